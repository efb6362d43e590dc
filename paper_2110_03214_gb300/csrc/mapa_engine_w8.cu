// Runner instantiations for 8-word vertex masks (graphs of up to 256 vertices).
#include "mapa_runner.cuh"

MAPA_DEFINE_W(8)
