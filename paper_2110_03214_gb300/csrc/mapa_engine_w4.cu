// Runner instantiations for 4-word vertex masks (graphs of up to 128 vertices).
#include "mapa_runner.cuh"

MAPA_DEFINE_W(4)
