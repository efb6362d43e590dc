// Runner instantiations for 2-word vertex masks (graphs of up to 64 vertices).
#include "mapa_runner.cuh"

MAPA_DEFINE_W(2)
