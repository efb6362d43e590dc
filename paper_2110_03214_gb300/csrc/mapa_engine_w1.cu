// Runner instantiations for 1-word vertex masks (graphs of up to 32 vertices).
#include "mapa_runner.cuh"

MAPA_DEFINE_W(1)
