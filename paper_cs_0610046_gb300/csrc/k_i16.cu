// Kernel instantiations for element type int16_t.
#include "kernels_blockscan.cuh"

MMF_INSTANTIATE_BLOCKSCAN(int16_t)
