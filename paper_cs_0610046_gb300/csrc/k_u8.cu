// Kernel instantiations for element type uint8_t.
#include "kernels_blockscan.cuh"

MMF_INSTANTIATE_BLOCKSCAN(uint8_t)
