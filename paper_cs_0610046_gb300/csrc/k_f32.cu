// Kernel instantiations for element type float.
#include "kernels_blockscan.cuh"

MMF_INSTANTIATE_BLOCKSCAN(float)
