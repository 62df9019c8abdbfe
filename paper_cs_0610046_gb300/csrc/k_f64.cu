// Kernel instantiations for element type double.
#include "kernels_blockscan.cuh"

MMF_INSTANTIATE_BLOCKSCAN(double)
