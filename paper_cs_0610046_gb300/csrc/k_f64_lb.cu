// Block-scan kernels for element type double in their envelope lower-bound form.
#include "kernels_blockscan_lb.cuh"

MMF_INSTANTIATE_BLOCKSCAN_LB(double)
