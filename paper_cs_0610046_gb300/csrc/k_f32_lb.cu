// Block-scan kernels for element type float in their envelope lower-bound form.
#include "kernels_blockscan_lb.cuh"

MMF_INSTANTIATE_BLOCKSCAN_LB(float)
