// Block-scan kernels for element type int16_t in their envelope lower-bound form.
#include "kernels_blockscan_lb.cuh"

MMF_INSTANTIATE_BLOCKSCAN_LB(int16_t)
