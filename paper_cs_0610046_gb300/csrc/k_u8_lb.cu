// Block-scan kernels for element type uint8_t in their envelope lower-bound form.
#include "kernels_blockscan_lb.cuh"

MMF_INSTANTIATE_BLOCKSCAN_LB(uint8_t)
