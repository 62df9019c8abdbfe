// Packed 2D kernel instantiations: int16_t, column windows 6, 7, 8, 9.
#include "pack2d.cuh"

MMF_INSTANTIATE_PACK2D(int16_t, 6)
MMF_INSTANTIATE_PACK2D(int16_t, 7)
MMF_INSTANTIATE_PACK2D(int16_t, 8)
MMF_INSTANTIATE_PACK2D(int16_t, 9)
