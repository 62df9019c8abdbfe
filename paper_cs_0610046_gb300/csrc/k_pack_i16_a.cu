// Packed 2D kernel instantiations: int16_t, column windows 1, 2, 3, 4, 5.
#include "pack2d.cuh"

MMF_INSTANTIATE_PACK2D(int16_t, 1)
MMF_INSTANTIATE_PACK2D(int16_t, 2)
MMF_INSTANTIATE_PACK2D(int16_t, 3)
MMF_INSTANTIATE_PACK2D(int16_t, 4)
MMF_INSTANTIATE_PACK2D(int16_t, 5)
