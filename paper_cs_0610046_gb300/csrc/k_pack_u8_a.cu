// Packed 2D kernel instantiations: uint8_t, column windows 1, 2, 3.
#include "pack2d.cuh"

MMF_INSTANTIATE_PACK2D(uint8_t, 1)
MMF_INSTANTIATE_PACK2D(uint8_t, 2)
MMF_INSTANTIATE_PACK2D(uint8_t, 3)
