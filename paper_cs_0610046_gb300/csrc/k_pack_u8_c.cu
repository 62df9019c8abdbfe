// Packed 2D kernel instantiations: uint8_t, column windows 7, 8, 9.
#include "pack2d.cuh"

MMF_INSTANTIATE_PACK2D(uint8_t, 7)
MMF_INSTANTIATE_PACK2D(uint8_t, 8)
MMF_INSTANTIATE_PACK2D(uint8_t, 9)
