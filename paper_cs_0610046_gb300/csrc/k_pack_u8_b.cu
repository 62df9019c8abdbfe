// Packed 2D kernel instantiations: uint8_t, column windows 4, 5, 6.
#include "pack2d.cuh"

MMF_INSTANTIATE_PACK2D(uint8_t, 4)
MMF_INSTANTIATE_PACK2D(uint8_t, 5)
MMF_INSTANTIATE_PACK2D(uint8_t, 6)
