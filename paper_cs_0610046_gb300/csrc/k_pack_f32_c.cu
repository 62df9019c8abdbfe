// Register-streaming 2D kernel instantiations: float, column windows 7, 8, 9.
#include "pack2d.cuh"

MMF_INSTANTIATE_PACK2D(float, 7)
MMF_INSTANTIATE_PACK2D(float, 8)
MMF_INSTANTIATE_PACK2D(float, 9)
