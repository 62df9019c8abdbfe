// Register-streaming 2D kernel instantiations: float, column windows 4, 5, 6.
#include "pack2d.cuh"

MMF_INSTANTIATE_PACK2D(float, 4)
MMF_INSTANTIATE_PACK2D(float, 5)
MMF_INSTANTIATE_PACK2D(float, 6)
