// Register-streaming 2D kernel instantiations: float, column windows 1, 2, 3.
#include "pack2d.cuh"

MMF_INSTANTIATE_PACK2D(float, 1)
MMF_INSTANTIATE_PACK2D(float, 2)
MMF_INSTANTIATE_PACK2D(float, 3)
