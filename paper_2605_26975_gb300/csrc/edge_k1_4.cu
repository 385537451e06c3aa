// Edge kernels for k = 1..4 (explicit instantiations).
#include "edge_launch.cuh"
PSPEC_INSTANTIATE_EDGES(1)
PSPEC_INSTANTIATE_EDGES(2)
PSPEC_INSTANTIATE_EDGES(3)
PSPEC_INSTANTIATE_EDGES(4)
