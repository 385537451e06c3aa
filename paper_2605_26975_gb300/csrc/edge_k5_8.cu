// Edge kernels for k = 5..8 (explicit instantiations).
#include "edge_launch.cuh"
PSPEC_INSTANTIATE_EDGES(5)
PSPEC_INSTANTIATE_EDGES(6)
PSPEC_INSTANTIATE_EDGES(7)
PSPEC_INSTANTIATE_EDGES(8)
