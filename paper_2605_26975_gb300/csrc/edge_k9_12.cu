// Edge kernels for k = 9..12 (explicit instantiations).
#include "edge_launch.cuh"
PSPEC_INSTANTIATE_EDGES(9)
PSPEC_INSTANTIATE_EDGES(10)
PSPEC_INSTANTIATE_EDGES(11)
PSPEC_INSTANTIATE_EDGES(12)
