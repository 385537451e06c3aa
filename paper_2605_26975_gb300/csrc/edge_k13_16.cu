// Edge kernels for k = 13..16 (explicit instantiations).
#include "edge_launch.cuh"
PSPEC_INSTANTIATE_EDGES(13)
PSPEC_INSTANTIATE_EDGES(14)
PSPEC_INSTANTIATE_EDGES(15)
PSPEC_INSTANTIATE_EDGES(16)
