// 3D instantiation of the level kernels and their launchers.
#define MG_DIM 3
#define MG_NS d3
#include "ops_dim.cuh"
