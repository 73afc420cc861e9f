// 2D instantiation of the level kernels and their launchers.
#define MG_DIM 2
#define MG_NS d2
#include "ops_dim.cuh"
