// Objective kernels for l = 4 marginals.
#include "objective.cuh"
MMOT_INSTANTIATE_OBJECTIVE(4)
