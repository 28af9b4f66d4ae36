// Objective kernels for l = 3 marginals.
#include "objective.cuh"
MMOT_INSTANTIATE_OBJECTIVE(3)
