// Objective kernels for l = 7 marginals.
#include "objective.cuh"
MMOT_INSTANTIATE_OBJECTIVE(7)
