// Instantiations of the solver update for rows of width 32, F32 master and F64 Y.
#include "update_kernel.cuh"

SPED_UPDATE_INSTANTIATE_PAIR(float, double, 32)
