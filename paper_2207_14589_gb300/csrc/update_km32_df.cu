// Instantiations of the solver update for rows of width 32, F64 master and F32 Y.
#include "update_kernel.cuh"

SPED_UPDATE_INSTANTIATE_PAIR(double, float, 32)
