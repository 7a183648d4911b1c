// Instantiations of the solver update for rows of width 24, F32 master.
#include "update_kernel.cuh"

SPED_UPDATE_INSTANTIATE_PAIR(float, float, 24)
SPED_UPDATE_INSTANTIATE_PAIR(float, double, 24)
