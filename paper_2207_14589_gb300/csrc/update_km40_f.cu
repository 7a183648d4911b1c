// Instantiations of the solver update for rows of width 40, F32 master.
#include "update_kernel.cuh"

SPED_UPDATE_INSTANTIATE_PAIR(float, float, 40)
SPED_UPDATE_INSTANTIATE_PAIR(float, double, 40)
