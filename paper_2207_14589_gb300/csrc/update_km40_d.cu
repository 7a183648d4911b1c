// Instantiations of the solver update for rows of width 40, F64 master.
#include "update_kernel.cuh"

SPED_UPDATE_INSTANTIATE_PAIR(double, double, 40)
SPED_UPDATE_INSTANTIATE_PAIR(double, float, 40)
