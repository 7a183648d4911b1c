// Instantiations of the solver update for rows of width 20.
#include "update_kernel.cuh"

SPED_UPDATE_INSTANTIATE(20)
