// Instantiations of the solver update for rows of width 8 and 16.
#include "update_kernel.cuh"

SPED_UPDATE_INSTANTIATE(8)
SPED_UPDATE_INSTANTIATE(16)
