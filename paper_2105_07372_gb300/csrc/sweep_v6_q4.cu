// Paired-warp sweep instances for rows of 32 coefficients (QV = 4).
#include "sweep6_impl.cuh"
MRA_SWEEP_V6_TABLE(4, MRA_SWEEP_V6_CASE(4, 1))
