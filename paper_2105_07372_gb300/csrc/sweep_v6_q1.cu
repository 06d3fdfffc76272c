// Paired-warp sweep instances for rows of 8 coefficients (QV = 1).
#include "sweep6_impl.cuh"
MRA_SWEEP_V6_TABLE(1, MRA_SWEEP_V6_CASE(1, 1) MRA_SWEEP_V6_CASE(1, 2) MRA_SWEEP_V6_CASE(1, 3))
