// Paired-warp sweep instances for rows of 16 coefficients (QV = 2).
#include "sweep6_impl.cuh"
MRA_SWEEP_V6_TABLE(2, MRA_SWEEP_V6_CASE(2, 1) MRA_SWEEP_V6_CASE(2, 2) MRA_SWEEP_V6_CASE(2, 3))
