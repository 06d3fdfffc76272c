// Paired-warp sweep instances for rows of 24 coefficients (QV = 3).
#include "sweep6_impl.cuh"
MRA_SWEEP_V6_TABLE(3, MRA_SWEEP_V6_CASE(3, 1) MRA_SWEEP_V6_CASE(3, 2))
