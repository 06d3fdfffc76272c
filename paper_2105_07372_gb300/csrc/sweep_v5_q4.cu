// Lean warp sweep instances for rows of 32 coefficients (QV = 4).
#include "sweep5_impl.cuh"
MRA_SWEEP_V5_TABLE(4)
