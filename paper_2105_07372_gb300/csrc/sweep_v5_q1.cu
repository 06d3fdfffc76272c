// Lean warp sweep instances for rows of 8 coefficients (QV = 1).
#include "sweep5_impl.cuh"
MRA_SWEEP_V5_TABLE(1)
