// Lean warp sweep instances for rows of 24 coefficients (QV = 3).
#include "sweep5_impl.cuh"
MRA_SWEEP_V5_TABLE(3)
