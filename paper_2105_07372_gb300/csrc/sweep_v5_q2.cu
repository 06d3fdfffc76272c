// Lean warp sweep instances for rows of 16 coefficients (QV = 2).
#include "sweep5_impl.cuh"
MRA_SWEEP_V5_TABLE(2)
