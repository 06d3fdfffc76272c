// Warp-per-image EM sweep for rows of 32 coefficients (4 float4 per lane per row).
#include "sweep_impl.cuh"

MRA_SWEEP_V2_TABLE(4)
