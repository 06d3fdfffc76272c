// Warp-per-image EM sweep for rows of 8 coefficients (1 float4 per lane per row).
#include "sweep_impl.cuh"

MRA_SWEEP_V2_TABLE(1)
