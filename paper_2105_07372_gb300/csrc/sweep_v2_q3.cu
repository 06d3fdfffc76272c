// Warp-per-image EM sweep for rows of 24 coefficients (3 float4 per lane per row).
#include "sweep_impl.cuh"

MRA_SWEEP_V2_TABLE(3)
