// Warp-per-image EM sweep for rows of 16 coefficients (2 float4 per lane per row).
#include "sweep_impl.cuh"

MRA_SWEEP_V2_TABLE(2)
