// CTA-cooperative batch EM sweep for rows of 32 coefficients (16 float4 per row).
#include "sweep3_impl.cuh"

MRA_SWEEP_V3_TABLE(16)
