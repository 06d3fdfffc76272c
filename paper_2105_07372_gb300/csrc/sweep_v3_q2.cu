// CTA-cooperative batch EM sweep for rows of 16 coefficients (8 float4 per row).
#include "sweep3_impl.cuh"

MRA_SWEEP_V3_TABLE(8)
