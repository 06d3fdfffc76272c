// CTA-cooperative batch EM sweep for rows of 24 coefficients (12 float4 per row).
#include "sweep3_impl.cuh"

MRA_SWEEP_V3_TABLE(12)
