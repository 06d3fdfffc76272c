// CTA-cooperative batch EM sweep for rows of 8 coefficients (4 float4 per row).
#include "sweep3_impl.cuh"

MRA_SWEEP_V3_TABLE(4)
