// EM sweeps for rows of 24 coefficients: warp per image (3 float4 per lane per row),
// CTA-cooperative batches (12 float4 per row) and chunked two-read streaming.
#include "sweep_impl.cuh"
#include "sweep3_impl.cuh"
#include "sweep4_impl.cuh"

MRA_SWEEP_V2_TABLE(3)
MRA_SWEEP_V3_TABLE(12)
MRA_SWEEP_V4_TABLE(3)
