// EM sweeps for rows of 32 coefficients: warp per image (4 float4 per lane per row),
// CTA-cooperative batches (16 float4 per row) and chunked two-read streaming.
#include "sweep_impl.cuh"
#include "sweep3_impl.cuh"
#include "sweep4_impl.cuh"

MRA_SWEEP_V2_TABLE(4)
MRA_SWEEP_V3_TABLE(16)
MRA_SWEEP_V4_TABLE(4)
