// EM sweeps for rows of 16 coefficients: warp per image (2 float4 per lane per row),
// CTA-cooperative batches (8 float4 per row) and chunked two-read streaming.
#include "sweep_impl.cuh"
#include "sweep3_impl.cuh"
#include "sweep4_impl.cuh"

MRA_SWEEP_V2_TABLE(2)
MRA_SWEEP_V3_TABLE(8)
MRA_SWEEP_V4_TABLE(2)
