// EM sweeps for rows of 8 coefficients: warp per image (1 float4 per lane per row),
// CTA-cooperative batches (4 float4 per row) and chunked two-read streaming.
#include "sweep_impl.cuh"
#include "sweep3_impl.cuh"
#include "sweep4_impl.cuh"

MRA_SWEEP_V2_TABLE(1)
MRA_SWEEP_V3_TABLE(4)
MRA_SWEEP_V4_TABLE(1)
