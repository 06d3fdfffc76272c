// Chunked two-read EM sweep for rows of 32 coefficients (4 float4 per lane per row), y in FP32.
#include "sweep4_impl.cuh"

MRA_SWEEP_V4_TABLE(4, 0)
