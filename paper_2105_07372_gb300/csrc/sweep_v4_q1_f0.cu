// Chunked two-read EM sweep for rows of 8 coefficients (1 float4 per lane per row), y in FP32.
#include "sweep4_impl.cuh"

MRA_SWEEP_V4_TABLE(1, 0)
