// Chunked two-read EM sweep for rows of 24 coefficients (3 float4 per lane per row), y in FP32.
#include "sweep4_impl.cuh"

MRA_SWEEP_V4_TABLE(3, 0)
