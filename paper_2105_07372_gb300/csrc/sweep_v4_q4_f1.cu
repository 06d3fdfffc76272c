// Chunked two-read EM sweep for rows of 32 coefficients (4 float4 per lane per row), y as the BF16 hi/lo split.
#include "sweep4_impl.cuh"

MRA_SWEEP_V4_TABLE(4, 1)
