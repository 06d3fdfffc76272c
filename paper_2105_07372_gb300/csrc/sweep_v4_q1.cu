// Chunked two-read EM sweep for rows of 8 coefficients (1 float4 per lane per row).
#include "sweep4_impl.cuh"

MRA_SWEEP_V4_TABLE(1)
