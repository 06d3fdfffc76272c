// Split-sweep stream kernels (correlation, accumulation) for rows of 24 coefficients.
#include "sweep_tc_impl.cuh"
MRA_SWEEP_TC_STREAM_TABLE(3)
