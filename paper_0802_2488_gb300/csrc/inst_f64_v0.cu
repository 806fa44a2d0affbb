// double instantiation of the fused passes, tiling variant 0.
#define EPFFT_REAL double
#define EPFFT_VAR 0
#define EPFFT_L4096(X) X(4096)
#include "inst_impl.cuh"
