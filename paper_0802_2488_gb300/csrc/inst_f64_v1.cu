// double instantiation of the fused passes, tiling variant 1.
#define EPFFT_REAL double
#define EPFFT_VAR 1
#define EPFFT_L4096(X) X(4096)
#include "inst_impl.cuh"
