// FP64 instantiation of the fused passes, lattice sides 4 .. 2048.
#define EPFFT_REAL double
#define EPFFT_L4096(X)
#include "inst_impl.cuh"
