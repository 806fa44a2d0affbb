// FP32 instantiation of the fused passes, lattice sides 4 .. 4096.
#define EPFFT_REAL float
#define EPFFT_L4096(X) X(4096)
#include "inst_impl.cuh"
