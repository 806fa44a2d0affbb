// Defect-correction kernels, tiling variant 1.
#define EPFFT_VAR 1
#include "inst_def_impl.cuh"
