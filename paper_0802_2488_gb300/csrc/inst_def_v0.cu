// Defect-correction kernels, tiling variant 0.
#define EPFFT_VAR 0
#include "inst_def_impl.cuh"
