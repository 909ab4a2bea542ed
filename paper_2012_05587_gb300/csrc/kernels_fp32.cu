// FP32-mixed particle kernels: int32 cell + FP32 offset and momentum, FP32
// per-CTA current accumulation in shared memory, FP64 for the grid-wide
// current reduction, the Ampere update, the energy diagnostics and the
// threshold test of leptons above gamma = 1e6.
#include "cascade_kernels.cuh"

CASCADE_DEFINE_LAUNCHERS(fp32, float)
