// FP64 particle kernels.  Built with -fmad=false: every product and sum
// rounds separately, in the order the step is written, as in the plain
// double-precision definition of the method.
#include "cascade_kernels.cuh"

CASCADE_DEFINE_LAUNCHERS(fp64, double)
