// Gauss's-law residual of a caller-held state, computed without allocating
// any memory.  This serves callers that cannot call cudaMalloc: code running
// while a stream is being captured into a CUDA graph (allocation would break
// the capture), hosts that give a library a fixed device-memory budget up
// front, and plug-ins whose host application owns every allocation.  The
// paper has no counterpart; cascade_gauss is the same check on a handle.
//
// Scratch lives in the file-scope array below.  Every GPU that loads the
// library holds it (kNoAllocMaxNx + 32 doubles, 512.25 KiB) until the process
// exits.  In host code the array's name is only a host-side stand-in, so the
// host obtains its device address once per device with cudaGetSymbolAddress
// and passes that address to the kernels.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>

#include <mutex>

#include "cascade_internal.h"

namespace {

constexpr int kNoAllocMaxNx = CASCADE_NOALLOC_MAX_NX;
constexpr int kMaxDevices = 64;

// [0, kNoAllocMaxNx): charge per node times dx; [kNoAllocMaxNx]: the result.
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocMaxNx + 32];

std::mutex g_setup_mu;
double* g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device (looked up on the
// first call for that device; that first call must not happen during a stream
// capture, because cudaGetSymbolAddress may initialise the module).
cudaError_t scratch_for(int device, double** out) {
  if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_setup_mu);
  if (!g_scratch_ptr[device]) {
    double* ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress((void**)&ptr, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[device] = ptr;
  }
  *out = g_scratch_ptr[device];
  return cudaSuccess;
}

template <class Real>
__global__ void k_noalloc_rho(int nx, double w, long long n_elec, const int32_t* __restrict__ cell_e,
                              const Real* __restrict__ off_e, long long n_posi, const int32_t* __restrict__ cell_p,
                              const Real* __restrict__ off_p, double* rho_dx) {
  const long long total = n_elec + n_posi;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const bool pos = t >= n_elec;
    const long long p = pos ? t - n_elec : t;
    const int c = pos ? cell_p[p] : cell_e[p];
    const double o = (double)(pos ? off_p[p] : off_e[p]);
    if (c < 0 || c >= nx) continue;  // outside the grid: not a valid particle
    const int c1 = (c + 1 == nx) ? 0 : c + 1;
    const double qw = (pos ? 1.0 : -1.0) * w;
    atomicAdd(&rho_dx[c], qw * (1.0 - o));
    atomicAdd(&rho_dx[c1], qw * o);
  }
}

__global__ void k_noalloc_resid(int nx, const double* __restrict__ E, const double* __restrict__ rho_dx,
                                double* out) {
  __shared__ double sh[32];
  double v = 0.0;
  for (int i = threadIdx.x; i < nx; i += blockDim.x) {
    const int im = (i == 0) ? nx - 1 : i - 1;
    v = fmax(v, fabs(E[i] - E[im] - rho_dx[i]));
  }
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    v = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
    if (threadIdx.x == 0) *out = v;
  }
}

}  // namespace

extern "C" int cascade_gauss_noalloc(int32_t nx, double dx, double w, int32_t precision, int64_t n_elec,
                                     const int32_t* cell_e, const void* off_e, int64_t n_posi,
                                     const int32_t* cell_p, const void* off_p, const double* E,
                                     double* resid_out, void* cuda_stream) {
  (void)dx;
  if (nx < 2 || nx > kNoAllocMaxNx) {
    char msg[128];
    snprintf(msg, sizeof(msg), "cascade_gauss_noalloc: nx = %d outside 2 .. %d (CASCADE_NOALLOC_MAX_NX)", nx,
             kNoAllocMaxNx);
    cpic::set_error_message(msg);
    return CASCADE_ERR_INVALID_ARG;
  }
  if (n_elec < 0 || n_posi < 0 || !E || !resid_out) return CASCADE_ERR_INVALID_ARG;
  if ((n_elec > 0 && (!cell_e || !off_e)) || (n_posi > 0 && (!cell_p || !off_p))) return CASCADE_ERR_INVALID_ARG;
  if (precision != CASCADE_FP64 && precision != CASCADE_FP32_MIXED) return CASCADE_ERR_INVALID_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return CASCADE_ERR_CUDA;
  double* scratch = nullptr;
  if (scratch_for(dev, &scratch) != cudaSuccess) return CASCADE_ERR_CUDA;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  double* rho_dx = scratch;
  double* out = scratch + kNoAllocMaxNx;
  // the array keeps the previous call's contents: clear the accumulator
  if (cudaMemsetAsync(rho_dx, 0, sizeof(double) * nx, st) != cudaSuccess) return CASCADE_ERR_CUDA;
  const long long total = (long long)n_elec + n_posi;
  long long blocks = (total + 255) / 256;
  if (blocks < 1) blocks = 1;
  if (blocks > 4096) blocks = 4096;
  if (precision == CASCADE_FP64) {
    k_noalloc_rho<double><<<(int)blocks, 256, 0, st>>>(nx, w, n_elec, cell_e, static_cast<const double*>(off_e),
                                                      n_posi, cell_p, static_cast<const double*>(off_p), rho_dx);
  } else {
    k_noalloc_rho<float><<<(int)blocks, 256, 0, st>>>(nx, w, n_elec, cell_e, static_cast<const float*>(off_e),
                                                     n_posi, cell_p, static_cast<const float*>(off_p), rho_dx);
  }
  k_noalloc_resid<<<1, 1024, 0, st>>>(nx, E, rho_dx, out);
  if (cudaGetLastError() != cudaSuccess) return CASCADE_ERR_CUDA;
  if (cudaMemcpyAsync(resid_out, out, sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return CASCADE_ERR_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return CASCADE_ERR_CUDA;
  return CASCADE_OK;
}
