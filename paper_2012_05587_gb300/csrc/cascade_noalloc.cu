// Gauss's-law residual of a caller-held state, computed without allocating
// any memory.  This serves callers that cannot call cudaMalloc: hosts that
// give a library a fixed device-memory budget up front and reserve the rest
// for their own pool, plug-ins whose host application owns every allocation,
// and real-time loops where an allocation (which may synchronise the whole
// device) is not allowed.  The paper has no counterpart; cascade_gauss is the
// same check on a handle.  The call synchronises the caller's stream and
// copies the result to the host before it returns.
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
// first call for that device, which may initialise the module).
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

// CIC charge of every particle on its two nodes (periodic: node nx is node 0;
// open boundaries: node nx is outside the grid and not kept).
template <class Real>
__global__ void k_noalloc_rho(int nx, int open_bc, double w, long long n_elec, const int32_t* __restrict__ cell_e,
                              const Real* __restrict__ off_e, long long n_posi, const int32_t* __restrict__ cell_p,
                              const Real* __restrict__ off_p, double* rho_dx) {
  const long long total = n_elec + n_posi;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const bool pos = t >= n_elec;
    const long long p = pos ? t - n_elec : t;
    const int c = pos ? cell_p[p] : cell_e[p];
    const double o = (double)(pos ? off_p[p] : off_e[p]);
    if (c < 0 || c >= nx) continue;  // departed (open boundaries) or outside the grid
    const double qw = (pos ? 1.0 : -1.0) * w;
    atomicAdd(&rho_dx[c], qw * (1.0 - o));
    if (c + 1 < nx) atomicAdd(&rho_dx[c + 1], qw * o);
    else if (!open_bc) atomicAdd(&rho_dx[0], qw * o);
  }
}

// max_i |E_{i+1/2} - E_{i-1/2} - dx (rho_i - rho_GJ)| (Eq. 25; rho_GJ = 0
// outside the co-rotating frame); with open boundaries the interior nodes.
__global__ void k_noalloc_resid(int nx, int open_bc, double rho_gj_dx, const double* __restrict__ E,
                                const double* __restrict__ rho_dx, double* out) {
  __shared__ double sh[32];
  double v = 0.0;
  for (int i = threadIdx.x + (open_bc ? 1 : 0); i < nx; i += blockDim.x) {
    const int im = (i == 0) ? nx - 1 : i - 1;
    v = fmax(v, fabs(E[i] - E[im] - (rho_dx[i] - rho_gj_dx)));
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

int invalid(const char* why) {
  char msg[160];
  snprintf(msg, sizeof(msg), "cascade_gauss_noalloc: %s", why);
  cpic::set_error_message(msg);
  return CASCADE_ERR_INVALID_ARG;
}

int cuda_failed(cudaError_t e, const char* step) {
  char msg[200];
  snprintf(msg, sizeof(msg), "cascade_gauss_noalloc: %s: %s", step, cudaGetErrorString(e));
  cpic::set_error_message(msg);
  return CASCADE_ERR_CUDA;
}

}  // namespace

extern "C" int cascade_gauss_noalloc(int32_t nx, double dx, double w, double rho_gj, int32_t open_bc,
                                     int32_t precision, int64_t n_elec, const int32_t* cell_e, const void* off_e,
                                     int64_t n_posi, const int32_t* cell_p, const void* off_p, const double* E,
                                     double* resid_out, void* cuda_stream) {
  cpic::set_error_message("");  // a message describes this call only
  if (nx < 2 || nx > kNoAllocMaxNx) {
    char msg[96];
    snprintf(msg, sizeof(msg), "nx = %d outside 2 .. %d (CASCADE_NOALLOC_MAX_NX)", nx, kNoAllocMaxNx);
    return invalid(msg);
  }
  if (!(dx > 0) || !isfinite(w) || !isfinite(rho_gj)) return invalid("dx must be positive, w and rho_gj finite");
  if (open_bc != 0 && open_bc != 1) return invalid("open_bc must be 0 or 1");
  if (n_elec < 0 || n_posi < 0) return invalid("negative particle count");
  if (!E || !resid_out) return invalid("E and resid_out are required");
  if ((n_elec > 0 && (!cell_e || !off_e)) || (n_posi > 0 && (!cell_p || !off_p)))
    return invalid("particle arrays are required for nonzero counts");
  if (precision != CASCADE_FP64 && precision != CASCADE_FP32_MIXED && precision != CASCADE_FP32_MIXED_FINE)
    return invalid("unknown precision");
  // an error left pending by earlier, unrelated launches is not this call's
  (void)cudaGetLastError();
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_failed(e, "cudaGetDevice");
  double* scratch = nullptr;
  if ((e = scratch_for(dev, &scratch)) != cudaSuccess) return cuda_failed(e, "cudaGetSymbolAddress of the scratch");
  cudaStream_t st = (cudaStream_t)cuda_stream;
  double* rho_dx = scratch;
  double* out = scratch + kNoAllocMaxNx;
  // the array keeps the previous call's contents: clear the accumulator
  if ((e = cudaMemsetAsync(rho_dx, 0, sizeof(double) * nx, st)) != cudaSuccess)
    return cuda_failed(e, "clearing the scratch");
  const long long total = (long long)n_elec + n_posi;
  long long blocks = (total + 255) / 256;
  if (blocks < 1) blocks = 1;
  if (blocks > 4096) blocks = 4096;
  if (precision == CASCADE_FP64) {
    k_noalloc_rho<double><<<(int)blocks, 256, 0, st>>>(nx, open_bc, w, n_elec, cell_e,
                                                      static_cast<const double*>(off_e), n_posi, cell_p,
                                                      static_cast<const double*>(off_p), rho_dx);
  } else {
    k_noalloc_rho<float><<<(int)blocks, 256, 0, st>>>(nx, open_bc, w, n_elec, cell_e,
                                                     static_cast<const float*>(off_e), n_posi, cell_p,
                                                     static_cast<const float*>(off_p), rho_dx);
  }
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_failed(e, "charge kernel launch");
  k_noalloc_resid<<<1, 1024, 0, st>>>(nx, open_bc, rho_gj * dx, E, rho_dx, out);
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_failed(e, "residual kernel launch");
  if ((e = cudaMemcpyAsync(resid_out, out, sizeof(double), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
    return cuda_failed(e, "copy of the result");
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_failed(e, "cudaStreamSynchronize");
  return CASCADE_OK;
}
