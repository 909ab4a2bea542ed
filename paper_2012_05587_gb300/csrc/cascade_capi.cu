// Host side of the C ABI declared in include/cascade.h: parameter validation,
// device memory, initial state, CUDA-graph replay of the step, diagnostics.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <mutex>
#include <new>
#include <vector>

#include "cascade_internal.h"

using namespace cpic;

namespace {

constexpr int kGraphSteps = 16;   // steps per captured CUDA graph
constexpr int kDefaultRing = 4096;

cascade_alloc_fn g_alloc = nullptr;
cascade_free_fn g_free = nullptr;
void* g_ctx = nullptr;
std::mutex g_alloc_mu;

thread_local char g_msg[512] = "";

int cuda_fail(cudaError_t e, const char* what) {
  snprintf(g_msg, sizeof(g_msg), "%s: %s", what, cudaGetErrorString(e));
  return CASCADE_ERR_CUDA;
}

#define CUDA_TRY(expr)                                 \
  do {                                                 \
    cudaError_t e_ = (expr);                           \
    if (e_ != cudaSuccess) return cuda_fail(e_, #expr); \
  } while (0)

long long next_pow2(long long v) {
  long long p = 1;
  while (p < v) p <<= 1;
  return p;
}

int validate(const cascade_params* p) {
  if (!p) return CASCADE_ERR_INVALID_ARG;
  const char* why = nullptr;
  if (p->nx < 2) why = "nx < 2";
  else if (p->ppc < 1) why = "ppc < 1";
  else if (!(p->dx > 0) || !(p->dt > 0)) why = "dx and dt must be positive";
  else if (!(p->dt < p->dx)) why = "c dt must be below dx";
  else if (!(p->n0 >= 0)) why = "n0 < 0";
  else if (!(p->u_spread >= 0)) why = "u_spread < 0";
  else if (!(p->l_pp >= 0)) why = "l_pp < 0";
  else if (!(p->eps_gamma >= 2.0)) why = "eps_gamma below the pair rest mass (2)";
  else if (!(p->gamma_thr - p->eps_gamma >= 1.0)) why = "gamma_thr - eps_gamma < 1";
  else if (!(p->eps_gamma / p->gamma_thr < 2.0 / 3.0)) why = "f = eps_gamma / gamma_thr >= 2/3";
  else if (p->particle_cap < 1) why = "particle_cap < 1";
  else if (p->photon_cap < 0) why = "photon_cap < 0";
  else if (p->precision != CASCADE_FP64 && p->precision != CASCADE_FP32_MIXED &&
           p->precision != CASCADE_FP32_MIXED_FINE)
    why = "unknown precision";
  else if (p->diag_ring < 0) why = "diag_ring < 0";
  if (why) {
    snprintf(g_msg, sizeof(g_msg), "invalid parameters: %s", why);
    return CASCADE_ERR_INVALID_ARG;
  }
  return CASCADE_OK;
}

int n_pp_of(const cascade_params* p) {
  const double v = ceil(p->l_pp / p->dt - 1e-9);
  return v < 0 ? 0 : (int)v;
}

}  // namespace

struct cascade {
  cascade_params p{};
  Dev d{};
  int device = 0;
  int num_sms = 0;
  cudaStream_t stream = nullptr;      // caller's stream
  cudaStream_t cap_stream = nullptr;  // private stream used only for graph capture
  cudaGraphExec_t graph = nullptr;
  std::vector<void*> allocs;
  cascade_alloc_fn alloc_fn = nullptr;
  cascade_free_fn free_fn = nullptr;
  void* alloc_ctx = nullptr;
  double* rho_dx = nullptr;
  double* scalar = nullptr;
  size_t real_size = 8;
  size_t bytes = 0;
  int sticky = 0;
  // kernel timing (cascade_set_timing)
  bool timing = false;
  std::vector<cudaEvent_t> ev_pool;
  size_t ev_used = 0;
  long long kernels_launched = 0;

  void* dalloc(size_t n) {
    n = (n + 255) & ~size_t(255);
    void* ptr = nullptr;
    if (alloc_fn) {
      ptr = alloc_fn(n, (void*)stream, alloc_ctx);
    } else if (cudaMalloc(&ptr, n) != cudaSuccess) {
      cudaGetLastError();
      ptr = nullptr;
    }
    if (ptr) {
      allocs.push_back(ptr);
      bytes += n;
    }
    return ptr;
  }

  cudaError_t launch_step() {
    if (timing) {
      while (ev_pool.size() < ev_used + 2) {
        cudaEvent_t e;
        cudaError_t r = cudaEventCreate(&e);
        if (r != cudaSuccess) return r;
        ev_pool.push_back(e);
      }
      cudaEvent_t b = ev_pool[ev_used], a = ev_pool[ev_used + 1];
      ev_used += 2;
      kernels_launched += 3;
      return p.precision == CASCADE_FP64 ? step_timed_fp64(d, stream, b, a) : step_timed_fp32(d, stream, b, a);
    }
    return p.precision == CASCADE_FP64 ? step_fp64(d, stream) : step_fp32(d, stream);
  }
};

namespace {

// Layout and sizes shared by cascade_footprint and allocation.
struct Plan {
  long long cap4, ph_cap;
  int n_pp, ring;
  size_t real;
};

Plan plan_of(const cascade_params* p) {
  Plan pl;
  pl.real = p->precision == CASCADE_FP64 ? sizeof(double) : sizeof(float);
  pl.cap4 = (p->particle_cap + 3) & ~3LL;
  pl.ph_cap = next_pow2(p->photon_cap > 0 ? p->photon_cap : p->particle_cap);
  pl.n_pp = n_pp_of(p);
  pl.ring = p->diag_ring > 0 ? p->diag_ring : kDefaultRing;
  return pl;
}

int setup(const cascade_params* params, void* stream, cascade_t** out) {
  *out = nullptr;
  int rc = validate(params);
  if (rc) return rc;
  cascade_t* h = new (std::nothrow) cascade_t();
  if (!h) return CASCADE_ERR_OOM;
  h->p = *params;
  h->stream = (cudaStream_t)stream;
  {
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    h->alloc_fn = g_alloc;
    h->free_fn = g_free;
    h->alloc_ctx = g_ctx;
  }
  *out = h;
  cudaError_t e = cudaGetDevice(&h->device);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  e = cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device);
  if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceGetAttribute");

  const Plan pl = plan_of(params);
  h->real_size = pl.real;
  Dev& d = h->d;
  d.nx = params->nx;
  d.n_pp = pl.n_pp;
  const double L = params->l_pp / params->dx;
  d.lpp_int = (int)floor(L);
  d.lpp_frac = L - (double)d.lpp_int;
  d.cap = params->particle_cap;
  d.ph_cap = pl.ph_cap;
  d.dx = params->dx;
  d.dt = params->dt;
  d.dtdx = params->dt / params->dx;
  d.jscale = params->n0 * params->dx / ((double)params->ppc * params->dt);
  d.w = params->n0 * params->dx / (double)params->ppc;
  d.gamma_thr = params->gamma_thr;
  d.eps_gamma = params->eps_gamma;
  const double hh = 0.5 * params->eps_gamma;
  d.u_pair = sqrt(hh * hh - 1.0);
  d.ring_n = pl.ring;
  d.fine_deposit = params->precision == CASCADE_FP32_MIXED_FINE ? 1 : 0;
  e = params->precision == CASCADE_FP64 ? configure_fp64(d, h->num_sms) : configure_fp32(d, h->num_sms);
  if (e != cudaSuccess) return cuda_fail(e, "configure");

  // device memory
  const size_t R = pl.real;
  for (int s = 0; s < 2; ++s) {
    d.cell[s] = static_cast<int32_t*>(h->dalloc(sizeof(int32_t) * pl.cap4));
    d.off[s] = h->dalloc(R * pl.cap4);
    d.u[s] = h->dalloc(R * pl.cap4);
    if (!d.cell[s] || !d.off[s] || !d.u[s]) return CASCADE_ERR_OOM;
  }
  d.ph_cell = static_cast<int32_t*>(h->dalloc(sizeof(int32_t) * pl.ph_cap));
  d.ph_off = h->dalloc(R * pl.ph_cap);
  d.E = static_cast<double*>(h->dalloc(sizeof(double) * d.nx));
  d.J = static_cast<double*>(h->dalloc(sizeof(double) * d.nx));
  const size_t acc = params->precision == CASCADE_FP64 ? partial_bytes_fp64() : partial_bytes_fp32();
  if (d.variant == kSmemESmemS) {
    d.S_part = h->dalloc(acc * (size_t)d.grid_push * d.nxp);
    if (!d.S_part) return CASCADE_ERR_OOM;
  } else {
    d.S_glob = static_cast<double*>(h->dalloc(sizeof(double) * d.nx));
    if (!d.S_glob) return CASCADE_ERR_OOM;
  }
  d.uk_part = static_cast<double*>(h->dalloc(sizeof(double) * d.grid_push));
  d.diag_part = static_cast<double*>(h->dalloc(sizeof(double) * 4 * d.grid_field));
  d.emit_end = static_cast<long long*>(h->dalloc(sizeof(long long) * (d.n_pp + 1)));
  d.ctl = static_cast<Ctl*>(h->dalloc(sizeof(Ctl)));
  d.ring = static_cast<cascade_diag_t*>(h->dalloc(sizeof(cascade_diag_t) * d.ring_n));
  h->rho_dx = static_cast<double*>(h->dalloc(sizeof(double) * d.nx));
  h->scalar = static_cast<double*>(h->dalloc(sizeof(double) * 4));
  if (!d.ph_cell || !d.ph_off || !d.E || !d.J || !d.uk_part || !d.diag_part || !d.emit_end || !d.ctl ||
      !d.ring || !h->rho_dx || !h->scalar)
    return CASCADE_ERR_OOM;

  CUDA_TRY(cudaMemsetAsync(d.ctl, 0, sizeof(Ctl), h->stream));
  CUDA_TRY(cudaMemsetAsync(d.emit_end, 0, sizeof(long long) * (d.n_pp + 1), h->stream));
  CUDA_TRY(cudaMemsetAsync(d.ring, 0, sizeof(cascade_diag_t) * d.ring_n, h->stream));
  CUDA_TRY(cudaMemsetAsync(d.J, 0, sizeof(double) * d.nx, h->stream));
  if (d.S_glob) CUDA_TRY(cudaMemsetAsync(d.S_glob, 0, sizeof(double) * d.nx, h->stream));
  return CASCADE_OK;
}

int upload_E(cascade_t* h, const double* E_host) {
  std::vector<double> E(h->d.nx, h->p.E0);
  if (E_host) memcpy(E.data(), E_host, sizeof(double) * h->d.nx);
  CUDA_TRY(cudaMemcpyAsync(h->d.E, E.data(), sizeof(double) * h->d.nx, cudaMemcpyHostToDevice, h->stream));
  CUDA_TRY(cudaStreamSynchronize(h->stream));
  return CASCADE_OK;
}

int upload_species(cascade_t* h, int s, long long n, const int32_t* cell, const double* off, const double* u) {
  if (n == 0) return CASCADE_OK;
  for (long long i = 0; i < n; ++i) {
    if (cell[i] < 0 || cell[i] >= h->p.nx || !(off[i] >= 0.0) || !(off[i] < 1.0) || !isfinite(u[i])) {
      snprintf(g_msg, sizeof(g_msg), "particle %lld of species %d outside the grid or not finite", i, s);
      return CASCADE_ERR_INVALID_ARG;
    }
  }
  CUDA_TRY(cudaMemcpyAsync(h->d.cell[s], cell, sizeof(int32_t) * n, cudaMemcpyHostToDevice, h->stream));
  if (h->real_size == sizeof(double)) {
    CUDA_TRY(cudaMemcpyAsync(h->d.off[s], off, sizeof(double) * n, cudaMemcpyHostToDevice, h->stream));
    CUDA_TRY(cudaMemcpyAsync(h->d.u[s], u, sizeof(double) * n, cudaMemcpyHostToDevice, h->stream));
    CUDA_TRY(cudaStreamSynchronize(h->stream));
  } else {
    std::vector<float> fo(n), fu(n);
    for (long long i = 0; i < n; ++i) {
      float o = (float)off[i];
      if (o >= 1.0f) o = 0x1.fffffep-1f;  // keep the offset inside the cell
      fo[i] = o;
      fu[i] = (float)u[i];
    }
    CUDA_TRY(cudaMemcpyAsync(h->d.off[s], fo.data(), sizeof(float) * n, cudaMemcpyHostToDevice, h->stream));
    CUDA_TRY(cudaMemcpyAsync(h->d.u[s], fu.data(), sizeof(float) * n, cudaMemcpyHostToDevice, h->stream));
    CUDA_TRY(cudaStreamSynchronize(h->stream));
  }
  return CASCADE_OK;
}

int set_counts(cascade_t* h, long long ne, long long np) {
  Ctl c;
  memset(&c, 0, sizeof(c));
  c.n[0] = ne;
  c.n[1] = np;
  CUDA_TRY(cudaMemcpyAsync(h->d.ctl, &c, sizeof(Ctl), cudaMemcpyHostToDevice, h->stream));
  CUDA_TRY(cudaStreamSynchronize(h->stream));
  return CASCADE_OK;
}

int read_ctl(cascade_t* h, Ctl* c) {
  CUDA_TRY(cudaStreamSynchronize(h->stream));
  CUDA_TRY(cudaMemcpy(c, h->d.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost));
  if (c->err && !h->sticky) h->sticky = c->err;
  return CASCADE_OK;
}

int capture_graph(cascade_t* h) {
  if (!h->cap_stream) CUDA_TRY(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
  cudaGraph_t g = nullptr;
  CUDA_TRY(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
  cudaError_t e = cudaSuccess;
  for (int k = 0; k < kGraphSteps && e == cudaSuccess; ++k)
    e = h->p.precision == CASCADE_FP64 ? step_fp64(h->d, h->cap_stream) : step_fp32(h->d, h->cap_stream);
  cudaError_t e2 = cudaStreamEndCapture(h->cap_stream, &g);
  if (e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return cuda_fail(e, "capture step");
  }
  if (e2 != cudaSuccess) return cuda_fail(e2, "cudaStreamEndCapture");
  e = cudaGraphInstantiate(&h->graph, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
  return CASCADE_OK;
}

}  // namespace

extern "C" {

int cascade_set_allocator(cascade_alloc_fn alloc_fn, cascade_free_fn free_fn, void* ctx) {
  if ((alloc_fn == nullptr) != (free_fn == nullptr)) return CASCADE_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(g_alloc_mu);
  g_alloc = alloc_fn;
  g_free = free_fn;
  g_ctx = ctx;
  return CASCADE_OK;
}

int cascade_create(const cascade_params* params, void* cuda_stream, cascade_t** out) {
  if (!out) return CASCADE_ERR_INVALID_ARG;
  cascade_t* h = nullptr;
  int rc = setup(params, cuda_stream, &h);
  if (rc == CASCADE_OK) {
    const long long npairs = (long long)params->nx * params->ppc;
    if (npairs > params->particle_cap) {
      snprintf(g_msg, sizeof(g_msg), "seed needs %lld particles per species, cap is %lld", npairs,
               (long long)params->particle_cap);
      rc = CASCADE_ERR_CAPACITY;
    }
    if (rc == CASCADE_OK) rc = upload_E(h, nullptr);
    if (rc == CASCADE_OK) {
      cudaError_t e = params->precision == CASCADE_FP64
                          ? seed_fp64(h->d, npairs, params->ppc, params->seed, params->u_spread, h->stream)
                          : seed_fp32(h->d, npairs, params->ppc, params->seed, params->u_spread, h->stream);
      if (e != cudaSuccess) rc = cuda_fail(e, "seed kernel");
    }
    if (rc == CASCADE_OK) rc = set_counts(h, npairs, npairs);
  }
  if (rc != CASCADE_OK) {
    cascade_destroy(h);
    return rc;
  }
  *out = h;
  return CASCADE_OK;
}

int cascade_create_from_state(const cascade_params* params, int64_t n_elec, const int32_t* cell_e,
                              const double* off_e, const double* u_e, int64_t n_posi, const int32_t* cell_p,
                              const double* off_p, const double* u_p, const double* E_host, void* cuda_stream,
                              cascade_t** out) {
  if (!out || n_elec < 0 || n_posi < 0) return CASCADE_ERR_INVALID_ARG;
  if ((n_elec > 0 && (!cell_e || !off_e || !u_e)) || (n_posi > 0 && (!cell_p || !off_p || !u_p)))
    return CASCADE_ERR_INVALID_ARG;
  cascade_t* h = nullptr;
  int rc = setup(params, cuda_stream, &h);
  if (rc == CASCADE_OK && (n_elec > params->particle_cap || n_posi > params->particle_cap)) {
    snprintf(g_msg, sizeof(g_msg), "state exceeds particle_cap");
    rc = CASCADE_ERR_CAPACITY;
  }
  if (rc == CASCADE_OK) rc = upload_E(h, E_host);
  if (rc == CASCADE_OK) rc = upload_species(h, 0, n_elec, cell_e, off_e, u_e);
  if (rc == CASCADE_OK) rc = upload_species(h, 1, n_posi, cell_p, off_p, u_p);
  if (rc == CASCADE_OK) rc = set_counts(h, n_elec, n_posi);
  if (rc != CASCADE_OK) {
    cascade_destroy(h);
    return rc;
  }
  *out = h;
  return CASCADE_OK;
}

int cascade_step(cascade_t* h, int32_t nsteps) {
  if (!h || nsteps < 0) return CASCADE_ERR_INVALID_ARG;
  cudaSetDevice(h->device);
  int left = nsteps;
  if (h->timing) {
    for (; left > 0; --left) CUDA_TRY(h->launch_step());
    return CASCADE_OK;
  }
  if (left >= kGraphSteps && !h->graph) {
    int rc = capture_graph(h);
    if (rc) return rc;
  }
  while (left >= kGraphSteps) {
    CUDA_TRY(cudaGraphLaunch(h->graph, h->stream));
    left -= kGraphSteps;
  }
  for (; left > 0; --left) CUDA_TRY(h->launch_step());
  return CASCADE_OK;
}

int cascade_sync(cascade_t* h) {
  if (!h) return CASCADE_ERR_INVALID_ARG;
  cudaSetDevice(h->device);
  Ctl c;
  int rc = read_ctl(h, &c);
  if (rc) return rc;
  return h->sticky;
}

int cascade_diag(cascade_t* h, cascade_diag_t* host_out, int32_t max, int32_t* n_out, double* E_host,
                 double* J_host) {
  if (!h || max < 0 || (max > 0 && !host_out)) return CASCADE_ERR_INVALID_ARG;
  cudaSetDevice(h->device);
  Ctl c;
  int rc = read_ctl(h, &c);
  if (rc) return rc;
  const long long kept = c.step < h->d.ring_n ? c.step : h->d.ring_n;
  const long long n = kept < max ? kept : max;
  const long long first = c.step - n;  // records of steps first+1 .. c.step
  long long done = 0;
  while (done < n) {
    const long long slot = (first + done) % h->d.ring_n;
    long long run = h->d.ring_n - slot;
    if (run > n - done) run = n - done;
    CUDA_TRY(cudaMemcpy(host_out + done, h->d.ring + slot, sizeof(cascade_diag_t) * run, cudaMemcpyDeviceToHost));
    done += run;
  }
  if (n_out) *n_out = (int32_t)n;
  if (E_host) CUDA_TRY(cudaMemcpy(E_host, h->d.E, sizeof(double) * h->d.nx, cudaMemcpyDeviceToHost));
  if (J_host) CUDA_TRY(cudaMemcpy(J_host, h->d.J, sizeof(double) * h->d.nx, cudaMemcpyDeviceToHost));
  return h->sticky;
}

int cascade_gauss(cascade_t* h, double* resid_out) {
  if (!h || !resid_out) return CASCADE_ERR_INVALID_ARG;
  cudaSetDevice(h->device);
  cudaError_t e = h->p.precision == CASCADE_FP64 ? gauss_fp64(h->d, h->rho_dx, h->scalar, h->stream)
                                                 : gauss_fp32(h->d, h->rho_dx, h->scalar, h->stream);
  if (e != cudaSuccess) return cuda_fail(e, "gauss kernels");
  CUDA_TRY(cudaStreamSynchronize(h->stream));
  CUDA_TRY(cudaMemcpy(resid_out, h->scalar, sizeof(double), cudaMemcpyDeviceToHost));
  return CASCADE_OK;
}

int cascade_counts(cascade_t* h, int64_t* n_elec, int64_t* n_posi, int64_t* n_photon, int64_t* step) {
  if (!h) return CASCADE_ERR_INVALID_ARG;
  cudaSetDevice(h->device);
  Ctl c;
  int rc = read_ctl(h, &c);
  if (rc) return rc;
  if (n_elec) *n_elec = c.n[0];
  if (n_posi) *n_posi = c.n[1];
  if (n_photon) *n_photon = c.ph_tail - c.ph_head;
  if (step) *step = c.step;
  return h->sticky;
}

int cascade_particles(cascade_t* h, int32_t species, int64_t max, int32_t* cell, double* off, double* u,
                      int64_t* n_out) {
  if (!h || species < 0 || species > 1 || max < 0) return CASCADE_ERR_INVALID_ARG;
  cudaSetDevice(h->device);
  Ctl c;
  int rc = read_ctl(h, &c);
  if (rc) return rc;
  const long long n = c.n[species] < max ? c.n[species] : max;
  if (n_out) *n_out = n;
  if (n == 0) return CASCADE_OK;
  if (cell) CUDA_TRY(cudaMemcpy(cell, h->d.cell[species], sizeof(int32_t) * n, cudaMemcpyDeviceToHost));
  if (h->real_size == sizeof(double)) {
    if (off) CUDA_TRY(cudaMemcpy(off, h->d.off[species], sizeof(double) * n, cudaMemcpyDeviceToHost));
    if (u) CUDA_TRY(cudaMemcpy(u, h->d.u[species], sizeof(double) * n, cudaMemcpyDeviceToHost));
  } else {
    std::vector<float> tmp(n);
    if (off) {
      CUDA_TRY(cudaMemcpy(tmp.data(), h->d.off[species], sizeof(float) * n, cudaMemcpyDeviceToHost));
      for (long long i = 0; i < n; ++i) off[i] = tmp[i];
    }
    if (u) {
      CUDA_TRY(cudaMemcpy(tmp.data(), h->d.u[species], sizeof(float) * n, cudaMemcpyDeviceToHost));
      for (long long i = 0; i < n; ++i) u[i] = tmp[i];
    }
  }
  return h->sticky;
}

int cascade_set_timing(cascade_t* h, int32_t enable) {
  if (!h) return CASCADE_ERR_INVALID_ARG;
  h->timing = enable != 0;
  return CASCADE_OK;
}

int cascade_timing(cascade_t* h, double* particle_kernel_ms, int64_t* particle_kernel_launches,
                   int64_t* kernels_launched) {
  if (!h) return CASCADE_ERR_INVALID_ARG;
  cudaSetDevice(h->device);
  CUDA_TRY(cudaStreamSynchronize(h->stream));
  double total = 0.0;
  for (size_t i = 0; i + 1 < h->ev_used; i += 2) {
    float ms = 0.f;
    CUDA_TRY(cudaEventElapsedTime(&ms, h->ev_pool[i], h->ev_pool[i + 1]));
    total += ms;
  }
  if (particle_kernel_ms) *particle_kernel_ms = total;
  if (particle_kernel_launches) *particle_kernel_launches = (int64_t)(h->ev_used / 2);
  if (kernels_launched) *kernels_launched = h->kernels_launched;
  h->ev_used = 0;
  h->kernels_launched = 0;
  return CASCADE_OK;
}

int cascade_destroy(cascade_t* h) {
  if (!h) return CASCADE_OK;
  cudaSetDevice(h->device);
  if (h->stream || !h->allocs.empty()) cudaStreamSynchronize(h->stream);
  for (cudaEvent_t e : h->ev_pool) cudaEventDestroy(e);
  if (h->graph) cudaGraphExecDestroy(h->graph);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  for (void* ptr : h->allocs) {
    if (h->free_fn) h->free_fn(ptr, (void*)h->stream, h->alloc_ctx);
    else cudaFree(ptr);
  }
  delete h;
  return CASCADE_OK;
}

int cascade_footprint(const cascade_params* params, int32_t* n_pp_out, size_t* device_bytes_out) {
  int rc = validate(params);
  if (rc) return rc;
  const Plan pl = plan_of(params);
  if (n_pp_out) *n_pp_out = pl.n_pp;
  if (device_bytes_out) {
    size_t b = 2 * (sizeof(int32_t) + 2 * pl.real) * (size_t)pl.cap4;
    b += (sizeof(int32_t) + pl.real) * (size_t)pl.ph_cap;
    b += sizeof(double) * (size_t)params->nx * 4;
    // per-CTA partials: at most 4 CTAs per SM on a 152-SM part
    b += pl.real * (size_t)(4 * 152) * (size_t)((params->nx + 31) & ~31);
    b += sizeof(cascade_diag_t) * (size_t)pl.ring + 64 * 1024;
    *device_bytes_out = b;
  }
  return CASCADE_OK;
}

const char* cascade_status_string(int status) {
  switch (status) {
    case CASCADE_OK: return "ok";
    case CASCADE_ERR_INVALID_ARG: return "invalid argument";
    case CASCADE_ERR_OOM: return "out of device memory";
    case CASCADE_ERR_CAPACITY: return "particle capacity exceeded";
    case CASCADE_ERR_CUDA: return "CUDA error";
    case CASCADE_ERR_TIMEOUT: return "device wait timed out";
    case CASCADE_ERR_UNIMPLEMENTED: return "not implemented";
    case CASCADE_ERR_PHOTON_CAPACITY: return "photon capacity exceeded";
    case CASCADE_ERR_BUSY: return "no free slot or memory";
    case CASCADE_ERR_NONFINITE: return "non-finite particle energy";
    default: return "unknown status";
  }
}

const char* cascade_last_error_message(void) { return g_msg; }

}  // extern "C"

namespace cpic {
void set_error_message(const char* msg) { snprintf(g_msg, sizeof(g_msg), "%s", msg); }
}  // namespace cpic

extern "C" {

}  // extern "C"
