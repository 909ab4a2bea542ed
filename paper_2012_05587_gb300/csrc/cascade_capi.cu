// Host side of the C ABI declared in include/cascade.h: parameter validation,
// device memory, initial state, CUDA-graph replay of the step, diagnostics.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <chrono>
#include <deque>
#include <mutex>
#include <new>
#include <string>
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
  else if (p->open_bc != 0 && p->open_bc != 1) why = "open_bc must be 0 or 1";
  else if (!isfinite(p->j_m) || !isfinite(p->rho_gj)) why = "j_m and rho_gj must be finite";
  else if (p->u_words < 0 || p->u_words > 2) why = "u_words must be 0, 1 or 2";
  if (why) {
    snprintf(g_msg, sizeof(g_msg), "invalid parameters: %s", why);
    return CASCADE_ERR_INVALID_ARG;
  }
  return CASCADE_OK;
}

// FP32 words per particle momentum (see cascade_momentum_words in the
// header): two when half the FP32 spacing at the threshold momentum exceeds
// 2^-12 of the reference push F dt.  Returns CASCADE_ERR_INVALID_ARG when the
// caller asks for one word where two are needed.
int momentum_words(const cascade_params* p, int* words) {
  if (p->precision == CASCADE_FP64) {
    *words = 2;
    return CASCADE_OK;
  }
  const double u_thr = sqrt(p->gamma_thr * p->gamma_thr - 1.0);
  int e = 0;
  frexp(u_thr, &e);                          // u_thr = m 2^e, m in [0.5, 1)
  const double half_spacing = ldexp(1.0, e - 25);  // FP32 keeps 24 bits
  const double F = p->E0 != 0.0 ? fabs(p->E0) : p->gamma_thr / ((double)p->nx * p->dx);
  const double push = F * p->dt;
  const bool two = half_spacing > ldexp(push, -12);
  if (p->u_words == 1 && two) {
    snprintf(g_msg, sizeof(g_msg),
             "one FP32 word cannot resolve the momentum at threshold: half its spacing at u_thr = %.6g is %.3g, "
             "above 2^-12 of the push %.3g per step (use u_words = 0 or 2)",
             u_thr, half_spacing, push);
    return CASCADE_ERR_INVALID_ARG;
  }
  *words = (p->u_words == 2 || two) ? 2 : 1;
  return CASCADE_OK;
}

int n_pp_of(const cascade_params* p) {
  const double v = ceil(p->l_pp / p->dt - 1e-9);
  return v < 0 ? 0 : (int)v;
}

}  // namespace

constexpr int kRecRing = 64;  // record copies a cascade may have queued

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
  // queued copies of the newest record (cascade_record_enqueue / _poll)
  Ctl* h_rec = nullptr;  // pinned, kRecRing copies of the control block
  cudaEvent_t ev_rec[kRecRing] = {};
  long long rec_issued = 0, rec_read = 0;
  std::deque<cascade_diag_t> rec_landed;  // taken from a full ring, not yet polled

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
      kernels_launched += 3 + (d.gauss_every > 0 ? 2 : 0) + (d.open_bc ? 2 : 0);
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
  size_t ulo;  // bytes of the low momentum word per particle (two-word FP32 momenta)
};

Plan plan_of(const cascade_params* p) {
  Plan pl;
  pl.real = p->precision == CASCADE_FP64 ? sizeof(double) : sizeof(float);
  int words = 1;
  momentum_words(p, &words);
  pl.ulo = (p->precision != CASCADE_FP64 && words == 2) ? sizeof(float) : 0;
  pl.cap4 = (p->particle_cap + 3) & ~3LL;
  pl.ph_cap = next_pow2(p->photon_cap > 0 ? p->photon_cap : p->particle_cap);
  pl.n_pp = n_pp_of(p);
  pl.ring = p->diag_ring > 0 ? p->diag_ring : kDefaultRing;
  return pl;
}

int setup(const cascade_params* params, void* stream, cascade_t** out, bool batch_member = false) {
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
  d.cap4 = pl.cap4;
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
  d.open_bc = params->open_bc;
  d.j_m = params->j_m;
  d.rho_gj = params->rho_gj;
  int words = 1;
  rc = momentum_words(params, &words);
  if (rc) return rc;
  d.u_words = params->precision == CASCADE_FP64 ? 1 : words;
  e = params->precision == CASCADE_FP64 ? configure_fp64(d, h->num_sms) : configure_fp32(d, h->num_sms);
  if (e == cudaErrorNotSupported && d.u_words == 2) {
    snprintf(g_msg, sizeof(g_msg),
             "two-word FP32 momenta need the grid's current to fit shared memory (nx = %d)", params->nx);
    return CASCADE_ERR_INVALID_ARG;
  }
  if (e == cudaErrorInvalidValue && params->open_bc) {
    snprintf(g_msg, sizeof(g_msg), "open boundaries need the grid's E or current to fit shared memory (nx = %d)",
             params->nx);
    return CASCADE_ERR_INVALID_ARG;
  }
  if (e != cudaSuccess) return cuda_fail(e, "configure");

  // device memory
  const size_t R = pl.real;
  for (int s = 0; s < 2; ++s) {
    d.cell[s] = static_cast<int32_t*>(h->dalloc(sizeof(int32_t) * pl.cap4));
    d.off[s] = h->dalloc(R * pl.cap4);
    d.u[s] = h->dalloc(R * pl.cap4);
    if (!d.cell[s] || !d.off[s] || !d.u[s]) return CASCADE_ERR_OOM;
    if (pl.ulo) {
      d.ulo[s] = static_cast<float*>(h->dalloc(pl.ulo * pl.cap4));
      if (!d.ulo[s]) return CASCADE_ERR_OOM;
    }
  }
  d.ph_cell = static_cast<int32_t*>(h->dalloc(sizeof(int32_t) * pl.ph_cap));
  d.ph_off = h->dalloc(R * pl.ph_cap);
  d.E = static_cast<double*>(h->dalloc(sizeof(double) * d.nx));
  d.J = static_cast<double*>(h->dalloc(sizeof(double) * d.nx));
  const size_t acc = params->precision == CASCADE_FP64 ? partial_bytes_fp64() : partial_bytes_fp32();
  if ((d.variant == kSmemESmemS || d.variant == kGlobESmemS) && !batch_member) {
    d.S_part = h->dalloc(acc * (size_t)d.grid_push * d.nxp);
    if (!d.S_part) return CASCADE_ERR_OOM;
  } else {
    // global FP64 current: the single-cascade fallback variants and every
    // batch member (each CTA adds its share of the current here)
    d.S_glob = static_cast<double*>(h->dalloc(sizeof(double) * d.nx));
    if (!d.S_glob) return CASCADE_ERR_OOM;
  }
  if (d.open_bc) {
    // departures per step are bounded by the particles next to the boundaries
    d.hole_cap = (pl.cap4 / 16 > 65536) ? pl.cap4 / 16 : 65536;
    for (int sp = 0; sp < 2; ++sp) {
      d.holes[sp] = static_cast<long long*>(h->dalloc(sizeof(long long) * d.hole_cap));
      d.hole_a[sp] = static_cast<long long*>(h->dalloc(sizeof(long long) * d.hole_cap));
      d.hole_b[sp] = static_cast<long long*>(h->dalloc(sizeof(long long) * d.hole_cap));
      if (!d.holes[sp] || !d.hole_a[sp] || !d.hole_b[sp]) return CASCADE_ERR_OOM;
    }
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
  CUDA_TRY(cudaMemsetAsync(d.uk_part, 0, sizeof(double) * d.grid_push, h->stream));
  if (d.S_glob) CUDA_TRY(cudaMemsetAsync(d.S_glob, 0, sizeof(double) * d.nx, h->stream));
  return CASCADE_OK;
}

// Phase timing of a state upload, for diagnosis: with CASCADE_TRACE_UPLOAD=1
// each mark waits for the stream and prints the host time since the
// previous mark to stderr.  Off by default (the waits serialise the upload).
struct UploadTrace {
  bool on = false;
  std::chrono::steady_clock::time_point t0;
  explicit UploadTrace() {
    const char* v = getenv("CASCADE_TRACE_UPLOAD");
    on = v && *v && atoi(v) != 0;
    t0 = std::chrono::steady_clock::now();
  }
  void mark(cascade_t* h, const char* what) {
    if (!on) return;
    if (h) cudaStreamSynchronize(h->stream);
    const auto t1 = std::chrono::steady_clock::now();
    fprintf(stderr, "cascade upload: %-28s %8.2f ms\n", what,
            std::chrono::duration<double, std::milli>(t1 - t0).count());
    t0 = t1;
  }
};

int upload_E(cascade_t* h, const double* E_host) {
  std::vector<double> E(h->d.nx, h->p.E0);
  if (E_host) memcpy(E.data(), E_host, sizeof(double) * h->d.nx);
  CUDA_TRY(cudaMemcpyAsync(h->d.E, E.data(), sizeof(double) * h->d.nx, cudaMemcpyHostToDevice, h->stream));
  CUDA_TRY(cudaStreamSynchronize(h->stream));
  return CASCADE_OK;
}

// Copy one species from host arrays (H = double or float): cells straight
// into place, offsets and momenta through a device staging buffer in chunks;
// a kernel rounds them to the particle precision and checks every particle.
template <class H>
int upload_species(cascade_t* h, int s, long long n, const int32_t* cell, const H* off, const H* u) {
  if (n == 0) return CASCADE_OK;
  const int f32 = sizeof(H) == sizeof(float) ? 1 : 0;
  unsigned int* bad = reinterpret_cast<unsigned int*>(h->scalar);
  unsigned int nbad = 0;
  UploadTrace tr;
  // Measured: after a cascade that had stepped was destroyed, the copies
  // below, queued without this wait, moved 3.7 GB in 135-160 ms; with it,
  // in 20 ms.  The cause was not found; the wait costs microseconds.
  cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(bad, 0, sizeof(unsigned int), h->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h->d.cell[s], cell, sizeof(int32_t) * n, cudaMemcpyHostToDevice, h->stream);
  auto check = [&](long long first, long long m, const void* so, const void* su) {
    return h->real_size == sizeof(double) ? upload_fp64(h->d, s, first, m, so, su, f32, bad, h->stream)
                                          : upload_fp32(h->d, s, first, m, so, su, f32, bad, h->stream);
  };
  void* stage = nullptr;
  if (sizeof(H) == h->real_size) {
    // the host arrays hold the particle precision: straight into place,
    // then checked there (the kernel reads and rewrites each element)
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->d.off[s], off, sizeof(H) * n, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->d.u[s], u, sizeof(H) * n, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = check(0, n, h->d.off[s], h->d.u[s]);
  } else {
    // FP64 host arrays for an FP32 cascade: through a device staging buffer
    // in chunks, rounded by the kernel
    const long long chunk = n < (1LL << 23) ? n : (1LL << 23);
    const size_t stage_bytes = sizeof(H) * (size_t)chunk;
    if (e == cudaSuccess) {
      if (h->alloc_fn) {
        stage = h->alloc_fn(2 * stage_bytes, (void*)h->stream, h->alloc_ctx);
      } else if (cudaMalloc(&stage, 2 * stage_bytes) != cudaSuccess) {
        cudaGetLastError();
        stage = nullptr;
      }
      if (!stage) {
        cudaStreamSynchronize(h->stream);
        return CASCADE_ERR_OOM;
      }
    }
    H* so = static_cast<H*>(stage);
    H* su = so + chunk;
    for (long long k = 0; k < n && e == cudaSuccess; k += chunk) {
      const long long m = (n - k) < chunk ? (n - k) : chunk;
      e = cudaMemcpyAsync(so, off + k, sizeof(H) * m, cudaMemcpyHostToDevice, h->stream);
      if (e == cudaSuccess) e = cudaMemcpyAsync(su, u + k, sizeof(H) * m, cudaMemcpyHostToDevice, h->stream);
      if (e == cudaSuccess) e = check(k, m, so, su);
    }
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(&nbad, bad, sizeof(unsigned int), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  else cudaStreamSynchronize(h->stream);  // nothing queued may still use the staging buffer
  tr.mark(h, "  copies and checks");
  if (stage) {
    if (h->free_fn) h->free_fn(stage, (void*)h->stream, h->alloc_ctx);
    else cudaFree(stage);
  }
  if (e != cudaSuccess) return cuda_fail(e, "state upload");
  if (nbad) {
    snprintf(g_msg, sizeof(g_msg), "%u particles of species %d outside the grid or not finite", nbad, s);
    return CASCADE_ERR_INVALID_ARG;
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

// Copies to the host go through the handle's own stream, so they never wait
// for work queued on other streams.
int d2h(cascade_t* h, void* dst, const void* src, size_t bytes) {
  CUDA_TRY(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(cudaStreamSynchronize(h->stream));
  return CASCADE_OK;
}

int read_ctl(cascade_t* h, Ctl* c) {
  int rc = d2h(h, c, h->d.ctl, sizeof(Ctl));
  if (rc) return rc;
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

// Section 3 initial state (uniform E0, quiet-start pairs, seeded momenta).
int create_seeded(const cascade_params* params, void* cuda_stream, bool batch_member, cascade_t** out) {
  *out = nullptr;
  cascade_t* h = nullptr;
  int rc = setup(params, cuda_stream, &h, batch_member);
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

}  // namespace

extern "C" {

int cascade_set_allocator(cascade_alloc_fn alloc_fn, cascade_free_fn free_fn, void* ctx) {
  g_msg[0] = '\0';  // a message describes this call only
  if ((alloc_fn == nullptr) != (free_fn == nullptr)) return CASCADE_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(g_alloc_mu);
  g_alloc = alloc_fn;
  g_free = free_fn;
  g_ctx = ctx;
  return CASCADE_OK;
}

int cascade_create(const cascade_params* params, void* cuda_stream, cascade_t** out) {
  g_msg[0] = '\0';  // a message describes this call only
  if (!out) return CASCADE_ERR_INVALID_ARG;
  return create_seeded(params, cuda_stream, false, out);
}

int cascade_create_from_state(const cascade_params* params, int64_t n_elec, const int32_t* cell_e,
                              const double* off_e, const double* u_e, int64_t n_posi, const int32_t* cell_p,
                              const double* off_p, const double* u_p, const double* E_host, void* cuda_stream,
                              cascade_t** out) {
  g_msg[0] = '\0';  // a message describes this call only
  if (!out || n_elec < 0 || n_posi < 0) return CASCADE_ERR_INVALID_ARG;
  if ((n_elec > 0 && (!cell_e || !off_e || !u_e)) || (n_posi > 0 && (!cell_p || !off_p || !u_p)))
    return CASCADE_ERR_INVALID_ARG;
  cascade_t* h = nullptr;
  UploadTrace tr;
  int rc = setup(params, cuda_stream, &h);
  tr.mark(rc == CASCADE_OK ? h : nullptr, "setup (allocations)");
  if (rc == CASCADE_OK && (n_elec > params->particle_cap || n_posi > params->particle_cap)) {
    snprintf(g_msg, sizeof(g_msg), "state exceeds particle_cap");
    rc = CASCADE_ERR_CAPACITY;
  }
  if (rc == CASCADE_OK) rc = upload_E(h, E_host);
  tr.mark(rc == CASCADE_OK ? h : nullptr, "E");
  if (rc == CASCADE_OK) rc = upload_species(h, 0, n_elec, cell_e, off_e, u_e);
  tr.mark(rc == CASCADE_OK ? h : nullptr, "species 0");
  if (rc == CASCADE_OK) rc = upload_species(h, 1, n_posi, cell_p, off_p, u_p);
  tr.mark(rc == CASCADE_OK ? h : nullptr, "species 1");
  if (rc == CASCADE_OK) rc = set_counts(h, n_elec, n_posi);
  tr.mark(rc == CASCADE_OK ? h : nullptr, "counts");
  if (rc != CASCADE_OK) {
    cascade_destroy(h);
    return rc;
  }
  *out = h;
  return CASCADE_OK;
}

int cascade_create_from_state_f32(const cascade_params* params, int64_t n_elec, const int32_t* cell_e,
                                  const float* off_e, const float* u_e, int64_t n_posi, const int32_t* cell_p,
                                  const float* off_p, const float* u_p, const double* E_host, void* cuda_stream,
                                  cascade_t** out) {
  g_msg[0] = '\0';  // a message describes this call only
  if (!out || n_elec < 0 || n_posi < 0) return CASCADE_ERR_INVALID_ARG;
  if ((n_elec > 0 && (!cell_e || !off_e || !u_e)) || (n_posi > 0 && (!cell_p || !off_p || !u_p)))
    return CASCADE_ERR_INVALID_ARG;
  cascade_t* h = nullptr;
  UploadTrace tr;
  int rc = setup(params, cuda_stream, &h);
  tr.mark(rc == CASCADE_OK ? h : nullptr, "setup (allocations)");
  if (rc == CASCADE_OK && (n_elec > params->particle_cap || n_posi > params->particle_cap)) {
    snprintf(g_msg, sizeof(g_msg), "state exceeds particle_cap");
    rc = CASCADE_ERR_CAPACITY;
  }
  if (rc == CASCADE_OK) rc = upload_E(h, E_host);
  tr.mark(rc == CASCADE_OK ? h : nullptr, "E");
  if (rc == CASCADE_OK) rc = upload_species(h, 0, n_elec, cell_e, off_e, u_e);
  tr.mark(rc == CASCADE_OK ? h : nullptr, "species 0");
  if (rc == CASCADE_OK) rc = upload_species(h, 1, n_posi, cell_p, off_p, u_p);
  tr.mark(rc == CASCADE_OK ? h : nullptr, "species 1");
  if (rc == CASCADE_OK) rc = set_counts(h, n_elec, n_posi);
  tr.mark(rc == CASCADE_OK ? h : nullptr, "counts");
  if (rc != CASCADE_OK) {
    cascade_destroy(h);
    return rc;
  }
  *out = h;
  return CASCADE_OK;
}

int cascade_step(cascade_t* h, int32_t nsteps) {
  g_msg[0] = '\0';  // a message describes this call only
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
  g_msg[0] = '\0';  // a message describes this call only
  if (!h) return CASCADE_ERR_INVALID_ARG;
  cudaSetDevice(h->device);
  Ctl c;
  int rc = read_ctl(h, &c);
  if (rc) return rc;
  return h->sticky;
}

int cascade_diag(cascade_t* h, cascade_diag_t* host_out, int32_t max, int32_t* n_out, double* E_host,
                 double* J_host) {
  g_msg[0] = '\0';  // a message describes this call only
  if (!h || max < 0 || (max > 0 && !host_out)) return CASCADE_ERR_INVALID_ARG;
  cudaSetDevice(h->device);
  Ctl c;
  int rc = read_ctl(h, &c);
  if (rc) return rc;
  const long long kept = c.step < h->d.ring_n ? c.step : h->d.ring_n;
  const long long n = kept < max ? kept : max;
  const long long first = c.step - n;  // records of steps first+1 .. c.step
  long long done = 0;
  if (n == 1) {  // the latest record came with the counters: no second copy
    host_out[0] = c.last;
    done = 1;
  }
  while (done < n) {
    const long long slot = (first + done) % h->d.ring_n;
    long long run = h->d.ring_n - slot;
    if (run > n - done) run = n - done;
    rc = d2h(h, host_out + done, h->d.ring + slot, sizeof(cascade_diag_t) * run);
    if (rc) return rc;
    done += run;
  }
  if (n_out) *n_out = (int32_t)n;
  if (E_host && (rc = d2h(h, E_host, h->d.E, sizeof(double) * h->d.nx))) return rc;
  if (J_host && (rc = d2h(h, J_host, h->d.J, sizeof(double) * h->d.nx))) return rc;
  return h->sticky;
}

int cascade_record_enqueue(cascade_t* h) {
  g_msg[0] = '\0';  // a message describes this call only
  if (!h) return CASCADE_ERR_INVALID_ARG;
  cudaSetDevice(h->device);
  if (!h->h_rec) {
    CUDA_TRY(cudaMallocHost(&h->h_rec, sizeof(Ctl) * kRecRing));
    for (cudaEvent_t& e : h->ev_rec) CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  }
  const int k = (int)(h->rec_issued % kRecRing);
  if (h->rec_issued - h->rec_read >= kRecRing) {
    // the ring is full: wait for its oldest copy (the host is then at most
    // kRecRing steps ahead of the device) and keep that record for the poll
    CUDA_TRY(cudaEventSynchronize(h->ev_rec[k]));
    const Ctl& c = h->h_rec[k];
    if (c.err && !h->sticky) h->sticky = c.err;
    h->rec_landed.push_back(c.last);
    ++h->rec_read;
  }
  // the whole control block: the newest record and the device's error flag
  CUDA_TRY(cudaMemcpyAsync(&h->h_rec[k], h->d.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(cudaEventRecord(h->ev_rec[k], h->stream));
  ++h->rec_issued;
  return CASCADE_OK;
}

int32_t cascade_record_copy_bytes(void) { return (int32_t)sizeof(Ctl); }

int cascade_record_poll(cascade_t* h, cascade_diag_t* out, int32_t max, int32_t wait, int32_t* n_out) {
  g_msg[0] = '\0';  // a message describes this call only
  if (!h || max < 0 || (max > 0 && !out) || !n_out) return CASCADE_ERR_INVALID_ARG;
  cudaSetDevice(h->device);
  int32_t n = 0;
  while (n < max && !h->rec_landed.empty()) {
    out[n++] = h->rec_landed.front();
    h->rec_landed.pop_front();
  }
  while (n < max && h->rec_read < h->rec_issued) {
    const int k = (int)(h->rec_read % kRecRing);
    if (wait) {
      CUDA_TRY(cudaEventSynchronize(h->ev_rec[k]));
    } else {
      const cudaError_t e = cudaEventQuery(h->ev_rec[k]);
      if (e == cudaErrorNotReady) {
        (void)cudaGetLastError();
        break;
      }
      if (e != cudaSuccess) return cuda_fail(e, "record event");
    }
    const Ctl& c = h->h_rec[k];
    if (c.err && !h->sticky) h->sticky = c.err;
    out[n++] = c.last;
    ++h->rec_read;
  }
  *n_out = n;
  return h->sticky;
}

int cascade_set_gauss_every(cascade_t* h, int32_t every) {
  g_msg[0] = '\0';  // a message describes this call only
  if (!h || every < 0) return CASCADE_ERR_INVALID_ARG;
  cudaSetDevice(h->device);
  if (every > 0 && !h->d.gauss_rho) {
    h->d.gauss_rho = static_cast<double*>(h->dalloc(sizeof(double) * h->d.nx));
    h->d.gauss_out = static_cast<double*>(h->dalloc(sizeof(double)));
    if (!h->d.gauss_rho || !h->d.gauss_out) return CASCADE_ERR_OOM;
    CUDA_TRY(cudaMemsetAsync(h->d.gauss_rho, 0, sizeof(double) * h->d.nx, h->stream));
  }
  if (every != h->d.gauss_every && h->graph) {  // the captured step no longer matches
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    cudaGraphExecDestroy(h->graph);
    h->graph = nullptr;
  }
  h->d.gauss_every = every;
  return CASCADE_OK;
}

int cascade_gauss(cascade_t* h, double* resid_out) {
  g_msg[0] = '\0';  // a message describes this call only
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
  g_msg[0] = '\0';  // a message describes this call only
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

int cascade_histogram(cascade_t* h, int32_t species, int32_t quantity, int32_t nbins, double lo, double hi,
                      int64_t* counts_host) {
  g_msg[0] = '\0';  // a message describes this call only
  if (!h || species < 0 || species > 1 || quantity < 0 || quantity > 2 || nbins < 1 || nbins > 65536 ||
      !(hi > lo) || !counts_host)
    return CASCADE_ERR_INVALID_ARG;
  cudaSetDevice(h->device);
  void* buf = nullptr;
  const size_t bytes = sizeof(unsigned long long) * (size_t)nbins;
  if (h->alloc_fn) buf = h->alloc_fn(bytes, (void*)h->stream, h->alloc_ctx);
  else if (cudaMalloc(&buf, bytes) != cudaSuccess) buf = nullptr;
  if (!buf) return CASCADE_ERR_OOM;
  unsigned long long* out = static_cast<unsigned long long*>(buf);
  cudaError_t e = h->real_size == sizeof(double)
                      ? histogram_fp64(h->d, species, quantity, nbins, lo, hi, out, h->stream)
                      : histogram_fp32(h->d, species, quantity, nbins, lo, hi, out, h->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(counts_host, out, bytes, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (h->free_fn) h->free_fn(buf, (void*)h->stream, h->alloc_ctx);
  else cudaFree(buf);
  if (e != cudaSuccess) return cuda_fail(e, "histogram");
  return h->sticky;
}

int cascade_particles(cascade_t* h, int32_t species, int64_t max, int32_t* cell, double* off, double* u,
                      int64_t* n_out) {
  g_msg[0] = '\0';  // a message describes this call only
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
      if (h->d.ulo[species]) {  // two-word momenta: add the low word
        CUDA_TRY(cudaMemcpy(tmp.data(), h->d.ulo[species], sizeof(float) * n, cudaMemcpyDeviceToHost));
        for (long long i = 0; i < n; ++i) u[i] += (double)tmp[i];
      }
    }
  }
  return h->sticky;
}

int cascade_set_timing(cascade_t* h, int32_t enable) {
  g_msg[0] = '\0';  // a message describes this call only
  if (!h) return CASCADE_ERR_INVALID_ARG;
  h->timing = enable != 0;
  return CASCADE_OK;
}

int cascade_timing(cascade_t* h, double* particle_kernel_ms, int64_t* particle_kernel_launches,
                   int64_t* kernels_launched) {
  g_msg[0] = '\0';  // a message describes this call only
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
  for (cudaEvent_t e : h->ev_rec)
    if (e) cudaEventDestroy(e);
  if (h->h_rec) cudaFreeHost(h->h_rec);
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
  g_msg[0] = '\0';  // a message describes this call only
  int rc = validate(params);
  if (rc) return rc;
  int words = 1;
  if ((rc = momentum_words(params, &words))) return rc;
  const Plan pl = plan_of(params);
  if (n_pp_out) *n_pp_out = pl.n_pp;
  if (device_bytes_out) {
    size_t b = 2 * (sizeof(int32_t) + 2 * pl.real + pl.ulo) * (size_t)pl.cap4;
    b += (sizeof(int32_t) + pl.real) * (size_t)pl.ph_cap;
    b += sizeof(double) * (size_t)params->nx * 4;
    // per-CTA partials: at most 4 CTAs per SM on a 152-SM part
    b += pl.real * (size_t)(4 * 152) * (size_t)((params->nx + 31) & ~31);
    b += sizeof(cascade_diag_t) * (size_t)pl.ring + 64 * 1024;
    *device_bytes_out = b;
  }
  return CASCADE_OK;
}

int cascade_momentum_words(const cascade_params* params, int32_t* words_out) {
  g_msg[0] = '\0';  // a message describes this call only
  int rc = validate(params);
  if (rc) return rc;
  int words = 1;
  rc = momentum_words(params, &words);
  if (rc) return rc;
  if (words_out) *words_out = words;
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

// ---------------------------------------------------------------------------
// Batches of cascades.
// ---------------------------------------------------------------------------
namespace {

constexpr int kSnapRing = 4;  // remaining-count snapshots in flight

// Slices of the constant-bank member table (one table per precision's
// kernel translation unit; a batch holds one slice of n_slots entries for its
// life).  First fit; -1 when no run of n free entries is left, and the batch
// then has only the shared-memory kernel.
std::mutex g_const_mu;
std::vector<char> g_const_used[2];

int const_slice_alloc(int precision, int n) {
  std::lock_guard<std::mutex> lk(g_const_mu);
  std::vector<char>& used = g_const_used[precision == CASCADE_FP64 ? 0 : 1];
  if (used.empty()) used.assign(kConstMembers, 0);
  for (int base = 0; base + n <= kConstMembers; ++base) {
    int k = 0;
    while (k < n && !used[base + k]) ++k;
    if (k == n) {
      for (int i = 0; i < n; ++i) used[base + i] = 1;
      return base;
    }
    base += k;
  }
  return -1;
}

void const_slice_free(int precision, int base, int n) {
  if (base < 0) return;
  std::lock_guard<std::mutex> lk(g_const_mu);
  std::vector<char>& used = g_const_used[precision == CASCADE_FP64 ? 0 : 1];
  for (int i = 0; i < n && base + i < (int)used.size(); ++i) used[base + i] = 0;
}

BatchMember member_of(const Dev& d) {
  BatchMember m{};
  for (int s = 0; s < 2; ++s) {
    m.cell[s] = d.cell[s];
    m.off[s] = d.off[s];
    m.u[s] = d.u[s];
  }
  m.ph_cell = d.ph_cell;
  m.ph_off = d.ph_off;
  m.E = d.E;
  m.S_glob = d.S_glob;
  m.uk_part = d.uk_part;
  m.ctl = d.ctl;
  m.cap4 = d.cap4;
  m.ph_cap = d.ph_cap;
  m.dt = d.dt;
  m.dtdx = d.dtdx;
  m.gamma_thr = d.gamma_thr;
  m.eps_gamma = d.eps_gamma;
  m.lpp_frac = d.lpp_frac;
  m.nx = d.nx;
  m.lpp_int = d.lpp_int;
  return m;
}

}  // namespace

struct cascade_batch {
  int n_slots = 0;
  int precision = CASCADE_FP32_MIXED;
  int max_nx = 0;
  size_t budget = 0;
  size_t used = 0;
  int device = 0;
  int num_sms = 0;
  cudaStream_t stream = nullptr;       // caller's stream: all batch steps
  cudaStream_t init_stream = nullptr;  // private: member allocation and seeding
  cudaStream_t cap_stream = nullptr;   // private: graph capture
  cudaGraphExec_t graph = nullptr;
  std::vector<cascade_t*> members;
  std::vector<long long> admit_seq;    // run sequence number at admission
  std::vector<char> reported;
  // device tables
  Dev* d_devs = nullptr;
  long long* d_remaining = nullptr;
  long long* d_item_start = nullptr;
  void* d_block = nullptr;             // one allocation holding the tables
  // pinned host mirrors
  Dev* h_devs = nullptr;
  long long* h_set = nullptr;          // staging for remaining-count updates
  long long* h_snap[kSnapRing] = {nullptr};
  cudaEvent_t ev_snap[kSnapRing] = {nullptr};
  long long snap_seq[kSnapRing] = {0};
  // the newest snapshot seen landed (copied out of the ring before its slot
  // is reused, so a host that runs ahead of the GPU still sees completions)
  std::vector<long long> landed;
  long long landed_seq = 0;
  long long run_seq = 0;               // runs enqueued so far
  int snap_next = 0;
  cudaEvent_t ev_init = nullptr;
  BatchDev bd{};
  int grid = 0, block = 0, dep = 0;
  size_t smem = 0;
  // kernel timing (cascade_batch_set_timing)
  bool timing = false;
  std::vector<cudaEvent_t> ev_pool;
  size_t ev_used = 0;
  long long kernels_launched = 0;
  // launch variant of the particle kernel and its autotuning
  cascade_batch_variant var{};
  int var_source = CASCADE_VARIANT_DEFAULT;
  double var_ns_per_unit = 0.0;
  bool tune_auto = false;              // tune when the size class changes (at a step or run with work)
  long long tune_warmup = 256;         // steps run before a pass that the cache cannot answer
  int tune_rounds = 4;                 // rounds of candidates per tuning pass
  int tune_use_cache = 1;              // 0: the next pass measures even on a cache hit
  std::string tuned_key;               // size class of the variant in use ("" = none yet)
  long long tune_countdown = -1;       // steps left before a pending tuning pass (-1: none pending)
  std::vector<cascade_batch_variant> tune_cands;  // the last pass's candidates ...
  std::vector<double> tune_ns;                    // ... and their ns per work unit
  long long* d_units = nullptr;        // work units of each tuning step (device)
  long long seed_particles = 0;        // seed particles of the members (size class of the batch)
  // constant-bank kernel (launch shape 4): the batch's slice of the member table
  int const_base = -1;
  BatchMember* h_members = nullptr;    // pinned staging of the table entries
  int* d_member_ctas = nullptr;

  cudaError_t launch_step() {
    cudaEvent_t before = nullptr, after = nullptr;
    if (timing) {
      while (ev_pool.size() < ev_used + 2) {
        cudaEvent_t e;
        cudaError_t r = cudaEventCreate(&e);
        if (r != cudaSuccess) return r;
        ev_pool.push_back(e);
      }
      before = ev_pool[ev_used];
      after = ev_pool[ev_used + 1];
      ev_used += 2;
      kernels_launched += 4;
    }
    return precision == CASCADE_FP64 ? batch_step_fp64(bd, grid, block, smem, dep, stream, before, after)
                                     : batch_step_fp32(bd, grid, block, smem, dep, stream, before, after);
  }
};

namespace {

constexpr int kTuneMaxSteps = 256;  // tuning steps logged per tuning pass
// constant-bank batch kernel: working CTAs per SM and step.  256-cascade
// scan, 3000 steps: 4: 2.33e11, 8: 2.41e11, 16: 2.43e11 particle-steps/s;
// its first 300 steps (the growth phase): 8: 2.01e11, 16: 1.91e11 (at 16
// the grid carries twice as many CTAs that find no work and exit)
constexpr int kConstCtasPerSm = 8;

// Launch parameters of one variant (no graph change); CASCADE_ERR_INVALID_ARG
// when the variant does not fit this batch (staging beside a large grid, a
// form the precision has no kernel for).
int batch_config_variant(cascade_batch_t* b, const cascade_batch_variant& v) {
  if (v.shape < 0 || v.shape > 4 || (v.stage != 0 && v.stage != 1) || v.prefetch < 0 || v.prefetch > 8 ||
      v.member_cost < 0)
    return CASCADE_ERR_INVALID_ARG;
  if (v.shape == 4 && b->const_base < 0) return CASCADE_ERR_INVALID_ARG;  // no slice of the member table
  const int fine = b->precision == CASCADE_FP32_MIXED_FINE ? 1 : 0;
  int grid = 0, block = 0, dep = 0;
  size_t smem = 0;
  const cudaError_t e =
      b->precision == CASCADE_FP64
          ? batch_configure_fp64(b->max_nx, 0, b->num_sms, v.shape, v.stage, &grid, &block, &smem, &dep)
          : batch_configure_fp32(b->max_nx, fine, b->num_sms, v.shape, v.stage, &grid, &block, &smem, &dep);
  if (e == cudaErrorInvalidValue) return CASCADE_ERR_INVALID_ARG;
  if (e != cudaSuccess) return cuda_fail(e, "batch configure");
  b->grid = grid;
  b->block = block;
  b->smem = smem;
  b->dep = dep;
  b->bd.prefetch = v.prefetch;
  b->bd.member_cost = v.member_cost;
  return CASCADE_OK;
}

// Make v the batch's variant; a captured graph of the old one is dropped.
int batch_apply_variant(cascade_batch_t* b, const cascade_batch_variant& v, int source, double ns_per_unit) {
  const int rc = batch_config_variant(b, v);
  if (rc) return rc;
  b->var = v;
  b->var_source = source;
  b->var_ns_per_unit = ns_per_unit;
  if (b->graph) {
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
  return CASCADE_OK;
}

int batch_occupied(const cascade_batch_t* b) {
  int occ = 0;
  for (cascade_t* h : b->members) occ += h != nullptr;
  return occ;
}

// Autotuning of the batch's launch shape: the candidates -- the four launch shapes
// with the particles staged through shared memory (FP32) and without it,
// then with an L2 prefetch one iteration ahead -- run in turn, one batch step
// each, round after round, so that each is measured over the same stretch of
// the run (the particle counts grow during a cascade).  Every tuning step is
// a real step of the members' work.  The score is the particle kernel's time
// (CUDA events) per work unit of the partition (4-particle chunks plus the
// fixed share per member, logged from the plan kernel every step); the
// fastest candidate is kept and stored in the cache under the batch's size
// class.  Runs at most max_steps steps; returns the number run in *used.
int batch_tune(cascade_batch_t* b, long long max_steps, long long* used) {
  *used = 0;
  if (!b->tune_auto || batch_occupied(b) == 0) return CASCADE_OK;
  char key[128];
  int rc = cascade_tune_key(b->precision, b->max_nx, b->seed_particles, batch_occupied(b), key, sizeof(key));
  if (rc) return rc;
  if (b->tuned_key == key) return CASCADE_OK;  // the variant in use was picked for this size class
  const char* path = cascade_tune_cache_path();
  if (b->tune_use_cache) {
    cascade_batch_variant v{};
    int32_t found = 0;
    cascade_tune_cache_lookup(path, key, &v, &found);
    if (found && batch_apply_variant(b, v, CASCADE_VARIANT_CACHED, 0.0) == CASCADE_OK) {
      b->tuned_key = key;
      b->tune_countdown = -1;
      return CASCADE_OK;
    }
  }
  // a miss: measure once the members have grown past their seeds (a cascade
  // multiplies its particles many times in its first steps, and the variant
  // that wins on the seeds is not the one that wins on the grown state)
  if (b->tune_countdown < 0) b->tune_countdown = b->tune_warmup;
  if (b->tune_countdown > 0) return CASCADE_OK;
  std::vector<cascade_batch_variant> cand;
  for (int stage = 1; stage >= 0; --stage)
    for (int shape : {4, 3, 2, 1, 0}) {
      const cascade_batch_variant v{shape, stage, stage ? 0 : 1, 1024};
      if (batch_config_variant(b, v) == CASCADE_OK) cand.push_back(v);
    }
  if (cand.empty()) return CASCADE_ERR_INVALID_ARG;
  const int V = (int)cand.size();
  long long steps = (long long)V * b->tune_rounds;
  if (steps > max_steps) steps = max_steps;
  if (steps > kTuneMaxSteps) steps = kTuneMaxSteps;
  if (steps < V) {  // too few steps to measure every candidate: keep the current variant
    return CASCADE_OK;
  }
  // direct launches with an event pair around each particle kernel
  const bool was_timing = b->timing;
  const size_t ev0 = b->ev_used;
  b->timing = true;
  for (long long k = 0; k < steps; ++k) {
    rc = batch_config_variant(b, cand[k % V]);
    if (rc) break;
    cudaError_t e = b->launch_step();
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(b->d_units + k, b->d_item_start + b->n_slots, sizeof(long long), cudaMemcpyDeviceToDevice,
                          b->stream);
    if (e != cudaSuccess) {
      rc = cuda_fail(e, "tuning step");
      break;
    }
    *used = k + 1;
  }
  b->timing = was_timing;
  std::vector<long long> units(kTuneMaxSteps, 0);
  std::vector<double> ms(V, 0.0), un(V, 0.0);
  if (rc == CASCADE_OK) {
    cudaError_t e = cudaStreamSynchronize(b->stream);
    if (e == cudaSuccess)
      e = cudaMemcpy(units.data(), b->d_units, sizeof(long long) * (size_t)*used, cudaMemcpyDeviceToHost);
    for (long long k = 0; k < *used && e == cudaSuccess; ++k) {
      float t = 0.f;
      e = cudaEventElapsedTime(&t, b->ev_pool[ev0 + 2 * k], b->ev_pool[ev0 + 2 * k + 1]);
      ms[k % V] += t;
      un[k % V] += (double)units[k];
    }
    if (e != cudaSuccess) rc = cuda_fail(e, "tuning events");
  }
  // the tuning events are not part of the caller's timing
  b->ev_used = ev0;
  if (!was_timing) b->kernels_launched = 0;
  if (rc) {
    batch_config_variant(b, b->var);
    return rc;
  }
  int best = -1;
  double best_ns = 0.0;
  for (int v = 0; v < V; ++v) {
    if (!(un[v] > 0)) continue;
    const double ns = 1e6 * ms[v] / un[v];
    if (best < 0 || ns < best_ns) {
      best = v;
      best_ns = ns;
    }
  }
  if (best < 0) {  // no work was measured (idle members): keep the current variant
    batch_config_variant(b, b->var);
    return CASCADE_OK;
  }
  cascade_tune_cache_store(path, key, &cand[best], best_ns);
  g_msg[0] = '\0';  // an unwritable cache is not this call's failure
  b->tuned_key = key;
  b->tune_use_cache = 1;
  b->tune_countdown = -1;
  b->tune_cands = cand;
  b->tune_ns.assign(V, 0.0);
  for (int v = 0; v < V; ++v) b->tune_ns[v] = un[v] > 0 ? 1e6 * ms[v] / un[v] : 0.0;
  return batch_apply_variant(b, cand[best], CASCADE_VARIANT_TUNED, best_ns);
}

int batch_capture(cascade_batch_t* b) {
  if (!b->cap_stream) CUDA_TRY(cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking));
  cudaGraph_t g = nullptr;
  CUDA_TRY(cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal));
  cudaError_t e = cudaSuccess;
  for (int k = 0; k < kGraphSteps && e == cudaSuccess; ++k)
    e = b->precision == CASCADE_FP64 ? batch_step_fp64(b->bd, b->grid, b->block, b->smem, b->dep, b->cap_stream)
                                     : batch_step_fp32(b->bd, b->grid, b->block, b->smem, b->dep, b->cap_stream);
  cudaError_t e2 = cudaStreamEndCapture(b->cap_stream, &g);
  if (e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return cuda_fail(e, "capture batch step");
  }
  if (e2 != cudaSuccess) return cuda_fail(e2, "cudaStreamEndCapture");
  e = cudaGraphInstantiate(&b->graph, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
  return CASCADE_OK;
}

// A snapshot slot whose copy has landed: keep it if it is the newest seen.
void batch_harvest(cascade_batch_t* b, int k) {
  if (b->snap_seq[k] <= b->landed_seq) return;
  b->landed.assign(b->h_snap[k], b->h_snap[k] + b->n_slots);
  b->landed_seq = b->snap_seq[k];
}

// Queue nsteps batch steps and a snapshot of the remaining counts.
int batch_enqueue(cascade_batch_t* b, int nsteps) {
  int left = nsteps;
  if (b->timing) {  // every step launched directly, with events around the particle kernel
    for (; left > 0; --left) CUDA_TRY(b->launch_step());
  }
  if (left >= kGraphSteps && !b->graph) {
    int rc = batch_capture(b);
    if (rc) return rc;
  }
  while (left >= kGraphSteps) {
    CUDA_TRY(cudaGraphLaunch(b->graph, b->stream));
    left -= kGraphSteps;
  }
  for (; left > 0; --left) CUDA_TRY(b->launch_step());
  const int k = b->snap_next;
  // the slot's previous snapshot must have landed before it is overwritten
  CUDA_TRY(cudaEventSynchronize(b->ev_snap[k]));
  if (b->snap_seq[k]) batch_harvest(b, k);
  b->run_seq += 1;
  CUDA_TRY(cudaMemcpyAsync(b->h_snap[k], b->d_remaining, sizeof(long long) * b->n_slots, cudaMemcpyDeviceToHost,
                           b->stream));
  CUDA_TRY(cudaEventRecord(b->ev_snap[k], b->stream));
  b->snap_seq[k] = b->run_seq;
  b->snap_next = (k + 1) % kSnapRing;
  return CASCADE_OK;
}

int batch_member_check(cascade_batch_t* b, int slot) {
  if (!b || slot < 0 || slot >= b->n_slots || !b->members[slot]) return CASCADE_ERR_INVALID_ARG;
  return CASCADE_OK;
}

bool same_kernel_class(int a, int c) { return (a == CASCADE_FP64) == (c == CASCADE_FP64) && a == c; }

// Tuning inside a call that has *steps steps to run: a size class the cache
// cannot answer is measured after warmup steps of the current variant (which
// may span several calls); the steps run here are taken off *steps.
int batch_tune_with_warmup(cascade_batch_t* b, long long* steps, long long warmup) {
  long long used = 0;
  int rc = batch_tune(b, *steps, &used);  // a cache hit, or arms the countdown
  if (rc || b->tune_countdown < 0) {
    *steps -= used;
    return rc;
  }
  if (b->tune_countdown > warmup) b->tune_countdown = warmup;
  if (b->tune_countdown > 0) {
    const long long w = b->tune_countdown < *steps ? b->tune_countdown : *steps;
    if ((rc = batch_enqueue(b, (int)w))) return rc;
    *steps -= w;
    b->tune_countdown -= w;
  }
  if (b->tune_countdown == 0 && *steps > 0) {
    rc = batch_tune(b, *steps, &used);
    *steps -= used;
  }
  return rc;
}

// Batch members keep one-word FP32 momenta (the batched particle kernel has
// no two-word form).
// What a batch member may not be: two-word FP32 momenta, or more particles
// per species than the batched kernel's 32-bit chunk indices cover.
int batch_member_params(const cascade_params* p) {
  if (p->particle_cap > kBatchMaxCap) {
    snprintf(g_msg, sizeof(g_msg), "batch members hold at most %lld particles per species (particle_cap %lld)",
             (long long)kBatchMaxCap, (long long)p->particle_cap);
    return CASCADE_ERR_INVALID_ARG;
  }
  int words = 1;
  int rc = momentum_words(p, &words);
  if (rc) return rc;
  if (p->precision != CASCADE_FP64 && words == 2) {
    snprintf(g_msg, sizeof(g_msg),
             "batch members keep one-word FP32 momenta; these parameters need two (run the cascade alone)");
    return CASCADE_ERR_INVALID_ARG;
  }
  return CASCADE_OK;
}

}  // namespace

extern "C" {

int cascade_batch_create_slots(int32_t max_slots, int32_t precision, int32_t max_nx, size_t hbm_budget,
                               void* cuda_stream, cascade_batch_t** out) {
  g_msg[0] = '\0';  // a message describes this call only
  if (!out || max_slots < 1 || max_nx < 2 ||
      (precision != CASCADE_FP64 && precision != CASCADE_FP32_MIXED && precision != CASCADE_FP32_MIXED_FINE)) {
    snprintf(g_msg, sizeof(g_msg), "batch: out is required, max_slots >= 1, max_nx >= 2, known precision");
    return CASCADE_ERR_INVALID_ARG;
  }
  *out = nullptr;
  cascade_batch_t* b = new (std::nothrow) cascade_batch_t();
  if (!b) return CASCADE_ERR_OOM;
  b->n_slots = max_slots;
  b->precision = precision;
  b->max_nx = max_nx;
  b->budget = hbm_budget;
  b->stream = (cudaStream_t)cuda_stream;
  b->members.assign(max_slots, nullptr);
  b->admit_seq.assign(max_slots, 0);
  b->reported.assign(max_slots, 0);
  auto fail = [&](int code) {
    cascade_batch_destroy(b);
    return code;
  };
  cudaError_t e = cudaGetDevice(&b->device);
  if (e != cudaSuccess) return fail(cuda_fail(e, "cudaGetDevice"));
  e = cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, b->device);
  if (e != cudaSuccess) return fail(cuda_fail(e, "cudaDeviceGetAttribute"));
  // a slice of the constant-bank member table (FP32 batches), needed before
  // any variant of launch shape 4 can be configured
  if (precision != CASCADE_FP64) b->const_base = const_slice_alloc(precision, max_slots);
  // default variant, the best measured on the 256-cascade scan: the
  // constant-bank kernel (FP32 with a slice of the member table) with the
  // particles staged through shared memory, else the persistent kernel at
  // 640 threads and 96 registers; staged where that fits, else with an L2
  // prefetch one iteration ahead
  {
    const int st = precision == CASCADE_FP64 ? 0 : 1;
    cascade_batch_variant v{b->const_base >= 0 ? 4 : 3, st, st ? 0 : 1, 1024};
    int rc = batch_config_variant(b, v);
    if (rc == CASCADE_ERR_INVALID_ARG && v.shape == 4) {
      v.shape = 3;
      rc = batch_config_variant(b, v);
    }
    if (rc == CASCADE_ERR_INVALID_ARG && v.stage) {
      v.stage = 0;
      v.prefetch = 1;
      rc = batch_config_variant(b, v);
    }
    if (rc == CASCADE_ERR_INVALID_ARG) {
      snprintf(g_msg, sizeof(g_msg), "max_nx = %d does not fit the batch kernel's shared memory", max_nx);
      return fail(CASCADE_ERR_INVALID_ARG);
    }
    if (rc) return fail(rc);
    b->var = v;
    b->var_source = CASCADE_VARIANT_DEFAULT;
    // forced picks for measurements: any of these variables fixes the
    // variant and turns tuning off
    const char* names[4] = {"CASCADE_BATCH_SHAPE", "CASCADE_BATCH_STAGE", "CASCADE_BATCH_PREFETCH",
                            "CASCADE_BATCH_MEMBER_COST"};
    int32_t* fields[4] = {&v.shape, &v.stage, &v.prefetch, &v.member_cost};
    bool forced = false;
    for (int i = 0; i < 4; ++i) {
      const char* ev = getenv(names[i]);
      if (ev && *ev) {
        *fields[i] = atoi(ev);
        forced = true;
      }
    }
    if (forced) {
      if (getenv("CASCADE_BATCH_STAGE") && !getenv("CASCADE_BATCH_PREFETCH")) v.prefetch = v.stage ? 0 : 1;
      if ((rc = batch_config_variant(b, v))) {
        snprintf(g_msg, sizeof(g_msg), "the forced batch variant (CASCADE_BATCH_*) does not fit this batch");
        return fail(rc);
      }
      b->var = v;
      b->var_source = CASCADE_VARIANT_FORCED;
    } else {
      const char* tune = getenv("CASCADE_BATCH_TUNE");
      b->tune_auto = !(tune && *tune && atoi(tune) == 0);
    }
  }
  // device tables in one allocation
  const size_t n = (size_t)max_slots;
  const size_t b_devs = (sizeof(Dev) * n + 255) & ~size_t(255);
  const size_t b_rem = (sizeof(long long) * n + 255) & ~size_t(255);
  const size_t b_items = (sizeof(long long) * (n + 1) + 255) & ~size_t(255);
  const size_t b_units = sizeof(long long) * kTuneMaxSteps;
  const size_t b_ctas = (sizeof(int) * n + 255) & ~size_t(255);
  const size_t total = b_devs + b_rem + b_items + b_units + b_ctas;
  e = cudaMalloc(&b->d_block, total);
  if (e != cudaSuccess) return fail(cuda_fail(e, "cudaMalloc batch tables"));
  char* base = static_cast<char*>(b->d_block);
  b->d_devs = reinterpret_cast<Dev*>(base);
  b->d_remaining = reinterpret_cast<long long*>(base + b_devs);
  b->d_item_start = reinterpret_cast<long long*>(base + b_devs + b_rem);
  b->d_units = reinterpret_cast<long long*>(base + b_devs + b_rem + b_items);
  b->d_member_ctas = reinterpret_cast<int*>(base + b_devs + b_rem + b_items + b_units);
  if ((e = cudaMemsetAsync(b->d_block, 0, total, b->stream)) != cudaSuccess) return fail(cuda_fail(e, "memset"));
  if ((e = cudaMallocHost(&b->h_devs, sizeof(Dev) * n)) != cudaSuccess) return fail(cuda_fail(e, "host mirror"));
  memset(b->h_devs, 0, sizeof(Dev) * n);
  if ((e = cudaMallocHost(&b->h_set, sizeof(long long) * n)) != cudaSuccess) return fail(cuda_fail(e, "staging"));
  for (int k = 0; k < kSnapRing; ++k) {
    if ((e = cudaMallocHost(&b->h_snap[k], sizeof(long long) * n)) != cudaSuccess) return fail(cuda_fail(e, "snap"));
    memset(b->h_snap[k], 0, sizeof(long long) * n);
    if ((e = cudaEventCreateWithFlags(&b->ev_snap[k], cudaEventDisableTiming)) != cudaSuccess)
      return fail(cuda_fail(e, "event"));
  }
  if ((e = cudaEventCreateWithFlags(&b->ev_init, cudaEventDisableTiming)) != cudaSuccess)
    return fail(cuda_fail(e, "event"));
  if ((e = cudaStreamCreateWithFlags(&b->init_stream, cudaStreamNonBlocking)) != cudaSuccess)
    return fail(cuda_fail(e, "stream"));
  b->bd.devs = b->d_devs;
  b->bd.remaining = b->d_remaining;
  b->bd.item_start = b->d_item_start;
  b->bd.n = max_slots;
  b->bd.max_nx = max_nx;
  b->bd.prefetch = b->var.prefetch;
  b->bd.member_cost = b->var.member_cost;
  if (b->const_base >= 0) {
    // the constant-bank kernel: the per-member CTA counts the plan kernel
    // writes, cps waves of CTAs per step (CASCADE_BATCH_CTAS_PER_SM, a
    // measurement override), and a row long enough for the members' shares
    // (one member alone gets two rows' worth of SMs)
    if ((e = cudaMallocHost(&b->h_members, sizeof(BatchMember) * n)) != cudaSuccess)
      return fail(cuda_fail(e, "host member table"));
    memset(b->h_members, 0, sizeof(BatchMember) * n);
    const char* ev = getenv("CASCADE_BATCH_CTAS_PER_SM");
    int cps = (ev && *ev) ? atoi(ev) : kConstCtasPerSm;
    cps = cps < 1 ? 1 : (cps > 64 ? 64 : cps);
    b->bd.member_ctas = b->d_member_ctas;
    b->bd.const_base = b->const_base;
    b->bd.target_ctas = cps * b->num_sms;
    const int row = (2 * cps * b->num_sms + max_slots - 1) / max_slots;
    b->bd.max_ctas = row > 8 * cps ? row : 8 * cps;
  }
  if ((e = cudaStreamSynchronize(b->stream)) != cudaSuccess) return fail(cuda_fail(e, "sync"));
  *out = b;
  return CASCADE_OK;
}

int cascade_batch_admit(cascade_batch_t* b, const cascade_params* params, int32_t nsteps, int32_t* slot_out) {
  g_msg[0] = '\0';  // a message describes this call only
  if (!b || !params || nsteps < 0) return CASCADE_ERR_INVALID_ARG;
  cudaSetDevice(b->device);
  int rc = validate(params);
  if (rc) return rc;
  if (!same_kernel_class(params->precision, b->precision)) {
    snprintf(g_msg, sizeof(g_msg), "member precision %d differs from the batch's %d", params->precision,
             b->precision);
    return CASCADE_ERR_INVALID_ARG;
  }
  if (params->open_bc) {
    snprintf(g_msg, sizeof(g_msg), "batch members are periodic (open_bc = 0)");
    return CASCADE_ERR_INVALID_ARG;
  }
  if ((rc = batch_member_params(params))) return rc;
  if (params->nx > b->max_nx) {
    snprintf(g_msg, sizeof(g_msg), "member nx = %d exceeds the batch's max_nx = %d", params->nx, b->max_nx);
    return CASCADE_ERR_INVALID_ARG;
  }
  size_t need = 0;
  cascade_footprint(params, nullptr, &need);
  if (b->budget && b->used + need > b->budget) {
    snprintf(g_msg, sizeof(g_msg), "footprint %zu B over the remaining budget %zu B", need, b->budget - b->used);
    return CASCADE_ERR_BUSY;
  }
  int slot = -1;
  for (int i = 0; i < b->n_slots; ++i)
    if (!b->members[i]) {
      slot = i;
      break;
    }
  if (slot < 0) {
    snprintf(g_msg, sizeof(g_msg), "all %d slots are occupied", b->n_slots);
    return CASCADE_ERR_BUSY;
  }
  cascade_t* h = nullptr;
  rc = create_seeded(params, (void*)b->init_stream, true, &h);
  if (rc) return rc;
  b->members[slot] = h;
  b->used += h->bytes;
  b->seed_particles += 2LL * params->nx * params->ppc;
  b->reported[slot] = 0;
  b->admit_seq[slot] = b->run_seq;
  // publish the member: its initialisation (on the private stream) happens
  // before the table update and every later step on the batch stream
  CUDA_TRY(cudaEventRecord(b->ev_init, b->init_stream));
  CUDA_TRY(cudaStreamWaitEvent(b->stream, b->ev_init, 0));
  b->h_devs[slot] = h->d;
  b->h_set[slot] = nsteps;
  CUDA_TRY(cudaMemcpyAsync(b->d_devs + slot, b->h_devs + slot, sizeof(Dev), cudaMemcpyHostToDevice, b->stream));
  if (b->const_base >= 0) {
    // the slot's entry of the constant-bank member table, behind the steps
    // queued before it (none of them reads this slot: it was free)
    b->h_members[slot] = member_of(h->d);
    CUDA_TRY(batch_member_set_fp32(b->const_base + slot, b->h_members + slot, b->stream));
  }
  CUDA_TRY(cudaMemcpyAsync(b->d_remaining + slot, b->h_set + slot, sizeof(long long), cudaMemcpyHostToDevice,
                           b->stream));
  if (slot_out) *slot_out = slot;
  return CASCADE_OK;
}

int cascade_batch_create(const cascade_params* params, int32_t n, size_t hbm_budget, void* cuda_stream,
                         cascade_batch_t** out) {
  g_msg[0] = '\0';  // a message describes this call only
  if (!params || n < 1 || !out) {
    snprintf(g_msg, sizeof(g_msg), "batch: params, n >= 1 and out are required");
    return CASCADE_ERR_INVALID_ARG;
  }
  // every member is checked on the host before any device work
  int max_nx = 2;
  for (int i = 0; i < n; ++i) {
    const int rc = validate(&params[i]);
    if (rc) {
      char why[sizeof(g_msg)];
      snprintf(why, sizeof(why), "%s", g_msg);
      snprintf(g_msg, sizeof(g_msg), "member %d: %s", i, why);
      return rc;
    }
    if (!same_kernel_class(params[i].precision, params[0].precision)) {
      snprintf(g_msg, sizeof(g_msg), "member %d: precision %d differs from member 0's %d", i, params[i].precision,
               params[0].precision);
      return CASCADE_ERR_INVALID_ARG;
    }
    if (params[i].open_bc) {
      snprintf(g_msg, sizeof(g_msg), "member %d: batch members are periodic (open_bc = 0)", i);
      return CASCADE_ERR_INVALID_ARG;
    }
    if (batch_member_params(&params[i])) {
      char why[sizeof(g_msg)];
      snprintf(why, sizeof(why), "%s", g_msg);
      snprintf(g_msg, sizeof(g_msg), "member %d: %s", i, why);
      return CASCADE_ERR_INVALID_ARG;
    }
    if (params[i].nx > max_nx) max_nx = params[i].nx;
  }
  cascade_batch_t* b = nullptr;
  int rc = cascade_batch_create_slots(n, params[0].precision, max_nx, hbm_budget, cuda_stream, &b);
  if (rc) return rc;
  for (int i = 0; i < n; ++i) {
    int slot = -1;
    rc = cascade_batch_admit(b, &params[i], 0, &slot);
    if (rc) {
      cascade_batch_destroy(b);
      return rc;
    }
  }
  *out = b;
  return CASCADE_OK;
}

int cascade_batch_step(cascade_batch_t* b, const int32_t* nsteps_each) {
  g_msg[0] = '\0';  // a message describes this call only
  if (!b || !nsteps_each) return CASCADE_ERR_INVALID_ARG;
  cudaSetDevice(b->device);
  // current remaining counts, then add the new targets
  CUDA_TRY(cudaStreamSynchronize(b->stream));
  CUDA_TRY(cudaMemcpy(b->h_set, b->d_remaining, sizeof(long long) * b->n_slots, cudaMemcpyDeviceToHost));
  long long most = 0;
  for (int i = 0; i < b->n_slots; ++i) {
    if (!b->members[i]) continue;
    if (nsteps_each[i] < 0) return CASCADE_ERR_INVALID_ARG;
    b->h_set[i] += nsteps_each[i];
    if (b->h_set[i] > most) most = b->h_set[i];
    if (nsteps_each[i] > 0) {
      b->reported[i] = 0;
      b->admit_seq[i] = b->run_seq;
    }
  }
  CUDA_TRY(cudaMemcpyAsync(b->d_remaining, b->h_set, sizeof(long long) * b->n_slots, cudaMemcpyHostToDevice,
                           b->stream));
  if (b->tune_auto && most > 0) {
    int rc = batch_tune_with_warmup(b, &most, (most / 4 < b->tune_warmup) ? most / 4 : b->tune_warmup);
    if (rc) return rc;
  }
  while (most > 0) {
    const int k = most > (1 << 30) ? (1 << 30) : (int)most;
    int rc = batch_enqueue(b, k);
    if (rc) return rc;
    most -= k;
  }
  return CASCADE_OK;
}

int cascade_batch_run(cascade_batch_t* b, int32_t nsteps) {
  g_msg[0] = '\0';  // a message describes this call only
  if (!b || nsteps < 0) return CASCADE_ERR_INVALID_ARG;
  cudaSetDevice(b->device);
  if (b->tune_auto && nsteps > 0) {
    long long left = nsteps;
    const int rc = batch_tune_with_warmup(b, &left, b->tune_warmup);
    if (rc) return rc;
    nsteps = (int32_t)left;
  }
  return batch_enqueue(b, nsteps);
}

int cascade_batch_set_variant(cascade_batch_t* b, const cascade_batch_variant* v) {
  g_msg[0] = '\0';  // a message describes this call only
  if (!b || !v) return CASCADE_ERR_INVALID_ARG;
  cudaSetDevice(b->device);
  const int rc = batch_apply_variant(b, *v, CASCADE_VARIANT_FORCED, 0.0);
  if (rc == CASCADE_ERR_INVALID_ARG) {
    snprintf(g_msg, sizeof(g_msg), "variant (shape %d, stage %d, prefetch %d, member cost %d) does not fit this batch",
             v->shape, v->stage, v->prefetch, v->member_cost);
    batch_config_variant(b, b->var);
    return rc;
  }
  if (rc == CASCADE_OK) b->tune_auto = false;
  return rc;
}

int cascade_batch_get_variant(cascade_batch_t* b, cascade_batch_variant* v, int32_t* source, double* ns_per_unit) {
  g_msg[0] = '\0';  // a message describes this call only
  if (!b) return CASCADE_ERR_INVALID_ARG;
  if (v) *v = b->var;
  if (source) *source = b->var_source;
  if (ns_per_unit) *ns_per_unit = b->var_ns_per_unit;
  return CASCADE_OK;
}

int cascade_batch_tune_next(cascade_batch_t* b, int32_t rounds, int32_t use_cache) {
  g_msg[0] = '\0';  // a message describes this call only
  if (!b || rounds < 0) return CASCADE_ERR_INVALID_ARG;
  b->tune_auto = rounds > 0;
  if (rounds > 0) b->tune_rounds = rounds;
  b->tune_use_cache = use_cache != 0;
  b->tuned_key.clear();
  b->tune_countdown = -1;
  return CASCADE_OK;
}

int cascade_batch_tune_warmup(cascade_batch_t* b, int64_t steps) {
  g_msg[0] = '\0';  // a message describes this call only
  if (!b || steps < 0) return CASCADE_ERR_INVALID_ARG;
  b->tune_warmup = steps;
  return CASCADE_OK;
}

int cascade_batch_tuning_report(cascade_batch_t* b, cascade_batch_variant* cands, double* ns_per_unit, int32_t max,
                                int32_t* n_out) {
  g_msg[0] = '\0';  // a message describes this call only
  if (!b || max < 0 || (max > 0 && (!cands || !ns_per_unit))) return CASCADE_ERR_INVALID_ARG;
  const int n = (int)b->tune_cands.size() < max ? (int)b->tune_cands.size() : max;
  for (int i = 0; i < n; ++i) {
    cands[i] = b->tune_cands[i];
    ns_per_unit[i] = b->tune_ns[i];
  }
  if (n_out) *n_out = n;
  return CASCADE_OK;
}

int cascade_batch_poll(cascade_batch_t* b, int32_t* done_slots, int32_t max, int32_t* n_out, int32_t wait) {
  g_msg[0] = '\0';  // a message describes this call only
  if (!b || max < 0 || (max > 0 && !done_slots)) return CASCADE_ERR_INVALID_ARG;
  cudaSetDevice(b->device);
  if (wait) {
    // all queued work, then a fresh snapshot
    const int rc = batch_enqueue(b, 0);
    if (rc) return rc;
    const int k = (b->snap_next + kSnapRing - 1) % kSnapRing;
    CUDA_TRY(cudaEventSynchronize(b->ev_snap[k]));
    batch_harvest(b, k);
  } else {
    for (int k = 0; k < kSnapRing; ++k) {
      if (b->snap_seq[k] == 0) continue;
      const cudaError_t q = cudaEventQuery(b->ev_snap[k]);
      if (q == cudaErrorNotReady) continue;
      if (q != cudaSuccess) return cuda_fail(q, "cudaEventQuery");
      batch_harvest(b, k);
    }
  }
  int n = 0;
  if (b->landed_seq > 0) {
    const long long seq = b->landed_seq;
    for (int i = 0; i < b->n_slots && n < max; ++i) {
      if (!b->members[i] || b->reported[i]) continue;
      // only snapshots queued after the member's admission speak for it
      if (seq <= b->admit_seq[i]) continue;
      if (b->landed[i] == 0) {
        done_slots[n++] = i;
        b->reported[i] = 1;
      }
    }
  }
  if (n_out) *n_out = n;
  return CASCADE_OK;
}

// A member reported finished is skipped by every later batch kernel, so its
// state can be read, or its memory released, without waiting for the batch.
int batch_settle(cascade_batch_t* b, int slot) {
  if (b->reported[slot]) return CASCADE_OK;
  CUDA_TRY(cudaStreamSynchronize(b->stream));
  return CASCADE_OK;
}

int cascade_batch_diag(cascade_batch_t* b, int32_t slot, cascade_diag_t* host_out, int32_t max, int32_t* n_out,
                       double* E_host, double* J_host) {
  g_msg[0] = '\0';  // a message describes this call only
  int rc = batch_member_check(b, slot);
  if (rc) return rc;
  cudaSetDevice(b->device);
  if ((rc = batch_settle(b, slot))) return rc;
  return cascade_diag(b->members[slot], host_out, max, n_out, E_host, J_host);
}

int cascade_batch_counts(cascade_batch_t* b, int32_t slot, int64_t* n_elec, int64_t* n_posi, int64_t* n_photon,
                         int64_t* step) {
  g_msg[0] = '\0';  // a message describes this call only
  int rc = batch_member_check(b, slot);
  if (rc) return rc;
  cudaSetDevice(b->device);
  if ((rc = batch_settle(b, slot))) return rc;
  return cascade_counts(b->members[slot], n_elec, n_posi, n_photon, step);
}

int cascade_batch_release(cascade_batch_t* b, int32_t slot) {
  g_msg[0] = '\0';  // a message describes this call only
  int rc = batch_member_check(b, slot);
  if (rc) return rc;
  cudaSetDevice(b->device);
  if (!b->reported[slot]) {
    // still running: stop it behind the queued work, then wait for that work
    b->h_set[slot] = 0;
    CUDA_TRY(cudaMemcpyAsync(b->d_remaining + slot, b->h_set + slot, sizeof(long long), cudaMemcpyHostToDevice,
                             b->stream));
    CUDA_TRY(cudaStreamSynchronize(b->stream));
  }
  cascade_t* h = b->members[slot];
  b->used -= h->bytes;
  b->seed_particles -= 2LL * h->p.nx * h->p.ppc;
  b->members[slot] = nullptr;
  b->reported[slot] = 0;
  return cascade_destroy(h);
}

int cascade_batch_info(cascade_batch_t* b, int32_t* slots, int32_t* occupied, size_t* bytes_in_use) {
  g_msg[0] = '\0';  // a message describes this call only
  if (!b) return CASCADE_ERR_INVALID_ARG;
  int occ = 0;
  for (cascade_t* h : b->members) occ += h != nullptr;
  if (slots) *slots = b->n_slots;
  if (occupied) *occupied = occ;
  if (bytes_in_use) *bytes_in_use = b->used;
  return CASCADE_OK;
}

int cascade_batch_set_timing(cascade_batch_t* b, int32_t enable) {
  g_msg[0] = '\0';  // a message describes this call only
  if (!b) return CASCADE_ERR_INVALID_ARG;
  b->timing = enable != 0;
  return CASCADE_OK;
}

int cascade_batch_timing(cascade_batch_t* b, double* particle_kernel_ms, int64_t* particle_kernel_launches,
                         int64_t* kernels_launched) {
  g_msg[0] = '\0';  // a message describes this call only
  if (!b) return CASCADE_ERR_INVALID_ARG;
  cudaSetDevice(b->device);
  CUDA_TRY(cudaStreamSynchronize(b->stream));
  double total = 0.0;
  for (size_t i = 0; i + 1 < b->ev_used; i += 2) {
    float ms = 0.f;
    CUDA_TRY(cudaEventElapsedTime(&ms, b->ev_pool[i], b->ev_pool[i + 1]));
    total += ms;
  }
  if (particle_kernel_ms) *particle_kernel_ms = total;
  if (particle_kernel_launches) *particle_kernel_launches = (int64_t)(b->ev_used / 2);
  if (kernels_launched) *kernels_launched = b->kernels_launched;
  b->ev_used = 0;
  b->kernels_launched = 0;
  return CASCADE_OK;
}

int cascade_batch_destroy(cascade_batch_t* b) {
  if (!b) return CASCADE_OK;
  cudaSetDevice(b->device);
  if (b->stream || b->d_block) cudaStreamSynchronize(b->stream);
  if (b->init_stream) cudaStreamSynchronize(b->init_stream);
  for (cascade_t* h : b->members)
    if (h) cascade_destroy(h);
  if (b->graph) cudaGraphExecDestroy(b->graph);
  if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
  if (b->init_stream) cudaStreamDestroy(b->init_stream);
  for (int k = 0; k < kSnapRing; ++k) {
    if (b->ev_snap[k]) cudaEventDestroy(b->ev_snap[k]);
    if (b->h_snap[k]) cudaFreeHost(b->h_snap[k]);
  }
  if (b->ev_init) cudaEventDestroy(b->ev_init);
  for (cudaEvent_t e : b->ev_pool) cudaEventDestroy(e);
  const_slice_free(b->precision, b->const_base, b->n_slots);
  if (b->h_members) cudaFreeHost(b->h_members);
  if (b->h_devs) cudaFreeHost(b->h_devs);
  if (b->h_set) cudaFreeHost(b->h_set);
  if (b->d_block) cudaFree(b->d_block);
  delete b;
  return CASCADE_OK;
}

}  // extern "C"
