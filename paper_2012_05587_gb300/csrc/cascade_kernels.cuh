// Device kernels of one pair-cascade PIC step (arXiv:2012.05587, Sections 2-3),
// templated on the particle precision.  Included by kernels_fp64.cu (built
// without FMA contraction, so its arithmetic rounds like the plain FP64
// definition) and kernels_fp32.cu (FP32 particles, FP64 grid reductions).
//
// Per step, on one stream:
//   k_convert  photons due this step -> e-/e+ pairs appended to both species
//   k_push     persistent grid over all leptons: gather E, push, move,
//              charge-conserving deposit into a per-CTA shared-memory copy of
//              the current, threshold emission with warp-aggregated photon
//              appends; per-CTA current partials and sum(gamma) to global
//   k_field    FP64 sum of the per-CTA partials in a fixed order, Ampere
//              update, field diagnostics; its last CTA advances the counters
//              and writes the per-step record
#pragma once

#include <type_traits>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>

#include "cascade_internal.h"

namespace cpic {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kFieldGroups = 8;  // row groups of the field kernel (kFieldBlock / 32)
constexpr int kBatchSmemSlots = 1024;  // batches up to this size keep the cost offsets in shared memory
// Upper bound on photons one lepton emits in one step (a step that needs more
// is far too coarse for the model; the count is clamped).
constexpr int kMaxPhotonsPerStep = 1 << 16;

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11): ten rounds of the 4x32
// S-box, multipliers 0xD2511F53 / 0xCD9E8D57, Weyl key steps 0x9E3779B9 /
// 0xBB67AE85.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t hi0 = __umulhi(0xD2511F53u, c[0]);
    const uint32_t lo0 = 0xD2511F53u * c[0];
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c[2]);
    const uint32_t lo1 = 0xCD9E8D57u * c[2];
    const uint32_t n0 = hi1 ^ c[1] ^ k0;
    const uint32_t n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
}

__device__ __forceinline__ void set_error(Ctl* ctl, int code) { atomicCAS(&ctl->err, 0, code); }

// Bulk prefetch of [ptr, ptr + bytes) into L2 (a hint; bytes a multiple of 16,
// ptr 16-byte aligned, the range inside an allocation).
__device__ __forceinline__ void prefetch_l2(const void* ptr, unsigned bytes) {
  if (bytes >= 16) asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(ptr), "r"(bytes) : "memory");
}

// Asynchronous copy of one 16-byte chunk into shared memory (both addresses
// 16-byte aligned); only the first `bytes` are read, the rest is zero-filled.
// The issuing thread waits for its own copies with cp.async.wait_group, a
// hardware wait that ends when the copies land (no spin loop).
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, unsigned bytes) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(sa), "l"(gmem), "r"(bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_prev() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

// ---------------------------------------------------------------------------
// Seed: quiet start, pair j in cell j mod nx at offset (j div nx + 1/2)/ppc,
// momenta u_spread * Box-Muller(Philox(counter = (j, 0), key = seed)).
// ---------------------------------------------------------------------------
template <class Real>
__global__ void k_seed(Dev d, long long npairs, int ppc, unsigned long long seed, double u_spread) {
  Real* off0 = static_cast<Real*>(d.off[0]);
  Real* off1 = static_cast<Real*>(d.off[1]);
  Real* u0 = static_cast<Real*>(d.u[0]);
  Real* u1 = static_cast<Real*>(d.u[1]);
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < npairs;
       j += (long long)gridDim.x * blockDim.x) {
    const int cell = (int)(j % d.nx);
    const long long k = j / d.nx;
    const double off = ((double)k + 0.5) / (double)ppc;
    uint32_t c[4] = {(uint32_t)j, (uint32_t)(j >> 32), 0u, 0u};
    philox4x32_10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
    const unsigned long long a = ((unsigned long long)c[0] << 32) | c[1];
    const unsigned long long b = ((unsigned long long)c[2] << 32) | c[3];
    const double r1 = ((double)(a >> 11) + 0.5) * (1.0 / 9007199254740992.0);
    const double r2 = ((double)(b >> 11) + 0.5) * (1.0 / 9007199254740992.0);
    const double rad = sqrt(-2.0 * log(r1));
    const double ang = 6.283185307179586 * r2;
    const double ze = rad * cos(ang);
    const double zp = rad * sin(ang);
    d.cell[0][j] = cell;
    d.cell[1][j] = cell;
    off0[j] = (Real)off;
    off1[j] = (Real)off;
    const double ue = u_spread * ze, up = u_spread * zp;
    u0[j] = (Real)ue;
    u1[j] = (Real)up;
    if (d.ulo[0]) {  // two-word momenta: the rounding residual
      d.ulo[0][j] = (float)(ue - (double)(Real)ue);
      d.ulo[1][j] = (float)(up - (double)(Real)up);
    }
  }
}

// ---------------------------------------------------------------------------
// Photon conversion (Section 2: equal split, gamma = eps/2 each, along the
// photon).  The FIFO holds photons in emission-step order; those emitted at
// step n - 1 - n_pp end at emit_end[(n - 1 - n_pp) mod (n_pp + 1)].
// ---------------------------------------------------------------------------
template <class Real>
__global__ void k_convert(Dev d) {
  Ctl* ctl = d.ctl;
  const long long step = ctl->step;
  const long long src = step - 1 - d.n_pp;
  const long long head = ctl->ph_head;
  const long long end = (src >= 0) ? d.emit_end[src % (d.n_pp + 1)] : head;
  const long long n0 = ctl->n[0], n1 = ctl->n[1];
  long long cnt = end - head;
  const long long room = min(d.cap - n0, d.cap - n1);
  const bool over = cnt > room;
  if (over) cnt = room;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    ctl->conv_count = cnt;
    ctl->conv_end = end;  // photons beyond the capacity are dropped (error below)
    if (over) set_error(ctl, CASCADE_ERR_CAPACITY);
    const long long N = n0 + n1 + 2 * cnt;
    long long g = (N + d.min_per_cta - 1) / d.min_per_cta;
    if (g < 1) g = 1;
    if (g > d.grid_push) g = d.grid_push;
    ctl->active_blocks = (int)g;
  }
  const Real up = (Real)d.u_pair;
  const Real* ph_off = static_cast<const Real*>(d.ph_off);
  Real* off0 = static_cast<Real*>(d.off[0]);
  Real* off1 = static_cast<Real*>(d.off[1]);
  Real* u0 = static_cast<Real*>(d.u[0]);
  Real* u1 = static_cast<Real*>(d.u[1]);
  const long long mask = d.ph_cap - 1;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < cnt;
       i += (long long)gridDim.x * blockDim.x) {
    const long long slot = (head + i) & mask;
    const int enc = d.ph_cell[slot];
    const int cell = enc & 0x7fffffff;
    const Real oc = ph_off[slot];
    const Real uv = (enc < 0) ? -up : up;
    d.cell[0][n0 + i] = cell;
    off0[n0 + i] = oc;
    u0[n0 + i] = uv;
    d.cell[1][n1 + i] = cell;
    off1[n1 + i] = oc;
    u1[n1 + i] = uv;
    if (d.ulo[0]) {  // two-word momenta: the rounding residual of u_pair
      const float lo = (float)(d.u_pair - (double)up);
      d.ulo[0][n0 + i] = (enc < 0) ? -lo : lo;
      d.ulo[1][n1 + i] = (enc < 0) ? -lo : lo;
    }
  }
}

// ---------------------------------------------------------------------------
// Vector loads of four consecutive particles.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void ld4(const int* p, int v[4]) {
  const int4 t = *reinterpret_cast<const int4*>(p);
  v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
}
__device__ __forceinline__ void st4(int* p, const int v[4]) {
  *reinterpret_cast<int4*>(p) = make_int4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void ld4(const float* p, float v[4]) {
  const float4 t = *reinterpret_cast<const float4*>(p);
  v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
}
__device__ __forceinline__ void st4(float* p, const float v[4]) {
  *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void ld4(const double* p, double v[4]) {
  const double2 a = reinterpret_cast<const double2*>(p)[0];
  const double2 b = reinterpret_cast<const double2*>(p)[1];
  v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}
__device__ __forceinline__ void st4(double* p, const double v[4]) {
  reinterpret_cast<double2*>(p)[0] = make_double2(v[0], v[1]);
  reinterpret_cast<double2*>(p)[1] = make_double2(v[2], v[3]);
}

// ---------------------------------------------------------------------------
// gamma and velocity.  Exact: gamma = sqrt(1 + u^2) and v = u / gamma rounded
// as written (the plain definition).  Fast (FP32 only): one reciprocal square
// root, r = 1/sqrt(1 + u^2), gamma = (1 + u^2) r, v = u r.
// ---------------------------------------------------------------------------
template <class Real, bool FAST>
struct Kin {
  __device__ static __forceinline__ void eval(Real u, Real dtdx, Real& g, Real& dd) {
    g = sqrt(Real(1) + u * u);
    dd = u / g * dtdx;
  }
};
template <>
struct Kin<float, true> {
  __device__ static __forceinline__ void eval(float u, float dtdx, float& g, float& dd) {
    const float a = 1.0f + u * u;
    const float r = rsqrtf(a);
    g = a * r;
    dd = (u * r) * dtdx;
  }
};

// Per-CTA current accumulator in shared memory, one entry per edge:
//   DEP 0  Real atomics (FP64 mode; shared-memory FP32 atomic adds measured
//          1.6x slower than integer ones on this part)
//   DEP 1  int32 fixed point at 2^-k.  Every contribution is below dt/dx in
//          magnitude and a CTA handles at most P particles in a launch, so k
//          = floor(log2(2^30 / (P dt/dx))) keeps every sum below 2^30: no
//          overflow is possible.  Rounding to nearest, unbiased, error at most
//          2^-(k+1) per contribution.
//   DEP 4  two int32 words: the DEP 1 word plus a second word holding the
//          rounding residual of the first at a finer scale; the residual is at
//          most half a coarse step, so that sum cannot overflow either.
//          Resolution about 2^-20, one more atomic per contribution.
template <class Real, int DEP>
struct AccOf {
  typedef Real type;
};
template <class Real>
struct AccOf<Real, 1> {
  typedef int type;
};
template <class Real>
struct AccOf<Real, 4> {
  typedef int type;
};

// ---------------------------------------------------------------------------
// The particle update, shared by the single-cascade and the batched kernels.
// PushState holds what one CTA set up for one cascade: the shared-memory E and
// current accumulator, the fixed-point scales, the photon-ring window.
// ---------------------------------------------------------------------------
template <class Real, int DEP>
struct PushState {
  typedef typename AccOf<Real, DEP>::type Acc;
  Ctl* ctl;
  Real* Es;
  Acc* Ss;
  int* Ls;
  float fx_scale, fx_inv, lo_scale, lo_inv;
  long long ph_tail, room, ph_mask;
};

// Fixed-point scales for a CTA that deposits at most pcount particles.  Every
// contribution is below dt/dx in magnitude, so each edge's sum stays below
// 2^30 at 2^k; the DEP 4 residual word sums pcount values of at most
// 2^-(k+1) at a finer scale 2^(k+1+m), again below 2^30.
template <class Real, int DEP>
__device__ __forceinline__ void set_scales(PushState<Real, DEP>& st, double pcount, double dtdx) {
  st.fx_scale = st.fx_inv = st.lo_scale = st.lo_inv = 1.0f;
  if (DEP == 1 || DEP == 4) {
    const double pc = pcount + 1.0;
    int k = (int)floor(log2(1073741824.0 / (pc * dtdx + 1.0)));
    k = k < 0 ? 0 : (k > 30 ? 30 : k);
    st.fx_scale = ldexpf(1.0f, k);
    st.fx_inv = ldexpf(1.0f, -k);
    if (DEP == 4) {
      int m = (int)floor(log2(1073741824.0 / pc));
      m = m < 0 ? 0 : m;
      int kl = k + 1 + m;
      kl = kl > 60 ? 60 : kl;
      st.lo_scale = ldexpf(1.0f, kl);
      st.lo_inv = ldexpf(1.0f, -kl);
    }
  }
}

// Advance four consecutive particles of species s starting at index base
// (cnt of them valid; the whole warp calls this together).  Returns the sum
// of their gamma after the step.
// OPEN: open boundaries (Section 7 runs): the gather clamps to the outermost
// edges, a particle crossing x = 0 or x = L deposits the part of its path
// inside and is marked departed (cell -1, index appended to the hole list),
// a photon whose conversion point lies outside is not kept.
// STG: the four particles were already copied into this thread's shared
// memory slots stg[0..2] (cell, offset, momentum; zero beyond cnt) by
// cp.async; otherwise they are loaded from global memory here.
// COMP (FP32 only): the momentum is a compensated pair of FP32 words, u + ulo
// with |ulo| at most half the spacing of u.  The push adds q dt E to the pair
// exactly up to the rounding of the low word (Knuth's TwoSum, written with
// round-to-nearest intrinsics so that no operation is contracted), so pushes
// far below the spacing of u still accumulate; the threshold test and the
// recoil of a lepton near or above gamma_thr use the pair's sum in FP64.
// DevT: the cascade's descriptor -- Dev (the single-cascade kernel's kernel
// parameter) or BatchMember (a batch member's entry in the constant bank).
template <class Real, int V, int DEP, bool FAST, bool OPEN, bool STG = false, bool COMP = false, class DevT = Dev>
__device__ __forceinline__ Real process4(const DevT& d, const PushState<Real, DEP>& st, int s, long long base,
                                         int cnt, int lane, const unsigned char* const* stg = nullptr) {
  static_assert(!COMP || (sizeof(Real) == 4 && !STG), "two-word momenta: FP32, direct loads");
  typedef typename AccOf<Real, DEP>::type Acc;
  const int nx = d.nx;
  const Real dt = (Real)d.dt, dtdx = (Real)d.dtdx;
  const Real thr = (Real)d.gamma_thr, eps = (Real)d.eps_gamma, lpf = (Real)d.lpp_frac;
  const Real one = Real(1), half = Real(0.5), zero = Real(0);
  int* cellp = d.cell[s] + base;
  Real* offp = static_cast<Real*>(d.off[s]) + base;
  Real* up = static_cast<Real*>(d.u[s]) + base;
  int cl[4] = {0, 0, 0, 0};
  Real of[4] = {zero, zero, zero, zero}, uu[4] = {zero, zero, zero, zero};
  float ul[4] = {0.f, 0.f, 0.f, 0.f};
  float* ulp = nullptr;
  if constexpr (COMP) {
    ulp = d.ulo[s] + base;
    if (cnt == 4) {
      ld4(ulp, ul);
    } else {
#pragma unroll
      for (int j = 0; j < 4; ++j)
        if (j < cnt) ul[j] = ulp[j];
    }
  }
  if (STG) {
    if (cnt > 0) {
      ld4(reinterpret_cast<const int*>(stg[0]), cl);
      ld4(reinterpret_cast<const Real*>(stg[1]), of);
      ld4(reinterpret_cast<const Real*>(stg[2]), uu);
    }
  } else if (cnt == 4) {
    ld4(cellp, cl);
    ld4(offp, of);
    ld4(up, uu);
  } else {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      if (j < cnt) {
        cl[j] = cellp[j];
        of[j] = offp[j];
        uu[j] = up[j];
      }
    }
  }
  const Real q = s ? one : -one;
  const Real qdt = s ? dt : -dt;
  // live[j]: particle j exists and has not departed (a departed particle is
  // only still stored if the hole list overflowed; it stays inert)
  bool live[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    live[j] = j < cnt;
    if (OPEN && cl[j] < 0) {
      live[j] = false;
      cl[j] = 0;
    }
  }

  // gather: linear between the two edges bracketing each particle
  Real Ep[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int c = cl[j];
    const Real o = of[j];
    const bool hi = o >= half;
    const int ia = hi ? c : ((c == 0) ? (OPEN ? 0 : nx - 1) : c - 1);
    const int ib = hi ? ((c + 1 == nx) ? (OPEN ? nx - 1 : 0) : c + 1) : c;
    const Real w = hi ? o - half : o + half;
    Real Ea, Eb;
    if (V == kGlobEGlobS || V == kGlobESmemS) {
      Ea = (Real)__ldg(d.E + ia);
      Eb = (Real)__ldg(d.E + ib);
    } else {
      Ea = st.Es[ia];
      Eb = st.Es[ib];
    }
    Ep[j] = (one - w) * Ea + w * Eb;
  }

  // push (du/dt = q E), move (dx/dt = u / gamma, cell units) and the
  // charge-conserving current: q * (offset change) per edge crossed
  Real g[4], a1[4], a2[4];
  int e1[4], e2[4];
  bool departed[4] = {false, false, false, false};
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int c = cl[j];
    const Real o = of[j];
    Real u;
    if constexpr (COMP) {
      // (uu, ul) + du as a new pair: TwoSum of the high words, the error and
      // the low word added, then renormalised (Fast2Sum)
      const float du = __fmul_rn((float)qdt, (float)Ep[j]);
      const float sh = __fadd_rn((float)uu[j], du);
      const float bv = __fsub_rn(sh, (float)uu[j]);
      const float er = __fadd_rn(__fsub_rn((float)uu[j], __fsub_rn(sh, bv)), __fsub_rn(du, bv));
      const float lo = __fadd_rn(ul[j], er);
      const float hi = __fadd_rn(sh, lo);
      ul[j] = __fsub_rn(lo, __fsub_rn(hi, sh));
      u = (Real)hi;
    } else {
      u = uu[j] + qdt * Ep[j];
    }
    Real gj, dd;
    Kin<Real, FAST>::eval(u, dtdx, gj, dd);
    Real o2 = o + dd;
    int c2 = c;
    Real b1, b2 = zero;
    int f2 = -1;
    bool gone = false;
    if (o2 >= one) {
      b1 = q * (one - o);
      if (OPEN && c + 1 == nx) {
        gone = true;  // left through x = L: the part inside is deposited
      } else {
        c2 = (c + 1 == nx) ? 0 : c + 1;
        o2 = o2 - one;
        f2 = c2;
        b2 = q * o2;
      }
    } else if (o2 < zero) {
      b1 = q * (zero - o);
      if (OPEN && c == 0) {
        gone = true;  // left through x = 0
      } else {
        c2 = (c == 0) ? nx - 1 : c - 1;
        o2 = o2 + one;
        f2 = c2;
        b2 = q * (o2 - one);
        if (o2 >= one) {
          o2 = zero;
          c2 = c;
        }
      }
    } else {
      b1 = q * (o2 - o);
    }
    const bool valid = live[j];
    e1[j] = valid ? c : -1;
    e2[j] = valid ? f2 : -1;
    a1[j] = b1;
    a2[j] = b2;
    if (OPEN && valid && gone) {
      departed[j] = true;
      live[j] = false;
      c2 = -1;
    }
    g[j] = live[j] ? gj : one;
    cl[j] = c2;
    of[j] = o2;
    uu[j] = u;
  }

  // deposit
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    if (V == kSmemESmemS || V == kGlobESmemS) {
      if (DEP == 1) {
        if (e1[j] >= 0) atomicAdd(&st.Ss[e1[j]], __float2int_rn((float)a1[j] * st.fx_scale));
        if (e2[j] >= 0) atomicAdd(&st.Ss[e2[j]], __float2int_rn((float)a2[j] * st.fx_scale));
      } else if (DEP == 4) {
        if (e1[j] >= 0) {
          const float a = (float)a1[j];
          const int qh = __float2int_rn(a * st.fx_scale);
          const int ql = __float2int_rn((a - (float)qh * st.fx_inv) * st.lo_scale);  // residual is exact
          atomicAdd(&st.Ss[e1[j]], qh);
          if (ql != 0) atomicAdd(&st.Ls[e1[j]], ql);
        }
        if (e2[j] >= 0) {
          const float a = (float)a2[j];
          const int qh = __float2int_rn(a * st.fx_scale);
          const int ql = __float2int_rn((a - (float)qh * st.fx_inv) * st.lo_scale);
          atomicAdd(&st.Ss[e2[j]], qh);
          if (ql != 0) atomicAdd(&st.Ls[e2[j]], ql);
        }
      } else {
        if (e1[j] >= 0) atomicAdd(&st.Ss[e1[j]], (Acc)a1[j]);
        if (e2[j] >= 0) atomicAdd(&st.Ss[e2[j]], (Acc)a2[j]);
      }
    } else {
      if (e1[j] >= 0) atomicAdd(&d.S_glob[e1[j]], (double)a1[j]);
      if (e2[j] >= 0) atomicAdd(&d.S_glob[e2[j]], (double)a2[j]);
    }
  }

  // QED (Section 2): threshold emission with recoil; photons appended with
  // one warp-wide scan and one global atomic per slot that has emitters
  if constexpr (OPEN) {
    // departed particles: their indices join their species' hole list (a
    // warp can hold both species, so one warp-wide scan and one atomic per
    // species present)
    const int nd = (int)departed[0] + (int)departed[1] + (int)departed[2] + (int)departed[3];
    if (__any_sync(kFull, nd > 0)) {
#pragma unroll
      for (int sp = 0; sp < 2; ++sp) {
        const int mine = (s == sp) ? nd : 0;
        int incl = mine;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int v = __shfl_up_sync(kFull, incl, o);
          if (lane >= o) incl += v;
        }
        const int tot = __shfl_sync(kFull, incl, 31);
        if (tot == 0) continue;
        unsigned long long b0 = 0;
        if (lane == 0) b0 = atomicAdd(&st.ctl->n_holes[sp], (unsigned long long)tot);
        b0 = __shfl_sync(kFull, b0, 0);
        if (mine == 0) continue;
        unsigned long long pos = b0 + incl - mine;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          if (departed[j]) {
            if ((long long)pos < d.hole_cap) d.holes[sp][pos] = base + j;
            else set_error(st.ctl, CASCADE_ERR_CAPACITY);
            ++pos;
          }
        }
      }
    }
  }

  // two-word momenta: the FP32 gamma only preselects (its rounding is far
  // below 2^-20 relative); the FP64 test below decides
  const Real thr_pre = COMP ? thr * Real(0.999999) : thr;
  const bool hot = (g[0] >= thr_pre) | (g[1] >= thr_pre) | (g[2] >= thr_pre) | (g[3] >= thr_pre) |
                   !(g[0] <= Real(1e30)) | !(g[1] <= Real(1e30)) | !(g[2] <= Real(1e30)) |
                   !(g[3] <= Real(1e30));
  if (__any_sync(kFull, hot)) {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int k = 0;
      int enc = 0;
      Real oc = zero;
      Real u = uu[j], gj = g[j];
      bool emit;
      const bool fwd = u > zero;  // direction kept through the recoil
      if (!(gj <= Real(1e30))) {
        // non-finite or absurd gamma: the run has blown up; flag it, no emission
        set_error(st.ctl, CASCADE_ERR_NONFINITE);
        emit = false;
      } else if (COMP || (sizeof(Real) == 4 && gj > Real(1e6))) {
        // large gamma, or a two-word momentum: threshold test and recoil in
        // FP64 (of the pair's sum for a two-word momentum)
        const double ud = (double)u + (double)ul[j];
        const double gd = sqrt(1.0 + ud * ud);
        emit = gd >= d.gamma_thr;
        if (emit) {
          k = 1 + (int)fmin(floor((gd - d.gamma_thr) / d.eps_gamma), (double)kMaxPhotonsPerStep);
          const double g2 = gd - (double)k * d.eps_gamma;
          const double un = (fwd ? 1.0 : -1.0) * sqrt(g2 * g2 - 1.0);
          u = (Real)un;
          if (COMP) ul[j] = (float)(un - (double)u);
          gj = (Real)g2;
        }
      } else {
        emit = gj >= thr;
        if (emit) {
          k = 1 + (int)fmin(floor((gj - thr) / eps), (Real)kMaxPhotonsPerStep);
          const Real g2 = gj - (Real)k * eps;
          const Real sg = fwd ? one : -one;
          u = sg * sqrt(g2 * g2 - one);
          gj = g2;
        }
      }
      if (emit) {
        // conversion point x + dir * l_pp, wrapped
        const Real o2 = of[j];
        const int c2 = cl[j];
        long long ci;
        if (fwd) {
          oc = o2 + lpf;
          ci = (long long)c2 + d.lpp_int;
          if (oc >= one) {
            oc = oc - one;
            ci += 1;
          }
        } else {
          oc = o2 - lpf;
          ci = (long long)c2 - d.lpp_int;
          if (oc < zero) {
            oc = oc + one;
            ci -= 1;
            if (oc >= one) {
              oc = zero;
              ci += 1;
            }
          }
        }
        long long m = ci % nx;
        if (m < 0) m += nx;
        enc = (int)m | (fwd ? 0 : (int)0x80000000);
        if (k > 1) atomicAdd(reinterpret_cast<unsigned long long*>(&st.ctl->emit_multi), 1ull);
        uu[j] = u;
        g[j] = gj;
        if (OPEN && (ci < 0 || ci >= nx)) k = 0;  // converts outside the domain: not kept
      }
      const unsigned em = __ballot_sync(kFull, k > 0);
      if (em) {
        const unsigned long long kk = (unsigned long long)k;
        unsigned long long incl = kk;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const unsigned long long v = __shfl_up_sync(kFull, incl, o);
          if (lane >= o) incl += v;
        }
        const unsigned long long tot = __shfl_sync(kFull, incl, 31);
        unsigned long long b0 = 0;
        if (lane == 0) b0 = atomicAdd(&st.ctl->emit_count, tot);
        b0 = __shfl_sync(kFull, b0, 0);
        const unsigned long long first = b0 + incl - kk;
        for (int m = 0; m < k; ++m) {
          const unsigned long long pos = first + m;
          if ((long long)pos < st.room) {
            const long long slot = (st.ph_tail + (long long)pos) & st.ph_mask;
            d.ph_cell[slot] = enc;
            static_cast<Real*>(d.ph_off)[slot] = oc;
          } else {
            set_error(st.ctl, CASCADE_ERR_PHOTON_CAPACITY);
          }
        }
      }
    }
  }

  if (OPEN) {
#pragma unroll
    for (int j = 0; j < 4; ++j)
      if (!live[j]) cl[j] = -1;  // departed now or before
  }
  if (cnt == 4) {
    st4(cellp, cl);
    st4(offp, of);
    st4(up, uu);
    if (COMP) st4(ulp, ul);
  } else {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      if (j < cnt) {
        cellp[j] = cl[j];
        offp[j] = of[j];
        up[j] = uu[j];
        if (COMP) ulp[j] = ul[j];
      }
    }
  }
  Real gs = zero;
#pragma unroll
  for (int j = 0; j < 4; ++j) gs += live[j] ? g[j] : zero;
  return gs;
}

// ---------------------------------------------------------------------------
// The particle kernel of one cascade.  V: where E and the current accumulator
// live (see PushVariant).  Persistent grid; the number of working CTAs
// follows the particle count.
// ---------------------------------------------------------------------------
// FP32: 1024 threads (64 registers); FP64 needs more registers per particle,
// so 512 threads with up to 128 registers and no spills.
template <class Real>
struct PushBlock {
  static constexpr int value = sizeof(Real) == 8 ? 512 : 1024;
};

// Shared memory of the particle kernel for E and the current accumulator:
// E (Real) plus one Real or int32 word per edge, two int32 words for DEP 4.
template <class Real>
__host__ __device__ inline size_t smem_field_bytes(int nx, int variant, int dep) {
  const size_t eb = ((size_t)nx * sizeof(Real) + 15) & ~size_t(15);
  if (variant == kSmemESmemS) return (dep == 4 ? 3 : 2) * eb;
  if (variant == kSmemEGlobS || variant == kGlobESmemS) return eb;
  return 0;
}

// Bytes of the cp.async staging area of the particle kernel: two stages of
// three 16-byte slots (cell, offset, momentum of four particles) per thread.
constexpr size_t kStageBytesPerThread = 2 * 3 * 16;

// STG (FP32 only): the particles of the next iteration are copied into
// shared memory with cp.async while the current ones are processed, so each
// thread keeps one iteration of loads in flight at all times.
// COMP: two-word momenta (see process4); direct loads.
template <class Real, int V, int DEP, bool FAST, bool OPEN, bool STG = false, bool COMP = false>
__global__ void __launch_bounds__(PushBlock<Real>::value, 1) k_push(Dev d) {
  static_assert(!STG || sizeof(Real) == 4, "the staging slots hold four 4-byte values");
  typedef typename AccOf<Real, DEP>::type Acc;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[32];
  Ctl* ctl = d.ctl;
  const int G = ctl->active_blocks;
  if ((int)blockIdx.x >= G) return;

  const int nx = d.nx;
  const size_t eb = ((size_t)nx * sizeof(Real) + 15) & ~size_t(15);
  PushState<Real, DEP> st;
  st.ctl = ctl;
  st.Es = reinterpret_cast<Real*>(smem_raw);
  st.Ss = reinterpret_cast<Acc*>(smem_raw + (V == kGlobESmemS ? 0 : eb));
  st.Ls = reinterpret_cast<int*>(smem_raw + 2 * eb);  // DEP 4 residual word
  if (V == kSmemESmemS || V == kSmemEGlobS) {
    for (int i = threadIdx.x; i < nx; i += blockDim.x) st.Es[i] = (Real)d.E[i];
  }
  if (V == kSmemESmemS || V == kGlobESmemS) {
    for (int i = threadIdx.x; i < nx; i += blockDim.x) {
      st.Ss[i] = Acc(0);
      if (DEP == 4) st.Ls[i] = 0;
    }
  }
  __syncthreads();

  const long long cc = ctl->conv_count;
  const long long N0 = ctl->n[0] + cc, N1 = ctl->n[1] + cc;
  const long long C0 = (N0 + 3) >> 2, C1 = (N1 + 3) >> 2, C = C0 + C1;
  st.ph_tail = ctl->ph_tail;
  st.room = d.ph_cap - (st.ph_tail - ctl->conv_end);
  st.ph_mask = d.ph_cap - 1;
  const long long stride = (long long)G * blockDim.x;
  const long long first_wb = (long long)blockIdx.x * blockDim.x;
  const long long iters_cta = (C > first_wb) ? (C - first_wb + stride - 1) / stride : 0;
  // every CTA takes the scale of the busiest one (CTA 0), so the int32 rows
  // of DEP 1 share one scale and the field kernel sums them exactly
  const long long iters_max = (C + stride - 1) / stride;
  set_scales<Real, DEP>(st, (double)(iters_max * blockDim.x * 4), d.dtdx);
  if (DEP == 1 && blockIdx.x == 0 && threadIdx.x == 0) ctl->part_inv = st.fx_inv;

  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  // this thread's staging slots: [stage][array][thread][16 B]
  unsigned char* stage = smem_raw + smem_field_bytes<Real>(nx, V, DEP);
  const size_t slab = (size_t)blockDim.x * 16;
  auto slot = [&](int b, int a) { return stage + (size_t)(b * 3 + a) * slab + (size_t)threadIdx.x * 16; };
  auto issue = [&](long long it) {  // cp.async of iteration it's chunk into stage it & 1
    const long long ch = first_wb + it * stride + warp * 32 + lane;
    if (it < iters_cta && ch < C) {
      const int sp = ch < C0 ? 0 : 1;
      const long long bp = (ch - (sp ? C0 : 0)) * 4;
      const unsigned bytes = (unsigned)min(4LL, (sp ? N1 : N0) - bp) * 4u;
      const int b = (int)(it & 1);
      cp_async16(slot(b, 0), d.cell[sp] + bp, bytes);
      cp_async16(slot(b, 1), static_cast<const Real*>(d.off[sp]) + bp, bytes);
      cp_async16(slot(b, 2), static_cast<const Real*>(d.u[sp]) + bp, bytes);
    }
    cp_async_commit();  // one group per iteration, empty or not
  };
  if (STG) issue(0);
  double gsum_total = 0.0;
  const int pf = d.prefetch;  // iterations ahead that lane 0 prefetches its warp's particles
  for (long long it = 0; it < iters_cta; ++it) {
    if (pf > 0 && lane == 0) {
      const long long chp = first_wb + (it + pf) * stride + warp * 32;  // the warp's first chunk then
      if (chp < C) {
        const int sp = chp < C0 ? 0 : 1;
        const long long bp = (chp - (sp ? C0 : 0)) * 4;
        long long np = d.cap4 - bp;  // stay inside the allocation
        if (np > 128) np = 128;
        if (np > 0) {
          prefetch_l2(d.cell[sp] + bp, (unsigned)(np * 4) & ~15u);
          prefetch_l2(static_cast<const Real*>(d.off[sp]) + bp, (unsigned)(np * sizeof(Real)) & ~15u);
          prefetch_l2(static_cast<const Real*>(d.u[sp]) + bp, (unsigned)(np * sizeof(Real)) & ~15u);
          if (COMP) prefetch_l2(d.ulo[sp] + bp, (unsigned)(np * 4) & ~15u);
        }
      }
    }
    const long long ch = first_wb + it * stride + warp * 32 + lane;
    int s = 0, cnt = 0;
    long long base = 0;
    if (ch < C) {
      s = ch < C0 ? 0 : 1;
      base = (ch - (s ? C0 : 0)) * 4;
      const long long N = s ? N1 : N0;
      cnt = (int)min(4LL, N - base);
    }
    if (STG) {
      issue(it + 1);
      cp_async_wait_prev();  // iteration it's copies have landed
      const int b = (int)(it & 1);
      const unsigned char* stg[3] = {slot(b, 0), slot(b, 1), slot(b, 2)};
      gsum_total += (double)process4<Real, V, DEP, FAST, OPEN, true>(d, st, s, base, cnt, lane, stg);
    } else {
      gsum_total += (double)process4<Real, V, DEP, FAST, OPEN, false, COMP>(d, st, s, base, cnt, lane);
    }
  }

  // sum of gamma over the CTA (FP64)
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) gsum_total += __shfl_down_sync(kFull, gsum_total, o);
  if (lane == 0) red[warp] = gsum_total;
  __syncthreads();
  if (warp == 0) {
    double v = (lane < (int)(blockDim.x >> 5)) ? red[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(kFull, v, o);
    if (lane == 0) d.uk_part[blockIdx.x] = v;
  }
  if (V == kSmemESmemS || V == kGlobESmemS) {
    if (DEP == 1) {
      // the raw int32 sums at the common scale ctl->part_inv
      int* P = static_cast<int*>(d.S_part) + (size_t)blockIdx.x * d.nxp;
      for (int i = threadIdx.x; i < nx; i += blockDim.x) P[i] = (int)st.Ss[i];
    } else {
      Real* P = static_cast<Real*>(d.S_part) + (size_t)blockIdx.x * d.nxp;
      for (int i = threadIdx.x; i < nx; i += blockDim.x) {
        if (DEP == 4) P[i] = (Real)((double)st.Ss[i] * (double)st.fx_inv + (double)st.Ls[i] * (double)st.lo_inv);
        else P[i] = (Real)st.Ss[i];
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Ampere update and field diagnostics; the last CTA finishes the step.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void block_reduce4(double v[4], double* sh /* [4][32] */) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    v[0] += __shfl_down_sync(kFull, v[0], o);
    v[1] += __shfl_down_sync(kFull, v[1], o);
    v[2] = fmax(v[2], __shfl_down_sync(kFull, v[2], o));
    v[3] += __shfl_down_sync(kFull, v[3], o);
  }
  if (lane == 0) {
    sh[warp] = v[0];
    sh[32 + warp] = v[1];
    sh[64 + warp] = v[2];
    sh[96 + warp] = v[3];
  }
  __syncthreads();
  if (warp == 0) {
    const int nw = blockDim.x >> 5;
    v[0] = lane < nw ? sh[lane] : 0.0;
    v[1] = lane < nw ? sh[32 + lane] : 0.0;
    v[2] = lane < nw ? sh[64 + lane] : 0.0;
    v[3] = lane < nw ? sh[96 + lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      v[0] += __shfl_down_sync(kFull, v[0], o);
      v[1] += __shfl_down_sync(kFull, v[1], o);
      v[2] = fmax(v[2], __shfl_down_sync(kFull, v[2], o));
      v[3] += __shfl_down_sync(kFull, v[3], o);
    }
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// End of a step (one thread): pairs and photons of this step join the
// counters, the step advances, the per-step record is written.  r holds
// sum E, sum J, max |E|, U_E over the edges; gsum is the sum of gamma.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void finish_step(const Dev& d, const double r[4], double gsum) {
  Ctl* ctl = d.ctl;
  const long long cc = ctl->conv_count;
  ctl->n[0] += cc;
  ctl->n[1] += cc;
  if (d.open_bc) {
    // departed particles are gone (compaction filled their slots)
    for (int sp = 0; sp < 2; ++sp) {
      const long long h = (long long)ctl->n_holes[sp];
      ctl->n[sp] -= h < d.hole_cap ? h : d.hole_cap;
      ctl->n_holes[sp] = 0ull;
      ctl->na[sp] = 0ull;
      ctl->nb[sp] = 0ull;
    }
  }
  ctl->pairs_total += cc;
  ctl->ph_head = ctl->conv_end;
  unsigned long long em = ctl->emit_count;
  const long long room = d.ph_cap - (ctl->ph_tail - ctl->conv_end);
  if ((long long)em > room) em = (unsigned long long)room;
  ctl->ph_tail += (long long)em;
  d.emit_end[ctl->step % (d.n_pp + 1)] = ctl->ph_tail;
  ctl->emit_count = 0ull;
  ctl->conv_count = 0;
  ctl->step += 1;
  const long long st = ctl->step;
  cascade_diag_t rec;
  rec.step = st;
  rec.t = (double)st * d.dt;
  rec.E_mean = r[0] / d.nx;
  rec.J_mean = r[1] / d.nx;
  rec.E_absmax = r[2];
  rec.U_E = r[3];
  rec.U_K = d.w * gsum;
  const long long nph = ctl->ph_tail - ctl->ph_head;
  rec.U_gamma = (double)nph * d.w * d.eps_gamma;
  rec.gauss_resid = __longlong_as_double(0x7ff8000000000000LL);
  rec.n_elec = ctl->n[0];
  rec.n_posi = ctl->n[1];
  rec.n_photon = nph;
  rec.n_pairs_total = ctl->pairs_total;
  rec.n_emit_multi = ctl->emit_multi;
  d.ring[(st - 1) % d.ring_n] = rec;
  ctl->last = rec;
}

// Sums of four values over the 32 lanes of a warp (sum, sum, max, sum);
// lane 0 holds the result.
__device__ __forceinline__ void warp_reduce4(double v[4]) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    v[0] += __shfl_down_sync(kFull, v[0], o);
    v[1] += __shfl_down_sync(kFull, v[1], o);
    v[2] = fmax(v[2], __shfl_down_sync(kFull, v[2], o));
    v[3] += __shfl_down_sync(kFull, v[3], o);
  }
}

// Acc: element type of the per-CTA current rows (int: FP32 int32 sums at
// the common scale ctl->part_inv, added exactly in int64; float/double: FP64
// sums in a fixed row order).  kPartials: rows in S_part, else the FP64
// global current S_glob.  On this part the FP64 pipe issues one warp
// instruction per 16 cycles per SM, so the kernel keeps FP64 work off the
// row sums (int64) and reduces its diagnostics in one warp.
template <class Acc, bool kPartials>
__global__ void __launch_bounds__(kFieldBlock) k_field(Dev d) {
  // 32 edges per CTA; the 8 warps each sum every 8th per-CTA partial row of
  // those edges (coalesced), then warp 0 adds the 8 group sums in order
  __shared__ double grp[kFieldGroups][32];
  __shared__ long long grp_i[kFieldGroups][32];
  __shared__ int s_last;
  Ctl* ctl = d.ctl;
  const int lane = threadIdx.x & 31, g = threadIdx.x >> 5;
  const int i = blockIdx.x * 32 + lane;
  const int G = ctl->active_blocks;
  constexpr bool kInt = std::is_integral<Acc>::value;
  if (kPartials) {
    const Acc* P = static_cast<const Acc*>(d.S_part) + i;
    const size_t pitch = d.nxp;
    if (kInt) {
      long long S = 0;
      if (i < d.nx)
        for (int b = g; b < G; b += kFieldGroups) S += (long long)P[(size_t)b * pitch];
      grp_i[g][lane] = S;
    } else {
      double S = 0.0;
      if (i < d.nx) {
        // four independent loads in flight, added in row order
        int b = g;
        for (; b + 3 * kFieldGroups < G; b += 4 * kFieldGroups) {
          const double v0 = (double)P[(size_t)b * pitch];
          const double v1 = (double)P[(size_t)(b + kFieldGroups) * pitch];
          const double v2 = (double)P[(size_t)(b + 2 * kFieldGroups) * pitch];
          const double v3 = (double)P[(size_t)(b + 3 * kFieldGroups) * pitch];
          S += v0;
          S += v1;
          S += v2;
          S += v3;
        }
        for (; b < G; b += kFieldGroups) S += (double)P[(size_t)b * pitch];
      }
      grp[g][lane] = S;
    }
    __syncthreads();
  }
  if (g == 0) {
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    if (i < d.nx) {
      double S = 0.0;
      if (kPartials && kInt) {
        long long Si = 0;
#pragma unroll
        for (int k = 0; k < kFieldGroups; ++k) Si += grp_i[k][lane];
        S = (double)Si * (double)ctl->part_inv;
      } else if (kPartials) {
#pragma unroll
        for (int k = 0; k < kFieldGroups; ++k) S += grp[k][lane];
      } else {
        S = d.S_glob[i];
        d.S_glob[i] = 0.0;
      }
      const double J = d.jscale * S;
      const double E = d.E[i] - d.dt * (J - d.j_m);  // Eq. 26 (j_m = 0 outside the co-rotating frame)
      d.E[i] = E;
      d.J[i] = J;
      v[0] = E;
      v[1] = J;
      v[2] = fabs(E);
      v[3] = 0.5 * E * E * d.dx;
    }
    warp_reduce4(v);
    if (lane == 0) {
      double* dp = d.diag_part + 4 * blockIdx.x;
      dp[0] = v[0];
      dp[1] = v[1];
      dp[2] = v[2];
      dp[3] = v[3];
      __threadfence();
      const unsigned t = atomicAdd(&ctl->field_ticket, 1u);
      s_last = (t == gridDim.x - 1);
    }
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  // last CTA: each thread folds a fixed share of the per-CTA partials and of
  // the particle kernel's sums of gamma, each warp reduces its lanes, and
  // thread 0 adds the warps' results in warp order
  double r[4] = {0.0, 0.0, 0.0, 0.0};
  for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) {
    const double2 a = __ldcg(reinterpret_cast<const double2*>(d.diag_part + 4 * b));
    const double2 c = __ldcg(reinterpret_cast<const double2*>(d.diag_part + 4 * b + 2));
    r[0] += a.x;
    r[1] += a.y;
    r[2] = fmax(r[2], c.x);
    r[3] += c.y;
  }
  double gs = 0.0;
  for (int b = threadIdx.x; b < G; b += blockDim.x) gs += __ldcg(d.uk_part + b);
  warp_reduce4(r);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) gs += __shfl_down_sync(kFull, gs, o);
  if (lane == 0) {
    grp[0][g] = r[0];
    grp[1][g] = r[1];
    grp[2][g] = r[2];
    grp[3][g] = r[3];
    grp[4][g] = gs;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t[4] = {0.0, 0.0, 0.0, 0.0}, ts = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      t[0] += grp[0][w];
      t[1] += grp[1][w];
      t[2] = fmax(t[2], grp[2][w]);
      t[3] += grp[3][w];
      ts += grp[4][w];
    }
    ctl->field_ticket = 0u;
    finish_step(d, t, ts);
  }
}

// ---------------------------------------------------------------------------
// Open boundaries: fill the slots of departed particles.  With N particles
// processed and H departed, the new count is N - H; live particles at or
// above it move into the holes below it (there are as many of each), so the
// cost is O(H), not O(N).
// ---------------------------------------------------------------------------
template <class Real>
__global__ void k_compact_plan(Dev d) {
  Ctl* ctl = d.ctl;
  const long long cc = ctl->conv_count;
  for (int s = 0; s < 2; ++s) {
    const long long N = ctl->n[s] + cc;
    long long H = (long long)ctl->n_holes[s];
    H = H < d.hole_cap ? H : d.hole_cap;
    const long long N2 = N - H;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < H;
         t += (long long)gridDim.x * blockDim.x) {
      if (d.cell[s][N2 + t] >= 0) d.hole_b[s][atomicAdd(&ctl->nb[s], 1ull)] = N2 + t;
      const long long h = d.holes[s][t];
      if (h < N2) d.hole_a[s][atomicAdd(&ctl->na[s], 1ull)] = h;
    }
  }
}

template <class Real>
__global__ void k_compact_move(Dev d) {
  Ctl* ctl = d.ctl;
  for (int s = 0; s < 2; ++s) {
    const long long na = (long long)ctl->na[s];
    const long long nb = (long long)ctl->nb[s];
    const long long n = na < nb ? na : nb;  // equal unless the hole list overflowed
    Real* off = static_cast<Real*>(d.off[s]);
    Real* u = static_cast<Real*>(d.u[s]);
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x) {
      const long long to = d.hole_a[s][k], from = d.hole_b[s][k];
      d.cell[s][to] = d.cell[s][from];
      off[to] = off[from];
      u[to] = u[from];
      if (d.ulo[s]) d.ulo[s][to] = d.ulo[s][from];
    }
  }
}

// ---------------------------------------------------------------------------
// Batched cascades.  Per step: conversion for every member (one row of CTAs
// per member), a one-CTA plan that prices every member's particles and scans
// the costs, the persistent particle kernel whose CTAs each take an equal
// contiguous part of the total cost (staging each member's E and
// accumulating its current in shared memory, then adding it to the member's
// FP64 current with global atomics), and the field kernel (one CTA per
// member).  Members whose remaining step count is zero are skipped by all
// four.
// ---------------------------------------------------------------------------
template <class Real>
__global__ void k_batch_convert(BatchDev b) {
  const int slot = blockIdx.y;
  if (b.remaining[slot] <= 0) return;
  const Dev& d = b.devs[slot];
  Ctl* ctl = d.ctl;
  const long long step = ctl->step;
  const long long src = step - 1 - d.n_pp;
  const long long head = ctl->ph_head;
  const long long end = (src >= 0) ? d.emit_end[src % (d.n_pp + 1)] : head;
  const long long n0 = ctl->n[0], n1 = ctl->n[1];
  long long cnt = end - head;
  const long long room = min(d.cap - n0, d.cap - n1);
  const bool over = cnt > room;
  if (over) cnt = room;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    ctl->conv_count = cnt;
    ctl->conv_end = end;
    if (over) set_error(ctl, CASCADE_ERR_CAPACITY);
  }
  const Real up = (Real)d.u_pair;
  const Real* ph_off = static_cast<const Real*>(d.ph_off);
  Real* off0 = static_cast<Real*>(d.off[0]);
  Real* off1 = static_cast<Real*>(d.off[1]);
  Real* u0 = static_cast<Real*>(d.u[0]);
  Real* u1 = static_cast<Real*>(d.u[1]);
  const long long mask = d.ph_cap - 1;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < cnt;
       i += (long long)gridDim.x * blockDim.x) {
    const long long slot_ph = (head + i) & mask;
    const int enc = d.ph_cell[slot_ph];
    const int cell = enc & 0x7fffffff;
    const Real oc = ph_off[slot_ph];
    const Real uv = (enc < 0) ? -up : up;
    d.cell[0][n0 + i] = cell;
    off0[n0 + i] = oc;
    u0[n0 + i] = uv;
    d.cell[1][n1 + i] = cell;
    off1[n1 + i] = oc;
    u1[n1 + i] = uv;
    if (d.ulo[0]) {  // two-word momenta: the rounding residual of u_pair
      const float lo = (float)(d.u_pair - (double)up);
      d.ulo[0][n0 + i] = (enc < 0) ? -lo : lo;
      d.ulo[1][n1 + i] = (enc < 0) ? -lo : lo;
    }
  }
}

// Work units of one active member this step: its 4-particle chunks plus a
// fixed share standing for staging E and flushing the current (member_cost +
// nx / 4 chunks), so that contiguous ranges of equal cost take about equal
// time.
__device__ __forceinline__ long long batch_units(const BatchDev& b, const Dev& d) {
  const long long cc = d.ctl->conv_count;
  const long long N0 = d.ctl->n[0] + cc, N1 = d.ctl->n[1] + cc;
  return ((N0 + 3) >> 2) + ((N1 + 3) >> 2) + b.member_cost + (d.nx >> 2);
}

// Exclusive scan of the members' work units over the slots.
template <class Real>
__global__ void __launch_bounds__(1024) k_batch_plan(BatchDev b) {
  __shared__ long long warp_tot[32];
  __shared__ long long s_total;
  const int per = (b.n + blockDim.x - 1) / blockDim.x;
  const int lo = threadIdx.x * per;
  const int hi = min(lo + per, b.n);
  long long mine = 0;
  for (int i = lo; i < hi; ++i)
    if (b.remaining[i] > 0) mine += batch_units(b, b.devs[i]);
  // block-wide exclusive scan of the per-thread totals
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  long long incl = mine;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const long long v = __shfl_up_sync(kFull, incl, o);
    if (lane >= o) incl += v;
  }
  if (lane == 31) warp_tot[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    long long v = lane < (int)(blockDim.x >> 5) ? warp_tot[lane] : 0;
    long long w = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const long long t = __shfl_up_sync(kFull, w, o);
      if (lane >= o) w += t;
    }
    warp_tot[lane] = w - v;  // exclusive prefix of the warps
  }
  __syncthreads();
  long long start = warp_tot[warp] + incl - mine;
  for (int i = lo; i < hi; ++i) {
    b.item_start[i] = start;
    if (b.remaining[i] > 0) start += batch_units(b, b.devs[i]);
  }
  if (threadIdx.x == blockDim.x - 1) {
    b.item_start[b.n] = warp_tot[warp] + incl;
    s_total = warp_tot[warp] + incl;
  }
  if (b.member_ctas) {
    // constant-bank kernel: each member's CTAs in proportion to its work
    // units (rounded up), at least one, at most the grid's row
    __syncthreads();
    const long long total = s_total;
    for (int i = lo; i < hi; ++i) {
      int k = 0;
      if (b.remaining[i] > 0 && total > 0) {
        const long long u = batch_units(b, b.devs[i]);
        const long long kk = (u * (long long)b.target_ctas + total - 1) / total;
        k = kk < 1 ? 1 : (kk > b.max_ctas ? b.max_ctas : (int)kk);
      }
      b.member_ctas[i] = k;
    }
  }
}

// Chunks [a, e) of member `slot` (species 0's chunks first, then species
// 1's), clipped to the member's chunk count: copy its descriptor, stage its E
// and clear the accumulator, advance the particles, then add the CTA's sum of
// gamma and current to the member's FP64 totals with global atomics.
template <class Real, int DEP, bool STG, class DevT>
__device__ __forceinline__ void batch_member_range(const BatchDev& b, const DevT& d, PushState<Real, DEP>& st,
                                                   double* red, unsigned char* stage, long long a, long long e,
                                                   long long C0, long long N0, long long N1);

template <class Real, int DEP, bool STG>
__device__ __forceinline__ void batch_range(const BatchDev& b, Dev& sd, PushState<Real, DEP>& st, double* red,
                                            unsigned char* stage, int slot, long long a, long long e) {
  {
    const long long* src = reinterpret_cast<const long long*>(b.devs + slot);
    long long* dst = reinterpret_cast<long long*>(&sd);
    for (int w = threadIdx.x; w < (int)(sizeof(Dev) / 8); w += blockDim.x) dst[w] = src[w];
  }
  __syncthreads();
  const Dev& d = sd;
  Ctl* ctl = d.ctl;
  const long long cc = ctl->conv_count;
  const long long N0 = ctl->n[0] + cc, N1 = ctl->n[1] + cc;
  const long long C0 = (N0 + 3) >> 2, C = C0 + ((N1 + 3) >> 2);
  if (e > C) e = C;
  if (a >= e) {
    __syncthreads();  // every thread has read sd before the next member overwrites it
    return;
  }
  batch_member_range<Real, DEP, STG>(b, d, st, red, stage, a, e, C0, N0, N1);
}

// The particles of chunks [a, e) of one member (descriptor d: in shared
// memory for k_batch_push, in the constant bank for k_batch_push_c): stage
// its E and clear the accumulator, advance the particles, then add the CTA's
// sum of gamma and current to the member's FP64 totals with global atomics.
template <class Real, int DEP, bool STG, class DevT>
__device__ __forceinline__ void batch_member_range(const BatchDev& b, const DevT& d, PushState<Real, DEP>& st,
                                                   double* red, unsigned char* stage, long long a, long long e,
                                                   long long C0, long long N0, long long N1) {
  typedef typename AccOf<Real, DEP>::type Acc;
  Ctl* ctl = d.ctl;
  const int nx = d.nx;
  for (int i = threadIdx.x; i < nx; i += blockDim.x) {
    st.Es[i] = (Real)d.E[i];
    st.Ss[i] = Acc(0);
    if (DEP == 4) st.Ls[i] = 0;
  }
  st.ctl = ctl;
  st.ph_tail = ctl->ph_tail;
  st.room = d.ph_cap - (st.ph_tail - ctl->conv_end);
  st.ph_mask = d.ph_cap - 1;
  set_scales<Real, DEP>(st, (double)((e - a) * 4), d.dtdx);
  __syncthreads();

  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double gsum = 0.0;
  // chunk and particle indices in 32 bits: a batch member holds at most
  // 2^30 particles per species (checked at admission)
  const int a32 = (int)a, e32 = (int)e, c0 = (int)C0, n0 = (int)N0, n1 = (int)N1;
  const int nthr = (int)blockDim.x, tid = (int)threadIdx.x;
  const int iters = (e32 - a32 + nthr - 1) / nthr;
  const int pf = b.prefetch;
  // this thread's staging slots (STG): [stage][array][thread][16 B]
  const size_t slab = (size_t)blockDim.x * 16;
  auto slot_of = [&](int bb, int arr) { return stage + (size_t)(bb * 3 + arr) * slab + (size_t)threadIdx.x * 16; };
  auto issue = [&](int it) {  // cp.async of iteration it's chunk into stage it & 1
    const int ch = a32 + it * nthr + tid;
    if (it < iters && ch < e32) {
      const int sp = ch < c0 ? 0 : 1;
      const int bp = (ch - (sp ? c0 : 0)) * 4;
      const unsigned bytes = (unsigned)min(4, (sp ? n1 : n0) - bp) * 4u;
      const int bb = it & 1;
      cp_async16(slot_of(bb, 0), d.cell[sp] + bp, bytes);
      cp_async16(slot_of(bb, 1), static_cast<const Real*>(d.off[sp]) + bp, bytes);
      cp_async16(slot_of(bb, 2), static_cast<const Real*>(d.u[sp]) + bp, bytes);
    }
    cp_async_commit();  // one group per iteration, empty or not
  };
  if (STG) issue(0);
  for (int it = 0; it < iters; ++it) {
    if (pf > 0 && lane == 0) {
      // the warp's particles pf iterations ahead, inside this range
      const int chp = a32 + (it + pf) * nthr + warp * 32;
      if (chp < e32) {
        const int sp = chp < c0 ? 0 : 1;
        const long long bp = (long long)(chp - (sp ? c0 : 0)) * 4;
        long long np = d.cap4 - bp;  // stay inside the allocation
        if (np > 128) np = 128;
        if (np > 0) {
          prefetch_l2(d.cell[sp] + bp, (unsigned)(np * 4) & ~15u);
          prefetch_l2(static_cast<const Real*>(d.off[sp]) + bp, (unsigned)(np * sizeof(Real)) & ~15u);
          prefetch_l2(static_cast<const Real*>(d.u[sp]) + bp, (unsigned)(np * sizeof(Real)) & ~15u);
        }
      }
    }
    const int ch = a32 + it * nthr + tid;
    int s = 0, cnt = 0, base = 0;
    if (ch < e32) {
      s = ch < c0 ? 0 : 1;
      base = (ch - (s ? c0 : 0)) * 4;
      cnt = min(4, (s ? n1 : n0) - base);
    }
    if (STG) {
      issue(it + 1);
      cp_async_wait_prev();  // iteration it's copies have landed
      const int bb = it & 1;
      const unsigned char* stg[3] = {slot_of(bb, 0), slot_of(bb, 1), slot_of(bb, 2)};
      gsum += (double)process4<Real, kSmemESmemS, DEP, true, false, true, false, DevT>(d, st, s, base, cnt, lane,
                                                                                    stg);
    } else {
      gsum += (double)process4<Real, kSmemESmemS, DEP, true, false, false, false, DevT>(d, st, s, base, cnt, lane);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) gsum += __shfl_down_sync(kFull, gsum, o);
  if (lane == 0) red[warp] = gsum;
  __syncthreads();
  if (threadIdx.x == 0) {
    double v = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += red[w];
    atomicAdd(d.uk_part, v);
  }
  for (int i = threadIdx.x; i < nx; i += blockDim.x) {
    double v;
    if (DEP == 1) v = (double)st.Ss[i] * (double)st.fx_inv;
    else if (DEP == 4) v = (double)st.Ss[i] * (double)st.fx_inv + (double)st.Ls[i] * (double)st.lo_inv;
    else v = (double)st.Ss[i];
    if (v != 0.0) atomicAdd(d.S_glob + i, v);
  }
  __syncthreads();
}

// CTA k takes the k-th of gridDim.x equal parts of the members' total cost
// (the exclusive scan in item_start): a contiguous run of chunks that changes
// member only at member boundaries, so each CTA stages a member's E and
// flushes its current once per launch, and its particles stream through in
// order (prefetched into L2 ahead of use).
// Launch shapes of the batched particle kernel: threads per CTA and the CTAs
// per SM its register budget is sized for (65536 registers per SM).  Shape 3
// is the default (see batch_configure).
template <int SHAPE>
struct BatchShape;
template <>
struct BatchShape<0> {  // 2 x 512 threads, 64 registers
  static constexpr int threads = 512, minb = 2;
};
template <>
struct BatchShape<1> {  // 1 x 512 threads, up to 128 registers
  static constexpr int threads = 512, minb = 1;
};
template <>
struct BatchShape<2> {  // 1 x 768 threads, up to 80 registers
  static constexpr int threads = 768, minb = 1;
};
template <>
struct BatchShape<3> {  // 1 x 640 threads, up to 96 registers
  static constexpr int threads = 640, minb = 1;
};

// STG (FP32): particles staged through shared memory with cp.async, as in
// the single-cascade kernel; the staging area follows E and the accumulator.
template <class Real, int DEP, int SHAPE, bool STG>
__global__ void __launch_bounds__(BatchShape<SHAPE>::threads, BatchShape<SHAPE>::minb) k_batch_push(BatchDev b) {
  static_assert(!STG || sizeof(Real) == 4, "the staging slots hold four 4-byte values");
  typedef typename AccOf<Real, DEP>::type Acc;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ __align__(16) Dev sd;
  __shared__ double red[32];
  __shared__ long long s_start[kBatchSmemSlots + 1];  // cost offsets of the members
  const long long total = b.item_start[b.n];
  const long long lo = total * (long long)blockIdx.x / gridDim.x;
  const long long hi = total * (long long)(blockIdx.x + 1) / gridDim.x;
  if (lo >= hi) return;
  const bool cached = b.n <= kBatchSmemSlots;
  if (cached)
    for (int i = threadIdx.x; i <= b.n; i += blockDim.x) s_start[i] = b.item_start[i];
  __syncthreads();
  const long long* starts = cached ? s_start : b.item_start;
  const size_t eb = ((size_t)b.max_nx * sizeof(Real) + 15) & ~size_t(15);
  PushState<Real, DEP> st;
  st.Es = reinterpret_cast<Real*>(smem_raw);
  st.Ss = reinterpret_cast<Acc*>(smem_raw + eb);
  st.Ls = reinterpret_cast<int*>(smem_raw + 2 * eb);
  unsigned char* stage = smem_raw + (DEP == 4 ? 3 : 2) * eb;
  int m = 0, top = b.n;  // last slot with starts[m] <= lo
  while (top - m > 1) {
    const int mid = (m + top) >> 1;
    if (starts[mid] <= lo) m = mid;
    else top = mid;
  }
  for (; m < b.n && starts[m] < hi; ++m) {
    const long long s0 = starts[m], s1 = starts[m + 1];
    if (s1 <= s0 || s1 <= lo) continue;  // idle member, or one that ends before this range
    batch_range<Real, DEP, STG>(b, sd, st, red, stage, m, (lo > s0 ? lo : s0) - s0, (hi < s1 ? hi : s1) - s0);
  }
}

// The member table of the constant-bank batch kernel (each batch owns a
// slice of it, from b.const_base).
__constant__ BatchMember c_members[kConstMembers];

// Constant-bank form of the batched particle kernel: grid (max_ctas, slots)
// of 1024-thread CTAs.  CTA (x, m) works on member m only, on the x-th of the
// member_ctas[m] equal parts of its chunks (the plan kernel sizes
// member_ctas[m] in proportion to the member's work); the other CTAs of the
// row return at once.  The member index is blockIdx.y, so its descriptor is
// read from the constant bank with a warp-uniform index and needs no
// per-thread registers: the kernel fits 1024 threads at 64 registers, like
// the single-cascade kernel, where the shared-memory descriptor of
// k_batch_push needs 96.  The hardware schedules the CTAs as SMs free up,
// which balances the members.
template <class Real, int DEP, bool STG>
__global__ void __launch_bounds__(1024, 1) k_batch_push_c(BatchDev b) {
  static_assert(!STG || sizeof(Real) == 4, "the staging slots hold four 4-byte values");
  const int slot = blockIdx.y;
  if (b.remaining[slot] <= 0) return;
  const int K = b.member_ctas[slot];
  if ((int)blockIdx.x >= K) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[32];
  const BatchMember& d = c_members[b.const_base + slot];
  Ctl* ctl = d.ctl;
  const long long cc = ctl->conv_count;
  const long long N0 = ctl->n[0] + cc, N1 = ctl->n[1] + cc;
  const long long C0 = (N0 + 3) >> 2, C = C0 + ((N1 + 3) >> 2);
  const long long a = C * blockIdx.x / K, e = C * (blockIdx.x + 1) / K;
  if (a >= e) return;  // the whole CTA returns together
  typedef typename AccOf<Real, DEP>::type Acc;
  const size_t eb = ((size_t)b.max_nx * sizeof(Real) + 15) & ~size_t(15);
  PushState<Real, DEP> st;
  st.Es = reinterpret_cast<Real*>(smem_raw);
  st.Ss = reinterpret_cast<Acc*>(smem_raw + eb);
  st.Ls = reinterpret_cast<int*>(smem_raw + 2 * eb);
  unsigned char* stage = smem_raw + (DEP == 4 ? 3 : 2) * eb;
  batch_member_range<Real, DEP, STG>(b, d, st, red, stage, a, e, C0, N0, N1);
}

template <class Real>
__global__ void __launch_bounds__(kFieldBlock) k_batch_field(BatchDev b) {
  __shared__ double sh[128];
  const int slot = blockIdx.x;
  if (b.remaining[slot] <= 0) return;
  const Dev& d = b.devs[slot];
  double v[4] = {0.0, 0.0, 0.0, 0.0};
  for (int i = threadIdx.x; i < d.nx; i += blockDim.x) {
    const double S = d.S_glob[i];
    d.S_glob[i] = 0.0;
    const double J = d.jscale * S;
    const double E = d.E[i] - d.dt * (J - d.j_m);
    d.E[i] = E;
    d.J[i] = J;
    v[0] += E;
    v[1] += J;
    v[2] = fmax(v[2], fabs(E));
    v[3] += 0.5 * E * E * d.dx;
  }
  block_reduce4(v, sh);
  if (threadIdx.x == 0) {
    const double gsum = *d.uk_part;
    *d.uk_part = 0.0;
    finish_step(d, v, gsum);
    b.remaining[slot] -= 1;
  }
}

// ---------------------------------------------------------------------------
// Upload of a caller's state: offsets and momenta arrive as FP64 in a staging
// buffer and are rounded to the particle precision (an offset that rounds up
// to 1 is kept just below it); every particle is checked (cell inside the
// grid, offset in [0, 1), finite momentum) and the number of bad ones is
// counted in *bad.
// ---------------------------------------------------------------------------
template <class Real, class Src>
__global__ void k_upload(Dev d, int s, long long first, long long count, const Src* off_src,
                         const Src* u_src, unsigned int* bad) {
  Real* off = static_cast<Real*>(d.off[s]) + first;
  Real* u = static_cast<Real*>(d.u[s]) + first;
  const int* cell = d.cell[s] + first;
  unsigned int nbad = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
       i += (long long)gridDim.x * blockDim.x) {
    const double o = off_src[i];
    const double uu = u_src[i];
    const int c = cell[i];
    const bool ok = c >= 0 && c < d.nx && o >= 0.0 && o < 1.0 && isfinite(uu);
    Real oo = (Real)o;
    if (!(oo < Real(1))) oo = Real(1) - (sizeof(Real) == 4 ? Real(5.9604645e-8) : Real(1.1102230246251565e-16));
    off[i] = ok ? oo : Real(0);
    const Real uh = ok ? (Real)uu : Real(0);
    u[i] = uh;
    if (d.ulo[s]) d.ulo[s][first + i] = ok ? (float)(uu - (double)uh) : 0.f;  // two-word momenta
    nbad += ok ? 0u : 1u;
  }
  if (nbad) atomicAdd(bad, nbad);
}

// ---------------------------------------------------------------------------
// Phase-space histogram of one species: per-CTA shared-memory counts, then
// one global atomic per non-empty bin.
// ---------------------------------------------------------------------------
template <class Real>
__global__ void k_histogram(Dev d, int s, int quantity, int nbins, double lo, double hi,
                            unsigned long long* out) {
  extern __shared__ unsigned int hcount[];
  for (int i = threadIdx.x; i < nbins; i += blockDim.x) hcount[i] = 0u;
  __syncthreads();
  const long long n = d.ctl->n[s];
  const double scale = nbins / (hi - lo);
  const Real* off = static_cast<const Real*>(d.off[s]);
  const Real* u = static_cast<const Real*>(d.u[s]);
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n;
       p += (long long)gridDim.x * blockDim.x) {
    if (d.cell[s][p] < 0) continue;  // departed (open boundaries)
    double v;
    const double up = (double)u[p] + (d.ulo[s] ? (double)d.ulo[s][p] : 0.0);
    if (quantity == 0) v = up;
    else if (quantity == 1) v = sqrt(1.0 + up * up);
    else v = ((double)d.cell[s][p] + (double)off[p]) * d.dx;
    if (v >= lo && v < hi) {
      int b = (int)((v - lo) * scale);
      b = b >= nbins ? nbins - 1 : b;
      atomicAdd(&hcount[b], 1u);
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < nbins; i += blockDim.x)
    if (hcount[i]) atomicAdd(out + i, (unsigned long long)hcount[i]);
}

// ---------------------------------------------------------------------------
// Gauss's-law residual of the current state (diagnostic, not in the step).
// ---------------------------------------------------------------------------
// every > 0: part of a step -- only every every-th step computes (the step
// counter lives on the device, so captured graphs keep the cadence); the
// reduce kernel leaves rho_dx zeroed for the next use.  every = 0: on demand.
template <class Real>
__global__ void k_gauss_deposit(Dev d, double* rho_dx, int every = 0) {
  Ctl* ctl = d.ctl;
  if (every > 0 && ctl->step % every != 0) return;
  const long long N0 = ctl->n[0], N1 = ctl->n[1];
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < N0 + N1;
       t += (long long)gridDim.x * blockDim.x) {
    const int s = t < N0 ? 0 : 1;
    const long long p = s ? t - N0 : t;
    const int c = d.cell[s][p];
    if (c < 0) continue;  // departed (open boundaries)
    const double o = (double)static_cast<const Real*>(d.off[s])[p];
    const double qw = (s ? 1.0 : -1.0) * d.w;
    atomicAdd(&rho_dx[c], qw * (1.0 - o));
    if (c + 1 < d.nx) atomicAdd(&rho_dx[c + 1], qw * o);
    else if (!d.open_bc) atomicAdd(&rho_dx[0], qw * o);  // periodic: node nx is node 0
  }
}

template <class Real>
__global__ void k_gauss_reduce(Dev d, double* rho_dx, double* out, int every = 0) {
  __shared__ double sh[128];
  if (every > 0 && d.ctl->step % every != 0) return;
  double v[4] = {0.0, 0.0, 0.0, 0.0};
  // dE/dx = rho - rho_GJ (Eq. 25); with open boundaries interior nodes only
  for (int i = threadIdx.x + (d.open_bc ? 1 : 0); i < d.nx; i += blockDim.x) {
    const int im = (i == 0) ? d.nx - 1 : i - 1;
    v[2] = fmax(v[2], fabs(d.E[i] - d.E[im] - (rho_dx[i] - d.rho_gj * d.dx)));
  }
  block_reduce4(v, sh);
  if (every > 0) {
    // every thread's reads of rho_dx are done (block_reduce4 synchronises)
    for (int i = threadIdx.x; i < d.nx; i += blockDim.x) rho_dx[i] = 0.0;
  }
  if (threadIdx.x == 0) {
    *out = v[2];
    const long long st = d.ctl->step;
    if (st > 0) {
      d.ring[(st - 1) % d.ring_n].gauss_resid = v[2];
      d.ctl->last.gauss_resid = v[2];
    }
  }
}

// ---------------------------------------------------------------------------
// Launchers (instantiated per precision by the including .cu file).
// ---------------------------------------------------------------------------
// Particle-kernel variants compiled for one precision: (V, DEP, FAST).  FP64
// keeps only the exact variants; FP32 adds the fast gamma and the fixed-point
// accumulator.
template <class Real>
struct PushTable {
  static const void* get(int V, int dep, bool fast, bool open, bool stage, bool comp = false);
};
template <>
inline const void* PushTable<double>::get(int V, int, bool, bool open, bool, bool) {
  if (V == kSmemESmemS)
    return open ? reinterpret_cast<const void*>(&k_push<double, kSmemESmemS, 0, false, true>)
                : reinterpret_cast<const void*>(&k_push<double, kSmemESmemS, 0, false, false>);
  if (V == kSmemEGlobS)
    return open ? reinterpret_cast<const void*>(&k_push<double, kSmemEGlobS, 0, false, true>)
                : reinterpret_cast<const void*>(&k_push<double, kSmemEGlobS, 0, false, false>);
  if (V == kGlobESmemS) return reinterpret_cast<const void*>(&k_push<double, kGlobESmemS, 0, false, false>);
  return reinterpret_cast<const void*>(&k_push<double, kGlobEGlobS, 0, false, false>);
}
template <>
inline const void* PushTable<float>::get(int V, int dep, bool, bool open, bool stage, bool comp) {
  if (comp) {  // two-word momenta: the shared-memory accumulator forms, direct loads
    if (V == kSmemESmemS) {
      if (open) return reinterpret_cast<const void*>(&k_push<float, kSmemESmemS, 1, true, true, false, true>);
      if (dep == 4) return reinterpret_cast<const void*>(&k_push<float, kSmemESmemS, 4, true, false, false, true>);
      return reinterpret_cast<const void*>(&k_push<float, kSmemESmemS, 1, true, false, false, true>);
    }
    if (V == kGlobESmemS) {
      if (open) return reinterpret_cast<const void*>(&k_push<float, kGlobESmemS, 1, true, true, false, true>);
      return reinterpret_cast<const void*>(&k_push<float, kGlobESmemS, 1, true, false, false, true>);
    }
    return nullptr;
  }
  if (V == kSmemESmemS) {
    if (stage && !open && dep == 1)
      return reinterpret_cast<const void*>(&k_push<float, kSmemESmemS, 1, true, false, true>);
    if (open) return reinterpret_cast<const void*>(&k_push<float, kSmemESmemS, 1, true, true>);
    if (dep == 4) return reinterpret_cast<const void*>(&k_push<float, kSmemESmemS, 4, true, false>);
    return reinterpret_cast<const void*>(&k_push<float, kSmemESmemS, 1, true, false>);
  }
  if (V == kSmemEGlobS) return reinterpret_cast<const void*>(&k_push<float, kSmemEGlobS, 0, true, false>);
  if (V == kGlobESmemS) {
    if (open) return reinterpret_cast<const void*>(&k_push<float, kGlobESmemS, 1, true, true>);
    return reinterpret_cast<const void*>(&k_push<float, kGlobESmemS, 1, true, false>);
  }
  return reinterpret_cast<const void*>(&k_push<float, kGlobEGlobS, 0, true, false>);
}

inline int env_int(const char* name, int dflt) {
  const char* v = getenv(name);
  return (v && *v) ? atoi(v) : dflt;
}

template <class Real>
struct Launchers {
  static size_t smem_bytes(int nx, int variant, int dep = 0) { return smem_field_bytes<Real>(nx, variant, dep); }

  // dynamic shared memory of one particle-kernel launch
  static size_t push_smem(const Dev& d) {
    return smem_bytes(d.nx, d.variant, d.push_dep) + (d.push_stage ? kStageBytesPerThread * d.block_push : 0);
  }

  static const void* push_fn(const Dev& d) {
    return PushTable<Real>::get(d.variant, d.push_dep, d.push_fast != 0, d.open_bc != 0, d.push_stage != 0,
                                sizeof(Real) == 4 && d.u_words == 2);
  }

  static cudaError_t configure(Dev& d, int num_sms) {
    const size_t limit = 200 * 1024;
    int dep = 0, fast = 0;
    if (sizeof(Real) == 4) {
      dep = d.fine_deposit ? 4 : 1;
      const int forced = env_int("CASCADE_PUSH_DEP", 0);  // measurement override: 1 or 4
      if (forced == 1 || forced == 4) dep = forced;
      fast = 1;
    }
    int variant = kGlobEGlobS;
    if (smem_bytes(d.nx, kSmemESmemS, dep) <= limit) variant = kSmemESmemS;
    else if (dep == 4 && smem_bytes(d.nx, kSmemESmemS, 1) <= limit) {
      dep = 1;  // the two-word accumulator does not fit: one word
      variant = kSmemESmemS;
    } else if (sizeof(Real) == 4 && smem_bytes(d.nx, kGlobESmemS) <= limit) {
      // E does not fit beside the accumulator: gather it through L1 (read
      // only).  FP32 only: FP64 shared-memory atomics are compare-and-swap
      // loops and measured slower than FP64 global atomics (variant 1).
      variant = kGlobESmemS;
      if (dep == 4) dep = 1;
    } else if (smem_bytes(d.nx, kSmemEGlobS) <= limit) {
      variant = kSmemEGlobS;
    }
    if (variant == kGlobEGlobS) dep = 0;
    const bool comp = sizeof(Real) == 4 && d.u_words == 2;
    if (comp) {
      // two-word momenta are built for the shared-memory accumulator forms
      if (variant != kSmemESmemS && variant != kGlobESmemS) return cudaErrorNotSupported;
      if (variant == kGlobESmemS && dep == 4) dep = 1;
    }
    if (d.open_bc) {
      // open boundaries are built for the shared-memory accumulator variants
      // (plus E in shared memory with global FP64 atomics in FP64)
      if (dep == 4) dep = 1;
      if (variant == kGlobEGlobS || (sizeof(Real) == 8 && variant == kGlobESmemS))
        return cudaErrorInvalidValue;
    }
    d.variant = variant;
    d.push_dep = dep;
    d.push_fast = fast;
    const int block = PushBlock<Real>::value;
    d.block_push = block;
    d.push_stage = 0;
    if (sizeof(Real) == 4 && variant == kSmemESmemS && dep == 1 && !d.open_bc && !comp &&
        env_int("CASCADE_PUSH_STAGE", 1) == 1) {
      // the staging area must fit beside E, the accumulator and the
      // kernel's static shared memory
      int dev = 0, optin = 0;
      cudaGetDevice(&dev);
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
      cudaFuncAttributes fa{};
      const cudaError_t ea = cudaFuncGetAttributes(&fa, PushTable<Real>::get(variant, dep, fast != 0, false, true));
      if (ea != cudaSuccess) return ea;
      if (smem_bytes(d.nx, variant, dep) + kStageBytesPerThread * block + fa.sharedSizeBytes <= (size_t)optin)
        d.push_stage = 1;
    }
    const size_t smem = push_smem(d);
    const void* fn = push_fn(d);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, block, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    d.grid_push = per_sm * num_sms;
    // L2 prefetch one iteration ahead: +4.6% with direct loads; with the
    // particles staged through shared memory it costs 8% and is off
    d.prefetch = env_int("CASCADE_PUSH_PREFETCH", d.push_stage ? 0 : 1);
    if (d.prefetch < 0 || d.prefetch > 8) d.prefetch = 0;
    d.grid_field = (d.nx + 31) / 32;
    d.nxp = (d.nx + 31) & ~31;
    d.min_per_cta = d.nx > 2048 ? d.nx : 2048;
    return cudaSuccess;
  }

  static cudaError_t seed(const Dev& d, long long npairs, int ppc, unsigned long long s, double spread,
                          cudaStream_t st) {
    if (npairs <= 0) return cudaSuccess;
    long long blocks = (npairs + 255) / 256;
    if (blocks > 65535) blocks = 65535;
    k_seed<Real><<<(int)blocks, 256, 0, st>>>(d, npairs, ppc, s, spread);
    return cudaGetLastError();
  }

  // One step: conversion, particle kernel, field kernel.  With events given,
  // they are recorded around the particle kernel.
  static cudaError_t step(const Dev& d, cudaStream_t st, cudaEvent_t before = nullptr,
                          cudaEvent_t after = nullptr) {
    k_convert<Real><<<d.grid_push, 256, 0, st>>>(d);
    if (before) cudaEventRecord(before, st);
    Dev arg = d;
    void* args[] = {&arg};
    cudaError_t e = cudaLaunchKernel(push_fn(d), dim3(d.grid_push), dim3(d.block_push), args,
                                     push_smem(d), st);
    if (e != cudaSuccess) return e;
    if (after) cudaEventRecord(after, st);
    if (d.open_bc) {
      k_compact_plan<Real><<<64, 256, 0, st>>>(d);
      k_compact_move<Real><<<64, 256, 0, st>>>(d);
    }
    if (d.variant == kSmemESmemS || d.variant == kGlobESmemS) {
      if (sizeof(Real) == 4 && d.push_dep == 1) k_field<int, true><<<d.grid_field, kFieldBlock, 0, st>>>(d);
      else k_field<Real, true><<<d.grid_field, kFieldBlock, 0, st>>>(d);
    } else {
      k_field<Real, false><<<d.grid_field, kFieldBlock, 0, st>>>(d);
    }
    if (d.gauss_every > 0) {  // the per-step Gauss residual, every gauss_every steps
      k_gauss_deposit<Real><<<d.grid_push, 256, 0, st>>>(d, d.gauss_rho, d.gauss_every);
      k_gauss_reduce<Real><<<1, 1024, 0, st>>>(d, d.gauss_rho, d.gauss_out, d.gauss_every);
    }
    return cudaGetLastError();
  }

  template <int DEP, bool STG>
  static const void* batch_push_shape(int shape) {
    switch (shape) {
      case 1: return reinterpret_cast<const void*>(&k_batch_push<Real, DEP, 1, STG>);
      case 2: return reinterpret_cast<const void*>(&k_batch_push<Real, DEP, 2, STG>);
      case 3: return reinterpret_cast<const void*>(&k_batch_push<Real, DEP, 3, STG>);
      default: return reinterpret_cast<const void*>(&k_batch_push<Real, DEP, 0, STG>);
    }
  }

  // shape: see BatchShape (0-3, the persistent kernel) or 4 (the
  // constant-bank kernel k_batch_push_c, FP32 only); stage: cp.async staging
  // (FP32 only).  nullptr: no such kernel.
  static const void* batch_push_fn(int dep, int shape, bool stage) {
    if constexpr (sizeof(Real) == 8) {
      if (shape == 4) return nullptr;
      return batch_push_shape<0, false>(shape);
    } else {
      if (shape == 4) {
        if (stage)
          return dep == 4 ? reinterpret_cast<const void*>(&k_batch_push_c<Real, 4, true>)
                          : reinterpret_cast<const void*>(&k_batch_push_c<Real, 1, true>);
        return dep == 4 ? reinterpret_cast<const void*>(&k_batch_push_c<Real, 4, false>)
                        : reinterpret_cast<const void*>(&k_batch_push_c<Real, 1, false>);
      }
      if (stage) return dep == 4 ? batch_push_shape<4, true>(shape) : batch_push_shape<1, true>(shape);
      return dep == 4 ? batch_push_shape<4, false>(shape) : batch_push_shape<1, false>(shape);
    }
  }

  static int batch_minb(int shape) { return shape == 0 ? BatchShape<0>::minb : 1; }

  static int batch_threads(int shape) {
    switch (shape) {
      case 1: return BatchShape<1>::threads;
      case 2: return BatchShape<2>::threads;
      case 3: return BatchShape<3>::threads;
      case 4: return 1024;
      default: return BatchShape<0>::threads;
    }
  }

  static cudaError_t batch_member_set(int index, const BatchMember* m, cudaStream_t st) {
    if (index < 0 || index >= kConstMembers) return cudaErrorInvalidValue;
    return cudaMemcpyToSymbolAsync(c_members, m, sizeof(BatchMember), sizeof(BatchMember) * (size_t)index,
                                   cudaMemcpyHostToDevice, st);
  }

  // Launch configuration of the batched particle kernel for one variant:
  // shape (see BatchShape) and stage (cp.async staging, FP32 only).  A stage
  // request that does not fit beside E, the accumulator and the kernel's
  // static shared memory (per CTA, and for the CTAs per SM of the shape, with
  // the 1 KB the system reserves per CTA) returns cudaErrorInvalidValue, as
  // does a grid too large for the shared-memory accumulator.
  static cudaError_t batch_configure(int max_nx, int fine, int num_sms, int shape, int stage, int* grid, int* block,
                                     size_t* smem, int* dep) {
    int dp = sizeof(Real) == 8 ? 0 : (fine ? 4 : 1);
    const size_t limit = 200 * 1024;
    if (smem_bytes(max_nx, kSmemESmemS, dp) > limit && dp == 4) dp = 1;
    const size_t sm = smem_bytes(max_nx, kSmemESmemS, dp);
    if (sm > limit) return cudaErrorInvalidValue;
    if (shape < 0 || shape > 4) return cudaErrorInvalidValue;
    if (stage && sizeof(Real) != 4) return cudaErrorInvalidValue;
    if (!batch_push_fn(dp, shape, stage != 0)) return cudaErrorInvalidValue;
    const int threads = batch_threads(shape);
    if (stage) {
      int dev = 0, optin = 0, per_sm_max = 0;
      cudaGetDevice(&dev);
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
      cudaDeviceGetAttribute(&per_sm_max, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
      cudaFuncAttributes fa{};
      const cudaError_t ea = cudaFuncGetAttributes(&fa, batch_push_fn(dp, shape, true));
      if (ea != cudaSuccess) return ea;
      const size_t per_cta = sm + kStageBytesPerThread * threads;
      if (per_cta + fa.sharedSizeBytes > (size_t)optin ||
          (per_cta + fa.sharedSizeBytes + 1024) * batch_minb(shape) > (size_t)per_sm_max)
        return cudaErrorInvalidValue;
    }
    const size_t smem_total = sm + (stage ? kStageBytesPerThread * threads : 0);
    const void* fn = batch_push_fn(dp, shape, stage != 0);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_total);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, smem_total);
    if (e != cudaSuccess) return e;
    *grid = (per_sm < 1 ? 1 : per_sm) * num_sms;
    *block = threads;
    *smem = smem_total;
    // kernel selector: accumulator form, launch shape, staging
    *dep = dp + 16 * shape + 256 * (stage ? 1 : 0);
    return cudaSuccess;
  }

  // One batch step; with events given, they are recorded around the
  // particle kernel.
  static cudaError_t batch_step(const BatchDev& b, int grid, int block, size_t smem, int dep, cudaStream_t st,
                                cudaEvent_t before = nullptr, cudaEvent_t after = nullptr) {
    k_batch_convert<Real><<<dim3(16, b.n), 256, 0, st>>>(b);
    k_batch_plan<Real><<<1, 1024, 0, st>>>(b);
    if (before) cudaEventRecord(before, st);
    BatchDev arg = b;
    void* args[] = {&arg};
    const int shape = (dep / 16) % 16;
    // the constant-bank kernel: one row of max_ctas CTAs per member slot
    const dim3 g = shape == 4 ? dim3(b.max_ctas, b.n) : dim3(grid);
    cudaError_t e = cudaLaunchKernel(batch_push_fn(dep % 16, shape, dep / 256 != 0), g, dim3(block), args, smem, st);
    if (e != cudaSuccess) return e;
    if (after) cudaEventRecord(after, st);
    k_batch_field<Real><<<b.n, kFieldBlock, 0, st>>>(b);
    return cudaGetLastError();
  }

  // src_f32: the staged offsets and momenta are float (else double)
  static cudaError_t upload(const Dev& d, int sp, long long first, long long count, const void* off_src,
                            const void* u_src, int src_f32, unsigned int* bad, cudaStream_t st) {
    if (count <= 0) return cudaSuccess;
    long long blocks = (count + 255) / 256;
    if (blocks > 8192) blocks = 8192;
    if (src_f32)
      k_upload<Real, float><<<(int)blocks, 256, 0, st>>>(d, sp, first, count, static_cast<const float*>(off_src),
                                                         static_cast<const float*>(u_src), bad);
    else
      k_upload<Real, double><<<(int)blocks, 256, 0, st>>>(d, sp, first, count, static_cast<const double*>(off_src),
                                                          static_cast<const double*>(u_src), bad);
    return cudaGetLastError();
  }

  static cudaError_t histogram(const Dev& d, int sp, int quantity, int nbins, double lo, double hi,
                               unsigned long long* out, cudaStream_t st) {
    const size_t sm = sizeof(unsigned int) * (size_t)nbins;
    cudaError_t e = cudaFuncSetAttribute(reinterpret_cast<const void*>(&k_histogram<Real>),
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(out, 0, sizeof(unsigned long long) * nbins, st);
    if (e != cudaSuccess) return e;
    k_histogram<Real><<<d.grid_push, 512, sm, st>>>(d, sp, quantity, nbins, lo, hi, out);
    return cudaGetLastError();
  }

  static cudaError_t gauss(const Dev& d, double* rho_dx, double* out, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(rho_dx, 0, sizeof(double) * d.nx, st);
    if (e != cudaSuccess) return e;
    k_gauss_deposit<Real><<<d.grid_push, 256, 0, st>>>(d, rho_dx);
    k_gauss_reduce<Real><<<1, 1024, 0, st>>>(d, rho_dx, out);
    return cudaGetLastError();
  }
};

}  // namespace cpic

#define CASCADE_DEFINE_LAUNCHERS(SUFFIX, REAL)                                               \
  namespace cpic {                                                                             \
  cudaError_t seed_##SUFFIX(const Dev& d, long long npairs, int ppc, unsigned long long seed,    \
                            double u_spread, cudaStream_t s) {                                    \
    return Launchers<REAL>::seed(d, npairs, ppc, seed, u_spread, s);                         \
  }                                                                                               \
  cudaError_t step_##SUFFIX(const Dev& d, cudaStream_t s) { return Launchers<REAL>::step(d, s); } \
  cudaError_t step_timed_##SUFFIX(const Dev& d, cudaStream_t s, cudaEvent_t b, cudaEvent_t a) {  \
    return Launchers<REAL>::step(d, s, b, a);                                                \
  }                                                                                               \
  cudaError_t gauss_##SUFFIX(const Dev& d, double* rho_dx, double* out, cudaStream_t s) {         \
    return Launchers<REAL>::gauss(d, rho_dx, out, s);                                        \
  }                                                                                               \
  cudaError_t configure_##SUFFIX(Dev& d, int num_sms) { return Launchers<REAL>::configure(d, num_sms); } \
  cudaError_t batch_configure_##SUFFIX(int max_nx, int fine, int num_sms, int shape, int stage, int* grid, \
                                       int* block, size_t* smem, int* dep) {                    \
    return Launchers<REAL>::batch_configure(max_nx, fine, num_sms, shape, stage, grid, block, smem, dep); \
  }                                                                                               \
  cudaError_t batch_step_##SUFFIX(const BatchDev& b, int grid, int block, size_t smem, int dep,   \
                                  cudaStream_t s, cudaEvent_t before, cudaEvent_t after) {        \
    return Launchers<REAL>::batch_step(b, grid, block, smem, dep, s, before, after);              \
  }                                                                                               \
  size_t partial_bytes_##SUFFIX() { return sizeof(REAL); }                                       \
  cudaError_t batch_member_set_##SUFFIX(int index, const BatchMember* m, cudaStream_t s) {          \
    return Launchers<REAL>::batch_member_set(index, m, s);                                        \
  }                                                                                               \
  cudaError_t histogram_##SUFFIX(const Dev& d, int sp, int q, int nb, double lo, double hi,          \
                                 unsigned long long* out, cudaStream_t s) {                       \
    return Launchers<REAL>::histogram(d, sp, q, nb, lo, hi, out, s);                              \
  }                                                                                               \
  cudaError_t upload_##SUFFIX(const Dev& d, int sp, long long first, long long count, const void* o,  \
                              const void* u, int src_f32, unsigned int* bad, cudaStream_t s) {      \
    return Launchers<REAL>::upload(d, sp, first, count, o, u, src_f32, bad, s);                   \
  }                                         \
  }
