// Internal types shared by the host side (cascade_capi.cu) and the kernel
// translation units (kernels_fp64.cu, kernels_fp32.cu).  Not part of the ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "cascade.h"

namespace cpic {

// Device-resident counters of one cascade.  Every kernel of a step reads the
// counters it needs from here, so a step has no host synchronisation and a
// captured CUDA graph of steps can be replayed unchanged.
struct Ctl {
  long long n[2];                 // particles per species (0 = e-, 1 = e+)
  long long ph_head, ph_tail;     // photon FIFO: [ph_head, ph_tail) in flight (monotone)
  long long pairs_total;          // pairs created since the start
  long long emit_multi;           // emissions of k > 1 photons
  long long step;                 // steps completed
  long long conv_count;           // pairs created by the current step's conversion
  long long conv_end;             // FIFO head once the current step's photons are converted
  unsigned long long emit_count;  // photons appended by the current step
  int err;                        // first device-side error (cascade_status), 0 if none
  int active_blocks;              // particle-kernel CTAs that work in the current step
  unsigned int field_ticket;      // last-block detection in the field kernel
  float part_inv;                 // FP32 int32 current partials: the common scale 2^-k
  // open boundaries: departed particles of the current step and the
  // compaction that fills their slots
  unsigned long long n_holes[2];  // departed (hole-list entries, may exceed the list)
  unsigned long long na[2];       // holes below the new count
  unsigned long long nb[2];       // live particles at or above the new count
  cascade_diag_t last;            // the latest per-step record (also in the ring), read with the counters
};

// Everything a kernel needs about one cascade, passed by value.
struct Dev {
  // grid and model constants
  int nx;              // cells
  int nxp;             // row pitch of the per-CTA current partials (nx rounded up to 32)
  int n_pp;            // photon flight in steps
  int lpp_int;         // floor(l_pp / dx)
  long long cap;       // particle capacity per species
  long long cap4;      // allocated particles per species (cap rounded up to 4)
  long long ph_cap;    // photon ring capacity (power of two)
  double dx, dt, dtdx, jscale, w;
  double gamma_thr, eps_gamma, lpp_frac, u_pair;
  // particle storage (SoA, one array per species; Real = float or double)
  int32_t* cell[2];
  void* off[2];
  void* u[2];
  float* ulo[2];       // FP32 two-word momentum: the low word (u = u + ulo), else null
  // photon ring: conversion cell (bit 31 = direction is -x) and offset
  int32_t* ph_cell;
  void* ph_off;
  // fields and reduction buffers
  double* E;           // E_{i+1/2}, nx
  double* J;           // J_{i+1/2}^{n+1/2}, nx
  void* S_part;        // per-CTA charge-flux partials, [grid_push][nxp]: int32 at the scale
                       // ctl->part_inv (FP32, one-word accumulator), else Real
  double* S_glob;      // nx, when the partials do not fit in shared memory
  double* uk_part;     // per-CTA sum of gamma, [grid_push]
  double* diag_part;   // per-CTA field diagnostics of the field kernel, [grid_field][4]
  long long* emit_end; // FIFO tail after step m, ring of n_pp + 1
  Ctl* ctl;
  cascade_diag_t* ring;
  int ring_n;
  int grid_push;       // CTAs of the persistent particle kernel
  int block_push;      // threads per CTA of the particle kernel
  int grid_field;      // CTAs of the field kernel
  int variant;         // particle-kernel variant, see PushVariant
  int push_dep;        // current accumulator, see AccOf in cascade_kernels.cuh
  int push_fast;       // 1: gamma from one reciprocal square root (FP32 only)
  int push_stage;      // 1: particles staged through shared memory with cp.async (FP32)
  int fine_deposit;    // FP32: two-word accumulator (CASCADE_FP32_MIXED_FINE)
  int u_words;         // FP32: 2 = momentum as a compensated pair (u, ulo), else 1
  int prefetch;        // particle kernel: iterations ahead to prefetch into L2 (0 = off)
  int open_bc;         // 1: open boundaries (co-rotating frame runs), 0: periodic
  double j_m;          // background current in Ampere's law
  double rho_gj;       // background charge in Gauss's law (diagnostic)
  long long hole_cap;  // open boundaries: entries per species of each list below
  long long* holes[2]; // departed particle indices
  long long* hole_a[2];// holes below the new count
  long long* hole_b[2];// live particles at or above the new count
  long long min_per_cta;  // particles per active CTA before another CTA is woken
  int gauss_every;     // > 0: the step computes the Gauss residual every gauss_every steps
  double* gauss_rho;   // its charge per node times dx (nx, kept zeroed between uses)
  double* gauss_out;   // its result
};

// The part of a member's descriptor that the constant-bank batch kernel
// reads (k_batch_push_c): a table of these lives in __constant__ memory,
// indexed by blockIdx.y, so every field is a warp-uniform constant-bank
// operand instead of a per-thread register.
struct BatchMember {
  int32_t* cell[2];
  void* off[2];
  void* u[2];
  int32_t* ph_cell;
  void* ph_off;
  double* E;
  double* S_glob;
  double* uk_part;
  Ctl* ctl;
  long long cap4, ph_cap;
  double dt, dtdx, gamma_thr, eps_gamma, lpp_frac;
  int nx, lpp_int;
};

// Entries of the constant-bank member table in each kernel translation unit.
// particles per species a batch member may hold: the batched kernel indexes
// 4-particle chunks and particles of one member with 32-bit integers
constexpr long long kBatchMaxCap = 1LL << 30;
constexpr int kConstMembers = 64 * 1024 / sizeof(BatchMember) - 8;

// A batch of cascades advanced together (one launch per kernel per step).
struct BatchDev {
  const Dev* devs;               // [n] member descriptors
  long long* remaining;          // [n] steps left per member; 0 = idle or empty slot
  long long* item_start;         // [n + 1] exclusive scan of the members' work units (cost) this step
  int n;                         // slots
  int max_nx;                    // largest member grid (shared-memory sizing)
  int prefetch;                  // iterations ahead the particle kernel prefetches into L2
  long long member_cost;         // fixed cost of a member in the partition, in 4-particle chunks
  int* member_ctas;              // [n] constant-bank kernel: CTAs that work on each member this step
  int const_base;                // constant-bank kernel: the batch's first entry in the member table
  int target_ctas;               // constant-bank kernel: working CTAs the plan aims at per step
  int max_ctas;                  // constant-bank kernel: CTAs launched per member (grid x)
};

enum PushVariant {
  kSmemESmemS = 0,  // E and the charge-flux accumulator in shared memory
  kSmemEGlobS = 1,  // E in shared memory, flux through global FP64 atomics
  kGlobEGlobS = 2,  // both in global memory (very large grids)
  kGlobESmemS = 3,  // E read through L1 from global memory, accumulator in shared memory
};

constexpr int kFieldBlock = 256;

// Record the detail of a failure for cascade_last_error_message (calling thread).
void set_error_message(const char* msg);

// Kernel launchers, one set per precision (defined in kernels_fp64.cu and
// kernels_fp32.cu).  They return a cudaError_t.
#define CASCADE_DECLARE_LAUNCHERS(SUFFIX)                                                       \
  cudaError_t seed_##SUFFIX(const Dev& d, long long npairs, int ppc, unsigned long long seed,  \
                            double u_spread, cudaStream_t s);                                   \
  cudaError_t step_##SUFFIX(const Dev& d, cudaStream_t s);                                      \
  cudaError_t step_timed_##SUFFIX(const Dev& d, cudaStream_t s, cudaEvent_t before, cudaEvent_t after); \
  cudaError_t gauss_##SUFFIX(const Dev& d, double* rho_dx, double* out, cudaStream_t s);       \
  cudaError_t configure_##SUFFIX(Dev& d, int num_sms);                                         \
  cudaError_t batch_configure_##SUFFIX(int max_nx, int fine, int num_sms, int shape, int stage, int* grid, \
                                       int* block, size_t* smem, int* dep);                     \
  cudaError_t batch_step_##SUFFIX(const BatchDev& b, int grid, int block, size_t smem, int dep,   \
                                  cudaStream_t s, cudaEvent_t before = nullptr,                 \
                                  cudaEvent_t after = nullptr);                                 \
  size_t partial_bytes_##SUFFIX();                                                             \
  cudaError_t batch_member_set_##SUFFIX(int index, const BatchMember* m, cudaStream_t s);       \
  cudaError_t histogram_##SUFFIX(const Dev& d, int sp, int quantity, int nbins, double lo, double hi,    \
                                 unsigned long long* out, cudaStream_t s);                           \
  cudaError_t upload_##SUFFIX(const Dev& d, int sp, long long first, long long count, const void* off_src, \
                              const void* u_src, int src_f32, unsigned int* bad, cudaStream_t s);

CASCADE_DECLARE_LAUNCHERS(fp64)
CASCADE_DECLARE_LAUNCHERS(fp32)

}  // namespace cpic
