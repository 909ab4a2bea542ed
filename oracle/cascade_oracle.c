/*
 * cascade_oracle.c -- plain FP64 CPU reference of the pair-cascade PIC step.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the oracle the CUDA library is checked
 * against.  Only the tests, the smoke check and the benchmark's CPU-baseline leg
 * may load it.  It shares no code, header, table or helper with the CUDA path.
 *
 * What it computes (Cruz, Grismayer & Silva, arXiv:2012.05587):
 *   - Section 3 setup: a 1D periodic electron-positron plasma of density n0 per
 *     species in a uniform initial field E0, in units c = 1, omega_p = 1
 *     (omega_p^2 = 4 pi e^2 n0 / m), E in m c omega_p / e.
 *   - the particle push du/dt = q E (the force term of the Vlasov equation, Eq. 6)
 *   - a charge-conserving current deposit and Ampere's law dE/dt = -J (Eq. 4 with
 *     the 4 pi absorbed by the normalisation), so Gauss's law dE/dx = rho holds
 *     (Eq. 25 with rho_GJ = 0).
 *   - the simplified QED model of Section 2: a lepton that reaches gamma_thr
 *     emits a photon of energy eps_gamma = f gamma_thr and keeps its direction
 *     with the energy reduced (the recoil that bounds population 1 to
 *     [gamma_thr - gamma_pair, gamma_thr] in Section 3); the photon becomes an
 *     e-/e+ pair whose members share its energy equally (Section 2).  The paper
 *     converts in place; a photon flight length l_pp (converted after
 *     n_pp = ceil(l_pp / (c dt)) steps at x_emit +- l_pp) generalises it, and
 *     l_pp = 0 gives back the in-place model.
 *
 * The loop, per step n -> n+1, in this order:
 *   1. photons whose conversion step is n become pairs (appended);
 *   2. every particle, in storage order: gather E^n, push, move, deposit;
 *   3. Ampere: E^{n+1} = E^n - dt J^{n+1/2};
 *   4. every lepton, in storage order: threshold emission with recoil;
 *   5. diagnostics at n+1.
 *
 * Co-rotating frame (Section 7, Eq. 25-26): an optional background charge
 * rho_GJ enters Gauss's law, dE/dx = rho - rho_GJ, and a background current
 * j_m enters Ampere's law, dE/dt = -(J - j_m).  With open boundaries the
 * field beyond the outermost edges equals the nearest edge, a particle that
 * crosses x = 0 or x = L deposits the part of its path inside the domain and
 * is removed at the end of the step, and a photon whose conversion point
 * lies outside is not kept.
 *
 * Representation: a particle sits at x = (cell + off) dx, cell integer,
 * off in [0, 1).  E and J live on edges: E[i] = E_{i+1/2}.  The charge of a
 * particle is shared between nodes cell and cell+1 with linear (CIC) weights.
 * A particle represents w = n0 dx / ppc physical particles per unit area.
 *
 * Floating point: plain double arithmetic, evaluated in source order; build
 * with -ffp-contract=off so no multiply-add is fused.
 *
 * Multi-core build (-fopenmp, used only to time the CPU on all host cores):
 * the particle loops of step 2 and of the diagnostics run over contiguous
 * blocks of particles, one per thread; each thread sums its deposit into a
 * row of its own and the rows are added in thread order.  Photon creation,
 * emission and removal stay sequential, so every list keeps its order.  With
 * one thread the result is bit-identical to the plain build; with more, the
 * sums of J, rho and U_K change order (round-off only).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------- */
/* Parameters and per-step diagnostics (oracle's own layout).                 */
/* ------------------------------------------------------------------------- */
typedef struct {
  int32_t nx;          /* cells, periodic */
  int32_t ppc;         /* seed macro-particles per cell per species */
  double dx, dt;       /* cell size and time step (c = 1, omega_p = 1) */
  double n0;           /* seed density per species */
  double u_spread;     /* seed momenta u ~ Normal(0, u_spread) */
  uint64_t seed;       /* Philox key */
  double E0;           /* initial uniform field */
  double gamma_thr;    /* emission threshold */
  double eps_gamma;    /* photon energy (m c^2) = f gamma_thr */
  double l_pp;         /* photon flight length before conversion */
  int64_t particle_cap;/* per species */
  double j_m;          /* background current (co-rotating frame), 0 otherwise */
  double rho_gj;       /* background charge density, 0 otherwise */
  int32_t open_bc;     /* 0: periodic; 1: open boundaries */
  int32_t pad_;
} orc_params;

typedef struct {
  int64_t step;
  double t, E_mean, J_mean, E_absmax, U_E, U_K, U_gamma, gauss_resid;
  int64_t n_elec, n_posi, n_photon, n_pairs_total, n_emit_multi;
} orc_diag;

enum { ORC_OK = 0, ORC_ERR_ARG = -1, ORC_ERR_OOM = -2, ORC_ERR_CAPACITY = -3 };

typedef struct {
  orc_params p;
  double w;            /* macro-particle weight n0 dx / ppc */
  double dtdx;         /* dt / dx */
  double jscale;       /* J = jscale * (sum of q * offset change) */
  int32_t n_pp;        /* photon flight in steps */
  int32_t lpp_int;     /* floor(l_pp / dx) */
  double lpp_frac;     /* l_pp / dx - floor(l_pp / dx) */
  int64_t step;

  /* particles, one list in storage order */
  int64_t np, np_alloc;
  int32_t *cell;
  double *off, *u, *gam;
  int8_t *q;
  int64_t n_species[2]; /* [0] electrons, [1] positrons */

  /* photons in flight, in emission order */
  int64_t nph, nph_alloc;
  int64_t *ph_conv_step;
  int32_t *ph_cell;
  double *ph_off;
  int8_t *ph_dir;

  double *E, *J, *S, *rho_dx;
  double *rows;        /* multi-core build: n_rows x nx per-thread sums */
  int32_t n_rows;
  int64_t pairs_total, emit_multi;
  int error;
} orc_sim;

/* ------------------------------------------------------------------------- */
/* Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11, "Parallel random        */
/* numbers: as easy as 1, 2, 3"): 10 rounds of the 4x32 Philox S-box with     */
/* multipliers 0xD2511F53, 0xCD9E8D57 and Weyl key increments 0x9E3779B9,     */
/* 0xBB67AE85.                                                                */
/* ------------------------------------------------------------------------- */
void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
  uint32_t c[4] = {ctr_in[0], ctr_in[1], ctr_in[2], ctr_in[3]};
  uint32_t k0 = key_in[0], k1 = key_in[1];
  for (int r = 0; r < 10; ++r) {
    uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c[0];
    uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c[2];
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c[1] ^ k0;
    uint32_t n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  out[0] = c[0]; out[1] = c[1]; out[2] = c[2]; out[3] = c[3];
}

/* Seed momenta of pair j: one Philox call with counter (j, step = 0), two
 * 53-bit uniforms in (0, 1), Box-Muller.  The cosine branch goes to the
 * electron, the sine branch to the positron. */
static void seed_normals(uint64_t seed, uint64_t j, double* z_elec, double* z_posi) {
  const uint32_t ctr[4] = {(uint32_t)j, (uint32_t)(j >> 32), 0u, 0u};
  const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t r[4];
  orc_philox4x32_10(ctr, key, r);
  uint64_t a = ((uint64_t)r[0] << 32) | r[1];
  uint64_t b = ((uint64_t)r[2] << 32) | r[3];
  double u1 = ((double)(a >> 11) + 0.5) * (1.0 / 9007199254740992.0);
  double u2 = ((double)(b >> 11) + 0.5) * (1.0 / 9007199254740992.0);
  double rad = sqrt(-2.0 * log(u1));
  double ang = 6.283185307179586 * u2;
  *z_elec = rad * cos(ang);
  *z_posi = rad * sin(ang);
}

void orc_seed_normals(uint64_t seed, uint64_t j, double* ze, double* zp) { seed_normals(seed, j, ze, zp); }

/* ------------------------------------------------------------------------- */
static int32_t wrap_cell(int64_t c, int32_t nx) {
  int64_t m = c % nx;
  if (m < 0) m += nx;
  return (int32_t)m;
}

static int grow_particles(orc_sim* s, int64_t need) {
  if (need <= s->np_alloc) return 0;
  int64_t na = s->np_alloc ? s->np_alloc : 1024;
  while (na < need) na *= 2;
  int32_t* c = realloc(s->cell, (size_t)na * sizeof(int32_t));
  if (!c) return -1; s->cell = c;
  double* o = realloc(s->off, (size_t)na * sizeof(double));
  if (!o) return -1; s->off = o;
  double* u = realloc(s->u, (size_t)na * sizeof(double));
  if (!u) return -1; s->u = u;
  double* g = realloc(s->gam, (size_t)na * sizeof(double));
  if (!g) return -1; s->gam = g;
  int8_t* q = realloc(s->q, (size_t)na);
  if (!q) return -1; s->q = q;
  s->np_alloc = na;
  return 0;
}

static int grow_photons(orc_sim* s, int64_t need) {
  if (need <= s->nph_alloc) return 0;
  int64_t na = s->nph_alloc ? s->nph_alloc : 1024;
  while (na < need) na *= 2;
  int64_t* cs = realloc(s->ph_conv_step, (size_t)na * sizeof(int64_t));
  if (!cs) return -1; s->ph_conv_step = cs;
  int32_t* c = realloc(s->ph_cell, (size_t)na * sizeof(int32_t));
  if (!c) return -1; s->ph_cell = c;
  double* o = realloc(s->ph_off, (size_t)na * sizeof(double));
  if (!o) return -1; s->ph_off = o;
  int8_t* d = realloc(s->ph_dir, (size_t)na);
  if (!d) return -1; s->ph_dir = d;
  s->nph_alloc = na;
  return 0;
}

static int push_particle(orc_sim* s, int32_t cell, double off, double u, int8_t q) {
  int sp = q > 0 ? 1 : 0;
  if (s->n_species[sp] + 1 > s->p.particle_cap) { s->error = ORC_ERR_CAPACITY; return -1; }
  if (grow_particles(s, s->np + 1)) { s->error = ORC_ERR_OOM; return -1; }
  s->cell[s->np] = cell; s->off[s->np] = off; s->u[s->np] = u; s->q[s->np] = q;
  s->gam[s->np] = sqrt(1.0 + u * u);
  s->np++;
  s->n_species[sp]++;
  return 0;
}

static int validate(const orc_params* p) {
  if (p->nx < 2 || p->ppc < 1) return ORC_ERR_ARG;
  if (!(p->dx > 0) || !(p->dt > 0) || !(p->dt < p->dx)) return ORC_ERR_ARG;
  if (!(p->n0 >= 0) || !(p->u_spread >= 0) || !(p->l_pp >= 0)) return ORC_ERR_ARG;
  if (!(p->eps_gamma >= 2.0)) return ORC_ERR_ARG;                 /* pair rest mass */
  if (!(p->gamma_thr - p->eps_gamma >= 1.0)) return ORC_ERR_ARG;  /* recoil stays physical */
  if (!(p->eps_gamma / p->gamma_thr < 2.0 / 3.0)) return ORC_ERR_ARG; /* Eq. 1 delay > 0 */
  if (p->particle_cap < 1) return ORC_ERR_ARG;
  if (p->open_bc != 0 && p->open_bc != 1) return ORC_ERR_ARG;
  return ORC_OK;
}

static orc_sim* alloc_sim(const orc_params* p) {
  orc_sim* s = calloc(1, sizeof(orc_sim));
  if (!s) return NULL;
  s->p = *p;
  s->w = p->n0 * p->dx / (double)p->ppc;
  s->dtdx = p->dt / p->dx;
  s->jscale = p->n0 * p->dx / ((double)p->ppc * p->dt);
  /* photon flight in whole steps, from the flight time l_pp / c */
  s->n_pp = (int32_t)ceil(p->l_pp / p->dt - 1e-9);
  if (s->n_pp < 0) s->n_pp = 0;
  double L = p->l_pp / p->dx;
  s->lpp_int = (int32_t)floor(L);
  s->lpp_frac = L - (double)s->lpp_int;
  s->E = calloc((size_t)p->nx, sizeof(double));
  s->J = calloc((size_t)p->nx, sizeof(double));
  s->S = calloc((size_t)p->nx, sizeof(double));
  s->rho_dx = calloc((size_t)p->nx, sizeof(double));
  if (!s->E || !s->J || !s->S || !s->rho_dx) return NULL;
  for (int32_t i = 0; i < p->nx; ++i) s->E[i] = p->E0;
  return s;
}

void orc_destroy(orc_sim* s) {
  if (!s) return;
  free(s->cell); free(s->off); free(s->u); free(s->gam); free(s->q);
  free(s->ph_conv_step); free(s->ph_cell); free(s->ph_off); free(s->ph_dir);
  free(s->E); free(s->J); free(s->S); free(s->rho_dx); free(s->rows);
  free(s);
}

/* Quiet start (Section 3 setup): in every cell, ppc co-located e-/e+ pairs at
 * offsets (k + 1/2) / ppc, so rho = 0 and the uniform E0 satisfies Gauss.
 * Pair j sits in cell j mod nx with k = j div nx; its momenta come from
 * Philox(counter = (j, 0), key = seed). */
int orc_create(const orc_params* p, orc_sim** out) {
  *out = NULL;
  int rc = validate(p);
  if (rc) return rc;
  if ((int64_t)p->nx * p->ppc > p->particle_cap) return ORC_ERR_CAPACITY;
  orc_sim* s = alloc_sim(p);
  if (!s) return ORC_ERR_OOM;
  int64_t npairs = (int64_t)p->nx * p->ppc;
  if (grow_particles(s, 2 * npairs)) { orc_destroy(s); return ORC_ERR_OOM; }
  for (int64_t j = 0; j < npairs; ++j) {
    int32_t cell = (int32_t)(j % p->nx);
    int64_t k = j / p->nx;
    double off = ((double)k + 0.5) / (double)p->ppc;
    double ze, zp;
    seed_normals(p->seed, (uint64_t)j, &ze, &zp);
    push_particle(s, cell, off, p->u_spread * ze, -1);
    push_particle(s, cell, off, p->u_spread * zp, +1);
  }
  *out = s;
  return ORC_OK;
}

/* Hand-built state: n particles with explicit cell, offset, momentum, charge;
 * E on edges (NULL = uniform E0). */
int orc_create_state(const orc_params* p, int64_t n, const int32_t* cell, const double* off,
                     const double* u, const int8_t* q, const double* E_init, orc_sim** out) {
  *out = NULL;
  int rc = validate(p);
  if (rc) return rc;
  orc_sim* s = alloc_sim(p);
  if (!s) return ORC_ERR_OOM;
  for (int64_t i = 0; i < n; ++i) {
    if (cell[i] < 0 || cell[i] >= p->nx || !(off[i] >= 0.0) || !(off[i] < 1.0) || (q[i] != 1 && q[i] != -1)) {
      orc_destroy(s); return ORC_ERR_ARG;
    }
    if (push_particle(s, cell[i], off[i], u[i], q[i])) { int e = s->error; orc_destroy(s); return e; }
  }
  if (E_init) memcpy(s->E, E_init, (size_t)p->nx * sizeof(double));
  *out = s;
  return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* One step n -> n+1.                                                        */
/* ------------------------------------------------------------------------- */
static void convert_photons(orc_sim* s) {
  /* Section 2: the photon energy is split equally, gamma = eps / 2 per member,
   * both moving along the photon direction. */
  const double h = 0.5 * s->p.eps_gamma;
  const double u_pair = sqrt(h * h - 1.0);
  int64_t kept = 0;
  for (int64_t i = 0; i < s->nph; ++i) {
    if (s->ph_conv_step[i] == s->step && !s->error) {
      double ud = s->ph_dir[i] > 0 ? u_pair : -u_pair;
      if (push_particle(s, s->ph_cell[i], s->ph_off[i], ud, -1) ||
          push_particle(s, s->ph_cell[i], s->ph_off[i], ud, +1)) {
        break;
      }
      s->pairs_total++;
    } else {
      s->ph_conv_step[kept] = s->ph_conv_step[i];
      s->ph_cell[kept] = s->ph_cell[i];
      s->ph_off[kept] = s->ph_off[i];
      s->ph_dir[kept] = s->ph_dir[i];
      kept++;
    }
  }
  if (!s->error) s->nph = kept;
}

/* Step 2 for particle p: gather, push, move, and deposit into S. */
static void move_particle(orc_sim* s, int64_t p, double* S) {
  const int32_t nx = s->p.nx;
  const int open = s->p.open_bc;
  const double dt = s->p.dt, dtdx = s->dtdx;
  const double q = (double)s->q[p];
  int32_t c = s->cell[p];
  double o = s->off[p];
  /* gather: linear interpolation between the two edges bracketing x (open
   * boundaries: beyond the outermost edges the field is that edge's) */
  int32_t ia, ib;
  double w;
  if (o >= 0.5) { ia = c; ib = (c + 1 == nx) ? (open ? nx - 1 : 0) : c + 1; w = o - 0.5; }
  else          { ia = (c == 0) ? (open ? 0 : nx - 1) : c - 1; ib = c; w = o + 0.5; }
  double Ep = (1.0 - w) * s->E[ia] + w * s->E[ib];
  /* push: du/dt = q E */
  double u = s->u[p] + q * dt * Ep;
  double g = sqrt(1.0 + u * u);
  /* move: dx/dt = u / gamma, in cell units */
  double d = u / g * dtdx;
  double o2 = o + d;
  int32_t c2 = c;
  /* deposit: charge-conserving current of the CIC shape, one term per
   * sub-segment between nodes; sum q * (offset change) per edge */
  if (o2 >= 1.0) {
    S[c] += q * (1.0 - o);
    if (open && c + 1 == nx) {
      c2 = -1;  /* left through x = L: the part inside is deposited */
    } else {
      c2 = (c + 1 == nx) ? 0 : c + 1;
      o2 = o2 - 1.0;
      S[c2] += q * o2;
    }
  } else if (o2 < 0.0) {
    S[c] += q * (0.0 - o);
    if (open && c == 0) {
      c2 = -1;  /* left through x = 0 */
    } else {
      c2 = (c == 0) ? nx - 1 : c - 1;
      o2 = o2 + 1.0;
      S[c2] += q * (o2 - 1.0);
      if (o2 >= 1.0) { o2 = 0.0; c2 = c; }  /* rounding landed on the node itself */
    }
  } else {
    S[c] += q * (o2 - o);
  }
  s->cell[p] = c2;
  s->off[p] = o2;
  s->u[p] = u;
  s->gam[p] = g;
}

#ifdef _OPENMP
/* Multi-core build: n_rows x nx scratch for per-thread sums. */
static double* thread_rows(orc_sim* s) {
  int32_t nt = (int32_t)omp_get_max_threads();
  if (nt > s->n_rows) {
    free(s->rows);
    s->rows = malloc((size_t)nt * (size_t)s->p.nx * sizeof(double));
    s->n_rows = s->rows ? nt : 0;
  }
  return s->rows;
}

/* Adds the first nt rows into out, in row order. */
static void sum_rows(const orc_sim* s, int32_t nt, double* out) {
  for (int32_t i = 0; i < s->p.nx; ++i) out[i] = 0.0;
  for (int32_t t = 0; t < nt; ++t)
    for (int32_t i = 0; i < s->p.nx; ++i) out[i] += s->rows[(size_t)t * s->p.nx + i];
}
#endif

static void push_move_deposit(orc_sim* s) {
  const int32_t nx = s->p.nx;
#ifdef _OPENMP
  if (thread_rows(s)) {
    int32_t nt = 1;
#pragma omp parallel
    {
      double* S = s->rows + (size_t)omp_get_thread_num() * nx;
      for (int32_t i = 0; i < nx; ++i) S[i] = 0.0;
#pragma omp single
      nt = (int32_t)omp_get_num_threads();
#pragma omp for schedule(static)
      for (int64_t p = 0; p < s->np; ++p) move_particle(s, p, S);
    }
    sum_rows(s, nt, s->S);
    return;
  }
#endif
  for (int32_t i = 0; i < nx; ++i) s->S[i] = 0.0;
  for (int64_t p = 0; p < s->np; ++p) move_particle(s, p, s->S);
}

/* Open boundaries: particles that left (cell -1) are removed, keeping the
 * storage order of the rest. */
static void remove_departed(orc_sim* s) {
  int64_t k = 0;
  for (int64_t p = 0; p < s->np; ++p) {
    if (s->cell[p] < 0) {
      s->n_species[s->q[p] > 0 ? 1 : 0]--;
      continue;
    }
    s->cell[k] = s->cell[p]; s->off[k] = s->off[p]; s->u[k] = s->u[p];
    s->gam[k] = s->gam[p]; s->q[k] = s->q[p];
    k++;
  }
  s->np = k;
}

/* Ampere: dE/dt = -(J - j_m) (Eq. 26; j_m = 0 outside the co-rotating frame). */
static void ampere(orc_sim* s) {
  const double dt = s->p.dt;
  for (int32_t i = 0; i < s->p.nx; ++i) {
    s->J[i] = s->jscale * s->S[i];
    s->E[i] = s->E[i] - dt * (s->J[i] - s->p.j_m);
  }
}

static void qed_emission(orc_sim* s) {
  const double thr = s->p.gamma_thr, eps = s->p.eps_gamma;
  const int64_t conv = s->step + 1 + s->n_pp;
  for (int64_t p = 0; p < s->np; ++p) {
    double g = s->gam[p];
    if (!(g >= thr)) continue;
    int64_t k = 1 + (int64_t)floor((g - thr) / eps);
    double g2 = g - (double)k * eps;
    double sgn = s->u[p] > 0.0 ? 1.0 : -1.0;
    s->u[p] = sgn * sqrt(g2 * g2 - 1.0);
    s->gam[p] = g2;
    if (k > 1) s->emit_multi++;
    /* conversion point x + dir * l_pp, wrapped (open boundaries: a photon
     * that would convert outside the domain is not kept) */
    int32_t cc;
    double oc;
    int64_t ci;
    if (sgn > 0) {
      oc = s->off[p] + s->lpp_frac;
      ci = (int64_t)s->cell[p] + s->lpp_int;
      if (oc >= 1.0) { oc = oc - 1.0; ci += 1; }
    } else {
      oc = s->off[p] - s->lpp_frac;
      ci = (int64_t)s->cell[p] - s->lpp_int;
      if (oc < 0.0) { oc = oc + 1.0; ci -= 1; if (oc >= 1.0) { oc = 0.0; ci += 1; } }
    }
    if (s->p.open_bc && (ci < 0 || ci >= s->p.nx)) continue;
    cc = wrap_cell(ci, s->p.nx);
    if (grow_photons(s, s->nph + k)) { s->error = ORC_ERR_OOM; return; }
    for (int64_t m = 0; m < k; ++m) {
      s->ph_conv_step[s->nph] = conv;
      s->ph_cell[s->nph] = cc;
      s->ph_off[s->nph] = oc;
      s->ph_dir[s->nph] = (int8_t)(sgn > 0 ? 1 : -1);
      s->nph++;
    }
  }
}

/* CIC charge of particle p into rho_dx (node cell and cell + 1). */
static void particle_charge(const orc_sim* s, int64_t p, double* rho_dx) {
  const int32_t nx = s->p.nx;
  int32_t c = s->cell[p];
  double qw = (double)s->q[p] * s->w;
  rho_dx[c] += qw * (1.0 - s->off[p]);
  if (c + 1 < nx) rho_dx[c + 1] += qw * s->off[p];
  else if (!s->p.open_bc) rho_dx[0] += qw * s->off[p];  /* periodic node nx = node 0 */
}

static void charge_density(orc_sim* s) {
  const int32_t nx = s->p.nx;
#ifdef _OPENMP
  if (thread_rows(s)) {
    int32_t nt = 1;
#pragma omp parallel
    {
      double* R = s->rows + (size_t)omp_get_thread_num() * nx;
      for (int32_t i = 0; i < nx; ++i) R[i] = 0.0;
#pragma omp single
      nt = (int32_t)omp_get_num_threads();
#pragma omp for schedule(static)
      for (int64_t p = 0; p < s->np; ++p) particle_charge(s, p, R);
    }
    sum_rows(s, nt, s->rho_dx);
    return;
  }
#endif
  for (int32_t i = 0; i < nx; ++i) s->rho_dx[i] = 0.0;
  for (int64_t p = 0; p < s->np; ++p) particle_charge(s, p, s->rho_dx);
}

static void diagnostics(orc_sim* s, orc_diag* d) {
  const int32_t nx = s->p.nx;
  double se = 0, sj = 0, amax = 0, ue = 0, uk = 0, gres = 0;
  for (int32_t i = 0; i < nx; ++i) {
    se += s->E[i];
    sj += s->J[i];
    double a = fabs(s->E[i]);
    if (a > amax) amax = a;
    ue += 0.5 * s->E[i] * s->E[i] * s->p.dx;
  }
#ifdef _OPENMP
#pragma omp parallel for schedule(static) reduction(+ : uk)
#endif
  for (int64_t p = 0; p < s->np; ++p) uk += s->w * s->gam[p];
  /* Gauss on node i between edges i-1/2 and i+1/2: E[i] - E[i-1] =
   * dx (rho_i - rho_GJ); with open boundaries only the interior nodes */
  charge_density(s);
  for (int32_t i = s->p.open_bc ? 1 : 0; i < nx; ++i) {
    int32_t im = (i == 0) ? nx - 1 : i - 1;
    double r = fabs(s->E[i] - s->E[im] - (s->rho_dx[i] - s->p.rho_gj * s->p.dx));
    if (r > gres) gres = r;
  }
  d->step = s->step;
  d->t = (double)s->step * s->p.dt;
  d->E_mean = se / nx;
  d->J_mean = sj / nx;
  d->E_absmax = amax;
  d->U_E = ue;
  d->U_K = uk;
  d->U_gamma = (double)s->nph * s->w * s->p.eps_gamma;
  d->gauss_resid = gres;
  d->n_elec = s->n_species[0];
  d->n_posi = s->n_species[1];
  d->n_photon = s->nph;
  d->n_pairs_total = s->pairs_total;
  d->n_emit_multi = s->emit_multi;
}

int orc_step(orc_sim* s, int32_t nsteps, orc_diag* out) {
  for (int32_t k = 0; k < nsteps; ++k) {
    if (s->error) return s->error;
    convert_photons(s);
    if (s->error) return s->error;
    push_move_deposit(s);
    if (s->p.open_bc) remove_departed(s);
    ampere(s);
    qed_emission(s);
    if (s->error) return s->error;
    s->step++;
    if (out) diagnostics(s, &out[k]);
  }
  return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Accessors.                                                                */
/* ------------------------------------------------------------------------- */
int64_t orc_num_particles(const orc_sim* s) { return s->np; }
int64_t orc_num_photons(const orc_sim* s) { return s->nph; }
int32_t orc_n_pp(const orc_sim* s) { return s->n_pp; }
int64_t orc_step_index(const orc_sim* s) { return s->step; }

void orc_get_fields(const orc_sim* s, double* E, double* J) {
  if (E) memcpy(E, s->E, (size_t)s->p.nx * sizeof(double));
  if (J) memcpy(J, s->J, (size_t)s->p.nx * sizeof(double));
}

void orc_get_particles(const orc_sim* s, int32_t* cell, double* off, double* u, int8_t* q) {
  for (int64_t p = 0; p < s->np; ++p) {
    if (cell) cell[p] = s->cell[p];
    if (off) off[p] = s->off[p];
    if (u) u[p] = s->u[p];
    if (q) q[p] = s->q[p];
  }
}

void orc_get_photons(const orc_sim* s, int64_t* conv_step, int32_t* cell, double* off, int8_t* dir) {
  for (int64_t i = 0; i < s->nph; ++i) {
    if (conv_step) conv_step[i] = s->ph_conv_step[i];
    if (cell) cell[i] = s->ph_cell[i];
    if (off) off[i] = s->ph_off[i];
    if (dir) dir[i] = s->ph_dir[i];
  }
}

/* Current diagnostics without stepping (state at the present step). */
void orc_diag_now(orc_sim* s, orc_diag* d) { diagnostics(s, d); }

/* Threads the particle loops use: 1 in the plain build. */
int32_t orc_threads(void) {
#ifdef _OPENMP
  return (int32_t)omp_get_max_threads();
#else
  return 1;
#endif
}

/* Multi-core build: sets the thread count (no effect in the plain build). */
void orc_set_threads(int32_t n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}
