/*
 * polyrx oracle: plain FP64 CPU restatement of de Buyl & Nies,
 * "A parallel algorithm for step- and chain-growth polymerization in
 * Molecular Dynamics" (arXiv:1409.7498).
 *
 * TEST INFRASTRUCTURE ONLY: the test suite, the package smoke check and the
 * CPU-baseline leg of the benchmark are its only users.  It shares no code,
 * header, table or helper with the CUDA path.
 *
 * Everything here is written for a reader checking it against the paper:
 * no blocking, no fusion, no reordering beyond what each definition states.
 * Compile with -ffp-contract=off so that every product and sum is rounded
 * exactly as written; fused multiply-adds appear only where fma() is called.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------
 * Philox4x32-10, the counter-based generator of Salmon, Moraes, Dror and
 * Shaw, "Parallel random numbers: as easy as 1, 2, 3" (SC'11).  One round
 * multiplies counter words 0 and 2 by the two round multipliers, swaps the
 * halves and xors in the round key; the key is bumped by the two Weyl
 * constants between rounds.  Ten rounds.
 * ---------------------------------------------------------------------- */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += W0;
      k1 += W1;
    }
    uint64_t p0 = (uint64_t)M0 * (uint64_t)c0;
    uint64_t p1 = (uint64_t)M1 * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Uniform in [0,1) with 53 random bits: the top 53 bits of (hi:lo) times
 * 2^-53.  Every value is exactly representable in double. */
double orc_u53(uint32_t hi, uint32_t lo) {
  uint64_t w = ((uint64_t)hi << 32) | (uint64_t)lo;
  return (double)(w >> 11) * 0x1.0p-53;
}

/* Uniform in [0,1) with 24 random bits (exact in float and double). */
double orc_u24(uint32_t w) { return (double)(w >> 8) * 0x1.0p-24; }

/* Counter layout shared by every keyed draw: word 0 = low 32 bits of the
 * step, words 1 and 2 = the particle ids, word 3 = tag | (step >> 32) << 8. */
static void draw(uint64_t seed, int64_t step, uint32_t a, uint32_t b, uint32_t tag,
                 uint32_t out[4]) {
  uint64_t s = (uint64_t)step;
  uint32_t ctr[4] = {(uint32_t)s, a, b, tag | ((uint32_t)(s >> 32) << 8)};
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  orc_philox4x32_10(ctr, key, out);
}

/* ------------------------------------------------------------------------
 * Geometry helpers
 * ---------------------------------------------------------------------- */

/* Minimum image of one separation component by compare-and-shift. */
static double min_image(double d, double L) {
  double half = 0.5 * L;
  if (d > half) return d - L;
  if (d < -half) return d + L;
  return d;
}

/* r_ij = x_j - x_i under the minimum image (j relative to i). */
static void separation(const double* x, int64_t i, int64_t j, const double L[3], double d[3]) {
  for (int k = 0; k < 3; ++k) d[k] = min_image(x[3 * j + k] - x[3 * i + k], L[k]);
}

/* Squared distance in the fixed order used for the reaction test:
 * fma(dz, dz, fma(dy, dy, dx*dx)). */
static double dist2_fixed(const double d[3]) {
  return fma(d[2], d[2], fma(d[1], d[1], d[0] * d[0]));
}

/* A plain linked-cell list: every cell is at least `rcut` wide, so any pair
 * closer than rcut sits in the same or an adjacent cell.  Used only when
 * each box edge holds at least three cells; otherwise callers fall back to
 * the all-pairs loop. */
typedef struct {
  int nc[3];
  int64_t* head;
  int64_t* next;
} cells_t;

static int cells_build(const orc_system* s, const double L[3], double rcut, cells_t* c) {
  c->head = NULL;
  c->next = NULL;
  for (int k = 0; k < 3; ++k) {
    c->nc[k] = (int)floor(L[k] / (rcut * (1.0 + 1e-9)));
    if (c->nc[k] < 3) return 0;
  }
  int64_t ncell = (int64_t)c->nc[0] * c->nc[1] * c->nc[2];
  c->head = (int64_t*)malloc(sizeof(int64_t) * (size_t)ncell);
  c->next = (int64_t*)malloc(sizeof(int64_t) * (size_t)(s->n > 0 ? s->n : 1));
  if (!c->head || !c->next) {
    free(c->head);
    free(c->next);
    c->head = c->next = NULL;
    return -1;
  }
  for (int64_t q = 0; q < ncell; ++q) c->head[q] = -1;
  for (int64_t i = s->n - 1; i >= 0; --i) {
    int cc[3];
    for (int k = 0; k < 3; ++k) {
      int v = (int)floor(s->x[3 * i + k] / L[k] * c->nc[k]);
      if (v < 0) v = 0;
      if (v >= c->nc[k]) v = c->nc[k] - 1;
      cc[k] = v;
    }
    int64_t q = ((int64_t)cc[2] * c->nc[1] + cc[1]) * c->nc[0] + cc[0];
    c->next[i] = c->head[q];
    c->head[q] = i;
  }
  return 1;
}

static void cells_free(cells_t* c) {
  free(c->head);
  free(c->next);
}

static int64_t cell_of(const cells_t* c, const double* x, const double L[3], int cc[3]) {
  for (int k = 0; k < 3; ++k) {
    int v = (int)floor(x[k] / L[k] * c->nc[k]);
    if (v < 0) v = 0;
    if (v >= c->nc[k]) v = c->nc[k] - 1;
    cc[k] = v;
  }
  return ((int64_t)cc[2] * c->nc[1] + cc[1]) * c->nc[0] + cc[0];
}

/* Calls visit(j) for every particle j != i that may lie within the cell
 * list's cutoff of i (all particles when `c` is NULL). */
typedef void (*visit_fn)(int64_t i, int64_t j, void* ctx);

static void for_each_neighbor(const orc_system* s, const cells_t* c, const double L[3],
                              int64_t i, visit_fn visit, void* ctx) {
  if (!c) {
    for (int64_t j = 0; j < s->n; ++j)
      if (j != i) visit(i, j, ctx);
    return;
  }
  int cc[3];
  cell_of(c, &s->x[3 * i], L, cc);
  for (int dz = -1; dz <= 1; ++dz)
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx) {
        int qx = (cc[0] + dx + c->nc[0]) % c->nc[0];
        int qy = (cc[1] + dy + c->nc[1]) % c->nc[1];
        int qz = (cc[2] + dz + c->nc[2]) % c->nc[2];
        int64_t q = ((int64_t)qz * c->nc[1] + qy) * c->nc[0] + qx;
        for (int64_t j = c->head[q]; j >= 0; j = c->next[j])
          if (j != i) visit(i, j, ctx);
      }
}

/* ------------------------------------------------------------------------
 * Potentials (Sec. II.C)
 * ---------------------------------------------------------------------- */

/* Cutoff of the truncated and shifted LJ (WCA): sigma_c = 2^(1/6) sigma,
 * where the shifted potential of Eq. 15 reaches zero with zero slope. */
static double wca_cutoff(const orc_md_params* md) { return pow(2.0, 1.0 / 6.0) * md->sigma; }

/* Eq. 15: V = 4 eps ((s/r)^12 - (s/r)^6 + 1/4) for r < sigma_c, else 0.
 * Returns V and writes the magnitude factor g with F_i = -g * r_ij
 * (r_ij = x_j - x_i), i.e. g = -(dV/dr)/r. */
static double wca_pair(double r2, const orc_md_params* md, double* g) {
  double rc = wca_cutoff(md);
  if (r2 >= rc * rc) {
    *g = 0.0;
    return 0.0;
  }
  double sr2 = md->sigma * md->sigma / r2;
  double sr6 = sr2 * sr2 * sr2;
  double sr12 = sr6 * sr6;
  double V = 4.0 * md->eps * (sr12 - sr6 + 0.25);
  /* -dV/dr = 24 eps (2 sr12 - sr6) / r */
  double minus_dVdr_over_r = 24.0 * md->eps * (2.0 * sr12 - sr6) / r2;
  if (md->force_cap > 0.0) {
    double r = sqrt(r2);
    double fmag = minus_dVdr_over_r * r;
    if (fmag > md->force_cap) minus_dVdr_over_r = md->force_cap / r;
  }
  *g = minus_dVdr_over_r;
  return V;
}

/* FENE, Sec. II.C: V = -1/2 k R0^2 ln(1 - (r/R0)^2).
 * -dV/dr / r = -k / (1 - r^2/R0^2). */
static int fene_pair(double r2, const orc_md_params* md, double* V, double* g) {
  double R02 = md->fene_r0 * md->fene_r0;
  if (!(r2 < R02)) return ORC_EOVERSTRETCH;
  double q = 1.0 - r2 / R02;
  *V = -0.5 * md->fene_k * R02 * log(q);
  *g = -md->fene_k / q;
  return ORC_OK;
}

/* Mirror LJ, Eq. 17: V_b(r) = V_LJ(2 sigma_c - r) for sigma_c < r < 2 sigma_c,
 * else 0.  With s = 2 sigma_c - r, dV_b/dr = 24 eps (2 (sigma/s)^12 -
 * (sigma/s)^6) / s. */
static void mirror_lj_pair(double r2, const orc_md_params* md, double* V, double* g) {
  double rc = wca_cutoff(md);
  double r = sqrt(r2);
  if (!(r > rc && r < 2.0 * rc)) {
    *V = 0.0;
    *g = 0.0;
    return;
  }
  double sd = 2.0 * rc - r;
  double ss2 = md->sigma * md->sigma / (sd * sd);
  double ss6 = ss2 * ss2 * ss2;
  double ss12 = ss6 * ss6;
  *V = 4.0 * md->eps * (ss12 - ss6 + 0.25);
  double dVdr = 24.0 * md->eps * (2.0 * ss12 - ss6) / sd;
  *g = -dVdr / r;
}

/* ------------------------------------------------------------------------
 * Conservative forces: WCA on every pair (no exclusions, Kremer-Grest
 * convention) plus the bond potential on every bond.
 * ---------------------------------------------------------------------- */
typedef struct {
  const orc_system* s;
  const orc_md_params* md;
  double* f;
  double epot2; /* pair energy counted from both sides */
} force_ctx;

static void force_visit(int64_t i, int64_t j, void* vctx) {
  force_ctx* ctx = (force_ctx*)vctx;
  double d[3];
  separation(ctx->s->x, i, j, ctx->md->L, d);
  double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
  double g;
  double V = wca_pair(r2, ctx->md, &g);
  /* F_i = -dV/dr * (x_i - x_j)/r = g * (x_i - x_j) = -g * d */
  for (int k = 0; k < 3; ++k) ctx->f[3 * i + k] -= g * d[k];
  ctx->epot2 += V;
}

int orc_forces(const orc_system* s, const orc_md_params* md, int use_cells, double* f,
               double* epot) {
  if (!s || !md || !f) return ORC_EINVAL;
  for (int64_t q = 0; q < 3 * s->n; ++q) f[q] = 0.0;
  force_ctx ctx = {s, md, f, 0.0};
  cells_t cl;
  int have = 0;
  if (use_cells) {
    have = cells_build(s, md->L, wca_cutoff(md), &cl);
    if (have < 0) return ORC_ENOMEM;
  }
  for (int64_t i = 0; i < s->n; ++i) for_each_neighbor(s, have ? &cl : NULL, md->L, i, force_visit, &ctx);
  if (have) cells_free(&cl);
  double ebond2 = 0.0;
  for (int64_t i = 0; i < s->n; ++i) {
    for (int b = 0; b < s->nadj[i]; ++b) {
      int64_t j = s->adj[(int64_t)s->cap * i + b];
      double d[3];
      separation(s->x, i, j, md->L, d);
      double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
      double V = 0.0, g = 0.0;
      if (s->adj_style[(int64_t)s->cap * i + b] == ORC_BOND_MIRROR_LJ) {
        mirror_lj_pair(r2, md, &V, &g);
      } else {
        int rc = fene_pair(r2, md, &V, &g);
        if (rc) return rc;
      }
      for (int k = 0; k < 3; ++k) f[3 * i + k] -= g * d[k];
      ebond2 += V;
    }
  }
  if (epot) *epot = 0.5 * ctx.epot2 + 0.5 * ebond2;
  return ORC_OK;
}

/* ------------------------------------------------------------------------
 * One MD step.  Velocity Verlet (Sec. II.C) with a Langevin thermostat
 * written in its kick-drift form, the half-step velocity being the stored
 * velocity:
 *   F      = F_c(x) - gamma m v + R,   R_k = sqrt(24 gamma kT m / dt)(u_k - 1/2)
 *   v_new  = v + (dt/m) F
 *   x_new  = x + dt v_new          (then wrapped into [0, L))
 * u_k is a 24-bit uniform from Philox keyed by (seed, step, id), so the
 * random force has variance 2 gamma kT m / dt.  With gamma = 0 this is plain
 * velocity Verlet.  `ke_full` (optional) receives the kinetic energy of the
 * full-step velocities (v + v_new)/2.
 * ---------------------------------------------------------------------- */
int orc_step(orc_system* s, const orc_md_params* md, int use_cells, double* ke_full) {
  if (!s || !md) return ORC_EINVAL;
  int64_t step = s->step + 1;
  double* f = (double*)malloc(sizeof(double) * (size_t)(3 * (s->n > 0 ? s->n : 1)));
  if (!f) return ORC_ENOMEM;
  int rc = orc_forces(s, md, use_cells, f, NULL);
  if (rc) {
    free(f);
    return rc;
  }
  double cR = sqrt(24.0 * md->gamma * md->kT * md->mass / md->dt);
  double ke = 0.0;
  for (int64_t i = 0; i < s->n; ++i) {
    double R[3] = {0.0, 0.0, 0.0};
    if (md->gamma > 0.0) {
      uint32_t w[4];
      draw(md->seed, step, (uint32_t)i, 0u, ORC_TAG_THERMO, w);
      for (int k = 0; k < 3; ++k) R[k] = cR * (orc_u24(w[k]) - 0.5);
    }
    for (int k = 0; k < 3; ++k) {
      double v = s->v[3 * i + k];
      double F = f[3 * i + k] - md->gamma * md->mass * v + R[k];
      double vn = v + (md->dt / md->mass) * F;
      double vf = 0.5 * (v + vn);
      ke += 0.5 * md->mass * vf * vf;
      double xn = s->x[3 * i + k] + md->dt * vn;
      if (xn >= md->L[k]) xn -= md->L[k];
      if (xn < 0.0) xn += md->L[k];
      if (!isfinite(xn) || !isfinite(vn)) {
        free(f);
        return ORC_ENONFINITE;
      }
      s->v[3 * i + k] = vn;
      s->x[3 * i + k] = xn;
    }
  }
  free(f);
  s->step = step;
  if (ke_full) *ke_full = ke;
  return ORC_OK;
}

/* ------------------------------------------------------------------------
 * Reaction step: Table I of Sec. III, steps 1-9, on one process (the three
 * communication steps Pi have nothing to exchange).
 * ---------------------------------------------------------------------- */
static int eligible_A(const orc_system* s, const orc_rx_params* rx, int64_t i) {
  return ((rx->mask_A >> s->type[i]) & 1u) && s->state[i] >= rx->a_lo && s->state[i] <= rx->a_hi;
}
static int eligible_T(const orc_system* s, const orc_rx_params* rx, int64_t i) {
  return ((rx->mask_T >> s->type[i]) & 1u) && s->state[i] >= rx->t_lo && s->state[i] <= rx->t_hi;
}
static int bonded(const orc_system* s, int64_t i, int64_t j) {
  for (int b = 0; b < s->nadj[i]; ++b)
    if (s->adj[(int64_t)s->cap * i + b] == (uint32_t)j) return 1;
  return 0;
}

int orc_check_reaction(const orc_rx_params* rx) {
  if (!rx) return ORC_EINVAL;
  if (rx->a_lo > rx->a_hi || rx->t_lo > rx->t_hi) return ORC_EINVAL;
  if (rx->theta < 1 || !(rx->k >= 0.0) || !(rx->r_react > 0.0)) return ORC_EINVAL;
  if (rx->bond_style != ORC_BOND_FENE && rx->bond_style != ORC_BOND_MIRROR_LJ) return ORC_EINVAL;
  if (rx->selection != ORC_SELECT_RANDOM && rx->selection != ORC_SELECT_NEAREST) return ORC_EINVAL;
  if ((rx->mask_A | rx->mask_T) >> 8) return ORC_EINVAL;
  /* A particle may not be eligible as A and as T at once: for a type in
   * both masks the two state windows must be disjoint. */
  if ((rx->mask_A & rx->mask_T) && !(rx->a_hi < rx->t_lo || rx->t_hi < rx->a_lo)) return ORC_EINVAL;
  return ORC_OK;
}

typedef struct {
  uint32_t a, t;
  uint64_t key;
} pair_t;

static int cmp_by_a(const void* p, const void* q) {
  const pair_t* x = (const pair_t*)p;
  const pair_t* y = (const pair_t*)q;
  if (x->a != y->a) return x->a < y->a ? -1 : 1;
  if (x->t != y->t) return x->t < y->t ? -1 : 1;
  return 0;
}
static int cmp_by_t(const void* p, const void* q) {
  const pair_t* x = (const pair_t*)p;
  const pair_t* y = (const pair_t*)q;
  if (x->t != y->t) return x->t < y->t ? -1 : 1;
  if (x->a != y->a) return x->a < y->a ? -1 : 1;
  return 0;
}

typedef struct {
  const orc_system* s;
  const orc_md_params* md;
  const orc_rx_params* rx;
  double p, rr2;
  int64_t step;
  pair_t* list;
  int64_t nlist, caplist;
  int64_t candidates;
  int oom;
} find_ctx;

/* Steps 1 and 2 for one (A = i, T = j) pair. */
static void find_visit(int64_t i, int64_t j, void* vctx) {
  find_ctx* c = (find_ctx*)vctx;
  if (!eligible_T(c->s, c->rx, j)) return;
  if (bonded(c->s, i, j)) return;
  double d[3];
  separation(c->s->x, i, j, c->md->L, d);
  if (!(dist2_fixed(d) < c->rr2)) return;
  c->candidates++;
  uint32_t w[4];
  draw(c->md->seed, c->step, (uint32_t)i, (uint32_t)j, ORC_TAG_ACCEPT, w);
  if (!(orc_u53(w[0], w[1]) < c->p)) return; /* Eq. 4 */
  if (c->nlist == c->caplist) {
    int64_t nc = c->caplist ? 2 * c->caplist : 1024;
    pair_t* nl = (pair_t*)realloc(c->list, sizeof(pair_t) * (size_t)nc);
    if (!nl) {
      c->oom = 1;
      return;
    }
    c->list = nl;
    c->caplist = nc;
  }
  c->list[c->nlist].a = (uint32_t)i;
  c->list[c->nlist].t = (uint32_t)j;
  c->list[c->nlist].key = 0;
  c->nlist++;
}

/* Step 9 for the final pairs, in ascending id of A: both adjacency rows,
 * the bond list, and the state shifts delta_A and delta_T (Eq. 2). */
static int add_bonds(orc_system* s, const orc_rx_params* rx, const pair_t* list, int64_t nfin,
                     int64_t step) {
  int status = ORC_OK;
  for (int64_t q = 0; q < nfin; ++q) {
    uint32_t a = list[q].a, t = list[q].t;
    int capA = s->cap < rx->max_valence[s->type[a] & 7] ? s->cap : rx->max_valence[s->type[a] & 7];
    int capT = s->cap < rx->max_valence[s->type[t] & 7] ? s->cap : rx->max_valence[s->type[t] & 7];
    if (s->nadj[a] >= capA || s->nadj[t] >= capT || s->nb >= s->nb_cap) {
      status = ORC_ECAPACITY;
      continue;
    }
    s->adj[(int64_t)s->cap * a + s->nadj[a]] = t;
    s->adj_style[(int64_t)s->cap * a + s->nadj[a]] = (uint8_t)rx->bond_style;
    s->nadj[a]++;
    s->adj[(int64_t)s->cap * t + s->nadj[t]] = a;
    s->adj_style[(int64_t)s->cap * t + s->nadj[t]] = (uint8_t)rx->bond_style;
    s->nadj[t]++;
    s->bond_a[s->nb] = a;
    s->bond_t[s->nb] = t;
    s->bond_step[s->nb] = step;
    s->bond_style[s->nb] = (uint8_t)rx->bond_style;
    s->nb++;
    s->state[a] = (int8_t)(s->state[a] + rx->dA);
    s->state[t] = (int8_t)(s->state[t] + rx->dT);
  }
  return status;
}

/* Nearest-partner search of the LAMMPS rule: for particle i (an A when
 * want_T, else a T), the eligible partner j of the other kind within the
 * reaction cutoff, not bonded to i, of smallest r^2 (ties to the smaller
 * id). */
typedef struct {
  const orc_system* s;
  const orc_md_params* md;
  const orc_rx_params* rx;
  double rr2;
  int want_T;
  int64_t best;
  double best_r2;
  int64_t in_range;
} nearest_ctx;

static void nearest_visit(int64_t i, int64_t j, void* vctx) {
  nearest_ctx* c = (nearest_ctx*)vctx;
  if (c->want_T ? !eligible_T(c->s, c->rx, j) : !eligible_A(c->s, c->rx, j)) return;
  if (bonded(c->s, i, j)) return;
  double d[3];
  separation(c->s->x, i, j, c->md->L, d);
  const double r2 = dist2_fixed(d);
  if (!(r2 < c->rr2)) return;
  c->in_range++;
  if (c->best < 0 || r2 < c->best_r2 || (r2 == c->best_r2 && j < c->best)) {
    c->best = j;
    c->best_r2 = r2;
  }
}

/* The LAMMPS fix bond/create selection (Sec. IV.A): every eligible A records
 * its nearest eligible T and every eligible T its nearest eligible A; a pair
 * whose two particles picked each other is a candidate, and it reacts when
 * u < k dt Theta, the draw keyed by the pair's ids with the smaller first
 * (the probability is evaluated on the particle of lowest identifier). */
static int react_nearest(orc_system* s, const orc_md_params* md, const orc_rx_params* rx,
                         int use_cells, int64_t step, orc_rx_trace* trace) {
  const double p = rx->k * md->dt * (double)rx->theta;
  const double rr2 = rx->r_react * rx->r_react;
  int64_t* near = (int64_t*)malloc(sizeof(int64_t) * (size_t)(s->n ? s->n : 1));
  pair_t* list = (pair_t*)malloc(sizeof(pair_t) * (size_t)(s->n ? s->n : 1));
  if (!near || !list) {
    free(near);
    free(list);
    return ORC_ENOMEM;
  }
  cells_t cl;
  int have = 0;
  if (use_cells) {
    have = cells_build(s, md->L, rx->r_react, &cl);
    if (have < 0) {
      free(near);
      free(list);
      return ORC_ENOMEM;
    }
  }
  int64_t in_range = 0;
  for (int64_t i = 0; i < s->n; ++i) {
    near[i] = -1;
    const int isA = eligible_A(s, rx, i), isT = eligible_T(s, rx, i);
    if (!isA && !isT) continue;
    nearest_ctx c = {s, md, rx, rr2, isA, -1, 0.0, 0};
    for_each_neighbor(s, have ? &cl : NULL, md->L, i, nearest_visit, &c);
    near[i] = c.best;
    if (isA) in_range += c.in_range; /* every (A, T) pair in range, counted once */
  }
  if (have) cells_free(&cl);
  int64_t mutual = 0, accepted = 0;
  for (int64_t a = 0; a < s->n; ++a) {
    if (!eligible_A(s, rx, a) || near[a] < 0) continue;
    const int64_t t = near[a];
    if (near[t] != a) continue;
    mutual++;
    const uint32_t lo = (uint32_t)(a < t ? a : t), hi = (uint32_t)(a < t ? t : a);
    uint32_t w[4];
    draw(md->seed, step, lo, hi, ORC_TAG_NEAREST, w);
    if (!(orc_u53(w[0], w[1]) < p)) continue; /* Eq. 4 */
    list[accepted].a = (uint32_t)a;
    list[accepted].t = (uint32_t)t;
    list[accepted].key = 0;
    accepted++;
  }
  free(near);
  const int status = add_bonds(s, rx, list, accepted, step);
  if (trace) {
    trace->candidates = in_range;
    trace->retained = mutual;
    trace->a_winners = accepted;
    trace->formed = accepted;
  }
  free(list);
  return status;
}

int orc_react(orc_system* s, const orc_md_params* md, const orc_rx_params* rx, int use_cells,
              int64_t step, orc_rx_trace* trace) {
  if (!s || !md) return ORC_EINVAL;
  int rc = orc_check_reaction(rx);
  if (rc) return rc;
  if (rx->selection == ORC_SELECT_NEAREST) return react_nearest(s, md, rx, use_cells, step, trace);
  find_ctx c;
  memset(&c, 0, sizeof(c));
  c.s = s;
  c.md = md;
  c.rx = rx;
  c.p = rx->k * md->dt * (double)rx->theta; /* acceptance probability, Eqs. 3-4 */
  c.rr2 = rx->r_react * rx->r_react;
  c.step = step;

  /* Steps 1-2: every eligible (A, T) pair within the reaction cutoff that
   * is not already bonded, retained when u < k dt Theta. */
  cells_t cl;
  int have = 0;
  if (use_cells) {
    have = cells_build(s, md->L, rx->r_react, &cl);
    if (have < 0) return ORC_ENOMEM;
  }
  for (int64_t i = 0; i < s->n; ++i)
    if (eligible_A(s, rx, i)) for_each_neighbor(s, have ? &cl : NULL, md->L, i, find_visit, &c);
  if (have) cells_free(&cl);
  if (c.oom) {
    free(c.list);
    return ORC_ENOMEM;
  }

  /* Step 3: L_A, the retained pairs ordered by id_A. */
  qsort(c.list, (size_t)c.nlist, sizeof(pair_t), cmp_by_a);

  /* Step 5: one T per A, chosen uniformly at random: the smallest of the
   * keys Philox(step, id_A, id_T), ties to the smaller id_T. */
  int64_t nwin = 0;
  for (int64_t q = 0; q < c.nlist;) {
    int64_t e = q;
    int64_t best = -1;
    uint64_t bestkey = 0;
    while (e < c.nlist && c.list[e].a == c.list[q].a) {
      uint32_t w[4];
      draw(md->seed, step, c.list[e].a, c.list[e].t, ORC_TAG_SEL_A, w);
      uint64_t key = ((uint64_t)w[0] << 32) | w[1];
      if (best < 0 || key < bestkey || (key == bestkey && c.list[e].t < c.list[best].t)) {
        best = e;
        bestkey = key;
      }
      ++e;
    }
    c.list[nwin++] = c.list[best];
    q = e;
  }

  /* Step 6: L_T, the A winners ordered by id_T. */
  qsort(c.list, (size_t)nwin, sizeof(pair_t), cmp_by_t);

  /* Step 7: one A per T, chosen uniformly at random among the A's that
   * picked it: the smallest key Philox(step, id_T, id_A), ties to the
   * smaller id_A. */
  int64_t nfin = 0;
  for (int64_t q = 0; q < nwin;) {
    int64_t e = q;
    int64_t best = -1;
    uint64_t bestkey = 0;
    while (e < nwin && c.list[e].t == c.list[q].t) {
      uint32_t w[4];
      draw(md->seed, step, c.list[e].t, c.list[e].a, ORC_TAG_SEL_T, w);
      uint64_t key = ((uint64_t)w[0] << 32) | w[1];
      if (best < 0 || key < bestkey || (key == bestkey && c.list[e].a < c.list[best].a)) {
        best = e;
        bestkey = key;
      }
      ++e;
    }
    c.list[nfin++] = c.list[best];
    q = e;
  }
  qsort(c.list, (size_t)nfin, sizeof(pair_t), cmp_by_a);

  /* Step 9: add the bonds and shift the states by delta_A and delta_T. */
  const int status = add_bonds(s, rx, c.list, nfin, step);
  if (trace) {
    trace->candidates = c.candidates;
    trace->retained = c.nlist;
    trace->a_winners = nwin;
    trace->formed = nfin;
  }
  free(c.list);
  return status;
}

/* ------------------------------------------------------------------------
 * Observables: particles per (type, state) (the populations M, P, P* of
 * Sec. V and X_s of Sec. II.B), bonds, energies and momentum.
 * ---------------------------------------------------------------------- */
int orc_observables(const orc_system* s, const orc_md_params* md, orc_obs* o) {
  if (!s || !o) return ORC_EINVAL;
  memset(o, 0, sizeof(*o));
  for (int64_t i = 0; i < s->n; ++i) {
    int t = s->type[i], st = s->state[i];
    if (t < 8 && st >= 0 && st < 16) o->counts[t][st]++;
    for (int k = 0; k < 3; ++k) {
      o->ke_half += 0.5 * md->mass * s->v[3 * i + k] * s->v[3 * i + k];
      o->momentum[k] += md->mass * s->v[3 * i + k];
    }
  }
  o->bonds = s->nb;
  double* f = (double*)malloc(sizeof(double) * (size_t)(3 * (s->n > 0 ? s->n : 1)));
  if (!f) return ORC_ENOMEM;
  int rc = orc_forces(s, md, 1, f, &o->epot);
  free(f);
  return rc;
}

/* nsteps MD steps; after the step s with s % Theta == 0 the reaction runs
 * on the positions of step s (the extension hooks in after velocity Verlet
 * and the thermostat, Sec. III), so new bonds act from the next force
 * evaluation.  Observables are recorded after every reaction step. */
int orc_run(orc_system* s, const orc_md_params* md, const orc_rx_params* rx, int64_t nsteps,
            int use_cells, orc_obs* obs_per_reaction, int64_t obs_cap) {
  int64_t nobs = 0;
  for (int64_t q = 0; q < nsteps; ++q) {
    int rc = orc_step(s, md, use_cells, NULL);
    if (rc) return rc;
    if (rx && s->step % rx->theta == 0) {
      rc = orc_react(s, md, rx, use_cells, s->step, NULL);
      if (rc) return rc;
      if (obs_per_reaction && nobs < obs_cap) {
        rc = orc_observables(s, md, &obs_per_reaction[nobs++]);
        if (rc) return rc;
      }
    }
  }
  return ORC_OK;
}

/* ------------------------------------------------------------------------
 * Pair-distance histogram between two particle classes (the data behind
 * g_AB(r) and <N_AB>, Secs. V-VI), all pairs.
 * ---------------------------------------------------------------------- */
static int in_class(const orc_system* s, const orc_class* c, int64_t i) {
  return ((c->type_mask >> (s->type[i] & 31)) & 1u) && s->state[i] >= c->s_lo && s->state[i] <= c->s_hi;
}

int orc_pair_histogram(const orc_system* s, const orc_md_params* md, const orc_class* a,
                       const orc_class* b, double r_max, int32_t nbins, int64_t* counts,
                       int64_t* n_a, int64_t* n_b) {
  if (!s || !md || !a || !b || !counts || nbins < 1 || !(r_max > 0.0)) return ORC_EINVAL;
  double* e2 = (double*)malloc(sizeof(double) * (size_t)(nbins + 1));
  if (!e2) return ORC_ENOMEM;
  for (int32_t k = 0; k <= nbins; ++k) {
    const double e = r_max * (double)k / (double)nbins;
    e2[k] = e * e;
  }
  for (int32_t k = 0; k < nbins; ++k) counts[k] = 0;
  int64_t na = 0, nb = 0;
  for (int64_t i = 0; i < s->n; ++i) {
    nb += in_class(s, b, i);
    if (!in_class(s, a, i)) continue;
    na++;
    for (int64_t j = 0; j < s->n; ++j) {
      if (j == i || !in_class(s, b, j)) continue;
      double d[3];
      separation(s->x, i, j, md->L, d);
      const double r2 = dist2_fixed(d);
      if (!(r2 < e2[nbins])) continue;
      int32_t k = 0;
      while (k + 1 < nbins && e2[k + 1] <= r2) ++k;
      counts[k]++;
    }
  }
  if (n_a) *n_a = na;
  if (n_b) *n_b = nb;
  free(e2);
  return ORC_OK;
}

/* ------------------------------------------------------------------------
 * Several concurrent reactions.  The paper names this extension (Secs. III.B
 * and VII: reactions with different intrinsic rates, following the reactive
 * multiparticle collision scheme of Rohlf et al.) without giving the
 * algorithm.  Reading used here:
 *   - the reactions share Theta and the structure of Table I.  A particle may
 *     be an A of several reactions or a T of several, never an A of one and
 *     a T of another (checked), so a reaction step still forms at most one
 *     bond per particle (Sec. III.A);
 *   - the pair (A, T) is a candidate of reaction r when A is in r's A
 *     window, T in r's T window, r^2 < r_react,r^2 and the two are not
 *     bonded.  Its candidate reactions c_1 < ... < c_m (in the scheme's
 *     order) share one acceptance draw u, as the reaction channels of one
 *     collision do in that scheme: the pair is retained for reaction c_j, the
 *     first j with u < P_j, where P_j = p_c1 + ... + p_cj is summed in that
 *     order and p_r = k_r dt Theta (Eqs. 3-4 per reaction); with
 *     u >= P_m it is not retained.  The pair thus reacts with probability
 *     min(1, p_c1 + ... + p_cm), and with reaction r with probability p_r
 *     over that sum when the sum is at most 1; one reaction reduces to
 *     u < p exactly;
 *   - steps 3-9 of Table I run on the pooled retained pairs with the same
 *     keyed choices (the keys do not depend on the reaction); the bond of a
 *     final pair takes the increments, bond style and valence limit of its
 *     reaction.
 * ---------------------------------------------------------------------- */
int orc_check_reactions(const orc_rx_params* rx, int nrx) {
  if (!rx || nrx < 1 || nrx > ORC_MAX_REACTIONS) return ORC_EINVAL;
  for (int r = 0; r < nrx; ++r) {
    int rc = orc_check_reaction(&rx[r]);
    if (rc) return rc;
    if (rx[r].theta != rx[0].theta) return ORC_EINVAL;
    if (nrx > 1 && rx[r].selection != ORC_SELECT_RANDOM) return ORC_EINVAL;
  }
  /* no (type, state) is an A of one reaction and a T of another */
  for (int r = 0; r < nrx; ++r)
    for (int q = 0; q < nrx; ++q)
      if ((rx[r].mask_A & rx[q].mask_T) && !(rx[r].a_hi < rx[q].t_lo || rx[q].t_hi < rx[r].a_lo))
        return ORC_EINVAL;
  return ORC_OK;
}

typedef struct {
  uint32_t a, t;
  int32_t rx;
} rpair_t;

static int rcmp_by_a(const void* p, const void* q) {
  const rpair_t* x = (const rpair_t*)p;
  const rpair_t* y = (const rpair_t*)q;
  if (x->a != y->a) return x->a < y->a ? -1 : 1;
  if (x->t != y->t) return x->t < y->t ? -1 : 1;
  return 0;
}
static int rcmp_by_t(const void* p, const void* q) {
  const rpair_t* x = (const rpair_t*)p;
  const rpair_t* y = (const rpair_t*)q;
  if (x->t != y->t) return x->t < y->t ? -1 : 1;
  if (x->a != y->a) return x->a < y->a ? -1 : 1;
  return 0;
}

typedef struct {
  const orc_system* s;
  const orc_md_params* md;
  const orc_rx_params* rx;
  int nrx;
  int64_t step;
  rpair_t* list;
  int64_t nlist, caplist;
  int64_t candidates;
  int oom;
} rfind_ctx;

/* Steps 1 and 2 for one pair (i, j): its candidate reactions, then one
 * draw against their cumulative acceptance probabilities. */
static void rfind_visit(int64_t i, int64_t j, void* vctx) {
  rfind_ctx* c = (rfind_ctx*)vctx;
  const orc_system* s = c->s;
  double d[3];
  separation(s->x, i, j, c->md->L, d);
  const double r2 = dist2_fixed(d);
  int cand[ORC_MAX_REACTIONS];
  int m = 0;
  for (int r = 0; r < c->nrx; ++r) {
    const orc_rx_params* x = &c->rx[r];
    if (!eligible_A(s, x, i) || !eligible_T(s, x, j)) continue;
    if (!(r2 < x->r_react * x->r_react)) continue;
    cand[m++] = r;
  }
  if (m == 0 || bonded(s, i, j)) return;
  c->candidates++;
  uint32_t w[4];
  draw(c->md->seed, c->step, (uint32_t)i, (uint32_t)j, ORC_TAG_ACCEPT, w);
  const double u = orc_u53(w[0], w[1]);
  double P = 0.0;
  int chosen = -1;
  for (int q = 0; q < m && chosen < 0; ++q) {
    const orc_rx_params* x = &c->rx[cand[q]];
    P = P + x->k * c->md->dt * (double)x->theta;
    if (u < P) chosen = cand[q];
  }
  if (chosen < 0) return;
  if (c->nlist == c->caplist) {
    int64_t nc = c->caplist ? 2 * c->caplist : 1024;
    rpair_t* nl = (rpair_t*)realloc(c->list, sizeof(rpair_t) * (size_t)nc);
    if (!nl) {
      c->oom = 1;
      return;
    }
    c->list = nl;
    c->caplist = nc;
  }
  c->list[c->nlist].a = (uint32_t)i;
  c->list[c->nlist].t = (uint32_t)j;
  c->list[c->nlist].rx = chosen;
  c->nlist++;
}

int orc_react_set(orc_system* s, const orc_md_params* md, const orc_rx_params* rx, int nrx,
                  int use_cells, int64_t step, orc_rx_trace* trace, int64_t* formed_per_rx) {
  if (!s || !md) return ORC_EINVAL;
  int rc = orc_check_reactions(rx, nrx);
  if (rc) return rc;
  rfind_ctx c;
  memset(&c, 0, sizeof(c));
  c.s = s;
  c.md = md;
  c.rx = rx;
  c.nrx = nrx;
  c.step = step;
  double rmax = 0.0;
  for (int r = 0; r < nrx; ++r) rmax = rx[r].r_react > rmax ? rx[r].r_react : rmax;

  /* Steps 1-2 for every particle that is an A of some reaction. */
  cells_t cl;
  int have = 0;
  if (use_cells) {
    have = cells_build(s, md->L, rmax, &cl);
    if (have < 0) return ORC_ENOMEM;
  }
  for (int64_t i = 0; i < s->n; ++i) {
    int isA = 0;
    for (int r = 0; r < nrx; ++r) isA |= eligible_A(s, &rx[r], i);
    if (isA) for_each_neighbor(s, have ? &cl : NULL, md->L, i, rfind_visit, &c);
  }
  if (have) cells_free(&cl);
  if (c.oom) {
    free(c.list);
    return ORC_ENOMEM;
  }

  /* Steps 3 and 5: L_A by id_A, one T per A (smallest key, ties to the
   * smaller id_T). */
  qsort(c.list, (size_t)c.nlist, sizeof(rpair_t), rcmp_by_a);
  int64_t nwin = 0;
  for (int64_t q = 0; q < c.nlist;) {
    int64_t e = q, best = -1;
    uint64_t bestkey = 0;
    while (e < c.nlist && c.list[e].a == c.list[q].a) {
      uint32_t w[4];
      draw(md->seed, step, c.list[e].a, c.list[e].t, ORC_TAG_SEL_A, w);
      uint64_t key = ((uint64_t)w[0] << 32) | w[1];
      if (best < 0 || key < bestkey || (key == bestkey && c.list[e].t < c.list[best].t)) {
        best = e;
        bestkey = key;
      }
      ++e;
    }
    c.list[nwin++] = c.list[best];
    q = e;
  }

  /* Steps 6-7: L_T by id_T, one A per T (smallest key, ties to the
   * smaller id_A). */
  qsort(c.list, (size_t)nwin, sizeof(rpair_t), rcmp_by_t);
  int64_t nfin = 0;
  for (int64_t q = 0; q < nwin;) {
    int64_t e = q, best = -1;
    uint64_t bestkey = 0;
    while (e < nwin && c.list[e].t == c.list[q].t) {
      uint32_t w[4];
      draw(md->seed, step, c.list[e].t, c.list[e].a, ORC_TAG_SEL_T, w);
      uint64_t key = ((uint64_t)w[0] << 32) | w[1];
      if (best < 0 || key < bestkey || (key == bestkey && c.list[e].a < c.list[best].a)) {
        best = e;
        bestkey = key;
      }
      ++e;
    }
    c.list[nfin++] = c.list[best];
    q = e;
  }
  qsort(c.list, (size_t)nfin, sizeof(rpair_t), rcmp_by_a);

  /* Step 9, in ascending id of A, each bond with its reaction's increments,
   * style and valence limits. */
  int status = ORC_OK;
  if (formed_per_rx)
    for (int r = 0; r < nrx; ++r) formed_per_rx[r] = 0;
  for (int64_t q = 0; q < nfin; ++q) {
    const uint32_t a = c.list[q].a, t = c.list[q].t;
    const orc_rx_params* x = &rx[c.list[q].rx];
    if (formed_per_rx) formed_per_rx[c.list[q].rx]++;
    int capA = s->cap < x->max_valence[s->type[a] & 7] ? s->cap : x->max_valence[s->type[a] & 7];
    int capT = s->cap < x->max_valence[s->type[t] & 7] ? s->cap : x->max_valence[s->type[t] & 7];
    if (s->nadj[a] >= capA || s->nadj[t] >= capT || s->nb >= s->nb_cap) {
      status = ORC_ECAPACITY;
      continue;
    }
    s->adj[(int64_t)s->cap * a + s->nadj[a]] = t;
    s->adj_style[(int64_t)s->cap * a + s->nadj[a]] = (uint8_t)x->bond_style;
    s->nadj[a]++;
    s->adj[(int64_t)s->cap * t + s->nadj[t]] = a;
    s->adj_style[(int64_t)s->cap * t + s->nadj[t]] = (uint8_t)x->bond_style;
    s->nadj[t]++;
    s->bond_a[s->nb] = a;
    s->bond_t[s->nb] = t;
    s->bond_step[s->nb] = step;
    s->bond_style[s->nb] = (uint8_t)x->bond_style;
    if (s->bond_rx) s->bond_rx[s->nb] = (uint8_t)c.list[q].rx;
    s->nb++;
    s->state[a] = (int8_t)(s->state[a] + x->dA);
    s->state[t] = (int8_t)(s->state[t] + x->dT);
  }
  if (trace) {
    trace->candidates = c.candidates;
    trace->retained = c.nlist;
    trace->a_winners = nwin;
    trace->formed = nfin;
  }
  free(c.list);
  return status;
}

/* nsteps MD steps with the reaction set applied after every step s with
 * s % Theta == 0 (as orc_run). */
int orc_run_set(orc_system* s, const orc_md_params* md, const orc_rx_params* rx, int nrx,
                int64_t nsteps, int use_cells) {
  int rc = orc_check_reactions(rx, nrx);
  if (rc) return rc;
  for (int64_t q = 0; q < nsteps; ++q) {
    rc = orc_step(s, md, use_cells, NULL);
    if (rc) return rc;
    if (s->step % rx[0].theta == 0) {
      rc = orc_react_set(s, md, rx, nrx, use_cells, s->step, NULL, NULL);
      if (rc) return rc;
    }
  }
  return ORC_OK;
}
