/*
 * OpenMP timing driver of the polyrx oracle.
 *
 * TEST INFRASTRUCTURE ONLY: the benchmark's CPU-baseline leg uses it to time
 * the oracle on every host core, beside the single-threaded timing of
 * orc_run.  It includes oracle.c unchanged, so every potential, the
 * Langevin update, the keyed draws and the reaction step (Table I) are the
 * pinned functions themselves; only the two per-particle loops of an MD step
 * are spread over threads:
 *   - the conservative force on particle i (its WCA pairs in the cell list's
 *     visiting order, then its bonds, Sec. II.C), which writes f[i] alone;
 *   - the Langevin velocity-Verlet update of particle i, which writes x[i]
 *     and v[i] alone.
 * Per particle the operations and their order are those of orc_forces and
 * orc_step, so orc_run_omp produces the same trajectory, bit for bit, as
 * orc_run (a CPU test checks it).  The cell list is built and the reaction
 * step runs on one thread, as in orc_run.
 */
#include "oracle.c"

#include <omp.h>

/* Conservative forces, one particle per loop iteration. */
static int forces_omp(const orc_system* s, const orc_md_params* md, double* f) {
  cells_t cl;
  const int have = cells_build(s, md->L, wca_cutoff(md), &cl);
  if (have < 0) return ORC_ENOMEM;
  int bad = 0;
#pragma omp parallel for schedule(static) reduction(| : bad)
  for (int64_t i = 0; i < s->n; ++i) {
    for (int k = 0; k < 3; ++k) f[3 * i + k] = 0.0;
    force_ctx ctx = {s, md, f, 0.0};
    for_each_neighbor(s, have ? &cl : NULL, md->L, i, force_visit, &ctx);
    for (int b = 0; b < s->nadj[i]; ++b) {
      int64_t j = s->adj[(int64_t)s->cap * i + b];
      double d[3];
      separation(s->x, i, j, md->L, d);
      double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
      double V = 0.0, g = 0.0;
      if (s->adj_style[(int64_t)s->cap * i + b] == ORC_BOND_MIRROR_LJ) {
        mirror_lj_pair(r2, md, &V, &g);
      } else if (fene_pair(r2, md, &V, &g)) {
        bad = 1;
        continue;
      }
      for (int k = 0; k < 3; ++k) f[3 * i + k] -= g * d[k];
    }
  }
  if (have) cells_free(&cl);
  return bad ? ORC_EOVERSTRETCH : ORC_OK;
}

/* One MD step with the update of orc_step, one particle per iteration. */
static int step_omp(orc_system* s, const orc_md_params* md, double* f) {
  const int64_t step = s->step + 1;
  int rc = forces_omp(s, md, f);
  if (rc) return rc;
  const double cR = sqrt(24.0 * md->gamma * md->kT * md->mass / md->dt);
  int bad = 0;
#pragma omp parallel for schedule(static) reduction(| : bad)
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
      double xn = s->x[3 * i + k] + md->dt * vn;
      if (xn >= md->L[k]) xn -= md->L[k];
      if (xn < 0.0) xn += md->L[k];
      if (!isfinite(xn) || !isfinite(vn)) bad = 1;
      s->v[3 * i + k] = vn;
      s->x[3 * i + k] = xn;
    }
  }
  if (bad) return ORC_ENONFINITE;
  s->step = step;
  return ORC_OK;
}

/* orc_run on `threads` threads (0: OpenMP's default); observables are not
 * recorded.  Returns the status of the first failing step. */
int orc_run_omp(orc_system* s, const orc_md_params* md, const orc_rx_params* rx, int64_t nsteps,
                int threads) {
  if (!s || !md) return ORC_EINVAL;
  if (threads > 0) omp_set_num_threads(threads);
  double* f = (double*)malloc(sizeof(double) * (size_t)(3 * (s->n > 0 ? s->n : 1)));
  if (!f) return ORC_ENOMEM;
  int rc = ORC_OK;
  for (int64_t q = 0; q < nsteps && rc == ORC_OK; ++q) {
    rc = step_omp(s, md, f);
    if (rc == ORC_OK && rx && s->step % rx->theta == 0) rc = orc_react(s, md, rx, 1, s->step, NULL);
  }
  free(f);
  return rc;
}

/* Threads an OpenMP parallel region gets by default on this host. */
int orc_omp_max_threads(void) { return omp_get_max_threads(); }
