/*
 * polyrx oracle: plain FP64 CPU restatement of de Buyl & Nies, "A parallel
 * algorithm for step- and chain-growth polymerization in Molecular Dynamics"
 * (arXiv:1409.7498).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check of the
 * package entry file and the CPU-baseline leg of the benchmark may load this
 * library.  The CUDA path never links, calls or includes anything from here,
 * and nothing here includes anything from the CUDA path.
 *
 * All arrays are indexed by particle id 0..n-1.  Positions are absolute
 * coordinates in [0, L) on a periodic orthorhombic box.
 */
#ifndef POLYRX_ORACLE_H
#define POLYRX_ORACLE_H
#include <stdint.h>

#define ORC_OK 0
#define ORC_EINVAL (-1)
#define ORC_ENOMEM (-2)
#define ORC_ECAPACITY (-3)
#define ORC_EOVERSTRETCH (-4)
#define ORC_ENONFINITE (-5)

/* Bond styles. FENE: Sec. II.C (Kremer-Grest bond).  Mirror LJ: Sec. II.C,
 * Eq. 17 (the paper's created-bond potential). */
#define ORC_BOND_FENE 0
#define ORC_BOND_MIRROR_LJ 1

/* Counter tags of the keyed Philox draws (fourth counter word, low byte). */
#define ORC_TAG_THERMO 1u
#define ORC_TAG_ACCEPT 2u
#define ORC_TAG_SEL_A 3u
#define ORC_TAG_SEL_T 4u
#define ORC_TAG_NEAREST 5u

/* Partner selection: the paper's algorithm (one T per A and one A per T,
 * each chosen at random; Table I), or the nearest-partner rule of the LAMMPS
 * fix bond/create that the paper compares it with (Sec. IV.A). */
#define ORC_SELECT_RANDOM 0
#define ORC_SELECT_NEAREST 1

typedef struct {
  double L[3];        /* box edges */
  double dt;          /* time step */
  double kT;          /* thermostat temperature */
  double gamma;       /* Langevin friction (0 = plain velocity Verlet) */
  double mass;        /* particle mass (all equal, Sec. II.C) */
  double eps, sigma;  /* WCA parameters, Eq. 15 */
  double fene_k;      /* FENE spring constant k_F */
  double fene_r0;     /* FENE maximum extension R_0 */
  double force_cap;   /* > 0: cap on the WCA pair-force magnitude (warm-up) */
  uint64_t seed;      /* Philox key */
} orc_md_params;

typedef struct {
  uint32_t mask_A;    /* bit t set: type t may act as the active A */
  uint32_t mask_T;    /* bit t set: type t may act as the target T */
  int32_t a_lo, a_hi; /* state window of A (inclusive) */
  int32_t t_lo, t_hi; /* state window of T (inclusive) */
  int32_t dA, dT;     /* state increments delta_A, delta_T, Eq. 2 */
  double k;           /* intrinsic rate */
  int64_t theta;      /* reaction interval Theta in MD steps */
  double r_react;     /* reaction cutoff */
  int32_t bond_style; /* style of the created bonds */
  int32_t selection;  /* ORC_SELECT_RANDOM (Table I) or ORC_SELECT_NEAREST (Sec. IV.A) */
  uint8_t max_valence[8]; /* per type: bonds a particle may hold */
} orc_rx_params;

typedef struct {
  int64_t n;          /* particles */
  int32_t cap;        /* adjacency capacity per particle */
  int32_t pad_;
  double* x;          /* [n][3] positions */
  double* v;          /* [n][3] velocities (half-step, see orc_step) */
  uint8_t* type;      /* [n] */
  int8_t* state;      /* [n] */
  uint8_t* nadj;      /* [n] bonds held */
  uint32_t* adj;      /* [n][cap] partner ids */
  uint8_t* adj_style; /* [n][cap] bond style of each entry */
  int64_t nb;         /* bonds in the list */
  int64_t nb_cap;     /* capacity of the bond list */
  uint32_t* bond_a;   /* [nb_cap] id of A (or first particle of an initial bond) */
  uint32_t* bond_t;   /* [nb_cap] id of T */
  int64_t* bond_step; /* [nb_cap] step the bond formed (0: initial) */
  uint8_t* bond_style;/* [nb_cap] */
  int64_t step;       /* completed MD steps */
  uint8_t* bond_rx;   /* [nb_cap] reaction that formed the bond (orc_react_set; may be NULL) */
} orc_system;

typedef struct {
  int64_t candidates;  /* Table I step 1 */
  int64_t retained;    /* step 2 */
  int64_t a_winners;   /* step 5 */
  int64_t formed;      /* step 7 / 9 */
} orc_rx_trace;

typedef struct {
  int64_t counts[8][16]; /* particles per (type, state) for state in 0..15 */
  int64_t bonds;
  double ke_half;        /* kinetic energy of the stored (half-step) velocities */
  double epot;           /* WCA + bond potential energy */
  double momentum[3];
} orc_obs;

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
double orc_u53(uint32_t hi, uint32_t lo);
double orc_u24(uint32_t w);

int orc_forces(const orc_system* s, const orc_md_params* md, int use_cells,
               double* f, double* epot);
int orc_step(orc_system* s, const orc_md_params* md, int use_cells, double* ke_full);
int orc_check_reaction(const orc_rx_params* rx);
int orc_react(orc_system* s, const orc_md_params* md, const orc_rx_params* rx,
              int use_cells, int64_t step, orc_rx_trace* trace);
int orc_observables(const orc_system* s, const orc_md_params* md, orc_obs* o);

/* A particle class: type in the mask and state in [s_lo, s_hi]. */
typedef struct {
  uint32_t type_mask;
  int32_t s_lo, s_hi;
} orc_class;

/* Pair-distance histogram between two classes, the raw data of the radial
 * distribution g_AB(r) whose integral up to the reaction cutoff gives the
 * mean number of available partners <N_AB> (Secs. V, VI):
 *   counts[k] = #{(i, j): i in a, j in b, j != i, e_k^2 <= r_ij^2 < e_(k+1)^2}
 * with e_k = r_max k / nbins, r_ij^2 = fma(dz, dz, fma(dy, dy, dx dx)) under
 * the minimum image.  *n_a, *n_b receive the class sizes. */
int orc_pair_histogram(const orc_system* s, const orc_md_params* md, const orc_class* a,
                       const orc_class* b, double r_max, int32_t nbins, int64_t* counts,
                       int64_t* n_a, int64_t* n_b);
int orc_run(orc_system* s, const orc_md_params* md, const orc_rx_params* rx,
            int64_t nsteps, int use_cells, orc_obs* obs_per_reaction, int64_t obs_cap);

/* Several concurrent reactions (the extension named in Secs. III.B and VII;
 * see orc_react_set in oracle.c for the reading).  At most ORC_MAX_REACTIONS
 * reactions sharing Theta; formed_per_rx (may be NULL) receives, per
 * reaction, the final pairs of that reaction. */
#define ORC_MAX_REACTIONS 4
int orc_check_reactions(const orc_rx_params* rx, int nrx);
int orc_react_set(orc_system* s, const orc_md_params* md, const orc_rx_params* rx, int nrx,
                  int use_cells, int64_t step, orc_rx_trace* trace, int64_t* formed_per_rx);
int orc_run_set(orc_system* s, const orc_md_params* md, const orc_rx_params* rx, int nrx,
                int64_t nsteps, int use_cells);

#endif
