/*
 * polyrx: C ABI of the GB300 (sm_103a) reactive coarse-grained MD library.
 *
 * It implements the data-parallel hot path of de Buyl & Nies, "A parallel
 * algorithm for step- and chain-growth polymerization in Molecular
 * Dynamics" (arXiv:1409.7498):
 *   - the MD step: WCA pair forces (Sec. II.C, Eq. 15) from Verlet
 *     neighbour lists built on a cell grid, FENE bond forces (Sec. II.C) or
 *     mirror-LJ created bonds (Eq. 17), and a Langevin velocity-Verlet
 *     integrator (velocity Verlet, Sec. II.C);
 *   - the reaction step run every Theta steps after the integration
 *     (Sec. III): candidate A/T pairs by type, state and distance, accepted
 *     with probability k dt Theta (Eqs. 3-4), one T per A and one A per T
 *     chosen at random (Table I, steps 1-9), bonds appended and states
 *     shifted by delta_A and delta_T (Eq. 2).
 *
 * Conventions for every entry point:
 *   - Return value: PRX_OK (0) or a negative PRX_E* status.  No C++
 *     exception crosses this boundary.  prx_last_error() gives a message.
 *   - Host arrays are indexed by particle id 0..n-1 and are owned by the
 *     caller; the library copies what it needs and never keeps a pointer to
 *     them.  All device memory is owned by the library.
 *   - Work is queued on the system's CUDA stream (the caller's stream when
 *     one is passed to prx_create, else a library-owned non-blocking
 *     stream).  Calls that return data to the host synchronise that stream.
 *     Device-side errors (FENE overstretch, capacity, non-finite values) are
 *     sticky: they surface at the next synchronising call or prx_sync().
 *   - Not thread-safe per system: one host thread drives one system.
 *   - Steps are numbered from 1.  A reaction runs after step s when
 *     s % Theta == 0, on the positions of step s; new bonds act from the
 *     next force evaluation.
 */
#ifndef POLYRX_H
#define POLYRX_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------- */
#define PRX_OK 0
#define PRX_EINVAL (-1)       /* bad argument, descriptor or call order */
#define PRX_ENOMEM (-2)       /* device or host allocation failed */
#define PRX_ECAPACITY (-3)    /* adjacency, valence, bond-list or buffer capacity exceeded */
#define PRX_EOVERSTRETCH (-4) /* a FENE bond reached r >= R0 */
#define PRX_ENONFINITE (-5)   /* a position, velocity or force became non-finite,
                                 or a particle crossed more than one cell in a step */
#define PRX_ETIMEOUT (-6)     /* a bounded device wait gave up (reserved: no kernel of
                                 this version waits on a flag) */
#define PRX_ECUDA (-7)        /* a CUDA runtime call failed */
#define PRX_EIO (-8)          /* checkpoint file could not be read or written */

/* ---- constants ------------------------------------------------------- */
#define PRX_BOND_FENE 0       /* Kremer-Grest FENE, Sec. II.C */
#define PRX_BOND_MIRROR_LJ 1  /* mirror Lennard-Jones, Eq. 17 */
#define PRX_SELECT_RANDOM 0   /* Table I: one T per A, one A per T, each at random */
#define PRX_SELECT_NEAREST 1  /* LAMMPS fix bond/create (Sec. IV.A): mutual nearest
                                 A-T pairs, then the acceptance test */
#define PRX_FORCE_FP32 0      /* pair and bond forces in FP32, integration in FP64 */
#define PRX_FORCE_FP64 1      /* everything in FP64 */
#define PRX_MAX_TYPES 8
#define PRX_MAX_STATES 16     /* states tracked by the observables: 0..15 */
#define PRX_MAX_ADJ 8         /* largest adjacency capacity per particle */
#define PRX_MAX_REACTIONS 4   /* concurrent reactions of one scheme */

typedef struct prx_system prx_system; /* opaque, library-owned */
typedef struct prx_batch prx_batch;   /* opaque, library-owned (see below) */

/* System descriptor.  Units are reduced LJ units (Sec. II.C). */
typedef struct {
  uint32_t n;             /* particles (0 allowed) */
  uint32_t adj_cap;       /* bonds a particle may hold, 1..PRX_MAX_ADJ */
  double box[3];          /* periodic box edges */
  double dt;              /* time step */
  double kT;              /* thermostat temperature */
  double gamma;           /* Langevin friction; 0 = plain velocity Verlet */
  double mass;            /* particle mass */
  double wca_eps;         /* WCA epsilon (Eq. 15) */
  double wca_sigma;       /* WCA sigma; cutoff sigma_c = 2^(1/6) sigma */
  double fene_k;          /* FENE k_F */
  double fene_r0;         /* FENE R_0 */
  double force_cap;       /* > 0: cap on the WCA pair-force magnitude (warm-up); 0: off */
  double skin;            /* Verlet-list skin: list radius = cutoff + skin, lists rebuilt
                             when a particle moved skin/2; < 0 selects the default (0.3);
                             shrunk automatically in boxes shorter than 3 list radii */
  int32_t force_precision;/* PRX_FORCE_FP32 or PRX_FORCE_FP64 */
  int32_t reserved;       /* must be 0 */
  uint64_t seed;          /* key of every random draw */
} prx_system_desc;

/* Reaction scheme T^t + A^a -> T^(t+dT)-A^(a+dA) (Eq. 2).  A particle of
 * type t is an eligible A when bit t of type_mask_A is set and its state is
 * in [a_lo, a_hi]; likewise for T.  For a type in both masks the two
 * windows must be disjoint, so no particle is A and T at once. */
typedef struct {
  uint32_t type_mask_A;
  uint32_t type_mask_T;
  int32_t a_lo, a_hi;
  int32_t t_lo, t_hi;
  int32_t dA, dT;
  double k;               /* intrinsic rate; acceptance probability p = k dt Theta */
  double r_react;         /* reaction cutoff (strict: r^2 < r_react^2, FP64) */
  uint32_t theta;         /* reaction interval Theta >= 1 */
  int32_t bond_style;     /* style of the created bonds */
  int32_t selection;      /* PRX_SELECT_RANDOM or PRX_SELECT_NEAREST */
  uint8_t max_valence[PRX_MAX_TYPES]; /* per type: bonds a particle may hold */
} prx_reaction_desc;

/* One bond of the bond list (the FixedPairList of Sec. III.A).  For a
 * created bond a is the active A and t the target T. */
typedef struct {
  uint32_t a, t;
  int64_t step;           /* step the bond formed; 0 for bonds given at creation */
  uint32_t style;
  uint32_t reaction;      /* index in the scheme of the reaction that formed it
                             (0 for initial bonds and single-reaction schemes) */
} prx_bond;

/* Counts of Table I for one reaction step.  With PRX_SELECT_NEAREST:
 * retained = mutual nearest pairs, a_winners = those accepted. */
typedef struct {
  int64_t candidates;     /* step 1: eligible pairs within the cutoff */
  int64_t retained;       /* step 2: accepted by u < k dt Theta */
  int64_t a_winners;      /* step 5: A's left with one T */
  int64_t formed;         /* steps 7-9: bonds created */
} prx_rx_trace;

typedef struct {
  int64_t step;
  int64_t bonds;
  int64_t counts[PRX_MAX_TYPES][PRX_MAX_STATES]; /* particles per (type, state) */
  double ke_half;         /* sum of m v^2 / 2 over the stored half-step velocities */
  double momentum[3];
} prx_observables;

/* One record of the per-reaction history kept on the device. */
typedef struct {
  int64_t step;
  int64_t bonds;
  int32_t counts[PRX_MAX_TYPES][PRX_MAX_STATES];
} prx_history_record;

typedef struct {
  uint64_t steps;         /* MD steps completed */
  uint64_t reactions;     /* reaction steps completed */
  uint64_t rebins;        /* neighbour-list rebuilds (sort + lists), including the first */
  uint64_t step_launches; /* step-kernel launches */
  uint64_t kernel_launches; /* all kernels launched by this system so far */
  uint32_t cells[3];      /* cell grid */
  double cell_edge[3];
} prx_stats;

/* Per-kernel device time recorded with CUDA events while profiling is on. */
typedef struct {
  char name[32];
  uint64_t launches;
  double total_ms;
} prx_kernel_time;

/* ---- lifecycle --------------------------------------------------------- */

/* Creates a system.  pos: [n][3] in [0, box) (a coordinate outside is
 * wrapped once; farther outside is PRX_EINVAL).  vel: [n][3] or NULL for
 * zero.  type: [n] values < PRX_MAX_TYPES.  state: [n].  bonds: n_bonds
 * initial bonds (a != t, ids < n) or NULL; they count against adj_cap.
 * cuda_stream: a cudaStream_t to use, or NULL for a library-owned stream.
 * On success *out receives the system. */
int prx_create(const prx_system_desc* desc, const double* pos, const double* vel,
               const uint8_t* type, const int8_t* state, const prx_bond* bonds,
               uint64_t n_bonds, void* cuda_stream, prx_system** out);

/* Frees every device and host resource of the system (NULL is a no-op). */
void prx_destroy(prx_system* sys);

/* Device bytes a system of this descriptor holds once created (prx_create)
 * and given the reaction scheme rx (NULL: none; a reaction cutoff above the
 * WCA cutoff widens the Verlet lists).  The admission unit of a batch's
 * memory budget (prx_batch_admit).  PRX_EINVAL for a NULL desc or bytes. */
int prx_estimate_bytes(const prx_system_desc* desc, const prx_reaction_desc* rx, uint64_t* bytes);

/* Sets (or, with rx == NULL, clears) the reaction scheme.  PRX_EINVAL when
 * the state windows of a type in both masks overlap, theta == 0, k < 0,
 * r_react <= 0, or a bond style or selection rule is unknown.  If r_react
 * exceeds the cell list's cutoff the cell grid is rebuilt.  The same as
 * prx_set_reactions(sys, rx, 1). */
int prx_set_reaction(prx_system* sys, const prx_reaction_desc* rx);

/* Sets n_rx concurrent reactions (1..PRX_MAX_REACTIONS; n_rx == 0 clears the
 * scheme).  The paper names several concurrent reactions with different
 * intrinsic rates as an extension of its algorithm (Secs. III.B, VII) without
 * giving one; this library's rule:
 *   - the reactions share Theta and the steps of Table I; a particle may be
 *     an A of several reactions or a T of several, never an A of one and a T
 *     of another, so each reaction step forms at most one bond per particle;
 *   - a pair is a candidate of reaction r when A and T lie in r's windows,
 *     r^2 < r_react,r^2 and they are not bonded; its candidate reactions
 *     c_1 < ... < c_m share one acceptance draw u (Eq. 4): it is retained for
 *     c_j, the first j with u < p_c1 + ... + p_cj (p_r = k_r dt Theta, summed
 *     in FP64 in this order), else not retained;
 *   - one T per A and one A per T are chosen among the retained pairs of all
 *     reactions as in Table I; a bond takes the increments, style and valence
 *     limits of its reaction, and its record names the reaction.
 * PRX_EINVAL when a reaction is invalid (as prx_set_reaction), the thetas
 * differ, a (type, state) is an A of one reaction and a T of another, or
 * n_rx > 1 with the nearest-partner rule. */
int prx_set_reactions(prx_system* sys, const prx_reaction_desc* rx, uint32_t n_rx);

/* ---- execution --------------------------------------------------------- */

/* Queues nsteps MD steps (with the reaction every Theta steps) on the
 * system's stream and returns without waiting.  The run is one device-driven
 * chain: after each step a kernel on the GPU launches the list rebuild when
 * a particle moved more than skin/2, the reaction step when it is due, and
 * the next step (device graph launches); where device graphs are not
 * available the library replays host-launched CUDA graphs with a
 * conditional rebuild node after each step instead, with the same kernels
 * and the same result. */
int prx_run(prx_system* sys, uint64_t nsteps);

/* Waits for queued work; returns the sticky device status. */
int prx_sync(prx_system* sys);

/* Runs only the reaction step (Table I) on the current state, numbering the
 * draws with `step` (parity entry point; no MD step is taken).  trace may
 * be NULL.  Synchronises. */
int prx_react_once(prx_system* sys, uint64_t step, prx_rx_trace* trace);

/* Conservative forces (WCA + bonds, no thermostat) at the current positions,
 * f_out [n][3] by id, and the potential energy.  Synchronises. */
int prx_compute_forces(prx_system* sys, double* f_out, double* epot_out);

/* ---- read-back (all synchronise) ------------------------------------------ */
int prx_get_step(prx_system* sys, uint64_t* step);
int prx_get_positions(prx_system* sys, double* out /* [n][3] by id, wrapped into [0, box) */);
int prx_get_velocities(prx_system* sys, double* out /* [n][3] by id, half-step */);
int prx_get_states(prx_system* sys, int8_t* out /* [n] by id */);
int prx_get_types(prx_system* sys, uint8_t* out /* [n] by id */);
/* Bonds in canonical order (step, a, t).  *n_out receives the bond count;
 * PRX_ECAPACITY if cap is smaller (out then holds the first cap). */
int prx_get_bonds(prx_system* sys, prx_bond* out, uint64_t cap, uint64_t* n_out);
int prx_get_observables(prx_system* sys, prx_observables* out);

/* Pipelined observables (the populations of Secs. V-VI, bonds, kinetic
 * energy, momentum) for monitoring a running system without stalling it.
 * prx_observables_begin enqueues their computation and the copy into pinned
 * host slot `slot` (0..PRX_OBS_SLOTS-1) on the system's stream and returns
 * at once; runs enqueued afterwards proceed on the device meanwhile.
 * prx_observables_end waits for that slot and fills *out with the values as
 * of the begin call.  PRX_EINVAL for a slot out of range or one without a
 * pending begin; a device error status is reported by the end call.  Not
 * allowed for batch members (the batch owns their stream). */
#define PRX_OBS_SLOTS 4
int prx_observables_begin(prx_system* sys, int slot);
int prx_observables_end(prx_system* sys, int slot, prx_observables* out);
/* Pipelined read of the newest reaction record (the populations per
 * (type, state) of Secs. V-VI and the bond count after the latest reaction
 * step, with its step): the reaction step itself leaves it at a fixed place,
 * so prx_history_begin launches no kernel; it enqueues the copy into pinned
 * host slot `slot` (0..PRX_OBS_SLOTS-1, shared with the observables calls)
 * on the system's stream and returns at once; prx_history_end waits for
 * that slot and fills *out (all zero before the first reaction step).
 * States change only at reaction steps, so after a run of whole reaction
 * intervals this is the run's current population record.  Not allowed for
 * batch members.  PRX_EINVAL for a slot out of range or busy / not
 * pending; a device error status is reported by the end call. */
int prx_history_begin(prx_system* sys, int slot);
int prx_history_end(prx_system* sys, int slot, prx_history_record* out);

/* The last min(cap, recorded) per-reaction records, oldest first.  The
 * device keeps the most recent `history_cap` records (default 8192). */
int prx_get_history(prx_system* sys, prx_history_record* out, uint64_t cap, uint64_t* n_out);
int prx_get_stats(prx_system* sys, prx_stats* out);

/* ---- analysis ----------------------------------------------------------------- */
/* A particle class: type bit set in type_mask, state in [s_lo, s_hi]. */
typedef struct {
  uint32_t type_mask;
  int32_t s_lo, s_hi;
} prx_class;

/* Pair-distance histogram between class a and class b at the current
 * positions: counts[k] (host, nbins entries) receives the number of ordered
 * pairs (i in a, j in b, j != i) with e_k^2 <= r_ij^2 < e_(k+1)^2, where
 * e_k = r_max k / nbins and r_ij^2 is the exact FP64 minimum-image distance
 * of the reaction test.  These are the data of the radial distribution
 * g_ab(r) whose integral up to the reaction cutoff is the mean number of
 * available partners <N_ab> (Secs. V-VI); *n_a, *n_b (may be NULL) receive
 * the class sizes.  The pairs come from the Verlet lists, which hold every
 * pair closer than the larger of the WCA and reaction cutoffs: r_max above
 * it, or nbins outside 1..2048, is PRX_EINVAL.  Read-only: allowed for a batch
 * member (it waits for the batch's stream).  Synchronises. */
int prx_pair_histogram(prx_system* sys, const prx_class* a, const prx_class* b, double r_max,
                       uint32_t nbins, uint64_t* counts, uint64_t* n_a, uint64_t* n_b);

/* ---- checkpoint ------------------------------------------------------------ */
/* Writes positions, velocities, types, states, bonds, step, descriptor and
 * reaction scheme.  Every random draw is keyed by (seed, step, ids), so a
 * loaded system continues bit for bit. */
int prx_save(prx_system* sys, const char* path);
int prx_load(const char* path, void* cuda_stream, prx_system** out);

/* ---- profiling ------------------------------------------------------------- */
/* While on, prx_run launches kernels one by one (no CUDA graph), brackets
 * each with CUDA events on the system's stream, and reads the cell-list
 * flag after every step to launch a rebuild only when needed. */
int prx_profile_begin(prx_system* sys);
/* Ends profiling and returns per-kernel launch counts and device time. */
int prx_profile_end(prx_system* sys, prx_kernel_time* out, uint32_t cap, uint32_t* n_out);

/* ---- allocation-free reaction step ------------------------------------------ */
/* Largest system prx_react_noalloc accepts. */
#define PRX_NOALLOC_MAX_N 16384

/* One reaction step (the same rules, draws and tie-breaking as
 * prx_react_once: rx->selection picks Table I's random rule or the
 * nearest-partner rule of Sec. IV.A) on device arrays the caller owns,
 * allocating nothing.
 * The paper has no counterpart: this entry point exists for callers that
 * cannot allocate device memory themselves, e.g. code that must stay within
 * a memory budget fixed by a host framework, or that runs inside an
 * allocator hook.
 *
 * Inputs (device pointers, indexed by particle id 0..n-1): d_pos [n][3]
 * positions in [0, box); d_type [n].  Updated in place: d_state [n], d_nadj
 * [n] and d_adj [n][adj_cap] (partner ids, bit 31 = bond style).  Outputs:
 * d_bonds_out receives the new bonds in ascending id of A (at most
 * bonds_cap), *d_nbonds_out (device) their number; trace (host, may be
 * NULL) the Table I counts.  The candidate search is all-pairs.
 *
 * Scratch memory: one static device array sized for PRX_NOALLOC_MAX_N
 * particles, held by every GPU that loads the library until the process
 * exits; n above that limit returns PRX_ECAPACITY.  The first call on a
 * device looks up the array's device address with that device current.
 * Every call shares the array: calls whose work overlaps on the GPU race, so
 * serialise them.  The call is queued on cuda_stream (NULL: the legacy
 * default stream), copies its counters into host memory and waits for the
 * stream before returning, so it must not be called while that stream is
 * being captured into a CUDA graph.
 *
 * Errors: PRX_EINVAL for a bad descriptor (as prx_set_reaction, including an
 * unknown selection rule) or a missing pointer.  PRX_ECAPACITY when a pair
 * would exceed a particle's valence (min(max_valence[type], adj_cap): that
 * pair forms no bond and takes no place in the output) or more bonds formed
 * than bonds_cap (the first bonds_cap, in ascending id of A, are applied and
 * written; the rest are not applied); every other pair is still applied and
 * written, and the trace counts every surviving pair, as prx_react_once
 * does. */
int prx_react_noalloc(const prx_reaction_desc* rx, const double* box, double dt, uint64_t seed,
                      uint64_t step, uint32_t n, const double* d_pos, const uint8_t* d_type,
                      int8_t* d_state, uint32_t adj_cap, uint8_t* d_nadj, uint32_t* d_adj,
                      prx_bond* d_bonds_out, uint32_t bonds_cap, uint32_t* d_nbonds_out,
                      void* cuda_stream, prx_rx_trace* trace);

/* ---- autotuner ---------------------------------------------------------------- */
/* Times the MD step (with the reaction every Theta steps when rx != NULL) of
 * the system described by desc and the host arrays (as for prx_create) for
 * each of the n_skins candidate skins, and writes the fastest to *best_skin.
 * Each candidate is a temporary system built from the same inputs on a
 * library stream, so the call needs the device memory of one extra system; it
 * runs steps / 4 + 1 warm-up steps, then times `steps` steps with CUDA
 * events.  ms_per_step (n_skins entries, may be NULL) receives each
 * candidate's time, -1 for a candidate that could not run (e.g. a box too
 * small for that list radius).  The skin sets the Verlet-list radius
 * r_c + skin, the cell edge and how often the lists are rebuilt; it does not
 * change the model: runs that differ only in the skin differ only in the
 * order of floating-point sums.  The choice depends on timing, so a run that
 * must be reproducible records the chosen skin in its descriptor.
 * PRX_EINVAL when no candidate could run. */
int prx_autotune_skin(const prx_system_desc* desc, const double* pos, const double* vel,
                      const uint8_t* type, const int8_t* state, const prx_reaction_desc* rx,
                      uint32_t steps, const double* skins, uint32_t n_skins, double* best_skin,
                      double* ms_per_step);

/* Launch configuration of a system's kernels.  The block shape and the
 * interval batching change only the speed: a run gives the same result, bit
 * for bit, under any of them (one thread computes each particle's forces and
 * update whatever the block shape, and a graph replay of m intervals
 * launches the same kernels as m replays of one).  The lanes per particle
 * change, like the skin, only the order of the FP32 force sums: with 4 a
 * particle's list is split over four lanes whose partial sums are combined
 * in a fixed order (more warps in flight for systems too small to fill the
 * GPU). */
typedef struct {
  uint32_t step_threads;       /* threads per block of the step kernel: 128, 256 or 512 (0: 256) */
  uint32_t step_blocks_per_sm; /* blocks per SM of its persistent grid (0: as many as fit) */
  uint32_t chunk_intervals;    /* reaction intervals per CUDA-graph replay in prx_run, 1..64
                                  (0: 1); without a scheme, chunks of 10 steps; used only
                                  when runs fall back to host-replayed graphs */
  uint32_t step_lanes;         /* lanes per particle of the FP32 step: 1 or 4 (0: 1) */
} prx_launch_config;

/* PRX_EINVAL for values out of range, a batch member, or a FP64-force
 * system with step_threads other than 0 or 256 or step_lanes other than
 * 0 or 1 (its kernels are fixed).  A system with step_lanes 4 cannot join a
 * batch (batched members run the one-lane kernel, so that each computes
 * exactly what it computes alone). */
int prx_set_launch_config(prx_system* sys, const prx_launch_config* cfg);
int prx_get_launch_config(prx_system* sys, prx_launch_config* cfg);

/* One autotuner candidate: skin, launch configuration, measured time. */
typedef struct {
  double skin;
  prx_launch_config launch;
  double ms_per_step;     /* -1: the candidate could not run */
  uint32_t stage;         /* 0 skin, 1 block shape, 2 interval batching */
  uint32_t cached;        /* 1: taken from the cache, not timed in this call */
} prx_tune_choice;

/* The library's autotuner over the Verlet skin (cell size and rebuild
 * interval), the step kernel's block shape and the reaction-interval
 * batching, by coordinate search: every skin with the default launch, then
 * every (threads, blocks per SM, lanes per particle) shape at the best
 * skin, then every chunk length at the best of those.  Each candidate is a temporary system built
 * from the inputs (as prx_autotune_skin), timed with CUDA events over
 * `steps` steps (rounded up to whole chunks) after a warm-up.  Empty lists
 * (count 0) keep the default of that dimension.  *best receives the fastest
 * candidate of the last stage; tried (may be NULL) up to tried_cap of the
 * timed candidates, *n_tried their count.  Results are cached for the
 * process, keyed by particle count, density, adjacency capacity, force
 * precision and reaction scheme (cutoff, Theta, rate), and by the candidate
 * lists; with cache_path non-NULL also in that text file (read before
 * timing, appended after), so another run can reuse them.  A cached
 * result comes back with best->cached = 1 and no candidate timed. */
int prx_autotune(const prx_system_desc* desc, const double* pos, const double* vel,
                 const uint8_t* type, const int8_t* state, const prx_reaction_desc* rx,
                 uint32_t steps, const double* skins, uint32_t n_skins, const uint32_t* threads,
                 const uint32_t* blocks_per_sm, const uint32_t* lanes, uint32_t n_shapes,
                 const uint32_t* chunks, uint32_t n_chunks, const char* cache_path,
                 prx_tune_choice* best, prx_tune_choice* tried, uint32_t tried_cap,
                 uint32_t* n_tried);

/* ---- batched ensemble -------------------------------------------------------- */
/* A batch advances many independent systems (replicas of different sizes,
 * schemes, rates and seeds) together: every MD step is ONE kernel launch
 * over all members, each block serving one part of one member; the
 * neighbour-list rebuild and the reaction step are one launch per kernel
 * too, in which members that need no rebuild (or have no reaction scheme)
 * return at once.  The steps, rebuilds and reactions of a batch are replayed
 * from CUDA graphs.  Every member computes exactly what it computes alone
 * (prx_run): the same kernels on the same data, bit for bit.
 *
 * The paper runs one system at a time; batching is this library's addition
 * for ensembles of replicas (the 32-seed kinetics averages of Sec. IV) and
 * for serving many jobs on one GPU. */
typedef struct {
  uint32_t members;         /* systems in the batch */
  uint32_t active;          /* members with at least one particle */
  uint64_t particles;       /* sum of the members' particle counts */
  uint64_t steps;           /* steps run by the batch */
  uint64_t rebuilds;        /* steps after which some member rebuilt its lists */
  uint64_t reactions;       /* reaction steps run */
  uint64_t kernel_launches; /* kernels launched by the batch */
  uint64_t graph_launches;  /* CUDA graph replays */
  uint32_t max_slots;       /* as given to prx_batch_create (0: no limit) */
  uint32_t slots_used;      /* admitted systems not yet reported by prx_batch_poll */
  uint64_t mem_budget;      /* as given to prx_batch_create (0: no limit) */
  uint64_t bytes_admitted;  /* prx_estimate_bytes summed over the members and the
                               admitted systems not yet reported */
  uint64_t epochs;          /* prx_batch_step_epoch calls that ran steps */
} prx_batch_stats;

/* Creates an empty batch whose work is queued on cuda_stream (NULL: a
 * library-owned stream).  max_slots bounds the systems held at once and
 * mem_budget the device bytes they hold together (prx_estimate_bytes of
 * each); 0 means no limit.  Admission beyond either is PRX_ENOMEM. */
int prx_batch_create(uint32_t max_slots, uint64_t mem_budget, void* cuda_stream, prx_batch** out);

/* Waits for the batch, returns every member to standalone use (on its own
 * stream, state kept) and frees the batch.  NULL is a no-op. */
void prx_batch_destroy(prx_batch* b);

/* Adds a system with no step target (advanced by prx_batch_run).  PRX_ENOMEM
 * when it would exceed the batch's slots or memory budget; PRX_EINVAL when
 * the system is in a batch already, uses
 * PRX_FORCE_FP64 (batches run FP32 forces only), is being profiled, or has
 * a reaction scheme whose Theta differs from that of the batch's reacting
 * members or whose step is at another point of the Theta cycle.  The
 * system's own stream is synchronised first.  While it is a member,
 * prx_run, prx_react_once, prx_set_reaction, prx_compute_forces and
 * prx_profile_begin on it return PRX_EINVAL; read-back calls and prx_save
 * work and wait for the batch's stream. */
int prx_batch_add(prx_batch* b, prx_system* sys);

/* Waits for the batch and removes a member (PRX_EINVAL if it is not one);
 * its slot and budget are freed. */
int prx_batch_remove(prx_batch* b, prx_system* sys);

/* Queues nsteps steps of every member (reactions every Theta steps as in
 * prx_run) on the batch's stream and returns without waiting.  PRX_EINVAL
 * while a member admitted with a step target (prx_batch_admit) is in the
 * batch: such batches advance by prx_batch_step_epoch. */
int prx_batch_run(prx_batch* b, uint64_t nsteps);

/* ---- serving: admission by slots and device memory, epochs, completion ----
 * The request loop of a server that keeps many jobs resident on one GPU:
 * jobs arrive as systems created by the caller, are admitted while a slot
 * and memory are free, advance together epoch by epoch, and are reported
 * when their steps are done so that the caller reads their results and the
 * slot takes the next job.  The paper runs one system at a time; this is the
 * library's continuous batching of many. */

/* Admits sys as a member that is to run exactly nsteps more steps (its result
 * is then the same as that of prx_run(sys, nsteps) alone, bit for bit).
 * *slot receives its slot number (0..max_slots-1; a running number when
 * max_slots is 0).  PRX_ENOMEM when no slot is free or when its
 * prx_estimate_bytes plus bytes_admitted exceeds the budget: the system is
 * then not admitted and stays usable alone.  PRX_EINVAL as prx_batch_add.
 * Queued work of the system is ordered before the batch's (no host wait). */
int prx_batch_admit(prx_batch* b, prx_system* sys, uint64_t nsteps, int32_t* slot);

/* Queues one epoch on the batch's stream:
 *  - admitted members with fewer steps left than one chunk (Theta steps;
 *    10 when no member reacts) leave the batch and run their last steps
 *    alone on their own streams, after the batch's queued work;
 *  - the others advance together by E steps, E = min(max_steps, the fewest
 *    steps left of an admitted member), rounded down to whole chunks;
 *  - admitted members whose steps are then done leave the batch.
 * *steps_run (may be NULL) receives E.  It returns without waiting while at
 * most two earlier epochs are still running on the device; otherwise it
 * first waits for the oldest (flow control).  A member's status (e.g. FENE
 * overstretch) surfaces in its own read-backs. */
int prx_batch_step_epoch(prx_batch* b, uint64_t max_steps, uint64_t* steps_run);

/* Reports, without waiting, admitted systems whose steps are all done and
 * whose device work has finished: up to cap slot numbers into done_slots,
 * their count into *n_done (0 when none).  A reported system has left the
 * batch, its slot and budget are free again, and it is back in standalone
 * use: read its results with the prx_get_* calls, then destroy it or keep
 * using it. */
int prx_batch_poll(prx_batch* b, int32_t* done_slots, int32_t cap, int32_t* n_done);

/* Waits for the batch; returns the first non-zero member status (its index
 * in *failed when failed != NULL, else -1 there). */
int prx_batch_sync(prx_batch* b, int32_t* failed);

int prx_batch_stats_get(prx_batch* b, prx_batch_stats* out);
const char* prx_batch_last_error(const prx_batch* b);

/* ---- errors ---------------------------------------------------------------- */
const char* prx_last_error(const prx_system* sys);
const char* prx_status_string(int status);

#ifdef __cplusplus
}
#endif
#endif /* POLYRX_H */
