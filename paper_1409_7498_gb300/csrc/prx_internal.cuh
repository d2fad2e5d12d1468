// Internal layout and device helpers of the polyrx CUDA library.
//
// Data layout in HBM (one system, n particles, slot order = sorted by cell at
// the last rebuild):
//   two SoA sets (the current one and the rebuild target):
//     x, y, z, vx, vy, vz : double[n]   absolute positions, half-step velocities
//     id                  : u32[n]      particle id of the slot
//     type, state, nadj   : u8/i8/u8[n]
//     adj                 : u32[n*cap]  partner slots; bit 31 = bond style
//   P[2] : uint4[n]  periodic fixed-point position X = floor(x / L 2^32) mod
//                    2^32 per axis (the int32 difference of two X is the
//                    minimum-image displacement, exactly, in units L / 2^32),
//                    .w = coarse copy of X at the last list build (3 x 10 bits,
//                    for the displacement trigger); double-buffered across
//                    steps (neighbours read the old copy while the new one is
//                    written)
//   nl  : Verlet neighbour list, column-major [list_cap][n] (list_cap a
//         multiple of 4), entries are the neighbours' slots (16-bit up to
//         65,535 particles, else 32-bit), each list padded with the owner's
//         own slot to a whole stage of four; nn : u8[n] entry counts
//         (without the padding)
//   cell_start : u32[ncell+1]  CSR offsets of the cells (z-major), valid at
//         the last rebuild; used only to build the lists
// A device control block (Ctl) holds the current set / buffer phase, the
// step counter, the rebuild flag and the sticky error status, so that one
// CUDA graph can be replayed without host involvement.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>

#include "../../include/polyrx.h"

namespace prx {

constexpr uint32_t NONE = 0xFFFFFFFFu;
constexpr uint32_t SLOT_MASK = 0x7FFFFFFFu;
constexpr int STEP_THREADS = 128;
constexpr int RX_THREADS = 256;
constexpr int SCAN_TILE = 2048;  // elements per scan tile (256 threads x 8)

// Counter tags of the keyed Philox draws (fourth counter word, low byte).
constexpr uint32_t TAG_THERMO = 1u, TAG_ACCEPT = 2u, TAG_SEL_A = 3u, TAG_SEL_T = 4u,
                   TAG_NEAREST = 5u;

struct SoA {
  double *x, *y, *z, *vx, *vy, *vz;
  uint32_t* id;
  uint8_t* type;
  int8_t* state;
  uint8_t* nadj;
  uint32_t* adj;
};

struct BondRec {
  uint32_t a, t;
  int64_t step;
  uint32_t style, reaction;
};
static_assert(sizeof(BondRec) == sizeof(prx_bond), "bond record layout");

struct HistRec {
  int64_t step;
  int64_t bonds;
  int32_t counts[PRX_MAX_TYPES][PRX_MAX_STATES];
};
static_assert(sizeof(HistRec) == sizeof(prx_history_record), "history record layout");

struct Ctl {
  int set;                  // current SoA set
  int phase;                // current off buffer
  int rebin_flag;           // a particle left its extended cell
  int status;               // sticky PRX_E* status (0 = ok)
  unsigned int done_step;   // last-block counters
  unsigned int done_rebin;
  unsigned int done_rx;
  unsigned int done_obs;
  unsigned long long step;  // completed MD steps
  unsigned long long rebins;
  unsigned long long reactions;
  unsigned long long nbonds;
  unsigned long long hist_count;
  long long trace[4];          // candidates, retained, a_winners, formed
  unsigned int n_active;       // eligible A's of the current reaction step
  unsigned int input_err;      // creation: first bad input kind (1 non-finite
                               // position, 2 outside the box, 3 type >= 8)
  // device-driven runs (dg.cu): steps left in the run, and the device graphs
  // k_dg_next launches (as cudaGraphExec_t values)
  unsigned long long steps_left;
  unsigned long long dg_rebuild, dg_react;
};

constexpr int MAX_RX = PRX_MAX_REACTIONS;
constexpr int POP_REPLICAS = 32;

// The scheme's reactions.  The scalar fields describe reaction 0 and serve
// the single-reaction kernels as before; with nr > 1 (concurrent reactions)
// the kernels take the per-reaction arrays.  A particle is an A of the
// reactions whose A window holds it, a T of those whose T window holds it
// (never both kinds, checked at set-up); a candidate pair's reactions
// partition one acceptance draw: reaction c_j of its candidate set m is taken
// when the draw's 53-bit word is below p53c[m][j] = ceil(P_j 2^53),
// P_j = p_c1 + ... + p_cj summed in FP64 in the scheme's order.
struct RxParams {
  uint32_t mask_A, mask_T;
  int32_t a_lo, a_hi, t_lo, t_hi, dA, dT;
  double p;         // k dt Theta
  uint64_t p53;     // ceil(p 2^53) (2^53 when p >= 1): u < p as an integer test
  double rr2;       // r_react^2 (exact test)
  float rr2_pre;    // (r_react + margin)^2 (FP32 prefilter, always conservative)
  float rr2_in;     // r_react^2 minus twice the FP32 error bound: inside for sure
  uint32_t style;
  int32_t rule;     // PRX_SELECT_RANDOM or PRX_SELECT_NEAREST
  uint8_t maxval[PRX_MAX_TYPES];
  // concurrent reactions (nr > 1)
  int32_t nr;
  uint32_t mA[MAX_RX], mT[MAX_RX];
  int32_t alo[MAX_RX], ahi[MAX_RX], tlo[MAX_RX], thi[MAX_RX], dAr[MAX_RX], dTr[MAX_RX];
  uint32_t styler[MAX_RX];
  uint8_t maxvalr[MAX_RX][PRX_MAX_TYPES];
  double rr2r[MAX_RX];
  uint64_t p53c[1 << MAX_RX][MAX_RX];
};

// Reactions (bit r) whose A window holds a particle of type t in state s,
// and likewise for T.
__device__ __forceinline__ uint32_t rx_elig_A(const RxParams& R, uint32_t t, int s) {
  uint32_t m = 0;
  for (int r = 0; r < R.nr; ++r)
    m |= (((R.mA[r] >> t) & 1u) && s >= R.alo[r] && s <= R.ahi[r]) ? (1u << r) : 0u;
  return m;
}
__device__ __forceinline__ uint32_t rx_elig_T(const RxParams& R, uint32_t t, int s) {
  uint32_t m = 0;
  for (int r = 0; r < R.nr; ++r)
    m |= (((R.mT[r] >> t) & 1u) && s >= R.tlo[r] && s <= R.thi[r]) ? (1u << r) : 0u;
  return m;
}

// A particle class of the pair histogram: type in the mask, state in [lo, hi].
struct PairClass {
  uint32_t mask;
  int32_t lo, hi;
};

// Control block shared by the members of a batch.
struct BatchCtl {
  int any_rebuild;          // some member needs a rebuild after this step
  unsigned int done_step;   // members whose step finished (last-member detection)
  unsigned long long rebuilds;  // steps after which the rebuild pipeline ran
  // device-driven batch runs (dg.cu): the last step's rebuild decision, the
  // steps left, the reaction phase (steps mod theta) and the device graphs
  int rebuild_now;
  int any_rx;
  int dg_err;                   // a device-side graph launch failed
  int pad_;
  unsigned long long steps_left, phase, theta;
  unsigned long long dg_rebuild, dg_react;
};

struct Sys {
  uint32_t n, cap;
  int nc[3];
  int ncell;
  // geometry
  double L[3], halfL[3];
  long long Lfx[3];               // L in 2^-32 units
  unsigned long long M64[3];      // round(2^64 / L): X = hi64((x + L) 2^32 M64)
  float scale[3];                 // L / 2^32 (physical length of one X unit)
  float scale_sq_ref;             // (L_0 / 2^32)^2
  int wshift[3];                  // coarse reference: bits (X >> wshift) & 1023
  float wunit[3];                 // physical length of one coarse unit
  float disp2_max;                // (skin/2 - margin)^2: rebuild when exceeded
  // Verlet list
  void* nl;                       // u16 or u32 entries, [list_cap][n]
  uint8_t* nn;
  int nl16;                       // 1: 16-bit entries
  int list_cap;
  float rv2_build;                // (r_c + skin + rounding margin)^2, list build test (FP32)
  // list-build tiling (cells of edge >= r_c + skin)
  int tile_y, tiles_y, tile_threads, tile_cap;
  // physics (FP32 and FP64 copies)
  float rc2f, sig2f, eps24f, eps4f, fcapf, fkf, fr02f, fr02if, rcf, sigf;
  int cubic;        // equal edges: the neighbour loop runs in position units
  float s2f, rc2u;  // scale^2 and the WCA cutoff^2 in position units^2
  double rc2, sig2, eps24, eps4, fcap, fk, fr02, rc, sig;
  double dt, a_fric, b_kick;  // v' = a v + b F ; x' = x + dt v'
  double gm;                  // gamma m (FP64 mode writes the friction force out)
  double mass;
  float b_kickf, cRf;
  double cR;
  int thermo;                 // gamma > 0
  uint64_t seed;
  // buffers
  SoA s0, s1;
  uint4 *P0, *P1;
  uint32_t* cell_start;
  uint32_t *count, *fill;
  uint32_t *key, *tmp, *new_of_old;
  uint32_t *win, *blk_count, *blk_off;
  uint8_t* wch;             // reaction of each A's chosen pair (concurrent reactions)
  BondRec* bonds;
  unsigned long long bond_cap;
  HistRec* hist;
  unsigned int hist_cap;
  int32_t* pop;             // particles per (type, state), kept current by the reaction
                            // step: POP_REPLICAS arrays of 128 whose sum is the count
  double *fout, *eout;
  double* red;              // per-block partial sums (observables)
  Ctl* ctl;
  // reaction scheme (has_rx = 0: none)
  RxParams R;
  int has_rx;
  // batch membership: in_batch = 1 inside a batched launch; batch = the
  // batch's control block
  int in_batch;
  BatchCtl* batch;
  // launch configuration of the single-system step kernel (host side)
  int step_bt;              // threads per block: 128, 256 or 512
  int step_bpsm;            // blocks per SM of the persistent grid (0: all that fit)
  int step_lanes;           // lanes per slot: 1, or 4 (k_step_nl4, small systems)
  unsigned int n_members;   // members of the batch (last-member detection)
};

// Part of a grid that belongs to one system: local block index and block
// count (the whole grid for a single system).
struct Blk {
  uint32_t b, nb;
};

// One entry of a batched launch's block map: system, local block, block count.
struct BlkMap {
  uint32_t sys, b, nb, pad;
};

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two
// 32x32->64 multiplies by the round constants, a word permutation and a xor
// with the round key, the key advancing by the two Weyl constants.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    k.x += 0x9E3779B9u;
    k.y += 0xBB67AE85u;
  }
  return c;
}

// Counter layout of every keyed draw: (step lo, id a, id b, tag | step hi << 8),
// key = (seed lo, seed hi).
__device__ __forceinline__ uint4 keyed_draw(uint64_t seed, unsigned long long step, uint32_t a,
                                            uint32_t b, uint32_t tag) {
  return philox4x32_10(make_uint4((uint32_t)step, a, b, tag | ((uint32_t)(step >> 32) << 8)),
                       make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
}

// 53-bit uniform in [0,1): top 53 bits of (hi:lo) times 2^-53 (exact).
// ceil(p 2^53) for the integer acceptance test (p 2^53 is exact in binary64).
inline uint64_t p53_of(double p) {
  if (!(p < 1.0)) return 1ull << 53;
  if (!(p > 0.0)) return 0ull;
  return (uint64_t)std::ceil(std::ldexp(p, 53));
}
// u < p for the uniform u = m 2^-53 in [0, 1) of a draw, m = the top 53 bits
// of the 64-bit word w = hi:lo (m = w >> 11), decided on the integer pipe:
// m 2^-53 < p exactly when m < ceil(p 2^53).
__device__ __forceinline__ bool u53_below(uint32_t hi, uint32_t lo, uint64_t p53) {
  return ((((unsigned long long)hi << 32) | lo) >> 11) < p53;
}

// Small unsigned integer v < 2^23 as float, exactly, on the integer and FP32
// pipes: the bit pattern 0x4B000000 | v is the float 2^23 + v.
__device__ __forceinline__ float small_u2f(uint32_t v) {
  return __fsub_rn(__uint_as_float(0x4B000000u | v), 8388608.0f);
}

// 24-bit uniform in [0,1): (w >> 8) 2^-24, exact in float.
__device__ __forceinline__ float u24f(uint32_t w) {
  const uint32_t v = w >> 8;
  const float half = small_u2f(v >> 1);
  return __fmul_rn(__fmaf_rn(half, 2.0f, (v & 1u) ? 1.0f : 0.0f), 0x1.0p-24f);
}

// binary32 -> binary64 by re-biasing the exponent field: exact for normal
// numbers and zero (binary32 subnormals become zero; the kernels run with
// flush-to-zero).  Costs integer operations only, no FP64-pipe instruction.
__device__ __forceinline__ double f2d_exact(float f) {
  const uint32_t u = __float_as_uint(f);
  const uint32_t mag = u & 0x7FFFFFFFu;
  uint32_t hi = (u & 0x80000000u) | ((mag >> 3) + 0x38000000u);
  uint32_t lo = u << 29;
  if (mag < 0x00800000u) {
    hi = u & 0x80000000u;
    lo = 0u;
  }
  return __hiloint2double((int)hi, (int)lo);
}

// trunc(x * 2^32) for |x| < 2^29, read off the binary64 fields (integer pipe).
__device__ __forceinline__ long long fx32(double x) {
  const long long b = __double_as_longlong(x);
  const int e = (int)((b >> 52) & 0x7FF);
  const long long m = (b & 0x000FFFFFFFFFFFFFLL) | 0x0010000000000000LL;
  const int sh = 1043 - e;  // x 2^32 = m 2^(e - 1075 + 32)
  // |x| >= 2^29 (or inf/nan) saturates to 2^62: far outside any cell, which
  // the callers report as an error
  long long r = (sh >= 63) ? 0LL : (sh >= 0 ? (m >> sh) : (sh >= -9 ? (m << (-sh)) : (1LL << 62)));
  return (b < 0) ? -r : r;
}

// Periodic fixed point of a coordinate: floor(x / L 2^32) mod 2^32, from
// the binary64 fields and one 64x64 high multiply (integer pipe only).
// Valid for -L < x < 2^29.
__device__ __forceinline__ uint32_t periodic_fx(double x, long long Lfx, unsigned long long M) {
  const unsigned long long a = (unsigned long long)(fx32(x) + Lfx);
  return (uint32_t)__umul64hi(a, M);
}

// Minimum-image displacement X_j - X_i of two periodic coordinates, in X units.
__device__ __forceinline__ int pdiff(uint32_t xj, uint32_t xi) { return (int)(xj - xi); }

__device__ __forceinline__ uint32_t coarse_ref(uint32_t X, uint32_t Y, uint32_t Z, const int* sh) {
  return ((X >> sh[0]) & 1023u) | (((Y >> sh[1]) & 1023u) << 10) | (((Z >> sh[2]) & 1023u) << 20);
}

__device__ __forceinline__ int wrap_cell(int q, int n) { return q < 0 ? q + n : (q >= n ? q - n : q); }

__device__ __forceinline__ void set_status(Ctl* ctl, int code) { atomicCAS(&ctl->status, 0, code); }

// Minimum image of one FP64 separation component by compare-and-shift.
__device__ __forceinline__ double min_image(double d, double L, double half) {
  if (d > half) return __dsub_rn(d, L);
  if (d < -half) return __dadd_rn(d, L);
  return d;
}

// Block maps of a batched launch, one per kernel family (device arrays).
struct BatchLaunch {
  const Sys* T;             // member table
  const BlkMap *part, *cell, *tile, *one, *build;
  unsigned n_part, n_cell, n_tile, n_one, n_build;
  int build_threads;
  size_t build_smem;
  // rebuild work of the members whose flag is set, compacted each rebuild
  // step: the same five families (part, cell, tile, one, build) at the same
  // offsets as the full maps, and their entry counts (zeroed by the step)
  BlkMap* act;
  uint32_t* act_n;
  // the part map is ordered by step-kernel variant (nl16, cubic): 00, 01,
  // 10, 11; the blocks of variant v are part[step_off[v] .. + step_n[v])
  unsigned step_off[4], step_n[4];
};

// ---- host-side launchers (defined in the kernel translation units) ----------
void launch_batch_step(const BatchLaunch& L, cudaStream_t st, cudaGraphConditionalHandle h,
                       int use_cond);
void launch_batch_rebuild(const BatchLaunch& L, cudaStream_t st);
void launch_batch_rx(const BatchLaunch& L, cudaStream_t st);
int configure_batch_build_kernel(size_t smem_bytes);
int batch_rebuild_kernel_count();
int batch_rx_kernel_count();
void launch_step(const Sys& S, cudaStream_t st, int fp64, int forces_only,
                 cudaGraphConditionalHandle h, int use_cond);
void launch_rebin(const Sys& S, cudaStream_t st, int mode, void (*hook)(void*, const char*, int),
                  void* hook_ctx);
void launch_rx(const Sys& S, cudaStream_t st, long long step_arg,
               void (*hook)(void*, const char*, int), void* hook_ctx);
void launch_observables(const Sys& S, cudaStream_t st, int nblocks);
// Counts the populations per (type, state) into S.pop (creation).
void launch_pop_init(const Sys& S, cudaStream_t st);
void launch_pair_hist(const Sys& S, cudaStream_t st, const PairClass& a, const PairClass& b,
                      const double* e2, int nbins, unsigned long long* counts,
                      unsigned long long* nab);
int rebin_kernel_count(const Sys& S);
int rx_kernel_count(int rule);
int step_kernel_count(int fp64);
size_t build_tile_smem(const Sys& S);
// Creation without a saved slot order: particle p goes to slot p.  `buf`
// holds the caller's (n, 3) positions (which = 0: validated, wrapped once
// into the box, ids and types checked) or velocities (which = 1), copied to
// the device; errors land in ctl->input_err.
void launch_stage_input(const Sys& S, cudaStream_t st, const double* buf, int which);
// Per-particle arrays in particle (id) order into device buffer `out`:
// 0 states, 1 types, 2 positions wrapped into the box, 3 velocities.
void launch_gather_by_id(const Sys& S, cudaStream_t st, int what, void* out);
int configure_build_kernel(size_t smem_bytes);
// Device-driven runs (dg.cu): k_dg_arm stores the run's step count and the
// rebuild and reaction device graphs in the control block; k_dg_next, the
// last kernel of the step's device graph, tail-launches what follows.
void launch_dg_arm(const Sys& S, cudaStream_t st, unsigned long long steps,
                   unsigned long long rebuild, unsigned long long react);
void launch_dg_next(const Sys& S, cudaStream_t st, unsigned int theta);
// The same for a batch: k_dgb_next follows the batch's step kernels.
void launch_dgb_arm(BatchCtl* c, cudaStream_t st, unsigned long long steps, unsigned long long phase,
                    unsigned long long theta, int any_rx, unsigned long long rebuild,
                    unsigned long long react);
void launch_dgb_next(BatchCtl* c, cudaStream_t st);

}  // namespace prx
