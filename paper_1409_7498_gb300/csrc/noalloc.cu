// Reaction step on caller-owned device arrays, with no device allocation.
//
// Some callers cannot call cudaMalloc at all: code that runs against a fixed
// memory budget handed out by a host framework, or inside an allocator hook
// where allocating again would re-enter the allocator.  prx_react_noalloc
// serves them: inputs and outputs are the caller's device buffers, and the
// only scratch (per-particle choices and a few counters) lives in one
// file-scope __device__ array of fixed size, held by every GPU that loads the
// library until the process exits.
//
// The candidate search is all-pairs (at most PRX_NOALLOC_MAX_N particles), so
// no cell list or neighbour list is needed.  Both selection rules of
// prx_react_once are implemented with its keyed Philox draws, its FP64
// distance test and its tie-breaking, so the two agree bit for bit on the
// same state: Table I's random rule (one T per A, then one A per T, each the
// smallest selection key) and the LAMMPS nearest-partner rule of Sec. IV.A
// (mutual nearest A-T pairs, then the acceptance draw).
#include <cuda_runtime.h>

#include <mutex>

#include "prx_internal.cuh"

namespace {

using namespace prx;

struct NaScratch {
  uint32_t win[PRX_NOALLOC_MAX_N];  // random rule: chosen T of each A (Table I step 5);
                                    // nearest rule: nearest partner of each A and T
  uint32_t fin[PRX_NOALLOC_MAX_N];  // surviving pairs (step 7), by A
  unsigned long long trace[4];
  unsigned int nbonds;
  int status;
};

// The scratch.  Every call shares it and it keeps the last call's contents;
// the counters are cleared at the start of each call and win/fin are fully
// rewritten.  Calls whose work overlaps on the GPU race on it.
static __device__ __align__(256) NaScratch g_na_scratch;

struct NaArgs {
  uint32_t n, cap;
  double L[3], halfL[3];
  const double* pos;
  const uint8_t* type;
  int8_t* state;
  uint8_t* nadj;
  uint32_t* adj;
  prx_bond* bonds;
  uint32_t bonds_cap;
  uint32_t* nbonds_out;
  uint64_t seed;
  unsigned long long step;
  RxParams R;
  NaScratch* sc;
};

__device__ __forceinline__ bool na_window(uint32_t mask, int lo, int hi, uint32_t t, int s) {
  return ((mask >> t) & 1u) && s >= lo && s <= hi;
}

__device__ __forceinline__ unsigned long long na_key64(uint4 w) {
  return ((unsigned long long)w.x << 32) | w.y;
}

// Exact FP64 test of Table I step 1 for the pair (i, j): the minimum-image
// separation x_j - x_i, r^2 = fma(dz, dz, fma(dy, dy, dx dx)), strict
// r^2 < r_react^2.  Returns r^2, or a negative value when out of range.
__device__ __forceinline__ double na_r2(const NaArgs& a, uint32_t i, uint32_t j, double xi,
                                        double yi, double zi) {
  const double dx = min_image(__dsub_rn(a.pos[3 * (size_t)j], xi), a.L[0], a.halfL[0]);
  const double dy = min_image(__dsub_rn(a.pos[3 * (size_t)j + 1], yi), a.L[1], a.halfL[1]);
  const double dz = min_image(__dsub_rn(a.pos[3 * (size_t)j + 2], zi), a.L[2], a.halfL[2]);
  const double r2 = __fma_rn(dz, dz, __fma_rn(dy, dy, __dmul_rn(dx, dx)));
  return r2 < a.R.rr2 ? r2 : -1.0;
}

__device__ __forceinline__ bool na_bonded(const NaArgs& a, uint32_t i, uint32_t j) {
  const uint32_t nb = a.nadj[i];
  bool bonded = false;
  for (uint32_t b = 0; b < nb; ++b) bonded |= (a.adj[(size_t)i * a.cap + b] & SLOT_MASK) == j;
  return bonded;
}

// LAMMPS rule (Sec. IV.A): the eligible partner of the other kind (a T when
// want_T, else an A) within r_react of particle i, not bonded to it, of
// smallest exact r^2, ties to the smaller id; in_range counts the pairs in
// range.
__device__ __forceinline__ uint32_t na_nearest(const NaArgs& a, uint32_t i, bool want_T,
                                               unsigned long long& in_range) {
  const double xi = a.pos[3 * (size_t)i], yi = a.pos[3 * (size_t)i + 1], zi = a.pos[3 * (size_t)i + 2];
  uint32_t best = NONE;
  double best_r2 = 0.0;
  for (uint32_t j = 0; j < a.n; ++j) {
    if (j == i) continue;
    const bool ok = want_T ? na_window(a.R.mask_T, a.R.t_lo, a.R.t_hi, a.type[j], a.state[j])
                           : na_window(a.R.mask_A, a.R.a_lo, a.R.a_hi, a.type[j], a.state[j]);
    if (!ok) continue;
    const double r2 = na_r2(a, i, j, xi, yi, zi);
    if (r2 < 0.0 || na_bonded(a, i, j)) continue;
    ++in_range;
    // j ascends, so a tie keeps the earlier (smaller) id
    if (best == NONE || r2 < best_r2) {
      best = j;
      best_r2 = r2;
    }
  }
  return best;
}

// Steps 1-5, one thread per particle id, all pairs (random rule); for the
// nearest rule each eligible A records its nearest eligible T.
__global__ void k_na_find(NaArgs a) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.n) return;
  uint32_t best = NONE;
  unsigned long long cand = 0, ret = 0;
  const bool isA = na_window(a.R.mask_A, a.R.a_lo, a.R.a_hi, a.type[i], a.state[i]);
  if (isA && a.R.rule == PRX_SELECT_NEAREST) {
    best = na_nearest(a, i, true, cand);
  } else if (isA) {
    const double xi = a.pos[3 * (size_t)i], yi = a.pos[3 * (size_t)i + 1], zi = a.pos[3 * (size_t)i + 2];
    unsigned long long bestkey = 0ull;
    for (uint32_t j = 0; j < a.n; ++j) {
      if (j == i || !na_window(a.R.mask_T, a.R.t_lo, a.R.t_hi, a.type[j], a.state[j])) continue;
      if (na_r2(a, i, j, xi, yi, zi) < 0.0 || na_bonded(a, i, j)) continue;
      ++cand;
      const uint4 wa = keyed_draw(a.seed, a.step, i, j, TAG_ACCEPT);
      if (!u53_below(wa.x, wa.y, a.R.p53)) continue;
      ++ret;
      const unsigned long long k = na_key64(keyed_draw(a.seed, a.step, i, j, TAG_SEL_A));
      if (best == NONE || k < bestkey || (k == bestkey && j < best)) {
        best = j;
        bestkey = k;
      }
    }
  }
  a.sc->win[i] = best;
  if (cand) atomicAdd(&a.sc->trace[0], cand);
  if (ret) atomicAdd(&a.sc->trace[1], ret);
}

// Nearest rule: each eligible T records its nearest eligible A.  A and T
// are disjoint sets, so the two kinds share win[].
__global__ void k_na_find_T(NaArgs a) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.n || !na_window(a.R.mask_T, a.R.t_lo, a.R.t_hi, a.type[i], a.state[i])) return;
  unsigned long long unused = 0;
  a.sc->win[i] = na_nearest(a, i, false, unused);
}

// Steps 6-7 (random rule): an A keeps its T only if its key
// Philox(step, id_T, id_A) is the smallest among the A's that chose the same
// T.  Nearest rule: an A and the T it picked react when the T picked it too
// and u < k dt Theta, drawn with the pair's smaller id first.
__global__ void k_na_select(NaArgs a) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.n) return;
  const uint32_t T = a.sc->win[i];
  uint32_t fin = NONE;
  const bool isA = na_window(a.R.mask_A, a.R.a_lo, a.R.a_hi, a.type[i], a.state[i]);
  if (T != NONE && isA && a.R.rule == PRX_SELECT_NEAREST) {
    if (a.sc->win[T] == i) {
      atomicAdd(&a.sc->trace[1], 1ull);  // mutual pairs
      const uint4 w = keyed_draw(a.seed, a.step, min(i, T), max(i, T), TAG_NEAREST);
      if (u53_below(w.x, w.y, a.R.p53)) {
        atomicAdd(&a.sc->trace[2], 1ull);  // accepted pairs
        fin = T;
      }
    }
  } else if (T != NONE && isA) {
    atomicAdd(&a.sc->trace[2], 1ull);
    const unsigned long long mine = na_key64(keyed_draw(a.seed, a.step, T, i, TAG_SEL_T));
    bool keep = true;
    for (uint32_t k = 0; k < a.n && keep; ++k) {
      if (k == i || a.sc->win[k] != T) continue;
      const unsigned long long other = na_key64(keyed_draw(a.seed, a.step, T, k, TAG_SEL_T));
      if (other < mine || (other == mine && k < i)) keep = false;
    }
    if (keep) fin = T;
  }
  a.sc->fin[i] = fin;
}

// Step 9 in one block: bonds appended in ascending id of A (a running count
// over the ids, no atomics), adjacency rows and states updated.  A pair that
// would exceed a particle's valence forms no bond and takes no place in the
// bond list (status PRX_ECAPACITY); the surviving pairs are all counted in
// the trace, as prx_react_once counts them.  Each A and each T is in at most
// one pair, so the valence reads see the rows as they were before this step.
__global__ void k_na_apply(NaArgs a) {
  __shared__ uint32_t wtot[32];
  __shared__ uint32_t carry, surv;
  if (threadIdx.x == 0) carry = surv = 0u;
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (uint32_t base = 0; base < a.n; base += blockDim.x) {
    const uint32_t i = base + threadIdx.x;
    const uint32_t T = i < a.n ? a.sc->fin[i] : NONE;
    bool has = false;
    uint32_t na = 0, nt = 0;
    if (T != NONE) {
      const uint32_t ta = a.type[i], tt = a.type[T];
      const uint32_t capA = a.R.maxval[ta] < a.cap ? a.R.maxval[ta] : a.cap;
      const uint32_t capT = a.R.maxval[tt] < a.cap ? a.R.maxval[tt] : a.cap;
      na = a.nadj[i];
      nt = a.nadj[T];
      has = na < capA && nt < capT;
      if (!has) atomicCAS(&a.sc->status, 0, PRX_ECAPACITY);
    }
    const uint32_t sbal = __ballot_sync(0xFFFFFFFFu, T != NONE);
    if (lane == 0 && sbal) atomicAdd(&surv, __popc(sbal));
    const uint32_t bal = __ballot_sync(0xFFFFFFFFu, has);
    if (lane == 0) wtot[wid] = __popc(bal);
    __syncthreads();
    uint32_t before = carry;
    for (int w = 0; w < wid; ++w) before += wtot[w];
    const uint32_t pos = before + __popc(bal & ((1u << lane) - 1u));
    if (has) {
      if (pos >= a.bonds_cap) {
        atomicCAS(&a.sc->status, 0, PRX_ECAPACITY);
      } else {
        const uint32_t sbit = a.R.style << 31;
        a.adj[(size_t)i * a.cap + na] = T | sbit;
        a.nadj[i] = (uint8_t)(na + 1);
        a.adj[(size_t)T * a.cap + nt] = i | sbit;
        a.nadj[T] = (uint8_t)(nt + 1);
        a.state[i] = (int8_t)(a.state[i] + a.R.dA);
        a.state[T] = (int8_t)(a.state[T] + a.R.dT);
        prx_bond b;
        b.a = i;
        b.t = T;
        b.step = (int64_t)a.step;
        b.style = a.R.style;
        b.reaction = 0u;
        a.bonds[pos] = b;
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      uint32_t t = 0;
      for (int w = 0; w < nw; ++w) t += wtot[w];
      carry += t;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const uint32_t formed = carry < a.bonds_cap ? carry : a.bonds_cap;
    a.sc->nbonds = formed;
    a.sc->trace[3] = surv;
    *a.nbonds_out = formed;
  }
}

std::mutex g_na_mutex;
NaScratch* g_na_addr[256];
bool g_na_ready[256];

// Device address of the scratch on the current device.  The first call on a
// device looks it up (with that device current); later calls reuse it.
int na_scratch(NaScratch** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) return PRX_ECUDA;
  std::lock_guard<std::mutex> lock(g_na_mutex);
  if (!g_na_ready[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_na_scratch) != cudaSuccess || !p) return PRX_ECUDA;
    g_na_addr[dev] = static_cast<NaScratch*>(p);
    g_na_ready[dev] = true;
  }
  *out = g_na_addr[dev];
  return PRX_OK;
}

}  // namespace

extern "C" int prx_react_noalloc(const prx_reaction_desc* rx, const double* box, double dt,
                                 uint64_t seed, uint64_t step, uint32_t n, const double* d_pos,
                                 const uint8_t* d_type, int8_t* d_state, uint32_t adj_cap,
                                 uint8_t* d_nadj, uint32_t* d_adj, prx_bond* d_bonds_out,
                                 uint32_t bonds_cap, uint32_t* d_nbonds_out, void* cuda_stream,
                                 prx_rx_trace* trace) {
  if (n > PRX_NOALLOC_MAX_N) return PRX_ECAPACITY;  // beyond the static scratch
  if (!rx || !box || !d_nbonds_out || !(dt > 0.0)) return PRX_EINVAL;
  if (adj_cap < 1 || adj_cap > PRX_MAX_ADJ) return PRX_EINVAL;
  if (n && (!d_pos || !d_type || !d_state || !d_nadj || !d_adj || (bonds_cap && !d_bonds_out)))
    return PRX_EINVAL;
  if (rx->a_lo > rx->a_hi || rx->t_lo > rx->t_hi || rx->theta < 1 || !(rx->k >= 0.0) ||
      !(rx->r_react > 0.0) || (rx->bond_style != PRX_BOND_FENE && rx->bond_style != PRX_BOND_MIRROR_LJ) ||
      ((rx->type_mask_A | rx->type_mask_T) >> PRX_MAX_TYPES) ||
      (rx->selection != PRX_SELECT_RANDOM && rx->selection != PRX_SELECT_NEAREST) ||
      ((rx->type_mask_A & rx->type_mask_T) && !(rx->a_hi < rx->t_lo || rx->t_hi < rx->a_lo)))
    return PRX_EINVAL;
  for (int k = 0; k < 3; ++k)
    if (!(box[k] > 0.0)) return PRX_EINVAL;
  NaScratch* sc = nullptr;
  int rc = na_scratch(&sc);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)cuda_stream;

  NaArgs a;
  a.R = RxParams{};
  a.R.nr = 1;
  a.n = n;
  a.cap = adj_cap;
  for (int k = 0; k < 3; ++k) {
    a.L[k] = box[k];
    a.halfL[k] = 0.5 * box[k];
  }
  a.pos = d_pos;
  a.type = d_type;
  a.state = d_state;
  a.nadj = d_nadj;
  a.adj = d_adj;
  a.bonds = d_bonds_out;
  a.bonds_cap = bonds_cap;
  a.nbonds_out = d_nbonds_out;
  a.seed = seed;
  a.step = step;
  a.R.mask_A = rx->type_mask_A;
  a.R.mask_T = rx->type_mask_T;
  a.R.a_lo = rx->a_lo;
  a.R.a_hi = rx->a_hi;
  a.R.t_lo = rx->t_lo;
  a.R.t_hi = rx->t_hi;
  a.R.dA = rx->dA;
  a.R.dT = rx->dT;
  a.R.p = rx->k * dt * (double)rx->theta;
  a.R.p53 = p53_of(a.R.p);
  a.R.rr2 = rx->r_react * rx->r_react;
  a.R.rr2_pre = 0.f;
  a.R.style = (uint32_t)rx->bond_style;
  a.R.rule = rx->selection;
  for (int t = 0; t < PRX_MAX_TYPES; ++t) a.R.maxval[t] = rx->max_valence[t];
  a.sc = sc;

  // counters and status start at zero on every call
  if (cudaMemsetAsync(&sc->trace[0], 0, sizeof(sc->trace) + sizeof(sc->nbonds) + sizeof(sc->status),
                      st) != cudaSuccess)
    return PRX_ECUDA;
  const unsigned g = n ? (n + 255u) / 256u : 1u;
  k_na_find<<<g, 256, 0, st>>>(a);
  if (a.R.rule == PRX_SELECT_NEAREST) k_na_find_T<<<g, 256, 0, st>>>(a);
  k_na_select<<<g, 256, 0, st>>>(a);
  k_na_apply<<<1, 1024, 0, st>>>(a);
  if (cudaGetLastError() != cudaSuccess) return PRX_ECUDA;
  unsigned long long tr[4];
  int status = 0;
  if (cudaMemcpyAsync(tr, &sc->trace[0], sizeof(tr), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaMemcpyAsync(&status, &sc->status, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return PRX_ECUDA;
  if (trace) {
    trace->candidates = (int64_t)tr[0];
    trace->retained = (int64_t)tr[1];
    trace->a_winners = (int64_t)tr[2];
    trace->formed = (int64_t)tr[3];
  }
  return status;
}
