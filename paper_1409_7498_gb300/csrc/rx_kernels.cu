// Reaction step (Sec. III, Table I) and observables.
//
// The three selection stages are atomic-free and independent of thread
// scheduling: every random choice is the minimum of Philox keys that depend
// only on (seed, step, particle ids), so the outcome is a function of the
// state alone.
//   rx_find      steps 1-5: each eligible A scans its 27 neighbour cells for
//                eligible T (type mask, state window, not yet bonded to A) with
//                r^2 < r_react^2 tested in FP64 on absolute positions (after an
//                FP32 prefilter that can only widen the set), accepts each with
//                u < k dt Theta (Eq. 4) and keeps the accepted T of smallest
//                key Philox(step, id_A, id_T): one T per A.
//   rx_select_T  steps 6-7: each A winner scans the cells around its T for the
//                other A's that picked the same T and keeps the pair only if
//                its key Philox(step, id_T, id_A) is the smallest: one A per T.
//   rx_select_apply  steps 6-9 fused: one A per T, then the bonds, both
//                adjacency rows and the states; the running populations per
//                (type, state) move with each bond, and the last block writes
//                the reaction's history record from them.
#include <cuda_runtime.h>

#include "prx_internal.cuh"

namespace prx {

namespace {

__device__ __forceinline__ bool in_window(uint32_t mask, int lo, int hi, uint32_t t, int s) {
  return ((mask >> t) & 1u) && s >= lo && s <= hi;
}

// One particle of type t moves from state s0 to s1 in the block's
// population changes (states outside 0..15 are not counted).
__device__ __forceinline__ void pop_move(int32_t* dpop, uint32_t t, int s0, int s1) {
  if (t >= PRX_MAX_TYPES) return;
  if (s0 >= 0 && s0 < PRX_MAX_STATES) atomicSub(&dpop[t * PRX_MAX_STATES + s0], 1);
  if (s1 >= 0 && s1 < PRX_MAX_STATES) atomicAdd(&dpop[t * PRX_MAX_STATES + s1], 1);
}

__device__ __forceinline__ unsigned long long key64(uint4 w) {
  return ((unsigned long long)w.x << 32) | w.y;
}

__device__ __forceinline__ bool last_block_rx(unsigned int* counter, uint32_t nb) {
  __shared__ bool is_last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    is_last = (atomicAdd(counter, 1u) == nb - 1);
  }
  __syncthreads();
  return is_last && threadIdx.x == 0;
}

__device__ __forceinline__ long long block_sum_ll(long long v) {
  __shared__ long long part[RX_THREADS / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xFFFFFFFFu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) part[wid] = v;
  __syncthreads();
  long long t = 0;
  if (threadIdx.x == 0)
    for (int w = 0; w < RX_THREADS / 32; ++w) t += part[w];
  return t;
}

template <bool NL16>
__device__ __forceinline__ uint32_t nl_get_rx(const Sys& S, int k, uint32_t i) {
  if constexpr (NL16) return ((const uint16_t*)S.nl)[(size_t)k * S.n + i];
  else return ((const uint32_t*)S.nl)[(size_t)k * S.n + i];
}

// Work list of the eligible A's (their order does not matter: each A's
// result goes to its own slot), and win[] cleared for every slot.
__device__ __forceinline__ void rx_compact_body(const Sys& S, const Blk blk) {
  const RxParams& R = S.R;

  Ctl* ctl = S.ctl;
  const SoA B = ctl->set ? S.s1 : S.s0;
  const uint32_t i = blk.b * blockDim.x + threadIdx.x;
  bool el = false;
  if (i < S.n) {
    S.win[i] = NONE;
    el = R.nr > 1 ? rx_elig_A(R, B.type[i], B.state[i]) != 0u
                  : in_window(R.mask_A, R.a_lo, R.a_hi, B.type[i], B.state[i]);
  }
  // one atomic per block: warp ballots, block prefix in shared memory
  __shared__ uint32_t wcnt[RX_THREADS / 32];
  __shared__ uint32_t bbase;
  const uint32_t bal = __ballot_sync(0xFFFFFFFFu, el);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) wcnt[wid] = __popc(bal);
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t t = 0;
    for (int w = 0; w < RX_THREADS / 32; ++w) {
      const uint32_t c = wcnt[w];
      wcnt[w] = t;
      t += c;
    }
    bbase = t ? atomicAdd(&ctl->n_active, t) : 0u;
  }
  __syncthreads();
  if (el) S.tmp[bbase + wcnt[wid] + __popc(bal & ((1u << lane) - 1u))] = i;
}

// The compaction of a single system: four slots per thread (one 4-byte load
// of types and one of states, one 16-byte clear of win), so a quarter of
// the blocks and of the block-level atomics on the work-list counter.  The
// list's order differs from rx_compact_body's, which does not matter.
__global__ void __launch_bounds__(RX_THREADS) k_rx_compact4(Sys S) {
  const RxParams& R = S.R;
  Ctl* ctl = S.ctl;
  const SoA B = ctl->set ? S.s1 : S.s0;
  const uint32_t i0 = (blockIdx.x * blockDim.x + threadIdx.x) * 4u;
  uint32_t bits = 0u;
  if (i0 + 3u < S.n) {
    const uchar4 t4 = *reinterpret_cast<const uchar4*>(B.type + i0);
    const char4 s4 = *reinterpret_cast<const char4*>(B.state + i0);
    *reinterpret_cast<uint4*>(S.win + i0) = make_uint4(NONE, NONE, NONE, NONE);
    const uint32_t tt[4] = {t4.x, t4.y, t4.z, t4.w};
    const int ss[4] = {s4.x, s4.y, s4.z, s4.w};
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const bool el = R.nr > 1 ? rx_elig_A(R, tt[u], ss[u]) != 0u
                               : in_window(R.mask_A, R.a_lo, R.a_hi, tt[u], ss[u]);
      bits |= (el ? 1u : 0u) << u;
    }
  } else {
    for (uint32_t u = 0; u < 4u && i0 + u < S.n; ++u) {
      const uint32_t i = i0 + u;
      S.win[i] = NONE;
      const bool el = R.nr > 1 ? rx_elig_A(R, B.type[i], B.state[i]) != 0u
                               : in_window(R.mask_A, R.a_lo, R.a_hi, B.type[i], B.state[i]);
      bits |= (el ? 1u : 0u) << u;
    }
  }
  // warp inclusive scan of the counts, block prefix in shared memory, one
  // atomic per block
  const uint32_t c = __popc(bits);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint32_t x = c;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
    if (lane >= o) x += y;
  }
  __shared__ uint32_t wcnt[RX_THREADS / 32];
  __shared__ uint32_t bbase;
  if (lane == 31) wcnt[wid] = x;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t t = 0;
    for (int w = 0; w < RX_THREADS / 32; ++w) {
      const uint32_t v = wcnt[w];
      wcnt[w] = t;
      t += v;
    }
    bbase = t ? atomicAdd(&ctl->n_active, t) : 0u;
  }
  __syncthreads();
  uint32_t pos = bbase + wcnt[wid] + x - c;
  for (uint32_t u = 0; u < 4u; ++u)
    if ((bits >> u) & 1u) S.tmp[pos++] = i0 + u;
}

__global__ void __launch_bounds__(RX_THREADS)
    kb_rx_compact(const Sys* __restrict__ T, const BlkMap* __restrict__ M) {
  const BlkMap m = M[blockIdx.x];
  const Sys& S = T[m.sys];
  if (!S.has_rx) return;  // this member has no reaction scheme
  rx_compact_body(S, Blk{m.b, m.nb});
}

// LAMMPS rule (Sec. IV.A): the eligible partner of the other kind (a T when
// want_T, else an A) within r_react of slot i, not bonded to it, of smallest
// exact r^2 (ties to the smaller id); `in_range` counts the pairs in range.
template <bool NL16>
__device__ __forceinline__ uint32_t nearest_partner(const Sys& S, const SoA& B, const uint4* P,
                                                    uint32_t i, bool want_T, long long& in_range) {
  const RxParams& R = S.R;
  const uint4 pi = P[i];
  const double xi = B.x[i], yi = B.y[i], zi = B.z[i];
  const uint32_t nb = B.nadj[i];
  uint32_t best = NONE, bestid = 0u;
  double best_r2 = 0.0;
  const int cnt = S.nn[i];
  for (int k = 0; k < cnt; ++k) {
    const uint32_t j = nl_get_rx<NL16>(S, k, i);
    // distance prefilter first (as in the random rule's search)
    const uint4 pj = P[j];
    const float ex = __int2float_rn(pdiff(pj.x, pi.x)) * S.scale[0];
    const float ey = __int2float_rn(pdiff(pj.y, pi.y)) * S.scale[1];
    const float ez = __int2float_rn(pdiff(pj.z, pi.z)) * S.scale[2];
    if (!(fmaf(ez, ez, fmaf(ey, ey, ex * ex)) < R.rr2_pre)) continue;
    const bool ok = want_T ? in_window(R.mask_T, R.t_lo, R.t_hi, B.type[j], B.state[j])
                           : in_window(R.mask_A, R.a_lo, R.a_hi, B.type[j], B.state[j]);
    if (!ok) continue;
    const double ddx = min_image(__dsub_rn(B.x[j], xi), S.L[0], S.halfL[0]);
    const double ddy = min_image(__dsub_rn(B.y[j], yi), S.L[1], S.halfL[1]);
    const double ddz = min_image(__dsub_rn(B.z[j], zi), S.L[2], S.halfL[2]);
    const double r2 = __fma_rn(ddz, ddz, __fma_rn(ddy, ddy, __dmul_rn(ddx, ddx)));
    if (!(r2 < R.rr2)) continue;
    bool bonded = false;
    for (uint32_t b = 0; b < nb; ++b) bonded |= (B.adj[(size_t)i * S.cap + b] & SLOT_MASK) == j;
    if (bonded) continue;
    ++in_range;
    const uint32_t idj = B.id[j];
    if (best == NONE || r2 < best_r2 || (r2 == best_r2 && idj < bestid)) {
      best = j;
      best_r2 = r2;
      bestid = idj;
    }
  }
  return best;
}

// Table I steps 2 and 5 for one candidate pair (A = idi, T = slot j):
// retained when u < k dt Theta (Eq. 4), then the smallest selection key wins
// (ties to the smaller id).
__device__ __forceinline__ void rx_accept_and_key(const Sys& S, const SoA& B,
                                                  unsigned long long step, uint32_t idi, uint32_t j,
                                                  uint64_t p53, long long& nret, uint32_t& best,
                                                  unsigned long long& bestkey, uint32_t& bestid) {
  const uint32_t idj = B.id[j];
  const uint4 wa = keyed_draw(S.seed, step, idi, idj, TAG_ACCEPT);
  if (!u53_below(wa.x, wa.y, p53)) return;
  ++nret;
  const unsigned long long key = key64(keyed_draw(S.seed, step, idi, idj, TAG_SEL_A));
  if (best == NONE || key < bestkey || (key == bestkey && idj < bestid)) {
    best = j;
    bestkey = key;
    bestid = idj;
  }
}

// Steps 1-5 for one eligible A of a scheme of concurrent reactions: its
// candidate pairs, each with its set m of candidate reactions (A and T in the
// reaction's windows, exact FP64 r^2 below the reaction's cutoff, not
// bonded), one acceptance draw against the cumulative bounds of m, and the
// retained pair of smallest selection key.  `ch` receives the chosen pair's
// reaction.
template <bool NL16>
__device__ __forceinline__ uint32_t rx_find_multi(const Sys& S, const SoA& B, const uint4* P,
                                                  unsigned long long step, uint32_t i,
                                                  long long& ncand, long long& nret, uint32_t& ch) {
  const RxParams& R = S.R;
  const uint32_t elA = rx_elig_A(R, B.type[i], B.state[i]);
  const uint4 pi = P[i];
  const uint32_t idi = B.id[i];
  const uint32_t nb = B.nadj[i];
  uint32_t best = NONE, bestid = 0u;
  unsigned long long bestkey = 0ull;
  const int cnt = S.nn[i];
  for (int k = 0; k < cnt; ++k) {
    const uint32_t j = nl_get_rx<NL16>(S, k, i);
    const uint4 pj = P[j];
    const float ex = __int2float_rn(pdiff(pj.x, pi.x)) * S.scale[0];
    const float ey = __int2float_rn(pdiff(pj.y, pi.y)) * S.scale[1];
    const float ez = __int2float_rn(pdiff(pj.z, pi.z)) * S.scale[2];
    if (!(fmaf(ez, ez, fmaf(ey, ey, ex * ex)) < R.rr2_pre)) continue;  // beyond every cutoff
    const uint32_t el = elA & rx_elig_T(R, B.type[j], B.state[j]);
    if (!el) continue;
    const double ddx = min_image(__dsub_rn(B.x[j], B.x[i]), S.L[0], S.halfL[0]);
    const double ddy = min_image(__dsub_rn(B.y[j], B.y[i]), S.L[1], S.halfL[1]);
    const double ddz = min_image(__dsub_rn(B.z[j], B.z[i]), S.L[2], S.halfL[2]);
    const double r2 = __fma_rn(ddz, ddz, __fma_rn(ddy, ddy, __dmul_rn(ddx, ddx)));
    uint32_t m = 0u;
    for (int r = 0; r < R.nr; ++r)
      if (((el >> r) & 1u) && r2 < R.rr2r[r]) m |= 1u << r;
    if (!m) continue;
    bool bonded = false;
    for (uint32_t b = 0; b < nb; ++b) bonded |= (B.adj[(size_t)i * S.cap + b] & SLOT_MASK) == j;
    if (bonded) continue;
    ++ncand;
    const uint32_t idj = B.id[j];
    const uint4 wa = keyed_draw(S.seed, step, idi, idj, TAG_ACCEPT);
    const unsigned long long u53 = (((unsigned long long)wa.x << 32) | wa.y) >> 11;
    int c = -1, q = 0;
    for (int r = 0; r < R.nr && c < 0; ++r) {
      if (!((m >> r) & 1u)) continue;
      if (u53 < R.p53c[m][q]) c = r;
      ++q;
    }
    if (c < 0) continue;
    ++nret;
    const unsigned long long key = key64(keyed_draw(S.seed, step, idi, idj, TAG_SEL_A));
    if (best == NONE || key < bestkey || (key == bestkey && idj < bestid)) {
      best = j;
      bestkey = key;
      bestid = idj;
      ch = (uint32_t)c;
    }
  }
  return best;
}

// Steps 1-5 for the single-reaction random rule, over the work list of
// eligible A's (grid-stride).  An A's Verlet list holds every particle within
// the list cutoff, which includes r_react, hence every candidate.  Four lanes
// per eligible A:
// lane q of an A's group takes its list entries q, q + 4, ..., marks its
// candidates, draws for them, and keeps its retained pair of smallest
// (key, id); the group then takes the smallest of the four.  That pair is
// the unique minimum over all of the A's retained pairs, the same one the
// list walk of a single thread finds, so the choice does not depend on the
// split; four lanes per A shorten each A's chain of dependent list ->
// position -> type loads fourfold.  The loop's trip count is uniform over a
// warp (8 A's per warp and pass), so the group shuffles see every lane.
template <bool NL16>
__device__ __forceinline__ void rx_find_random4(const Sys& S, const Blk blk, const SoA& B,
                                                const uint4* P, unsigned long long step,
                                                uint32_t nact, long long& ncand, long long& nret) {
  const RxParams& R = S.R;
  const uint32_t q = threadIdx.x & 3u;
  const uint32_t gstride = (blk.nb * blockDim.x) >> 2;
  for (uint32_t wb = (blk.b * blockDim.x + (threadIdx.x & ~31u)) >> 2; wb < nact; wb += gstride) {
    const uint32_t w = wb + ((threadIdx.x & 31u) >> 2);
    const bool valid = w < nact;
    uint32_t best = NONE, bestid = 0u;
    unsigned long long bestkey = 0ull;
    const uint32_t i = valid ? S.tmp[w] : 0u;
    if (valid) {
      const uint4 pi = P[i];
      const uint32_t idi = B.id[i];
      const uint32_t nb = B.nadj[i];
      const int cnt = S.nn[i];
      // pass 1 marks this lane's candidates (bit k / 4 for list entry k);
      // pass 2 draws for them
      unsigned long long mask = 0ull;
      for (int k0 = (int)q; k0 < cnt; k0 += 16) {
        // up to four of this lane's entries at once: their slots, then their
        // positions, then the types and states of those within the prefilter
        uint32_t jj[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) jj[u] = k0 + 4 * u < cnt ? nl_get_rx<NL16>(S, k0 + 4 * u, i) : i;
        float r2v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const uint4 pj = P[jj[u]];
          const float ex = __int2float_rn(pdiff(pj.x, pi.x)) * S.scale[0];
          const float ey = __int2float_rn(pdiff(pj.y, pi.y)) * S.scale[1];
          const float ez = __int2float_rn(pdiff(pj.z, pi.z)) * S.scale[2];
          r2v[u] = fmaf(ez, ez, fmaf(ey, ey, ex * ex));
        }
        uint32_t tw = 0u;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const bool near = k0 + 4 * u < cnt && r2v[u] < R.rr2_pre;
          if (near && in_window(R.mask_T, R.t_lo, R.t_hi, B.type[jj[u]], B.state[jj[u]])) tw |= 1u << u;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          if (!((tw >> u) & 1u)) continue;
          const uint32_t j = jj[u];
          if (!(r2v[u] < R.rr2_in)) {  // near the cutoff: the exact FP64 test
            const double ddx = min_image(__dsub_rn(B.x[j], B.x[i]), S.L[0], S.halfL[0]);
            const double ddy = min_image(__dsub_rn(B.y[j], B.y[i]), S.L[1], S.halfL[1]);
            const double ddz = min_image(__dsub_rn(B.z[j], B.z[i]), S.L[2], S.halfL[2]);
            const double r2 = __fma_rn(ddz, ddz, __fma_rn(ddy, ddy, __dmul_rn(ddx, ddx)));
            if (!(r2 < R.rr2)) continue;
          }
          bool bonded = false;
          for (uint32_t b = 0; b < nb; ++b) bonded |= (B.adj[(size_t)i * S.cap + b] & SLOT_MASK) == j;
          if (bonded) continue;
          const int m = (k0 + 4 * u) >> 2;
          if (m < 64) {
            mask |= 1ull << m;
          } else {
            ++ncand;
            rx_accept_and_key(S, B, step, idi, j, R.p53, nret, best, bestkey, bestid);
          }
        }
      }
      while (mask) {
        const int m = __ffsll((long long)mask) - 1;
        mask &= mask - 1ull;
        ++ncand;
        rx_accept_and_key(S, B, step, idi, nl_get_rx<NL16>(S, 4 * m + (int)q, i), R.p53, nret,
                          best, bestkey, bestid);
      }
    }
#pragma unroll
    for (int off = 1; off < 4; off <<= 1) {
      const unsigned long long ok = __shfl_xor_sync(0xFFFFFFFFu, bestkey, off);
      const uint32_t oid = __shfl_xor_sync(0xFFFFFFFFu, bestid, off);
      const uint32_t ob = __shfl_xor_sync(0xFFFFFFFFu, best, off);
      if (ob != NONE && (best == NONE || ok < bestkey || (ok == bestkey && oid < bestid))) {
        best = ob;
        bestkey = ok;
        bestid = oid;
      }
    }
    if (valid && q == 0u) S.win[i] = best;
  }
}

template <bool NL16>
__device__ __forceinline__ void rx_find_body(const Sys& S, const Blk blk, long long step_arg) {
  const RxParams& R = S.R;

  Ctl* ctl = S.ctl;
  const unsigned long long step = step_arg >= 0 ? (unsigned long long)step_arg : ctl->step;
  const SoA B = ctl->set ? S.s1 : S.s0;
  const uint4* P = ctl->phase ? S.P1 : S.P0;
  const uint32_t nact = ctl->n_active;
  long long ncand = 0, nret = 0;
  if (R.rule != PRX_SELECT_NEAREST && R.nr <= 1) {
    rx_find_random4<NL16>(S, blk, B, P, step, nact, ncand, nret);
  } else {
    // the nearest rule and concurrent reactions: one thread per eligible A
    for (uint32_t w = blk.b * blockDim.x + threadIdx.x; w < nact; w += blk.nb * blockDim.x) {
      const uint32_t i = S.tmp[w];
      uint32_t best = NONE;
      if (R.rule == PRX_SELECT_NEAREST) {
        best = nearest_partner<NL16>(S, B, P, i, true, ncand);
      } else {
        uint32_t ch = 0u;
        best = rx_find_multi<NL16>(S, B, P, step, i, ncand, nret, ch);
        S.wch[i] = (uint8_t)ch;
      }
      S.win[i] = best;
    }
  }
  const long long c = block_sum_ll(ncand);
  const long long r = block_sum_ll(nret);
  if (threadIdx.x == 0 && (c | r)) {
    atomicAdd((unsigned long long*)&ctl->trace[0], (unsigned long long)c);
    atomicAdd((unsigned long long*)&ctl->trace[1], (unsigned long long)r);
  }
}

template <bool NL16>
__global__ void __launch_bounds__(RX_THREADS) k_rx_find(Sys S, long long step_arg) {
  rx_find_body<NL16>(S, Blk{blockIdx.x, gridDim.x}, step_arg);
}
__global__ void __launch_bounds__(RX_THREADS)
    kb_rx_find(const Sys* __restrict__ T, const BlkMap* __restrict__ M) {
  const BlkMap m = M[blockIdx.x];
  const Sys& S = T[m.sys];
  if (!S.has_rx) return;  // this member has no reaction scheme
  if (S.nl16) rx_find_body<true>(S, Blk{m.b, m.nb}, -1LL);
  else rx_find_body<false>(S, Blk{m.b, m.nb}, -1LL);
}

// Steps 6-7 for one A winner: every other A that picked the same T lies
// within r_react of T, hence in T's Verlet list.
template <bool NL16>
__device__ __forceinline__ void rx_find_T_body(const Sys& S, const Blk blk) {
  const RxParams& R = S.R;
  if (R.rule != PRX_SELECT_NEAREST) return;
  Ctl* ctl = S.ctl;
  const SoA B = ctl->set ? S.s1 : S.s0;
  const uint4* P = ctl->phase ? S.P1 : S.P0;
  const uint32_t i = blk.b * blockDim.x + threadIdx.x;
  if (i >= S.n || !in_window(R.mask_T, R.t_lo, R.t_hi, B.type[i], B.state[i])) return;
  long long unused = 0;
  S.win[i] = nearest_partner<NL16>(S, B, P, i, false, unused);
}

template <bool NL16>
__global__ void __launch_bounds__(RX_THREADS) k_rx_find_T(Sys S) {
  rx_find_T_body<NL16>(S, Blk{blockIdx.x, gridDim.x});
}
__global__ void __launch_bounds__(RX_THREADS)
    kb_rx_find_T(const Sys* __restrict__ T, const BlkMap* __restrict__ M) {
  const BlkMap m = M[blockIdx.x];
  const Sys& S = T[m.sys];
  if (!S.has_rx) return;  // this member has no reaction scheme
  if (S.nl16) rx_find_T_body<true>(S, Blk{m.b, m.nb});
  else rx_find_T_body<false>(S, Blk{m.b, m.nb});
}

// Table I steps 6-9 in one pass over the eligible A's (the compacted list
// S.tmp): the T that an A picked keeps the A with the smallest key_T
// (random rule), or a mutual nearest pair is accepted with probability
// k dt Theta (nearest rule); an A that keeps its T forms the bond at once:
// adjacency of both, states, and a record in the bond list.  The decisions
// read only the choices (win) and ids, which no bond changes, and each A
// and each T take part in at most one bond, so forming bonds while other
// A's still decide changes nothing.  Bond-list positions come from one
// atomic per warp: the list's order may vary between runs (it is read back
// sorted), its content does not.
template <bool NL16>
__device__ __forceinline__ uint32_t rx_decide(const Sys& S, const SoA& B, unsigned long long step,
                                              uint32_t i, bool& winner) {
  const RxParams& R = S.R;
  const uint32_t T = S.win[i];
  winner = false;
  if (T == NONE) return NONE;
  if (R.rule == PRX_SELECT_NEAREST) {
    // LAMMPS rule: an A and the T it picked react when the T picked it too
    // and u < k dt Theta, drawn with the pair's smaller id first
    if (S.win[T] != i) return NONE;
    winner = true;
    const uint32_t ida = B.id[i], idt = B.id[T];
    const uint4 w = keyed_draw(S.seed, step, min(ida, idt), max(ida, idt), TAG_NEAREST);
    return u53_below(w.x, w.y, R.p53) ? T : NONE;
  }
  winner = true;
  const uint32_t idi = B.id[i], idT = B.id[T];
  const unsigned long long mine = key64(keyed_draw(S.seed, step, idT, idi, TAG_SEL_T));
  bool keep = true;
  const int cnt = S.nn[T];
  // four list entries of T at a time (independent loads go out together)
  for (int k0 = 0; k0 < cnt && keep; k0 += 4) {
    uint32_t aa[4], wa[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) aa[u] = k0 + u < cnt ? nl_get_rx<NL16>(S, k0 + u, T) : i;
#pragma unroll
    for (int u = 0; u < 4; ++u) wa[u] = S.win[aa[u]];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const uint32_t a = aa[u];
      if (!keep || k0 + u >= cnt || a == i || wa[u] != T) continue;
      const uint32_t ida = B.id[a];
      const unsigned long long other = key64(keyed_draw(S.seed, step, idT, ida, TAG_SEL_T));
      if (other < mine || (other == mine && ida < idi)) keep = false;
    }
  }
  return keep ? T : NONE;
}

template <bool NL16>
__device__ __forceinline__ void rx_select_apply_body(const Sys& S, const Blk blk, long long step_arg) {
  const RxParams& R = S.R;
  Ctl* ctl = S.ctl;
  const unsigned long long step = step_arg >= 0 ? (unsigned long long)step_arg : ctl->step;
  const SoA B = ctl->set ? S.s1 : S.s0;
  const uint32_t nact = ctl->n_active;
  const int lane = threadIdx.x & 31;
  long long nwin = 0, nfin = 0;
  // population changes of this block's bonds, per (type, state)
  __shared__ int32_t dpop[PRX_MAX_TYPES * PRX_MAX_STATES];
  for (int k = threadIdx.x; k < PRX_MAX_TYPES * PRX_MAX_STATES; k += blockDim.x) dpop[k] = 0;
  __syncthreads();
  // block-strided over the eligible A's, warp-uniform trip count
  for (uint32_t base = blk.b * blockDim.x; base < nact; base += blk.nb * blockDim.x) {
    const uint32_t w = base + threadIdx.x;
    uint32_t i = NONE, T = NONE;
    if (w < nact) {
      i = S.tmp[w];
      bool winner;
      T = rx_decide<NL16>(S, B, step, i, winner);
      nwin += winner ? 1 : 0;
    }
    bool form = false;
    uint32_t na = 0, nt = 0, ch = 0;
    if (T != NONE) {
      ++nfin;
      const uint32_t ta = B.type[i], tt = B.type[T];
      // the pair's reaction sets the valence limits, increments and style
      ch = R.nr > 1 ? (uint32_t)S.wch[i] : 0u;
      const uint32_t mva = R.nr > 1 ? R.maxvalr[ch][ta] : R.maxval[ta];
      const uint32_t mvt = R.nr > 1 ? R.maxvalr[ch][tt] : R.maxval[tt];
      const uint32_t capA = mva < S.cap ? mva : S.cap;
      const uint32_t capT = mvt < S.cap ? mvt : S.cap;
      na = B.nadj[i];
      nt = B.nadj[T];
      form = na < capA && nt < capT;
      if (!form) set_status(ctl, PRX_ECAPACITY);
    }
    // one bond-list reservation per warp
    const unsigned bal = __ballot_sync(0xFFFFFFFFu, form);
    if (!bal) continue;
    unsigned long long first = 0ull;
    if (lane == __ffs(bal) - 1) first = atomicAdd(&ctl->nbonds, (unsigned long long)__popc(bal));
    first = __shfl_sync(0xFFFFFFFFu, first, __ffs(bal) - 1);
    if (!form) continue;
    const unsigned long long pos = first + __popc(bal & ((1u << lane) - 1u));
    if (pos >= S.bond_cap) {
      set_status(ctl, PRX_ECAPACITY);
      continue;
    }
    const uint32_t style = R.nr > 1 ? R.styler[ch] : R.style;
    const uint32_t sbit = style << 31;
    B.adj[(size_t)i * S.cap + na] = T | sbit;
    B.nadj[i] = (uint8_t)(na + 1);
    B.adj[(size_t)T * S.cap + nt] = i | sbit;
    B.nadj[T] = (uint8_t)(nt + 1);
    const int sa = B.state[i], stt = B.state[T];
    const int sa1 = (int8_t)(sa + (R.nr > 1 ? R.dAr[ch] : R.dA));
    const int st1 = (int8_t)(stt + (R.nr > 1 ? R.dTr[ch] : R.dT));
    B.state[i] = (int8_t)sa1;
    B.state[T] = (int8_t)st1;
    pop_move(dpop, B.type[i], sa, sa1);
    pop_move(dpop, B.type[T], stt, st1);
    BondRec rec;
    rec.a = B.id[i];
    rec.t = B.id[T];
    rec.step = (int64_t)step;
    rec.style = style;
    rec.reaction = ch;
    S.bonds[pos] = rec;
  }
  const long long cw = block_sum_ll(nwin);
  const long long cf = block_sum_ll(nfin);
  if (threadIdx.x == 0) {
    if (R.rule == PRX_SELECT_NEAREST) {  // mutual pairs, accepted pairs
      if (cw) atomicAdd((unsigned long long*)&ctl->trace[1], (unsigned long long)cw);
      if (cf) atomicAdd((unsigned long long*)&ctl->trace[2], (unsigned long long)cf);
    } else if (cw) {
      atomicAdd((unsigned long long*)&ctl->trace[2], (unsigned long long)cw);
    }
    if (cf) atomicAdd((unsigned long long*)&ctl->trace[3], (unsigned long long)cf);
  }
  // the block's population changes into its replica of the running counts
  // (POP_REPLICAS copies, so that blocks do not all meet on the same few
  // counters); the last block sums the replicas into the reaction record
  // (populations, bonds, step)
  __syncthreads();
  int32_t* rep = S.pop + (size_t)(blk.b % POP_REPLICAS) * (PRX_MAX_TYPES * PRX_MAX_STATES);
  for (int k = threadIdx.x; k < PRX_MAX_TYPES * PRX_MAX_STATES; k += blockDim.x)
    if (dpop[k]) atomicAdd(rep + k, dpop[k]);
  __threadfence();
  __shared__ bool is_last;
  __syncthreads();
  if (threadIdx.x == 0) is_last = atomicAdd(&ctl->done_rx, 1u) == blk.nb - 1;
  __syncthreads();
  if (is_last) {
    const unsigned long long slot = ctl->hist_count % S.hist_cap;
    HistRec* rec = &S.hist[slot];
    HistRec* latest = &S.hist[S.hist_cap + 1];
    for (int k = threadIdx.x; k < PRX_MAX_TYPES * PRX_MAX_STATES; k += blockDim.x) {
      int32_t c = 0;
      for (int r = 0; r < POP_REPLICAS; ++r) c += __ldcg(S.pop + r * (PRX_MAX_TYPES * PRX_MAX_STATES) + k);
      (&rec->counts[0][0])[k] = c;
      (&latest->counts[0][0])[k] = c;
    }
    if (threadIdx.x == 0) {
      ctl->done_rx = 0u;
      const long long st = step_arg >= 0 ? step_arg : (long long)ctl->step;
      const long long nb = (long long)atomicAdd(&ctl->nbonds, 0ull);
      rec->step = latest->step = st;
      rec->bonds = latest->bonds = nb;
      ctl->hist_count += 1ull;
      ctl->reactions += 1ull;
    }
  }
}

template <bool NL16>
__global__ void __launch_bounds__(RX_THREADS) k_rx_select_apply(Sys S, long long step_arg) {
  rx_select_apply_body<NL16>(S, Blk{blockIdx.x, gridDim.x}, step_arg);
}
__global__ void __launch_bounds__(RX_THREADS)
    kb_rx_select_apply(const Sys* __restrict__ T, const BlkMap* __restrict__ M) {
  const BlkMap m = M[blockIdx.x];
  const Sys& S = T[m.sys];
  if (!S.has_rx) return;  // this member has no reaction scheme
  if (S.nl16) rx_select_apply_body<true>(S, Blk{m.b, m.nb}, -1LL);
  else rx_select_apply_body<false>(S, Blk{m.b, m.nb}, -1LL);
}

// Populations per (type, state) counted over every slot into out[128]
// (integer atomics: the counts do not depend on their order).  With rec set,
// the last block also stamps rec's step and bond count (on-demand
// observables, into the spare history slot).
__device__ __forceinline__ void pop_count_body(const Sys& S, const Blk blk, int32_t* out,
                                               HistRec* rec) {
  Ctl* ctl = S.ctl;
  const SoA B = ctl->set ? S.s1 : S.s0;
  __shared__ int32_t h[PRX_MAX_TYPES * PRX_MAX_STATES];
  for (int k = threadIdx.x; k < PRX_MAX_TYPES * PRX_MAX_STATES; k += blockDim.x) h[k] = 0;
  __syncthreads();
  // Block-strided over the slots; within a warp, lanes with the same
  // (type, state) bin are counted by one shared atomic of their leader.
  const int lane = threadIdx.x & 31;
  for (uint32_t base = blk.b * blockDim.x; base < S.n; base += blk.nb * blockDim.x) {
    const uint32_t i = base + threadIdx.x;
    int key = -1;
    if (i < S.n) {
      const uint32_t t = B.type[i];
      const int s = B.state[i];
      if (t < PRX_MAX_TYPES && s >= 0 && s < PRX_MAX_STATES) key = (int)t * PRX_MAX_STATES + s;
    }
    const unsigned grp = __match_any_sync(0xFFFFFFFFu, key);
    if (key >= 0 && lane == __ffs(grp) - 1) atomicAdd(&h[key], __popc(grp));
  }
  __syncthreads();
  for (int k = threadIdx.x; k < PRX_MAX_TYPES * PRX_MAX_STATES; k += blockDim.x)
    if (h[k]) atomicAdd(out + k, h[k]);
  if (!rec) return;
  __threadfence();
  if (last_block_rx(&ctl->done_obs, blk.nb)) {
    ctl->done_obs = 0u;
    rec->step = (long long)ctl->step;
    rec->bonds = (long long)ctl->nbonds;
  }
}

__global__ void __launch_bounds__(RX_THREADS) k_obs_hist(Sys S) {
  pop_count_body(S, Blk{blockIdx.x, gridDim.x}, &S.hist[S.hist_cap].counts[0][0], &S.hist[S.hist_cap]);
}
__global__ void __launch_bounds__(RX_THREADS) k_pop_init(Sys S) {
  pop_count_body(S, Blk{blockIdx.x, gridDim.x}, S.pop, nullptr);
}

// Per-block FP64 partial sums of m v^2 / 2 and m v (fixed-order tree).
__global__ void __launch_bounds__(RX_THREADS) k_obs_sums(Sys S, double mass) {
  Ctl* ctl = S.ctl;
  const SoA B = ctl->set ? S.s1 : S.s0;
  // grid-strided sums per thread, then a fixed warp tree and the warps in
  // order: few FP64 additions per slot, the same order on every call
  double ke = 0.0, px = 0.0, py = 0.0, pz = 0.0;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < S.n; i += gridDim.x * blockDim.x) {
    const double vx = B.vx[i], vy = B.vy[i], vz = B.vz[i];
    ke += vx * vx + vy * vy + vz * vz;
    px += vx;
    py += vy;
    pz += vz;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    ke += __shfl_down_sync(0xFFFFFFFFu, ke, o);
    px += __shfl_down_sync(0xFFFFFFFFu, px, o);
    py += __shfl_down_sync(0xFFFFFFFFu, py, o);
    pz += __shfl_down_sync(0xFFFFFFFFu, pz, o);
  }
  __shared__ double red[4][RX_THREADS / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
    red[0][wid] = ke;
    red[1][wid] = px;
    red[2][wid] = py;
    red[3][wid] = pz;
  }
  __syncthreads();
  if (threadIdx.x < 4) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[threadIdx.x][w];
    S.red[4 * (size_t)blockIdx.x + threadIdx.x] = (threadIdx.x == 0 ? 0.5 * mass : mass) * t;
  }
}

// The nsum per-block sums reduced to one value each, in a fixed order (thread
// t adds blocks t, t + 256, ...; then a fixed tree), written to
// red[4 nblk .. 4 nblk + 3].
__global__ void __launch_bounds__(RX_THREADS) k_obs_final(Sys S, uint32_t nsum, uint32_t nblk) {
  __shared__ double part[4][RX_THREADS];
  double a[4] = {0.0, 0.0, 0.0, 0.0};
  for (uint32_t b = threadIdx.x; b < nsum; b += blockDim.x)
    for (int q = 0; q < 4; ++q) a[q] += S.red[4 * (size_t)b + q];
  for (int q = 0; q < 4; ++q) part[q][threadIdx.x] = a[q];
  __syncthreads();
  for (int w = RX_THREADS / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w)
      for (int q = 0; q < 4; ++q) part[q][threadIdx.x] += part[q][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x < 4) S.red[4 * (size_t)nblk + threadIdx.x] = part[threadIdx.x][0];
}

// Batched reaction steps clear each member's counters in a kernel.
__global__ void kb_rx_begin(const Sys* __restrict__ T, const BlkMap* __restrict__ M) {
  const Sys& S = T[M[blockIdx.x].sys];
  if (!S.has_rx || threadIdx.x != 0) return;
  for (int q = 0; q < 4; ++q) S.ctl->trace[q] = 0;
  S.ctl->n_active = 0u;
}

// Pair-distance histogram between two particle classes (the data of
// g_AB(r), Secs. V-VI): one thread per slot of class a runs over its Verlet
// list; pairs are binned by the exact FP64 r^2 (minimum image, the reaction
// test's fma order) against the squared bin edges e2[0..nbins].  Counts are
// integers, so the result does not depend on the order of the atomics.
template <bool NL16>
__global__ void __launch_bounds__(RX_THREADS)
    k_pair_hist(Sys S, PairClass a, PairClass b, const double* __restrict__ e2, int nbins,
                unsigned long long* counts, unsigned long long* nab) {
  extern __shared__ __align__(16) unsigned char smem_h[];
  double* se2 = reinterpret_cast<double*>(smem_h);
  unsigned int* sc = reinterpret_cast<unsigned int*>(se2 + nbins + 1);
  for (int k = threadIdx.x; k <= nbins; k += blockDim.x) se2[k] = e2[k];
  for (int k = threadIdx.x; k < nbins; k += blockDim.x) sc[k] = 0u;
  __syncthreads();
  Ctl* ctl = S.ctl;
  const SoA B = ctl->set ? S.s1 : S.s0;
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  bool ia = false, ib = false;
  if (i < S.n) {
    ia = in_window(a.mask, a.lo, a.hi, B.type[i], B.state[i]);
    ib = in_window(b.mask, b.lo, b.hi, B.type[i], B.state[i]);
  }
  if (ia) {
    const double xi = B.x[i], yi = B.y[i], zi = B.z[i];
    const double rmax2 = se2[nbins];
    const int cnt = S.nn[i];
    for (int k = 0; k < cnt; ++k) {
      const uint32_t j = nl_get_rx<NL16>(S, k, i);
      if (!in_window(b.mask, b.lo, b.hi, B.type[j], B.state[j])) continue;
      const double ddx = min_image(__dsub_rn(B.x[j], xi), S.L[0], S.halfL[0]);
      const double ddy = min_image(__dsub_rn(B.y[j], yi), S.L[1], S.halfL[1]);
      const double ddz = min_image(__dsub_rn(B.z[j], zi), S.L[2], S.halfL[2]);
      const double r2 = __fma_rn(ddz, ddz, __fma_rn(ddy, ddy, __dmul_rn(ddx, ddx)));
      if (!(r2 < rmax2)) continue;
      int lo = 0, hi = nbins - 1;  // largest bin whose lower edge is <= r
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (se2[mid] <= r2) lo = mid;
        else hi = mid - 1;
      }
      atomicAdd(&sc[lo], 1u);
    }
  }
  const int na = __syncthreads_count(ia), nb = __syncthreads_count(ib);
  for (int k = threadIdx.x; k < nbins; k += blockDim.x)
    if (sc[k]) atomicAdd(&counts[k], (unsigned long long)sc[k]);
  if (threadIdx.x == 0) {
    if (na) atomicAdd(&nab[0], (unsigned long long)na);
    if (nb) atomicAdd(&nab[1], (unsigned long long)nb);
  }
}

inline unsigned blocks_rx(uint32_t n) { return n ? (n + RX_THREADS - 1) / RX_THREADS : 1u; }

}  // namespace

int rx_kernel_count(int rule) { return rule == PRX_SELECT_NEAREST ? 4 : 3; }

void launch_rx(const Sys& S, cudaStream_t st, long long step_arg,
               void (*hook)(void*, const char*, int), void* ctx) {
  const unsigned g = blocks_rx(S.n);
  auto H = [&](const char* nm, int p) {
    if (hook) hook(ctx, nm, p);
  };
  cudaMemsetAsync(&S.ctl->trace[0], 0, sizeof(long long) * 4 + sizeof(unsigned int), st);
  H("rx_compact", 0);
  {
    const unsigned g4 = blocks_rx((S.n + 3u) / 4u);
    k_rx_compact4<<<g4, RX_THREADS, 0, st>>>(S);
  }
  H("rx_compact", 1);
  const unsigned gf = g < 1216u ? g : 1216u;
  H("rx_find", 0);
  if (S.nl16) k_rx_find<true><<<gf, RX_THREADS, 0, st>>>(S, step_arg);
  else k_rx_find<false><<<gf, RX_THREADS, 0, st>>>(S, step_arg);
  H("rx_find", 1);
  if (S.R.rule == PRX_SELECT_NEAREST) {
    H("rx_find_T", 0);
    if (S.nl16) k_rx_find_T<true><<<g, RX_THREADS, 0, st>>>(S);
    else k_rx_find_T<false><<<g, RX_THREADS, 0, st>>>(S);
    H("rx_find_T", 1);
  }
  H("rx_select_apply", 0);
  if (S.nl16) k_rx_select_apply<true><<<gf, RX_THREADS, 0, st>>>(S, step_arg);
  else k_rx_select_apply<false><<<gf, RX_THREADS, 0, st>>>(S, step_arg);
  H("rx_select_apply", 1);
}

void launch_pair_hist(const Sys& S, cudaStream_t st, const PairClass& a, const PairClass& b,
                      const double* e2, int nbins, unsigned long long* counts,
                      unsigned long long* nab) {
  const unsigned g = blocks_rx(S.n);
  const size_t sm = 8 * (size_t)(nbins + 1) + 4 * (size_t)nbins;
  if (S.nl16) k_pair_hist<true><<<g, RX_THREADS, sm, st>>>(S, a, b, e2, nbins, counts, nab);
  else k_pair_hist<false><<<g, RX_THREADS, sm, st>>>(S, a, b, e2, nbins, counts, nab);
}

// On-demand observables: the spare history slot (index hist_cap) receives the
// populations; S.red the per-block sums and, after them, their totals.
void launch_observables(const Sys& S, cudaStream_t st, int nblocks) {
  cudaMemsetAsync(&S.hist[S.hist_cap], 0, sizeof(HistRec), st);
  k_obs_hist<<<nblocks, RX_THREADS, 0, st>>>(S);
  // the sums on at most 8 blocks per SM, strided over the slots
  const unsigned nsum = nblocks < 1216 ? (unsigned)nblocks : 1216u;
  k_obs_sums<<<nsum, RX_THREADS, 0, st>>>(S, S.mass);
  k_obs_final<<<1, RX_THREADS, 0, st>>>(S, nsum, (uint32_t)nblocks);
}

void launch_pop_init(const Sys& S, cudaStream_t st) {
  cudaMemsetAsync(S.pop, 0, sizeof(int32_t) * POP_REPLICAS * PRX_MAX_TYPES * PRX_MAX_STATES, st);
  if (S.n) k_pop_init<<<blocks_rx(S.n) < 1216u ? blocks_rx(S.n) : 1216u, RX_THREADS, 0, st>>>(S);
}

int batch_rx_kernel_count() { return 5; }

void launch_batch_rx(const BatchLaunch& L, cudaStream_t st) {
  kb_rx_begin<<<L.n_one, 32, 0, st>>>(L.T, L.one);
  kb_rx_compact<<<L.n_part, RX_THREADS, 0, st>>>(L.T, L.part);
  kb_rx_find<<<L.n_part, RX_THREADS, 0, st>>>(L.T, L.part);
  kb_rx_find_T<<<L.n_part, RX_THREADS, 0, st>>>(L.T, L.part);
  kb_rx_select_apply<<<L.n_part, RX_THREADS, 0, st>>>(L.T, L.part);
}

}  // namespace prx
