// MD kernels: the fused force + Langevin velocity-Verlet step, and the
// rebuild (deterministic counting sort of the slots by cell, then the Verlet
// neighbour lists from a shared-memory sweep of the neighbour cells).
//
// Step kernel, one thread per slot (FP32 force mode):
//   WCA (Sec. II.C, Eq. 15) over the Verlet list, displacements taken
//   exactly from the periodic fixed-point positions and rounded once to FP32;
//   FENE (Sec. II.C) or mirror LJ (Eq. 17) over the adjacency row; Langevin
//   random force keyed by (seed, step, id); then in FP64: v' = a v + b F (one
//   DFMA per component), x' = x + dt v' (one DFMA).  The new fixed-point
//   position comes from x' through integer operations on its binary64
//   fields, so the FP64 pipe (about 70x slower than FP32 on this part) sees
//   only the six DFMAs.
#include <mutex>
#include <type_traits>
#include <cuda_runtime.h>

#include "prx_internal.cuh"

namespace prx {

namespace {

// WCA pair term in FP32; d = x_j - x_i.  Adds -g d to f and V/2 to e.
// Reciprocals and quotients use the hardware approximation (relative error
// about 2^-22), well inside the FP32 force tolerance.
__device__ __forceinline__ void wca32(const Sys& S, float dx, float dy, float dz, float r2,
                                      float& fx, float& fy, float& fz, float& e) {
  const float r2i = __fdividef(1.0f, r2);
  const float sr2 = S.sig2f * r2i;
  const float sr6 = sr2 * sr2 * sr2;
  float g = S.eps24f * sr6 * (2.0f * sr6 - 1.0f) * r2i;
  if (S.fcapf > 0.0f) {
    const float r = sqrtf(r2);
    if (g * r > S.fcapf) g = __fdividef(S.fcapf, r);
  }
  fx -= g * dx;
  fy -= g * dy;
  fz -= g * dz;
  e += 0.5f * S.eps4f * (sr6 * sr6 - sr6 + 0.25f);
}

// Bond term in FP32 (FENE or mirror LJ by style); returns false on FENE overstretch.
__device__ __forceinline__ bool bond32(const Sys& S, uint32_t style, float dx, float dy, float dz,
                                       float& fx, float& fy, float& fz, float& e) {
  const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
  float g;
  if (style == 0u) {
    if (!(r2 < S.fr02f)) return false;
    const float q = 1.0f - r2 * S.fr02if;
    g = -__fdividef(S.fkf, q);
    e += 0.5f * (-0.5f * S.fkf * S.fr02f * logf(q));
  } else {
    const float r = sqrtf(r2);
    if (!(r > S.rcf && r < 2.0f * S.rcf)) return true;
    const float sd = 2.0f * S.rcf - r;
    const float ss2 = __fdividef(S.sig2f, sd * sd);
    const float ss6 = ss2 * ss2 * ss2;
    const float dVdr = __fdividef(S.eps24f * (2.0f * ss6 * ss6 - ss6), sd);
    g = -__fdividef(dVdr, r);
    e += 0.5f * S.eps4f * (ss6 * ss6 - ss6 + 0.25f);
  }
  fx -= g * dx;
  fy -= g * dy;
  fz -= g * dz;
  return true;
}

// FP64 versions, arithmetic written as in the plain definitions.
template <bool ENERGY = true>
__device__ __forceinline__ void wca64(const Sys& S, double dx, double dy, double dz, double r2,
                                      double& fx, double& fy, double& fz, double& e) {
  const double sr2 = __ddiv_rn(S.sig2, r2);
  const double sr6 = __dmul_rn(__dmul_rn(sr2, sr2), sr2);
  const double sr12 = __dmul_rn(sr6, sr6);
  double g = __ddiv_rn(__dmul_rn(S.eps24, __dsub_rn(__dmul_rn(2.0, sr12), sr6)), r2);
  if (S.fcap > 0.0) {
    const double r = __dsqrt_rn(r2);
    if (__dmul_rn(g, r) > S.fcap) g = __ddiv_rn(S.fcap, r);
  }
  fx = __dsub_rn(fx, __dmul_rn(g, dx));
  fy = __dsub_rn(fy, __dmul_rn(g, dy));
  fz = __dsub_rn(fz, __dmul_rn(g, dz));
  if constexpr (ENERGY)
    e = __dadd_rn(e, __dmul_rn(0.5, __dmul_rn(S.eps4, __dadd_rn(__dsub_rn(sr12, sr6), 0.25))));
}

template <bool ENERGY = true>
__device__ __forceinline__ bool bond64(const Sys& S, uint32_t style, double dx, double dy,
                                       double dz, double& fx, double& fy, double& fz, double& e) {
  const double r2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
  double g;
  if (style == 0u) {
    if (!(r2 < S.fr02)) return false;
    const double q = __dsub_rn(1.0, __ddiv_rn(r2, S.fr02));
    g = __ddiv_rn(-S.fk, q);
    if constexpr (ENERGY)
      e = __dadd_rn(e, __dmul_rn(0.5, __dmul_rn(__dmul_rn(__dmul_rn(-0.5, S.fk), S.fr02), log(q))));
  } else {
    const double r = __dsqrt_rn(r2);
    if (!(r > S.rc && r < 2.0 * S.rc)) return true;
    const double sd = __dsub_rn(2.0 * S.rc, r);
    const double ss2 = __ddiv_rn(S.sig2, __dmul_rn(sd, sd));
    const double ss6 = __dmul_rn(__dmul_rn(ss2, ss2), ss2);
    const double ss12 = __dmul_rn(ss6, ss6);
    const double dVdr = __ddiv_rn(__dmul_rn(S.eps24, __dsub_rn(__dmul_rn(2.0, ss12), ss6)), sd);
    g = __ddiv_rn(-dVdr, r);
    if constexpr (ENERGY)
      e = __dadd_rn(e, __dmul_rn(0.5, __dmul_rn(S.eps4, __dadd_rn(__dsub_rn(ss12, ss6), 0.25))));
  }
  fx = __dsub_rn(fx, __dmul_rn(g, dx));
  fy = __dsub_rn(fy, __dmul_rn(g, dy));
  fz = __dsub_rn(fz, __dmul_rn(g, dz));
  return true;
}

// Last warp of a grid to finish, without a block barrier: each warp counts
// itself out of its block in shared memory, and the last warp of a block
// counts the block out of the grid.  `warps_left` is set to the block's warp
// count before the block's work starts.
// The only data the last warp reads is the rebuild flag, whose setters
// fence after setting it; warps therefore fence only once per block.
__device__ __forceinline__ bool last_warp(unsigned int* counter, unsigned int* warps_left,
                                          uint32_t nb) {
  __syncwarp();
  bool last = false;
  if ((threadIdx.x & 31) == 0) {
    if (atomicSub(warps_left, 1u) == 1u) {
      __threadfence();
      last = atomicAdd(counter, 1u) == nb - 1;
    }
  }
  return last;
}

// A particle moved more than skin/2: flag the system (and its batch).
__device__ __forceinline__ void raise_rebuild(const Sys& S) {
  atomicExch(&S.ctl->rebin_flag, 1);
  if (S.in_batch) atomicExch(&S.batch->any_rebuild, 1);
  __threadfence();
}

// End of a step: the system's last warp advances its step counter and
// buffer phase; for a single system it also sets the graph's rebuild
// condition, for a batch the last system to finish sets it for all.
__device__ __forceinline__ void step_epilogue(const Sys& S, int ph, unsigned long long step,
                                              cudaGraphConditionalHandle cond, int use_cond,
                                              unsigned int* warps_left, uint32_t nb) {
  Ctl* ctl = S.ctl;
  if (last_warp(&ctl->done_step, warps_left, nb)) {
    ctl->done_step = 0u;
    ctl->phase = ph ^ 1;
    ctl->step = step;
    if (!S.in_batch) {
      const int flag = atomicAdd(&ctl->rebin_flag, 0);
      if (use_cond) cudaGraphSetConditional(cond, flag ? 1u : 0u);
    } else {
      __threadfence();
      if (atomicAdd(&S.batch->done_step, 1u) == S.n_members - 1) {
        S.batch->done_step = 0u;
        const int flag = atomicExch(&S.batch->any_rebuild, 0);
        if (flag) S.batch->rebuilds += 1ull;
        S.batch->rebuild_now = flag;  // for a device-driven run (dg.cu)
        if (use_cond) cudaGraphSetConditional(cond, flag ? 1u : 0u);
      }
    }
  }
}

// k-th Verlet-list entry of slot i: the neighbour's slot (16-bit for systems
// of at most 65,535 particles).  Entries past a slot's count hold stale
// slots of some earlier list: still valid slots.
template <bool NL16>
__device__ __forceinline__ uint32_t nl_raw(const Sys& S, int k, uint32_t i) {
  if constexpr (NL16) return __ldg(((const uint16_t*)S.nl) + (size_t)k * S.n + i);
  else return __ldg(((const uint32_t*)S.nl) + (size_t)k * S.n + i);
}
template <bool NL16>
__device__ __forceinline__ uint32_t nl_get(const Sys& S, int k, uint32_t i) {
  return nl_raw<NL16>(S, k, i);
}

// Fetch the line holding *a into L2 (no register result).
__device__ __forceinline__ void prefetch_l2(const void* a) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(a));
}

// Physical minimum-image displacement x_j - x_i: exact in fixed point,
// converted with one rounding, scaled by L / 2^32.
__device__ __forceinline__ void disp(const Sys& S, uint4 pj, uint4 pi, float& dx, float& dy,
                                     float& dz) {
  dx = __int2float_rn(pdiff(pj.x, pi.x)) * S.scale[0];
  dy = __int2float_rn(pdiff(pj.y, pi.y)) * S.scale[1];
  dz = __int2float_rn(pdiff(pj.z, pi.z)) * S.scale[2];
}

// Displacement since the last list build exceeds skin/2 (coarse reference in .w).
__device__ __forceinline__ bool moved_beyond_skin(const Sys& S, uint32_t X, uint32_t Y, uint32_t Z,
                                                  uint32_t W) {
  const int ax = (int)(((X >> S.wshift[0]) - W) << 22) >> 22;
  const int ay = (int)(((Y >> S.wshift[1]) - (W >> 10)) << 22) >> 22;
  const int az = (int)(((Z >> S.wshift[2]) - (W >> 20)) << 22) >> 22;
  const float ex = (float)ax * S.wunit[0], ey = (float)ay * S.wunit[1], ez = (float)az * S.wunit[2];
  return fmaf(ez, ez, fmaf(ey, ey, ex * ex)) > S.disp2_max;
}

// periodic_fx for the step kernel: the scaling by 2^32 added to the binary64
// exponent field (exact for normal x; zero and subnormals stay below 1) and
// the truncation done by the hardware FP64 -> s64 conversion, which costs
// one FP64-pipe instruction instead of fx32's variable 64-bit shifts.  The
// same value as periodic_fx for |x| < 2^29.
__device__ __forceinline__ uint32_t periodic_fx_cvt(double x, long long Lfx, unsigned long long M) {
  const double y = __longlong_as_double(__double_as_longlong(x) + (32LL << 52));
  const unsigned long long a = (unsigned long long)(__double2ll_rz(y) + Lfx);
  return (uint32_t)__umul64hi(a, M);
}

// End of an FP32-mode step for one slot: Langevin kick (friction applied
// exactly in FP64), drift, new fixed-point position, rebuild trigger.
//   v' = a v + b (F_c + R),  x' = x + dt v'
__device__ __forceinline__ void integrate32(const Sys& S, Ctl* ctl, const SoA& B, uint4* Pn,
                                            uint32_t i, uint32_t pid, uint32_t W,
                                            unsigned long long step, float fx, float fy, float fz,
                                            double xi, double yi, double zi, double vx, double vy,
                                            double vz) {
  float Rx = 0.f, Ry = 0.f, Rz = 0.f;
  if (S.thermo) {
    const uint4 w = keyed_draw(S.seed, step, pid, 0u, TAG_THERMO);
    Rx = S.cRf * (u24f(w.x) - 0.5f);
    Ry = S.cRf * (u24f(w.y) - 0.5f);
    Rz = S.cRf * (u24f(w.z) - 0.5f);
  }
  const float kx = S.b_kickf * (fx + Rx), ky = S.b_kickf * (fy + Ry), kz = S.b_kickf * (fz + Rz);
  if (!(fabsf(kx) + fabsf(ky) + fabsf(kz) < 1e30f)) set_status(ctl, PRX_ENONFINITE);
  vx = __fma_rn(vx, S.a_fric, f2d_exact(kx));
  vy = __fma_rn(vy, S.a_fric, f2d_exact(ky));
  vz = __fma_rn(vz, S.a_fric, f2d_exact(kz));
  const double nx = __fma_rn(S.dt, vx, xi);
  const double ny = __fma_rn(S.dt, vy, yi);
  const double nz = __fma_rn(S.dt, vz, zi);
  const uint32_t X = periodic_fx_cvt(nx, S.Lfx[0], S.M64[0]);
  const uint32_t Y = periodic_fx_cvt(ny, S.Lfx[1], S.M64[1]);
  const uint32_t Z = periodic_fx_cvt(nz, S.Lfx[2], S.M64[2]);
  if (moved_beyond_skin(S, X, Y, Z, W)) raise_rebuild(S);
  B.vx[i] = vx;
  B.vy[i] = vy;
  B.vz[i] = vz;
  B.x[i] = nx;
  B.y[i] = ny;
  B.z[i] = nz;
  Pn[i] = make_uint4(X, Y, Z, W);
}

// ---------------------------------------------------------------------------
// FP32 step kernel: one thread per slot, WCA over the Verlet list.
// ---------------------------------------------------------------------------
// The step of slot i: forces over its list and bonds, then the integration
// (or, FORCES_ONLY, the forces written out).
template <bool NL16, bool FORCES_ONLY, bool CUBIC>
__device__ __forceinline__ void step_one(const Sys& S, Ctl* ctl, const SoA& B,
                                         const uint4* __restrict__ P, uint4* __restrict__ Pn,
                                         uint32_t i, unsigned long long step) {
  // every load that does not depend on another goes out first
  const int cnt = __ldg(S.nn + i);
  uint32_t rn[4];
#pragma unroll
  for (int u = 0; u < 4; ++u) rn[u] = nl_raw<NL16>(S, u, i);
  const uint4 pi = __ldg(P + i);
  // the bond count and adjacency row are read after the list loop; a
  // prefetch into L2 now hides their DRAM latency without holding
  // registers across the loop
  prefetch_l2(B.nadj + i);
  prefetch_l2(B.adj + (size_t)i * S.cap);
  float fx = 0.f, fy = 0.f, fz = 0.f, e = 0.f;
  // software pipeline over the list, four entries per stage: the next
  // stage's list entries (when this list has one) load while this stage's
  // four gathers complete.
  // The build pads every list to whole stages with the slot itself (r = 0,
  // skipped).  In a cubic box displacements stay in position units and the
  // neighbour force is scaled once at the end.
  for (int k = 0; k < cnt; k += 4) {
    uint4 pj[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) pj[u] = __ldg(P + rn[u]);
#pragma unroll
    for (int u = 0; u < 4; ++u) rn[u] = k + 4 < cnt ? nl_raw<NL16>(S, k + 4 + u, i) : 0u;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      if constexpr (CUBIC) {
        const float ux = __int2float_rn(pdiff(pj[u].x, pi.x));
        const float uy = __int2float_rn(pdiff(pj[u].y, pi.y));
        const float uz = __int2float_rn(pdiff(pj[u].z, pi.z));
        const float r2u = fmaf(uz, uz, fmaf(uy, uy, ux * ux));
        if (r2u > 0.f && r2u < S.rc2u) wca32(S, ux, uy, uz, r2u * S.s2f, fx, fy, fz, e);
      } else {
        float dx, dy, dz;
        disp(S, pj[u], pi, dx, dy, dz);
        const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
        if (r2 > 0.f && r2 < S.rc2f) wca32(S, dx, dy, dz, r2, fx, fy, fz, e);
      }
    }
  }
  if constexpr (CUBIC) {
    fx *= S.scale[0];
    fy *= S.scale[0];
    fz *= S.scale[0];
  }
  bool ok = true;
  // bonds two at a time: both entries, then both partners' positions, in
  // flight together (half the dependent load chains).  The first pair's
  // entries load beside the bond count, and its gathers do not wait for it:
  // entries past the count (stale or never written) are clamped to a valid
  // slot and their terms skipped.
  const uint32_t* arow0 = B.adj + (size_t)i * S.cap;
  const uint32_t nb = __ldg(B.nadj + i);
  {
    const uint32_t e0 = __ldg(arow0), e1 = S.cap > 1 ? __ldg(arow0 + 1) : i;
    const uint32_t s0 = min(e0 & SLOT_MASK, S.n - 1u), s1 = min(e1 & SLOT_MASK, S.n - 1u);
    const uint4 p0 = __ldg(P + s0), p1 = __ldg(P + s1);
    float dx, dy, dz;
    if (nb > 0u) {
      disp(S, p0, pi, dx, dy, dz);
      ok = bond32(S, e0 >> 31, dx, dy, dz, fx, fy, fz, e) && ok;
    }
    if (nb > 1u) {
      disp(S, p1, pi, dx, dy, dz);
      ok = bond32(S, e1 >> 31, dx, dy, dz, fx, fy, fz, e) && ok;
    }
  }
  for (int b = 2; b < (int)nb; b += 2) {
    const uint32_t* arow = B.adj + (size_t)i * S.cap + b;
    const bool two = b + 1 < (int)nb;
    const uint32_t e0 = __ldg(arow), e1 = two ? __ldg(arow + 1) : i;
    const uint4 p0 = __ldg(P + (e0 & SLOT_MASK)), p1 = __ldg(P + (e1 & SLOT_MASK));
    float dx, dy, dz;
    disp(S, p0, pi, dx, dy, dz);
    ok = bond32(S, e0 >> 31, dx, dy, dz, fx, fy, fz, e) && ok;
    if (two) {
      disp(S, p1, pi, dx, dy, dz);
      ok = bond32(S, e1 >> 31, dx, dy, dz, fx, fy, fz, e) && ok;
    }
  }
  if (!ok) set_status(ctl, PRX_EOVERSTRETCH);
  if constexpr (FORCES_ONLY) {
    S.fout[3 * (size_t)i + 0] = (double)fx;
    S.fout[3 * (size_t)i + 1] = (double)fy;
    S.fout[3 * (size_t)i + 2] = (double)fz;
    S.eout[i] = (double)e;
  } else {
    const double xi = B.x[i], yi = B.y[i], zi = B.z[i];
    const double vx = B.vx[i], vy = B.vy[i], vz = B.vz[i];
    const uint32_t pid = __ldg(B.id + i);
    integrate32(S, ctl, B, Pn, i, pid, pi.w, step, fx, fy, fz, xi, yi, zi, vx, vy, vz);
  }
}

template <bool NL16, bool FORCES_ONLY, bool CUBIC>
__device__ __forceinline__ void step_nl_body(const Sys& S, const Blk blk,
                                             cudaGraphConditionalHandle cond, int use_cond) {
  __shared__ unsigned int warps_left;
  if (threadIdx.x == 0) warps_left = blockDim.x >> 5;
  __syncthreads();
  Ctl* ctl = S.ctl;
  const int set = ctl->set;
  const int ph = ctl->phase;
  const unsigned long long step = ctl->step + 1ull;
  const SoA B = set ? S.s1 : S.s0;
  const uint4* __restrict__ P = ph ? S.P1 : S.P0;
  uint4* __restrict__ Pn = ph ? S.P0 : S.P1;
  const uint32_t i = blk.b * blockDim.x + threadIdx.x;
  if (i < S.n) step_one<NL16, FORCES_ONLY, CUBIC>(S, ctl, B, P, Pn, i, step);
  if constexpr (!FORCES_ONLY) step_epilogue(S, ph, step, cond, use_cond, &warps_left, blk.nb);
}

// Single system: as many blocks as are resident at once (or the launch
// configuration's blocks per SM), each warp taking 32-slot chunks strided by
// the grid's warp count, so that every SM stays fully occupied to the end
// instead of running a partial last wave.  BT threads per block, with the
// register budget of 48 resident warps per SM for every BT; the block shape
// changes only the scheduling, not any particle's arithmetic.
template <bool NL16, bool FORCES_ONLY, bool CUBIC, int BT>
__global__ void __launch_bounds__(BT, 1536 / BT)
    k_step_nl(Sys S, cudaGraphConditionalHandle cond, int use_cond) {
  __shared__ unsigned int warps_left;
  if (threadIdx.x == 0) warps_left = blockDim.x >> 5;
  __syncthreads();
  Ctl* ctl = S.ctl;
  const int ph = ctl->phase;
  const unsigned long long step = ctl->step + 1ull;
  const uint4* __restrict__ P = ph ? S.P1 : S.P0;
  uint4* __restrict__ Pn = ph ? S.P0 : S.P1;
  const uint32_t W = gridDim.x * (blockDim.x >> 5);
  // one loop per SoA set (a uniform branch), so that the set's array
  // pointers are read from the kernel parameters where they are used
  // instead of occupying registers across the loop
  auto run = [&](const SoA& B) {
    for (uint32_t c = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); c * 32u < S.n; c += W) {
      const uint32_t i = c * 32u + (threadIdx.x & 31u);
      if (i < S.n) step_one<NL16, FORCES_ONLY, CUBIC>(S, ctl, B, P, Pn, i, step);
    }
  };
  if (ctl->set) run(S.s1);
  else run(S.s0);
  if constexpr (!FORCES_ONLY) step_epilogue(S, ph, step, cond, use_cond, &warps_left, gridDim.x);
}
// The same step with four lanes per slot, for systems too small to fill the
// GPU with one thread per slot: a warp takes 8 consecutive slots; lane q of
// a slot's group sums its list entries q, q + 4, ... and bonds q, q + 4, ...;
// the four partial forces are combined by a fixed butterfly (the same order
// every step), and lanes 0-7 then integrate the 8 slots as in the one-lane
// kernel.  Four times as many warps per slot hide the dependent
// list -> position gathers that a small grid leaves exposed.  The sum order
// differs from the one-lane kernel's (FP32 rounding only).
template <bool NL16, bool FORCES_ONLY, bool CUBIC, int BT>
__global__ void __launch_bounds__(BT, 1536 / BT)
    k_step_nl4(Sys S, cudaGraphConditionalHandle cond, int use_cond) {
  __shared__ unsigned int warps_left;
  if (threadIdx.x == 0) warps_left = blockDim.x >> 5;
  __syncthreads();
  Ctl* ctl = S.ctl;
  const int ph = ctl->phase;
  const unsigned long long step = ctl->step + 1ull;
  const uint4* __restrict__ P = ph ? S.P1 : S.P0;
  uint4* __restrict__ Pn = ph ? S.P0 : S.P1;
  const uint32_t W = gridDim.x * (blockDim.x >> 5);
  const int lane = threadIdx.x & 31, q = lane & 3;
  auto run = [&](const SoA& B) {
    for (uint32_t c = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); c * 8u < S.n; c += W) {
      const uint32_t i = c * 8u + (uint32_t)(lane >> 2);
      float fx = 0.f, fy = 0.f, fz = 0.f, e = 0.f;
      uint32_t wref = 0u;
      bool ok = true;
      if (i < S.n) {
        const int cnt = __ldg(S.nn + i);
        const uint4 pi = __ldg(P + i);
        wref = pi.w;
        for (int k0 = q; k0 < cnt; k0 += 16) {
          uint32_t rn[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) rn[u] = k0 + 4 * u < cnt ? nl_raw<NL16>(S, k0 + 4 * u, i) : i;
          uint4 pj[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) pj[u] = __ldg(P + rn[u]);
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            if constexpr (CUBIC) {
              const float ux = __int2float_rn(pdiff(pj[u].x, pi.x));
              const float uy = __int2float_rn(pdiff(pj[u].y, pi.y));
              const float uz = __int2float_rn(pdiff(pj[u].z, pi.z));
              const float r2u = fmaf(uz, uz, fmaf(uy, uy, ux * ux));
              if (r2u > 0.f && r2u < S.rc2u) wca32(S, ux, uy, uz, r2u * S.s2f, fx, fy, fz, e);
            } else {
              float dx, dy, dz;
              disp(S, pj[u], pi, dx, dy, dz);
              const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
              if (r2 > 0.f && r2 < S.rc2f) wca32(S, dx, dy, dz, r2, fx, fy, fz, e);
            }
          }
        }
        if constexpr (CUBIC) {
          fx *= S.scale[0];
          fy *= S.scale[0];
          fz *= S.scale[0];
        }
        const uint32_t nb = __ldg(B.nadj + i);
        for (uint32_t b = (uint32_t)q; b < nb; b += 4) {
          const uint32_t ent = __ldg(B.adj + (size_t)i * S.cap + b);
          const uint4 pj = __ldg(P + (ent & SLOT_MASK));
          float dx, dy, dz;
          disp(S, pj, pi, dx, dy, dz);
          ok = bond32(S, ent >> 31, dx, dy, dz, fx, fy, fz, e) && ok;
        }
      }
      if (!ok) set_status(ctl, PRX_EOVERSTRETCH);
#pragma unroll
      for (int o = 1; o < 4; o <<= 1) {
        fx += __shfl_xor_sync(0xFFFFFFFFu, fx, o);
        fy += __shfl_xor_sync(0xFFFFFFFFu, fy, o);
        fz += __shfl_xor_sync(0xFFFFFFFFu, fz, o);
        if constexpr (FORCES_ONLY) e += __shfl_xor_sync(0xFFFFFFFFu, e, o);
      }
      // lane g (< 8) takes slot c * 8 + g from the group's first lane
      const int src = (lane & 7) * 4;
      const float gx = __shfl_sync(0xFFFFFFFFu, fx, src);
      const float gy = __shfl_sync(0xFFFFFFFFu, fy, src);
      const float gz = __shfl_sync(0xFFFFFFFFu, fz, src);
      const float ge = __shfl_sync(0xFFFFFFFFu, e, src);
      const uint32_t gw = __shfl_sync(0xFFFFFFFFu, wref, src);
      const uint32_t ii = c * 8u + (uint32_t)lane;
      if (lane < 8 && ii < S.n) {
        if constexpr (FORCES_ONLY) {
          S.fout[3 * (size_t)ii + 0] = (double)gx;
          S.fout[3 * (size_t)ii + 1] = (double)gy;
          S.fout[3 * (size_t)ii + 2] = (double)gz;
          S.eout[ii] = (double)ge;
        } else {
          const double xi = B.x[ii], yi = B.y[ii], zi = B.z[ii];
          const double vx = B.vx[ii], vy = B.vy[ii], vz = B.vz[ii];
          const uint32_t pid = __ldg(B.id + ii);
          integrate32(S, ctl, B, Pn, ii, pid, gw, step, gx, gy, gz, xi, yi, zi, vx, vy, vz);
        }
      }
    }
  };
  if (ctl->set) run(S.s1);
  else run(S.s0);
  if constexpr (!FORCES_ONLY) step_epilogue(S, ph, step, cond, use_cond, &warps_left, gridDim.x);
}

// Members of a batch may differ in list width and box shape: the batch step
// runs one launch per (list width, cubic) variant present, each over the
// blocks of its members, with the single-system kernel's register budget.
template <bool NL16, bool CUBIC>
__global__ void __launch_bounds__(256, 5)
    kb_step_nl(const Sys* __restrict__ T, const BlkMap* __restrict__ M,
               cudaGraphConditionalHandle cond, int use_cond, uint32_t* __restrict__ act_n) {
  if (blockIdx.x == 0 && threadIdx.x < 5) act_n[threadIdx.x] = 0u;  // for this step's rebuild plan
  const BlkMap m = M[blockIdx.x];
  step_nl_body<NL16, false, CUBIC>(T[m.sys], Blk{m.b, m.nb}, cond, use_cond);
}

// ---------------------------------------------------------------------------
// FP64 force mode (small systems): conservative forces per slot from the
// absolute positions over the same Verlet list, written to fout (and, for
// prx_compute_forces, the energies to eout); the integration runs as a second
// kernel so that no thread reads a position another thread updates.
// Arithmetic per pair in the order of the plain definitions.  FP64 issues
// at about 1/64 of the FP32 rate on this part, so the few particles of an
// FP64 system are spread over every SM: four lanes per slot (lane q takes
// the list entries and bonds q, q + 4, ...), one warp per block, and the
// four partial sums combined by a fixed butterfly (the same order every
// step).
// ---------------------------------------------------------------------------
constexpr int F64_LANES = 4;

template <bool NL16, bool ENERGY>
__global__ void __launch_bounds__(32) k_forces64(Sys S) {
  Ctl* ctl = S.ctl;
  const SoA B = ctl->set ? S.s1 : S.s0;
  const int lane = threadIdx.x & 31, q = lane & (F64_LANES - 1);
  const uint32_t i = blockIdx.x * (32 / F64_LANES) + (uint32_t)(lane / F64_LANES);
  double fx = 0.0, fy = 0.0, fz = 0.0, e = 0.0;
  bool ok = true;
  if (i < S.n) {
    const double xi = B.x[i], yi = B.y[i], zi = B.z[i];
    const int cnt = S.nn[i];
    for (int k = q; k < cnt; k += F64_LANES) {
      const uint32_t j = nl_get<NL16>(S, k, i);
      const double ddx = min_image(__dsub_rn(B.x[j], xi), S.L[0], S.halfL[0]);
      const double ddy = min_image(__dsub_rn(B.y[j], yi), S.L[1], S.halfL[1]);
      const double ddz = min_image(__dsub_rn(B.z[j], zi), S.L[2], S.halfL[2]);
      const double r2 = __dadd_rn(__dadd_rn(__dmul_rn(ddx, ddx), __dmul_rn(ddy, ddy)), __dmul_rn(ddz, ddz));
      if (r2 < S.rc2) wca64<ENERGY>(S, ddx, ddy, ddz, r2, fx, fy, fz, e);
    }
    const uint32_t nb = B.nadj[i];
    for (uint32_t b = (uint32_t)q; b < nb; b += F64_LANES) {
      const uint32_t ent = B.adj[(size_t)i * S.cap + b];
      const uint32_t j = ent & SLOT_MASK;
      const double ddx = min_image(__dsub_rn(B.x[j], xi), S.L[0], S.halfL[0]);
      const double ddy = min_image(__dsub_rn(B.y[j], yi), S.L[1], S.halfL[1]);
      const double ddz = min_image(__dsub_rn(B.z[j], zi), S.L[2], S.halfL[2]);
      ok = bond64<ENERGY>(S, ent >> 31, ddx, ddy, ddz, fx, fy, fz, e) && ok;
    }
  }
  if (!ok) set_status(ctl, PRX_EOVERSTRETCH);
#pragma unroll
  for (int o = 1; o < F64_LANES; o <<= 1) {
    fx = __dadd_rn(fx, __shfl_xor_sync(0xFFFFFFFFu, fx, o));
    fy = __dadd_rn(fy, __shfl_xor_sync(0xFFFFFFFFu, fy, o));
    fz = __dadd_rn(fz, __shfl_xor_sync(0xFFFFFFFFu, fz, o));
    if constexpr (ENERGY) e = __dadd_rn(e, __shfl_xor_sync(0xFFFFFFFFu, e, o));
  }
  if (q == 0 && i < S.n) {
    S.fout[3 * (size_t)i + 0] = fx;
    S.fout[3 * (size_t)i + 1] = fy;
    S.fout[3 * (size_t)i + 2] = fz;
    if constexpr (ENERGY) S.eout[i] = e;
  }
}

// FP64 integration in the oracle's order of operations:
//   F = F_c - gamma m v + R,  v' = v + (dt/m) F,  x' = x + dt v'.
__global__ void __launch_bounds__(STEP_THREADS)
    k_integrate64(Sys S, cudaGraphConditionalHandle cond, int use_cond) {
  __shared__ unsigned int warps_left;
  if (threadIdx.x == 0) warps_left = blockDim.x >> 5;
  __syncthreads();
  Ctl* ctl = S.ctl;
  const int set = ctl->set;
  const int ph = ctl->phase;
  const unsigned long long step = ctl->step + 1ull;
  const SoA B = set ? S.s1 : S.s0;
  const uint4* __restrict__ P = ph ? S.P1 : S.P0;
  uint4* __restrict__ Pn = ph ? S.P0 : S.P1;
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < S.n) {
    const uint32_t W = P[i].w;
    const uint32_t pid = B.id[i];
    double R[3] = {0.0, 0.0, 0.0};
    if (S.thermo) {
      const uint4 w = keyed_draw(S.seed, step, pid, 0u, TAG_THERMO);
      R[0] = __dmul_rn(S.cR, __dsub_rn(f2d_exact(u24f(w.x)), 0.5));
      R[1] = __dmul_rn(S.cR, __dsub_rn(f2d_exact(u24f(w.y)), 0.5));
      R[2] = __dmul_rn(S.cR, __dsub_rn(f2d_exact(u24f(w.z)), 0.5));
    }
    double* xs[3] = {B.x, B.y, B.z};
    double* vs[3] = {B.vx, B.vy, B.vz};
    uint32_t Xn[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const double v = vs[d][i];
      const double F = __dadd_rn(__dsub_rn(S.fout[3 * (size_t)i + d], __dmul_rn(S.gm, v)), R[d]);
      const double vn = __dadd_rn(v, __dmul_rn(S.b_kick, F));
      const double xn = __dadd_rn(xs[d][i], __dmul_rn(S.dt, vn));
      if (!isfinite(vn) || !isfinite(xn)) set_status(ctl, PRX_ENONFINITE);
      vs[d][i] = vn;
      xs[d][i] = xn;
      Xn[d] = periodic_fx(xn, S.Lfx[d], S.M64[d]);
    }
    if (moved_beyond_skin(S, Xn[0], Xn[1], Xn[2], W)) raise_rebuild(S);
    Pn[i] = make_uint4(Xn[0], Xn[1], Xn[2], W);
  }
  step_epilogue(S, ph, step, cond, use_cond, &warps_left, gridDim.x);
}

// ---------------------------------------------------------------------------
// Rebuild.  Keys (wrapping x into [0, L)), counting sort with a stable
// (ascending old slot) order inside each cell, permutation of every
// per-particle array into the other SoA set with fresh fixed-point positions,
// adjacency remap, then the Verlet lists.
// ---------------------------------------------------------------------------
// v >= L: v - L; then v < 0: v + L.  The tests compare binary64 bit
// patterns on the integer pipe (for non-negative doubles the bit order is the
// numeric order; -0.0 counts as 0), so the FP64 pipe only sees the rare
// particle that left the box.
__device__ __forceinline__ double wrap_into_box(double v, double L) {
  if (__double_as_longlong(v) >= __double_as_longlong(L)) v = __dsub_rn(v, L);
  const long long b = __double_as_longlong(v);
  if (b < 0 && (b << 1) != 0) v = __dadd_rn(v, L);
  return v;
}

// Cell of every slot from the fixed-point position the last step wrote.
__device__ __forceinline__ void rebin_keys_body(const Sys& S, const Blk blk) {
  Ctl* ctl = S.ctl;
  const uint4* __restrict__ P = ctl->phase ? S.P1 : S.P0;
  const uint32_t i = blk.b * blockDim.x + threadIdx.x;
  if (i >= S.n) return;
  const uint4 q = P[i];
  const uint32_t cx = __umulhi(q.x, (uint32_t)S.nc[0]);
  const uint32_t cy = __umulhi(q.y, (uint32_t)S.nc[1]);
  const uint32_t cz = __umulhi(q.z, (uint32_t)S.nc[2]);
  const uint32_t k = (cz * (uint32_t)S.nc[1] + cy) * (uint32_t)S.nc[0] + cx;
  S.key[i] = k;
  atomicAdd(&S.count[k], 1u);
}

__global__ void k_rebin_keys(Sys S) { rebin_keys_body(S, Blk{blockIdx.x, gridDim.x}); }

// First binning of a system (no step has written fixed-point positions yet):
// cells from the FP64 positions, which are wrapped into the box in place.
__global__ void k_rebin_keys_x(Sys S) {
  Ctl* ctl = S.ctl;
  const SoA B = ctl->set ? S.s1 : S.s0;
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= S.n) return;
  double* xs[3] = {B.x, B.y, B.z};
  uint32_t c[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const double v0 = xs[d][i];
    const double v = wrap_into_box(v0, S.L[d]);
    if (v != v0) xs[d][i] = v;
    c[d] = __umulhi(periodic_fx(v, S.Lfx[d], S.M64[d]), (uint32_t)S.nc[d]);
  }
  const uint32_t k = (c[2] * (uint32_t)S.nc[1] + c[1]) * (uint32_t)S.nc[0] + c[0];
  S.key[i] = k;
  atomicAdd(&S.count[k], 1u);
}
__global__ void kb_rebin_keys(const Sys* __restrict__ T, const BlkMap* __restrict__ M, const uint32_t* __restrict__ C) {
  if (blockIdx.x >= *C) return;  // compacted map: members that rebuild
  const BlkMap m = M[blockIdx.x];
  const Sys& S = T[m.sys];
  if (!S.ctl->rebin_flag) return;  // this member needs no rebuild
  rebin_keys_body(S, Blk{m.b, m.nb});
}

// Restore: keys were uploaded (a checkpoint's cells); only count them.
__device__ __forceinline__ void count_keys_body(const Sys& S, const Blk blk) {
  const uint32_t i = blk.b * blockDim.x + threadIdx.x;
  if (i >= S.n) return;
  atomicAdd(&S.count[S.key[i]], 1u);
}

__global__ void k_count_keys(Sys S) { count_keys_body(S, Blk{blockIdx.x, gridDim.x}); }

// Exclusive scan of count[0..ncell) into cell_start[0..ncell], three passes.
__device__ __forceinline__ void scan_tiles_body(const Sys& S, const Blk blk) {
  __shared__ uint32_t red[256];
  const uint32_t* __restrict__ in = S.count;
  const uint32_t n = (uint32_t)S.ncell;
  const uint32_t base = blk.b * SCAN_TILE;
  uint32_t s = 0;
  for (int k = 0; k < SCAN_TILE / 256; ++k) {
    const uint32_t idx = base + k * 256 + threadIdx.x;
    if (idx < n) s += in[idx];
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) S.blk_off[blk.b] = red[0];
}
__global__ void k_scan_tiles(Sys S) { scan_tiles_body(S, Blk{blockIdx.x, gridDim.x}); }
__global__ void kb_scan_tiles(const Sys* __restrict__ T, const BlkMap* __restrict__ M, const uint32_t* __restrict__ C) {
  if (blockIdx.x >= *C) return;
  const BlkMap m = M[blockIdx.x];
  const Sys& S = T[m.sys];
  if (!S.ctl->rebin_flag) return;
  scan_tiles_body(S, Blk{m.b, m.nb});
}

__device__ __forceinline__ uint32_t block_exclusive_scan_256(uint32_t v, uint32_t& total) {
  __shared__ uint32_t warp_tot[8];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_tot[wid] = x;
  __syncthreads();
  if (wid == 0) {
    uint32_t t = lane < 8 ? warp_tot[lane] : 0u;
#pragma unroll
    for (int o = 1; o < 8; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, t, o);
      if (lane >= o) t += y;
    }
    if (lane < 8) warp_tot[lane] = t;
  }
  __syncthreads();
  const uint32_t before = wid ? warp_tot[wid - 1] : 0u;
  total = warp_tot[7];
  __syncthreads();
  return before + x - v;
}

// Single block: exclusive scan of the tile sums in place.
__device__ __forceinline__ void scan_top_body(const Sys& S) {
  uint32_t* tsum = S.blk_off;
  const uint32_t ntiles = ((uint32_t)S.ncell + SCAN_TILE - 1) / SCAN_TILE;
  uint32_t carry = 0;
  for (uint32_t base = 0; base < ntiles; base += 256) {
    const uint32_t idx = base + threadIdx.x;
    const uint32_t v = idx < ntiles ? tsum[idx] : 0u;
    uint32_t total;
    const uint32_t ex = block_exclusive_scan_256(v, total);
    if (idx < ntiles) tsum[idx] = carry + ex;
    carry += total;
  }
}
__global__ void k_scan_top(Sys S) { scan_top_body(S); }
__global__ void kb_scan_top(const Sys* __restrict__ T, const BlkMap* __restrict__ M, const uint32_t* __restrict__ C) {
  if (blockIdx.x >= *C) return;
  const Sys& S = T[M[blockIdx.x].sys];
  if (!S.ctl->rebin_flag) return;
  scan_top_body(S);
}

__device__ __forceinline__ void scan_down_body(const Sys& S, const Blk blk) {
  const uint32_t* __restrict__ in = S.count;
  const uint32_t n = (uint32_t)S.ncell;
  uint32_t* __restrict__ out = S.cell_start;
  const uint32_t base = blk.b * SCAN_TILE + threadIdx.x * (SCAN_TILE / 256);
  uint32_t loc[SCAN_TILE / 256];
  uint32_t s = 0;
#pragma unroll
  for (int k = 0; k < SCAN_TILE / 256; ++k) {
    loc[k] = (base + k < n) ? in[base + k] : 0u;
    s += loc[k];
  }
  uint32_t total;
  uint32_t run = S.blk_off[blk.b] + block_exclusive_scan_256(s, total);
  if (blk.b == 0 && threadIdx.x == 0) out[0] = 0u;
#pragma unroll
  for (int k = 0; k < SCAN_TILE / 256; ++k) {
    run += loc[k];
    if (base + k < n) out[base + k + 1] = run;
  }
}
// The same with the tile's offset summed from the tile sums by the block
// itself (no scan_top pass; for grids of at most 1,024 tiles).
__device__ __forceinline__ void scan_down_self_body(const Sys& S, const Blk blk) {
  const uint32_t* __restrict__ in = S.count;
  const uint32_t n = (uint32_t)S.ncell;
  uint32_t* __restrict__ out = S.cell_start;
  uint32_t part = 0;
  for (uint32_t t = threadIdx.x; t < blk.b; t += blockDim.x) part += S.blk_off[t];
  uint32_t off;
  (void)block_exclusive_scan_256(part, off);
  const uint32_t base = blk.b * SCAN_TILE + threadIdx.x * (SCAN_TILE / 256);
  uint32_t loc[SCAN_TILE / 256];
  uint32_t s = 0;
#pragma unroll
  for (int k = 0; k < SCAN_TILE / 256; ++k) {
    loc[k] = (base + k < n) ? in[base + k] : 0u;
    s += loc[k];
  }
  uint32_t total;
  uint32_t run = off + block_exclusive_scan_256(s, total);
  if (blk.b == 0 && threadIdx.x == 0) out[0] = 0u;
#pragma unroll
  for (int k = 0; k < SCAN_TILE / 256; ++k) {
    run += loc[k];
    if (base + k < n) out[base + k + 1] = run;
  }
}
__global__ void k_scan_down(Sys S) { scan_down_body(S, Blk{blockIdx.x, gridDim.x}); }
__global__ void k_scan_down_self(Sys S) { scan_down_self_body(S, Blk{blockIdx.x, gridDim.x}); }
__global__ void kb_scan_down(const Sys* __restrict__ T, const BlkMap* __restrict__ M, const uint32_t* __restrict__ C) {
  if (blockIdx.x >= *C) return;
  const BlkMap m = M[blockIdx.x];
  const Sys& S = T[m.sys];
  if (!S.ctl->rebin_flag) return;
  scan_down_body(S, Blk{m.b, m.nb});
}

// Batched rebuilds clear the cell counters in a kernel (a single system uses memsets).
__global__ void kb_rebin_clear(const Sys* __restrict__ T, const BlkMap* __restrict__ M, const uint32_t* __restrict__ C) {
  if (blockIdx.x >= *C) return;
  const BlkMap m = M[blockIdx.x];
  const Sys& S = T[m.sys];
  if (!S.ctl->rebin_flag) return;
  const uint32_t c = m.b * blockDim.x + threadIdx.x;
  if (c < (uint32_t)S.ncell) {
    S.count[c] = 0u;
    S.fill[c] = 0u;
  }
}

__device__ __forceinline__ void rebin_scatter_body(const Sys& S, const Blk blk) {
  const uint32_t i = blk.b * blockDim.x + threadIdx.x;
  if (i >= S.n) return;
  const uint32_t k = S.key[i];
  const uint32_t pos = atomicAdd(&S.fill[k], 1u);
  S.tmp[S.cell_start[k] + pos] = i;
}

__global__ void k_rebin_scatter(Sys S) { rebin_scatter_body(S, Blk{blockIdx.x, gridDim.x}); }
__global__ void kb_rebin_scatter(const Sys* __restrict__ T, const BlkMap* __restrict__ M, const uint32_t* __restrict__ C) {
  if (blockIdx.x >= *C) return;
  const BlkMap m = M[blockIdx.x];
  const Sys& S = T[m.sys];
  if (!S.ctl->rebin_flag) return;  // this member needs no rebuild
  rebin_scatter_body(S, Blk{m.b, m.nb});
}

// Sorts each cell's members by old slot: the order inside a cell then does
// not depend on the order in which the scatter's atomics completed.  Then
// records every member's new slot (new_of_old), for the permutation.
__device__ __forceinline__ void cas_u32(uint32_t& a, uint32_t& b) {
  const uint32_t lo = min(a, b), hi = max(a, b);
  a = lo;
  b = hi;
}
__device__ __forceinline__ void rebin_cellsort_body(const Sys& S, const Blk blk) {
  const uint32_t c = blk.b * blockDim.x + threadIdx.x;
  if (c >= (uint32_t)S.ncell) return;
  const uint32_t s0 = S.cell_start[c], s1 = S.cell_start[c + 1];
  if (s1 - s0 <= 8u) {
    // the common case: an 8-input sorting network in registers (absent
    // members padded with the largest key)
    uint32_t v[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) v[q] = s0 + q < s1 ? S.tmp[s0 + q] : 0xFFFFFFFFu;
    cas_u32(v[0], v[1]); cas_u32(v[2], v[3]); cas_u32(v[4], v[5]); cas_u32(v[6], v[7]);
    cas_u32(v[0], v[2]); cas_u32(v[1], v[3]); cas_u32(v[4], v[6]); cas_u32(v[5], v[7]);
    cas_u32(v[1], v[2]); cas_u32(v[5], v[6]); cas_u32(v[0], v[4]); cas_u32(v[3], v[7]);
    cas_u32(v[1], v[5]); cas_u32(v[2], v[6]);
    cas_u32(v[1], v[4]); cas_u32(v[3], v[6]);
    cas_u32(v[2], v[4]); cas_u32(v[3], v[5]);
    cas_u32(v[3], v[4]);
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      if (s0 + q < s1) {
        S.tmp[s0 + q] = v[q];
        S.new_of_old[v[q]] = s0 + q;
      }
    }
    return;
  }
  for (uint32_t a = s0 + 1; a < s1; ++a) {
    const uint32_t v = S.tmp[a];
    uint32_t b = a;
    while (b > s0 && S.tmp[b - 1] > v) {
      S.tmp[b] = S.tmp[b - 1];
      --b;
    }
    S.tmp[b] = v;
  }
  for (uint32_t a = s0; a < s1; ++a) S.new_of_old[S.tmp[a]] = a;
}

__global__ void k_rebin_cellsort(Sys S) { rebin_cellsort_body(S, Blk{blockIdx.x, gridDim.x}); }
__global__ void kb_rebin_cellsort(const Sys* __restrict__ T, const BlkMap* __restrict__ M, const uint32_t* __restrict__ C) {
  if (blockIdx.x >= *C) return;
  const BlkMap m = M[blockIdx.x];
  const Sys& S = T[m.sys];
  if (!S.ctl->rebin_flag) return;  // this member needs no rebuild
  rebin_cellsort_body(S, Blk{m.b, m.nb});
}

// New slot s takes old slot tmp[s]: copies every per-particle array into the
// other set (bond partners renamed to their new slots) and writes the
// fixed-point position with a fresh displacement reference; tmp[s] then
// receives the cell the sort put the slot in (read by the list build).
__device__ __forceinline__ void rebin_permute_one(const Sys& S, uint32_t s, bool wrap) {
  Ctl* ctl = S.ctl;
  const int set = ctl->set;
  const SoA A = set ? S.s1 : S.s0;
  const SoA B = set ? S.s0 : S.s1;
  uint4* P = ctl->phase ? S.P1 : S.P0;
  const uint32_t o = S.tmp[s];
  // every load first: a store into set B could alias a later load from set A
  // as far as the compiler knows, and would hold that load back
  double x = __ldg(A.x + o), y = __ldg(A.y + o), z = __ldg(A.z + o);
  const double vx = __ldg(A.vx + o), vy = __ldg(A.vy + o), vz = __ldg(A.vz + o);
  const uint32_t pid = __ldg(A.id + o);
  const uint8_t ty = __ldg(A.type + o);
  const int8_t st = __ldg(A.state + o);
  const uint32_t nb = __ldg(A.nadj + o);
  const uint32_t key = __ldg(S.key + o);
  uint32_t e[4];  // partners renamed to their new slots (the first four at once)
#pragma unroll
  for (int b = 0; b < 4; ++b) e[b] = b < (int)nb ? __ldg(A.adj + (size_t)o * S.cap + b) : 0u;
#pragma unroll
  for (int b = 0; b < 4; ++b)
    if (b < (int)nb) e[b] = __ldg(S.new_of_old + (e[b] & SLOT_MASK)) | (e[b] & ~SLOT_MASK);
  // positions re-enter the box here (a checkpoint restore keeps them as
  // saved, so that the continued run wraps them at the same step as the
  // original run)
  if (wrap) {
    x = wrap_into_box(x, S.L[0]);
    y = wrap_into_box(y, S.L[1]);
    z = wrap_into_box(z, S.L[2]);
  }
  B.x[s] = x;
  B.y[s] = y;
  B.z[s] = z;
  B.vx[s] = vx;
  B.vy[s] = vy;
  B.vz[s] = vz;
  B.id[s] = pid;
  B.type[s] = ty;
  B.state[s] = st;
  B.nadj[s] = (uint8_t)nb;
#pragma unroll
  for (int b = 0; b < 4; ++b)
    if (b < (int)nb) B.adj[(size_t)s * S.cap + b] = e[b];
  for (uint32_t b = 4; b < nb; ++b) {
    const uint32_t f = A.adj[(size_t)o * S.cap + b];
    B.adj[(size_t)s * S.cap + b] = S.new_of_old[f & SLOT_MASK] | (f & ~SLOT_MASK);
  }
  const uint32_t X = periodic_fx(x, S.Lfx[0], S.M64[0]);
  const uint32_t Y = periodic_fx(y, S.Lfx[1], S.M64[1]);
  const uint32_t Z = periodic_fx(z, S.Lfx[2], S.M64[2]);
  P[s] = make_uint4(X, Y, Z, coarse_ref(X, Y, Z, S.wshift));
  S.tmp[s] = key;
}

__device__ __forceinline__ void rebin_permute_body(const Sys& S, const Blk blk, bool wrap) {
  const uint32_t s = blk.b * blockDim.x + threadIdx.x;
  if (s < S.n) rebin_permute_one(S, s, wrap);
}
// Single system: the resident blocks' warps take 32-slot chunks strided by
// the grid's warp count (no partial last wave, as in k_step_nl).
__global__ void k_rebin_permute(Sys S, int wrap) {
  const uint32_t W = gridDim.x * (blockDim.x >> 5);
  for (uint32_t c = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); c * 32u < S.n; c += W) {
    const uint32_t i = c * 32u + (threadIdx.x & 31u);
    if (i < S.n) rebin_permute_one(S, i, wrap != 0);
  }
}
__global__ void kb_rebin_permute(const Sys* __restrict__ T, const BlkMap* __restrict__ M, const uint32_t* __restrict__ C) {
  if (blockIdx.x >= *C) return;
  const BlkMap m = M[blockIdx.x];
  const Sys& S = T[m.sys];
  if (!S.ctl->rebin_flag) return;  // this member needs no rebuild
  rebin_permute_body(S, Blk{m.b, m.nb}, true);
}

// ---------------------------------------------------------------------------
// Verlet-list build.  One block per tile of TY consecutive cell rows (cy0 ..
// cy0+TY-1 at one cz); threads = the tile's particles, contiguous in slot
// order (in passes of blockDim when a tile is longer).  All (TY+2) x 3
// neighbour rows are staged in shared memory as FP32 coordinates in the
// tile's frame (one pass in the common case), each row extended by one
// periodic image cell at both ends, so every particle's 3 x 3 x 3 cell
// neighbourhood is 9 contiguous ranges.  A pair enters the list when its
// FP32 distance is below r_c + skin (widened by the rounding bound).
// ---------------------------------------------------------------------------
// 16-byte copy global -> shared that does not wait for the data (cp.async,
// L2 only); cp_async_wait_all() waits for every copy the thread issued.
__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gsrc) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

struct RowInfo {
  int base;        // first staged index of the row
  int padL;        // particles of the left image cell (cell nx-1)
  int rowcount;    // particles of the row
  int tot;         // padL + rowcount + padR
  int row_lo;      // first slot of the row
  int left_start;  // first slot of cell nx-1
  int c1;          // first slot of cell 1 (end of cell 0)
  uint32_t yref;   // fixed-point lower edge of the (wrapped) row in y
  uint32_t zref;   // and in z
  float yoff;      // that edge's offset from the tile's lower edge, unwrapped
  float zoff;
  int pad;
};
constexpr int TILE_ROWS_MAX = 18;  // (TY + 2) x 3 for TY <= 4

// FP32 coordinates of a staged particle in the tile's frame: y and z relative
// to the tile's lower cell edges (each row's images unwrapped), x in [0, L)
// with the left and right image cells shifted by -L and +L.  A slot keyed to
// cell 0 (nx-1) whose position rounds to the far end of the box (possible by
// one rounding step after a restore) is taken back to the near side.  The
// values carry ~1e-5 sigma of rounding; the list radius has a margin for it.
__device__ __forceinline__ float4 build_coords(const uint4 p, const RowInfo& r, int kr,
                                               uint32_t slot, float sx, float sy, float sz,
                                               float Lx) {
  float xf = __uint2float_rn(p.x) * sx;
  if (slot < (uint32_t)r.c1 && p.x >= 0x80000000u) xf -= Lx;
  if (slot >= (uint32_t)r.left_start && p.x < 0x80000000u) xf += Lx;
  if (kr < r.padL) xf -= Lx;
  else if (kr >= r.padL + r.rowcount) xf += Lx;
  const float yf = fmaf(__int2float_rn(pdiff(p.y, r.yref)), sy, r.yoff);
  const float zf = fmaf(__int2float_rn(pdiff(p.z, r.zref)), sz, r.zoff);
  return make_float4(xf, yf, zf, __uint_as_float(slot));
}

// One candidate: hit = r2 < rv2; a hit is written to row `cnt` of the
// slot's column while cnt < cap, and cnt counts every hit (cnt > cap
// afterwards means the list overflowed).  The caller never passes the
// particle itself.  Predicated PTX, so that the warp does not diverge on the
// (frequent) hits.
template <bool NL16>
__device__ __forceinline__ void list_candidate(unsigned char* col, uint32_t stride, float r2,
                                               float rv2, uint32_t qslot, int cap, int& cnt) {
  if constexpr (NL16) {
    asm volatile(
        "{\n\t.reg .pred h, w;\n\t.reg .u64 a;\n\t"
        "setp.lt.f32 h, %1, %2;\n\t"
        "setp.lt.and.s32 w, %0, %4, h;\n\t"
        "mad.wide.u32 a, %0, %5, %6;\n\t"
        "@w st.global.u16 [a], %7;\n\t"
        "@h add.s32 %0, %0, 1;\n\t}"
        : "+r"(cnt)
        : "f"(r2), "f"(rv2), "r"(qslot), "r"(cap), "r"(stride), "l"(col), "h"((uint16_t)qslot)
        : "memory");
  } else {
    asm volatile(
        "{\n\t.reg .pred h, w;\n\t.reg .u64 a;\n\t"
        "setp.lt.f32 h, %1, %2;\n\t"
        "setp.lt.and.s32 w, %0, %4, h;\n\t"
        "mad.wide.u32 a, %0, %5, %6;\n\t"
        "@w st.global.u32 [a], %3;\n\t"
        "@h add.s32 %0, %0, 1;\n\t}"
        : "+r"(cnt)
        : "f"(r2), "f"(rv2), "r"(qslot), "r"(cap), "r"(stride), "l"(col)
        : "memory");
  }
}

template <bool NL16>
__device__ __forceinline__ void build_nlist_body(const Sys& S, const Blk blk, unsigned char* smem) {
  const int CAP = S.tile_cap;
  float4* sX = reinterpret_cast<float4*>(smem);
  RowInfo* ri = reinterpret_cast<RowInfo*>(smem + 16 * (size_t)CAP);
  uint32_t* sCS = reinterpret_cast<uint32_t*>(ri + TILE_ROWS_MAX);
  __shared__ int sTOT;
  __shared__ unsigned int warps_left;
  if (threadIdx.x == 0) warps_left = blockDim.x >> 5;

  Ctl* ctl = S.ctl;
  const uint4* __restrict__ P = ctl->phase ? S.P1 : S.P0;
  const int nx = S.nc[0], ny = S.nc[1], nz = S.nc[2];
  const int ty = blk.b % S.tiles_y, cz = blk.b / S.tiles_y;
  const int cy0 = ty * S.tile_y;
  const int TYb = min(S.tile_y, ny - cy0);
  const int RY = TYb + 2, R = 3 * RY;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const uint32_t rs = S.cell_start[(cz * ny + cy0) * nx];
  const uint32_t re = S.cell_start[(cz * ny + cy0 + TYb - 1) * nx + nx];

  for (int k = threadIdx.x; k < R * (nx + 1); k += blockDim.x) {
    const int sr = k / (nx + 1), c = k - sr * (nx + 1);
    const int dzi = sr / RY, yi = sr - dzi * RY;
    const int qz = wrap_cell(cz - 1 + dzi, nz), qy = wrap_cell(cy0 - 1 + yi, ny);
    sCS[k] = S.cell_start[(qz * ny + qy) * nx + c];
  }
  __syncthreads();
  if (threadIdx.x < R) {
    const uint32_t* cs = sCS + threadIdx.x * (nx + 1);
    const int dzi = threadIdx.x / RY, yi = threadIdx.x - dzi * RY;
    const int uy = cy0 - 1 + yi, uz = cz - 1 + dzi;  // unwrapped row indices
    const int qy = wrap_cell(uy, ny), qz = wrap_cell(uz, nz);
    RowInfo r;
    r.padL = (int)(cs[nx] - cs[nx - 1]);
    r.rowcount = (int)(cs[nx] - cs[0]);
    r.tot = r.padL + r.rowcount + (int)(cs[1] - cs[0]);
    r.row_lo = (int)cs[0];
    r.left_start = (int)cs[nx - 1];
    r.c1 = (int)cs[1];
    r.yref = (uint32_t)(((unsigned long long)qy << 32) / (unsigned)ny);
    r.zref = (uint32_t)(((unsigned long long)qz << 32) / (unsigned)nz);
    r.yoff = (float)((double)(uy - cy0) * (S.L[1] / ny));
    r.zoff = (float)((double)(uz - cz) * (S.L[2] / nz));
    r.base = 0;
    r.pad = 0;
    ri[threadIdx.x] = r;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int run = 0;
    for (int sr = 0; sr < R; ++sr) {
      ri[sr].base = run;
      run += ri[sr].tot;
    }
    sTOT = run;
  }
  __syncthreads();
  const int TOT = sTOT;
  const float sx = S.scale[0], sy = S.scale[1], sz = S.scale[2], rv2 = S.rv2_build;
  const float Lx = (float)S.L[0];

  // Stages entries [c0, c0 + cn) of the neighbour rows, one warp per row:
  // raw copies in flight at once (cp.async), then each lane turns the
  // entries it copied into tile-frame FP32 coordinates in place (the same
  // warp/lane mapping, so no block barrier in between).
  auto stage = [&](int c0, int cn) {
    for (int sr = warp; sr < R; sr += nwarps) {
      const RowInfo& r = ri[sr];
      const int k0 = max(r.base, c0), k1 = min(r.base + r.tot, c0 + cn);
      const int padL = r.padL, rc = r.rowcount, lo = r.row_lo, ls = r.left_start, b = r.base;
      for (int ent = k0 + lane; ent < k1; ent += 32) {
        const int kr = ent - b;
        const int slot = kr < padL ? ls + kr : (kr < padL + rc ? lo + kr - padL : lo + kr - padL - rc);
        cp_async16(&sX[ent - c0], P + slot);
      }
    }
    cp_async_wait_all();
    __syncwarp();
    for (int sr = warp; sr < R; sr += nwarps) {
      const RowInfo r = ri[sr];
      const int k0 = max(r.base, c0), k1 = min(r.base + r.tot, c0 + cn);
      for (int ent = k0 + lane; ent < k1; ent += 32) {
        const int kr = ent - r.base;
        const int slot = kr < r.padL ? r.left_start + kr
                                     : r.row_lo + (kr < r.padL + r.rowcount ? kr - r.padL
                                                                            : kr - r.padL - r.rowcount);
        const float4 raw = sX[ent - c0];
        const uint4 p = make_uint4(__float_as_uint(raw.x), __float_as_uint(raw.y),
                                   __float_as_uint(raw.z), 0u);
        sX[ent - c0] = build_coords(p, r, kr, (uint32_t)slot, sx, sy, sz, Lx);
      }
    }
  };
  const bool one = TOT <= CAP;  // the common case: every row staged once
  if (one) {
    stage(0, TOT);
    __syncthreads();
  }

  for (uint32_t base = rs; base < re; base += blockDim.x) {
    const uint32_t i = base + threadIdx.x;
    const bool act = i < re;
    const uint4 pi = act ? P[i] : make_uint4(0u, 0u, 0u, 0u);
    // the cell the sort put this slot in (not the one its current position
    // maps to: after a checkpoint restore the two can differ by one)
    const uint32_t kc = act ? S.tmp[i] : (uint32_t)((cz * ny + cy0) * nx);
    int cx = (int)(kc % (uint32_t)nx);
    int yrel = (int)((kc / (uint32_t)nx) % (uint32_t)ny) - cy0;
    if (yrel < 0 || yrel >= TYb) {  // cannot happen for a consistent sort
      set_status(ctl, PRX_EINVAL);
      yrel = 0;
      cx = 0;
    }
    uint32_t win[9];
#pragma unroll
    for (int w = 0; w < 9; ++w) {
      const int sr = (w / 3) * RY + yrel + (w % 3);
      const uint32_t* cs = sCS + sr * (nx + 1);
      const RowInfo& r = ri[sr];
      const int lo = r.base + (cx == 0 ? 0 : r.padL + (int)cs[cx - 1] - r.row_lo);
      const int hi = r.base + (cx + 2 > nx ? r.tot : r.padL + (int)cs[cx + 2] - r.row_lo);
      win[w] = (uint32_t)lo | ((uint32_t)hi << 16);
    }
    float4 fi;
    int kself0;  // the particle's own entry in the staged centre row
    {
      const RowInfo& r = ri[RY + yrel + 1];
      fi = build_coords(pi, r, r.padL + ((int)i - r.row_lo), i, sx, sy, sz, Lx);
      kself0 = r.base + r.padL + ((int)i - r.row_lo);
    }
    int cnt = 0;
    const int cap = S.list_cap;
    unsigned char* col = (unsigned char*)S.nl + (size_t)i * (NL16 ? 2 : 4);
    const uint32_t stride = S.n * (NL16 ? 2u : 4u);
    for (int c0 = 0; c0 < TOT; c0 += CAP) {
      const int cn = min(CAP, TOT - c0);
      if (!one) {  // neighbour rows longer than the buffer: staged per chunk
        __syncthreads();
        stage(c0, cn);
        __syncthreads();
      }
      if (act) {
        // the particle itself is staged once, in the centre row's window
        // (w = 4), whose walk skips it: no candidate needs a self test
        const int kself = kself0 - c0;
#pragma unroll
        for (int w = 0; w < 9; ++w) {
          const int lo = max((int)(win[w] & 0xFFFFu), c0) - c0;
          const int hi = min((int)(win[w] >> 16), c0 + cn) - c0;
          auto walk = [&](int a, int b) {
#pragma unroll 2
            for (int k = a; k < b; ++k) {
              const float4 q = sX[k];
              const float dx = q.x - fi.x, dy = q.y - fi.y, dz = q.z - fi.z;
              list_candidate<NL16>(col, stride, fmaf(dz, dz, fmaf(dy, dy, dx * dx)), rv2,
                                   __float_as_uint(q.w), cap, cnt);
            }
          };
          if (w == 4) {
            walk(lo, min(hi, max(lo, kself)));
            walk(max(lo, kself + 1), hi);
          } else {
            walk(lo, hi);
          }
        }
      }
    }
    if (act) {
      const int m = min(cnt, cap);
      S.nn[i] = (uint8_t)m;
      if (cnt > cap) set_status(ctl, PRX_ECAPACITY);
      // pad to a whole stage of four with the slot itself (the step kernel
      // gathers four entries at a time; the self pair has r = 0 and no force)
      for (int k = m; k < ((m + 3) & ~3); ++k) {
        if constexpr (NL16) ((uint16_t*)S.nl)[(size_t)k * S.n + i] = (uint16_t)i;
        else ((uint32_t*)S.nl)[(size_t)k * S.n + i] = i;
      }
    }
  }
  // the last warp of the system's tiles flips the SoA set and clears the
  // flag (a warp count, not a block barrier: warps that finish early leave)
  if (last_warp(&ctl->done_rebin, &warps_left, blk.nb)) {
    ctl->done_rebin = 0u;
    ctl->set ^= 1;
    ctl->rebin_flag = 0;
    ctl->rebins += 1ull;
  }
}

template <bool NL16>
__global__ void __launch_bounds__(256) k_build_nlist(Sys S) {
  extern __shared__ __align__(16) unsigned char smem_b[];
  build_nlist_body<NL16>(S, Blk{blockIdx.x, gridDim.x}, smem_b);
}
__global__ void __launch_bounds__(256)
    kb_build_nlist(const Sys* __restrict__ T, const BlkMap* __restrict__ M, const uint32_t* __restrict__ C) {
  extern __shared__ __align__(16) unsigned char smem_b[];
  if (blockIdx.x >= *C) return;
  const BlkMap m = M[blockIdx.x];
  const Sys& S = T[m.sys];
  if (!S.ctl->rebin_flag) return;
  if (S.nl16) build_nlist_body<true>(S, Blk{m.b, m.nb}, smem_b);
  else build_nlist_body<false>(S, Blk{m.b, m.nb}, smem_b);
}

inline unsigned blocks_for(uint64_t n, int t) { return (unsigned)((n + t - 1) / t); }

// Rebuild plan of a batch: the entries of the five block maps (stored one
// after the other: part, cell, tile, one, build) that belong to members
// whose rebuild flag is set, compacted into `act` at the same family offsets,
// with their counts in act_n.  The lanes of a warp that append to the same
// family reserve their places with one atomic; the order of the compacted
// entries does not matter (every block's work depends only on its entry).
__global__ void kb_rebuild_plan(const Sys* __restrict__ T, const BlkMap* __restrict__ maps,
                                uint4 off, uint32_t n_all, BlkMap* __restrict__ act,
                                uint32_t* __restrict__ act_n) {
  const uint32_t e = blockIdx.x * blockDim.x + threadIdx.x;
  int fam = -1;
  BlkMap m{};
  if (e < n_all) {
    m = maps[e];
    if (T[m.sys].ctl->rebin_flag)
      fam = e < off.x ? 0 : e < off.y ? 1 : e < off.z ? 2 : e < off.w ? 3 : 4;
  }
  const unsigned grp = __match_any_sync(0xFFFFFFFFu, fam);
  const int lane = threadIdx.x & 31, lead = __ffs(grp) - 1;
  uint32_t base = 0u;
  if (fam >= 0 && lane == lead) base = atomicAdd(&act_n[fam], (uint32_t)__popc(grp));
  base = __shfl_sync(0xFFFFFFFFu, base, lead);
  if (fam >= 0) {
    const uint32_t start = fam == 0 ? 0u : fam == 1 ? off.x : fam == 2 ? off.y : fam == 3 ? off.z : off.w;
    act[start + base + __popc(grp & ((1u << lane) - 1u))] = m;
  }
}

// Input staging for a plain creation (slot = particle index).  Positions are
// wrapped by at most one box edge (v >= L: v - L; v < 0: v + L, FP64), the
// same operations as the host-side restore path.
__global__ void k_stage_input(Sys S, const double* __restrict__ buf, int which) {
  const uint32_t s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= S.n) return;
  const SoA& B = S.s0;
  double c[3];
  unsigned err = 0u;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    double v = buf[3 * (size_t)s + k];
    if (which == 0) {
      if (!isfinite(v)) {
        err = max(err, 1u);
      } else {
        if (v >= S.L[k]) v = __dsub_rn(v, S.L[k]);
        if (v < 0.0) v = __dadd_rn(v, S.L[k]);
        if (!(v >= 0.0 && v < S.L[k])) err = max(err, 2u);
      }
    }
    c[k] = v;
  }
  if (which == 0) {
    B.x[s] = c[0];
    B.y[s] = c[1];
    B.z[s] = c[2];
    B.id[s] = s;
    if (B.type[s] >= PRX_MAX_TYPES) err = max(err, 3u);
    if (err) atomicMax(&S.ctl->input_err, err);
  } else {
    B.vx[s] = c[0];
    B.vy[s] = c[1];
    B.vz[s] = c[2];
  }
}

}  // namespace

// Read-back in particle order: slot s of the current set goes to index id[s]
// of `out` (device): 0 states (i8), 1 types (u8), 2 positions wrapped once
// into the box (the permutation's rule), [n][3], 3 velocities [n][3].
__global__ void k_gather_by_id(Sys S, int what, void* __restrict__ out) {
  const uint32_t s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= S.n) return;
  const SoA B = S.ctl->set ? S.s1 : S.s0;
  const uint32_t p = B.id[s];
  if (what == 0) {
    ((int8_t*)out)[p] = B.state[s];
  } else if (what == 1) {
    ((uint8_t*)out)[p] = B.type[s];
  } else if (what == 2) {
    double* o = (double*)out + 3 * (size_t)p;
    o[0] = wrap_into_box(B.x[s], S.L[0]);
    o[1] = wrap_into_box(B.y[s], S.L[1]);
    o[2] = wrap_into_box(B.z[s], S.L[2]);
  } else {
    double* o = (double*)out + 3 * (size_t)p;
    o[0] = B.vx[s];
    o[1] = B.vy[s];
    o[2] = B.vz[s];
  }
}

void launch_gather_by_id(const Sys& S, cudaStream_t st, int what, void* out) {
  if (S.n) k_gather_by_id<<<blocks_for(S.n, 256), 256, 0, st>>>(S, what, out);
}

void launch_stage_input(const Sys& S, cudaStream_t st, const double* buf, int which) {
  if (S.n) k_stage_input<<<blocks_for(S.n, 256), 256, 0, st>>>(S, buf, which);
}

// Blocks of `threads` threads of kernel `kern` resident on the whole current
// device at once (cached per device and kernel id: the step kernel's
// variants and block sizes).
// Multiprocessors of the current device (cached per device).
unsigned device_sms() {
  static unsigned cache[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 1u;
  if (!cache[dev]) {
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) {
      cudaGetLastError();
      return 1u;
    }
    cache[dev] = (unsigned)sms;
  }
  return cache[dev];
}

unsigned resident_blocks(int variant, const void* kern, int threads) {
  static std::mutex mu;
  static unsigned cache[64][64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 1u;
  std::lock_guard<std::mutex> lk(mu);
  unsigned& c = cache[dev][variant & 63];
  if (!c) {
    int sms = 0, per = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, threads, 0) != cudaSuccess) {
      cudaGetLastError();
      return 1u;
    }
    c = sms * per > 0 ? (unsigned)(sms * per) : 1u;
  }
  return c;
}

void launch_step(const Sys& S, cudaStream_t st, int fp64, int forces_only,
                 cudaGraphConditionalHandle h, int use_cond) {
  if (fp64) {
    const unsigned gf = blocks_for(S.n, 32 / F64_LANES) > 0 ? blocks_for(S.n, 32 / F64_LANES) : 1;
    if (forces_only) {
      if (S.nl16) k_forces64<true, true><<<gf, 32, 0, st>>>(S);
      else k_forces64<false, true><<<gf, 32, 0, st>>>(S);
    } else {
      if (S.nl16) k_forces64<true, false><<<gf, 32, 0, st>>>(S);
      else k_forces64<false, false><<<gf, 32, 0, st>>>(S);
      const unsigned gi = blocks_for(S.n, 32) > 0 ? blocks_for(S.n, 32) : 1;
      k_integrate64<<<gi, 32, 0, st>>>(S, h, use_cond);
    }
  } else {
    // forces-only launches keep 256 threads; the step takes the launch
    // configuration's block size and blocks per SM; both take its lanes per
    // slot (so that prx_compute_forces sums as the step does)
    const int bt = forces_only ? 256 : S.step_bt;
    auto K = [&](auto nl16, auto fo, auto cub) {
      constexpr bool N16 = decltype(nl16)::value, FO = decltype(fo)::value, CU = decltype(cub)::value;
      constexpr int v = (N16 ? 4 : 0) + (FO ? 2 : 0) + (CU ? 1 : 0);
      auto go = [&](auto btc) {
        constexpr int BT = decltype(btc)::value;
        const bool four = S.step_lanes == 4;
        auto* kern = four ? k_step_nl4<N16, FO, CU, BT> : k_step_nl<N16, FO, CU, BT>;
        const unsigned per = four ? BT / 4 : BT;  // slots per block
        const unsigned g0 = blocks_for(S.n, per) > 0 ? blocks_for(S.n, per) : 1;
        unsigned r = resident_blocks(v + 8 * (BT == 128 ? 1 : (BT == 512 ? 2 : 0)) + (four ? 32 : 0),
                                     (const void*)kern, BT);
        if (!FO && S.step_bpsm > 0) {
          const unsigned want = (unsigned)S.step_bpsm * (unsigned)device_sms();
          r = want < r ? want : r;
        }
        kern<<<(g0 < r ? g0 : r), BT, 0, st>>>(S, h, use_cond);
      };
      if constexpr (FO) {
        go(std::integral_constant<int, 256>{});
      } else {
        if (bt == 128) go(std::integral_constant<int, 128>{});
        else if (bt == 512) go(std::integral_constant<int, 512>{});
        else go(std::integral_constant<int, 256>{});
      }
    };
    using T_ = std::true_type;
    using F_ = std::false_type;
    if (S.cubic) {
      if (S.nl16) forces_only ? K(T_{}, T_{}, T_{}) : K(T_{}, F_{}, T_{});
      else forces_only ? K(F_{}, T_{}, T_{}) : K(F_{}, F_{}, T_{});
    } else {
      if (S.nl16) forces_only ? K(T_{}, T_{}, F_{}) : K(T_{}, F_{}, F_{});
      else forces_only ? K(F_{}, T_{}, F_{}) : K(F_{}, F_{}, F_{});
    }
  }
}

int step_kernel_count(int fp64) { return fp64 ? 2 : 1; }

size_t build_tile_smem(const Sys& S) {
  return 16 * (size_t)S.tile_cap + sizeof(RowInfo) * TILE_ROWS_MAX +
         4 * (size_t)TILE_ROWS_MAX * (S.nc[0] + 1);
}

// The dynamic shared-memory limit is an attribute of the kernel (per device),
// shared by every system: it only ever grows, to the largest tile any system
// on the device has asked for, so that systems of different sizes coexist.
namespace {
std::mutex g_smem_mu;
size_t g_smem_set[2][64];  // [single, batched][device]
int raise_smem_limit(int which, size_t bytes) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return -1;
  std::lock_guard<std::mutex> lk(g_smem_mu);
  if (bytes <= g_smem_set[which][dev]) return 0;
  bool ok;
  if (which == 0) {
    ok = cudaFuncSetAttribute(k_build_nlist<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)bytes) == cudaSuccess &&
         cudaFuncSetAttribute(k_build_nlist<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)bytes) == cudaSuccess;
  } else {
    ok = cudaFuncSetAttribute(kb_build_nlist, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)bytes) == cudaSuccess;
  }
  if (!ok) return -1;
  g_smem_set[which][dev] = bytes;
  return 0;
}
}  // namespace

int configure_build_kernel(size_t smem_bytes) { return raise_smem_limit(0, smem_bytes); }

constexpr unsigned kScanSelfTiles = 1024;  // tiles up to which the scan has two passes

int rebin_kernel_count(const Sys& S) {
  return (S.ncell + SCAN_TILE - 1) / SCAN_TILE <= (int)kScanSelfTiles ? 7 : 8;
}

// Whole rebuild: keys and counts (mode 0: from the fixed-point positions of
// the last step; 1: from the FP64 positions; 2: given), scan, scatter,
// per-cell sort, permutation (with the adjacency renamed), Verlet lists.  `hook`
// (optional) is called before (0) and after (1) each launch with the
// kernel's name, for event timing.
void launch_rebin(const Sys& S, cudaStream_t st, int mode, void (*hook)(void*, const char*, int),
                  void* ctx) {
  const unsigned gp = blocks_for(S.n, 256) ? blocks_for(S.n, 256) : 1;
  const unsigned gc = blocks_for(S.ncell, 256);
  const unsigned tiles = blocks_for(S.ncell, SCAN_TILE);
  auto H = [&](const char* nm, int p) {
    if (hook) hook(ctx, nm, p);
  };
  cudaMemsetAsync(S.count, 0, sizeof(uint32_t) * S.ncell, st);
  cudaMemsetAsync(S.fill, 0, sizeof(uint32_t) * S.ncell, st);
  H(mode == 2 ? "count_keys" : "rebin_keys", 0);
  if (mode == 2) k_count_keys<<<gp, 256, 0, st>>>(S);
  else if (mode == 1) k_rebin_keys_x<<<gp, 256, 0, st>>>(S);
  else k_rebin_keys<<<gp, 256, 0, st>>>(S);
  H(mode == 2 ? "count_keys" : "rebin_keys", 1);
  H("scan_tiles", 0);
  k_scan_tiles<<<tiles, 256, 0, st>>>(S);
  H("scan_tiles", 1);
  if (tiles <= kScanSelfTiles) {
    H("scan_down", 0);
    k_scan_down_self<<<tiles, 256, 0, st>>>(S);
    H("scan_down", 1);
  } else {
    H("scan_top", 0);
    k_scan_top<<<1, 256, 0, st>>>(S);
    H("scan_top", 1);
    H("scan_down", 0);
    k_scan_down<<<tiles, 256, 0, st>>>(S);
    H("scan_down", 1);
  }
  H("rebin_scatter", 0);
  k_rebin_scatter<<<gp, 256, 0, st>>>(S);
  H("rebin_scatter", 1);
  H("rebin_cellsort", 0);
  k_rebin_cellsort<<<gc, 256, 0, st>>>(S);
  H("rebin_cellsort", 1);
  H("rebin_permute", 0);
  {
    const unsigned r = resident_blocks(8, (const void*)k_rebin_permute, 256);
    k_rebin_permute<<<(gp < r ? gp : r), 256, 0, st>>>(S, mode != 2);
  }
  H("rebin_permute", 1);
  const unsigned gt = (unsigned)(S.tiles_y * S.nc[2]);
  const size_t sm = build_tile_smem(S);
  H("build_nlist", 0);
  if (S.nl16) k_build_nlist<true><<<gt, S.tile_threads, sm, st>>>(S);
  else k_build_nlist<false><<<gt, S.tile_threads, sm, st>>>(S);
  H("build_nlist", 1);
}

void launch_batch_step(const BatchLaunch& L, cudaStream_t st, cudaGraphConditionalHandle h,
                       int use_cond) {
  // variants in the order of the part map: (nl16, cubic) = 00, 01, 10, 11
  if (L.step_n[0]) kb_step_nl<false, false><<<L.step_n[0], 256, 0, st>>>(L.T, L.part + L.step_off[0], h, use_cond, L.act_n);
  if (L.step_n[1]) kb_step_nl<false, true><<<L.step_n[1], 256, 0, st>>>(L.T, L.part + L.step_off[1], h, use_cond, L.act_n);
  if (L.step_n[2]) kb_step_nl<true, false><<<L.step_n[2], 256, 0, st>>>(L.T, L.part + L.step_off[2], h, use_cond, L.act_n);
  if (L.step_n[3]) kb_step_nl<true, true><<<L.step_n[3], 256, 0, st>>>(L.T, L.part + L.step_off[3], h, use_cond, L.act_n);
}

// The rebuild pipeline over the members whose flag is set: a plan kernel
// compacts their blocks, then every kernel runs the full grid of its family,
// its blocks beyond the compacted count returning at once.
void launch_batch_rebuild(const BatchLaunch& L, cudaStream_t st) {
  const uint32_t o1 = L.n_part, o2 = o1 + L.n_cell, o3 = o2 + L.n_tile, o4 = o3 + L.n_one;
  const uint32_t n_all = o4 + L.n_build;
  kb_rebuild_plan<<<blocks_for(n_all, 256), 256, 0, st>>>(L.T, L.part, make_uint4(o1, o2, o3, o4), n_all,
                                                           L.act, L.act_n);
  const BlkMap *part = L.act, *cell = L.act + o1, *tile = L.act + o2, *one = L.act + o3, *build = L.act + o4;
  const uint32_t *c_part = L.act_n, *c_cell = L.act_n + 1, *c_tile = L.act_n + 2, *c_one = L.act_n + 3,
                 *c_build = L.act_n + 4;
  kb_rebin_clear<<<L.n_cell, 256, 0, st>>>(L.T, cell, c_cell);
  kb_rebin_keys<<<L.n_part, 256, 0, st>>>(L.T, part, c_part);
  kb_scan_tiles<<<L.n_tile, 256, 0, st>>>(L.T, tile, c_tile);
  kb_scan_top<<<L.n_one, 256, 0, st>>>(L.T, one, c_one);
  kb_scan_down<<<L.n_tile, 256, 0, st>>>(L.T, tile, c_tile);
  kb_rebin_scatter<<<L.n_part, 256, 0, st>>>(L.T, part, c_part);
  kb_rebin_cellsort<<<L.n_cell, 256, 0, st>>>(L.T, cell, c_cell);
  kb_rebin_permute<<<L.n_part, 256, 0, st>>>(L.T, part, c_part);
  kb_build_nlist<<<L.n_build, L.build_threads, L.build_smem, st>>>(L.T, build, c_build);
}

int batch_rebuild_kernel_count() { return 10; }

int configure_batch_build_kernel(size_t smem_bytes) { return raise_smem_limit(1, smem_bytes); }

}  // namespace prx
