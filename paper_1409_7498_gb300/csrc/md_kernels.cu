// MD kernels: the fused force + Langevin velocity-Verlet step, and the
// cell-list rebuild (deterministic counting sort of the slots by cell).
//
// Step kernel, one thread per slot (FP32 force mode):
//   WCA (Sec. II.C, Eq. 15) over the 27 neighbour cells on FP32 positions
//   relative to each particle's cell origin; FENE (Sec. II.C) or mirror LJ
//   (Eq. 17) over the adjacency row; Langevin random force keyed by
//   (seed, step, id); then in FP64: v' = a v + b F (one DFMA per component),
//   x' = x + dt v' (one DFMA).  The new FP32 offset comes from x' through an
//   exact fixed-point read of its binary64 fields, so the FP64 pipe (which
//   runs about 70x slower than FP32 on this part) sees only the six DFMAs.
#include <cuda_runtime.h>

#include "prx_internal.cuh"

namespace prx {

namespace {

// WCA pair term in FP32; d = x_j - x_i.  Adds -g d to f and V/2 to e.
__device__ __forceinline__ void wca32(const Sys& S, float dx, float dy, float dz, float r2,
                                      float& fx, float& fy, float& fz, float& e) {
  const float r2i = __fdiv_rn(1.0f, r2);
  const float sr2 = S.sig2f * r2i;
  const float sr6 = sr2 * sr2 * sr2;
  float g = S.eps24f * sr6 * (2.0f * sr6 - 1.0f) * r2i;
  if (S.fcapf > 0.0f) {
    const float r = sqrtf(r2);
    if (g * r > S.fcapf) g = S.fcapf / r;
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
    const float q = 1.0f - r2 / S.fr02f;
    g = -S.fkf / q;
    e += 0.5f * (-0.5f * S.fkf * S.fr02f * logf(q));
  } else {
    const float r = sqrtf(r2);
    if (!(r > S.rcf && r < 2.0f * S.rcf)) return true;
    const float sd = 2.0f * S.rcf - r;
    const float ss2 = S.sig2f / (sd * sd);
    const float ss6 = ss2 * ss2 * ss2;
    const float dVdr = S.eps24f * (2.0f * ss6 * ss6 - ss6) / sd;
    g = -dVdr / r;
    e += 0.5f * S.eps4f * (ss6 * ss6 - ss6 + 0.25f);
  }
  fx -= g * dx;
  fy -= g * dy;
  fz -= g * dz;
  return true;
}

// FP64 versions, arithmetic written as in the plain definitions.
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
  e = __dadd_rn(e, __dmul_rn(0.5, __dmul_rn(S.eps4, __dadd_rn(__dsub_rn(sr12, sr6), 0.25))));
}

__device__ __forceinline__ bool bond64(const Sys& S, uint32_t style, double dx, double dy,
                                       double dz, double& fx, double& fy, double& fz, double& e) {
  const double r2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
  double g;
  if (style == 0u) {
    if (!(r2 < S.fr02)) return false;
    const double q = __dsub_rn(1.0, __ddiv_rn(r2, S.fr02));
    g = __ddiv_rn(-S.fk, q);
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
    e = __dadd_rn(e, __dmul_rn(0.5, __dmul_rn(S.eps4, __dadd_rn(__dsub_rn(ss12, ss6), 0.25))));
  }
  fx = __dsub_rn(fx, __dmul_rn(g, dx));
  fy = __dsub_rn(fy, __dmul_rn(g, dy));
  fz = __dsub_rn(fz, __dmul_rn(g, dz));
  return true;
}

// New cell offset of a freshly integrated coordinate, in 2^-32 fixed point.
__device__ __forceinline__ long long cell_offset_fx(double x, int c, long long H) {
  return fx32(x) - (long long)c * H;
}

// Last block of a grid: returns true in thread 0 of the block that finished last.
__device__ __forceinline__ bool last_block(unsigned int* counter) {
  __shared__ bool is_last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned int prev = atomicAdd(counter, 1u);
    is_last = (prev == gridDim.x - 1);
  }
  __syncthreads();
  return is_last && threadIdx.x == 0;
}

// Exact displacement x_j - x_i in 2^-29 units from two cell-relative offsets,
// the cell difference wrapped to the nearest periodic image.  Unsigned
// arithmetic: the result is exact whenever it fits in 32 bits.
__device__ __forceinline__ int exact_d29(int oj, int oi, int cj, int ci, int n, int H, int corr) {
  int raw = cj - ci;
  uint32_t c = 0u;
  if (raw > n / 2) {
    raw -= n;
    c = (uint32_t)(-corr);
  } else if (raw < -(n / 2)) {
    raw += n;
    c = (uint32_t)corr;
  }
  return (int)((uint32_t)oj - (uint32_t)oi + (uint32_t)(raw * H) + c);
}

// End of a step for one slot: Langevin kick (friction applied exactly in
// FP64), drift, new fixed-point cell offset, rebuild trigger.
//   v' = a v + b (F_c + R),  x' = x + dt v'           (FP32 forces)
__device__ __forceinline__ void integrate32(const Sys& S, Ctl* ctl, const SoA& B, int4* offn,
                                            uint32_t i, int4 oi, int cx, int cy, int cz,
                                            unsigned long long step, float fx, float fy,
                                            float fz, double xi, double yi, double zi, double vx,
                                            double vy, double vz) {
  const uint32_t pid = B.id[i];
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
  const long long ox = cell_offset_fx(nx, cx, S.Hfx[0]);
  const long long oy = cell_offset_fx(ny, cy, S.Hfx[1]);
  const long long oz = cell_offset_fx(nz, cz, S.Hfx[2]);
  if (!(ox >= S.lofx[0] && ox < S.hifx[0] && oy >= S.lofx[1] && oy < S.hifx[1] &&
        oz >= S.lofx[2] && oz < S.hifx[2])) {
    // more than one cell edge away in one step: not a state a rebuild repairs
    if (ox < -S.Hfx[0] || ox >= 2 * S.Hfx[0] || oy < -S.Hfx[1] || oy >= 2 * S.Hfx[1] ||
        oz < -S.Hfx[2] || oz >= 2 * S.Hfx[2])
      set_status(ctl, PRX_ENONFINITE);
    atomicExch(&ctl->rebin_flag, 1);
  }
  B.vx[i] = vx;
  B.vy[i] = vy;
  B.vz[i] = vz;
  B.x[i] = nx;
  B.y[i] = ny;
  B.z[i] = nz;
  offn[i] = make_int4((int)(ox >> 3), (int)(oy >> 3), (int)(oz >> 3), oi.w);
}

__device__ __forceinline__ void step_epilogue(Ctl* ctl, int ph, unsigned long long step,
                                              cudaGraphConditionalHandle cond, int use_cond) {
  if (last_block(&ctl->done_step)) {
    ctl->done_step = 0u;
    ctl->phase = ph ^ 1;
    ctl->step = step;
    const int flag = atomicAdd(&ctl->rebin_flag, 0);
    if (use_cond) cudaGraphSetConditional(cond, flag ? 1u : 0u);
  }
}

// ---------------------------------------------------------------------------
// FP32 step kernel.  One block per tile of TY consecutive cell rows (cy0 ..
// cy0+TY-1 at one cz); threads = the tile's particles, which are contiguous
// in slot order (in passes of blockDim when a tile is longer).  All
// (TY+2) x 3 neighbour rows are staged in shared memory in one pass, each row
// extended by one periodic image cell at both ends, so that every
// particle's 3 x 3 x 3 cell neighbourhood is 9 contiguous ranges.  Staged
// per particle, in the tile frame:
//   P = FP32 position (prefilter only; its error is far below the margin),
//   Q = 2^-29 fixed-point position modulo 2^32 (periodic corrections folded
//       in): differences of two Q are exact displacements.
// Pairs passing r^2 < (r_c + 1e-3)^2 on P get their displacement from Q,
// rounded once to FP32, and the WCA force.
// ---------------------------------------------------------------------------
struct RowInfo {
  int base;        // first staged index of the row
  int padL;        // particles of the left image cell (cell nx-1)
  int rowcount;    // particles of the row
  int tot;         // padL + rowcount + padR
  int row_lo;      // first slot of the row
  int left_start;  // first slot of cell nx-1
  uint32_t qy, qz; // tile-frame fixed-point shifts of the row
  float fy, fz;    // tile-frame FP32 shifts of the row
  int pad0, pad1;
};
constexpr int TILE_ROWS_MAX = 18;  // (TY + 2) x 3 for TY <= 4

// 2^-29 fixed point to float by truncation to 2^-20 (one magic-number
// conversion): accurate to 1e-6, enough for the prefilter and cheaper than
// the correctly rounded conversion used for forces.
__device__ __forceinline__ float fx29_coarse(int d) {
  const uint32_t v = (uint32_t)((d >> 9) + 4194304);  // [0, 2^23) for |d| < 2^31
  return __fsub_rn(__uint_as_float(0x4B000000u | v), 12582912.0f) * 0x1.0p-20f;
}

constexpr int QMAX = 16;  // prefilter hits buffered per thread before the exact pass

template <bool FORCES_ONLY>
__global__ void __launch_bounds__(256)
    k_step_tiles(Sys S, cudaGraphConditionalHandle cond, int use_cond) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int CAP = S.tile_cap;
  float4* sP = reinterpret_cast<float4*>(smem);
  int4* sQ = reinterpret_cast<int4*>(smem + 16 * (size_t)CAP);
  RowInfo* ri = reinterpret_cast<RowInfo*>(smem + 32 * (size_t)CAP);
  uint32_t* sCS = reinterpret_cast<uint32_t*>(ri + TILE_ROWS_MAX);
  uint16_t* sHit = reinterpret_cast<uint16_t*>(sCS + TILE_ROWS_MAX * (S.nc[0] + 1));
  __shared__ int sTOT;

  Ctl* ctl = S.ctl;
  const int set = ctl->set;
  const int ph = ctl->phase;
  const unsigned long long step = ctl->step + 1ull;
  const SoA B = set ? S.s1 : S.s0;
  const int4* __restrict__ off = ph ? S.off1 : S.off0;
  int4* __restrict__ offn = ph ? S.off0 : S.off1;
  const int nx = S.nc[0], ny = S.nc[1], nz = S.nc[2];
  const int ty = blockIdx.x % S.tiles_y, cz = blockIdx.x / S.tiles_y;
  const int cy0 = ty * S.tile_y;
  const int TYb = min(S.tile_y, ny - cy0);
  const int RY = TYb + 2, R = 3 * RY;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const uint32_t rs = S.cell_start[(cz * ny + cy0) * nx];
  const uint32_t re = S.cell_start[(cz * ny + cy0 + TYb - 1) * nx + nx];

  // cell starts of the staged rows
  for (int k = threadIdx.x; k < R * (nx + 1); k += blockDim.x) {
    const int sr = k / (nx + 1), c = k - sr * (nx + 1);
    const int dzi = sr / RY, yi = sr - dzi * RY;
    const int qz = wrap_cell(cz - 1 + dzi, nz), qy = wrap_cell(cy0 - 1 + yi, ny);
    sCS[k] = S.cell_start[(qz * ny + qy) * nx + c];
  }
  __syncthreads();
  if (threadIdx.x < R) {
    const int sr = threadIdx.x;
    const int dzi = sr / RY, yi = sr - dzi * RY;
    const uint32_t* cs = sCS + sr * (nx + 1);
    const int qz = cz - 1 + dzi, qy = cy0 - 1 + yi;
    uint32_t cz_corr = 0u, cy_corr = 0u;
    if (qz < 0) cz_corr = (uint32_t)(-S.corr29[2]);
    else if (qz >= nz) cz_corr = (uint32_t)S.corr29[2];
    if (qy < 0) cy_corr = (uint32_t)(-S.corr29[1]);
    else if (qy >= ny) cy_corr = (uint32_t)S.corr29[1];
    RowInfo r;
    r.padL = (int)(cs[nx] - cs[nx - 1]);
    r.rowcount = (int)(cs[nx] - cs[0]);
    r.tot = r.padL + r.rowcount + (int)(cs[1] - cs[0]);
    r.row_lo = (int)cs[0];
    r.left_start = (int)cs[nx - 1];
    r.qy = (uint32_t)((yi - 1) * S.H29[1]) + cy_corr;
    r.qz = (uint32_t)((dzi - 1) * S.H29[2]) + cz_corr;
    r.fy = (float)(yi - 1) * S.hf[1];
    r.fz = (float)(dzi - 1) * S.hf[2];
    r.base = 0;
    r.pad0 = r.pad1 = 0;
    ri[sr] = r;
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
  uint16_t* myHit = sHit + threadIdx.x;  // column layout: hit q at myHit[q * blockDim]

  for (uint32_t base = rs; base < re; base += blockDim.x) {
    const uint32_t i = base + threadIdx.x;
    const bool act = i < re;
    const int4 oi = act ? off[i] : make_int4(0, 0, 0, 0);
    const int cx = oi.w & 511, cy = (oi.w >> 9) & 511;
    const int yrel = act ? cy - cy0 : 0;
    // own position in the tile frame (fixed point mod 2^32, and FP32)
    const uint32_t ox = (uint32_t)oi.x + (uint32_t)(cx * S.H29[0]);
    const uint32_t oy = (uint32_t)oi.y + (uint32_t)(yrel * S.H29[1]);
    const uint32_t oz = (uint32_t)oi.z;
    const float pix = __fmaf_rn((float)cx, S.hf[0], fx29_coarse(oi.x));
    const float piy = __fmaf_rn((float)yrel, S.hf[1], fx29_coarse(oi.y));
    const float piz = fx29_coarse(oi.z);
    double xi = 0.0, yi = 0.0, zi = 0.0, vx = 0.0, vy = 0.0, vz = 0.0;
    if (!FORCES_ONLY && act) {
      xi = B.x[i];
      yi = B.y[i];
      zi = B.z[i];
      vx = B.vx[i];
      vy = B.vy[i];
      vz = B.vz[i];
    }
    // the 9 windows (virtual cells cx-1 .. cx+1 of the 9 neighbour rows),
    // packed lo | hi << 16
    uint32_t win[9];
    int self = -1;
#pragma unroll
    for (int w = 0; w < 9; ++w) {
      const int sr = (w / 3) * RY + yrel + (w % 3);
      const uint32_t* cs = sCS + sr * (nx + 1);
      const RowInfo& r = ri[sr];
      const int lo = r.base + (cx == 0 ? 0 : r.padL + (int)cs[cx - 1] - r.row_lo);
      const int hi = r.base + (cx + 2 > nx ? r.tot : r.padL + (int)cs[cx + 2] - r.row_lo);
      win[w] = (uint32_t)lo | ((uint32_t)hi << 16);
      if (w == 4) self = r.base + r.padL + (int)i - r.row_lo;
    }
    float fx = 0.f, fy = 0.f, fz = 0.f, e = 0.f;

    for (int c0 = 0; c0 < TOT; c0 += CAP) {
      const int cn = min(CAP, TOT - c0);
      __syncthreads();  // previous users of the staging buffer are done
      // one warp per staged row, lanes over the row's particles
      for (int sr = warp; sr < R; sr += nwarps) {
        const RowInfo r = ri[sr];
        const int k0 = max(r.base, c0), k1 = min(r.base + r.tot, c0 + cn);
        for (int ent = k0 + lane; ent < k1; ent += 32) {
          const int kr = ent - r.base;
          int slot, vcx;
          uint32_t corx = 0u;
          if (kr < r.padL) {
            slot = r.left_start + kr;
            vcx = -1;
            corx = (uint32_t)(-S.corr29[0]);
          } else if (kr < r.padL + r.rowcount) {
            slot = r.row_lo + (kr - r.padL);
            vcx = -2;
          } else {
            slot = r.row_lo + (kr - r.padL - r.rowcount);
            vcx = nx;
            corx = (uint32_t)S.corr29[0];
          }
          const int4 q = off[slot];
          if (vcx == -2) vcx = q.w & 511;
          const int k = ent - c0;
          sQ[k] = make_int4((int)((uint32_t)q.x + (uint32_t)(vcx * S.H29[0]) + corx),
                            (int)((uint32_t)q.y + r.qy), (int)((uint32_t)q.z + r.qz), 0);
          sP[k] = make_float4(__fmaf_rn((float)vcx, S.hf[0], fx29_coarse(q.x)),
                              fx29_coarse(q.y) + r.fy, fx29_coarse(q.z) + r.fz, 0.f);
        }
      }
      __syncthreads();
      if (act) {
        const int sk = self - c0;
        int nh = 0;
        // exact pass over the buffered prefilter hits: displacement from the
        // fixed-point positions, rounded once to FP32
        auto flush = [&]() {
          for (int q = 0; q < nh; ++q) {
            const int4 qq = sQ[myHit[q * blockDim.x]];
            const float dxe = fx29_to_float((int)((uint32_t)qq.x - ox));
            const float dye = fx29_to_float((int)((uint32_t)qq.y - oy));
            const float dze = fx29_to_float((int)((uint32_t)qq.z - oz));
            const float r2 = fmaf(dze, dze, fmaf(dye, dye, dxe * dxe));
            if (r2 < S.rc2f) wca32(S, dxe, dye, dze, r2, fx, fy, fz, e);
          }
          nh = 0;
        };
#pragma unroll
        for (int w = 0; w < 9; ++w) {
          const int lo = max((int)(win[w] & 0xFFFFu), c0) - c0;
          const int hi = min((int)(win[w] >> 16), c0 + cn) - c0;
          for (int k = lo; k < hi; ++k) {
            const float4 p = sP[k];
            const float ddx = p.x - pix, ddy = p.y - piy, ddz = p.z - piz;
            const float r2p = fmaf(ddz, ddz, fmaf(ddy, ddy, ddx * ddx));
            if (r2p < S.rc2pre && k != sk) {
              myHit[nh * blockDim.x] = (uint16_t)k;
              if (++nh == QMAX) flush();
            }
          }
        }
        flush();
      }
    }

    if (act) {
      // bonds, with the exact fixed-point displacement to the partner
      const uint32_t nb = B.nadj[i];
      bool ok = true;
      for (uint32_t b = 0; b < nb; ++b) {
        const uint32_t ent = B.adj[(size_t)i * S.cap + b];
        const int4 q = off[ent & SLOT_MASK];
        const int ex = exact_d29(q.x, oi.x, q.w & 511, cx, nx, S.H29[0], S.corr29[0]);
        const int ey = exact_d29(q.y, oi.y, (q.w >> 9) & 511, cy, ny, S.H29[1], S.corr29[1]);
        const int ez = exact_d29(q.z, oi.z, (q.w >> 18) & 511, (oi.w >> 18) & 511, nz, S.H29[2],
                                 S.corr29[2]);
        ok = bond32(S, ent >> 31, fx29_to_float(ex), fx29_to_float(ey), fx29_to_float(ez), fx,
                    fy, fz, e) && ok;
      }
      if (!ok) set_status(ctl, PRX_EOVERSTRETCH);
      if constexpr (FORCES_ONLY) {
        S.fout[3 * (size_t)i + 0] = (double)fx;
        S.fout[3 * (size_t)i + 1] = (double)fy;
        S.fout[3 * (size_t)i + 2] = (double)fz;
        S.eout[i] = (double)e;
      } else {
        integrate32(S, ctl, B, offn, i, oi, cx, cy, (oi.w >> 18) & 511, step, fx, fy, fz, xi, yi,
                    zi, vx, vy, vz);
      }
    }
  }
  if constexpr (!FORCES_ONLY) step_epilogue(ctl, ph, step, cond, use_cond);
}

// ---------------------------------------------------------------------------
// FP64 force mode (small systems): conservative forces per slot from the
// absolute positions, written to fout / eout; the integration runs as a
// second kernel so that no thread reads a position another thread updates.
// Arithmetic is written in the order of the plain definitions.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(STEP_THREADS) k_forces64(Sys S) {
  Ctl* ctl = S.ctl;
  const SoA B = ctl->set ? S.s1 : S.s0;
  const int4* __restrict__ off = ctl->phase ? S.off1 : S.off0;
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= S.n) return;
  int cx, cy, cz;
  unpack_cell((uint32_t)off[i].w, cx, cy, cz);
  const double xi = B.x[i], yi = B.y[i], zi = B.z[i];
  double fx = 0.0, fy = 0.0, fz = 0.0, e = 0.0;
  for (int dz = -1; dz <= 1; ++dz) {
    const int qz = wrap_cell(cz + dz, S.nc[2]);
    for (int dy = -1; dy <= 1; ++dy) {
      const int qy = wrap_cell(cy + dy, S.nc[1]);
      const int rowbase = (qz * S.nc[1] + qy) * S.nc[0];
      for (int dx = -1; dx <= 1; ++dx) {
        const int q = rowbase + wrap_cell(cx + dx, S.nc[0]);
        const uint32_t s0 = S.cell_start[q], s1 = S.cell_start[q + 1];
        for (uint32_t j = s0; j < s1; ++j) {
          if (j == i) continue;
          const double ddx = min_image(__dsub_rn(B.x[j], xi), S.L[0], S.halfL[0]);
          const double ddy = min_image(__dsub_rn(B.y[j], yi), S.L[1], S.halfL[1]);
          const double ddz = min_image(__dsub_rn(B.z[j], zi), S.L[2], S.halfL[2]);
          const double r2 =
              __dadd_rn(__dadd_rn(__dmul_rn(ddx, ddx), __dmul_rn(ddy, ddy)), __dmul_rn(ddz, ddz));
          if (r2 < S.rc2) wca64(S, ddx, ddy, ddz, r2, fx, fy, fz, e);
        }
      }
    }
  }
  bool ok = true;
  const uint32_t nb = B.nadj[i];
  for (uint32_t b = 0; b < nb; ++b) {
    const uint32_t ent = B.adj[(size_t)i * S.cap + b];
    const uint32_t j = ent & SLOT_MASK;
    const double ddx = min_image(__dsub_rn(B.x[j], xi), S.L[0], S.halfL[0]);
    const double ddy = min_image(__dsub_rn(B.y[j], yi), S.L[1], S.halfL[1]);
    const double ddz = min_image(__dsub_rn(B.z[j], zi), S.L[2], S.halfL[2]);
    ok = bond64(S, ent >> 31, ddx, ddy, ddz, fx, fy, fz, e) && ok;
  }
  if (!ok) set_status(ctl, PRX_EOVERSTRETCH);
  S.fout[3 * (size_t)i + 0] = fx;
  S.fout[3 * (size_t)i + 1] = fy;
  S.fout[3 * (size_t)i + 2] = fz;
  S.eout[i] = e;
}

// FP64 integration in the oracle's order of operations:
//   F = F_c - gamma m v + R,  v' = v + (dt/m) F,  x' = x + dt v'.
__global__ void __launch_bounds__(STEP_THREADS)
    k_integrate64(Sys S, cudaGraphConditionalHandle cond, int use_cond) {
  Ctl* ctl = S.ctl;
  const int set = ctl->set;
  const int ph = ctl->phase;
  const unsigned long long step = ctl->step + 1ull;
  const SoA B = set ? S.s1 : S.s0;
  const int4* __restrict__ off = ph ? S.off1 : S.off0;
  int4* __restrict__ offn = ph ? S.off0 : S.off1;
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < S.n) {
    const int4 oi = off[i];
    int cc[3];
    unpack_cell((uint32_t)oi.w, cc[0], cc[1], cc[2]);
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
    long long o[3];
    bool inside = true, jump = false;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const double v = vs[d][i];
      const double F = __dadd_rn(__dsub_rn(S.fout[3 * (size_t)i + d], __dmul_rn(S.gm, v)), R[d]);
      const double vn = __dadd_rn(v, __dmul_rn(S.b_kick, F));
      const double xn = __dadd_rn(xs[d][i], __dmul_rn(S.dt, vn));
      if (!isfinite(vn) || !isfinite(xn)) set_status(ctl, PRX_ENONFINITE);
      vs[d][i] = vn;
      xs[d][i] = xn;
      o[d] = cell_offset_fx(xn, cc[d], S.Hfx[d]);
      inside = inside && o[d] >= S.lofx[d] && o[d] < S.hifx[d];
      jump = jump || o[d] < -S.Hfx[d] || o[d] >= 2 * S.Hfx[d];
    }
    if (!inside) {
      if (jump) set_status(ctl, PRX_ENONFINITE);
      atomicExch(&ctl->rebin_flag, 1);
    }
    offn[i] = make_int4((int)(o[0] >> 3), (int)(o[1] >> 3), (int)(o[2] >> 3), oi.w);
  }
  step_epilogue(ctl, ph, step, cond, use_cond);
}

// ---------------------------------------------------------------------------
// Cell-list rebuild.  Keys, counting sort with a stable (ascending old slot)
// order inside each cell, permutation of every per-particle array into the
// other SoA set, and remapping of the adjacency to the new slots.
// ---------------------------------------------------------------------------

// Incremental keys: a particle moved at most one cell since the last
// rebuild, so its new cell is its old one shifted by -1, 0 or +1 per axis.
// Coordinates that wrap through the box are shifted by one box edge.
__global__ void k_rebin_keys(Sys S) {
  Ctl* ctl = S.ctl;
  const int set = ctl->set;
  const SoA B = set ? S.s1 : S.s0;
  const int4* off = ctl->phase ? S.off1 : S.off0;
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= S.n) return;
  const int4 o = off[i];
  int c[3];
  unpack_cell((uint32_t)o.w, c[0], c[1], c[2]);
  double* xs[3] = {B.x, B.y, B.z};
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const long long od = cell_offset_fx(xs[d][i], c[d], S.Hfx[d]);
    int s = od < 0 ? -1 : (od >= S.Hfx[d] ? 1 : 0);
    int q = c[d] + s;
    if (q < 0) {
      q += S.nc[d];
      xs[d][i] = __dadd_rn(xs[d][i], S.L[d]);
    } else if (q >= S.nc[d]) {
      q -= S.nc[d];
      xs[d][i] = __dsub_rn(xs[d][i], S.L[d]);
    }
    c[d] = q;
  }
  const uint32_t k = (uint32_t)((c[2] * S.nc[1] + c[1]) * S.nc[0] + c[0]);
  S.key[i] = k;
  atomicAdd(&S.count[k], 1u);
}

// Full keys from absolute positions (creation, grid change): wraps x into
// [0, L) and takes floor(x / h).
__global__ void k_bin_full_keys(Sys S) {
  Ctl* ctl = S.ctl;
  const SoA B = ctl->set ? S.s1 : S.s0;
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= S.n) return;
  double* xs[3] = {B.x, B.y, B.z};
  int c[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    double v = xs[d][i];
    if (v >= S.L[d]) v = __dsub_rn(v, S.L[d]);
    if (v < 0.0) v = __dadd_rn(v, S.L[d]);
    xs[d][i] = v;
    int q = (int)floor(__dmul_rn(v, S.inv_h[d]));
    q = q < 0 ? 0 : (q >= S.nc[d] ? S.nc[d] - 1 : q);
    c[d] = q;
  }
  const uint32_t k = (uint32_t)((c[2] * S.nc[1] + c[1]) * S.nc[0] + c[0]);
  S.key[i] = k;
  atomicAdd(&S.count[k], 1u);
}

// Restore: keys were uploaded (a checkpoint's cells); only count them.
__global__ void k_count_keys(Sys S) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= S.n) return;
  atomicAdd(&S.count[S.key[i]], 1u);
}

// Exclusive scan of count[0..ncell) into cell_start[0..ncell], three passes.
__global__ void k_scan_tiles(const uint32_t* __restrict__ in, uint32_t n, uint32_t* __restrict__ tsum) {
  __shared__ uint32_t red[256];
  const uint32_t base = blockIdx.x * SCAN_TILE;
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
  if (threadIdx.x == 0) tsum[blockIdx.x] = red[0];
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
__global__ void k_scan_top(uint32_t* tsum, uint32_t ntiles) {
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

__global__ void k_scan_down(const uint32_t* __restrict__ in, uint32_t n,
                            const uint32_t* __restrict__ tsum, uint32_t* __restrict__ out) {
  const uint32_t base = blockIdx.x * SCAN_TILE + threadIdx.x * (SCAN_TILE / 256);
  uint32_t loc[SCAN_TILE / 256];
  uint32_t s = 0;
#pragma unroll
  for (int k = 0; k < SCAN_TILE / 256; ++k) {
    loc[k] = (base + k < n) ? in[base + k] : 0u;
    s += loc[k];
  }
  uint32_t total;
  uint32_t run = tsum[blockIdx.x] + block_exclusive_scan_256(s, total);
  if (blockIdx.x == 0 && threadIdx.x == 0) out[0] = 0u;
#pragma unroll
  for (int k = 0; k < SCAN_TILE / 256; ++k) {
    run += loc[k];
    if (base + k < n) out[base + k + 1] = run;
  }
}

__global__ void k_rebin_scatter(Sys S) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= S.n) return;
  const uint32_t k = S.key[i];
  const uint32_t pos = atomicAdd(&S.fill[k], 1u);
  S.tmp[S.cell_start[k] + pos] = i;
}

// Sorts each cell's members by old slot: the order inside a cell then does
// not depend on the order in which the scatter's atomics completed.
__global__ void k_rebin_cellsort(Sys S) {
  const uint32_t c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= (uint32_t)S.ncell) return;
  const uint32_t s0 = S.cell_start[c], s1 = S.cell_start[c + 1];
  for (uint32_t a = s0 + 1; a < s1; ++a) {
    const uint32_t v = S.tmp[a];
    uint32_t b = a;
    while (b > s0 && S.tmp[b - 1] > v) {
      S.tmp[b] = S.tmp[b - 1];
      --b;
    }
    S.tmp[b] = v;
  }
}

// New slot s takes old slot tmp[s]: copies every per-particle array into the
// other set and recomputes the FP32 offset against the new cell.
__global__ void k_rebin_permute(Sys S) {
  Ctl* ctl = S.ctl;
  const int set = ctl->set;
  const SoA A = set ? S.s1 : S.s0;
  const SoA B = set ? S.s0 : S.s1;
  int4* off = ctl->phase ? S.off1 : S.off0;
  const uint32_t s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= S.n) return;
  const uint32_t o = S.tmp[s];
  const uint32_t k = S.key[o];
  const int cx = (int)(k % (uint32_t)S.nc[0]);
  const int cy = (int)((k / (uint32_t)S.nc[0]) % (uint32_t)S.nc[1]);
  const int cz = (int)(k / ((uint32_t)S.nc[0] * (uint32_t)S.nc[1]));
  const double x = A.x[o], y = A.y[o], z = A.z[o];
  B.x[s] = x;
  B.y[s] = y;
  B.z[s] = z;
  B.vx[s] = A.vx[o];
  B.vy[s] = A.vy[o];
  B.vz[s] = A.vz[o];
  const uint32_t pid = A.id[o];
  B.id[s] = pid;
  B.type[s] = A.type[o];
  B.state[s] = A.state[o];
  const uint32_t nb = A.nadj[o];
  B.nadj[s] = (uint8_t)nb;
  for (uint32_t b = 0; b < nb; ++b) B.adj[(size_t)s * S.cap + b] = A.adj[(size_t)o * S.cap + b];
  S.new_of_old[o] = s;
  S.slot_of_id[pid] = s;
  const uint32_t w = pack_cell(cx, cy, cz);
  off[s] = make_int4((int)(cell_offset_fx(x, cx, S.Hfx[0]) >> 3), (int)(cell_offset_fx(y, cy, S.Hfx[1]) >> 3),
                     (int)(cell_offset_fx(z, cz, S.Hfx[2]) >> 3), (int)w);
}

__global__ void k_rebin_remap(Sys S) {
  Ctl* ctl = S.ctl;
  const int set = ctl->set;
  const SoA B = set ? S.s0 : S.s1;  // the set just written
  const uint32_t s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s < S.n) {
    const uint32_t nb = B.nadj[s];
    for (uint32_t b = 0; b < nb; ++b) {
      const uint32_t e = B.adj[(size_t)s * S.cap + b];
      B.adj[(size_t)s * S.cap + b] = S.new_of_old[e & SLOT_MASK] | (e & ~SLOT_MASK);
    }
  }
  if (last_block(&ctl->done_rebin)) {
    ctl->done_rebin = 0u;
    ctl->set = set ^ 1;
    ctl->rebin_flag = 0;
    ctl->rebins += 1ull;
  }
}

inline unsigned blocks_for(uint64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

void launch_step(const Sys& S, cudaStream_t st, int fp64, int forces_only,
                 cudaGraphConditionalHandle h, int use_cond) {
  if (fp64) {
    const unsigned g = blocks_for(S.n, STEP_THREADS) > 0 ? blocks_for(S.n, STEP_THREADS) : 1;
    k_forces64<<<g, STEP_THREADS, 0, st>>>(S);
    if (!forces_only) k_integrate64<<<g, STEP_THREADS, 0, st>>>(S, h, use_cond);
  } else {
    const unsigned tiles = (unsigned)(S.tiles_y * S.nc[2]);
    const size_t sm = step_tile_smem(S);
    if (forces_only) k_step_tiles<true><<<tiles, S.tile_threads, sm, st>>>(S, h, use_cond);
    else k_step_tiles<false><<<tiles, S.tile_threads, sm, st>>>(S, h, use_cond);
  }
}

size_t step_tile_smem(const Sys& S) {
  return 32 * (size_t)S.tile_cap + sizeof(RowInfo) * TILE_ROWS_MAX +
         4 * (size_t)TILE_ROWS_MAX * (S.nc[0] + 1) + 2 * (size_t)QMAX * S.tile_threads;
}

int configure_step_kernels(size_t smem_bytes) {
  if (cudaFuncSetAttribute(k_step_tiles<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem_bytes) != cudaSuccess)
    return -1;
  if (cudaFuncSetAttribute(k_step_tiles<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem_bytes) != cudaSuccess)
    return -1;
  return 0;
}

int step_kernel_count(int fp64) { return fp64 ? 2 : 1; }

int rebin_kernel_count() { return 8; }

// Whole rebuild: keys (mode 0 incremental, 1 full from positions, 2 given),
// scan, scatter, per-cell sort, permutation, adjacency remap.  `hook`
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
  const char* kn = mode == 0 ? "rebin_keys" : (mode == 1 ? "bin_full_keys" : "count_keys");
  H(kn, 0);
  if (mode == 0) k_rebin_keys<<<gp, 256, 0, st>>>(S);
  else if (mode == 1) k_bin_full_keys<<<gp, 256, 0, st>>>(S);
  else k_count_keys<<<gp, 256, 0, st>>>(S);
  H(kn, 1);
  H("scan_tiles", 0);
  k_scan_tiles<<<tiles, 256, 0, st>>>(S.count, S.ncell, S.blk_off);
  H("scan_tiles", 1);
  H("scan_top", 0);
  k_scan_top<<<1, 256, 0, st>>>(S.blk_off, tiles);
  H("scan_top", 1);
  H("scan_down", 0);
  k_scan_down<<<tiles, 256, 0, st>>>(S.count, S.ncell, S.blk_off, S.cell_start);
  H("scan_down", 1);
  H("rebin_scatter", 0);
  k_rebin_scatter<<<gp, 256, 0, st>>>(S);
  H("rebin_scatter", 1);
  H("rebin_cellsort", 0);
  k_rebin_cellsort<<<gc, 256, 0, st>>>(S);
  H("rebin_cellsort", 1);
  H("rebin_permute", 0);
  k_rebin_permute<<<gp, 256, 0, st>>>(S);
  H("rebin_permute", 1);
  H("rebin_remap", 0);
  k_rebin_remap<<<gp, 256, 0, st>>>(S);
  H("rebin_remap", 1);
}

}  // namespace prx
