// G7 on the tensor cores: the point-coupling part of the FP64 refinement residual,
//   r[(al,i),be] -= sum_{al' != al} W_i[al][al'] X[(al',i),be]     (every mesh point i)
// formed exactly enough for FP64 refinement from FP16 tensor-core products by
// error-free splitting into integer slices (Ozaki, Ogita, Oishi, Rump 2012; the
// variant for FP16 tensor cores of Mukunoki et al. 2020):
//
//   * every row of W_i (al fixed, the diagonal al' = al excluded: it is applied in
//     FP64 by the kinetic kernel) is scaled by 2^-e with e such that every |Re|,
//     |Im| of the row is below 1, and cut into S = 9 signed 6-bit digits:
//     w 2^-e = sum_s d_s 2^-6(s+1), |d_s| <= 63 (54 bits: bit fields of
//     floor(|w| 2^(54-e)), the sign of w on every digit); the same for every column
//     of X_i (be fixed) with its own exponent f;
//   * a digit product d_p e_q is an integer below 2^12, exact in an FP16 MMA with
//     FP32 accumulation, and so is a sum of them while it stays below 2^24: with K
//     terms per real product and two real products per complex part, up to
//     floor(2^24 / (2 K 63^2)) digit pairs (8 at K = 256) share one FP32 tensor-
//     memory accumulator exactly;
//   * pairs with p + q <= 8 are formed (the rest lies below 2^-54 of the row/column
//     scales), grouped by p + q, and every group's exact FP32 sums are drained from
//     tensor memory into FP64 registers with the weight 2^-6(p+q+2); the result is
//     scaled by 2^(e + f) and subtracted from r in FP64.
//
// Per 128 x 64 output tile of one mesh point: 45 digit pairs x 4 real products
// (Re = Wr Xr - Wi Xi, Im = Wr Xi + Wi Xr, the minus through the negate-A bit)
// of K = round_up(nch, 16) on tcgen05 (kind::f16, M = 128, N = 64), operands
// staged by TMA through a 12-stage mbarrier pipeline, four double-buffered
// accumulator sets of 2 x 64 TMEM columns so that a group's drain overlaps the
// next group's MMAs.
// Roles (320 threads, one CTA per SM, persistent over tiles): warp 0 TMA producer,
// warp 1 TMEM allocator + MMA issuer, warps 2..9 epilogue (warp w reads TMEM lane
// quadrant w % 4, column half (w - 2) / 4).  Every wait is bounded; on expiry the
// kernel raises an error word, lets its copies / MMAs drain, frees TMEM, returns.
#include <cuda.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <cmath>

#include "cplx.cuh"
#include "rmat_internal.h"
#include "tc_common.cuh"

namespace {

constexpr int OZ_S = 9;           // digits per operand value
constexpr int OZ_D = 8;           // digit pairs kept: p + q <= OZ_D
constexpr int OZ_BM = 128, OZ_BN = 64, OZ_BK = 16;
constexpr int OZ_STAGES = 12;
constexpr int OZ_THREADS = 320;
constexpr uint32_t OZ_A_BYTES = OZ_BM * 32, OZ_B_BYTES = OZ_BN * 32;
constexpr uint32_t OZ_STAGE = 2 * OZ_A_BYTES + 2 * OZ_B_BYTES;  // re + im planes of A and B
constexpr int OZ_NBUF = 4;        // accumulator sets (2 x 64 columns each)
constexpr size_t OZ_SMEM = (size_t)OZ_STAGES * OZ_STAGE + 1024 + 512;
constexpr int OZ_MAXG = 48, OZ_MAXP = 48;

struct OzPlan {
  int ngroups;
  unsigned char first[OZ_MAXG], count[OZ_MAXG], d[OZ_MAXG];  // pairs [first, first+count)
  unsigned char p[OZ_MAXP], q[OZ_MAXP];
};

struct OzMaps {
  CUtensorMap a;  // A digit planes: rows ((s*2 + part)*a_pts + pt)*a_rows + row
  CUtensorMap b;  // X digit planes: rows ((s*2 + part)*npts + pt)*nrhs + be
};

// Which product a launch forms.  Coupling: points = mesh points i, A = W_i (rows al,
// K = al', one per point, complex), output row (al, i).  Kinetic: points = channels
// al, A = the real kinetic matrix (rows i, K = j, shared by every channel), output
// row (al, i).
struct OzGeom {
  int npts;          // points (independent products)
  int mrows;         // A rows per point (nch or nlag)
  int a_rows;        // A plane rows per point (mrows, or padded to the tile)
  int a_pts;         // A planes per digit and part: npts, or 1 (shared by every point)
  int a_real;        // A is real: two MMAs per K-step, its imaginary planes never read
  int pt_major;      // output row pt * nlag + row (kinetic) instead of row * nlag + pt
  int ew_shared;     // A row exponents per row only (not per point)
  int nlag;
};

// The nine signed 6-bit digits of v (|v| < 1): the base-64 expansion of |v| cut after
// 54 bits, every digit with the sign of v (the same digits as repeated multiply-by-64
// and truncation), taken as bit fields of the integer floor(|v| 2^54) so that only two
// FP64 operations are spent per value (FP64 is ~2 FMA per clock per SM on this part).
// sh = 54 - e, sc = 2^sh: |w| 2^sh < 2^54 for the scaled value w 2^-e (sc is only
// formed when 2^sh is a finite double; rows of values below 2^-970 scale per value).
__device__ __forceinline__ double oz_scale(int e) { return e >= -960 ? ldexp(1.0, 54 - e) : 0.0; }
__device__ __forceinline__ void oz_digits(double w, double sc, int e, __half* d) {
  const double a = sc != 0.0 ? fabs(w) * sc : ldexp(fabs(w), 54 - e);
  const unsigned long long u = (unsigned long long)a;
  const bool neg = w < 0.0;
#pragma unroll
  for (int s = 0; s < OZ_S; ++s) {
    const int q = (int)((u >> (6 * (OZ_S - 1 - s))) & 63ull);
    d[s] = __int2half_rn(neg ? -q : q);
  }
}

// One warp per row (i, al) of W: exponent over al' != al, then the digit planes.
__global__ void __launch_bounds__(256)
oz_split_w_kernel(const double2* __restrict__ W, int nlag, int nch, int kpad,
                  __half* __restrict__ Wsl, int* __restrict__ ew) {
  const int row = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (row >= nlag * nch) return;
  const int i = row / nch, al = row - i * nch;
  const double2* w = W + (size_t)row * nch;
  double m = 0.0;
  for (int k = lane; k < nch; k += 32)
    if (k != al) m = fmax(m, fmax(fabs(w[k].x), fabs(w[k].y)));
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  const int e = m > 0.0 ? ilogb(m) + 1 : 0;  // |v| = |w| 2^-e < 1
  if (lane == 0) ew[row] = e;
  const size_t plane = (size_t)nlag * nch * kpad;
  const double sc = oz_scale(e);
  for (int k = lane; k < kpad; k += 32) {
    double vr = 0.0, vi = 0.0;
    if (k < nch && k != al) {
      vr = w[k].x;
      vi = w[k].y;
    }
    __half* o = Wsl + (size_t)row * kpad + k;
    __half dr[OZ_S], di[OZ_S];
    oz_digits(vr, sc, e, dr);
    oz_digits(vi, sc, e, di);
#pragma unroll
    for (int s = 0; s < OZ_S; ++s) {
      o[(size_t)(2 * s) * plane] = dr[s];
      o[(size_t)(2 * s + 1) * plane] = di[s];
    }
  }
}

// The real kinetic matrix K (nlag x nlag, FP64, row-major) -> digit planes
// [s][part 0][row][kpad] with rows padded to a_rows (zeros); one exponent per row
// over the whole row.  One warp per row.
__global__ void __launch_bounds__(256)
oz_split_k_kernel(const double* __restrict__ K, int nlag, int a_rows, int kpad,
                  __half* __restrict__ Ksl, int* __restrict__ ek) {
  const int row = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (row >= a_rows) return;
  const double* kr = K + (size_t)row * nlag;
  double m = 0.0;
  if (row < nlag)
    for (int k = lane; k < nlag; k += 32) m = fmax(m, fabs(kr[k]));
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  const int e = m > 0.0 ? ilogb(m) + 1 : 0;
  if (lane == 0) ek[row] = e;
  const size_t plane = (size_t)a_rows * kpad;
  const double sc = oz_scale(e);
  for (int k = lane; k < kpad; k += 32) {
    const double v = (row < nlag && k < nlag) ? kr[k] : 0.0;
    __half d[OZ_S];
    oz_digits(v, sc, e, d);
#pragma unroll
    for (int s = 0; s < OZ_S; ++s) Ksl[(size_t)(2 * s) * plane + (size_t)row * kpad + k] = d[s];
  }
}

// X (FP64, row-major [(al',j)][be]) -> digit planes [s][part][pt][be][k] with one
// exponent per (pt, be): max over k first, then 32 x 32 blocks transposed through
// shared memory so the planes are written along k.  The element of point pt and K
// index k is row pt * pt_stride + k * k_stride of X: the coupling product takes
// pt = mesh point i, k = channel al' (strides 1, nlag), the kinetic product pt =
// channel al, k = mesh point j (strides nlag, 1).
constexpr int OZ_XT = 32;
__global__ void __launch_bounds__(256)
oz_split_x_kernel(const double2* __restrict__ X, int nrhs, int npts, int kext, int pt_stride,
                  int k_stride, int kpad, __half* __restrict__ Xsl, int* __restrict__ fx,
                  const int* __restrict__ skip) {
  if (skip && *skip) return;
  __shared__ double red[8][OZ_XT];
  __shared__ int s_f[OZ_XT];
  __shared__ double s_sc[OZ_XT];
  __shared__ __align__(16) __half dig[OZ_S][2][OZ_XT][OZ_XT + 8];
  const int i = blockIdx.y, b0 = blockIdx.x * OZ_XT;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int be = b0 + lane;
  double m = 0.0;
  if (be < nrhs)
    for (int a = warp; a < kext; a += 8) {
      const double2 x = X[((size_t)i * pt_stride + (size_t)a * k_stride) * nrhs + be];
      m = fmax(m, fmax(fabs(x.x), fabs(x.y)));
    }
  red[warp][lane] = m;
  __syncthreads();
  if (warp == 0) {
    for (int w = 1; w < 8; ++w) m = fmax(m, red[w][lane]);
    const int f = m > 0.0 ? ilogb(m) + 1 : 0;
    s_f[lane] = f;
    s_sc[lane] = oz_scale(f);
    if (be < nrhs) fx[(size_t)i * nrhs + be] = f;
  }
  __syncthreads();
  const size_t plane = (size_t)npts * nrhs * kpad;
  for (int c0 = 0; c0 < kpad; c0 += OZ_XT) {
    for (int a = warp; a < OZ_XT; a += 8) {
      const int ga = c0 + a;
      double vr = 0.0, vi = 0.0;
      if (ga < kext && be < nrhs) {
        const double2 x = X[((size_t)i * pt_stride + (size_t)ga * k_stride) * nrhs + be];
        vr = x.x;
        vi = x.y;
      }
      __half dr[OZ_S], di[OZ_S];
      oz_digits(vr, s_sc[lane], s_f[lane], dr);
      oz_digits(vi, s_sc[lane], s_f[lane], di);
#pragma unroll
      for (int s = 0; s < OZ_S; ++s) {
        dig[s][0][lane][a] = dr[s];
        dig[s][1][lane][a] = di[s];
      }
    }
    __syncthreads();
    // rows (s, part, be) of 32 digits = 4 x 16 bytes along al'
    const int cw = min(OZ_XT, kpad - c0);  // multiple of 16
    for (int e = threadIdx.x; e < OZ_S * 2 * OZ_XT * 4; e += 256) {
      const int u = e & 3, rb = (e >> 2) % OZ_XT, sp = (e >> 2) / OZ_XT;
      const int s = sp >> 1, part = sp & 1;
      if (b0 + rb >= nrhs || 8 * u >= cw) continue;
      const uint4 v = *reinterpret_cast<const uint4*>(&dig[s][part][rb][8 * u]);
      __half* o = Xsl + (size_t)(2 * s + part) * plane + ((size_t)i * nrhs + b0 + rb) * kpad + c0 + 8 * u;
      *reinterpret_cast<uint4*>(o) = v;
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(OZ_THREADS, 1)
oz_product_kernel(const __grid_constant__ OzMaps maps, const __grid_constant__ OzPlan plan,
                  const OzGeom geo, double2* __restrict__ R, int nrhs, int kpad,
                  const int* __restrict__ ew, const int* __restrict__ fx,
                  const int* __restrict__ skip, int* __restrict__ err) {
  if (skip && *skip) return;  // before any barrier or TMEM allocation
  extern __shared__ unsigned char smem_raw[];
  unsigned char* stages =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  uint64_t* bars = reinterpret_cast<uint64_t*>(stages + OZ_STAGES * OZ_STAGE);
  // bars[0..S) full, [S..2S) empty, [2S + 2b] tmem_full of set b, [2S + 2b + 1] tmem_empty
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * OZ_STAGES + 2 * OZ_NBUF);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int mt = (geo.mrows + OZ_BM - 1) / OZ_BM, nt = (nrhs + OZ_BN - 1) / OZ_BN;
  const int ntiles = geo.npts * mt * nt;
  const int ksteps = kpad / OZ_BK;
  const int G = plan.ngroups;

  if (threadIdx.x == 0) {
    for (int s = 0; s < OZ_STAGES; ++s) {
      mbar_init(smem_u32(&bars[s]), 1);
      mbar_init(smem_u32(&bars[OZ_STAGES + s]), 1);
    }
    for (int b = 0; b < OZ_NBUF; ++b) {
      mbar_init(smem_u32(&bars[2 * OZ_STAGES + 2 * b]), 1);
      mbar_init(smem_u32(&bars[2 * OZ_STAGES + 2 * b + 1]), 8);
    }
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    // ------------------------------ TMA producer ------------------------------
    if (lane == 0) {
      uint32_t it = 0;
      bool ok = true;
      for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
        const int i = tile / (mt * nt), rem = tile % (mt * nt);
        const int m0 = (rem % mt) * OZ_BM, n0 = (rem / mt) * OZ_BN;
        for (int g = 0; g < G && ok; ++g)
          for (int pr = plan.first[g]; pr < plan.first[g] + plan.count[g] && ok; ++pr) {
            const int p = plan.p[pr], q = plan.q[pr];
            const int ia = geo.a_pts == 1 ? 0 : i;
            const int ar = ((2 * p) * geo.a_pts + ia) * geo.a_rows + m0;
            const int ai = ((2 * p + 1) * geo.a_pts + ia) * geo.a_rows + m0;
            const int br = ((2 * q) * geo.npts + i) * nrhs + n0;
            const int bi = ((2 * q + 1) * geo.npts + i) * nrhs + n0;
            for (int ks = 0; ks < ksteps; ++ks, ++it) {
              const uint32_t s = it % OZ_STAGES, ph = (it / OZ_STAGES) & 1;
              if (!mbar_wait(smem_u32(&bars[OZ_STAGES + s]), ph ^ 1, abort_flag)) { ok = false; break; }
              const uint32_t full = smem_u32(&bars[s]);
              mbar_expect_tx(full, geo.a_real ? OZ_STAGE - OZ_A_BYTES : OZ_STAGE);
              const uint32_t st = smem_u32(stages + s * OZ_STAGE);
              const int x = ks * OZ_BK;
              tma_load_2d(st, &maps.a, x, ar, full);
              if (!geo.a_real) tma_load_2d(st + OZ_A_BYTES, &maps.a, x, ai, full);
              tma_load_2d(st + 2 * OZ_A_BYTES, &maps.b, x, br, full);
              tma_load_2d(st + 2 * OZ_A_BYTES + OZ_B_BYTES, &maps.b, x, bi, full);
            }
          }
      }
      if (!ok) {
        *abort_flag = 1;
        atomicExch(err, 2);
      }
      for (uint32_t k = (it > OZ_STAGES ? it - OZ_STAGES : 0); k < it; ++k) {
        const unsigned long long t0 = gtimer();
        while (!mbar_try(smem_u32(&bars[k % OZ_STAGES]), (k / OZ_STAGES) & 1))
          if (gtimer() - t0 > RMAT_TC_WAIT_NS) break;
      }
    }
  } else if (warp == 1) {
    // ------------------------------- MMA issuer -------------------------------
    if (lane == 0) {
      uint32_t it = 0, gcount = 0;
      bool ok = true;
      const uint32_t id_pos = idesc_tc<OZ_BM, OZ_BN, 1>(false), id_neg = idesc_tc<OZ_BM, OZ_BN, 1>(true);
      for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
        for (int g = 0; g < G && ok; ++g, ++gcount) {
          const uint32_t buf = gcount % OZ_NBUF, use = gcount / OZ_NBUF;
          if (use > 0 &&
              !mbar_wait(smem_u32(&bars[2 * OZ_STAGES + 2 * buf + 1]), (use - 1) & 1, abort_flag)) {
            ok = false;
            break;
          }
          fence_after();
          const uint32_t dre = tmem + buf * 2 * OZ_BN, dim = dre + OZ_BN;
          bool first = true;
          for (int pr = plan.first[g]; pr < plan.first[g] + plan.count[g] && ok; ++pr)
            for (int ks = 0; ks < ksteps; ++ks, ++it) {
              const uint32_t s = it % OZ_STAGES, ph = (it / OZ_STAGES) & 1;
              if (!mbar_wait(smem_u32(&bars[s]), ph, abort_flag)) { ok = false; break; }
              fence_after();
              const uint32_t st = smem_u32(stages + s * OZ_STAGE);
              const uint64_t a_r = sdesc_sw32(st), a_i = sdesc_sw32(st + OZ_A_BYTES);
              const uint64_t b_r = sdesc_sw32(st + 2 * OZ_A_BYTES);
              const uint64_t b_i = sdesc_sw32(st + 2 * OZ_A_BYTES + OZ_B_BYTES);
              mma_issue<1>(dre, a_r, b_r, id_pos, first ? 0u : 1u);
              mma_issue<1>(dim, a_r, b_i, id_pos, first ? 0u : 1u);
              if (!geo.a_real) {
                mma_issue<1>(dre, a_i, b_i, id_neg, 1u);
                mma_issue<1>(dim, a_i, b_r, id_pos, 1u);
              }
              first = false;
              mma_commit(smem_u32(&bars[OZ_STAGES + s]));
            }
          if (!ok) break;
          mma_commit(smem_u32(&bars[2 * OZ_STAGES + 2 * buf]));
        }
      }
      if (!ok) {
        *abort_flag = 1;
        atomicExch(err, 2);
        const uint32_t buf = gcount % OZ_NBUF, use = gcount / OZ_NBUF;
        mma_commit(smem_u32(&bars[2 * OZ_STAGES + 2 * buf]));
        const unsigned long long t0 = gtimer();
        while (!mbar_try(smem_u32(&bars[2 * OZ_STAGES + 2 * buf]), use & 1))
          if (gtimer() - t0 > RMAT_TC_WAIT_NS) break;
      }
    }
  } else {
    // -------------------------------- epilogue --------------------------------
    const int quad = warp & 3, half = (warp - 2) >> 2;
    const int row = quad * 32 + lane;
    uint32_t gcount = 0;
    bool ok = true;
    for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
      const int i = tile / (mt * nt), rem = tile % (mt * nt);
      const int m0 = (rem % mt) * OZ_BM, n0 = (rem / mt) * OZ_BN;
      double acr[32], aci[32];
#pragma unroll
      for (int c = 0; c < 32; ++c) acr[c] = aci[c] = 0.0;
      for (int g = 0; g < G; ++g, ++gcount) {
        const uint32_t buf = gcount % OZ_NBUF, use = gcount / OZ_NBUF;
        if (!mbar_wait(smem_u32(&bars[2 * OZ_STAGES + 2 * buf]), use & 1, abort_flag)) {
          *abort_flag = 1;
          atomicExch(err, 2);
          ok = false;
          break;
        }
        fence_after();
        const double w = ldexp(1.0, -6 * (plan.d[g] + 2));
        const uint32_t ta = tmem + buf * 2 * OZ_BN + ((uint32_t)(quad * 32) << 16) + half * 32;
        float v[32];
        tmem_ld16(ta, v);
        tmem_ld16(ta + 16, v + 16);
        tmem_wait_ld();
#pragma unroll
        for (int c = 0; c < 32; ++c) acr[c] = fma((double)v[c], w, acr[c]);
        tmem_ld16(ta + OZ_BN, v);
        tmem_ld16(ta + OZ_BN + 16, v + 16);
        tmem_wait_ld();
        fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(&bars[2 * OZ_STAGES + 2 * buf + 1]));
#pragma unroll
        for (int c = 0; c < 32; ++c) aci[c] = fma((double)v[c], w, aci[c]);
      }
      if (!ok) break;
      const int arow = m0 + row;
      if (arow < geo.mrows) {
        const int e = ew[(geo.ew_shared ? 0 : (size_t)i * geo.mrows) + arow];
        double2* r = R + ((geo.pt_major ? (size_t)i * geo.nlag + arow
                                         : (size_t)arow * geo.nlag + i)) * nrhs;
#pragma unroll
        for (int c = 0; c < 32; ++c) {
          const int be = n0 + half * 32 + c;
          if (be < nrhs) {
            const int sc = e + fx[(size_t)i * nrhs + be];
            double2 v = r[be];
            v.x -= ldexp(acr[c], sc);
            v.y -= ldexp(aci[c], sc);
            r[be] = v;
          }
        }
      }
    }
  }
  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 1)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
}

// Digit pairs (p, q), p + q <= OZ_D, in groups that keep every FP32 sum exact.
bool make_plan(int kpad, OzPlan* pl) {
  const double per_pair = 2.0 * kpad * 63.0 * 63.0;  // |Re| bound of one pair's sum
  const int gmax = (int)std::floor(16777215.0 / per_pair);
  if (gmax < 1) return false;
  int np = 0, ng = 0;
  for (int d = 0; d <= OZ_D; ++d) {
    int left = d + 1, p = 0;
    while (left > 0) {
      const int cnt = std::min(left, gmax);
      if (ng >= OZ_MAXG || np + cnt > OZ_MAXP) return false;
      pl->first[ng] = (unsigned char)np;
      pl->count[ng] = (unsigned char)cnt;
      pl->d[ng] = (unsigned char)d;
      for (int k = 0; k < cnt; ++k, ++p, ++np) {
        pl->p[np] = (unsigned char)p;
        pl->q[np] = (unsigned char)(d - p);
      }
      ++ng;
      left -= cnt;
    }
  }
  pl->ngroups = ng;
  return true;
}

struct OzState {
  __half* wsl = nullptr; size_t wsl_cap = 0;
  __half* xsl = nullptr; size_t xsl_cap = 0;
  int* ew = nullptr;     size_t ew_cap = 0;
  int* fx = nullptr;     size_t fx_cap = 0;
  // kinetic product: K's digit planes (once per mesh), X's along the mesh index
  __half* ksl = nullptr; size_t ksl_cap = 0;
  __half* xksl = nullptr; size_t xksl_cap = 0;
  int* ek = nullptr;     size_t ek_cap = 0;
  int* fxk = nullptr;    size_t fxk_cap = 0;
  const void* k_src = nullptr;
  long long k_gen = -1;
  int k_nlag = -1;
  OzMaps kmaps;
  const void* kmap_k = nullptr;
  const void* kmap_x = nullptr;
  int kmap_key[3] = {-1, -1, -1};
  OzPlan kplan;
  int kplan_kpad = -1;
  const void* w_src = nullptr;  // W digit planes built from this table ...
  long long w_gen = -1;         // ... at this point-coupling generation
  OzMaps maps;
  const void* map_w = nullptr;
  const void* map_x = nullptr;
  int map_key[4] = {-1, -1, -1, -1};
  OzPlan plan;
  int plan_kpad = -1;
};

OzState& oz_state(rmat_ctx c) {
  if (!c->oz) c->oz = new OzState();
  return *reinterpret_cast<OzState*>(c->oz);
}

bool g_oz_attr = false;

int launch_product(rmat_ctx c, const OzMaps& maps, const OzPlan& plan, const OzGeom& geo,
                   double2* Rout, int kpad, const int* ew, const int* fx, const int* skip) {
  if (!g_oz_attr) {
    RMAT_CU(cudaFuncSetAttribute(oz_product_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)OZ_SMEM));
    g_oz_attr = true;
  }
  const int tiles = geo.npts * ceil_div(geo.mrows, OZ_BM) * ceil_div(c->nrhs, OZ_BN);
  const int grid = std::min(tiles, c->sm_count);
  oz_product_kernel<<<grid, OZ_THREADS, OZ_SMEM, c->stream>>>(maps, plan, geo, Rout, c->nrhs, kpad,
                                                              ew, fx, skip,
                                                              c->dstat + ST_TIMEOUT);
  c->launches++;
  RMAT_CU(cudaGetLastError());
  return RMAT_OK;
}

}  // namespace

// Whether the residual of this context takes the tensor-core coupling product.
bool oz_enabled(rmat_ctx c) {
  if (c->kind != 1 || c->resid_param == 1) return false;
  const int kpad = (int)round_up(c->nch, 16);
  if (kpad > 2048) return false;
  return c->resid_param >= 2 || c->nch >= 32;
}

// R -= (W_i off-diagonal) X_i at every mesh point on the tensor cores.
int launch_oz_coupling(rmat_ctx c, const double2* Xin, double2* Rout, const int* skip) {
  OzState& z = oz_state(c);
  const int nch = c->nch, nlag = c->nlag, nrhs = c->nrhs;
  const int kpad = (int)round_up(nch, 16);
  if (z.plan_kpad != kpad) {
    if (!make_plan(kpad, &z.plan)) return RMAT_ESTATE;
    z.plan_kpad = kpad;
  }
  const size_t wrows = (size_t)2 * OZ_S * nlag * nch, xrows = (size_t)2 * OZ_S * nlag * nrhs;
  RMAT_CHECK(rmat_grow(c, (void**)&z.wsl, &z.wsl_cap, wrows * kpad * sizeof(__half)));
  RMAT_CHECK(rmat_grow(c, (void**)&z.xsl, &z.xsl_cap, xrows * kpad * sizeof(__half)));
  RMAT_CHECK(rmat_grow(c, (void**)&z.ew, &z.ew_cap, (size_t)nlag * nch * sizeof(int)));
  RMAT_CHECK(rmat_grow(c, (void**)&z.fx, &z.fx_cap, (size_t)nlag * nrhs * sizeof(int)));
  if (z.w_src != c->Wpt || z.w_gen != c->wpt_gen || z.map_w != z.wsl) {
    // the point-coupling table changed (new assembly): its digit planes, once
    oz_split_w_kernel<<<ceil_div(nlag * nch, 8), 256, 0, c->stream>>>(c->Wpt, nlag, nch, kpad, z.wsl,
                                                                      z.ew);
    c->launches++;
    RMAT_CU(cudaGetLastError());
    z.w_src = c->Wpt;
    z.w_gen = c->wpt_gen;
  }
  const int key[4] = {nch, nlag, nrhs, kpad};
  if (z.map_w != z.wsl || z.map_x != z.xsl || !std::equal(key, key + 4, z.map_key)) {
    RMAT_CHECK(tc_make_plane_map_f16(&z.maps.a, z.wsl, kpad, (int)wrows, kpad, OZ_BM));
    RMAT_CHECK(tc_make_plane_map_f16(&z.maps.b, z.xsl, kpad, (int)xrows, kpad, OZ_BN));
    z.map_w = z.wsl;
    z.map_x = z.xsl;
    std::copy(key, key + 4, z.map_key);
  }
  dim3 gx(ceil_div(nrhs, OZ_XT), nlag);
  oz_split_x_kernel<<<gx, 256, 0, c->stream>>>(Xin, nrhs, nlag, nch, 1, nlag, kpad, z.xsl, z.fx,
                                               skip);
  c->launches++;
  RMAT_CU(cudaGetLastError());
  const OzGeom geo{nlag, nch, nch, nlag, 0, 0, 0, nlag};
  return launch_product(c, z.maps, z.plan, geo, Rout, kpad, z.ew, z.fx, skip);
}

// Whether the kinetic part of the residual takes the tensor-core digit product too.
bool oz_kinetic_enabled(rmat_ctx c) {
  if (!oz_enabled(c) || c->sector) return false;
  // only on request: the rows of K are dominated by their diagonal, so cutting each row
  // at 2^-54 of its largest entry leaves about nlag/2 u of |K||X| per row where FP64
  // products leave ~u, and the refinement's floor rises with it (measured at
  // N = 25600: max|r|/max|Phi| stalls near 2e-10 instead of 1e-12)
  return c->resid_param == 3 && c->nlag <= 2048;
}

// R -= K X_al for every channel al on the tensor cores (K the real kinetic matrix).
int launch_oz_kinetic(rmat_ctx c, const double2* Xin, double2* Rout, const int* skip) {
  OzState& z = oz_state(c);
  const int nch = c->nch, nlag = c->nlag, nrhs = c->nrhs;
  const int kpad = (int)round_up(nlag, 16), a_rows = (int)round_up(nlag, OZ_BM);
  if (z.kplan_kpad != kpad) {
    if (!make_plan(kpad, &z.kplan)) return RMAT_ESTATE;
    z.kplan_kpad = kpad;
  }
  const size_t krows = (size_t)2 * OZ_S * a_rows, xrows = (size_t)2 * OZ_S * nch * nrhs;
  RMAT_CHECK(rmat_grow(c, (void**)&z.ksl, &z.ksl_cap, krows * kpad * sizeof(__half)));
  RMAT_CHECK(rmat_grow(c, (void**)&z.xksl, &z.xksl_cap, xrows * kpad * sizeof(__half)));
  RMAT_CHECK(rmat_grow(c, (void**)&z.ek, &z.ek_cap, (size_t)a_rows * sizeof(int)));
  RMAT_CHECK(rmat_grow(c, (void**)&z.fxk, &z.fxk_cap, (size_t)nch * nrhs * sizeof(int)));
  if (z.k_src != c->Kmat || z.k_gen != c->kmat_gen || z.k_nlag != nlag ||
      z.kmap_k != z.ksl) {  // K's digit planes, once per mesh
    oz_split_k_kernel<<<ceil_div(a_rows, 8), 256, 0, c->stream>>>(c->Kmat, nlag, a_rows, kpad,
                                                                  z.ksl, z.ek);
    c->launches++;
    RMAT_CU(cudaGetLastError());
    z.k_src = c->Kmat;
    z.k_gen = c->kmat_gen;
    z.k_nlag = nlag;
  }
  const int key[3] = {nch, nrhs, kpad};
  if (z.kmap_k != z.ksl || z.kmap_x != z.xksl || !std::equal(key, key + 3, z.kmap_key)) {
    RMAT_CHECK(tc_make_plane_map_f16(&z.kmaps.a, z.ksl, kpad, (int)krows, kpad, OZ_BM));
    RMAT_CHECK(tc_make_plane_map_f16(&z.kmaps.b, z.xksl, kpad, (int)xrows, kpad, OZ_BN));
    z.kmap_k = z.ksl;
    z.kmap_x = z.xksl;
    std::copy(key, key + 3, z.kmap_key);
  }
  dim3 gx(ceil_div(nrhs, OZ_XT), nch);
  oz_split_x_kernel<<<gx, 256, 0, c->stream>>>(Xin, nrhs, nch, nlag, nlag, 1, kpad, z.xksl, z.fxk,
                                               skip);
  c->launches++;
  RMAT_CU(cudaGetLastError());
  const OzGeom geo{nch, nlag, a_rows, 1, 1, 1, 1, nlag};
  return launch_product(c, z.kmaps, z.kplan, geo, Rout, kpad, z.ek, z.fxk, skip);
}

void oz_release(rmat_ctx c) {
  if (!c->oz) return;
  OzState& z = oz_state(c);
  cudaFree(z.wsl);
  cudaFree(z.xsl);
  cudaFree(z.ew);
  cudaFree(z.fx);
  cudaFree(z.ksl);
  cudaFree(z.xksl);
  cudaFree(z.ek);
  cudaFree(z.fxk);
  delete &z;
  c->oz = nullptr;
}
