// G7/G8: FP64 residual and refinement update (Sec. 3.2; Sec. 3.4 step 7).
//
// The paper forms r = b - M x in double precision on the host (dense ZGEMM,
// 8 N^2 nrhs flops).  Here the residual of an assembled problem is formed on
// the device from the block structure of Eq. (block_structure):
//   r[(al,i),be] = delta_{al be} f_i(a) - sum_j K[i][j] X[(al,j),be]
//                  - sum_al' W_i[al][al'] X[(al',i),be]
// with K = hm T0 - hm (B/a) f f^T (nlag x nlag, real) and W_i the full local
// coupling at mesh point i (potential plus centrifugal/threshold/-E diagonal):
// 4 nlag^2 nch nrhs + 8 nch^2 nlag nrhs flops instead of 8 N^2 nrhs, and no
// N x N matrix in FP64.  A loaded dense system uses the dense FP64 product.
// All solution/residual arrays here are row-major N x nrhs.
#include <algorithm>

#include "cplx.cuh"
#include "rmat_internal.h"

namespace {

// r = Phi - K X  (one CTA per (channel, 32 right-hand sides); warps over mesh rows).
// MODE 0: FP64 sums; MODE 1: compensated sums (dot2_add; r rounded once at the end),
// which takes the rounding of the dominant kinetic part of C X off the refinement's
// floor; with Wd (the point-coupling table, may be null) the diagonal W_i[al][al] X is
// included here (the tensor-core product takes only al' != al).
// MODE 2: S[(al,i),be] = sum_j |K[i][j]| Ax[(al,j),be] into the real array S, from
// the magnitudes Ax = |X| (the kinetic part of |C||X|, the scale of the FP64 floor).
template <int MODE>
__global__ void __launch_bounds__(256)
resid_kinetic_kernel(double2* __restrict__ R, const double2* __restrict__ X,
                     const double* __restrict__ Ax, int nrhs, int nlag,
                     const double* __restrict__ K, const double* __restrict__ fa,
                     const double* __restrict__ faL, const int* __restrict__ skip,
                     double* __restrict__ S, const double2* __restrict__ Wd) {
  if (skip && *skip) return;
  const int al = blockIdx.y;
  const int be = blockIdx.x * 32 + (threadIdx.x & 31);
  const int warp = threadIdx.x >> 5;
  if (be >= nrhs) return;
  const size_t base = (size_t)al * nlag * nrhs + be;
  for (int i = warp; i < nlag; i += 8) {
    const double* Ki = K + (size_t)i * nlag;
    if (MODE == 2) {
      double sa = 0.0;
      for (int j = 0; j < nlag; ++j) sa = fma(fabs(__ldg(Ki + j)), Ax[base + (size_t)j * nrhs], sa);
      S[base + (size_t)i * nrhs] = sa;
      continue;
    }
    double sr = 0.0, si = 0.0, cr = 0.0, ci = 0.0;
    for (int j = 0; j < nlag; ++j) {
      const double k = __ldg(Ki + j);
      const double2 x = X[base + (size_t)j * nrhs];
      if (MODE == 1) {
        dot2_add(sr, cr, k, x.x);
        dot2_add(si, ci, k, x.y);
      } else {
        sr = fma(k, x.x, sr);
        si = fma(k, x.y, si);
      }
    }
    const int nch = gridDim.y;
    if (Wd) {
      const double2 w = Wd[((size_t)i * nch + al) * nch + al];
      const double2 x = X[base + (size_t)i * nrhs];
      if (MODE == 1) {
        dot2_add(sr, cr, w.x, x.x);
        dot2_add(sr, cr, -w.y, x.y);
        dot2_add(si, ci, w.x, x.y);
        dot2_add(si, ci, w.y, x.x);
      } else {
        sr = fma(w.x, x.x, fma(-w.y, x.y, sr));
        si = fma(w.x, x.y, fma(w.y, x.x, si));
      }
    }
    // surface terms: columns be < nch f_i(a) (or f_i(r2)), columns nch + be f_i(r1)
    const double phi = (faL && be >= nch) ? (al == be - nch ? faL[i] : 0.0)
                                          : (al == be ? fa[i] : 0.0);
    R[base + (size_t)i * nrhs] = make_double2((phi - sr) - cr, (-si) - ci);
  }
}

// R = Phi - Wd X: the surface right-hand side and the diagonal point coupling
// W_i[al][al] X[(al,i),be] in FP64, when the kinetic and the off-diagonal coupling
// products are both formed on the tensor cores.
__global__ void __launch_bounds__(256)
resid_diag_kernel(double2* __restrict__ R, const double2* __restrict__ X, int nrhs, int nlag,
                  int nch, const double2* __restrict__ Wd, const double* __restrict__ fa,
                  const int* __restrict__ skip) {
  if (skip && *skip) return;
  const size_t total = (size_t)nch * nlag * nrhs;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    const int be = (int)(e % nrhs);
    const size_t row = e / nrhs;
    const int i = (int)(row % nlag), al = (int)(row / nlag);
    const double2 w = Wd[((size_t)i * nch + al) * nch + al];
    const double2 x = X[e];
    const double phi = al == be ? fa[i] : 0.0;
    R[e] = make_double2(phi - fma(w.x, x.x, -w.y * x.y), -fma(w.x, x.y, w.y * x.x));
  }
}

__global__ void absx_kernel(const double2* __restrict__ X, double* __restrict__ Ax, size_t total) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x)
    Ax[e] = hypot(X[e].x, X[e].y);
}

// r -= W_i X_i at every mesh point: complex FP64 GEMM (nch x nch) x (nch x nrhs)
// per point on the FP64 tensor path (mma.m8n8k4.f64; the complex product as four
// real products, -Wi*Xi through a negated copy of the Wi fragment: the three-product
// form doubles the rounding of Im and with it the refinement's floor).  64 x 64
// output tile per CTA, 16-deep K chunks staged in shared memory as separate real
// and imaginary [k][64] planes (row pitch 72 doubles: the 4 k-rows x 8 entries a
// fragment load touches fall in distinct 8-byte bank slots, two wavefronts).
// Each of the 8 warps owns a 32 x 16 sub-tile: 4 x 2 tiles of 8 x 8.
constexpr int RC_T = 64, RC_K = 16, RC_LD = 72;

__device__ __forceinline__ void dmma(double& d0, double& d1, double a, double b) {
  asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};"
               : "+d"(d0), "+d"(d1)
               : "d"(a), "d"(b));
}

// ABS: one real product |W_i| |X_i| per tile (|.| the complex modulus), added to
// the kinetic part in S, and the maximum of the sum into *amax (the bit pattern of
// a non-negative double is monotone, so an integer atomicMax orders it).
template <bool ABS>
__global__ void __launch_bounds__(256)
resid_coupling_kernel(double2* __restrict__ R, const double2* __restrict__ X, int nrhs, int nlag,
                      int nch, const double2* __restrict__ W, const int* __restrict__ skip,
                      const double* __restrict__ S, unsigned long long* __restrict__ amax,
                      const double* __restrict__ Ax) {
  if (skip && *skip) return;
  __shared__ double Wr[RC_K][RC_LD], Wm[RC_K][RC_LD];  // W[a0 + a][k0 + k] -> [k][a]
  __shared__ double Xr[RC_K][RC_LD], Xm[RC_K][RC_LD];  // X[(k0 + k, i)][b0 + b] -> [k][b]
  const int i = blockIdx.z;
  const int a0 = blockIdx.y * RC_T, b0 = blockIdx.x * RC_T;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int wa = (warp >> 2) * 32, wb = (warp & 3) * 16;  // warp sub-tile origin
  const int g = lane >> 2, t = lane & 3;                   // fragment group / thread in group
  const double2* Wi = W + (size_t)i * nch * nch;
  double t1[4][2][2], t2[4][2][2];  // re, im (ABS: |W||X| in t1)
#pragma unroll
  for (int p = 0; p < 4; ++p)
#pragma unroll
    for (int q = 0; q < 2; ++q)
#pragma unroll
      for (int h = 0; h < 2; ++h) t1[p][q][h] = t2[p][q][h] = 0.0;
  for (int k0 = 0; k0 < nch; k0 += RC_K) {
    // W tile: 64 rows x 16 k (coalesced along k); X tile: 16 k x 64 columns
    for (int e = threadIdx.x; e < RC_T * RC_K; e += 256) {
      const int kk = e & (RC_K - 1), aa = e >> 4;
      const int ga = a0 + aa, gk = k0 + kk;
      const double2 w = (ga < nch && gk < nch) ? Wi[(size_t)ga * nch + gk] : make_double2(0, 0);
      Wr[kk][aa] = ABS ? hypot(w.x, w.y) : w.x;
      Wm[kk][aa] = w.y;
      const int kb = e >> 6, bb = e & (RC_T - 1);
      const int gk2 = k0 + kb, gb = b0 + bb;
      if (ABS) {
        Xr[kb][bb] = (gk2 < nch && gb < nrhs) ? Ax[((size_t)gk2 * nlag + i) * nrhs + gb] : 0.0;
      } else {
        const double2 x = (gk2 < nch && gb < nrhs) ? X[((size_t)gk2 * nlag + i) * nrhs + gb]
                                                  : make_double2(0, 0);
        Xr[kb][bb] = x.x;
        Xm[kb][bb] = x.y;
      }
    }
    __syncthreads();
#pragma unroll
    for (int k4 = 0; k4 < RC_K; k4 += 4) {
      double ar[4], ai[4], an[4], br[2], bi[2];
#pragma unroll
      for (int p = 0; p < 4; ++p) {
        ar[p] = Wr[k4 + t][wa + 8 * p + g];
        ai[p] = Wm[k4 + t][wa + 8 * p + g];
        an[p] = -ai[p];
      }
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        br[q] = Xr[k4 + t][wb + 8 * q + g];
        bi[q] = Xm[k4 + t][wb + 8 * q + g];
      }
      if (ABS) {
#pragma unroll
        for (int p = 0; p < 4; ++p)
#pragma unroll
          for (int q = 0; q < 2; ++q) dmma(t1[p][q][0], t1[p][q][1], ar[p], br[q]);
        continue;
      }
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          dmma(t1[p][q][0], t1[p][q][1], ar[p], br[q]);   // re
          dmma(t1[p][q][0], t1[p][q][1], an[p], bi[q]);
          dmma(t2[p][q][0], t2[p][q][1], ar[p], bi[q]);   // im
          dmma(t2[p][q][0], t2[p][q][1], ai[p], br[q]);
        }
    }
    __syncthreads();
  }
  // accumulator element (row g, columns 2t, 2t+1) of each 8 x 8 tile
  if (ABS) {
    double m = 0.0;
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      const int ga = a0 + wa + 8 * p + g;
#pragma unroll
      for (int q = 0; q < 2; ++q)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int gb = b0 + wb + 8 * q + 2 * t + h;
          if (ga < nch && gb < nrhs)
            m = fmax(m, S[((size_t)ga * nlag + i) * nrhs + gb] + t1[p][q][h]);
        }
    }
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) atomicMax(amax, (unsigned long long)__double_as_longlong(m));
    return;
  }
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    const int ga = a0 + wa + 8 * p + g;
    if (ga >= nch) continue;
#pragma unroll
    for (int q = 0; q < 2; ++q)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int gb = b0 + wb + 8 * q + 2 * t + h;
        if (gb >= nrhs) continue;
        double2* r = R + ((size_t)ga * nlag + i) * nrhs + gb;
        double2 v = *r;
        v.x -= t1[p][q][h];
        v.y -= t2[p][q][h];
        *r = v;
      }
  }
}

// max |r| (bit pattern of a non-negative double is monotone) and r -> solve precision
template <class T>
__global__ void resid_norm_convert_kernel(const double2* __restrict__ R, size_t total, int nrhs,
                                          const double* __restrict__ D, cplx<T>* __restrict__ Bw,
                                          unsigned long long* __restrict__ red,
                                          const int* __restrict__ skip) {
  if (skip && *skip) return;
  double m = 0.0;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    double2 z = R[e];
    m = fmax(m, hypot(z.x, z.y));
    if (D) {
      const double s = D[e / nrhs];
      z.x *= s;
      z.y *= s;
    }
    Bw[e] = to_c(z, T());
  }
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  __shared__ double sm[32];
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x < 32) {
    m = (threadIdx.x < (blockDim.x >> 5)) ? sm[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (threadIdx.x == 0) atomicMax(red, (unsigned long long)__double_as_longlong(m));
  }
}

__global__ void absmax_kernel(const double2* __restrict__ v, size_t total,
                              unsigned long long* __restrict__ red) {
  double m = 0.0;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x)
    m = fmax(m, hypot(v[e].x, v[e].y));
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  __shared__ double sm[32];
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x < 32) {
    m = (threadIdx.x < (blockDim.x >> 5)) ? sm[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (threadIdx.x == 0) atomicMax(red, (unsigned long long)__double_as_longlong(m));
  }
}

// max over (row, column) of sum_k |A[row][k]| |X[k][column]| for a loaded dense
// system (row-major A N x N, X N x nrhs): one thread per output entry.
__global__ void absprod_dense_kernel(const double2* __restrict__ A, const double2* __restrict__ X,
                                     int N, int nrhs, unsigned long long* __restrict__ amax) {
  const size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  double m = 0.0;
  if (e < (size_t)N * nrhs) {
    const int row = (int)(e / nrhs), col = (int)(e % nrhs);
    const double2* a = A + (size_t)row * N;
    for (int k = 0; k < N; ++k) {
      const double2 x = X[(size_t)k * nrhs + col];
      m = fma(hypot(a[k].x, a[k].y), hypot(x.x, x.y), m);
    }
  }
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(amax, (unsigned long long)__double_as_longlong(m));
}

template <class T>
__global__ void x_update_kernel(double2* __restrict__ X, const cplx<T>* __restrict__ W,
                                size_t total, int nrhs, const double* __restrict__ D,
                                const IrState* __restrict__ st) {
  if (st && st->done) return;  // device-driven refinement: already stopped
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    const double2 d = to_d(W[e]);
    const double s = D ? D[e / nrhs] : 1.0;
    double2 x = X[e];
    x.x += s * d.x;
    x.y += s * d.y;
    X[e] = x;
  }
}

template <class T>
__global__ void x_from_w_kernel(double2* __restrict__ X, const cplx<T>* __restrict__ W,
                                size_t total, int nrhs, const double* __restrict__ D) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    double2 x = to_d(W[e]);
    if (D) {
      const double s = D[e / nrhs];
      x.x *= s;
      x.y *= s;
    }
    X[e] = x;
  }
}

// right-hand sides into the solve buffer: surface terms (assembled) or B (dense)
template <class T>
__global__ void w_from_phi_kernel(cplx<T>* __restrict__ Bw, int N, int nrhs, int nlag,
                                  const double* __restrict__ fa, const double* __restrict__ faL,
                                  const double2* __restrict__ B64, const double* __restrict__ D) {
  const size_t total = (size_t)N * nrhs;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    const int row = (int)(e / nrhs), be = (int)(e % nrhs);
    double2 z;
    if (B64) {
      z = B64[e];
    } else {
      const int al = row / nlag, i = row - al * nlag, nch = N / nlag;
      if (faL && be >= nch) z = make_double2(al == be - nch ? faL[i] : 0.0, 0.0);
      else z = make_double2(al == be ? fa[i] : 0.0, 0.0);
    }
    if (D) {
      z.x *= D[row];
      z.y *= D[row];
    }
    Bw[e] = to_c(z, T());
  }
}

// row-major N x nrhs (internal) -> column-major N x nrhs with leading dimension ldx
__global__ void x_to_colmajor_kernel(const double2* __restrict__ X, int N, int nrhs,
                                     double2* __restrict__ Xo, int ldx) {
  __shared__ double2 tile[32][33];
  const int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int k = ty; k < 32; k += 8) {
    const int rr = r0 + k, cc = c0 + tx;
    tile[k][tx] = (rr < N && cc < nrhs) ? X[(size_t)rr * nrhs + cc] : make_double2(0, 0);
  }
  __syncthreads();
  for (int k = ty; k < 32; k += 8) {
    const int cc = c0 + k, rr = r0 + tx;
    if (rr < N && cc < nrhs) Xo[rr + (size_t)ldx * cc] = tile[tx][k];
  }
}

// column-major N x nrhs (leading dimension ldx) -> row-major N x nrhs (internal)
__global__ void x_from_colmajor_kernel(const double2* __restrict__ Xi, int ldx, int N, int nrhs,
                                       double2* __restrict__ X) {
  __shared__ double2 tile[32][33];
  const int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int k = ty; k < 32; k += 8) {
    const int cc = c0 + k, rr = r0 + tx;
    tile[tx][k] = (rr < N && cc < nrhs) ? Xi[rr + (size_t)ldx * cc] : make_double2(0, 0);
  }
  __syncthreads();
  for (int k = ty; k < 32; k += 8) {
    const int rr = r0 + k, cc = c0 + tx;
    if (rr < N && cc < nrhs) X[(size_t)rr * nrhs + cc] = tile[k][tx];
  }
}

// Device-side stopping rule of the graph-capturable refinement (the rule of the
// host loop of rmat_solve): tol reached; the FP64 floor (normwise backward error
// max|r| / (max|C||X| + max|Phi|) <= RMAT_FLOOR_CONV u) seen `need` times in a row:
// one last correction, then stop (RMAT_OK); non-finite residual; non-halving residual
// `patience` times in a row (RMAT_OK when within RMAT_FLOOR_STALL u of the floor, else
// RMAT_ENOCONV); or the last allowed step.
__global__ void ir_init_kernel(IrState* st) {
  st->prev = INFINITY;
  st->rel = 0.0;
  st->stagn = 0;
  st->done = 0;
  st->status = RMAT_OK;
  st->iters = 0;
  st->floor_hits = 0;
  st->final = 0;
}

__global__ void ir_state_kernel(const unsigned long long* __restrict__ red, double phi_max,
                                double tol, int patience, int need, int last, IrState* st) {
  if (st->done) return;
  if (st->final) {  // the correction after the floor has been applied: stop
    st->done = 1;
    return;
  }
  const double rmax = __longlong_as_double((long long)red[0]);
  const double r = rmax / phi_max;
  const double scale = __longlong_as_double((long long)red[1]) + phi_max;
  st->rel = r;
  if (rmax <= RMAT_FLOOR_CONV * RMAT_U64 * scale) ++st->floor_hits;
  else st->floor_hits = 0;
  if (!isfinite(r)) {
    st->done = 1;
    st->status = RMAT_ENOCONV;
  } else if (r < tol) {
    st->done = 1;
  } else if (last) {
    st->done = 1;
    st->status = (tol > 0 && rmax > RMAT_FLOOR_STALL * RMAT_U64 * scale) ? RMAT_ENOCONV : RMAT_OK;
  } else if (st->floor_hits >= need) {
    st->final = 1;  // one more correction, then stop
  } else if (r > 0.5 * st->prev) {
    if (++st->stagn >= patience) {
      st->done = 1;
      st->status = rmax <= RMAT_FLOOR_STALL * RMAT_U64 * scale ? RMAT_OK : RMAT_ENOCONV;
    }
  } else {
    st->stagn = 0;
  }
  st->prev = r;
  if (!st->done) st->iters++;
}

int grid_for(rmat_ctx c, size_t total) {
  return std::max(1, (int)std::min<size_t>((size_t)c->sm_count * 8, (total + 255) / 256));
}

}  // namespace

// Rout = Phi - C Xin through the block structure of C: kinetic part (and, with the
// tensor-core coupling product, the diagonal point coupling) in FP64 on CUDA cores,
// the point couplings on the FP64 tensor instruction or as exact digit products on
// the tcgen05 tensor cores.
int structured_residual(rmat_ctx c, const double2* Xin, double2* Rout, const int* skip) {
  const int nrhs = c->nrhs;
  const bool oz = oz_enabled(c);
  if (oz_kinetic_enabled(c)) {  // every product on the tensor cores
    resid_diag_kernel<<<grid_for(c, (size_t)c->N * nrhs), 256, 0, c->stream>>>(
        Rout, Xin, nrhs, c->nlag, c->nch, c->Wpt, c->fa, skip);
    c->launches++;
    RMAT_CU(cudaGetLastError());
    RMAT_CHECK(launch_oz_kinetic(c, Xin, Rout, skip));
    return launch_oz_coupling(c, Xin, Rout, skip);
  }
  dim3 gk(ceil_div(nrhs, 32), c->nch);
  const bool comp = c->resid_comp == 1 || (c->resid_comp == -1 && c->precision == RMAT_C128);
  if (comp)
    resid_kinetic_kernel<1><<<gk, 256, 0, c->stream>>>(
        Rout, Xin, nullptr, nrhs, c->nlag, c->Kmat, c->fa, c->sector ? c->faL : nullptr, skip,
        nullptr, oz ? c->Wpt : nullptr);
  else
    resid_kinetic_kernel<0><<<gk, 256, 0, c->stream>>>(
        Rout, Xin, nullptr, nrhs, c->nlag, c->Kmat, c->fa, c->sector ? c->faL : nullptr, skip,
        nullptr, oz ? c->Wpt : nullptr);
  c->launches++;
  RMAT_CU(cudaGetLastError());
  if (oz) return launch_oz_coupling(c, Xin, Rout, skip);
  dim3 gc(ceil_div(nrhs, RC_T), ceil_div(c->nch, RC_T), c->nlag);
  resid_coupling_kernel<false><<<gc, 256, 0, c->stream>>>(Rout, Xin, nrhs, c->nlag, c->nch, c->Wpt,
                                                          skip, nullptr, nullptr, nullptr);
  c->launches++;
  RMAT_CU(cudaGetLastError());
  return RMAT_OK;
}

// r = Phi - C X (FP64) and max|r| -> red[0]; r is also written to Bw in the
// factor precision for the correction solve.
int launch_residual(rmat_ctx c, double*) {
  const int N = c->N, nrhs = c->nrhs;
  const size_t total = (size_t)N * nrhs;
  KTimer kt(c, KT_RESID);
  RMAT_CU(cudaMemsetAsync(c->red, 0, sizeof(unsigned long long), c->stream));
  if (c->kind == 1) {
    RMAT_CHECK(structured_residual(c, c->X, c->Rres, c->skip));
  } else {
    RMAT_CU(cudaMemcpyAsync(c->Rres, c->B64, total * sizeof(double2), cudaMemcpyDeviceToDevice,
                            c->stream));
    RMAT_CHECK(gemm_sub_c128(c, N, nrhs, N, c->A64, N, c->X, nrhs, c->Rres, nrhs));
  }
  RMAT_CU(cudaGetLastError());
  const double* D = c->equil ? c->Dsc : nullptr;
  if (c->precision == RMAT_C128)
    resid_norm_convert_kernel<double><<<grid_for(c, total), 256, 0, c->stream>>>(
        c->Rres, total, nrhs, D, reinterpret_cast<double2*>(c->Bw), c->red, c->skip);
  else
    resid_norm_convert_kernel<float><<<grid_for(c, total), 256, 0, c->stream>>>(
        c->Rres, total, nrhs, D, reinterpret_cast<float2*>(c->Bw), c->red, c->skip);
  c->launches++;
  RMAT_CU(cudaGetLastError());
  kt.end();
  return RMAT_OK;
}

// Rout = Phi - C Xin (FP64, row-major N x nrhs) for any Xin: the structured
// product of an assembled problem or the dense product of a loaded one.
int launch_apply_resid(rmat_ctx c, const double2* Xin, double2* Rout) {
  const int N = c->N, nrhs = c->nrhs;
  if (c->kind == 1) {
    RMAT_CHECK(structured_residual(c, Xin, Rout, nullptr));
  } else {
    RMAT_CU(cudaMemcpyAsync(Rout, c->B64, (size_t)N * nrhs * sizeof(double2),
                            cudaMemcpyDeviceToDevice, c->stream));
    RMAT_CHECK(gemm_sub_c128(c, N, nrhs, N, c->A64, N, Xin, nrhs, Rout, nrhs));
  }
  RMAT_CU(cudaGetLastError());
  return RMAT_OK;
}

// red[1] = max over entries of |C||X| (|.| the complex modulus, X = c->X): the scale
// of the FP64 floor of the refinement residual.  Uses Rres as scratch.
int launch_absprod(rmat_ctx c) {
  const int N = c->N, nrhs = c->nrhs;
  RMAT_CU(cudaMemsetAsync(c->red + 1, 0, sizeof(unsigned long long), c->stream));
  if (c->kind == 1) {
    // Rres as scratch: S = |K||X| in its first N nrhs doubles, |X| in the next
    double* S = reinterpret_cast<double*>(c->Rres);
    double* Ax = S + (size_t)N * nrhs;
    absx_kernel<<<grid_for(c, (size_t)N * nrhs), 256, 0, c->stream>>>(c->X, Ax, (size_t)N * nrhs);
    dim3 gk(ceil_div(nrhs, 32), c->nch);
    resid_kinetic_kernel<2><<<gk, 256, 0, c->stream>>>(nullptr, nullptr, Ax, nrhs, c->nlag, c->Kmat,
                                                       nullptr, nullptr, c->skip, S, nullptr);
    dim3 gc(ceil_div(nrhs, RC_T), ceil_div(c->nch, RC_T), c->nlag);
    resid_coupling_kernel<true><<<gc, 256, 0, c->stream>>>(nullptr, c->X, nrhs, c->nlag, c->nch,
                                                           c->Wpt, c->skip, S, c->red + 1, Ax);
    c->launches += 3;
  } else {
    const size_t total = (size_t)N * nrhs;
    absprod_dense_kernel<<<(unsigned)((total + 255) / 256), 256, 0, c->stream>>>(c->A64, c->X, N,
                                                                                nrhs, c->red + 1);
    c->launches++;
  }
  RMAT_CU(cudaGetLastError());
  return RMAT_OK;
}

int launch_update(rmat_ctx c, const IrState* st) {
  const size_t total = (size_t)c->N * c->nrhs;
  const double* D = c->equil ? c->Dsc : nullptr;
  if (c->precision == RMAT_C128)
    x_update_kernel<double><<<grid_for(c, total), 256, 0, c->stream>>>(
        c->X, reinterpret_cast<const double2*>(c->Bw), total, c->nrhs, D, st);
  else
    x_update_kernel<float><<<grid_for(c, total), 256, 0, c->stream>>>(
        c->X, reinterpret_cast<const float2*>(c->Bw), total, c->nrhs, D, st);
  c->launches++;
  RMAT_CU(cudaGetLastError());
  return RMAT_OK;
}

int launch_x_from_w(rmat_ctx c) {
  const size_t total = (size_t)c->N * c->nrhs;
  const double* D = c->equil ? c->Dsc : nullptr;
  if (c->precision == RMAT_C128)
    x_from_w_kernel<double><<<grid_for(c, total), 256, 0, c->stream>>>(
        c->X, reinterpret_cast<const double2*>(c->Bw), total, c->nrhs, D);
  else
    x_from_w_kernel<float><<<grid_for(c, total), 256, 0, c->stream>>>(
        c->X, reinterpret_cast<const float2*>(c->Bw), total, c->nrhs, D);
  c->launches++;
  RMAT_CU(cudaGetLastError());
  return RMAT_OK;
}

int launch_w_from_phi(rmat_ctx c) {
  const size_t total = (size_t)c->N * c->nrhs;
  const double2* B64 = (c->kind == 2) ? c->B64 : nullptr;
  const double* D = c->equil ? c->Dsc : nullptr;
  if (c->precision == RMAT_C128)
    w_from_phi_kernel<double><<<grid_for(c, total), 256, 0, c->stream>>>(
        reinterpret_cast<double2*>(c->Bw), c->N, c->nrhs, c->nlag, c->fa,
        c->sector ? c->faL : nullptr, B64, D);
  else
    w_from_phi_kernel<float><<<grid_for(c, total), 256, 0, c->stream>>>(
        reinterpret_cast<float2*>(c->Bw), c->N, c->nrhs, c->nlag, c->fa,
        c->sector ? c->faL : nullptr, B64, D);
  c->launches++;
  RMAT_CU(cudaGetLastError());
  return RMAT_OK;
}

int launch_x_out(rmat_ctx c, double2* Xo, int ldx) { return launch_to_colmajor(c, c->X, Xo, ldx); }

int launch_to_colmajor(rmat_ctx c, const double2* src, double2* dst, int ld) {
  dim3 grid(ceil_div(c->nrhs, 32), ceil_div(c->N, 32));
  x_to_colmajor_kernel<<<grid, 256, 0, c->stream>>>(src, c->N, c->nrhs, dst, ld);
  c->launches++;
  RMAT_CU(cudaGetLastError());
  return RMAT_OK;
}

int launch_from_colmajor(rmat_ctx c, const double2* src, int ld, double2* dst) {
  dim3 grid(ceil_div(c->nrhs, 32), ceil_div(c->N, 32));
  x_from_colmajor_kernel<<<grid, 256, 0, c->stream>>>(src, ld, c->N, c->nrhs, dst);
  c->launches++;
  RMAT_CU(cudaGetLastError());
  return RMAT_OK;
}

int launch_absmax(rmat_ctx c, const double2* v, size_t n) {
  RMAT_CU(cudaMemsetAsync(c->red, 0, sizeof(unsigned long long), c->stream));
  absmax_kernel<<<grid_for(c, n), 256, 0, c->stream>>>(v, n, c->red);
  c->launches++;
  RMAT_CU(cudaGetLastError());
  return RMAT_OK;
}

int launch_ir_init(rmat_ctx c, IrState* st) {
  ir_init_kernel<<<1, 1, 0, c->stream>>>(st);
  c->launches++;
  RMAT_CU(cudaGetLastError());
  return RMAT_OK;
}

int launch_ir_state(rmat_ctx c, double tol, int patience, int last, IrState* st) {
  ir_state_kernel<<<1, 1, 0, c->stream>>>(c->red, c->phi_max, tol, patience,
                                          rmat_floor_need(c->precision), last, st);
  c->launches++;
  RMAT_CU(cudaGetLastError());
  return RMAT_OK;
}
