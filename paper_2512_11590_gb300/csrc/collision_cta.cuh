// The R-matrix contraction and the collision matrix of ONE system by one thread block,
// with its scratch (matching system, channel functions, status) in device memory the
// caller provides: used by the allocation-free entry point (one static array) and by
// the batched small-system kernel (one slot per CTA).  See rmat_collision for the
// formulas: R = (hm/a) Phi^T X;  R~ = a sqrt(k) R sqrt(k);
//   U = (diag O - R~ diag O')^-1 (diag I - R~ diag I'), open x open block,
// by Gaussian elimination with partial pivoting (largest |Re|+|Im|, first row on
// ties) carrying the right-hand sides, then back substitution.
#pragma once

#include "cplx.cuh"
#include "rmat_internal.h"
#include "special.cuh"

namespace {

constexpr int MAXC = RMAT_NOALLOC_MAX_NCH;
constexpr int NA_THREADS = 256;

struct NoallocScratch {
  double2 R[MAXC * MAXC];   // R-matrix, row-major
  double2 ZO[MAXC * MAXC];  // matching matrix diag O - R~ diag O'
  double2 ZI[MAXC * MAXC];  // right-hand sides diag I - R~ diag I' (open columns)
  double2 I[MAXC], O[MAXC], dI[MAXC], dO[MAXC];
  double k[MAXC];
  int status;               // 0 ok, 1 + column of an exactly zero pivot,
                            // -(1 + channel) for a channel function that did not converge
};

struct NoallocParams {
  int nch, nlag, nopen, ldx;
  double a, hm, B, E;
  int l[MAXC];
  double thresh[MAXC];
  double zz[MAXC];
  int open[MAXC];
};

// R and U of one system by one CTA of NA_THREADS threads.  X[(al,i), be] sits at
// X[(al*nlag + i) * xr + be * xc] (column-major: xr = 1, xc = ldx; row-major N x nch:
// xr = nch, xc = 1).  S: this CTA's scratch.  Returns through S->status.
__device__ void matching_cta(const NoallocParams& p, const double* __restrict__ fa,
                             const double2* __restrict__ X, size_t xr, size_t xc,
                             double2* __restrict__ Rout, double2* __restrict__ Uout,
                             NoallocScratch* __restrict__ S) {
  const int tid = threadIdx.x;
  const int nch = p.nch, no = p.nopen;
  __shared__ int s_piv;
  if (tid == 0) S->status = 0;  // must start at zero on every call
  // R[al][be] = (hm/a) sum_i f_i(a) X[(al,i), be]
  for (int e = tid; e < nch * nch; e += NA_THREADS) {
    const int al = e / nch, be = e % nch;
    double sr = 0.0, si = 0.0;
    for (int i = 0; i < p.nlag; ++i) {
      const double2 x = X[((size_t)al * p.nlag + i) * xr + (size_t)be * xc];
      sr = fma(fa[i], x.x, sr);
      si = fma(fa[i], x.y, si);
    }
    const double2 r = make_double2(p.hm / p.a * sr, p.hm / p.a * si);
    S->R[e] = r;
    if (Rout) Rout[al + (size_t)nch * be] = r;
  }
  __syncthreads();  // status cleared before any channel can report
  // channel functions at rho = k a
  for (int ch = tid; ch < nch; ch += NA_THREADS) {
    double2 I, O, dI, dO;
    double k;
    if (!channel_functions(p.l[ch], p.E - p.thresh[ch], p.hm, p.a, p.B, p.zz[ch], &I, &O, &dI,
                           &dO, &k))
      S->status = -(1 + ch);
    S->I[ch] = I;
    S->O[ch] = O;
    S->dI[ch] = dI;
    S->dO[ch] = dO;
    S->k[ch] = k;
  }
  __syncthreads();
  // matching system (every entry written, nothing relies on earlier contents)
  for (int e = tid; e < nch * (nch + no); e += NA_THREADS) {
    const int row = e / (nch + no), col = e % (nch + no);
    const int cp = col < nch ? col : p.open[col - nch];
    const double2 R = S->R[row * nch + cp];
    const double s = p.a * sqrt(S->k[row]) * sqrt(S->k[cp]);
    const double2 Rt = make_double2(s * R.x, s * R.y);
    const double2 f = col < nch ? S->dO[cp] : S->dI[cp];
    double2 z = cmul<double>(Rt, f);
    z.x = -z.x;
    z.y = -z.y;
    if (row == cp) {
      const double2 d = col < nch ? S->O[row] : S->I[row];
      z.x += d.x;
      z.y += d.y;
    }
    if (col < nch) S->ZO[row * nch + col] = z;
    else S->ZI[row * no + (col - nch)] = z;
  }
  __syncthreads();
  // Gaussian elimination with partial pivoting, right-hand sides carried along
  for (int j = 0; j < nch; ++j) {
    if (tid < 32) {
      double best = -1.0;
      int bi = nch;
      for (int r = j + tid; r < nch; r += 32) {
        const double m = cabs1<double>(S->ZO[r * nch + j]);
        if (m > best) { best = m; bi = r; }
      }
      for (int o = 16; o > 0; o >>= 1) {
        const double ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
      }
      if (tid == 0) {
        s_piv = bi;
        if (!(best > 0.0) && S->status == 0) S->status = j + 1;
      }
    }
    __syncthreads();
    const int pv = s_piv;
    if (pv != j && pv < nch) {
      for (int c = tid; c < nch + no; c += NA_THREADS) {
        double2* a = c < nch ? &S->ZO[j * nch + c] : &S->ZI[j * no + (c - nch)];
        double2* b = c < nch ? &S->ZO[pv * nch + c] : &S->ZI[pv * no + (c - nch)];
        const double2 t = *a;
        *a = *b;
        *b = t;
      }
    }
    __syncthreads();
    const double2 piv = S->ZO[j * nch + j];
    if (piv.x != 0.0 || piv.y != 0.0) {  // the same value in every thread
      // multipliers once per row, kept in the (otherwise unused) lower part of ZO
      for (int r = j + 1 + tid; r < nch; r += NA_THREADS)
        S->ZO[r * nch + j] = cdiv<double>(S->ZO[r * nch + j], piv);
      __syncthreads();
      const int rows = nch - j - 1, cols = nch - j - 1 + no;
      for (int e = tid; e < rows * cols; e += NA_THREADS) {
        const int r = j + 1 + e / cols, cc = e % cols;
        const double2 lm = S->ZO[r * nch + j];
        if (cc < nch - j - 1) {
          const int c = j + 1 + cc;
          csub_mul<double>(S->ZO[r * nch + c], lm, S->ZO[j * nch + c]);
        } else {
          const int c = cc - (nch - j - 1);
          csub_mul<double>(S->ZI[r * no + c], lm, S->ZI[j * no + c]);
        }
      }
    }
    __syncthreads();
  }
  // back substitution on the open columns
  for (int j = nch - 1; j >= 0; --j) {
    const double2 d = S->ZO[j * nch + j];
    for (int c = tid; c < no; c += NA_THREADS)
      if (d.x != 0.0 || d.y != 0.0) S->ZI[j * no + c] = cdiv<double>(S->ZI[j * no + c], d);
    __syncthreads();
    for (int e = tid; e < j * no; e += NA_THREADS) {
      const int r = e / no, c = e % no;
      csub_mul<double>(S->ZI[r * no + c], S->ZO[r * nch + j], S->ZI[j * no + c]);
    }
    __syncthreads();
  }
  // U(q, q2) = Ufull[open[q]][q2], column-major nopen x nopen
  for (int e = tid; e < no * no; e += NA_THREADS) {
    const int q = e % no, q2 = e / no;
    Uout[e] = S->ZI[p.open[q] * no + q2];
  }
}

}  // namespace
