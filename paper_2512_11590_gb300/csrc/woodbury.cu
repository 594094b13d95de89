// Woodbury-kinetic form of the internal-region system (Sec. 3.3, Type 3 solver).
//
// M = K_diag + V_coupling with K_diag = I_nch (x) K, K = hm*T0 - hm*(B/a) f f^T
// real and shared by every channel, and V_coupling everything of M that is
// diagonal in the radial index: W[j][al][al'] = V_al,al'(r_j) + delta (hm l(l+1)/r_j^2
// + E_al - E), the per-point table the FP64 residual already uses.  Then
//   M c = b  <=>  S c~ = (I (x) K^-1) b~,   S = I + (K^-1 (x) I) W   (radial-major),
//   S[(i,al),(j,al')] = delta_ij delta_al,al' + Kinv[i][j] W[j][al][al'],
// with (i, al) -> i*nch + al and c~ the radial-major reordering of c.
//
// Here S is the matrix that is factored (same N x N dense LU as M), but the
// refinement keeps the FP64 residual of the ORIGINAL system: every solve maps
// its channel-major right-hand side through K^-1 (FP64 accumulation) into
// radial-major order, solves with the factors of S and maps the result back.
// K^-1 removes the kinetic operator's conditioning from the factored matrix
// (cond S ~ 1e4 where cond M ~ 1e8 at nlag = 100), so a complex64 factor of S
// corrects 4-5 decimal digits per refinement step instead of ~2.  K^-1 depends
// on the mesh only (formed once per mesh on the host, FP64 Gauss-Jordan).
#include <cmath>
#include <vector>

#include "cplx.cuh"
#include "rmat_internal.h"

namespace {

// FP32 copy of the per-point coupling table for the complex64 Schur assembly.
__global__ void w_to_f32_kernel(float2* __restrict__ W32, const double2* __restrict__ W,
                                size_t total) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x)
    W32[e] = make_float2((float)W[e].x, (float)W[e].y);
}

// One warp per row (i, al) of S.  Column c = j*nch + al' reads W[j][al][al'],
// contiguous in al', and the broadcast Kinv[i][j]; lanes track (j, al') of
// their column incrementally.  Padding columns [N, ld) are written as zeros.
// Complex64 rows multiply in FP32 (both inputs rounded to FP32 once),
// complex128 rows in FP64.
template <class T, class WT>
__global__ void __launch_bounds__(256)
schur_assemble_kernel(cplx<T>* __restrict__ S, int ld, int N, int nch, int nlag,
                      const T* __restrict__ Kinv, const WT* __restrict__ W) {
  const int lane = threadIdx.x & 31;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  const int sq = 32 / nch, sr = 32 - sq * nch;  // 32 = sq*nch + sr
  for (int row = gw; row < N; row += nw) {
    const int i = row / nch, al = row - i * nch;
    cplx<T>* Srow = S + (size_t)row * ld;
    const T* Krow = Kinv + (size_t)i * nlag;
    int j = lane / nch, alp = lane - j * nch;
    for (int col = lane; col < ld; col += 32) {
      cplx<T> v = mkc<T>((T)0, (T)0);
      if (col < N) {
        const T k = Krow[j];
        const WT w = W[((size_t)j * nch + al) * nch + alp];
        v = mkc<T>(k * (T)w.x, k * (T)w.y);
        if (col == row) v.x += (T)1;
      }
      Srow[col] = v;
      alp += sr;
      j += sq;
      if (alp >= nch) { alp -= nch; j += 1; }
    }
  }
}

// Bs[(i,al), c] = sum_j Kinv[i][j] Bw[(al,j), c]   (FP64 accumulation).
// Grid (ceil(nrhs/32), ceil(nlag/64), nch); a CTA computes a 64 (i) x 32 (c)
// tile of one channel, a thread 4 x 2 outputs; j is staged 32 at a time.
constexpr int KA_TI = 64, KA_TC = 32, KA_TJ = 32;

template <class T>
__global__ void __launch_bounds__(256)
kinv_apply_kernel(const cplx<T>* __restrict__ Bw, cplx<T>* __restrict__ Bs, int nch, int nlag,
                  int nrhs, const double* __restrict__ Kinv, const int* __restrict__ skip) {
  if (skip && *skip) return;
  __shared__ double As[KA_TI][KA_TJ + 1];
  __shared__ double2 Xs[KA_TJ][KA_TC];
  const int al = blockIdx.z;
  const int i0 = blockIdx.y * KA_TI, c0 = blockIdx.x * KA_TC;
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;  // columns c0 + 2tx + {0,1}, rows i0 + 4ty + {0..3}
  double accr[4][2] = {}, acci[4][2] = {};
  for (int j0 = 0; j0 < nlag; j0 += KA_TJ) {
    for (int e = tid; e < KA_TI * KA_TJ; e += 256) {
      const int r = e / KA_TJ, q = e % KA_TJ;
      const int gi = i0 + r, gj = j0 + q;
      As[r][q] = (gi < nlag && gj < nlag) ? Kinv[(size_t)gi * nlag + gj] : 0.0;
    }
    for (int e = tid; e < KA_TJ * KA_TC; e += 256) {
      const int q = e / KA_TC, cc = e % KA_TC;
      const int gj = j0 + q, gc = c0 + cc;
      double2 x = make_double2(0.0, 0.0);
      if (gj < nlag && gc < nrhs) {
        const cplx<T> b = Bw[((size_t)al * nlag + gj) * nrhs + gc];
        x = make_double2((double)b.x, (double)b.y);
      }
      Xs[q][cc] = x;
    }
    __syncthreads();
    // padding rows (i >= nlag) and padding K steps (j >= nlag) skip the FP64 work:
    // at nlag = 100 the 64 x 32 tiling would otherwise issue 1.64x the useful FMAs
    const int qmax = (i0 + ty * 4 < nlag) ? min(KA_TJ, nlag - j0) : 0;
#pragma unroll 4
    for (int q = 0; q < qmax; ++q) {
      double a[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) a[r] = As[ty * 4 + r][q];
      const double2 x0 = Xs[q][tx * 2], x1 = Xs[q][tx * 2 + 1];
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        accr[r][0] = fma(a[r], x0.x, accr[r][0]);
        acci[r][0] = fma(a[r], x0.y, acci[r][0]);
        accr[r][1] = fma(a[r], x1.x, accr[r][1]);
        acci[r][1] = fma(a[r], x1.y, acci[r][1]);
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int gi = i0 + ty * 4 + r;
    if (gi >= nlag) continue;
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int gc = c0 + tx * 2 + u;
      if (gc < nrhs)
        Bs[((size_t)gi * nch + al) * nrhs + gc] = mkc<T>((T)accr[r][u], (T)acci[r][u]);
    }
  }
}

// Bs[(al,i), c] = Bw[(i,al), c]: radial-major rows back to channel-major.
template <class T>
__global__ void radial_to_channel_kernel(const cplx<T>* __restrict__ Bw, cplx<T>* __restrict__ Bs,
                                         int nch, int nlag, int nrhs,
                                         const int* __restrict__ skip) {
  if (skip && *skip) return;
  const size_t total = (size_t)nch * nlag * nrhs;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    const size_t row = e / nrhs;
    const int c = (int)(e - row * nrhs);
    const int al = (int)(row / nlag), i = (int)(row - (size_t)al * nlag);
    Bs[e] = Bw[((size_t)i * nch + al) * nrhs + c];
  }
}

// Gauss-Jordan inversion with partial pivoting (FP64, host); false if singular.
bool invert_host(std::vector<double>& A, int n, std::vector<double>& inv) {
  inv.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) inv[(size_t)i * n + i] = 1.0;
  for (int k = 0; k < n; ++k) {
    int p = k;
    for (int r = k + 1; r < n; ++r)
      if (std::fabs(A[(size_t)r * n + k]) > std::fabs(A[(size_t)p * n + k])) p = r;
    const double piv = A[(size_t)p * n + k];
    if (piv == 0.0 || !std::isfinite(piv)) return false;
    if (p != k)
      for (int c = 0; c < n; ++c) {
        std::swap(A[(size_t)p * n + c], A[(size_t)k * n + c]);
        std::swap(inv[(size_t)p * n + c], inv[(size_t)k * n + c]);
      }
    const double ip = 1.0 / piv;
    for (int c = 0; c < n; ++c) {
      A[(size_t)k * n + c] *= ip;
      inv[(size_t)k * n + c] *= ip;
    }
    for (int r = 0; r < n; ++r) {
      if (r == k) continue;
      const double f = A[(size_t)r * n + k];
      if (f == 0.0) continue;
      for (int c = 0; c < n; ++c) {
        A[(size_t)r * n + c] -= f * A[(size_t)k * n + c];
        inv[(size_t)r * n + c] -= f * inv[(size_t)k * n + c];
      }
    }
  }
  return true;
}

}  // namespace

// K^-1 of the current mesh (host FP64) into c->Kinv / c->Kinv32; once per mesh.
int woodbury_prepare(rmat_ctx c, const double* K_host) {
  const int n = c->nlag;
  std::vector<double> A(K_host, K_host + (size_t)n * n), inv;
  if (!invert_host(A, n, inv)) return RMAT_ESINGULAR;
  std::vector<float> inv32(inv.size());
  for (size_t e = 0; e < inv.size(); ++e) inv32[e] = (float)inv[e];
  RMAT_CHECK(rmat_grow(c, (void**)&c->Kinv, &c->Kinv_cap, inv.size() * sizeof(double)));
  RMAT_CHECK(rmat_grow(c, (void**)&c->Kinv32, &c->Kinv32_cap, inv32.size() * sizeof(float)));
  RMAT_CU(cudaMemcpy(c->Kinv, inv.data(), inv.size() * sizeof(double), cudaMemcpyHostToDevice));
  RMAT_CU(cudaMemcpy(c->Kinv32, inv32.data(), inv32.size() * sizeof(float),
                     cudaMemcpyHostToDevice));
  c->kinv_nlag = n;
  return RMAT_OK;
}

// S into c->C (needs the per-point table c->Wpt of this energy).
int launch_schur_assemble(rmat_ctx c) {
  const int blocks = std::max(1, std::min(c->sm_count * 8, ceil_div((long long)c->N * 32, 256)));
  if (c->precision == RMAT_C128) {
    schur_assemble_kernel<double, double2><<<blocks, 256, 0, c->stream>>>(
        reinterpret_cast<double2*>(c->C), c->ld, c->N, c->nch, c->nlag, c->Kinv, c->Wpt);
    c->launches++;
  } else {
    const size_t total = (size_t)c->nlag * c->nch * c->nch;
    RMAT_CHECK(rmat_grow(c, (void**)&c->W32, &c->W32_cap, total * sizeof(float2)));
    w_to_f32_kernel<<<std::max(1, std::min(c->sm_count * 4, ceil_div((long long)total, 256))), 256,
                      0, c->stream>>>(reinterpret_cast<float2*>(c->W32), c->Wpt, total);
    schur_assemble_kernel<float, float2><<<blocks, 256, 0, c->stream>>>(
        reinterpret_cast<float2*>(c->C), c->ld, c->N, c->nch, c->nlag, c->Kinv32,
        reinterpret_cast<const float2*>(c->W32));
    c->launches += 2;
  }
  RMAT_CU(cudaGetLastError());
  return RMAT_OK;
}

// Bw (channel-major) -> Bs = radial-major (I (x) K^-1) Bw -> copied back into Bw.
int launch_kinv_apply(rmat_ctx c) {
  const dim3 grid(ceil_div(c->nrhs, KA_TC), ceil_div(c->nlag, KA_TI), c->nch);
  const size_t bytes = (size_t)c->N * c->nrhs * (c->precision == RMAT_C128 ? 16 : 8);
  if (c->precision == RMAT_C128)
    kinv_apply_kernel<double><<<grid, 256, 0, c->stream>>>(
        reinterpret_cast<const double2*>(c->Bw), reinterpret_cast<double2*>(c->Bs), c->nch,
        c->nlag, c->nrhs, c->Kinv, c->skip);
  else
    kinv_apply_kernel<float><<<grid, 256, 0, c->stream>>>(
        reinterpret_cast<const float2*>(c->Bw), reinterpret_cast<float2*>(c->Bs), c->nch, c->nlag,
        c->nrhs, c->Kinv, c->skip);
  c->launches++;
  RMAT_CU(cudaGetLastError());
  RMAT_CU(cudaMemcpyAsync(c->Bw, c->Bs, bytes, cudaMemcpyDeviceToDevice, c->stream));
  return RMAT_OK;
}

// Bw (radial-major solution of S) -> Bs channel-major -> copied back into Bw.
int launch_radial_to_channel(rmat_ctx c) {
  const size_t total = (size_t)c->N * c->nrhs;
  const int blocks = std::max(1, std::min(c->sm_count * 8, ceil_div((long long)total, 256)));
  const size_t bytes = total * (c->precision == RMAT_C128 ? 16 : 8);
  if (c->precision == RMAT_C128)
    radial_to_channel_kernel<double><<<blocks, 256, 0, c->stream>>>(
        reinterpret_cast<const double2*>(c->Bw), reinterpret_cast<double2*>(c->Bs), c->nch,
        c->nlag, c->nrhs, c->skip);
  else
    radial_to_channel_kernel<float><<<blocks, 256, 0, c->stream>>>(
        reinterpret_cast<const float2*>(c->Bw), reinterpret_cast<float2*>(c->Bs), c->nch, c->nlag,
        c->nrhs, c->skip);
  c->launches++;
  RMAT_CU(cudaGetLastError());
  RMAT_CU(cudaMemcpyAsync(c->Bw, c->Bs, bytes, cudaMemcpyDeviceToDevice, c->stream));
  return RMAT_OK;
}
