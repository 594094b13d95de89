// GMRES-based iterative refinement (FGMRES-IR) for the complex64 factors.
//
// Classical refinement (Sec. 3.2) corrects x with d = M^-1 r, M^-1 the solve with
// the low-precision factors; it contracts by about cond(C) u_f per step and stalls
// once cond(C) u_f approaches 1.  GMRES-IR instead solves the correction equation
// C d = r by GMRES preconditioned with the same factors, in FP64 vectors with the
// FP64 product of C (Carson & Higham's GMRES-IR).  The preconditioner is applied
// in the factors' precision, so the flexible variant (FGMRES, right
// preconditioning, the preconditioned vectors z_k kept) is used:
//   beta = ||r||, v_0 = r / beta;  for k = 0, 1, ...:
//     z_k = M^-1 v_k,  w = C z_k,
//     h_jk = <v_j, w>, w -= sum_j h_jk v_j   (classical Gram-Schmidt, applied twice),
//     h_{k+1,k} = ||w||, v_{k+1} = w / h_{k+1,k},
//     Givens rotations reduce H to upper triangular and give the residual
//     estimate |g_{k+1}| of min ||beta e_1 - H y||;
//   d = sum_k y_k z_k.
// Every right-hand side (column of the N x nrhs row-major arrays) has its own
// Krylov space; the columns advance together and the inner loop ends when every
// column's estimate is below tau * beta or after m steps.  The small Hessenberg
// problems (at most 65 x 64 per column) are solved on the host.
#include <algorithm>
#include <cmath>
#include <complex>
#include <vector>

#include "cplx.cuh"
#include "rmat_internal.h"

namespace {

constexpr int GM_ROWS = 8;     // row groups per CTA of the column reductions
constexpr int GM_PARTS = 128;  // CTAs along the rows (partial sums per column)

// part[(p*k + j)*nrhs + c] = sum over this CTA's rows of conj(V_j[row][c]) * w[row][c]
__global__ void __launch_bounds__(32 * GM_ROWS)
col_dots_kernel(double2* __restrict__ part, const double2* __restrict__ V, size_t vstride, int k,
                const double2* __restrict__ w, int N, int nrhs) {
  const int c = blockIdx.x * 32 + threadIdx.x;
  const int p = blockIdx.y, P = gridDim.y;
  __shared__ double2 red[GM_ROWS][32];
  for (int j = 0; j < k; ++j) {
    const double2* Vj = V + (size_t)j * vstride;
    double sr = 0.0, si = 0.0;
    if (c < nrhs)
      for (int row = p * GM_ROWS + threadIdx.y; row < N; row += P * GM_ROWS) {
        const double2 a = Vj[(size_t)row * nrhs + c], b = w[(size_t)row * nrhs + c];
        sr = fma(a.x, b.x, fma(a.y, b.y, sr));  // Re(conj(a) b)
        si = fma(a.x, b.y, fma(-a.y, b.x, si)); // Im(conj(a) b)
      }
    red[threadIdx.y][threadIdx.x] = make_double2(sr, si);
    __syncthreads();
    if (threadIdx.y == 0 && c < nrhs) {
      double2 s = red[0][threadIdx.x];
      for (int q = 1; q < GM_ROWS; ++q) {
        s.x += red[q][threadIdx.x].x;
        s.y += red[q][threadIdx.x].y;
      }
      part[((size_t)p * k + j) * nrhs + c] = s;
    }
    __syncthreads();
  }
}

// out[j*nrhs + c] = sum_p part[(p*k + j)*nrhs + c]   (fixed order: deterministic)
__global__ void col_dots_finish_kernel(double2* __restrict__ out, const double2* __restrict__ part,
                                       int P, int k, int nrhs) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= k * nrhs) return;
  double2 s = make_double2(0.0, 0.0);
  for (int p = 0; p < P; ++p) {
    const double2 v = part[(size_t)p * k * nrhs + e];
    s.x += v.x;
    s.y += v.y;
  }
  out[e] = s;
}

// w[row][c] -= sum_j h[j][c] V_j[row][c]
__global__ void col_axpy_kernel(double2* __restrict__ w, const double2* __restrict__ V,
                                size_t vstride, int k, const double2* __restrict__ h, int N,
                                int nrhs) {
  const size_t total = (size_t)N * nrhs;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    const int c = (int)(e % nrhs);
    double2 acc = w[e];
    for (int j = 0; j < k; ++j) {
      const double2 a = h[j * nrhs + c], v = V[(size_t)j * vstride + e];
      acc.x -= a.x * v.x - a.y * v.y;
      acc.y -= a.x * v.y + a.y * v.x;
    }
    w[e] = acc;
  }
}

// v[row][c] = s[c] * w[row][c]  (s real)
__global__ void col_scale_kernel(double2* __restrict__ v, const double2* __restrict__ w,
                                 const double* __restrict__ s, int N, int nrhs) {
  const size_t total = (size_t)N * nrhs;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    const double f = s[e % nrhs];
    v[e] = make_double2(f * w[e].x, f * w[e].y);
  }
}

// X[row][c] += sum_j y[j][c] Z_j[row][c]
__global__ void col_combine_kernel(double2* __restrict__ X, const double2* __restrict__ Z,
                                   size_t zstride, int k, const double2* __restrict__ y, int N,
                                   int nrhs) {
  const size_t total = (size_t)N * nrhs;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    const int c = (int)(e % nrhs);
    double2 acc = X[e];
    for (int j = 0; j < k; ++j) {
      const double2 a = y[j * nrhs + c], z = Z[(size_t)j * zstride + e];
      acc.x += a.x * z.x - a.y * z.y;
      acc.y += a.x * z.y + a.y * z.x;
    }
    X[e] = acc;
  }
}

// Bw = D v in the factor precision (the equilibrated system's right-hand side)
template <class T>
__global__ void to_bw_kernel(cplx<T>* __restrict__ Bw, const double2* __restrict__ v, size_t total,
                             int nrhs, const double* __restrict__ D) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    double2 z = v[e];
    if (D) {
      const double s = D[e / nrhs];
      z.x *= s;
      z.y *= s;
    }
    Bw[e] = mkc<T>((T)z.x, (T)z.y);
  }
}

// z = D Bw in FP64
template <class T>
__global__ void from_bw_kernel(double2* __restrict__ z, const cplx<T>* __restrict__ Bw,
                               size_t total, int nrhs, const double* __restrict__ D) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    const double s = D ? D[e / nrhs] : 1.0;
    z[e] = make_double2(s * (double)Bw[e].x, s * (double)Bw[e].y);
  }
}

// w = Phi - t  (so that w = C z when t = Phi - C z)
__global__ void phi_minus_kernel(double2* __restrict__ w, const double2* __restrict__ t,
                                 size_t total, int nrhs, int nlag, const double* __restrict__ fa,
                                 const double* __restrict__ faL, int nch,
                                 const double2* __restrict__ B64) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    double2 phi;
    if (B64) {
      phi = B64[e];
    } else {
      const int row = (int)(e / nrhs), be = (int)(e % nrhs);
      const int al = row / nlag, i = row - al * nlag;
      if (faL && be >= nch) phi = make_double2(al == be - nch ? faL[i] : 0.0, 0.0);
      else phi = make_double2(al == be ? fa[i] : 0.0, 0.0);
    }
    w[e] = make_double2(phi.x - t[e].x, phi.y - t[e].y);
  }
}

int grid_of(rmat_ctx c, size_t total) {
  return std::max(1, (int)std::min<size_t>((size_t)c->sm_count * 8, (total + 255) / 256));
}

using cd = std::complex<double>;

struct Gmres {
  rmat_ctx c;
  int N, nrhs, m;
  size_t total;
  double2 *V, *Z, *T, *part, *dots, *hd;
  double* sd;
  std::vector<double2> hbuf;

  // dots[j][c] = <V_j, w> for j < k  (host copy in hbuf)
  int col_dots(const double2* Vb, int k, const double2* w) {
    const int P = std::max(1, std::min(GM_PARTS, ceil_div(N, GM_ROWS)));
    col_dots_kernel<<<dim3(ceil_div(nrhs, 32), P), dim3(32, GM_ROWS), 0, c->stream>>>(
        part, Vb, total, k, w, N, nrhs);
    col_dots_finish_kernel<<<ceil_div(k * nrhs, 256), 256, 0, c->stream>>>(dots, part, P, k, nrhs);
    c->launches += 2;
    RMAT_CU(cudaGetLastError());
    hbuf.resize((size_t)k * nrhs);
    RMAT_CU(cudaMemcpyAsync(hbuf.data(), dots, (size_t)k * nrhs * sizeof(double2),
                            cudaMemcpyDeviceToHost, c->stream));
    RMAT_CU(cudaStreamSynchronize(c->stream));
    return RMAT_OK;
  }
  int axpy(double2* w, const double2* Vb, int k, const std::vector<double2>& h) {
    RMAT_CU(cudaMemcpyAsync(hd, h.data(), (size_t)k * nrhs * sizeof(double2),
                            cudaMemcpyHostToDevice, c->stream));
    col_axpy_kernel<<<grid_of(c, total), 256, 0, c->stream>>>(w, Vb, total, k, hd, N, nrhs);
    c->launches++;
    RMAT_CU(cudaGetLastError());
    return RMAT_OK;
  }
  int scale(double2* v, const double2* w, const std::vector<double>& s) {
    RMAT_CU(cudaMemcpyAsync(sd, s.data(), nrhs * sizeof(double), cudaMemcpyHostToDevice,
                            c->stream));
    col_scale_kernel<<<grid_of(c, total), 256, 0, c->stream>>>(v, w, sd, N, nrhs);
    c->launches++;
    RMAT_CU(cudaGetLastError());
    return RMAT_OK;
  }
  // z = M^-1 v through the factors (Bw in the factor precision, D-scaled)
  int precond(double2* z, const double2* v) {
    const double* D = c->equil ? c->Dsc : nullptr;
    if (c->precision == RMAT_C128)
      to_bw_kernel<double><<<grid_of(c, total), 256, 0, c->stream>>>(
          reinterpret_cast<double2*>(c->Bw), v, total, nrhs, D);
    else
      to_bw_kernel<float><<<grid_of(c, total), 256, 0, c->stream>>>(
          reinterpret_cast<float2*>(c->Bw), v, total, nrhs, D);
    c->launches++;
    RMAT_CU(cudaGetLastError());
    RMAT_CHECK(rmat_solve_system(c));
    if (c->precision == RMAT_C128)
      from_bw_kernel<double><<<grid_of(c, total), 256, 0, c->stream>>>(
          z, reinterpret_cast<const double2*>(c->Bw), total, nrhs, D);
    else
      from_bw_kernel<float><<<grid_of(c, total), 256, 0, c->stream>>>(
          z, reinterpret_cast<const float2*>(c->Bw), total, nrhs, D);
    c->launches++;
    RMAT_CU(cudaGetLastError());
    return RMAT_OK;
  }
  // w = C z (FP64): t = Phi - C z, w = Phi - t
  int apply(double2* w, const double2* z) {
    RMAT_CHECK(launch_apply_resid(c, z, T));
    phi_minus_kernel<<<grid_of(c, total), 256, 0, c->stream>>>(
        w, T, total, nrhs, c->nlag, c->fa, c->sector ? c->faL : nullptr, c->nch,
        c->kind == 2 ? c->B64 : nullptr);
    c->launches++;
    RMAT_CU(cudaGetLastError());
    return RMAT_OK;
  }
};

}  // namespace

// One FGMRES correction of c->X for the residual r held in c->Rres (FP64):
// X += d with C d ~= r.  Returns the number of inner steps in *inner.
int gmres_correction(rmat_ctx c, int m, double tau, int* inner) {
  Gmres g;
  g.c = c;
  g.N = c->N;
  g.nrhs = c->nrhs;
  g.m = m;
  g.total = (size_t)g.N * g.nrhs;
  const int nrhs = g.nrhs;
  const int P = std::max(1, std::min(GM_PARTS, ceil_div(g.N, GM_ROWS)));
  const size_t vec = g.total * sizeof(double2);
  RMAT_CHECK(rmat_grow(c, &c->gm_V, &c->gm_V_cap, (size_t)(m + 1) * vec));
  RMAT_CHECK(rmat_grow(c, &c->gm_Z, &c->gm_Z_cap, (size_t)m * vec));
  RMAT_CHECK(rmat_grow(c, &c->gm_T, &c->gm_T_cap, vec));
  RMAT_CHECK(rmat_grow(c, &c->gm_small, &c->gm_small_cap,
                       ((size_t)P * (m + 2) * nrhs + 2 * (size_t)(m + 2) * nrhs) * sizeof(double2) +
                           nrhs * sizeof(double)));
  g.V = reinterpret_cast<double2*>(c->gm_V);
  g.Z = reinterpret_cast<double2*>(c->gm_Z);
  g.T = reinterpret_cast<double2*>(c->gm_T);
  g.part = reinterpret_cast<double2*>(c->gm_small);
  g.dots = g.part + (size_t)P * (m + 2) * nrhs;
  g.hd = g.dots + (size_t)(m + 2) * nrhs;
  g.sd = reinterpret_cast<double*>(g.hd + (size_t)(m + 2) * nrhs);

  // beta = ||r|| per column, v_0 = r / beta
  RMAT_CHECK(g.col_dots(c->Rres, 1, c->Rres));
  std::vector<double> beta(nrhs), s(nrhs);
  for (int q = 0; q < nrhs; ++q) {
    beta[q] = std::sqrt(std::max(0.0, g.hbuf[q].x));
    s[q] = beta[q] > 0.0 ? 1.0 / beta[q] : 0.0;
  }
  RMAT_CHECK(g.scale(g.V, c->Rres, s));
  // per column: H (m+1) x m column-major, Givens (cs real, sn complex), g
  std::vector<cd> H((size_t)nrhs * (m + 1) * m, cd(0)), sn((size_t)nrhs * m), gv((size_t)nrhs * (m + 1));
  std::vector<double> cs((size_t)nrhs * m);
  for (int q = 0; q < nrhs; ++q) gv[(size_t)q * (m + 1)] = beta[q];
  auto Hq = [&](int q, int i, int k) -> cd& { return H[((size_t)q * m + k) * (m + 1) + i]; };
  int k_used = 0;
  std::vector<double2> h1, h2;
  for (int k = 0; k < m; ++k) {
    double2* vk = g.V + (size_t)k * g.total;
    double2* zk = g.Z + (size_t)k * g.total;
    double2* w = g.V + (size_t)(k + 1) * g.total;
    RMAT_CHECK(g.precond(zk, vk));
    RMAT_CHECK(g.apply(w, zk));
    // classical Gram-Schmidt, twice
    RMAT_CHECK(g.col_dots(g.V, k + 1, w));
    h1 = g.hbuf;
    RMAT_CHECK(g.axpy(w, g.V, k + 1, h1));
    RMAT_CHECK(g.col_dots(g.V, k + 1, w));
    h2 = g.hbuf;
    RMAT_CHECK(g.axpy(w, g.V, k + 1, h2));
    RMAT_CHECK(g.col_dots(w, 1, w));
    double worst = 0.0;
    for (int q = 0; q < nrhs; ++q) {
      for (int j = 0; j <= k; ++j) {
        const size_t e = (size_t)j * nrhs + q;
        Hq(q, j, k) = cd(h1[e].x + h2[e].x, h1[e].y + h2[e].y);
      }
      const double hn = std::sqrt(std::max(0.0, g.hbuf[q].x));
      Hq(q, k + 1, k) = hn;
      s[q] = hn > 0.0 ? 1.0 / hn : 0.0;
      // previous rotations on column k, then the new one
      for (int j = 0; j < k; ++j) {
        const double cj = cs[(size_t)q * m + j];
        const cd sj = sn[(size_t)q * m + j];
        const cd a = Hq(q, j, k), b = Hq(q, j + 1, k);
        Hq(q, j, k) = cj * a + sj * b;
        Hq(q, j + 1, k) = -std::conj(sj) * a + cj * b;
      }
      const cd a = Hq(q, k, k), b = Hq(q, k + 1, k);
      const double t = std::sqrt(std::norm(a) + std::norm(b));
      double ck;
      cd sk;
      if (t == 0.0) {
        ck = 1.0;
        sk = 0.0;
      } else if (std::abs(a) == 0.0) {
        ck = 0.0;
        sk = std::conj(b) / std::abs(b);
      } else {
        ck = std::abs(a) / t;
        sk = (a / std::abs(a)) * std::conj(b) / t;
      }
      cs[(size_t)q * m + k] = ck;
      sn[(size_t)q * m + k] = sk;
      Hq(q, k, k) = ck * a + sk * b;
      Hq(q, k + 1, k) = 0.0;
      cd& gk = gv[(size_t)q * (m + 1) + k];
      gv[(size_t)q * (m + 1) + k + 1] = -std::conj(sk) * gk;
      gk = ck * gk;
      if (beta[q] > 0.0)
        worst = std::max(worst, std::abs(gv[(size_t)q * (m + 1) + k + 1]) / beta[q]);
    }
    k_used = k + 1;
    if (worst < tau || k + 1 == m) break;
    RMAT_CHECK(g.scale(w, w, s));  // v_{k+1}
  }
  // y = R^-1 g per column, X += sum_k y_k z_k
  std::vector<double2> y((size_t)k_used * nrhs);
  for (int q = 0; q < nrhs; ++q) {
    std::vector<cd> yq(k_used);
    for (int i = k_used - 1; i >= 0; --i) {
      cd acc = gv[(size_t)q * (m + 1) + i];
      for (int j = i + 1; j < k_used; ++j) acc -= Hq(q, i, j) * yq[j];
      const cd d = Hq(q, i, i);
      yq[i] = std::abs(d) > 0.0 ? acc / d : cd(0);
    }
    for (int i = 0; i < k_used; ++i) y[(size_t)i * nrhs + q] = make_double2(yq[i].real(), yq[i].imag());
  }
  RMAT_CU(cudaMemcpyAsync(g.hd, y.data(), y.size() * sizeof(double2), cudaMemcpyHostToDevice,
                          c->stream));
  col_combine_kernel<<<grid_of(c, g.total), 256, 0, c->stream>>>(c->X, g.Z, g.total, k_used, g.hd,
                                                                 g.N, nrhs);
  c->launches++;
  RMAT_CU(cudaGetLastError());
  RMAT_CU(cudaStreamSynchronize(c->stream));
  if (inner) *inner = k_used;
  return RMAT_OK;
}
