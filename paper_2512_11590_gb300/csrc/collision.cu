// G9/G10: R-matrix contraction and collision matrix (FP64, on the device).
//
// R (Sec. 3.1 step 4): R_{al be} = sum_i q2(r_i) X[(al,i), be] with q2 = f_i(a);
// with C in MeV the dimensionless R-matrix carries hm/a:
//   R = (hm/a) Phi^T X.
// U: matching to the free asymptotic solutions at the channel radius (Sec. 1,
// Coulomb/Whittaker functions of Sec. 4.1):
//   R~ = a sqrt(k) R sqrt(k),
//   U  = (diag O - R~ diag O')^-1 (diag I - R~ diag I'),  open x open block,
// I = G - iF, O = G + iF (Coulomb functions; Riccati-Bessel F = rho j_l,
// G = -rho y_l for eta = 0) for open channels; O = Whittaker function (or, for
// eta > 0, O = 1 and O' = W'/W), I = 0 for closed ones (special.cuh).  The
// matching system (nch x nch, nopen right-hand sides) is solved with this
// library's FP64 LU.
#include <algorithm>

#include "cplx.cuh"
#include "rmat_internal.h"
#include "special.cuh"

namespace {

__global__ void r_contract_kernel(const double2* __restrict__ X, int nch, int nlag, int nrhs,
                                  const double* __restrict__ fa, double scale,
                                  double2* __restrict__ Rint, double2* __restrict__ Rout) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nch * nch) return;
  const int al = e / nch, be = e % nch;
  double sr = 0.0, si = 0.0;
  for (int i = 0; i < nlag; ++i) {
    const double2 x = X[((size_t)al * nlag + i) * nrhs + be];
    sr = fma(fa[i], x.x, sr);
    si = fma(fa[i], x.y, si);
  }
  const double2 r = make_double2(scale * sr, scale * si);
  Rint[(size_t)al * nch + be] = r;
  if (Rout) Rout[al + (size_t)nch * be] = r;
}

struct ChanFn {
  double2 I, O, dI, dO;
  double k;
};

// One thread per channel; a channel function that does not converge sets
// status (1 + channel) and the host reports RMAT_ECHANFN.
__global__ void chan_fn_kernel(ChanFn* __restrict__ out, int nch, const int* __restrict__ l,
                               const double* __restrict__ th, const double* __restrict__ zz,
                               double E, double hm, double a, double B, int* __restrict__ status) {
  const int ch = blockIdx.x * blockDim.x + threadIdx.x;
  if (ch >= nch) return;
  ChanFn f;
  if (!channel_functions(l[ch], E - th[ch], hm, a, B, zz[ch], &f.I, &f.O, &f.dI, &f.dO, &f.k))
    *status = 1 + ch;
  out[ch] = f;
}

// ZO (nch x nch) and ZI (nch x nopen), row-major, from R and the channel functions.
__global__ void z_build_kernel(const double2* __restrict__ Rint, const ChanFn* __restrict__ f,
                               int nch, int nopen, const int* __restrict__ open, double a,
                               double2* __restrict__ ZO, double2* __restrict__ ZI) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  const int ncol = nch + nopen;
  if (e >= nch * ncol) return;
  const int row = e / ncol, col = e % ncol;
  const int cp = col < nch ? col : open[col - nch];
  const double2 R = Rint[(size_t)row * nch + cp];
  const double s = a * sqrt(f[row].k) * sqrt(f[cp].k);
  const double2 Rt = make_double2(s * R.x, s * R.y);
  if (col < nch) {
    double2 z = cmul<double>(Rt, f[cp].dO);
    z.x = -z.x;
    z.y = -z.y;
    if (row == cp) { z.x += f[row].O.x; z.y += f[row].O.y; }
    ZO[(size_t)row * nch + col] = z;
  } else {
    double2 z = cmul<double>(Rt, f[cp].dI);
    z.x = -z.x;
    z.y = -z.y;
    if (row == cp) { z.x += f[row].I.x; z.y += f[row].I.y; }
    ZI[(size_t)row * nopen + (col - nch)] = z;
  }
}

__global__ void u_extract_kernel(const double2* __restrict__ Ufull, int nopen,
                                 const int* __restrict__ open, double2* __restrict__ U) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nopen * nopen) return;
  const int q = e % nopen, q2 = e / nopen;  // U(q, q2), column-major
  U[e] = Ufull[(size_t)open[q] * nopen + q2];
}

}  // namespace

int launch_collision(rmat_ctx c, double2* R_dev, double2* U_dev, int nopen) {
  const int nch = c->nch;
  r_contract_kernel<<<ceil_div(nch * nch, 128), 128, 0, c->stream>>>(
      c->X, nch, c->nlag, c->nrhs, c->fa, c->hm / c->a, c->Rint, R_dev);
  c->launches++;
  RMAT_CU(cudaGetLastError());
  return launch_u_from_rint(c, U_dev, nopen);
}

int launch_u_from_rint(rmat_ctx c, double2* U_dev, int nopen) {
  const int nch = c->nch;
  if (!U_dev || nopen == 0) return RMAT_OK;
  ChanFn* fn = reinterpret_cast<ChanFn*>(c->Zbuf);
  double2* ZO = reinterpret_cast<double2*>(reinterpret_cast<char*>(c->Zbuf) +
                                           round_up(sizeof(ChanFn) * nch, 256));
  double2* ZI = ZO + (size_t)nch * nch;
  chan_fn_kernel<<<ceil_div(nch, 64), 64, 0, c->stream>>>(fn, nch, c->l_d, c->th_d, c->zz_d, c->E,
                                                           c->hm, c->a, c->bloch_B,
                                                           c->dstat + ST_CHANFN);
  z_build_kernel<<<ceil_div((long long)nch * (nch + nopen), 128), 128, 0, c->stream>>>(
      c->Rint, fn, nch, nopen, c->open_d, c->a, ZO, ZI);
  c->launches += 2;
  RMAT_CU(cudaGetLastError());
  const long long tl = c->tu_launches;
  const double tf = c->tu_flops;
  const size_t tev = c->tu_events.size();
  const int nb = std::min(64, nch);
  RMAT_CHECK(perm_reserve(c, c->perm_z, nch, nb));
  RMAT_CHECK(lu_factor_dev<double>(c, ZO, nch, nch, c->zpiv, nb, false, c->perm_z));
  RMAT_CHECK(lu_solve_dev<double>(c, ZO, nch, nch, c->perm_z, nb, ZI, nopen, nopen));
  c->tu_launches = tl;
  c->tu_flops = tf;
  c->tu_events.resize(tev);
  u_extract_kernel<<<ceil_div(nopen * nopen, 128), 128, 0, c->stream>>>(ZI, nopen, c->open_d, U_dev);
  c->launches++;
  RMAT_CU(cudaGetLastError());
  return RMAT_OK;
}

namespace {

// G[q][al][be] = hm sum_i f_q(i) X[(al, i), col_q(be)]: q = 0 RR (f_R, columns 0..nch),
// 1 RL (f_R, columns nch..2nch), 2 LR (f_L, columns 0..nch), 3 LL (f_L, nch..2nch).
__global__ void sector_g_kernel(double2* __restrict__ G, const double2* __restrict__ X, int nch,
                                int nlag, int nrhs, const double* __restrict__ fR,
                                const double* __restrict__ fL, double hm, int nblocks) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nblocks * nch * nch) return;
  const int q = e / (nch * nch), al = (e / nch) % nch, be = e % nch;
  const double* f = q < 2 ? fR : fL;
  const int col = (q & 1) ? nch + be : be;
  double sr = 0.0, si = 0.0;
  for (int i = 0; i < nlag; ++i) {
    const double2 x = X[((size_t)al * nlag + i) * nrhs + col];
    sr = fma(f[i], x.x, sr);
    si = fma(f[i], x.y, si);
  }
  G[e] = make_double2(hm * sr, hm * si);
}

}  // namespace

int launch_sector_g(rmat_ctx c, double2* G) {
  const int nch = c->nch, nb = c->sector ? 4 : 1;
  sector_g_kernel<<<ceil_div(nb * nch * nch, 128), 128, 0, c->stream>>>(
      G, c->X, nch, c->nlag, c->nrhs, c->fa, c->sector ? c->faL : nullptr, c->hm, nb);
  c->launches++;
  RMAT_CU(cudaGetLastError());
  return RMAT_OK;
}

namespace {

__global__ void prop_add_kernel(double2* __restrict__ P, const double2* __restrict__ A,
                                const double2* __restrict__ B, int n) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n) P[e] = make_double2(A[e].x + B[e].x, A[e].y + B[e].y);
}

// Rint = Rl / a (row-major) and, when requested, Rout column-major
__global__ void prop_finish_kernel(double2* __restrict__ Rint, double2* __restrict__ Rout,
                                   const double2* __restrict__ Rl, int nch, double inv_a) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nch * nch) return;
  const double2 r = make_double2(Rl[e].x * inv_a, Rl[e].y * inv_a);
  Rint[e] = r;
  if (Rout) Rout[(e / nch) + (size_t)nch * (e % nch)] = r;
}

}  // namespace

// One propagation step: Rl <- g_RR - g_RL (Rl + g_LL)^-1 g_LR (G = RR, RL, LR, LL).
int launch_prop_step(rmat_ctx c, double2* Rl, double2* G, double2* P) {
  const int nch = c->nch, n = nch * nch;
  const size_t blk = (size_t)n;
  double2 *gRR = G, *gRL = G + blk, *gLR = G + 2 * blk, *gLL = G + 3 * blk;
  prop_add_kernel<<<ceil_div(n, 128), 128, 0, c->stream>>>(P, Rl, gLL, n);
  c->launches++;
  RMAT_CU(cudaGetLastError());
  const long long tl = c->tu_launches;
  const double tf = c->tu_flops;
  const size_t tev = c->tu_events.size();
  const int nb = std::min(64, nch);
  RMAT_CHECK(perm_reserve(c, c->perm_z, nch, nb));
  RMAT_CHECK(lu_factor_dev<double>(c, P, nch, nch, c->zpiv, nb, false, c->perm_z));
  RMAT_CHECK(lu_solve_dev<double>(c, P, nch, nch, c->perm_z, nb, gLR, nch, nch));  // Y in gLR
  RMAT_CHECK(gemm_sub_c128(c, nch, nch, nch, gRL, nch, gLR, nch, gRR, nch));   // gRR -= gRL Y
  c->tu_launches = tl;
  c->tu_flops = tf;
  c->tu_events.resize(tev);
  RMAT_CU(cudaMemcpyAsync(Rl, gRR, blk * sizeof(double2), cudaMemcpyDeviceToDevice, c->stream));
  return RMAT_OK;
}

int launch_prop_finish(rmat_ctx c, const double2* Rl, double2* Rout) {
  const int nch = c->nch;
  prop_finish_kernel<<<ceil_div(nch * nch, 128), 128, 0, c->stream>>>(c->Rint, Rout, Rl, nch,
                                                                       1.0 / c->a);
  c->launches++;
  RMAT_CU(cudaGetLastError());
  return RMAT_OK;
}

size_t collision_workspace_bytes(int nch) {
  return round_up(sizeof(ChanFn) * nch, 256) + (size_t)nch * 2 * nch * sizeof(double2);
}
