// G1: assembly of the internal-region matrix C = T + L(B) + V - E*I on the device.
//
// Block structure of Eq. (block_structure) in Sec. 2: diagonal channel blocks
// K_alpha + D_alpha,alpha (full nlag x nlag kinetic + Bloch matrix plus the
// diagonal potential, centrifugal term, threshold and -E), off-diagonal blocks
// D_alpha,alpha' = diag(V_alpha,alpha'(r_i)) (local potentials).  Row-major
// storage; every entry of the N x ld matrix is written (HBM write-bound:
// 8 N ld bytes in complex64, 16 N ld in complex128; the few nonzeros that share
// a 16-byte chunk with zeros are written twice).
//
// Entries are formed in FP64 with explicitly rounded operations in this order:
//   K_ij     = hm*T0_ij - (hm*(B/a)) * (f_i*f_j)            (host table Kmat)
//   d_al,i   = (hm * (l(l+1))) / (r_i*r_i) + (E_al - E)
//   C_ii(re) = K_ii + (d_al,i + Re V_alal(r_i)),  C_ii(im) = Im V_alal(r_i)
// then rounded once to the storage type.
#include "cplx.cuh"
#include "rmat_internal.h"

namespace {

__device__ __forceinline__ double chan_diag(double hm, int l, double ri, double th, double E) {
  const double ll = (double)l;
  const double ll1 = __dmul_rn(ll, __dadd_rn(ll, 1.0));
  return __dadd_rn(__ddiv_rn(__dmul_rn(hm, ll1), __dmul_rn(ri, ri)), __dsub_rn(th, E));
}

// One warp per row.  The row is mostly structural zeros (all but the nlag
// same-channel columns and one column per other channel), so the warp first
// clears it with 16-byte stores, skipping the chunks that lie inside the
// same-channel block, and after __syncwarp writes the nonzeros: the
// same-channel block (contiguous, lane-strided) and the nch-1 entries
// (al', i) of the local couplings.  __syncwarp orders the two passes, so a
// nonzero that shares a 16-byte chunk with cleared columns is written last.
template <class T>
__global__ void __launch_bounds__(256)
assemble_kernel(cplx<T>* __restrict__ C, int ld, int N, int nch, int nlag,
                const double* __restrict__ K, const double* __restrict__ r,
                const int* __restrict__ l, const double* __restrict__ th,
                const double2* __restrict__ V, double hm, double E,
                const double* __restrict__ D) {
  constexpr int CPC = 16 / (int)sizeof(cplx<T>);  // complex entries per 16-byte chunk
  const int lane = threadIdx.x & 31;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int row = gw; row < N; row += nw) {
    const int al = row / nlag, i = row - al * nlag;
    const double d = chan_diag(hm, l[al], r[i], th[al], E);
    const double drow = D ? D[row] : 1.0;
    cplx<T>* Crow = C + (size_t)row * ld;
    const int b0 = al * nlag, b1 = b0 + nlag;  // same-channel columns [b0, b1)
    if ((reinterpret_cast<uintptr_t>(Crow) & 15) == 0 && ld % CPC == 0) {
      uint4* C4 = reinterpret_cast<uint4*>(Crow);
      const int nq = ld / CPC;
      const uint4 z = make_uint4(0u, 0u, 0u, 0u);
#pragma unroll 4
      for (int q = lane; q < nq; q += 32) {
        const int c0 = q * CPC;
        if (c0 >= b0 && c0 + CPC <= b1) continue;
        C4[q] = z;
      }
    } else {
      for (int col = lane; col < ld; col += 32)
        if (col < b0 || col >= b1) Crow[col] = mkc<T>((T)0, (T)0);
    }
    __syncwarp();
    for (int j = lane; j < nlag; j += 32) {  // same-channel block K_al + D_al,al
      double re = K[i * nlag + j], im = 0.0;
      if (j == i) {
        const double2 v = V[i + (size_t)nlag * (al + (size_t)nch * al)];
        re = __dadd_rn(re, __dadd_rn(d, v.x));
        im = v.y;
      }
      if (D) {
        const double sc = drow * D[b0 + j];
        re *= sc;
        im *= sc;
      }
      Crow[b0 + j] = mkc<T>((T)re, (T)im);
    }
    for (int alp = lane; alp < nch; alp += 32) {  // D_al,al' = diag(V_al,al'(r_i))
      if (alp == al) continue;
      const double2 v = V[i + (size_t)nlag * (al + (size_t)nch * alp)];
      double re = v.x, im = v.y;
      const int col = alp * nlag + i;
      if (D) {
        const double sc = drow * D[col];
        re *= sc;
        im *= sc;
      }
      Crow[col] = mkc<T>((T)re, (T)im);
    }
  }
}

// Symmetric equilibration D_(al,i) = |C_(al,i),(al,i)|^-1/2 (1 when the diagonal is 0).
__global__ void diag_scale_kernel(double* __restrict__ D, int N, int nch, int nlag,
                                  const double* __restrict__ K, const double* __restrict__ r,
                                  const int* __restrict__ l, const double* __restrict__ th,
                                  const double2* __restrict__ V, double hm, double E) {
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= N) return;
  const int al = row / nlag, i = row - al * nlag;
  const double2 v = V[i + (size_t)nlag * (al + (size_t)nch * al)];
  const double re = K[i * nlag + i] + chan_diag(hm, l[al], r[i], th[al], E) + v.x;
  const double m = hypot(re, v.y);
  D[row] = m > 0.0 ? 1.0 / sqrt(m) : 1.0;
}

// Full coupling matrix at each mesh point for the structured FP64 residual:
// W[i][al][al'] = V_al,al'(r_i) + delta_al,al' d_al,i.
__global__ void point_coupling_kernel(double2* __restrict__ W, int nch, int nlag,
                                      const double* __restrict__ r, const int* __restrict__ l,
                                      const double* __restrict__ th,
                                      const double2* __restrict__ V, double hm, double E) {
  const size_t total = (size_t)nlag * nch * nch;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    const int alp = (int)(e % nch);
    const int al = (int)((e / nch) % nch);
    const int i = (int)(e / ((size_t)nch * nch));
    double2 v = V[i + (size_t)nlag * (al + (size_t)nch * alp)];
    if (al == alp) v.x = __dadd_rn(chan_diag(hm, l[al], r[i], th[al], E), v.x);
    W[e] = v;
  }
}

// Dense system: column-major complex128 A (lda) -> row-major working copy in T
// and row-major complex128 copy for the residual; B (ldb) -> row-major B64.
template <class T>
__global__ void load_dense_kernel(cplx<T>* __restrict__ C, int ld, double2* __restrict__ A64,
                                  int n, const double2* __restrict__ A, int lda) {
  __shared__ double2 tile[32][33];
  const int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int k = ty; k < 32; k += 8) {  // read column c0+k, rows r0+tx (coalesced)
    const int rr = r0 + tx, cc = c0 + k;
    tile[k][tx] = (rr < n && cc < n) ? A[rr + (size_t)lda * cc] : make_double2(0, 0);
  }
  __syncthreads();
  for (int k = ty; k < 32; k += 8) {  // write row r0+k, columns c0+tx
    const int rr = r0 + k, cc = c0 + tx;
    if (rr < n && cc < ld) {
      const double2 z = (cc < n) ? tile[tx][k] : make_double2(0, 0);
      C[(size_t)rr * ld + cc] = mkc<T>((T)z.x, (T)z.y);
      if (cc < n) A64[(size_t)rr * n + cc] = z;
    }
  }
}

__global__ void load_rhs_kernel(double2* __restrict__ B64, int n, int nrhs,
                                const double2* __restrict__ B, int ldb) {
  const size_t total = (size_t)n * nrhs;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    const int row = (int)(e / nrhs), col = (int)(e % nrhs);
    B64[e] = B[row + (size_t)ldb * col];
  }
}

}  // namespace

int launch_assemble(rmat_ctx c, const double2* V, double E) {
  const int blocks = std::max(1, std::min(c->sm_count * 8, ceil_div((long long)c->N * 32, 256)));
  const double* D = c->equil ? c->Dsc : nullptr;
  if (D) {
    diag_scale_kernel<<<ceil_div(c->N, 256), 256, 0, c->stream>>>(
        c->Dsc, c->N, c->nch, c->nlag, c->Kmat, c->rmesh, c->l_d, c->th_d, V, c->hm, E);
    c->launches++;
  }
  if (c->precision == RMAT_C128) {
    assemble_kernel<double><<<blocks, 256, 0, c->stream>>>(
        reinterpret_cast<double2*>(c->C), c->ld, c->N, c->nch, c->nlag, c->Kmat, c->rmesh, c->l_d,
        c->th_d, V, c->hm, E, D);
  } else {
    assemble_kernel<float><<<blocks, 256, 0, c->stream>>>(
        reinterpret_cast<float2*>(c->C), c->ld, c->N, c->nch, c->nlag, c->Kmat, c->rmesh, c->l_d,
        c->th_d, V, c->hm, E, D);
  }
  c->launches++;
  RMAT_CU(cudaGetLastError());
  return RMAT_OK;
}

int launch_point_coupling(rmat_ctx c, const double2* V, double E) {
  const size_t total = (size_t)c->nlag * c->nch * c->nch;
  const int blocks = std::max(1, std::min(c->sm_count * 8, ceil_div((long long)total, 256)));
  point_coupling_kernel<<<blocks, 256, 0, c->stream>>>(c->Wpt, c->nch, c->nlag, c->rmesh, c->l_d,
                                                       c->th_d, V, c->hm, E);
  c->launches++;
  c->wpt_gen++;  // digit planes of the tensor-core residual are rebuilt from the new table
  RMAT_CU(cudaGetLastError());
  return RMAT_OK;
}

int launch_load_dense(rmat_ctx c, const double2* A, int lda, const double2* B, int ldb) {
  dim3 grid(ceil_div(c->ld, 32), ceil_div(c->N, 32));
  if (c->precision == RMAT_C128)
    load_dense_kernel<double><<<grid, 256, 0, c->stream>>>(reinterpret_cast<double2*>(c->C), c->ld,
                                                           c->A64, c->N, A, lda);
  else
    load_dense_kernel<float><<<grid, 256, 0, c->stream>>>(reinterpret_cast<float2*>(c->C), c->ld,
                                                          c->A64, c->N, A, lda);
  const size_t total = (size_t)c->N * c->nrhs;
  load_rhs_kernel<<<std::max(1, std::min(c->sm_count * 4, ceil_div((long long)total, 256))), 256, 0,
                    c->stream>>>(c->B64, c->N, c->nrhs, B, ldb);
  c->launches += 2;
  RMAT_CU(cudaGetLastError());
  return RMAT_OK;
}
