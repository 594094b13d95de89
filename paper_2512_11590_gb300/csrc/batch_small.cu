// a11: the small systems of a batch in ONE persistent launch.
//
// Every CTA of a persistent grid takes the next system from a device work counter
// and runs that system's whole hot path on its own SM, the matrix held in shared
// memory (N = nch * nlag up to 160 in complex64, 112 in complex128):
//   * assembly of C = T + L(B) + V - E (Eq. block_structure, Sec. 2) straight into
//     shared memory, in the factor precision;
//   * LU with partial pivoting (largest |Re| + |Im| in the column, first row on ties;
//     Sec. 3.1), right-looking, one column at a time;
//   * forward / backward substitution for the nch surface right-hand sides, one warp
//     per right-hand-side column (no block-wide barrier in the sweeps);
//   * FP64 refinement (Sec. 3.2): r = Phi - C X formed in FP64 from the block
//     structure (kinetic table, centrifugal + threshold - E, the point couplings V),
//     the stopping rule of rmat_solve (tol, FP64 floor + one final correction,
//     stagnation, max_refine), X += C^-1 r with the shared-memory factors;
//   * R and U of the system (collision_cta.cuh).
// Status words and refinement counts go to the batch's per-system arrays, exactly as
// the lane path writes them.  The systems are ordered largest first on the host.
#include <cmath>

#include "collision_cta.cuh"
#include "cplx.cuh"
#include "rmat_internal.h"

namespace {

constexpr int SB_THREADS = 256;

template <class T>
__global__ void __launch_bounds__(SB_THREADS, 1)
batch_small_kernel(const SmallSys* __restrict__ sys, int nsmall, int* __restrict__ next,
                   int max_refine, double tol, int need, int patience, int* __restrict__ st_all,
                   IrState* __restrict__ ir_all, SmallScratch scr) {
  using C2 = cplx<T>;
  extern __shared__ unsigned char smem_raw[];
  __shared__ int s_sys, s_piv, s_info;
  __shared__ double s_red[32];
  __shared__ NoallocParams s_p;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  double2* Xg = scr.X + (size_t)blockIdx.x * scr.slot;   // FP64 solution, row-major N x nch
  double2* Rg = scr.R + (size_t)blockIdx.x * scr.slot;   // FP64 residual
  NoallocScratch* S = reinterpret_cast<NoallocScratch*>(scr.coll) + blockIdx.x;

  // block-wide maximum of a non-negative double (all threads call)
  auto block_max = [&](double m) -> double {
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    __syncthreads();
    if (lane == 0) s_red[warp] = m;
    __syncthreads();
    double t = 0.0;
    for (int w = 0; w < SB_THREADS / 32; ++w) t = fmax(t, s_red[w]);
    return t;
  };

  for (;;) {
    if (tid == 0) s_sys = atomicAdd(next, 1);
    __syncthreads();
    const int k = s_sys;
    if (k >= nsmall) break;
    const SmallSys y = sys[k];
    const int N = y.N, nch = y.nch, nlag = y.nlag, ldc = N | 1;
    C2* C = reinterpret_cast<C2*>(smem_raw);                 // [N][ldc]
    C2* Bw = C + (size_t)N * ldc;                              // [N][nch]
    int* piv = reinterpret_cast<int*>(Bw + (size_t)N * nch);  // [N]
    // ---- assembly (FP64 values rounded once to T) ----
    for (int e = tid; e < N * N; e += SB_THREADS) {
      const int r = e / N, c = e - r * N;
      const int al = r / nlag, i = r - al * nlag, al2 = c / nlag, j = c - al2 * nlag;
      double2 v = make_double2(0.0, 0.0);
      if (al == al2) {
        v.x = y.K[i * nlag + j];
        if (i == j) {
          const double rr = y.r[i];
          const double2 w = y.V[i + (size_t)nlag * (al + (size_t)nch * al)];
          const int l = y.l[al];
          v.x += y.hm * l * (l + 1.0) / (rr * rr) + y.th[al] - y.E + w.x;
          v.y += w.y;
        }
      } else if (i == j) {
        v = y.V[i + (size_t)nlag * (al + (size_t)nch * al2)];
      }
      C[(size_t)r * ldc + c] = to_c(v, T());
    }
    if (tid == 0) s_info = 0;
    __syncthreads();
    // ---- LU with partial pivoting ----
    for (int j = 0; j < N; ++j) {
      if (warp == 0) {
        T best = (T)-1;
        int bi = N;
        for (int r = j + lane; r < N; r += 32) {
          const T m = cabs1<T>(C[(size_t)r * ldc + j]);
          if (m > best) { best = m; bi = r; }
        }
        for (int o = 16; o > 0; o >>= 1) {
          const T ob = __shfl_xor_sync(0xffffffffu, best, o);
          const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
          if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
        }
        if (lane == 0) {
          s_piv = bi < N ? bi : j;
          if (!(best > (T)0) && s_info == 0) s_info = j + 1;
        }
      }
      __syncthreads();
      const int p = s_piv;
      if (tid == 0) piv[j] = p;
      if (p != j)
        for (int c = tid; c < N; c += SB_THREADS) {
          const C2 t = C[(size_t)j * ldc + c];
          C[(size_t)j * ldc + c] = C[(size_t)p * ldc + c];
          C[(size_t)p * ldc + c] = t;
        }
      __syncthreads();
      const C2 pv = C[(size_t)j * ldc + j];
      if (pv.x != (T)0 || pv.y != (T)0) {  // the same value in every thread
        for (int r = j + 1 + tid; r < N; r += SB_THREADS)
          C[(size_t)r * ldc + j] = cdiv<T>(C[(size_t)r * ldc + j], pv);
        __syncthreads();
        const int m = N - j - 1;
        for (int e = tid; e < m * m; e += SB_THREADS) {
          const int r = j + 1 + e / m, c = j + 1 + e % m;
          csub_mul<T>(C[(size_t)r * ldc + c], C[(size_t)r * ldc + j], C[(size_t)j * ldc + c]);
        }
      }
      __syncthreads();
    }
    // ---- first right-hand sides: Phi[(al,i), be] = delta_{al be} f_i(a) ----
    for (int e = tid; e < N * nch; e += SB_THREADS) {
      const int r = e / nch, be = e - r * nch, al = r / nlag;
      Bw[e] = to_c(make_double2(al == be ? y.fa[r - al * nlag] : 0.0, 0.0), T());
    }
    __syncthreads();
    // solve with the factors, one warp per right-hand-side column, in place in Bw
    auto solve = [&]() {
      for (int be = warp; be < nch; be += SB_THREADS / 32) {
        for (int j = 0; j < N; ++j) {  // interchanges in order
          const int p = piv[j];
          if (p != j && lane == 0) {
            const C2 t = Bw[(size_t)j * nch + be];
            Bw[(size_t)j * nch + be] = Bw[(size_t)p * nch + be];
            Bw[(size_t)p * nch + be] = t;
          }
        }
        __syncwarp();
        for (int j = 0; j < N; ++j) {  // L, unit diagonal
          const C2 yj = Bw[(size_t)j * nch + be];
          for (int r = j + 1 + lane; r < N; r += 32)
            csub_mul<T>(Bw[(size_t)r * nch + be], C[(size_t)r * ldc + j], yj);
          __syncwarp();
        }
        for (int j = N - 1; j >= 0; --j) {  // U
          if (lane == 0) Bw[(size_t)j * nch + be] = cdiv<T>(Bw[(size_t)j * nch + be], C[(size_t)j * ldc + j]);
          __syncwarp();
          const C2 yj = Bw[(size_t)j * nch + be];
          for (int r = lane; r < j; r += 32)
            csub_mul<T>(Bw[(size_t)r * nch + be], C[(size_t)r * ldc + j], yj);
          __syncwarp();
        }
      }
      __syncthreads();
    };
    solve();
    for (int e = tid; e < N * nch; e += SB_THREADS) Xg[e] = to_d(Bw[e]);
    __syncthreads();
    // |C||X| of the first solution (scale of the FP64 floor) and the residual
    auto residual = [&](bool absval) -> double {
      double m = 0.0;
      for (int e = tid; e < N * nch; e += SB_THREADS) {
        const int r = e / nch, be = e - r * nch, al = r / nlag, i = r - al * nlag;
        // complex128: the kinetic and diagonal terms (the dominant ones) in compensated
        // sums, as the single-system residual does for this precision
        constexpr bool comp = sizeof(T) == 8;
        double sr = 0.0, si = 0.0, cr = 0.0, ci = 0.0;
        const double* Ki = y.K + (size_t)i * nlag;
        for (int j = 0; j < nlag; ++j) {
          const double2 x = Xg[(size_t)(al * nlag + j) * nch + be];
          if (absval) {
            sr = fma(fabs(Ki[j]), hypot(x.x, x.y), sr);
          } else if (comp) {
            dot2_add(sr, cr, Ki[j], x.x);
            dot2_add(si, ci, Ki[j], x.y);
          } else {
            sr = fma(Ki[j], x.x, sr);
            si = fma(Ki[j], x.y, si);
          }
        }
        const double rr = y.r[i];
        const int l = y.l[al];
        const double d = y.hm * l * (l + 1.0) / (rr * rr) + y.th[al] - y.E;
        const double2 xs = Xg[(size_t)r * nch + be];
        if (absval) {
          sr = fma(fabs(d), hypot(xs.x, xs.y), sr);
        } else if (comp) {
          dot2_add(sr, cr, d, xs.x);
          dot2_add(si, ci, d, xs.y);
        } else {
          sr = fma(d, xs.x, sr);
          si = fma(d, xs.y, si);
        }
        for (int a2 = 0; a2 < nch; ++a2) {
          const double2 w = y.V[i + (size_t)nlag * (al + (size_t)nch * a2)];
          const double2 x = Xg[(size_t)(a2 * nlag + i) * nch + be];
          if (absval) {
            sr = fma(hypot(w.x, w.y), hypot(x.x, x.y), sr);
          } else {
            sr = fma(w.x, x.x, fma(-w.y, x.y, sr));
            si = fma(w.x, x.y, fma(w.y, x.x, si));
          }
        }
        if (absval) {
          m = fmax(m, sr);
        } else {
          const double phi = al == be ? y.fa[i] : 0.0;
          const double2 rv = make_double2((phi - sr) - cr, (-si) - ci);
          Rg[e] = rv;
          m = fmax(m, hypot(rv.x, rv.y));
        }
      }
      return block_max(m);
    };
    const double scale = residual(true) + y.phi_max;
    // ---- refinement (the stopping rule of rmat_solve) ----
    int it = 0, stagn = 0, hits = 0, status = RMAT_OK;
    double prev = INFINITY, rel = 0.0;
    if (max_refine > 0 || tol > 0) {
      for (;;) {
        const double rmax = residual(false);
        rel = rmax / y.phi_max;
        hits = rmax <= RMAT_FLOOR_CONV * RMAT_U64 * scale ? hits + 1 : 0;
        bool stop = false, final = false;
        if (!isfinite(rel)) {
          status = RMAT_ENOCONV;
          stop = true;
        } else if (rel < tol) {
          stop = true;
        } else if (it >= max_refine) {
          status = (tol > 0 && rmax > RMAT_FLOOR_STALL * RMAT_U64 * scale) ? RMAT_ENOCONV : RMAT_OK;
          stop = true;
        } else if (hits >= need) {
          final = true;
        } else if (rel > 0.5 * prev) {
          if (++stagn >= patience) {
            status = rmax <= RMAT_FLOOR_STALL * RMAT_U64 * scale ? RMAT_OK : RMAT_ENOCONV;
            stop = true;
          }
        } else {
          stagn = 0;
        }
        if (stop) break;
        prev = rel;
        for (int e = tid; e < N * nch; e += SB_THREADS) Bw[e] = to_c(Rg[e], T());
        __syncthreads();
        solve();
        for (int e = tid; e < N * nch; e += SB_THREADS) {
          const double2 d = to_d(Bw[e]);
          Xg[e].x += d.x;
          Xg[e].y += d.y;
        }
        __syncthreads();
        ++it;
        if (final) break;
      }
    }
    // ---- R and U ----
    if (tid == 0) {
      s_p.nch = nch;
      s_p.nlag = nlag;
      s_p.nopen = y.nopen;
      s_p.ldx = N;
      s_p.a = y.a;
      s_p.hm = y.hm;
      s_p.B = y.B;
      s_p.E = y.E;
    }
    for (int c = tid; c < nch; c += SB_THREADS) {
      s_p.l[c] = y.l[c];
      s_p.thresh[c] = y.th[c];
      s_p.zz[c] = y.zz[c];
    }
    for (int c = tid; c < y.nopen; c += SB_THREADS) s_p.open[c] = y.open[c];
    __syncthreads();
    matching_cta(s_p, y.fa, Xg, (size_t)nch, 1, nullptr, y.U, S);
    __syncthreads();
    if (tid == 0) {
      int* st = st_all + (size_t)y.sys * ST_COUNT;
      for (int q = 0; q < ST_COUNT; ++q) st[q] = 0;
      if (s_info) st[ST_INFO] = s_info;
      const int cs = S->status;
      if (cs < 0) st[ST_CHANFN] = 1;
      else if (cs > 0 && !s_info) st[ST_INFO] = cs;  // exactly singular matching system
      IrState& w = ir_all[y.sys];
      w.prev = prev;
      w.rel = rel;
      w.stagn = stagn;
      w.done = 1;
      w.status = status;
      w.iters = it;
      w.floor_hits = hits;
      w.final = 0;
    }
    __syncthreads();
  }
}

}  // namespace

size_t small_coll_scratch_bytes() { return sizeof(NoallocScratch); }

size_t small_smem_bytes(int precision, int N, int nch) {
  const size_t e = precision == RMAT_C128 ? 16 : 8;
  return ((size_t)N * (N | 1) + (size_t)N * nch) * e + (size_t)N * sizeof(int);
}

int launch_batch_small(cudaStream_t st, int precision, const SmallSys* sys, int nsmall, int* next,
                       int grid, size_t smem, int max_refine, double tol, int* st_all,
                       IrState* ir_all, const SmallScratch& scr) {
  if (nsmall <= 0) return RMAT_OK;
  RMAT_CU(cudaMemsetAsync(next, 0, sizeof(int), st));
  const int need = rmat_floor_need(precision), patience = precision == RMAT_C128 ? 2 : 1;
  static size_t attr[2] = {0, 0};  // largest dynamic shared memory set so far (per type)
  size_t& a = attr[precision == RMAT_C128];
  if (smem > a) {
    if (precision == RMAT_C128)
      RMAT_CU(cudaFuncSetAttribute(batch_small_kernel<double>,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    else
      RMAT_CU(cudaFuncSetAttribute(batch_small_kernel<float>,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    a = smem;
  }
  if (precision == RMAT_C128)
    batch_small_kernel<double><<<grid, SB_THREADS, smem, st>>>(sys, nsmall, next, max_refine, tol,
                                                               need, patience, st_all, ir_all, scr);
  else
    batch_small_kernel<float><<<grid, SB_THREADS, smem, st>>>(sys, nsmall, next, max_refine, tol,
                                                              need, patience, st_all, ir_all, scr);
  RMAT_CU(cudaGetLastError());
  return RMAT_OK;
}
