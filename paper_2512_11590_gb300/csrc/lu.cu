// Blocked right-looking LU with partial pivoting and the triangular solves.
//
// Paper: Type-1 solver M = P L U with partial pivoting followed by forward and
// backward substitution for all nch right-hand sides (Sec. 3.1); the same
// factorisation in single precision for the mixed-precision solvers
// (Sec. 3.2, 3.4).  Layout: row-major working matrix (the R-matrix C is
// complex symmetric, so row-major C equals the paper's column-major C), block
// width nb.  For each block column k0:
//   G2  panel:  cooperative kernel over rows k0..n-1, columns k0..k0+jb; one
//               grid barrier per column; warp-shuffle argmax of |Re|+|Im|
//               (first row on ties); the pivot row travels through a slot in
//               global memory, so swap, scaling and rank-1 update need no
//               second barrier.
//   G3  swaps + TRSM: the panel's row interchanges applied to the trailing
//               columns, then U12 = L11^-1 A12.
//   G4  trailing update C22 -= L21 U12 (tensor cores, gemm_tc.cu, or the
//               SIMT kernel below).
// Interchanges are NOT applied to the columns left of the panel: the forward
// solve replays the panel permutations block by block, which is equivalent to
// LAPACK's P^T applied once.
#include <algorithm>
#include <climits>

#include <cooperative_groups.h>
#include <cuda_fp16.h>

#include "cplx.cuh"
#include "rmat_internal.h"

namespace {

constexpr int PANEL_THREADS = 256;
constexpr int MAX_RPC = 4096;  // rows per panel CTA

// SMEM: the CTA's panel rows live in shared memory for the whole column loop
// (loaded once, written back at the end); otherwise they are read and written
// in place in global memory (L2-resident), for panels too tall to stage.
template <class T, bool SMEM>
__global__ void __launch_bounds__(PANEL_THREADS)
panel_kernel(cplx<T>* __restrict__ A, int ld, int k0, int n, int jb, int* __restrict__ ipiv,
             int* __restrict__ stat, PanelScratch ps, int rpc, int ldr, long long spin_limit) {
  using C2 = cplx<T>;
  const int P = gridDim.x, cta = blockIdx.x, tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5, nwarp = PANEL_THREADS / 32;
  const int r_lo = k0 + cta * rpc;
  const int r_hi = min(k0 + (cta + 1) * rpc, n);
  T* cval = (T*)ps.cval;
  C2* crow = (C2*)ps.crow;
  C2* trow = (C2*)ps.trow;

  __shared__ T s_v[32];
  __shared__ int s_i[32];
  __shared__ int s_win, s_zero, s_abort;
  extern __shared__ unsigned char smem_raw[];
  C2* s_prow = reinterpret_cast<C2*>(smem_raw);  // [RMAT_MAX_NB] pivot row
  C2* s_trow = s_prow + RMAT_MAX_NB;             // [RMAT_MAX_NB] old row gj
  C2* s_l = s_trow + RMAT_MAX_NB;                // [rpc]
  C2* s_rows = s_l + rpc;                        // [rpc][ldr] when SMEM
  // own row r, panel-local column c (shared-memory rows padded to ldr = jb + 1 when
  // that fits, so a column read by consecutive rows spreads over the banks)
  auto at = [&](int r) -> C2* {
    return SMEM ? s_rows + (size_t)(r - r_lo) * ldr : A + (size_t)r * ld + k0;
  };
  if (tid == 0) s_abort = 0;
  if (SMEM) {
    for (int e = tid; e < (r_hi - r_lo) * jb; e += PANEL_THREADS) {
      const int rr = e / jb, cc = e - rr * jb;
      s_rows[(size_t)rr * ldr + cc] = A[(size_t)(r_lo + rr) * ld + k0 + cc];
    }
  }
  __syncthreads();

  // Column lookahead: right after column j's multipliers, only column j+1 of the
  // rank-1 update is applied and its local candidate found; the two rows published
  // before the barrier (the candidate and row gj+1) are brought fully up to date,
  // and the rest of column j's update runs while the grid barrier is in flight.
  __shared__ T s_cb;
  __shared__ int s_ci, s_pre0, s_pre1, s_zprev;
  // block-wide (best, bidx) -> s_cb, s_ci (first row on ties)
  auto block_cand = [&](T best, int bidx) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const T ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bidx, o);
      if (ob > best || (ob == best && oi < bidx)) { best = ob; bidx = oi; }
    }
    if (lane == 0) { s_v[warp] = best; s_i[warp] = bidx; }
    __syncthreads();
    if (warp == 0) {
      best = lane < nwarp ? s_v[lane] : (T)-1;
      bidx = lane < nwarp ? s_i[lane] : INT_MAX;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const T ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bidx, o);
        if (ob > best || (ob == best && oi < bidx)) { best = ob; bidx = oi; }
      }
      if (lane == 0) { s_cb = best; s_ci = bidx; }
    }
    __syncthreads();
  };
  // publish column jj's candidate (row s_ci) and row k0+jj, then arrive at barrier jj
  // complex64: the candidate (value, row, column generation) is one 64-bit record
  // per CTA and parity, stored with release semantics after the CTA's rows: the
  // records are the barrier, and the winner is known as soon as all have arrived.
  // complex128: value/row in cval/cidx and an arrival counter.
  unsigned long long* rec = reinterpret_cast<unsigned long long*>(ps.cval);
  auto publish_arrive = [&](int jj) {
    const int pp = jj & 1, gg = k0 + jj;
    if (warp == 0) {
      if (sizeof(T) == 8 && lane == 0) {
        cval[pp * RMAT_MAX_PANEL_CTAS + cta] = s_cb;
        ps.cidx[pp * RMAT_MAX_PANEL_CTAS + cta] = s_ci;
      }
      if (s_ci != INT_MAX) {
        C2* slot = crow + ((size_t)pp * RMAT_MAX_PANEL_CTAS + cta) * RMAT_MAX_NB;
        const C2* src = at(s_ci);
        for (int c = lane; c < jb; c += 32) slot[c] = src[c];
      }
    } else if (gg >= r_lo && gg < r_hi) {
      const C2* src = at(gg);
      for (int c = tid - 32; c < jb; c += PANEL_THREADS - 32) trow[(size_t)pp * RMAT_MAX_NB + c] = src[c];
    }
    __syncthreads();
    if (tid == 0) {
      if constexpr (sizeof(T) == 4) {
        const unsigned long long v =
            ((unsigned long long)__float_as_uint((float)(s_cb > (T)0 ? s_cb : (T)0)) << 32) |
            ((unsigned long long)(jj + 1) << 18) | (unsigned long long)(s_ci == INT_MAX ? 0x3FFFF : s_ci);
        asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(rec + pp * RMAT_MAX_PANEL_CTAS + cta),
                     "l"(v)
                     : "memory");
      } else {
        asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(ps.bar) : "memory");
      }
    }
  };

  {  // column 0: nothing pending
    T best = (T)-1;
    int bidx = INT_MAX;
    for (int r = r_lo + tid; r < r_hi; r += PANEL_THREADS) {
      const T m = cabs1<T>(at(r)[0]);
      if (m > best) { best = m; bidx = r; }
    }
    if (tid == 0) { s_pre0 = -1; s_pre1 = -1; s_zprev = 1; }
    block_cand(best, bidx);
    publish_arrive(0);
  }

  for (int j = 0; j < jb; ++j) {
    const int gj = k0 + j;
    const int par = j & 1;
    // ---- deferred: column j-1's update of columns j+1.. (rows > gj-1, not published) ----
    if (!s_zprev && j + 1 < jb) {
      const int p0 = s_pre0, p1 = s_pre1;
      for (int r = max(r_lo, gj) + warp; r < r_hi; r += nwarp) {
        if (r == p0 || r == p1) continue;
        const C2 lm = s_l[r - r_lo];
        C2* Ar = at(r);
        for (int c = j + 1 + lane; c < jb; c += 32) {
          C2 x = Ar[c];
          csub_mul<T>(x, lm, s_prow[c]);
          Ar[c] = x;
        }
      }
    }
    if constexpr (sizeof(T) == 4) {
      // ---- barrier j = all P records of parity j&1 carry generation j+1 (bounded) ----
      constexpr int QPL = RMAT_MAX_PANEL_CTAS / 32;
      unsigned long long r[QPL];
      if (warp == 0) {
        long long polls = 0;
        bool ok = false;
        for (;;) {
          bool mine = true;
#pragma unroll
          for (int u = 0; u < QPL; ++u) {
            const int q = lane + 32 * u;
            r[u] = 0ull;
            if (q < P)
              asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];"
                           : "=l"(r[u])
                           : "l"(rec + par * RMAT_MAX_PANEL_CTAS + q)
                           : "memory");
            if (q < P && (int)((r[u] >> 18) & 0x3FFF) != j + 1) mine = false;
          }
          if (__all_sync(0xffffffffu, mine)) { ok = true; break; }
          if (++polls > spin_limit) break;
        }
        if (!ok && lane == 0) {
          atomicExch(&stat[ST_TIMEOUT], 1);
          s_abort = 1;
        }
      }
      // every warp has finished the deferred update (it reads s_prow, rewritten below)
      __syncthreads();
      if (s_abort) return;
      if (warp == 0) {
        {
          asm volatile("fence.acq_rel.gpu;" ::: "memory");
          float best = -1.f;
          int bidx = INT_MAX, bc = -1;
#pragma unroll
          for (int u = 0; u < QPL; ++u) {
            const int q = lane + 32 * u;
            if (q >= P) continue;
            const float v = __uint_as_float((unsigned)(r[u] >> 32));
            int ix = (int)(r[u] & 0x3FFFF);
            if (ix == 0x3FFFF) ix = INT_MAX;
            if (v > best || (v == best && ix < bidx)) { best = v; bidx = ix; bc = q; }
          }
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) {
            const float ob = __shfl_xor_sync(0xffffffffu, best, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bidx, o);
            const int oc = __shfl_xor_sync(0xffffffffu, bc, o);
            if (ob > best || (ob == best && oi < bidx)) { best = ob; bidx = oi; bc = oc; }
          }
          // winner's row and the old row gj in one round trip
          const int wc = (bc >= 0 && bc < P) ? bc : 0;
          const C2* wslot = crow + ((size_t)par * RMAT_MAX_PANEL_CTAS + wc) * RMAT_MAX_NB;
          for (int c = lane; c < jb; c += 32) {
            s_prow[c] = ld_cg(wslot + c);
            s_trow[c] = ld_cg(trow + (size_t)par * RMAT_MAX_NB + c);
          }
          if (lane == 0) {
            s_win = bidx;
            s_zero = !(best > 0.f);
          }
        }
      }
      __syncthreads();
      if (s_abort) return;
    } else {
      // ---- grid barrier j (bounded spin): acquire-poll ----
      if (tid == 0) {
        const unsigned target = (unsigned)(j + 1) * (unsigned)P;
        long long polls = 0;
        while (ld_acquire_gpu(ps.bar) < target) {
          if (++polls > spin_limit) {
            atomicExch(&stat[ST_TIMEOUT], 1);
            s_abort = 1;
            break;
          }
        }
      }
      __syncthreads();
      if (s_abort) return;
      // ---- phase B: global winner (warp 0), old row gj prefetched (other warps) ----
      if (warp == 0) {
        T best = (T)-1;
        int bidx = INT_MAX;
        int bc = -1;
        // all candidates requested before any is compared: one L2 round trip
        constexpr int QPL = RMAT_MAX_PANEL_CTAS / 32;
        T cv[QPL];
        int ci[QPL];
  #pragma unroll
        for (int u = 0; u < QPL; ++u) {
          const int q = lane + 32 * u;
          cv[u] = q < P ? ld_cg(cval + par * RMAT_MAX_PANEL_CTAS + q) : (T)-1;
          ci[u] = q < P ? ld_cg(ps.cidx + par * RMAT_MAX_PANEL_CTAS + q) : INT_MAX;
        }
  #pragma unroll
        for (int u = 0; u < QPL; ++u)
          if (cv[u] > best || (cv[u] == best && ci[u] < bidx)) {
            best = cv[u];
            bidx = ci[u];
            bc = lane + 32 * u;
          }
  #pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          const T ob = __shfl_xor_sync(0xffffffffu, best, o);
          const int oi = __shfl_xor_sync(0xffffffffu, bidx, o);
          const int oc = __shfl_xor_sync(0xffffffffu, bc, o);
          if (ob > best || (ob == best && oi < bidx)) { best = ob; bidx = oi; bc = oc; }
        }
        const int wc = (bc >= 0 && bc < P) ? bc : 0;
        const C2* wslot = crow + ((size_t)par * RMAT_MAX_PANEL_CTAS + wc) * RMAT_MAX_NB;
        for (int c = lane; c < jb; c += 32) s_prow[c] = ld_cg(wslot + c);
        if (lane == 0) {
          s_win = bidx;
          s_zero = !(best > (T)0);
        }
      } else {
        for (int c = tid - 32; c < jb; c += PANEL_THREADS - 32)
          s_trow[c] = ld_cg(trow + (size_t)par * RMAT_MAX_NB + c);
      }
      __syncthreads();
    }
    const int p = (s_win >= gj && s_win < n) ? s_win : gj;
    if (cta == 0 && tid == 0) {
      ipiv[gj] = p;
      if (s_zero) atomicCAS(&stat[ST_INFO], 0, gj + 1);
    }
    if (p != gj) {
      if (gj >= r_lo && gj < r_hi) {
        C2* dst = at(gj);
        for (int c = tid; c < jb; c += PANEL_THREADS) dst[c] = s_prow[c];
      }
      if (p >= r_lo && p < r_hi) {
        C2* dst = at(p);
        for (int c = tid; c < jb; c += PANEL_THREADS) dst[c] = s_trow[c];
      }
    }
    __syncthreads();
    // ---- multipliers of column j (an exactly zero column keeps its entries: LAPACK) ----
    const bool zero = s_zero;
    const C2 piv = s_prow[j];
    const int r_first = max(r_lo, gj + 1);
    if (!zero)
      for (int r = r_first + tid; r < r_hi; r += PANEL_THREADS) {
        C2* ar = at(r);
        const C2 lm = cdiv<T>(ar[j], piv);
        ar[j] = lm;
        s_l[r - r_lo] = lm;
      }
    if (j + 1 == jb) break;
    __syncthreads();
    // ---- column j+1: its update, then its local candidate ----
    T best = (T)-1;
    int bidx = INT_MAX;
    for (int r = r_first + tid; r < r_hi; r += PANEL_THREADS) {
      C2* ar = at(r);
      C2 x = ar[j + 1];
      if (!zero) {
        csub_mul<T>(x, s_l[r - r_lo], s_prow[j + 1]);
        ar[j + 1] = x;
      }
      const T m = cabs1<T>(x);
      if (m > best) { best = m; bidx = r; }
    }
    block_cand(best, bidx);
    // rows published before barrier j+1: the candidate and row gj+1, fully updated
    const int q0 = (s_ci != INT_MAX) ? s_ci : -1;
    const int q1 = (gj + 1 >= r_lo && gj + 1 < r_hi && gj + 1 != q0) ? gj + 1 : -1;
    if (!zero && warp < 2) {
      const int r = warp == 0 ? q0 : q1;
      if (r >= 0) {
        const C2 lm = s_l[r - r_lo];
        C2* Ar = at(r);
        for (int c = j + 2 + lane; c < jb; c += 32) {
          C2 x = Ar[c];
          csub_mul<T>(x, lm, s_prow[c]);
          Ar[c] = x;
        }
      }
    }
    if (tid == 0) { s_pre0 = q0; s_pre1 = q1; s_zprev = zero; }
    __syncthreads();
    publish_arrive(j + 1);
  }
  __syncthreads();
  if (SMEM) {
    for (int e = tid; e < (r_hi - r_lo) * jb; e += PANEL_THREADS) {
      const int rr = e / jb, cc = e - rr * jb;
      A[(size_t)(r_lo + rr) * ld + k0 + cc] = s_rows[(size_t)rr * ldr + cc];
    }
  }
}

// Cluster variant of the panel for M rows that fit the shared memory of one thread
// block cluster (up to 16 CTAs): the same partial pivoting (largest |Re|+|Im|, first
// row on ties), with the per-column exchange through distributed shared memory and
// the hardware cluster barrier instead of a grid barrier in global memory.  Each CTA
// publishes its candidate (value, row, row contents) and, if it holds row gj, that
// row, in parity-double-buffered shared slots; one cluster barrier per column.
template <class T>
__global__ void __launch_bounds__(PANEL_THREADS)
panel_cluster_kernel(cplx<T>* __restrict__ A, int ld, int k0, int n, int jb,
                     int* __restrict__ ipiv, int* __restrict__ stat, int rpc, int ldr) {
  namespace cg = cooperative_groups;
  using C2 = cplx<T>;
  cg::cluster_group cluster = cg::this_cluster();
  const int CS = (int)cluster.num_blocks(), rank = (int)cluster.block_rank(), tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5, nwarp = PANEL_THREADS / 32;
  const int r_lo = k0 + rank * rpc;
  const int r_hi = min(k0 + (rank + 1) * rpc, n);
  __shared__ T s_v[32];
  __shared__ int s_i[32];
  __shared__ int s_win, s_zero;
  __shared__ T c_v[2];    // published candidate value (parity buffers)
  __shared__ int c_i[2];  // published candidate row
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C2* s_prow = reinterpret_cast<C2*>(smem_raw);  // [jb] pivot row
  C2* s_trow = s_prow + jb;                      // [jb] old row gj
  C2* crow = s_trow + jb;                        // [2][jb] published candidate row
  C2* trowp = crow + 2 * jb;                     // [2][jb] published row gj (its holder)
  C2* s_l = trowp + 2 * jb;                      // [rpc]
  C2* s_rows = s_l + rpc;                        // [rpc][ldr]
  auto at = [&](int r) -> C2* { return s_rows + (size_t)(r - r_lo) * ldr; };
  for (int e = tid; e < (r_hi - r_lo) * jb; e += PANEL_THREADS) {
    const int rr = e / jb, cc = e - rr * jb;
    s_rows[(size_t)rr * ldr + cc] = A[(size_t)(r_lo + rr) * ld + k0 + cc];
  }
  __syncthreads();
  for (int j = 0; j < jb; ++j) {
    const int gj = k0 + j, par = j & 1;
    T best = (T)-1;
    int bidx = INT_MAX;
    for (int r = max(r_lo, gj) + tid; r < r_hi; r += PANEL_THREADS) {
      const T m = cabs1<T>(at(r)[j]);
      if (m > best) { best = m; bidx = r; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const T ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bidx, o);
      if (ob > best || (ob == best && oi < bidx)) { best = ob; bidx = oi; }
    }
    if (lane == 0) { s_v[warp] = best; s_i[warp] = bidx; }
    if (gj >= r_lo && gj < r_hi && warp > 0) {
      const C2* src = at(gj);
      for (int c = tid - 32; c < jb; c += PANEL_THREADS - 32) trowp[par * jb + c] = src[c];
    }
    __syncthreads();
    if (warp == 0) {
      best = lane < nwarp ? s_v[lane] : (T)-1;
      bidx = lane < nwarp ? s_i[lane] : INT_MAX;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const T ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bidx, o);
        if (ob > best || (ob == best && oi < bidx)) { best = ob; bidx = oi; }
      }
      if (lane == 0) { c_v[par] = best; c_i[par] = bidx; }
      if (bidx != INT_MAX)
        for (int c = lane; c < jb; c += 32) crow[par * jb + c] = at(bidx)[c];
    }
    cluster.sync();  // every CTA's candidate and row gj are published
    if (warp == 0) {
      best = (T)-1;
      bidx = INT_MAX;
      int wr = 0;
      if (lane < CS) {
        best = *cluster.map_shared_rank(&c_v[par], lane);
        bidx = *cluster.map_shared_rank(&c_i[par], lane);
        wr = lane;
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const T ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bidx, o);
        const int orr = __shfl_xor_sync(0xffffffffu, wr, o);
        if (ob > best || (ob == best && oi < bidx)) { best = ob; bidx = oi; wr = orr; }
      }
      const C2* wrow = cluster.map_shared_rank(crow + par * jb, wr);
      for (int c = lane; c < jb; c += 32) s_prow[c] = wrow[c];
      if (lane == 0) {
        s_win = bidx;
        s_zero = !(best > (T)0);
      }
    } else {
      const int hr = min((gj - k0) / rpc, CS - 1);  // the CTA holding row gj
      const C2* hrow = cluster.map_shared_rank(trowp + par * jb, hr);
      for (int c = tid - 32; c < jb; c += PANEL_THREADS - 32) s_trow[c] = hrow[c];
    }
    __syncthreads();
    const int p = (s_win >= gj && s_win < n) ? s_win : gj;
    if (rank == 0 && tid == 0) {
      ipiv[gj] = p;
      if (s_zero) atomicCAS(&stat[ST_INFO], 0, gj + 1);
    }
    if (p != gj) {
      if (gj >= r_lo && gj < r_hi)
        for (int c = tid; c < jb; c += PANEL_THREADS) at(gj)[c] = s_prow[c];
      if (p >= r_lo && p < r_hi)
        for (int c = tid; c < jb; c += PANEL_THREADS) at(p)[c] = s_trow[c];
    }
    __syncthreads();
    if (s_zero) continue;  // exactly zero column: no scaling, no update (LAPACK)
    const C2 piv = s_prow[j];
    const int r_first = max(r_lo, gj + 1);
    for (int r = r_first + tid; r < r_hi; r += PANEL_THREADS) {
      C2* ar = at(r);
      const C2 lm = cdiv<T>(ar[j], piv);
      ar[j] = lm;
      s_l[r - r_lo] = lm;
    }
    __syncthreads();
    if (j + 1 < jb) {
      for (int r = r_first + warp; r < r_hi; r += nwarp) {
        const C2 lm = s_l[r - r_lo];
        C2* Ar = at(r);
        for (int c = j + 1 + lane; c < jb; c += 32) {
          C2 x = Ar[c];
          csub_mul<T>(x, lm, s_prow[c]);
          Ar[c] = x;
        }
      }
    }
    __syncthreads();
  }
  cluster.sync();  // no CTA leaves while a peer may still read its published slots
  for (int e = tid; e < (r_hi - r_lo) * jb; e += PANEL_THREADS) {
    const int rr = e / jb, cc = e - rr * jb;
    A[(size_t)(r_lo + rr) * ld + k0 + cc] = s_rows[(size_t)rr * ldr + cc];
  }
}

// ---- G3: row interchanges on the trailing columns + U12 = L11^-1 A12 ------
// (apply_perm_kernel and trsm_block_rhs_kernel below, on the trailing columns
// viewed as right-hand sides)

__device__ __forceinline__ float tf32_round(float x) {
  unsigned r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// Tensor operand planes, four per operand: [re_hi | re_lo | im_hi | im_lo].
//   fmt 0: TF32 hi/lo in fp32 words (hi = TF32 rounding, lo = exact remainder);
//   fmt 1: FP16 hi/lo of s*z, s a power of two chosen so that |s*z| <= 1.
//   F: the whole factor, row-major [n][ldf] — L21 blocks and U12 rows as they are
//      produced; the A operand of the trailing update and of the solve updates.
//   B: U12^T of the current block, [c][256] (K-major B operand of the trailing update).
//   Y: a solved right-hand-side block transposed, [rhs][256] (B operand of the solve updates).
// With fmt 1, L21 is stored unscaled (|l| <= sqrt(2) under |Re|+|Im| pivoting), each
// U12 block with one scale (inverse kept in uscale[block]), each Y column with its
// own (inverse in ycs[column]); the tensor-core epilogue multiplies the scales back.
__device__ __forceinline__ void put4(void* base, size_t plane, size_t o, float2 z, int fmt,
                                     float sc) {
  if (fmt == 0) {
    float* b = reinterpret_cast<float*>(base);
    const float rh = tf32_round(z.x), ih = tf32_round(z.y);
    b[o] = rh;
    b[plane + o] = z.x - rh;
    b[2 * plane + o] = ih;
    b[3 * plane + o] = z.y - ih;
  } else {
    __half* b = reinterpret_cast<__half*>(base);
    const float xr = z.x * sc, xi = z.y * sc;
    const __half hr = __float2half_rn(xr), hi = __float2half_rn(xi);
    b[o] = hr;
    b[plane + o] = __float2half_rn(xr - __half2float(hr));
    b[2 * plane + o] = hi;
    b[3 * plane + o] = __float2half_rn(xi - __half2float(hi));
  }
}

// Power-of-two s with m*s in [0.5, 1) (1 for m = 0 or non-finite m).
__device__ __forceinline__ float pow2_scale(float m) {
  if (!(m > 0.f) || !(m < INFINITY)) return 1.f;
  int e;
  frexpf(m, &e);
  e = max(-126, min(126, e));
  return ldexpf(1.f, -e);
}

__device__ __forceinline__ float cmaxabs(float2 z) { return fmaxf(fabsf(z.x), fabsf(z.y)); }

// L21 rows r in [k0+jb, n), columns k0..k0+jb-1 -> F (warp per row, lanes over columns).
__global__ void split_l21_kernel(const float2* __restrict__ A, int ld, int k0, int jb, int n,
                                 void* __restrict__ F, int ldf, size_t fplane, int fmt) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const int r = k0 + jb + warp;
  if (r >= n) return;
  for (int t = lane; t < jb; t += 32)
    put4(F, fplane, (size_t)r * ldf + k0 + t, A[(size_t)r * ld + k0 + t], fmt, 1.f);
}

// ---- inverse of a unit lower triangular diagonal block ------------------------
// X = L11^-1 for the JB x JB block at (k0, k0) (unit diagonal implied; JB = 64 or 128),
// written in full (ones on the diagonal, zeros above) to Xout [JB][JB].  One CTA:
//   level 0: each 32 x 32 diagonal block inverted in place by one warp, column by
//     column from the right: X[i][j] = -(L[i][j] + sum_{j<k<i} X[i][k] L[k][j]), the
//     column's L entries passed between lanes by shuffles before they are replaced;
//   level h = 32, 64: every 2h x 2h diagonal block [A 0; B C] with A^-1, C^-1 in place
//     gets its lower-left block -C^-1 (B A^-1): T = B A^-1 into a scratch block, then
//     -C^-1 T over B (thread: one column, every eighth row; the triangular factors'
//     zero parts skipped).
constexpr int TINV_THREADS = 512;
template <int JB>
__global__ void __launch_bounds__(TINV_THREADS)
tri_inv_lower_kernel(const float2* __restrict__ A, int ld, int k0, float2* __restrict__ Xout) {
  constexpr int LDX = JB + 1, LDT = JB / 2 + 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* X = reinterpret_cast<float2*>(smem_raw);  // [JB][LDX]
  float2* Tb = X + JB * LDX;                        // [JB / 2][LDT]
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const float2 zero = make_float2(0.f, 0.f);
  for (int e = tid; e < JB * JB; e += TINV_THREADS) {
    const int r = e / JB, c = e - r * JB;
    X[r * LDX + c] = c < r ? A[(size_t)(k0 + r) * ld + k0 + c] : zero;
  }
  __syncthreads();
  if (warp < JB / 32) {  // level 0
    float2* Xb = X + 32 * warp * (LDX + 1);
    for (int j = 30; j >= 0; --j) {
      const float2 lj = lane > j ? Xb[lane * LDX + j] : zero;
      float2 acc = lj;
      for (int k = j + 1; k < 31; ++k) {
        const float2 lk = make_float2(__shfl_sync(0xffffffffu, lj.x, k),
                                      __shfl_sync(0xffffffffu, lj.y, k));
        if (k < lane) cadd_mul<float>(acc, Xb[lane * LDX + k], lk);
      }
      __syncwarp();
      if (lane > j) Xb[lane * LDX + j] = make_float2(-acc.x, -acc.y);
      __syncwarp();
    }
  }
  __syncthreads();
#pragma unroll
  for (int h = 32; h < JB; h *= 2) {
    const int c = tid % h, r0 = (tid / h) % 8, d = tid / (8 * h);
    const bool on = d < JB / (2 * h);
    const int R0 = 2 * h * d + h, C0 = 2 * h * d;
    constexpr int MM = JB / 16;  // rows per thread at h = JB / 2 (the larger level)
    const int mm = h / 8;
    float2 t[MM];
    if (on) {
      // T = B A^-1:  T[i][c] = B[i][c] + sum_{k > c} B[i][k] X_A[k][c]
#pragma unroll
      for (int m = 0; m < MM; ++m) t[m] = m < mm ? X[(R0 + r0 + 8 * m) * LDX + C0 + c] : zero;
      for (int k = c + 1; k < h; ++k) {
        const float2 xk = X[(C0 + k) * LDX + C0 + c];
#pragma unroll
        for (int m = 0; m < MM; ++m)
          if (m < mm) cadd_mul<float>(t[m], X[(R0 + r0 + 8 * m) * LDX + C0 + k], xk);
      }
#pragma unroll
      for (int m = 0; m < MM; ++m)
        if (m < mm) Tb[(h * d + r0 + 8 * m) * LDT + c] = t[m];
    }
    __syncthreads();
    if (on) {
      // B := -C^-1 T:  X[R0+i][C0+c] = -(T[i][c] + sum_{k < i} X_C[i][k] T[k][c])
#pragma unroll
      for (int m = 0; m < MM; ++m) t[m] = m < mm ? Tb[(h * d + r0 + 8 * m) * LDT + c] : zero;
      const int imax = r0 + 8 * (mm - 1);
      for (int k = 0; k < imax; ++k) {
        const float2 tk = Tb[(h * d + k) * LDT + c];
#pragma unroll
        for (int m = 0; m < MM; ++m) {
          const int i = r0 + 8 * m;
          if (m < mm && k < i) cadd_mul<float>(t[m], X[(R0 + i) * LDX + R0 + k], tk);
        }
      }
#pragma unroll
      for (int m = 0; m < MM; ++m)
        if (m < mm) X[(R0 + r0 + 8 * m) * LDX + C0 + c] = make_float2(-t[m].x, -t[m].y);
    }
    __syncthreads();
  }
  for (int e = tid; e < JB * JB; e += TINV_THREADS) {
    const int r = e / JB, c = e - r * JB;
    Xout[e] = c < r ? X[r * LDX + c] : make_float2(c == r ? 1.f : 0.f, 0.f);
  }
}

// ---- complex-symmetric LDL^T without pivoting (C = C^T, Sec. 2) ----------------
// The jb x jb diagonal block (jb <= 128) factored in one CTA in shared memory: unit
// lower L11 below the diagonal, U11 = D11 L11^T on and above it (the unpivoted LU of
// the block), identity interchanges.  Right-looking in panels of DIAG_W columns:
//   column j of a panel: multipliers l_i = a_ij (1 / a_jj) for every row below j,
//     then the rank-1 update of the panel's columns right of j (all rows below j)
//     and of the panel's rows below j right of the panel (their U part);
//   after the panel: the block right of and below it -= L(panel columns) U(panel
//     rows), a GEMM of depth DIAG_W in which every thread keeps the U part of its two
//     columns in registers and reads each L row once (a warp-wide broadcast).
// A zero pivot is recorded in stat[ST_INFO] (first column, 1-based) and its column
// left as it is.
constexpr int DIAG_THREADS = 512, DIAG_W = 8;
template <class T>
__global__ void __launch_bounds__(DIAG_THREADS)
diag_nopiv_kernel(cplx<T>* __restrict__ A, int ld, int k0, int jb, int* __restrict__ ipiv,
                  int* __restrict__ stat) {
  using C2 = cplx<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C2* s = reinterpret_cast<C2*>(smem_raw);  // [jb][jb + 2]
  const int ls = jb + 2, tid = threadIdx.x;
  C2* D = A + (size_t)k0 * ld + k0;
  for (int e = tid; e < jb * jb; e += DIAG_THREADS) {
    const int r = e / jb, cc = e - r * jb;
    s[r * ls + cc] = D[(size_t)r * ld + cc];
  }
  for (int e = tid; e < jb; e += DIAG_THREADS) ipiv[k0 + e] = k0 + e;
  __syncthreads();
  for (int p0 = 0; p0 < jb; p0 += DIAG_W) {
    const int pe = min(p0 + DIAG_W, jb);  // panel columns [p0, pe)
    for (int j = p0; j < pe; ++j) {
      const C2 piv = s[j * ls + j];
      if (piv.x == (T)0 && piv.y == (T)0) {  // uniform: every thread reads the same pivot
        if (tid == 0) atomicCAS(&stat[ST_INFO], 0, k0 + j + 1);
        continue;
      }
      if (j + 1 == jb) break;
      const C2 inv = cdiv<T>(mkc<T>((T)1, (T)0), piv);
      if (tid > j && tid < jb) s[tid * ls + j] = cmul<T>(s[tid * ls + j], inv);
      __syncthreads();
      // region a: rows (j, jb) x panel columns (j, pe), a thread per (row, column) with
      // DIAG_W columns per row; region b: panel rows (j, pe) x columns [pe, jb), 128
      // columns per row (DIAG_W, 128 and the block size are powers of two: shifts)
      static_assert(DIAG_W == 8 && DIAG_THREADS == 512, "thread maps below");
      for (int t = tid; (t >> 3) < jb - 1 - j; t += DIAG_THREADS) {
        const int i = j + 1 + (t >> 3), c = j + 1 + (t & 7);
        if (c < pe) csub_mul<T>(s[i * ls + c], s[i * ls + j], s[j * ls + c]);
      }
      for (int t = tid; (t >> 7) < pe - 1 - j; t += DIAG_THREADS) {
        const int i = j + 1 + (t >> 7), c = pe + (t & 127);
        if (c < jb) csub_mul<T>(s[i * ls + c], s[i * ls + j], s[j * ls + c]);
      }
      __syncthreads();
    }
    if (pe >= jb) break;
    // trailing block [pe, jb) x [pe, jb) -= L[., p0:pe) U[p0:pe, .)
    const int c0 = pe + 2 * (tid & 63), r0 = tid >> 6;
    if (c0 < jb) {
      const bool two = c0 + 1 < jb;
      C2 u0[DIAG_W], u1[DIAG_W];
#pragma unroll
      for (int k = 0; k < DIAG_W; ++k) {
        const bool on = p0 + k < pe;
        u0[k] = on ? s[(p0 + k) * ls + c0] : mkc<T>((T)0, (T)0);
        u1[k] = on && two ? s[(p0 + k) * ls + c0 + 1] : mkc<T>((T)0, (T)0);
      }
      for (int i = pe + r0; i < jb; i += DIAG_THREADS / 64) {
        const C2* li = s + i * ls + p0;
        C2 a0 = s[i * ls + c0], a1 = two ? s[i * ls + c0 + 1] : mkc<T>((T)0, (T)0);
#pragma unroll
        for (int k = 0; k < DIAG_W; ++k) {
          const C2 l = p0 + k < pe ? li[k] : mkc<T>((T)0, (T)0);
          csub_mul<T>(a0, l, u0[k]);
          csub_mul<T>(a1, l, u1[k]);
        }
        s[i * ls + c0] = a0;
        if (two) s[i * ls + c0 + 1] = a1;
      }
    }
    __syncthreads();
  }
  for (int e = tid; e < jb * jb; e += DIAG_THREADS) {
    const int r = e / jb, cc = e - r * jb;
    D[(size_t)r * ld + cc] = s[r * ls + cc];
  }
}

// L21 = C21 U11^-1 = (L11 U12)^T U11^-1 = U12^T D11^-1, since C21 = C12^T and
// U11 = D11 L11^T:  L21[r][j] = U12[j][r] / U11[j][j], written into A's block column
// below the diagonal block (rows k0+jb.., columns k0..k0+jb-1).  32 x 32 tiles
// through shared memory (rows of U12 read and rows of L21 written coalesced).  The
// largest max(|Re|, |Im|) of L21 goes to *lmax (the element growth the unpivoted
// factor shows; float bits).
__global__ void __launch_bounds__(256)
l21_from_u12_kernel(float2* __restrict__ A, int ld, int k0, int jb, int n,
                    unsigned* __restrict__ lmax) {
  __shared__ float2 tile[32][33];
  __shared__ float2 dinv[32];
  const int r0 = k0 + jb + blockIdx.x * 32, j0 = blockIdx.y * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  if (threadIdx.x < 32) {
    const int j = j0 + threadIdx.x;
    float2 d = j < jb ? A[(size_t)(k0 + j) * ld + k0 + j] : make_float2(0.f, 0.f);
    dinv[threadIdx.x] = (d.x == 0.f && d.y == 0.f) ? make_float2(0.f, 0.f)
                                                   : cdiv<float>(make_float2(1.f, 0.f), d);
  }
  for (int t = ty; t < 32; t += 8) {  // tile[j][r] = U12[j0 + t][r0 + tx]
    const int j = j0 + t, r = r0 + tx;
    tile[t][tx] = (j < jb && r < n) ? A[(size_t)(k0 + j) * ld + r] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  float m = 0.f;
  for (int t = ty; t < 32; t += 8) {  // L21[r0 + t][j0 + tx]
    const int r = r0 + t, j = j0 + tx;
    if (r < n && j < jb) {
      const float2 l = cmul<float>(tile[tx][t], dinv[tx]);
      A[(size_t)r * ld + k0 + j] = l;
      m = fmaxf(m, cmaxabs(l));
    }
  }
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if (tx == 0 && m > 0.f) atomicMax(lmax, __float_as_uint(m));
}

// ipiv[i] = i: the interchange record of a factorisation without pivoting.
__global__ void identity_pivots_kernel(int* __restrict__ ipiv, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    ipiv[i] = i;
}

// The A operand of the tensor-core U12 product: M = I - L11^-1 (strictly lower, the
// negated entries of the inverse below its unit diagonal) split into four planes
// [JB][128]; FP16 planes carry the power-of-two scale of max |M|, its inverse to
// *inv_scale.  One CTA.
__global__ void __launch_bounds__(1024)
minv_planes_kernel(const float2* __restrict__ Linv, int JB, void* __restrict__ M, size_t mplane,
                   int fmt, float* __restrict__ inv_scale) {
  __shared__ float red[32];
  float m = 0.f;
  for (int e = threadIdx.x; e < JB * JB; e += 1024)
    if (e % JB < e / JB) m = fmaxf(m, cmaxabs(Linv[e]));
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  m = 0.f;
  for (int w = 0; w < 32; ++w) m = fmaxf(m, red[w]);
  const float sc = fmt == 1 ? pow2_scale(m) : 1.f;
  if (threadIdx.x == 0 && inv_scale) *inv_scale = 1.f / sc;
  for (int e = threadIdx.x; e < JB * JB; e += 1024) {
    const int i = e / JB, k = e - i * JB;
    const float2 v = k < i ? make_float2(-Linv[e].x, -Linv[e].y) : make_float2(0.f, 0.f);
    put4(M, mplane, (size_t)i * 128 + k, v, fmt, sc);
  }
}

// max(|Re|, |Im|) over rows k0..k0+jb-1, columns c0..c0+ncols-1 of A -> atomicMax on
// the float bits in *out (non-negative floats order like their bit patterns).
__global__ void __launch_bounds__(256)
block_absmax_kernel(const float2* __restrict__ A, int ld, int k0, int jb, int c0, int ncols,
                    unsigned* __restrict__ out, unsigned* __restrict__ out2) {
  float m = 0.f;
  const long long total = (long long)jb * ncols;
  for (long long e = blockIdx.x * 256ll + threadIdx.x; e < total; e += (long long)gridDim.x * 256)
    m = fmaxf(m, cmaxabs(A[(size_t)(k0 + e / ncols) * ld + c0 + e % ncols]));
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  __shared__ float sm[8];
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < 8; ++w) m = fmaxf(m, sm[w]);
    atomicMax(out, __float_as_uint(m));
    if (out2) atomicMax(out2, __float_as_uint(m));
  }
}

// 32 x 32 tile of a jb x ncols block S (rows t, columns c; row stride lds):
// optional row-major copy into F (rows frow0 + t, columns fcol0 + c) and optional
// transposed planes T[trow0 + c][tk0 + t], zero-filled for jb <= t < round_up(jb, 32).
// fmt 1: F's scale comes from the max in *smax, T's from *smaxT (default: F's);
// CTA (0, 0) records the inverse scales.
__global__ void __launch_bounds__(256)
split_block_kernel(const float2* __restrict__ S, int lds, int jb, int ncols, void* __restrict__ F,
                   int ldf, size_t fplane, int frow0, int fcol0, void* __restrict__ T,
                   size_t tplane, int trow0, int tk0, int fmt, const unsigned* __restrict__ smax,
                   float* __restrict__ sinv, const unsigned* __restrict__ smaxT,
                   float* __restrict__ sinvT) {
  __shared__ float2 tile[32][33];
  const float sc = (fmt == 1 && smax) ? pow2_scale(__uint_as_float(*smax)) : 1.f;
  const float scT = (fmt == 1 && smaxT) ? pow2_scale(__uint_as_float(*smaxT)) : sc;
  if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) {
    if (sinv) *sinv = 1.f / sc;
    if (sinvT) *sinvT = 1.f / scT;
  }
  const int c0 = blockIdx.x * 32, t0 = blockIdx.y * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
  for (int i = ty; i < 32; i += 8) {
    const int t = t0 + i, c = c0 + tx;
    float2 z = make_float2(0.f, 0.f);
    if (t < jb && c < ncols) {
      z = S[(size_t)t * lds + c];
      if (F) put4(F, fplane, (size_t)(frow0 + t) * ldf + fcol0 + c, z, fmt, sc);
    }
    tile[i][tx] = z;
  }
  if (!T) return;
  __syncthreads();
  for (int i = ty; i < 32; i += 8) {
    const int c = c0 + i, t = t0 + tx;
    if (c < ncols) put4(T, tplane, (size_t)(trow0 + c) * RMAT_MAX_NB + tk0 + t, tile[tx][i], fmt, scT);
  }
}

// Left interchanges on the split factor planes (tensor path): block blk's row moves
// applied to K-columns 0..k0 of F (the L parts of all earlier blocks), so F holds L
// in the final row order (P A = L U) that the forward solve uses after one gather of
// the right-hand sides.  The complex64 factor C keeps the deferred layout.
// One CTA per 32 columns: moved rows gathered to shared memory, then written back.
template <class E>
__global__ void __launch_bounds__(256)
permute_fpl_left_kernel(E* __restrict__ F, int ldf, size_t fplane, int k0,
                        const int* __restrict__ rows, const int* __restrict__ src,
                        const int* __restrict__ cnt, int blk, int nbp) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  E* vals = reinterpret_cast<E*>(smem_raw);  // [2 * nbp][32]
  const int c0 = blockIdx.x * 32, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int n_q = cnt[blk];
  const int* rw = rows + (size_t)blk * 2 * nbp;
  const int* sr = src + (size_t)blk * 2 * nbp;
  const int col = c0 + lane;
  for (int pl = 0; pl < 4; ++pl) {
    E* Fp = F + pl * fplane;
    for (int q = warp; q < n_q; q += 8)
      if (col < k0) vals[q * 32 + lane] = Fp[(size_t)rw[sr[q]] * ldf + col];
    __syncthreads();
    for (int q = warp; q < n_q; q += 8)
      if (col < k0) Fp[(size_t)rw[q] * ldf + col] = vals[q * 32 + lane];
    __syncthreads();
  }
}

// Composed row permutation of all blocks (applied in order): pf[i] = the original row
// whose content ends at position i.  One CTA; tmp holds one block's moved entries.
__global__ void __launch_bounds__(256)
compose_perm_kernel(int n, int nb, const int* __restrict__ rows, const int* __restrict__ src,
                    const int* __restrict__ cnt, int* __restrict__ pf) {
  __shared__ int tmp[2 * RMAT_MAX_NB];
  for (int i = threadIdx.x; i < n; i += 256) pf[i] = i;
  __syncthreads();
  const int nblk = (n + nb - 1) / nb;
  for (int b = 0; b < nblk; ++b) {
    const int* rw = rows + (size_t)b * 2 * nb;
    const int* sr = src + (size_t)b * 2 * nb;
    const int m = cnt[b];
    for (int q = threadIdx.x; q < m; q += 256) tmp[q] = pf[rw[sr[q]]];
    __syncthreads();
    for (int q = threadIdx.x; q < m; q += 256) pf[rw[q]] = tmp[q];
    __syncthreads();
  }
}

// Bt[i] = B[pf[i]] (rows of nrhs complex64), then the caller copies Bt back.
__global__ void row_gather_kernel(const float2* __restrict__ B, float2* __restrict__ Bt, int n,
                                  int nrhs, const int* __restrict__ pf,
                                  const int* __restrict__ skip) {
  if (skip && *skip) return;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < (size_t)n * nrhs;
       e += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / nrhs), cc = (int)(e % nrhs);
    Bt[e] = B[(size_t)pf[i] * nrhs + cc];
  }
}

// A solved right-hand-side block (jb rows of S, ncols columns) -> transposed planes
// Y[c][t], zero-filled for jb <= t < round_up(jb, 32); one warp per column, so the
// column's scale (fmt 1) is a warp reduction; ycs[c] = 1/s.
__global__ void __launch_bounds__(256)
split_y_kernel(const float2* __restrict__ S, int lds, int jb, int ncols, void* __restrict__ Y,
               size_t yplane, int fmt, float* __restrict__ ycs, const int* __restrict__ skip) {
  if (skip && *skip) return;
  const int c = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (c >= ncols) return;
  const int kpad = (jb + 31) / 32 * 32;
  float m = 0.f;
  for (int t = lane; t < jb; t += 32) m = fmaxf(m, cmaxabs(S[(size_t)t * lds + c]));
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  const float sc = fmt == 1 ? pow2_scale(m) : 1.f;
  if (ycs && lane == 0) ycs[c] = 1.f / sc;
  for (int t = lane; t < kpad; t += 32) {
    const float2 z = t < jb ? S[(size_t)t * lds + c] : make_float2(0.f, 0.f);
    put4(Y, yplane, (size_t)c * RMAT_MAX_NB + t, z, fmt, sc);
  }
}

// ---- SIMT complex GEMM: C -= A B (all row-major) -----------------------------
constexpr int GB_M = 64, GB_N = 64, GB_K = 16;

template <class T>
__global__ void __launch_bounds__(256)
cgemm_sub_kernel(int M, int N, int K, const cplx<T>* __restrict__ A, int lda,
                 const cplx<T>* __restrict__ B, int ldb, cplx<T>* __restrict__ C, int ldc,
                 const int* __restrict__ skip) {
  using C2 = cplx<T>;
  if (skip && *skip) return;
  __shared__ C2 As[GB_K][GB_M + 1];
  __shared__ C2 Bs[GB_K][GB_N];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int m0 = blockIdx.y * GB_M, n0 = blockIdx.x * GB_N;
  C2 acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = mkc<T>(0, 0);
  for (int kk = 0; kk < K; kk += GB_K) {
#pragma unroll
    for (int e = tid; e < GB_M * GB_K; e += 256) {
      const int m = e / GB_K, k = e % GB_K;
      const int gm = m0 + m, gk = kk + k;
      As[k][m] = (gm < M && gk < K) ? A[(size_t)gm * lda + gk] : mkc<T>(0, 0);
    }
#pragma unroll
    for (int e = tid; e < GB_K * GB_N; e += 256) {
      const int k = e / GB_N, nn = e % GB_N;
      const int gk = kk + k, gn = n0 + nn;
      Bs[k][nn] = (gk < K && gn < N) ? B[(size_t)gk * ldb + gn] : mkc<T>(0, 0);
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < GB_K; ++k) {
      C2 a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[k][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[k][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) cadd_mul<T>(acc[i][j], a[i], b[j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int gm = m0 + ty + 16 * i;
    if (gm >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gn = n0 + tx + 16 * j;
      if (gn >= N) continue;
      C2 c = C[(size_t)gm * ldc + gn];
      c.x -= acc[i][j].x;
      c.y -= acc[i][j].y;
      C[(size_t)gm * ldc + gn] = c;
    }
  }
}

// ---- solve kernels (right-hand sides row-major, ldb) -------------------------
// Triangular solve on a jb x jb diagonal block for 32 right-hand-side columns
// per CTA (lane = column).  The diagonal block is first staged in shared memory
// (coalesced), so the dependent inner products read shared memory only.  Rows
// are processed in groups of 8 (one per warp): each warp accumulates the
// contributions of all rows solved before its group in parallel, then warp 0
// finishes the 8 x 8 triangle sequentially.
// LOWER: unit lower, rows top-down; else upper (divide by the diagonal), bottom-up.
template <class T, bool LOWER>
__global__ void __launch_bounds__(256)
trsm_block_rhs_kernel(const cplx<T>* __restrict__ A, int ld, int k0, int jb,
                      cplx<T>* __restrict__ B, int ldb, int nrhs, const int* __restrict__ skip) {
  using C2 = cplx<T>;
  if (skip && *skip) return;
  extern __shared__ unsigned char smem_raw[];
  C2* xs = reinterpret_cast<C2*>(smem_raw);  // [jb][32]
  C2* Ls = xs + (size_t)jb * 32;               // [jb][jb + 1]
  const int lds = jb + 1;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int col = blockIdx.x * 32 + lane;
  const bool act = col < nrhs;
  // stage the diagonal block: 8 independent loads in flight per thread
  for (int e0 = threadIdx.x; e0 < jb * jb; e0 += 256 * 8) {
    C2 v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int e = e0 + u * 256;
      if (e < jb * jb) {
        const int i = e / jb, t = e - i * jb;
        v[u] = A[(size_t)(k0 + i) * ld + k0 + t];
      }
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int e = e0 + u * 256;
      if (e < jb * jb) {
        const int i = e / jb, t = e - i * jb;
        Ls[i * lds + t] = v[u];
      }
    }
  }
  __syncthreads();
  const int ngroups = (jb + 7) / 8;
  for (int g = 0; g < ngroups; ++g) {
    const int li = LOWER ? g * 8 + warp : jb - 1 - (g * 8 + warp);
    const bool rowok = (g * 8 + warp) < jb;
    if (rowok) {
      C2 acc = act ? B[(size_t)(k0 + li) * ldb + col] : mkc<T>(0, 0);
      const C2* Lr = Ls + li * lds;
      if (LOWER) {
        for (int t = 0; t < g * 8; ++t) csub_mul<T>(acc, Lr[t], xs[t * 32 + lane]);
      } else {
        for (int t = jb - g * 8; t < jb; ++t) csub_mul<T>(acc, Lr[t], xs[t * 32 + lane]);
      }
      xs[li * 32 + lane] = acc;
    }
    __syncthreads();
    if (warp == 0) {
      for (int w = 0; w < 8 && g * 8 + w < jb; ++w) {
        const int ri = LOWER ? g * 8 + w : jb - 1 - (g * 8 + w);
        const C2* Lr = Ls + ri * lds;
        C2 acc = xs[ri * 32 + lane];
        for (int w2 = 0; w2 < w; ++w2) {
          const int tj = LOWER ? g * 8 + w2 : jb - 1 - (g * 8 + w2);
          csub_mul<T>(acc, Lr[tj], xs[tj * 32 + lane]);
        }
        if (!LOWER) acc = cdiv<T>(acc, Lr[ri]);
        xs[ri * 32 + lane] = acc;
      }
    }
    __syncthreads();
  }
  if (act)
    for (int i = warp; i < jb; i += 8) B[(size_t)(k0 + i) * ldb + col] = xs[i * 32 + lane];
}

// Fused block solve for a block of exactly JB rows (JB in {32, 64, 128}),
// 32 right-hand-side columns per CTA (lane = column), 8 warps:
//   1. stage the diagonal block (L11 unit lower, or U11) in shared memory;
//   2. with a permutation list: gather the involved rows through the block's net
//      source map (the interchanges applied), write the rows below the block back;
//   3. right-looking substitution with the block's rows in registers (warp w
//      owns solve positions w, w+8, ...): per step the owner publishes x_s,
//      then every warp subtracts L[i][s] x_s from its remaining rows;
//   4. write the solved rows, and (float, Y != nullptr) their TF32 split
//      planes transposed, the B operand of the tensor-core block update.
template <class T, bool LOWER, int JB>
__global__ void __launch_bounds__(256)
solve_block_kernel(const cplx<T>* __restrict__ A, int ld, int k0, cplx<T>* __restrict__ B,
                   int ldb, int ncols, int nbp, const int* __restrict__ prow,
                   const int* __restrict__ psrc, const int* __restrict__ pcnt,
                   void* __restrict__ Y, size_t yplane, size_t bstride, int fmt,
                   float* __restrict__ ycs, const int* __restrict__ skip) {
  using C2 = cplx<T>;
  if (skip && *skip) return;
  if (bstride) {  // batched over diagonal blocks (inversion): block blockIdx.y, B rows 0..JB-1
    k0 = blockIdx.y * nbp;
    B += (size_t)blockIdx.y * bstride - (size_t)k0 * ldb;
  }
  constexpr int RPW = JB / 8;
  constexpr int LDS = JB + 2;  // 16-byte aligned rows for the asynchronous copy
  constexpr int CPR = JB * (int)sizeof(C2) / 16;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C2* Ls = reinterpret_cast<C2*>(smem_raw);  // [JB][LDS]
  C2* vals = Ls + JB * LDS;                  // [2*JB][32] gather; reused as xs [JB][33]
  C2* xs = vals;
  C2* dinv = vals + 2 * JB * 32;             // [JB]
  int* rows = reinterpret_cast<int*>(dinv + JB);  // [2*JB]
  int* idx = rows + 2 * JB;                  // [2*JB] net source slots
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int col = blockIdx.x * 32 + lane;
  const bool act = col < ncols;

  // diagonal block -> shared memory, every 16-byte copy in flight at once
  for (int q = threadIdx.x; q < JB * CPR; q += 256) {
    const int r = q / CPR, h = q - r * CPR;
    const unsigned dst = (unsigned)__cvta_generic_to_shared(
        reinterpret_cast<unsigned char*>(Ls + (size_t)r * LDS) + 16 * h);
    const unsigned char* sp = reinterpret_cast<const unsigned char*>(A + (size_t)(k0 + r) * ld + k0) + 16 * h;
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(sp) : "memory");
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
  int cnt = JB;
  if (prow) {
    const int blk = k0 / nbp;
    cnt = pcnt[blk];
    for (int q = threadIdx.x; q < cnt; q += 256) {
      rows[q] = prow[(size_t)blk * 2 * nbp + q];
      idx[q] = psrc[(size_t)blk * 2 * nbp + q];  // net source slot of slot q
    }
  } else {
    for (int q = threadIdx.x; q < JB; q += 256) {
      rows[q] = k0 + q;
      idx[q] = q;
    }
  }
  __syncthreads();
  // permuted gather: slot q receives the original content of slot idx[q]
#pragma unroll 4
  for (int q = warp; q < cnt; q += 8)
    vals[q * 32 + lane] = act ? B[(size_t)rows[idx[q]] * ldb + col] : mkc<T>(0, 0);
  asm volatile("cp.async.wait_group 0;" ::: "memory");
  __syncthreads();
  if (!LOWER) {
    for (int q = threadIdx.x; q < JB; q += 256) dinv[q] = cdiv<T>(mkc<T>(1, 0), Ls[q * LDS + q]);
    __syncthreads();
  }
  if (prow)
    for (int q = JB + warp; q < cnt; q += 8)
      if (act) B[(size_t)rows[q] * ldb + col] = vals[q * 32 + lane];
  C2 b[RPW];
#pragma unroll
  for (int r = 0; r < RPW; ++r) {
    const int sp = r * 8 + warp;
    b[r] = vals[(LOWER ? sp : JB - 1 - sp) * 32 + lane];
  }
  __syncthreads();  // vals is reused as xs below
  for (int sp = 0; sp < JB; ++sp) {
    const int is = LOWER ? sp : JB - 1 - sp;
    if (warp == (sp & 7)) {
      const int rs = sp >> 3;
      C2 x = b[0];
#pragma unroll
      for (int r = 1; r < RPW; ++r)
        if (r == rs) x = b[r];
      if (!LOWER) x = cmul<T>(x, dinv[is]);
      xs[is * 33 + lane] = x;
    }
    __syncthreads();
    const C2 xv = xs[is * 33 + lane];
#pragma unroll
    for (int r = 0; r < RPW; ++r) {
      const int s2 = r * 8 + warp;
      if (s2 > sp) csub_mul<T>(b[r], Ls[(LOWER ? s2 : JB - 1 - s2) * LDS + is], xv);
    }
  }
  __syncthreads();
  if (act)
    for (int i = warp; i < JB; i += 8) B[(size_t)(k0 + i) * ldb + col] = xs[i * 33 + lane];
  if (Y) {
    for (int cc = warp; cc < 32; cc += 8) {
      const int gc = blockIdx.x * 32 + cc;
      if (gc >= ncols) continue;
      float m = 0.f;
      for (int i = lane; i < JB; i += 32) {
        const C2 z = xs[i * 33 + cc];
        m = fmaxf(m, fmaxf(fabsf((float)z.x), fabsf((float)z.y)));
      }
      for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
      const float sc = fmt == 1 ? pow2_scale(m) : 1.f;
      if (ycs && lane == 0) ycs[gc] = 1.f / sc;
      for (int i = lane; i < JB; i += 32) {
        const C2 z = xs[i * 33 + cc];
        put4(Y, yplane, (size_t)gc * RMAT_MAX_NB + i, make_float2((float)z.x, (float)z.y), fmt, sc);
      }
    }
  }
}

template <class T>
__global__ void identity_blocks_kernel(cplx<T>* __restrict__ D, int JB, size_t total) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)((e / JB) % JB), j = (int)(e % JB);
    D[e] = mkc<T>(i == j ? (T)1 : (T)0, (T)0);
  }
}

// Solve-path block application with an inverted diagonal block:
//   Y = Dinv * B_k   (B_k = rows k0..k0+JB-1 of B after the block's interchanges,
//                     gathered through the net source map when one is given),
// Y written back over B_k and, when Y planes are requested, as TF32 split planes
// transposed (B operand of the tensor-core block update).
// One cluster of JB/16 CTAs owns 16 right-hand-side columns; CTA s of the cluster
// gathers permutation slots 32s..32s+31 and computes output rows 16s..16s+15.
// Every read of B happens before the first cluster barrier and every write after
// the second, and no two clusters touch the same column, so the in-place update
// has no race.
// One complex entry of split operand planes (fmt 0: TF32 hi/lo as fp32 words, 1: FP16
// hi/lo carrying a power-of-two scale, undone by the caller): hi + lo per real part.
__device__ __forceinline__ float2 get4(const void* base, size_t plane, size_t o, int fmt) {
  if (fmt == 0) {
    const float* b = reinterpret_cast<const float*>(base);
    return make_float2(b[o] + b[plane + o], b[2 * plane + o] + b[3 * plane + o]);
  }
  const __half* b = reinterpret_cast<const __half*>(base);
  return make_float2(__half2float(b[o]) + __half2float(b[plane + o]),
                     __half2float(b[2 * plane + o]) + __half2float(b[3 * plane + o]));
}

// The solves' look-ahead update of the next step's rows, fused into the diagonal-block
// application that produces its right operand: B[row0 + r, cols] -= F[row0 + r,
// kcol0 .. kcol0 + JB) * Y for r < nrows, Y the block's solution rows (JB x 16 per
// cluster, gathered from the CTAs' shared memory), F the factor's split planes (the
// final row order of the tensor path: L rows of the next block in the forward sweep,
// U rows of the block above in the backward sweep, FP16 planes scaled per rs_div rows
// by rowscale).  The far rows' update may still be reduce-adding into these rows from
// the side stream, so the subtraction is atomic.
struct NearUpd {
  const void* F = nullptr;  // null: no fused update
  size_t fplane = 0;
  int ldf = 0, fmt = 0;
  int row0 = 0, nrows = 0, kcol0 = 0;
  const float* rowscale = nullptr;
  int rs_div = 1;
};

template <int JB>
__global__ void __cluster_dims__(1, JB / 16, 1) __launch_bounds__(256)
apply_inv_kernel(const float2* __restrict__ Dinv, int k0, int nbp, float2* __restrict__ B,
                 int ldb, int ncols, const int* __restrict__ prow, const int* __restrict__ psrc,
                 const int* __restrict__ pcnt, void* __restrict__ Yp, size_t yplane, int fmt,
                 float* __restrict__ ycs, const int* __restrict__ skip, const NearUpd nu) {
  namespace cg = cooperative_groups;
  if (skip && *skip) return;  // uniform over the cluster: no CTA reaches a cluster barrier
  constexpr int CW = 16;          // columns per cluster
  constexpr int SL = 32;          // permutation slots gathered per CTA (2*JB over JB/16 CTAs)
  constexpr int LDD = JB + 2;     // 16-byte aligned rows; the two rows a warp reads use different banks
  constexpr int CPR = JB * 8 / 16;
  cg::cluster_group cluster = cg::this_cluster();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* Ds = reinterpret_cast<float2*>(smem_raw);  // [16][LDD] rows 16s.. of the inverse
  float2* vloc = Ds + 16 * LDD;                     // [SL][CW] own gathered slots
  float2* vk = vloc + SL * CW;                      // [JB][CW] permuted B_k (all slots < JB)
  float2* ys = vk + JB * CW;                        // [16][CW+1] output rows
  int* rows = reinterpret_cast<int*>(ys + 16 * (CW + 1));  // [2*JB]
  int* src = rows + 2 * JB;                                // [2*JB]
  const int tid = threadIdx.x, s = blockIdx.y;
  const int cl = tid & (CW - 1), qq = tid >> 4;
  const int col = blockIdx.x * CW + cl;
  const bool act = col < ncols;
  const int blk = k0 / nbp;
  const float2* D = Dinv + ((size_t)blk * JB + 16 * s) * JB;
  for (int q = tid; q < 16 * CPR; q += 256) {
    const int r = q / CPR, h = q - r * CPR;
    const unsigned dst = (unsigned)__cvta_generic_to_shared(
        reinterpret_cast<unsigned char*>(Ds + (size_t)r * LDD) + 16 * h);
    const unsigned char* sp = reinterpret_cast<const unsigned char*>(D + (size_t)r * JB) + 16 * h;
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(sp) : "memory");
  }
  int cnt = JB;
  if (!prow && (ldb & 1) == 0 && (ncols & 1) == 0) {
    // no interchanges to apply: every CTA stages the whole B_k tile (JB rows x CW
    // columns) straight from global memory, 16 bytes (two columns) per copy
    const int c0 = blockIdx.x * CW;
    for (int e = tid; e < JB * (CW / 2); e += 256) {
      const int t = e / (CW / 2), h2 = 2 * (e % (CW / 2));
      float2* dst = vk + t * CW + h2;
      if (c0 + h2 < ncols) {
        const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
        const float2* sp = B + (size_t)(k0 + t) * ldb + c0 + h2;
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(sp) : "memory");
      } else {
        dst[0] = make_float2(0.f, 0.f);
        dst[1] = make_float2(0.f, 0.f);
      }
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    __syncthreads();
    cluster.sync();  // every CTA's read of B_k is done before any CTA writes its rows
  } else {
  asm volatile("cp.async.commit_group;" ::: "memory");
  if (prow) {
    cnt = pcnt[blk];
    for (int q = tid; q < cnt; q += 256) {
      rows[q] = prow[(size_t)blk * 2 * nbp + q];
      src[q] = psrc[(size_t)blk * 2 * nbp + q];
    }
  } else {
    for (int q = tid; q < JB; q += 256) {
      rows[q] = k0 + q;
      src[q] = q;
    }
  }
  __syncthreads();
  // gather: slot q receives the original content of slot src[q]
#pragma unroll
  for (int u = 0; u < SL / 16; ++u) {
    const int q = SL * s + qq + 16 * u;
    if (q < cnt)
      vloc[(qq + 16 * u) * CW + cl] = act ? B[(size_t)rows[src[q]] * ldb + col] : make_float2(0.f, 0.f);
  }
  cluster.sync();  // every gather (read of B) of the cluster is done
  for (int e = tid; e < JB * CW; e += 256) {
    const int t = e / CW;
    const float2* peer = cluster.map_shared_rank(vloc, t / SL);
    vk[e] = peer[(t % SL) * CW + (e % CW)];
  }
  asm volatile("cp.async.wait_group 0;" ::: "memory");
  cluster.sync();  // peers may now overwrite B and exit
  }
  if (prow && act) {
#pragma unroll
    for (int u = 0; u < SL / 16; ++u) {
      const int q = SL * s + qq + 16 * u;
      if (q >= JB && q < cnt) B[(size_t)rows[q] * ldb + col] = vloc[(qq + 16 * u) * CW + cl];
    }
  }
  const int ri = qq;  // output row 16s + ri, column cl
  float2 acc = make_float2(0.f, 0.f);
#pragma unroll 8
  for (int t = 0; t < JB; ++t) cadd_mul<float>(acc, Ds[ri * LDD + t], vk[t * CW + cl]);
  const int i = 16 * s + ri;
  if (act) B[(size_t)(k0 + i) * ldb + col] = acc;
  if (Yp || nu.F) {
    ys[ri * (CW + 1) + cl] = acc;
    __syncthreads();
  }
  if (Yp) {
    __shared__ float cmax[CW];
    const int cc = tid >> 4, ii = tid & 15;
    float sc = 1.f;
    if (fmt == 1) {
      // column scale: max over the cluster's JB rows (16 per CTA, exchanged via DSMEM)
      if (tid < CW) {
        float m = 0.f;
        for (int r = 0; r < 16; ++r) m = fmaxf(m, cmaxabs(ys[r * (CW + 1) + tid]));
        cmax[tid] = m;
      }
      cluster.sync();
      float m = 0.f;
      for (int q = 0; q < JB / 16; ++q) m = fmaxf(m, *cluster.map_shared_rank(&cmax[cc], q));
      sc = pow2_scale(m);
      if (s == 0 && ii == 0 && blockIdx.x * CW + cc < ncols) ycs[blockIdx.x * CW + cc] = 1.f / sc;
      cluster.sync();  // peers' cmax reads are done
    }
    // transposed planes: plane row = column, K index = i (16 consecutive i per column)
    const int gc = blockIdx.x * CW + cc;
    if (gc < ncols)
      put4(Yp, yplane, (size_t)gc * RMAT_MAX_NB + 16 * s + ii, ys[ii * (CW + 1) + cc], fmt, sc);
  }
  if (nu.F) {
    cluster.sync();  // every CTA's 16 solution rows are in its ys
    for (int e = tid; e < JB * CW; e += 256) {
      const int t = e / CW;
      const float2* peer = cluster.map_shared_rank(ys, t / 16);
      vk[e] = peer[(t % 16) * (CW + 1) + (e % CW)];
    }
    // rows 16 s + q JB .. of the next step's block (the inverse rows in Ds are done)
    for (int q0 = 16 * s; q0 < nu.nrows; q0 += JB) {
      __syncthreads();
      for (int e = tid; e < 16 * JB; e += 256) {
        const int r = e / JB, t = e - r * JB;
        float2 v = make_float2(0.f, 0.f);
        if (q0 + r < nu.nrows) {
          const int row = nu.row0 + q0 + r;
          v = get4(nu.F, nu.fplane, (size_t)row * nu.ldf + nu.kcol0 + t, nu.fmt);
          if (nu.rowscale) {
            const float sc = nu.rowscale[row / nu.rs_div];
            v.x *= sc;
            v.y *= sc;
          }
        }
        Ds[r * LDD + t] = v;
      }
      __syncthreads();
      float2 a0 = make_float2(0.f, 0.f), a1 = make_float2(0.f, 0.f);
#pragma unroll 8
      for (int t = 0; t < JB; t += 2) {
        cadd_mul<float>(a0, Ds[ri * LDD + t], vk[t * CW + cl]);
        cadd_mul<float>(a1, Ds[ri * LDD + t + 1], vk[(t + 1) * CW + cl]);
      }
      if (act && q0 + ri < nu.nrows) {
        float2* dst = B + (size_t)(nu.row0 + q0 + ri) * ldb + col;
        atomicAdd(&dst->x, -(a0.x + a1.x));
        atomicAdd(&dst->y, -(a0.y + a1.y));
      }
    }
    cluster.sync();  // the peers' reads of this CTA's ys are done before it exits
  }
}

template <int JB>
size_t apply_inv_smem() {
  return (size_t)(16 * (JB + 2) + 32 * 16 + JB * 16 + 16 * 17) * sizeof(float2) +
         (size_t)4 * JB * sizeof(int);
}

template <class T, int JB>
size_t solve_block_smem() {
  return (size_t)JB * (JB + 2) * sizeof(cplx<T>) + (size_t)2 * JB * 32 * sizeof(cplx<T>) +
         (size_t)JB * sizeof(cplx<T>) + (size_t)4 * JB * sizeof(int);
}

template <class T>
size_t trsm_smem(int jb) {
  return (size_t)jb * 32 * sizeof(cplx<T>) + (size_t)jb * (jb + 1) * sizeof(cplx<T>);
}

// ---- row interchanges as one permutation per block -----------------------------
// perm_prep_kernel (one warp per block of jb pivots): the jb sequential swaps
// rows (k0+t) <-> ipiv[k0+t] touch the block rows k0..k0+jb-1 and at most jb
// rows below.  The involved rows are listed once (block rows first, then the
// distinct rows below in first-use order) with, for each step t, the list slot
// of its pivot row; the list serves the trailing columns of the factorisation
// and every forward solve.  Out-of-range pivots (only after a panel that gave
// up on a bounded wait) become no-ops and raise the status word.
__global__ void perm_prep_kernel(const int* __restrict__ ipiv, int n, int nb, int k0_first,
                                 int* __restrict__ prow, int* __restrict__ pidx,
                                 int* __restrict__ pcnt, int* __restrict__ psrc,
                                 int* __restrict__ stat) {
  const int blk = blockIdx.x;
  const int k0 = k0_first + blk * nb;
  if (k0 >= n) return;
  const int jb = min(nb, n - k0);
  const int lane = threadIdx.x;
  int* rows = prow + (size_t)(k0 / nb) * 2 * nb;
  int* idx = pidx + (size_t)(k0 / nb) * nb;
  for (int t = lane; t < jb; t += 32) rows[t] = k0 + t;
  int nout = 0;
  for (int t = 0; t < jb; ++t) {
    int p = ipiv[k0 + t];
    int slot;
    if (p < k0 + t || p >= n) {
      if (lane == 0) atomicExch(&stat[ST_BADARG], 1);
      slot = t;
    } else if (p < k0 + jb) {
      slot = p - k0;
    } else {
      slot = -1;
      for (int q0 = 0; q0 < nout && slot < 0; q0 += 32) {
        const int q = q0 + lane;
        const bool hit = q < nout && rows[jb + q] == p;
        const unsigned m = __ballot_sync(0xffffffffu, hit);
        if (m) slot = jb + q0 + __ffs(m) - 1;
      }
      if (slot < 0) {
        slot = jb + nout;
        if (lane == 0) rows[slot] = p;
        ++nout;
      }
      __syncwarp();
    }
    if (lane == 0) idx[t] = slot;
  }
  if (lane == 0) pcnt[k0 / nb] = jb + nout;
  // net effect of the sequential swaps: slot q ends up holding the original
  // content of slot src[q] (simulated once here, so gathers need no replay)
  __syncwarp();
  int* src = psrc + (size_t)(k0 / nb) * 2 * nb;
  const int cnt = jb + nout;
  for (int q = lane; q < cnt; q += 32) src[q] = q;
  __syncwarp();
  if (lane == 0) {
    for (int t = 0; t < jb; ++t) {
      const int sl = idx[t];
      if (sl != t) {
        const int u = src[t];
        src[t] = src[sl];
        src[sl] = u;
      }
    }
  }
  __syncwarp();
}

// Apply block k0's permutation to ncols columns of B (rows of B are matrix rows):
// gather the involved rows into shared memory, replay the swaps there, write back.
template <class T>
__global__ void __launch_bounds__(256)
apply_perm_kernel(cplx<T>* __restrict__ B, int ldb, int ncols, int k0, int nb, int jb,
                  const int* __restrict__ prow, const int* __restrict__ pidx,
                  const int* __restrict__ pcnt, const int* __restrict__ skip) {
  using C2 = cplx<T>;
  if (skip && *skip) return;
  extern __shared__ unsigned char smem_raw[];
  C2* vals = reinterpret_cast<C2*>(smem_raw);                      // [2*nb][32]
  int* rows = reinterpret_cast<int*>(vals + (size_t)2 * nb * 32);  // [2*nb]
  int* idx = rows + 2 * nb;                                        // [nb]
  const int blk = k0 / nb;
  const int cnt = pcnt[blk];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int q = threadIdx.x; q < cnt; q += 256) rows[q] = prow[(size_t)blk * 2 * nb + q];
  for (int q = threadIdx.x; q < jb; q += 256) idx[q] = pidx[(size_t)blk * nb + q];
  __syncthreads();
  const int col = blockIdx.x * 32 + lane;
  const bool act = col < ncols;
  for (int q = warp; q < cnt; q += 8)
    if (act) vals[q * 32 + lane] = B[(size_t)rows[q] * ldb + col];
  __syncthreads();
  if (warp == 0) {
    for (int t = 0; t < jb; ++t) {
      const int s = idx[t];
      if (s != t) {
        const C2 u = vals[t * 32 + lane];
        vals[t * 32 + lane] = vals[s * 32 + lane];
        vals[s * 32 + lane] = u;
      }
    }
  }
  __syncthreads();
  for (int q = warp; q < cnt; q += 8)
    if (act) B[(size_t)rows[q] * ldb + col] = vals[q * 32 + lane];
}

template <class T>
size_t perm_smem(int nb) {
  return (size_t)2 * nb * 32 * sizeof(cplx<T>) + (size_t)3 * nb * sizeof(int);
}

// ---- FP64 complex GEMM C -= A B (row-major) on the FP64 tensor instruction ------
// mma.sync.m8n8k4.f64 (tcgen05 has no f64 kind): the complex product as three real
// products (3M): T1 = Ar Br, T2 = Ai Bi, T3 = (Ar + Ai)(Br + Bi), Re = T1 - T2,
// Im = T3 - T1 - T2, the operand sums formed in registers.  64 x 64 output tile per
// CTA, 16-deep K chunks staged as separate real / imaginary [k][64] planes (row pitch
// 72 doubles: a fragment load's 4 k-rows x 8 entries hit distinct bank slots); each of
// the 8 warps owns 32 x 16 (4 x 2 tiles of 8 x 8).
constexpr int ZG_T = 64, ZG_K = 16, ZG_LD = 72;

__device__ __forceinline__ void dmma_acc(double& d0, double& d1, double a, double b) {
  asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};"
               : "+d"(d0), "+d"(d1)
               : "d"(a), "d"(b));
}

__global__ void __launch_bounds__(256)
zgemm_sub_dmma_kernel(int M, int N, int K, const double2* __restrict__ A, int lda,
                      const double2* __restrict__ B, int ldb, double2* __restrict__ C, int ldc,
                      const int* __restrict__ skip) {
  if (skip && *skip) return;
  __shared__ double Ar[ZG_K][ZG_LD], Am[ZG_K][ZG_LD];  // A[m0 + m][k0 + k] -> [k][m]
  __shared__ double Br[ZG_K][ZG_LD], Bm[ZG_K][ZG_LD];  // B[k0 + k][n0 + n] -> [k][n]
  const int m0 = blockIdx.y * ZG_T, n0 = blockIdx.x * ZG_T;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int wm = (warp >> 2) * 32, wn = (warp & 3) * 16;
  const int g = lane >> 2, t = lane & 3;
  double t1[4][2][2], t2[4][2][2], t3[4][2][2];
#pragma unroll
  for (int p = 0; p < 4; ++p)
#pragma unroll
    for (int q = 0; q < 2; ++q)
#pragma unroll
      for (int h = 0; h < 2; ++h) t1[p][q][h] = t2[p][q][h] = t3[p][q][h] = 0.0;
  for (int k0 = 0; k0 < K; k0 += ZG_K) {
    for (int e = threadIdx.x; e < ZG_T * ZG_K; e += 256) {
      const int kk = e & (ZG_K - 1), mm = e >> 4;
      const int gm = m0 + mm, gk = k0 + kk;
      const double2 a = (gm < M && gk < K) ? A[(size_t)gm * lda + gk] : make_double2(0, 0);
      Ar[kk][mm] = a.x;
      Am[kk][mm] = a.y;
      const int kb = e >> 6, nn = e & (ZG_T - 1);
      const int gk2 = k0 + kb, gn = n0 + nn;
      const double2 b = (gk2 < K && gn < N) ? B[(size_t)gk2 * ldb + gn] : make_double2(0, 0);
      Br[kb][nn] = b.x;
      Bm[kb][nn] = b.y;
    }
    __syncthreads();
#pragma unroll
    for (int k4 = 0; k4 < ZG_K; k4 += 4) {
      double ar[4], ai[4], as[4], br[2], bi[2], bs[2];
#pragma unroll
      for (int p = 0; p < 4; ++p) {
        ar[p] = Ar[k4 + t][wm + 8 * p + g];
        ai[p] = Am[k4 + t][wm + 8 * p + g];
        as[p] = ar[p] + ai[p];
      }
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        br[q] = Br[k4 + t][wn + 8 * q + g];
        bi[q] = Bm[k4 + t][wn + 8 * q + g];
        bs[q] = br[q] + bi[q];
      }
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          dmma_acc(t1[p][q][0], t1[p][q][1], ar[p], br[q]);
          dmma_acc(t2[p][q][0], t2[p][q][1], ai[p], bi[q]);
          dmma_acc(t3[p][q][0], t3[p][q][1], as[p], bs[q]);
        }
    }
    __syncthreads();
  }
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    const int gm = m0 + wm + 8 * p + g;
    if (gm >= M) continue;
#pragma unroll
    for (int q = 0; q < 2; ++q)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int gn = n0 + wn + 8 * q + 2 * t + h;
        if (gn >= N) continue;
        double2* cp = C + (size_t)gm * ldc + gn;
        double2 v = *cp;
        v.x -= t1[p][q][h] - t2[p][q][h];
        v.y -= t3[p][q][h] - t1[p][q][h] - t2[p][q][h];
        *cp = v;
      }
  }
}

template <class T>
int gemm_sub(rmat_ctx c, int M, int N, int K, const cplx<T>* A, int lda, const cplx<T>* B,
             int ldb, cplx<T>* C, int ldc) {
  if (M <= 0 || N <= 0 || K <= 0) return RMAT_OK;
  if constexpr (sizeof(T) == 8) {
    dim3 grid(ceil_div(N, ZG_T), ceil_div(M, ZG_T));
    zgemm_sub_dmma_kernel<<<grid, 256, 0, c->stream>>>(M, N, K, A, lda, B, ldb, C, ldc, c->skip);
  } else {
    dim3 grid(ceil_div(N, GB_N), ceil_div(M, GB_M));
    cgemm_sub_kernel<T><<<grid, 256, 0, c->stream>>>(M, N, K, A, lda, B, ldb, C, ldc, c->skip);
  }
  c->launches++;
  RMAT_CU(cudaGetLastError());
  return RMAT_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
int panel_ctas_for(rmat_ctx c, int M) {
  int P = c->panel_ctas_param > 0 ? c->panel_ctas_param : c->sm_count;
  P = std::min(P, RMAT_MAX_PANEL_CTAS);
  P = std::min(P, std::max(1, ceil_div(M, 32)));
  while (ceil_div(M, P) > MAX_RPC) ++P;
  return P;
}

// Dynamic shared memory a panel CTA may stage: the device's opt-in maximum per
// block less 1 KB for the kernel's static shared variables.
size_t panel_smem_limit(rmat_ctx c) { return (size_t)c->smem_optin - 1024; }

template <class T>
size_t panel_smem(int rpc, int ldr, bool in_smem) {
  return (size_t)(2 * RMAT_MAX_NB + rpc) * sizeof(cplx<T>) +
         (in_smem ? (size_t)rpc * ldr * sizeof(cplx<T>) : 0);
}

template <class T>
size_t panel_cluster_smem(int jb, int rpc, int ldr) {
  return (size_t)(6 * jb + rpc + (size_t)rpc * ldr) * sizeof(cplx<T>);
}

// Largest cluster the cluster panel may use on this device (16 needs the
// non-portable size opt-in; 8 is portable); 0 if cluster launches are unavailable.
template <class T>
int panel_cluster_max(rmat_ctx c) {
  static int cs_max[2] = {-1, -1};
  int& m = cs_max[sizeof(T) == 8];
  if (m >= 0) return m;
  m = 0;
  const int smem = (int)panel_smem_limit(c);
  if (cudaFuncSetAttribute(panel_cluster_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           smem) != cudaSuccess ||
      cudaFuncSetAttribute(panel_cluster_kernel<T>,
                           cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
    cudaGetLastError();
    return m;
  }
  for (int cs = 16; cs >= 1; cs /= 2) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cs);
    cfg.blockDim = dim3(PANEL_THREADS);
    cfg.dynamicSmemBytes = (size_t)smem;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = cs;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int nclusters = 0;
    if (cudaOccupancyMaxActiveClusters(&nclusters, panel_cluster_kernel<T>, &cfg) == cudaSuccess &&
        nclusters > 0) {
      m = cs;
      break;
    }
    cudaGetLastError();
  }
  return m;
}

// Cluster size for a panel of M rows: about 128 rows per CTA (complex64) or 32
// (complex128: the rank-1 updates run at this part's FP64 rate, ~2 FMA per clock per
// SM, so they are spread over more SMs), up to the device's maximum; 0 when the rows
// do not fit the cluster's shared memory (grid variant).
template <class T>
int panel_cluster_size(rmat_ctx c, int M, int jb, int* rpc_out, int* ldr_out) {
  const int cmax = panel_cluster_max<T>(c);
  if (cmax == 0) return 0;
  const int per = sizeof(T) == 8 ? 32 : 128;
  int cs = 1;
  while (cs < cmax && ceil_div(M, cs) > per) cs *= 2;
  const int rpc = ceil_div(M, cs);
  const size_t limit = panel_smem_limit(c);
  int ldr = jb + 1;
  if (panel_cluster_smem<T>(jb, rpc, ldr) > limit) ldr = jb;
  if (panel_cluster_smem<T>(jb, rpc, ldr) > limit) return 0;
  *rpc_out = rpc;
  *ldr_out = ldr;
  return cs;
}

int panel_cluster_fits(rmat_ctx c, int precision, int M, int jb) {
  int rpc = 0, ldr = 0;
  return precision == RMAT_C128 ? panel_cluster_size<double>(c, M, jb, &rpc, &ldr)
                                : panel_cluster_size<float>(c, M, jb, &rpc, &ldr);
}

// la_ctas > 0: a look-ahead panel beside a far update that leaves it about that many
// SMs: grid variant on at most la_ctas CTAs (a cluster would need its CTAs free in one
// GPC at once).  No kernel it runs beside waits for it, so its CTAs that are not yet
// resident start when those kernels' CTAs retire.
template <class T>
int launch_panel(rmat_ctx c, cplx<T>* A, int ld, int k0, int n, int jb, int* ipiv, int la_ctas = 0) {
  const int M = n - k0;
  if (c->panel_ctas_param <= 0 && la_ctas <= 0) {  // rows fit one cluster's shared memory
    int rpc = 0, ldr = 0;
    const int cs = panel_cluster_size<T>(c, M, jb, &rpc, &ldr);
    if (cs > 0) {
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(cs);
      cfg.blockDim = dim3(PANEL_THREADS);
      cfg.dynamicSmemBytes = panel_cluster_smem<T>(jb, rpc, ldr);
      cfg.stream = c->stream;
      cudaLaunchAttribute at[1];
      at[0].id = cudaLaunchAttributeClusterDimension;
      at[0].val.clusterDim.x = cs;
      at[0].val.clusterDim.y = 1;
      at[0].val.clusterDim.z = 1;
      cfg.attrs = at;
      cfg.numAttrs = 1;
      KTimer kt(c, KT_PANEL);
      RMAT_CU(cudaLaunchKernelEx(&cfg, panel_cluster_kernel<T>, A, ld, k0, n, jb, ipiv, c->dstat,
                                 rpc, ldr));
      kt.end();
      c->launches++;
      return RMAT_OK;
    }
  }
  int P = panel_ctas_for(c, M);
  if (la_ctas > 0) {
    P = std::min({la_ctas, RMAT_MAX_PANEL_CTAS, std::max(1, ceil_div(M, 32))});
    while (ceil_div(M, P) > MAX_RPC) ++P;
  }
  const int rpc = ceil_div(M, P);
  int ldr = jb + 1;
  const size_t limit = panel_smem_limit(c);
  if (panel_smem<T>(rpc, ldr, true) > limit) ldr = jb;
  const bool in_smem = panel_smem<T>(rpc, ldr, true) <= limit;
  const size_t smem = panel_smem<T>(rpc, ldr, in_smem);
  static bool attr_set[2] = {false, false};
  if (!attr_set[sizeof(T) == 8]) {
    RMAT_CU(cudaFuncSetAttribute(panel_kernel<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)limit));
    // the SM's unified memory as shared memory, so a look-ahead panel CTA fits beside a
    // far update's CTA
    RMAT_CU(cudaFuncSetAttribute(panel_kernel<T, true>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared));
    RMAT_CU(cudaFuncSetAttribute(panel_kernel<T, false>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)panel_smem<T>(MAX_RPC, 0, false)));
    attr_set[sizeof(T) == 8] = true;
  }
  // arrival counter and the candidate records (generation 0: nothing published)
  RMAT_CU(cudaMemsetAsync(c->ps.bar, 0, 256 + 2 * RMAT_MAX_PANEL_CTAS * sizeof(double), c->stream));
  PanelScratch ps = c->ps;
  long long spin = c->spin_limit;
  int* stat = c->dstat;
  void* args[] = {&A,   &ld,   (void*)&k0,  (void*)&n, (void*)&jb, &ipiv,
                  &stat, &ps,   (void*)&rpc, &ldr,      &spin};
  const void* kern = in_smem ? (const void*)panel_kernel<T, true> : (const void*)panel_kernel<T, false>;
  KTimer kt(c, KT_PANEL);
  RMAT_CU(cudaLaunchCooperativeKernel(kern, dim3(P), dim3(PANEL_THREADS), args, smem, c->stream));
  kt.end();
  c->launches++;
  return RMAT_OK;
}

// Largest block width whose diagonal block fits the TRSM's shared memory.
template <class T> constexpr int max_nb() { return sizeof(T) == 4 ? 128 : 64; }

template <class T>
int set_trsm_attrs() {
  static bool done = false;
  if (done) return RMAT_OK;
  const int smem_max = (int)trsm_smem<T>(max_nb<T>());
  RMAT_CU(cudaFuncSetAttribute(trsm_block_rhs_kernel<T, true>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, smem_max));
  RMAT_CU(cudaFuncSetAttribute(trsm_block_rhs_kernel<T, false>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, smem_max));
  RMAT_CU(cudaFuncSetAttribute(apply_perm_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)perm_smem<T>(max_nb<T>())));
  done = true;
  return RMAT_OK;
}

template <class T>
int apply_perm(rmat_ctx c, const LUPerm& pm, cplx<T>* B, int ldb, int ncols, int k0, int nb, int jb) {
  apply_perm_kernel<T><<<ceil_div(ncols, 32), 256, perm_smem<T>(nb), c->stream>>>(
      B, ldb, ncols, k0, nb, jb, pm.rows, pm.idx, pm.cnt, c->skip);
  c->launches++;
  RMAT_CU(cudaGetLastError());
  return RMAT_OK;
}

// Fused block solve when jb is a supported width; *done = false otherwise.
template <class T, bool LOWER, int JB>
int launch_solve_block(rmat_ctx c, const LUPerm* pm, const cplx<T>* A, int ld, int k0, int nb,
                       cplx<T>* B, int ldb, int ncols, void* Y) {
  static bool attr = false;
  const size_t smem = solve_block_smem<T, JB>();
  if (!attr) {
    RMAT_CU(cudaFuncSetAttribute(solve_block_kernel<T, LOWER, JB>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    attr = true;
  }
  solve_block_kernel<T, LOWER, JB><<<ceil_div(ncols, 32), 256, smem, c->stream>>>(
      A, ld, k0, B, ldb, ncols, nb, pm ? pm->rows : nullptr, pm ? pm->src : nullptr,
      pm ? pm->cnt : nullptr, Y, (size_t)RMAT_YPL_ROWS * RMAT_MAX_NB, (size_t)0,
      rmat_plane_fmt(c->precision), Y ? rmat_ycs_cur(c) : nullptr, c->skip);
  c->launches++;
  RMAT_CU(cudaGetLastError());
  return RMAT_OK;
}

template <class T, bool LOWER>
int solve_block(rmat_ctx c, const LUPerm* pm, const cplx<T>* A, int ld, int k0, int nb, int jb,
                cplx<T>* B, int ldb, int ncols, void* Y, bool* done) {
  *done = true;
  if (jb == 32) return launch_solve_block<T, LOWER, 32>(c, pm, A, ld, k0, nb, B, ldb, ncols, Y);
  if (jb == 64) return launch_solve_block<T, LOWER, 64>(c, pm, A, ld, k0, nb, B, ldb, ncols, Y);
  if constexpr (sizeof(T) == 4)
    if (jb == 128) return launch_solve_block<T, LOWER, 128>(c, pm, A, ld, k0, nb, B, ldb, ncols, Y);
  *done = false;
  return RMAT_OK;
}

// Inverses of all full-width diagonal blocks (L11^-1 unit lower, U11^-1 upper) of a
// complex64 factor, for the solve path: identity, then the batched block solve.
template <int JB>
int invert_diag_blocks(rmat_ctx c, const float2* A, int ld, int n, int nb, bool lower_done = false) {
  const int nfull = n / nb;
  c->inv_blocks = 0;
  if (nfull == 0) return RMAT_OK;
  const size_t per = (size_t)JB * JB, total = per * nfull;
  RMAT_CHECK(rmat_grow(c, &c->Dinv, &c->Dinv_cap, 2 * total * sizeof(float2)));
  float2* Linv = reinterpret_cast<float2*>(c->Dinv);
  float2* Uinv = Linv + total;
  // lower_done: the L11^-1 blocks were formed during the factorisation (U12 products)
  float2* first = lower_done ? Uinv : Linv;
  const size_t cnt = lower_done ? total : 2 * total;
  identity_blocks_kernel<float><<<std::min(c->sm_count * 4, ceil_div((long long)cnt, 256)), 256,
                                  0, c->stream>>>(first, JB, cnt);
  c->launches++;
  static bool attr[2] = {false, false};
  const size_t smem = solve_block_smem<float, JB>();
  if (!attr[JB == 128]) {
    RMAT_CU(cudaFuncSetAttribute(solve_block_kernel<float, true, JB>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    RMAT_CU(cudaFuncSetAttribute(solve_block_kernel<float, false, JB>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    attr[JB == 128] = true;
  }
  const dim3 grid(JB / 32, nfull);
  if (!lower_done) {
    solve_block_kernel<float, true, JB><<<grid, 256, smem, c->stream>>>(
        A, ld, 0, Linv, JB, JB, nb, nullptr, nullptr, nullptr, nullptr, 0, per, 0, nullptr, nullptr);
    c->launches++;
  }
  solve_block_kernel<float, false, JB><<<grid, 256, smem, c->stream>>>(
      A, ld, 0, Uinv, JB, JB, nb, nullptr, nullptr, nullptr, nullptr, 0, per, 0, nullptr, nullptr);
  c->launches++;
  RMAT_CU(cudaGetLastError());
  c->inv_blocks = nfull;
  c->inv_nb = nb;
  return RMAT_OK;
}

// ---- 256-row solve steps ----------------------------------------------------
// The inverses of pairs of 128-row diagonal blocks, for solve sweeps of half as many
// dependent steps:
//   [L1 0; L21 L2]^-1 = [L1^-1 0; -L2^-1 L21 L1^-1  L2^-1],
//   [U1 U12; 0 U2]^-1 = [U1^-1  -U1^-1 U12 U2^-1; 0 U2^-1],
// from the 128-row inverses already formed, L21 from the factor planes (final row
// order, hi + lo), U12 from C (rows of a block are final after its own panel).

namespace {

// Scratch blocks of pair q: L21 and U12 (128 x 128 each), the diagonal sub-blocks of
// both 256-row inverses, zeros above / below them.
template <class E>
__global__ void __launch_bounds__(256)
pair_gather_kernel(const float2* __restrict__ A, int ld, const E* __restrict__ F, int ldf,
                   size_t fplane, const float2* __restrict__ Linv, const float2* __restrict__ Uinv,
                   float2* __restrict__ L21, float2* __restrict__ U12, float2* __restrict__ L2,
                   float2* __restrict__ U2) {
  constexpr int H = 128, P = 256;
  const int q = blockIdx.y;
  const size_t k0 = (size_t)q * P;
  for (int e = blockIdx.x * 256 + threadIdx.x; e < H * H; e += gridDim.x * 256) {
    const int i = e / H, j = e - i * H;
    const size_t fo = (k0 + H + i) * ldf + k0 + j;
    L21[(size_t)q * H * H + e] =
        make_float2((float)F[fo] + (float)F[fplane + fo], (float)F[2 * fplane + fo] + (float)F[3 * fplane + fo]);
    U12[(size_t)q * H * H + e] = A[(k0 + i) * ld + k0 + H + j];
    const float2 z = make_float2(0.f, 0.f);
    float2* l = L2 + (size_t)q * P * P;
    float2* u = U2 + (size_t)q * P * P;
    l[(size_t)i * P + j] = Linv[(size_t)(2 * q) * H * H + e];
    l[(size_t)(H + i) * P + H + j] = Linv[(size_t)(2 * q + 1) * H * H + e];
    l[(size_t)i * P + H + j] = z;
    u[(size_t)i * P + j] = Uinv[(size_t)(2 * q) * H * H + e];
    u[(size_t)(H + i) * P + H + j] = Uinv[(size_t)(2 * q + 1) * H * H + e];
    u[(size_t)(H + i) * P + j] = z;
  }
}

// Out[b] = alpha A[b] B[b], 128 x 128 x 128 complex64 per b (B staged in shared memory):
// thread t forms row t / 2, columns 64 (t % 2) .. +63.
__global__ void __launch_bounds__(256)
pair_gemm_kernel(const float2* __restrict__ A, size_t sa, const float2* __restrict__ Bm,
                 size_t sb, float2* __restrict__ Out, size_t so, int ldo, float alpha) {
  constexpr int H = 128;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* Bs = reinterpret_cast<float2*>(smem_raw);
  const int b = blockIdx.x, tid = threadIdx.x;
  const float2* Ab = A + (size_t)b * sa;
  const float2* Bb = Bm + (size_t)b * sb;
  for (int e = tid; e < H * H; e += 256) Bs[e] = Bb[e];
  __syncthreads();
  const int i = tid >> 1, j0 = (tid & 1) * 64;
  float2 acc[64];
#pragma unroll
  for (int jj = 0; jj < 64; ++jj) acc[jj] = make_float2(0.f, 0.f);
  for (int k = 0; k < H; ++k) {
    const float2 a = Ab[(size_t)i * H + k];
#pragma unroll
    for (int jj = 0; jj < 64; ++jj) cadd_mul<float>(acc[jj], a, Bs[k * H + j0 + jj]);
  }
  float2* o = Out + (size_t)b * so + (size_t)i * ldo + j0;
#pragma unroll
  for (int jj = 0; jj < 64; ++jj) o[jj] = make_float2(alpha * acc[jj].x, alpha * acc[jj].y);
}

}  // namespace

// After invert_diag_blocks<128> of a tensor-path factor: the 256-row inverses of every
// pair of full blocks into c->Dinv2 ([L pairs][256][256], then [U pairs][256][256]).
int invert_pair_blocks(rmat_ctx c, const float2* A, int ld, int n) {
  constexpr int H = 128, P = 256;
  c->inv_pairs = 0;
  c->pairs_off = false;  // a new factorisation: try the pair steps again
  const int npairs = c->inv_blocks / 2;
  if (c->solve_blk == 128 || c->inv_nb != H || npairs == 0 || !c->Fpl) return RMAT_OK;
  const size_t per = (size_t)P * P, hh = (size_t)H * H;
  RMAT_CHECK(rmat_grow(c, &c->Dinv2, &c->Dinv2_cap, 2 * per * npairs * sizeof(float2)));
  RMAT_CHECK(rmat_grow(c, &c->Pscr, &c->Pscr_cap, 3 * hh * npairs * sizeof(float2)));
  float2* L2 = reinterpret_cast<float2*>(c->Dinv2);
  float2* U2 = L2 + per * npairs;
  float2* L21 = reinterpret_cast<float2*>(c->Pscr);
  float2* U12 = L21 + hh * npairs;
  float2* T = U12 + hh * npairs;
  const float2* Linv = reinterpret_cast<const float2*>(c->Dinv);
  const float2* Uinv = Linv + hh * c->inv_blocks;
  const size_t fplane = (size_t)n * c->ld;
  const dim3 gg(16, npairs);
  if (rmat_plane_fmt(c->precision) == 1)
    pair_gather_kernel<__half><<<gg, 256, 0, c->stream>>>(
        A, ld, reinterpret_cast<const __half*>(c->Fpl), c->ld, fplane, Linv, Uinv, L21, U12, L2, U2);
  else
    pair_gather_kernel<float><<<gg, 256, 0, c->stream>>>(
        A, ld, reinterpret_cast<const float*>(c->Fpl), c->ld, fplane, Linv, Uinv, L21, U12, L2, U2);
  static bool attr = false;
  const size_t smem = hh * sizeof(float2);
  if (!attr) {
    RMAT_CU(cudaFuncSetAttribute(pair_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem));
    attr = true;
  }
  // L: T = L21 L1^-1, lower-left = -L2^-1 T;  U: T = U12 U2^-1, upper-right = -U1^-1 T
  pair_gemm_kernel<<<npairs, 256, smem, c->stream>>>(L21, hh, Linv, 2 * hh, T, hh, H, 1.f);
  pair_gemm_kernel<<<npairs, 256, smem, c->stream>>>(Linv + hh, 2 * hh, T, hh, L2 + (size_t)H * P,
                                                     per, P, -1.f);
  pair_gemm_kernel<<<npairs, 256, smem, c->stream>>>(U12, hh, Uinv + hh, 2 * hh, T, hh, H, 1.f);
  pair_gemm_kernel<<<npairs, 256, smem, c->stream>>>(Uinv, 2 * hh, T, hh, U2 + H, per, P, -1.f);
  c->launches += 5;
  RMAT_CU(cudaGetLastError());
  c->inv_pairs = npairs;
  return RMAT_OK;
}

template <int JB>
int launch_apply_inv(rmat_ctx c, bool upper, int k0, int nb, float2* B, int ldb, int ncols,
                     const LUPerm* pm, void* Yp, const NearUpd& nu = NearUpd()) {
  static bool attr = false;
  const size_t smem = apply_inv_smem<JB>();
  if (!attr) {
    RMAT_CU(cudaFuncSetAttribute(apply_inv_kernel<JB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem));
    if (JB / 16 > 8)  // a 16-CTA cluster is beyond the portable size
      RMAT_CU(cudaFuncSetAttribute(apply_inv_kernel<JB>,
                                   cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    RMAT_CU(cudaFuncSetAttribute(apply_inv_kernel<JB>,
                                 cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared));
    attr = true;
  }
  // JB = 256: the pair inverses (blocks of 256 rows, table index k0 / 256)
  const size_t total = (size_t)JB * JB * (JB == 256 ? c->inv_pairs : c->inv_blocks);
  const float2* D = reinterpret_cast<const float2*>(JB == 256 ? c->Dinv2 : c->Dinv) +
                    (upper ? total : 0);
  KTimer kt(c, KT_APPLY_INV);
  apply_inv_kernel<JB><<<dim3(ceil_div(ncols, 16), JB / 16), 256, smem, c->stream>>>(
      D, k0, nb, B, ldb, ncols, pm ? pm->rows : nullptr, pm ? pm->src : nullptr,
      pm ? pm->cnt : nullptr, Yp, (size_t)RMAT_YPL_ROWS * RMAT_MAX_NB, rmat_plane_fmt(c->precision),
      rmat_ycs_cur(c), c->skip, nu);
  kt.end();
  c->launches++;
  RMAT_CU(cudaGetLastError());
  return RMAT_OK;
}

// Block blk's interchanges on K-columns 0..k0 of the split factor planes.
int permute_fpl_left(rmat_ctx c, int n, int ld, int k0, int nb, const LUPerm& pm) {
  if (k0 <= 0) return RMAT_OK;
  const size_t fplane = (size_t)n * ld;
  const int blk = k0 / nb;
  if (rmat_plane_esz(c->precision) == 2) {
    const size_t smem = (size_t)2 * nb * 32 * sizeof(__half);
    permute_fpl_left_kernel<__half><<<ceil_div(k0, 32), 256, smem, c->stream>>>(
        reinterpret_cast<__half*>(c->Fpl), ld, fplane, k0, pm.rows, pm.src, pm.cnt, blk, nb);
  } else {
    static bool attr = false;
    const size_t smem = (size_t)2 * nb * 32 * sizeof(float);
    if (!attr) {
      RMAT_CU(cudaFuncSetAttribute(permute_fpl_left_kernel<float>,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)(2 * RMAT_MAX_NB * 32 * sizeof(float))));
      attr = true;
    }
    permute_fpl_left_kernel<float><<<ceil_div(k0, 32), 256, smem, c->stream>>>(
        reinterpret_cast<float*>(c->Fpl), ld, fplane, k0, pm.rows, pm.src, pm.cnt, blk, nb);
  }
  c->launches++;
  RMAT_CU(cudaGetLastError());
  return RMAT_OK;
}

// End of a tensor-path factorisation: F holds L in the final row order; the forward
// solve gathers its right-hand sides once through the composed permutation.
int finish_fpl_order(rmat_ctx c, int n, int nb, const LUPerm& pm) {
  compose_perm_kernel<<<1, 256, 0, c->stream>>>(n, nb, pm.rows, pm.src, pm.cnt, c->pfwd);
  c->launches++;
  RMAT_CU(cudaGetLastError());
  c->fpl_final = true;
  c->fpl_nb = nb;
  return RMAT_OK;
}

// U12 = L11^-1 (P A12) for a full complex64 block through its inverse: L11^-1 is formed
// right after the panel (tri_inv_lower_kernel, one CTA) into its slot of the solve-path
// inverse table, then applied to all trailing columns on the tensor cores (the
// interchanges applied first; launch_u12_tc).
// Block widths 64 and 128; returns false when it does not apply.
// have_inv: L11^-1 of this block is in place already (an earlier call for other
// columns of the same block).
template <int JB>
int u12_by_inverse_jb(rmat_ctx c, float2* A, int ld, int n, int k0, const LUPerm* pm, int col0,
                      int ncols, bool have_inv) {
  const int nfull = n / JB;
  const size_t per = (size_t)JB * JB;
  RMAT_CHECK(rmat_grow(c, &c->Dinv, &c->Dinv_cap, 2 * per * nfull * sizeof(float2)));
  float2* Lk = reinterpret_cast<float2*>(c->Dinv) + (size_t)(k0 / JB) * per;
  static bool attr = false;
  const size_t smem = (size_t)(JB * (JB + 1) + (JB / 2) * (JB / 2 + 1)) * sizeof(float2);
  if (!attr) {
    RMAT_CU(cudaFuncSetAttribute(tri_inv_lower_kernel<JB>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    attr = true;
  }
  if (!have_inv) {
    tri_inv_lower_kernel<JB><<<1, TINV_THREADS, smem, c->stream>>>(A, ld, k0, Lk);
    c->launches++;
    RMAT_CU(cudaGetLastError());
  }
  if (ncols <= 0) return RMAT_OK;
  // On the tensor cores, in place: U12 = A12 - (I - L11^-1) A12, after the interchanges.
  // The FP16 planes carry one power-of-two scale per block, so only when the rows of a
  // block are of one magnitude: the symmetric equilibration (unit diagonal) sees to
  // that; otherwise the CUDA-core application keeps every entry's relative precision.
  if (!c->Mpl || !c->Bpl || !c->equil)
    return launch_apply_inv<JB>(c, false, k0, JB, A + col0, ld, ncols, pm, nullptr);
  if (pm) RMAT_CHECK(apply_perm<float>(c, *pm, A + col0, ld, ncols, k0, JB, JB));
  const int fmt = rmat_plane_fmt(c->precision);
  const int sa = ceil_div(n, JB) + 1, sm = sa + 1;  // scale slots past the per-block ones
  unsigned* um = fmt == 1 ? c->umax + sa : nullptr;
  if (um) {
    RMAT_CU(cudaMemsetAsync(um, 0, sizeof(unsigned), c->stream));
    block_absmax_kernel<<<std::min(c->sm_count * 2, ceil_div((long long)JB * ncols, 256)), 256, 0,
                          c->stream>>>(A, ld, k0, JB, col0, ncols, um, nullptr);
    c->launches++;
  }
  split_block_kernel<<<dim3(ceil_div(ncols, 32), JB / 32), 256, 0, c->stream>>>(
      A + (size_t)k0 * ld + col0, ld, JB, ncols, nullptr, 0, 0, 0, 0, c->Bpl,
      (size_t)n * RMAT_MAX_NB, col0, 0, fmt, um, fmt == 1 ? c->uscale + sa : nullptr, nullptr,
      nullptr);
  minv_planes_kernel<<<1, 1024, 0, c->stream>>>(Lk, JB, c->Mpl, (size_t)128 * 128, fmt,
                                                c->uscale + sm);
  c->launches += 2;
  RMAT_CU(cudaGetLastError());
  return launch_u12_tc(c, n, k0, JB, col0, ncols, c->uscale + sm, c->uscale + sa);
}

int u12_by_inverse(rmat_ctx c, float2* A, int ld, int n, int k0, int nb, const LUPerm* pm,
                   int col0, int ncols, bool* done, bool have_inv = false) {
  *done = true;
  if (nb == 128) return u12_by_inverse_jb<128>(c, A, ld, n, k0, pm, col0, ncols, have_inv);
  if (nb == 64) return u12_by_inverse_jb<64>(c, A, ld, n, k0, pm, col0, ncols, have_inv);
  *done = false;
  return RMAT_OK;
}

template <class T>
int launch_diag_nopiv(rmat_ctx c, cplx<T>* A, int ld, int k0, int jb, int* ipiv) {
  static bool attr = false;
  const size_t smem = (size_t)jb * (jb + 2) * sizeof(cplx<T>);
  if (!attr) {
    RMAT_CU(cudaFuncSetAttribute(diag_nopiv_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)((size_t)max_nb<T>() * (max_nb<T>() + 2) * sizeof(cplx<T>))));
    attr = true;
  }
  if (jb > max_nb<T>()) return RMAT_ESTATE;
  KTimer kt(c, KT_PANEL);
  diag_nopiv_kernel<T><<<1, DIAG_THREADS, smem, c->stream>>>(A, ld, k0, jb, ipiv, c->dstat);
  c->launches++;
  RMAT_CU(cudaGetLastError());
  kt.end();
  return RMAT_OK;
}

// Look-ahead panel (complex64): the block's jb columns factored as sub-panels of 32
// columns, whose rows (~47 KB per CTA at N = 25600 on every SM) fit in the shared
// memory a three-stage far update leaves on each SM, so the panel runs beside it on
// all SMs.  After each sub-panel: its interchanges applied to the block's other
// columns (left: the L parts of the earlier sub-panels follow every later
// interchange, as inside one panel; right: before they are updated) and to `extra`
// columns right of the block, then U12 = L11^-1 A12 of the sub-panel on all those
// right columns and A22 -= L21 U12 below it (CUDA cores: every kernel here stays
// small enough to share an SM with the far update).  With extra = the next block's
// width, that block leaves updated by this one, its U12 rows in place.  Same pivots
// as one panel (partial pivoting on the updated columns); results agree to rounding.
int la_panel(rmat_ctx c, float2* A, int ld, int k0, int n, int jb, int extra, int* ipiv,
             int la_ctas) {
  constexpr int W = 32;
  const LUPerm& ps = c->perm_sub;
  if (k0 % W || !ps.rows) return RMAT_ESTATE;
  for (int s0 = k0; s0 < k0 + jb; s0 += W) {
    const int w = std::min(W, k0 + jb - s0);
    RMAT_CHECK(launch_panel<float>(c, A, ld, s0, n, w, ipiv, la_ctas));
    const int r0 = s0 + w, rc = k0 + jb + extra - r0;
    if (s0 == k0 && rc <= 0) continue;
    perm_prep_kernel<<<1, 32, 0, c->stream>>>(ipiv, n, W, s0, ps.rows, ps.idx, ps.cnt, ps.src,
                                              c->dstat);
    c->launches++;
    if (s0 > k0) RMAT_CHECK(apply_perm<float>(c, ps, A + k0, ld, s0 - k0, s0, W, w));
    if (rc <= 0) continue;
    RMAT_CHECK(apply_perm<float>(c, ps, A + r0, ld, rc, s0, W, w));
    trsm_block_rhs_kernel<float, true><<<ceil_div(rc, 32), 256, trsm_smem<float>(w), c->stream>>>(
        A, ld, s0, w, A + r0, ld, rc, nullptr);
    c->launches++;
    RMAT_CU(cudaGetLastError());
    if (n > r0)
      RMAT_CHECK(gemm_sub<float>(c, n - r0, rc, w, A + (size_t)r0 * ld + s0, ld,
                                 A + (size_t)s0 * ld + r0, ld, A + (size_t)r0 * ld + r0, ld));
  }
  return RMAT_OK;
}

// Paired tensor-core factorisation (complex64): two panels share one trailing
// update with K = 2 nb, halving the read-modify-write passes over C22 (the update
// is bound by that traffic with FP16 operands).  For a pair (a at k0, b at k0b):
//   panel a; U12_a over all trailing columns; columns of b updated by a (narrow);
//   panel b; b's interchanges applied to the far columns and to a copy S of L21_a
//   (F keeps the deferred-interchange layout the solves replay); rows of b updated
//   by a (strip); U12_b; then C_far -= [S | L21_b] [U12_a ; U12_b] with one common
//   scale for both U12 halves.
// LDL^T (ldlt, C = C^T, no interchanges): diagonal block a; U12_a over all trailing
//   columns and L21_a = U12_a^T D_a^-1; rows of b updated by a over all trailing
//   columns (the diagonal block b and U12_b's rows); diagonal block b; U12_b and
//   L21_b; then the far update keeps only its tiles on or above the diagonal.
int factor_pairs_tc(rmat_ctx c, float2* A, int n, int ld, int* ipiv, int nb, const LUPerm& pm,
                    bool ldlt) {
  const int fmt = rmat_plane_fmt(c->precision);
  const size_t esz = rmat_plane_esz(c->precision);
  const size_t fplane = (size_t)n * ld, bplane = (size_t)n * RMAT_MAX_NB;
  const int pslot = ceil_div(n, nb);  // umax / uscale entry of the pair's common scale
  auto absmax = [&](int row0, int jb, int col0, int ncols, unsigned* o1, unsigned* o2) {
    block_absmax_kernel<<<std::min(c->sm_count * 2, ceil_div((long long)jb * ncols, 256)), 256, 0,
                          c->stream>>>(A, ld, row0, jb, col0, ncols, o1, o2);
    c->launches++;
  };
  auto split = [&](int row0, int jb, int col0, int ncols, bool f, bool t, int tk0,
                   const unsigned* sm, float* si, const unsigned* smT, float* siT) {
    split_block_kernel<<<dim3(ceil_div(ncols, 32), (int)round_up(jb, 32) / 32), 256, 0, c->stream>>>(
        A + (size_t)row0 * ld + col0, ld, jb, ncols, f ? c->Fpl : nullptr, ld, fplane, row0, col0,
        t ? c->Bpl : nullptr, bplane, col0, tk0, fmt, sm, si, smT, siT);
    c->launches++;
  };
  auto l21 = [&](int k0, int jb) {
    split_l21_kernel<<<ceil_div((long long)(n - k0 - jb) * 32, 256), 256, 0, c->stream>>>(
        A, ld, k0, jb, n, c->Fpl, ld, fplane, fmt);
    c->launches++;
  };
  auto prep = [&](int k0) -> int {
    if (ldlt) return RMAT_OK;  // identity interchanges, listed once before the loop
    perm_prep_kernel<<<1, 32, 0, c->stream>>>(ipiv, n, nb, k0, pm.rows, pm.idx, pm.cnt, pm.src,
                                              c->dstat);
    c->launches++;
    return permute_fpl_left(c, n, ld, k0, nb, pm);  // F's L parts follow every interchange
  };
  if (ldlt) {  // every block's (identity) row list at once, for the solves
    identity_pivots_kernel<<<ceil_div(n, 256), 256, 0, c->stream>>>(ipiv, n);
    perm_prep_kernel<<<ceil_div(n, nb), 32, 0, c->stream>>>(ipiv, n, nb, 0, pm.rows, pm.idx,
                                                           pm.cnt, pm.src, c->dstat);
    c->launches += 2;
    RMAT_CU(cudaGetLastError());
  }
  // U12 = L11^-1 (rows k0.., columns col0..col0+ncols), interchanges applied when perm
  auto trsm = [&](int k0, int jb, int col0, int ncols, bool perm, bool have_inv = false) -> int {
    bool fused = false;
    if (jb == nb) RMAT_CHECK(u12_by_inverse(c, A, ld, n, k0, nb, perm ? &pm : nullptr, col0, ncols,
                                            &fused, have_inv));
    if (!fused)
      RMAT_CHECK(solve_block<float, true>(c, perm ? &pm : nullptr, A, ld, k0, nb, jb, A + col0, ld,
                                          ncols, nullptr, &fused));
    if (!fused) {
      if (perm) RMAT_CHECK(apply_perm<float>(c, pm, A + col0, ld, ncols, k0, nb, jb));
      trsm_block_rhs_kernel<float, true><<<ceil_div(ncols, 32), 256, trsm_smem<float>(jb),
                                           c->stream>>>(A, ld, k0, jb, A + col0, ld, ncols, nullptr);
      c->launches++;
    }
    RMAT_CU(cudaGetLastError());
    return RMAT_OK;
  };
  auto panel = [&](int k0, int jb) -> int {
    return ldlt ? launch_diag_nopiv<float>(c, A, ld, k0, jb, ipiv)
                : launch_panel<float>(c, A, ld, k0, n, jb, ipiv);
  };
  // LDL^T: the multipliers below block k0 from its U12 (the block column below the
  // diagonal block was never updated)
  auto mult = [&](int k0, int jb) {
    if (!ldlt || n - k0 - jb <= 0) return;
    l21_from_u12_kernel<<<dim3(ceil_div(n - k0 - jb, 32), ceil_div(jb, 32)), 256, 0, c->stream>>>(
        A, ld, k0, jb, n, reinterpret_cast<unsigned*>(c->dstat + ST_LMAX));
    c->launches++;
  };
  unsigned* um = fmt == 1 ? c->umax : nullptr;
  float* us = fmt == 1 ? c->uscale : nullptr;
  // Look-ahead (pivoted LU): a pair's far update is issued as the next pair's 2 nb
  // columns (this stream) and the rest (far-far, side stream, three pipeline stages
  // so that every SM keeps room for a look-ahead panel CTA).  While the far-far update
  // runs, the next pair's panel a (32-column sub-panels, with U12_a on b's columns
  // and b's update by a) and panel b run beside it on the same SMs; everything that
  // touches the far-far columns or the earlier L columns of F (the far-far update's
  // A operand) waits for it: a's and b's interchanges there, U12_a on the far
  // columns, and the pair scale slot the far-far update reads.  Far blocks of at
  // least la_both_min rows take both panels beside their far-far update, those of
  // at least la_min rows only the first (a shorter far update would leave the second
  // exposed after the first), smaller ones none (the serial order is then faster).
  const bool la = !ldlt && c->factor_lookahead && c->side && (nb == 64 || nb == 128);
  const int la_ctas = c->la_panel_ctas > 0 ? c->la_panel_ctas : c->sm_count;
  const int la_min = c->la_min_rows > 0 ? c->la_min_rows : 6144;
  // the next pair's 32-column sub-panel CTAs (rows in shared memory) must fit beside a
  // far-part CTA on each SM, else they would wait for the far part to end: a far
  // block of M rows looks ahead only while that holds (up to ~25600 rows on 152 SMs)
  auto fits_beside = [&](int M) {
    const int P = std::min({la_ctas, RMAT_MAX_PANEL_CTAS, std::max(1, ceil_div(M, 32))});
    // the panel's dynamic shared memory plus its 288 static bytes, beside the far part's,
    // with the 1 KB each CTA reserves
    const size_t need = panel_smem<float>(ceil_div(M, P), 33, true) + 288;
    const size_t room = (size_t)c->smem_per_sm - tc_lean_smem() - 2 * 1024;
    return need <= room;
  };
  const int la_both_min = c->la_both_rows > 0 ? c->la_both_rows : 20480;
  cudaStream_t main_s = c->stream;
  bool pending = false;   // a far-far update is in flight on the side stream
  bool la_pair = false;   // this pair follows a split far update (look-ahead order)
  bool la_both = false;   // ... and both its panels run beside it (else only the first)
  const bool la_serial = c->factor_lookahead == 2;  // same order, one stream (timing)
  auto join = [&]() -> int {
    if (pending) {
      RMAT_CU(cudaStreamWaitEvent(main_s, c->la_ev[2], 0));
      pending = false;
    }
    return RMAT_OK;
  };
  auto perm_list = [&](int k0) {
    perm_prep_kernel<<<1, 32, 0, c->stream>>>(ipiv, n, nb, k0, pm.rows, pm.idx, pm.cnt, pm.src,
                                              c->dstat);
    c->launches++;
  };
  int k0 = 0;
  while (k0 < n) {
    const int jba = std::min(nb, n - k0), blka = k0 / nb;
    if (la_pair && la_both) {
      // the previous far block was wider than 2 nb: this is a full pair whose 2 nb
      // columns are up to date, beside the far-far update: panel a (with U12_a on b's
      // columns and b's update by a), panel b
      const int k0b = k0 + jba, jbb = nb, far0 = k0b + jbb, far = n - far0;
      const int resta = n - k0 - jba;
      RMAT_CHECK(la_panel(c, A, ld, k0, n, jba, jbb, ipiv, la_ctas));
      perm_list(k0);
      l21(k0, jba);  // F's L21_a (its own columns: the far-far update reads earlier ones)
      RMAT_CU(cudaGetLastError());
      RMAT_CHECK(la_panel(c, A, ld, k0b, n, jbb, 0, ipiv, la_ctas));
      perm_list(k0b);
      RMAT_CHECK(join());
      RMAT_CHECK(permute_fpl_left(c, n, ld, k0, nb, pm));
      RMAT_CHECK(permute_fpl_left(c, n, ld, k0b, nb, pm));  // b's interchanges reach L21_a too
      RMAT_CHECK(trsm(k0, jba, far0, far, true));          // U12_a on the far columns
      if (um) {
        RMAT_CU(cudaMemsetAsync(um + pslot, 0, sizeof(unsigned), c->stream));
        absmax(k0, jba, k0b, resta, um + blka, um + pslot);
      }
      // F rows of a (the backward solve's U12_a, one scale) and the U12_a^T planes
      split(k0, jba, k0b, resta, true, true, 0, um ? um + blka : nullptr, us ? us + blka : nullptr,
            nullptr, nullptr);
      RMAT_CHECK(apply_perm<float>(c, pm, A + far0, ld, far, k0b, nb, jbb));  // b's, far columns
      RMAT_CU(cudaGetLastError());
      // rows of b <- a in the far columns
      RMAT_CHECK(launch_factor_tc(c, n, k0b, jbb, far0, far, jba, k0, us ? us + blka : nullptr));
    } else {
      if (la_pair) {
        // panel a alone beside the far-far update (a shorter far update would leave
        // the second panel exposed anyway); then the serial order
        RMAT_CHECK(la_panel(c, A, ld, k0, n, jba, 0, ipiv, la_ctas));
        perm_list(k0);
        RMAT_CHECK(join());
        RMAT_CHECK(permute_fpl_left(c, n, ld, k0, nb, pm));
      } else {
        RMAT_CHECK(panel(k0, jba));
        RMAT_CHECK(prep(k0));
      }
      const int resta = n - k0 - jba;
      if (resta <= 0) break;
      RMAT_CHECK(trsm(k0, jba, k0 + jba, resta, !ldlt));
      mult(k0, jba);
      if (resta <= nb) {  // block b is the last one: a single update
        if (um) absmax(k0, jba, k0 + jba, resta, um + blka, nullptr);
        split(k0, jba, k0 + jba, resta, true, true, 0, um ? um + blka : nullptr,
              us ? us + blka : nullptr, nullptr, nullptr);
        l21(k0, jba);
        RMAT_CU(cudaGetLastError());
        RMAT_CHECK(launch_trailing_tc(c, A, ld, k0, jba, n, ldlt));
        k0 += jba;
        continue;
      }
      const int k0b = k0 + jba, jbb = nb, far0 = k0b + jbb, far = n - far0;
      if (um) {
        RMAT_CU(cudaMemsetAsync(um + pslot, 0, sizeof(unsigned), c->stream));
        absmax(k0, jba, k0b, resta, um + blka, um + pslot);
      }
      split(k0, jba, k0b, resta, true, true, 0, um ? um + blka : nullptr, us ? us + blka : nullptr,
            nullptr, nullptr);
      l21(k0, jba);
      RMAT_CU(cudaGetLastError());
      if (ldlt) {
        // rows of b <- a over all trailing columns: the diagonal block b and U12_b's rows
        RMAT_CHECK(launch_factor_tc(c, n, k0b, jbb, k0b, resta, jba, k0, us ? us + blka : nullptr));
        RMAT_CHECK(panel(k0b, jbb));
        RMAT_CHECK(prep(k0b));
      } else {
        // columns of b <- a (rows k0b.., in the row order before panel b)
        RMAT_CHECK(launch_factor_tc(c, n, k0b, n - k0b, k0b, jbb, jba, k0, us ? us + blka : nullptr));
        RMAT_CHECK(panel(k0b, jbb));
        RMAT_CHECK(prep(k0b));  // b's interchanges also reach F's L21_a
        RMAT_CHECK(apply_perm<float>(c, pm, A + far0, ld, far, k0b, nb, jbb));  // and the far columns
        // rows of b <- a in the far columns
        RMAT_CHECK(launch_factor_tc(c, n, k0b, jbb, far0, far, jba, k0, us ? us + blka : nullptr));
      }
    }
    const int k0b = k0 + jba, jbb = nb, blkb = k0b / nb, far0 = k0b + jbb, far = n - far0;
    RMAT_CHECK(trsm(k0b, jbb, far0, far, false));  // U12_b
    mult(k0b, jbb);
    if (um) absmax(k0b, jbb, far0, far, um + blkb, um + pslot);
    // F rows of b (own scale); U12^T planes of both halves with the pair's common scale
    split(k0b, jbb, far0, far, true, true, jba, um ? um + blkb : nullptr, us ? us + blkb : nullptr,
          um ? um + pslot : nullptr, us ? us + pslot : nullptr);
    split(k0, jba, far0, far, false, true, 0, um ? um + pslot : nullptr, nullptr, nullptr, nullptr);
    l21(k0b, jbb);
    RMAT_CU(cudaGetLastError());
    // C_far -= [L21_a | L21_b] [U12_a ; U12_b]: F's K-columns k0..k0+jba+jbb are contiguous
    if (la && far > 2 * nb && far >= la_min && fits_beside(far)) {
      // the next pair's columns here, then the far-far columns on the side stream
      // (forked after everything above); launched in this order so the narrow update's
      // CTAs are dispatched first and the side stream's fill the SMs they leave
      if (!la_serial) {
        RMAT_CU(cudaEventRecord(c->la_ev[0], main_s));
        RMAT_CU(cudaStreamWaitEvent(c->side, c->la_ev[0], 0));
      }
      RMAT_CHECK(launch_factor_tc(c, n, far0, far, far0, 2 * nb, jba + jbb, k0,
                                  us ? us + pslot : nullptr, false));
      if (!la_serial) c->stream = c->side;
      c->side_free = 0;
      c->tc_lean = true;
      const int st = launch_factor_tc(c, n, far0, far, far0 + 2 * nb, far - 2 * nb, jba + jbb, k0,
                                      us ? us + pslot : nullptr, false);
      c->tc_lean = false;
      c->side_free = -1;
      c->stream = main_s;
      RMAT_CHECK(st);
      if (!la_serial) {
        RMAT_CU(cudaEventRecord(c->la_ev[2], c->side));
        pending = true;
      }
      la_pair = true;
      la_both = far >= la_both_min;
    } else {
      la_pair = false;
      RMAT_CHECK(launch_factor_tc(c, n, far0, far, far0, far, jba + jbb, k0,
                                  us ? us + pslot : nullptr, ldlt));
    }
    k0 = far0;
  }
  RMAT_CHECK(join());
  c->inv_blocks = 0;
  c->inv_pairs = 0;
  // L11^-1 of every full block is already in place (formed for its U12), except the
  // last block when it has no trailing columns: form it here
  const int nfull = n / nb;
  if (nfull > 0 && nfull * nb == n) {
    bool done = false;
    RMAT_CHECK(u12_by_inverse(c, A, ld, n, (nfull - 1) * nb, nb, nullptr, n, 0, &done));
  }
  if (nb == 128) RMAT_CHECK(invert_diag_blocks<128>(c, A, ld, n, nb, true));
  if (nb == 64) RMAT_CHECK(invert_diag_blocks<64>(c, A, ld, n, nb, true));
  RMAT_CHECK(finish_fpl_order(c, n, nb, pm));
  return invert_pair_blocks(c, A, ld, n);
}

template <class T>
int lu_factor_dev(rmat_ctx c, void* Av, int n, int ld, int* ipiv, int nb, bool tensor,
                  const LUPerm& pm) {
  using C2 = cplx<T>;
  C2* A = reinterpret_cast<C2*>(Av);
  if (nb < 1 || nb > max_nb<T>()) return RMAT_ESTATE;
  RMAT_CHECK(set_trsm_attrs<T>());
  RMAT_CU(cudaMemsetAsync(ipiv, 0xff, (size_t)n * sizeof(int), c->stream));  // -1: "not pivoted"
  c->fpl_final = false;
  const int fmt = rmat_plane_fmt(c->precision);
  if (tensor && fmt == 1)
    RMAT_CU(cudaMemsetAsync(c->umax, 0, (size_t)ceil_div(n, nb) * sizeof(unsigned), c->stream));
  // complex-symmetric LDL^T without pivoting (tensor-core precisions): no panel, and
  // the trailing updates keep only the tiles on or above the diagonal
  const bool ldlt = tensor && sizeof(T) == 4 && c->factor_used == 1;  // set by rmat_factor
  if (ldlt) RMAT_CU(cudaMemsetAsync(c->dstat + ST_LMAX, 0, sizeof(int), c->stream));
  if constexpr (sizeof(T) == 4)
    if (tensor && c->paired && 2 * nb <= RMAT_MAX_NB)
      return factor_pairs_tc(c, reinterpret_cast<float2*>(A), n, ld, ipiv, nb, pm, ldlt);
  for (int k0 = 0; k0 < n; k0 += nb) {
    const int jb = std::min(nb, n - k0);
    if (ldlt)
      RMAT_CHECK(launch_diag_nopiv<T>(c, A, ld, k0, jb, ipiv));
    else
      RMAT_CHECK(launch_panel<T>(c, A, ld, k0, n, jb, ipiv));
    const int rest = n - k0 - jb;
    if (rest <= 0) {
      perm_prep_kernel<<<1, 32, 0, c->stream>>>(ipiv, n, nb, k0, pm.rows, pm.idx, pm.cnt, pm.src,
                                                c->dstat);
      c->launches++;
      if (tensor && sizeof(T) == 4) RMAT_CHECK(permute_fpl_left(c, n, ld, k0, nb, pm));
      continue;
    }
    // G3: interchanges on the trailing columns, then U12 = L11^-1 A12
    perm_prep_kernel<<<1, 32, 0, c->stream>>>(ipiv, n, nb, k0, pm.rows, pm.idx, pm.cnt, pm.src,
                                              c->dstat);
    c->launches++;
    if (tensor && sizeof(T) == 4) RMAT_CHECK(permute_fpl_left(c, n, ld, k0, nb, pm));
    bool fused = false;
    RMAT_CHECK(solve_block<T, true>(c, &pm, A, ld, k0, nb, jb, A + k0 + jb, ld, rest, nullptr,
                                    &fused));
    if (!fused) {
      RMAT_CHECK(apply_perm<T>(c, pm, A + k0 + jb, ld, rest, k0, nb, jb));
      trsm_block_rhs_kernel<T, true><<<ceil_div(rest, 32), 256, trsm_smem<T>(jb), c->stream>>>(
          A, ld, k0, jb, A + k0 + jb, ld, rest, nullptr);
      c->launches++;
    }
    RMAT_CU(cudaGetLastError());
    if (tensor && sizeof(T) == 4) {
      const size_t fplane = (size_t)n * ld, bplane = (size_t)n * RMAT_MAX_NB;
      const float2* Af = reinterpret_cast<const float2*>(A);
      const int kpad = (int)round_up(jb, 32);
      const int blk = k0 / nb;
      if (ldlt) {  // L21 from U12 (the block column below the diagonal was not updated)
        l21_from_u12_kernel<<<dim3(ceil_div(rest, 32), ceil_div(jb, 32)), 256, 0, c->stream>>>(
            reinterpret_cast<float2*>(A), ld, k0, jb, n,
            reinterpret_cast<unsigned*>(c->dstat + ST_LMAX));
        c->launches++;
      }
      if (fmt == 1) {  // the U12 block's scale: max over its entries first
        block_absmax_kernel<<<std::min(c->sm_count * 2, ceil_div((long long)jb * rest, 256)), 256, 0,
                              c->stream>>>(Af, ld, k0, jb, k0 + jb, rest, c->umax + blk, nullptr);
        c->launches++;
      }
      split_block_kernel<<<dim3(ceil_div(rest, 32), kpad / 32), 256, 0, c->stream>>>(
          Af + (size_t)k0 * ld + k0 + jb, ld, jb, rest, c->Fpl, ld, fplane, k0, k0 + jb, c->Bpl,
          bplane, k0 + jb, 0, fmt, fmt == 1 ? c->umax + blk : nullptr,
          fmt == 1 ? c->uscale + blk : nullptr, nullptr, nullptr);
      split_l21_kernel<<<ceil_div((long long)rest * 32, 256), 256, 0, c->stream>>>(
          Af, ld, k0, jb, n, c->Fpl, ld, fplane, fmt);
      c->launches += 2;
      RMAT_CU(cudaGetLastError());
      RMAT_CHECK(launch_trailing_tc(c, reinterpret_cast<float2*>(A), ld, k0, jb, n, ldlt));
    } else {
      cudaEvent_t e0 = nullptr, e1 = nullptr;
      if (c->timing) {
        e0 = rmat_event(c);
        e1 = rmat_event(c);
        RMAT_CU(cudaEventRecord(e0, c->stream));
      }
      RMAT_CHECK(gemm_sub<T>(c, rest, rest, jb, A + (size_t)(k0 + jb) * ld + k0, ld,
                             A + (size_t)k0 * ld + k0 + jb, ld, A + (size_t)(k0 + jb) * ld + k0 + jb,
                             ld));
      if (c->timing) {
        RMAT_CU(cudaEventRecord(e1, c->stream));
        c->tu_events.push_back({e0, e1});
      }
      c->tu_launches++;
      c->tu_flops += 8.0 * rest * (double)rest * jb;
    }
  }
  c->inv_blocks = 0;
  c->inv_pairs = 0;
  if (tensor && sizeof(T) == 4) {
    const float2* Af = reinterpret_cast<const float2*>(A);
    if (nb == 128) RMAT_CHECK(invert_diag_blocks<128>(c, Af, ld, n, nb));
    if (nb == 64) RMAT_CHECK(invert_diag_blocks<64>(c, Af, ld, n, nb));
    RMAT_CHECK(finish_fpl_order(c, n, nb, pm));
    RMAT_CHECK(invert_pair_blocks(c, Af, ld, n));
  }
  return RMAT_OK;
}

template <class T>
int lu_solve_dev(rmat_ctx c, const void* Av, int n, int ld, const LUPerm& pm, int nb, void* Bv,
                 int ldb, int nrhs, bool tensor) {
  using C2 = cplx<T>;
  const C2* A = reinterpret_cast<const C2*>(Av);
  C2* B = reinterpret_cast<C2*>(Bv);
  RMAT_CHECK(set_trsm_attrs<T>());
  // tensor-core block updates need the factor's split planes (written by a
  // tensor-path factorisation), an even row stride and at most RMAT_YPL_ROWS columns
  const bool tc = tensor && sizeof(T) == 4 && c->Fpl && nrhs % 2 == 0 && nrhs <= RMAT_YPL_ROWS &&
                  ldb == nrhs && Bv == c->Bw;
  const size_t yplane = (size_t)RMAT_YPL_ROWS * RMAT_MAX_NB;
  const int fmt = rmat_plane_fmt(c->precision);
  // forward.  Tensor path: F's L parts are in the final row order, so the right-hand
  // sides are permuted once (composed permutation) and the blocks need no replay;
  // otherwise each panel's interchanges are replayed block by block.
  const bool upfront = tc && c->fpl_final && c->fpl_nb == nb && c->Bt;
  if (upfront) {
    row_gather_kernel<<<std::min(c->sm_count * 8, ceil_div((long long)n * nrhs, 256)), 256, 0,
                        c->stream>>>(reinterpret_cast<const float2*>(B),
                                     reinterpret_cast<float2*>(c->Bt), n, nrhs, c->pfwd, c->skip);
    c->launches++;
    RMAT_CU(cudaGetLastError());
    RMAT_CU(cudaMemcpyAsync(B, c->Bt, (size_t)n * nrhs * sizeof(C2), cudaMemcpyDeviceToDevice,
                            c->stream));
  }
  const LUPerm* fpm = upfront ? nullptr : &pm;
  // Look-ahead (tensor path, no per-block interchanges to replay): after block k's
  // diagonal application, its update of the NEXT block's rows runs on the main
  // stream and its update of the far rows on the side stream, so block k+1 can start
  // at once.  Block k+2 waits for block k's far update (it covers block k+2's rows);
  // the Y planes alternate between two buffers (block parity) for the same reason.
  // The far and next-row updates of different blocks reduce-add into disjoint or
  // commuting rows of B (TMA reduce-add is atomic per element).
  const bool la_fwd = tc && c->solve_lookahead && fpm == nullptr && c->side;
  const bool la_bwd = tc && c->solve_lookahead && c->side;
  // mode 2: each step's update of the next step's rows inside its diagonal application
  // (the factor's split planes in their final row order), one launch less per step but
  // ~25 us more per diagonal application at N = 25600, so not the default
  const bool fuse_near = c->solve_lookahead == 2 && c->fpl_final;
  // 256-row steps over pairs of blocks with a composed inverse (rows pre-gathered)
  const bool pairs = tc && fpm == nullptr && nb == 128 && c->inv_nb == nb && c->inv_pairs > 0 &&
                     !c->pairs_off;
  auto pair_at = [&](int r0) { return pairs && r0 % 256 == 0 && r0 / 256 < c->inv_pairs; };
  // the look-ahead's update of the next step's rows (few output tiles, on the SMs the
  // far update leaves free) splits its K range over CTAs
  auto ksplit_for = [&](int jbk) {
    const int kst = fmt == 1 ? 16 : 8, steps = (int)round_up(jbk, kst) / kst;
    return steps % 4 == 0 ? 4 : steps % 2 == 0 ? 2 : 1;
  };
  const int last = ((n - 1) / nb) * nb;
  // a pair step covers block kb and the one above when kb is a pair's second block
  auto pair_end = [&](int kb) { return pairs && (kb / nb) % 2 == 1 && (kb / nb) / 2 < c->inv_pairs; };
  // Both sweeps for the right-hand-side columns col0..col0+nc, on streams main_s / side_s
  // with look-ahead events ev[0..3].  Column groups are independent, so the sweeps of
  // different groups run concurrently on their own streams.
  auto sweeps = [&](int col0, int nc, cudaStream_t main_s, cudaStream_t side_s,
                    cudaEvent_t* ev) -> int {
    C2* Bc = B + col0;
    const int gx_g = ceil_div(nc, 32);
    c->stream = main_s;
    c->ycol0 = col0;
    bool pending[2] = {false, false};
    auto la_wait = [&](int b) -> int {
      if (pending[b]) {
        RMAT_CU(cudaStreamWaitEvent(main_s, ev[2 + b], 0));
        pending[b] = false;
      }
      return RMAT_OK;
    };
    auto split_yg = [&](int row0, int jb) -> int {
      split_y_kernel<<<ceil_div(nc, 8), 256, 0, c->stream>>>(
          reinterpret_cast<const float2*>(Bc) + (size_t)row0 * ldb, ldb, jb, nc, rmat_ypl_cur(c),
          yplane, fmt, rmat_ycs_cur(c), c->skip);
      c->launches++;
      RMAT_CU(cudaGetLastError());
      return RMAT_OK;
    };
    // the far update of a step on the side stream, forked after the next-row update
    auto far_update = [&](int b, int row0, int M, int k0, int jb, const float* rs) -> int {
      RMAT_CU(cudaEventRecord(ev[b], main_s));
      RMAT_CU(cudaStreamWaitEvent(side_s, ev[b], 0));
      c->stream = side_s;
      const int st = launch_solve_tc(c, row0, M, nc, k0, jb, row0, n, rs, nb);
      c->stream = main_s;
      RMAT_CHECK(st);
      RMAT_CU(cudaEventRecord(ev[2 + b], side_s));
      pending[b] = true;
      return RMAT_OK;
    };
    int step = 0;
    for (int k0 = 0, jb = 0; k0 < n; k0 += jb, ++step) {
      const bool pstep = pair_at(k0);
      jb = pstep ? 256 : std::min(nb, n - k0);
      const int b = step & 1;
      if (tc) {
        RMAT_CHECK(la_wait(b));
        c->ybuf = b;
      }
      const bool need_y = tc && n - k0 - jb > 0;
      bool fused = false;
      // the next step's rows updated inside the diagonal application (look-ahead mode 2)
      NearUpd nu;
      const int nrow0 = k0 + jb, nM = n - k0 - jb;
      const int nnear = std::min(pair_at(nrow0) ? 256 : nb, nM);
      const bool fuse = need_y && la_fwd && fuse_near && nnear > 0;
      if (fuse) {
        nu.F = c->Fpl;
        nu.fplane = (size_t)n * ld;
        nu.ldf = ld;
        nu.fmt = fmt;
        nu.row0 = nrow0;
        nu.nrows = nnear;
        nu.kcol0 = k0;
      }
      bool near_done = false;
      if (pstep) {
        RMAT_CHECK(launch_apply_inv<256>(c, false, k0, 256, reinterpret_cast<float2*>(Bc), ldb, nc,
                                         nullptr, need_y ? rmat_ypl_cur(c) : nullptr, nu));
        fused = true;
        near_done = fuse;
      } else if (tc && jb == nb && k0 / nb < c->inv_blocks && c->inv_nb == nb) {
        float2* Bf = reinterpret_cast<float2*>(Bc);
        void* Yp = need_y ? rmat_ypl_cur(c) : nullptr;
        if (nb == 128) RMAT_CHECK(launch_apply_inv<128>(c, false, k0, nb, Bf, ldb, nc, fpm, Yp, nu));
        else RMAT_CHECK(launch_apply_inv<64>(c, false, k0, nb, Bf, ldb, nc, fpm, Yp, nu));
        fused = true;
        near_done = fuse;
      } else {
        RMAT_CHECK(solve_block<T, true>(c, fpm, A, ld, k0, nb, jb, Bc, ldb, nc,
                                        need_y ? rmat_ypl_cur(c) : nullptr, &fused));
      }
      if (!fused) {
        if (fpm) RMAT_CHECK(apply_perm<T>(c, pm, Bc, ldb, nc, k0, nb, jb));
        trsm_block_rhs_kernel<T, true><<<gx_g, 256, trsm_smem<T>(jb), c->stream>>>(A, ld, k0, jb, Bc,
                                                                                  ldb, nc, c->skip);
        c->launches++;
        RMAT_CU(cudaGetLastError());
        if (need_y) RMAT_CHECK(split_yg(k0, jb));
      }
      if (need_y) {
        const int row0 = k0 + jb, M = n - k0 - jb;
        const int near = std::min(pair_at(row0) ? 256 : nb, M);
        if (near_done) {
          if (near < M) RMAT_CHECK(far_update(b, row0 + near, M - near, k0, jb, nullptr));
        } else if (!la_fwd || near >= M) {
          RMAT_CHECK(launch_solve_tc(c, row0, M, nc, k0, jb, row0, n, nullptr, nb));
        } else {
          RMAT_CHECK(launch_solve_tc(c, row0, near, nc, k0, jb, row0, n, nullptr, nb,
                                     ksplit_for(jb)));
          RMAT_CHECK(far_update(b, row0 + near, M - near, k0, jb, nullptr));
        }
      } else {
        RMAT_CHECK(gemm_sub<T>(c, n - k0 - jb, nc, jb, A + (size_t)(k0 + jb) * ld + k0, ld,
                               Bc + (size_t)k0 * ldb, ldb, Bc + (size_t)(k0 + jb) * ldb, ldb));
      }
    }
    RMAT_CHECK(la_wait(0));
    RMAT_CHECK(la_wait(1));
    // backward: U11 solve, then update the rows above (right-looking); look-ahead as
    // in the forward sweep, the next block being the one above
    step = 0;
    for (int kb = last; kb >= 0; ++step) {
      const bool pstep = pair_end(kb);
      const int k0 = pstep ? kb - nb : kb;
      const int jb = pstep ? 256 : std::min(nb, n - k0);
      kb = k0 - nb;
      const int b = step & 1;
      if (tc) {
        RMAT_CHECK(la_wait(b));
        c->ybuf = b;
      }
      const bool need_y = tc && k0 > 0;
      bool fused = false;
      NearUpd nu;
      const int bnear = std::min(pair_end(kb) ? 256 : nb, k0);  // the next (upper) step's rows
      const bool fuse = need_y && la_bwd && fuse_near && bnear > 0;
      if (fuse) {
        nu.F = c->Fpl;
        nu.fplane = (size_t)n * ld;
        nu.ldf = ld;
        nu.fmt = fmt;
        nu.row0 = k0 - bnear;
        nu.nrows = bnear;
        nu.kcol0 = k0;
        nu.rowscale = fmt == 1 ? c->uscale : nullptr;  // U rows: one scale per row block
        nu.rs_div = nb;
      }
      bool near_done = false;
      if (pstep) {
        RMAT_CHECK(launch_apply_inv<256>(c, true, k0, 256, reinterpret_cast<float2*>(Bc), ldb, nc,
                                         nullptr, need_y ? rmat_ypl_cur(c) : nullptr, nu));
        fused = true;
        near_done = fuse;
      } else if (tc && jb == nb && k0 / nb < c->inv_blocks && c->inv_nb == nb) {
        float2* Bf = reinterpret_cast<float2*>(Bc);
        void* Yp = need_y ? rmat_ypl_cur(c) : nullptr;
        if (nb == 128) RMAT_CHECK(launch_apply_inv<128>(c, true, k0, nb, Bf, ldb, nc, nullptr, Yp, nu));
        else RMAT_CHECK(launch_apply_inv<64>(c, true, k0, nb, Bf, ldb, nc, nullptr, Yp, nu));
        fused = true;
        near_done = fuse;
      } else {
        RMAT_CHECK(solve_block<T, false>(c, nullptr, A, ld, k0, nb, jb, Bc, ldb, nc,
                                         need_y ? rmat_ypl_cur(c) : nullptr, &fused));
      }
      if (!fused) {
        trsm_block_rhs_kernel<T, false><<<gx_g, 256, trsm_smem<T>(jb), c->stream>>>(A, ld, k0, jb, Bc,
                                                                                   ldb, nc, c->skip);
        c->launches++;
        RMAT_CU(cudaGetLastError());
        if (need_y) RMAT_CHECK(split_yg(k0, jb));
      }
      if (need_y) {
        // A = U rows of earlier row blocks: their per-block scales apply row-wise
        const float* rs = fmt == 1 ? c->uscale : nullptr;
        const int near = std::min(pair_end(kb) ? 256 : nb, k0);  // the next (upper) step's rows
        if (near_done) {
          if (near < k0) RMAT_CHECK(far_update(b, 0, k0 - near, k0, jb, rs));
        } else if (!la_bwd || near >= k0) {
          RMAT_CHECK(launch_solve_tc(c, 0, k0, nc, k0, jb, 0, n, rs, nb));
        } else {
          RMAT_CHECK(launch_solve_tc(c, k0 - near, near, nc, k0, jb, k0 - near, n, rs, nb,
                                     ksplit_for(jb)));
          RMAT_CHECK(far_update(b, 0, k0 - near, k0, jb, rs));
        }
      } else {
        RMAT_CHECK(gemm_sub<T>(c, k0, nc, jb, A + k0, ld, Bc + (size_t)k0 * ldb, ldb, Bc, ldb));
      }
    }
    RMAT_CHECK(la_wait(0));
    RMAT_CHECK(la_wait(1));
    return RMAT_OK;
  };
  // Column groups (tensor path with look-ahead, on request): two groups of nrhs/2
  // columns when the halves stay multiples of 64 and the second group's streams exist.
  // Not the default: at N = 25600 with 256 right-hand sides two concurrent groups took
  // 11.2 ms per solve against 10.4 ms for one (their diagonal applications and far
  // updates compete for the same SMs)
  const int groups_want = c->solve_groups > 0 ? c->solve_groups : 1;
  const bool grouped = la_fwd && la_bwd && groups_want == 2 && nrhs % 128 == 0 && nrhs >= 256 &&
                       c->grp_main && c->grp_side;
  cudaStream_t caller = c->stream;
  c->ysolve_nrhs = nrhs;
  int st = RMAT_OK;
  if (!grouped) {
    c->tc_cap_div = 1;
    st = sweeps(0, nrhs, caller, c->side, c->la_ev);
  } else {
    const int half = nrhs / 2;
    c->tc_cap_div = 2;
    RMAT_CU(cudaEventRecord(c->grp_ev[4], caller));
    RMAT_CU(cudaStreamWaitEvent(c->grp_main, c->grp_ev[4], 0));
    st = sweeps(0, half, caller, c->side, c->la_ev);
    if (st == RMAT_OK) st = sweeps(half, half, c->grp_main, c->grp_side, c->grp_ev);
    c->stream = caller;
    // join: the caller's stream continues after both groups
    if (st == RMAT_OK) {
      RMAT_CU(cudaEventRecord(c->grp_ev[5], c->grp_main));
      RMAT_CU(cudaStreamWaitEvent(caller, c->grp_ev[5], 0));
    }
  }
  c->stream = caller;
  c->ycol0 = 0;
  c->tc_cap_div = 1;
  return st;
}

template int lu_factor_dev<float>(rmat_ctx, void*, int, int, int*, int, bool, const LUPerm&);
template int lu_factor_dev<double>(rmat_ctx, void*, int, int, int*, int, bool, const LUPerm&);
template int lu_solve_dev<float>(rmat_ctx, const void*, int, int, const LUPerm&, int, void*, int,
                                  int, bool);
template int lu_solve_dev<double>(rmat_ctx, const void*, int, int, const LUPerm&, int, void*, int,
                                   int, bool);

int gemm_sub_c128(rmat_ctx c, int M, int N, int K, const double2* A, int lda, const double2* B,
                  int ldb, double2* C, int ldc) {
  return gemm_sub<double>(c, M, N, K, A, lda, B, ldb, C, ldc);
}
