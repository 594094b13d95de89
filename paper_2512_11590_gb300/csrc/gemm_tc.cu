// G4 (tensor path): trailing update C22 -= L21 U12 on the tcgen05 tensor cores.
//
// The paper runs the single-precision factorisation's updates in FP32
// (cusolverDnCgetrf, Sec. 3.4).  Here each complex product is formed from TF32
// tensor-core products with FP32 accumulation in tensor memory:
//   x = x_hi + x_lo,  x_hi = tf32(x),  x_lo = x - x_hi          (per real plane)
//   a*b ~= a_hi b_hi + a_hi b_lo + a_lo b_hi                    (3 products)
//   Re += Ar Br - Ai Bi,   Im += Ar Bi + Ai Br                  (4 real GEMMs)
// i.e. 12 TF32 MMAs per K-step into two FP32 accumulators (re, im).  The
// -Ai Bi terms use the instruction descriptor's negate-A bit.
//
// Operand planes (written by split_l21_kernel / split_u12_kernel in lu.cu) are
// K-major fp32 [row][K] with a 256-float row stride: A rows = L21 rows, B rows =
// U12 columns.  Tile 128 x 256 per CTA (cta_group::1, M=128, N=256): the re and
// im accumulators take all 512 TMEM columns.  K-steps of 8 (32-byte rows,
// SWIZZLE_32B) flow through a 4-stage TMA -> mbarrier pipeline.
//
// Roles (192 threads, one CTA per SM, persistent over tiles):
//   warp 0      TMA producer (one elected lane)
//   warp 1      TMEM allocator + MMA issuer (one elected lane)
//   warps 2..5  epilogue: tcgen05.ld of re/im rows, C -= acc in global memory
// Every wait is bounded (~2 s of globaltimer); on expiry the kernel raises an
// error word, lets its issued copies/MMAs drain (bounded), frees TMEM, returns.
#include <cuda.h>

#include <cstring>

#include "rmat_internal.h"
#include "tc_common.cuh"

namespace {

constexpr int TC_BM = 128, TC_BN = 256, TC_BK = 8;
constexpr int TC_THREADS = 192;
constexpr uint32_t A_PLANE_BYTES = TC_BM * TC_BK * 4;                              // 4 KB
constexpr uint32_t STAGING_BYTES = TC_BM * 32 * 4;  // 16 complex columns x 128 rows, 128B swizzle

// Tile width BN = 256 (trailing updates) or 128 (solve updates: twice the tiles for
// the same rows, and two accumulator sets in the 512 TMEM columns, so the epilogue
// of one tile overlaps the MMAs of the next).
// BN = 128 keeps three pipeline stages (130 KB of shared memory), so a solve-path
// diagonal application (76 KB) fits beside a running update on the same SM.
// LEAN (BN = 256): three stages (177 KB), so a look-ahead panel CTA of up to ~48 KB
// fits beside each CTA of a far update that covers every SM.
template <int BN, bool LEAN = false>
struct TcCfg {
  static constexpr uint32_t B_PLANE = BN * TC_BK * 4;                 // 8 / 4 KB
  static constexpr uint32_t STAGE = 4 * A_PLANE_BYTES + 4 * B_PLANE;  // 48 / 32 KB
  static constexpr int NBUF = 512 / (2 * BN);                         // accumulator sets
  static constexpr int STAGES = (BN == 128 || LEAN) ? 3 : 4;
  static constexpr size_t SMEM = (size_t)STAGES * STAGE + 2 * STAGING_BYTES + 1024 + 256;
};

struct TcMaps {
  CUtensorMap a[4];  // A operand planes: re_hi, re_lo, im_hi, im_lo
  CUtensorMap b[4];  // B operand planes
  CUtensorMap c;     // output C viewed as fp32 [rows][2*cols], reduce-add target
};

__device__ __forceinline__ void epi_bar() {  // the 128 epilogue threads only
  asm volatile("bar.sync 1, 128;" ::: "memory");
}
template <int BN, int KIND>
__host__ __device__ constexpr uint32_t idesc_mma(bool negA) {
  return idesc_tc<TC_BM, BN, KIND>(negA);
}
// Product p of the 12 per K-step (p = 6*acc + 3*part + t):
//   acc 0 (re): part 0 Ar*Br, part 1 -Ai*Bi;  acc 1 (im): part 0 Ar*Bi, part 1 Ai*Br
//   t: 0 hi*hi, 1 hi*lo, 2 lo*hi.   Planes: 0 re_hi, 1 re_lo, 2 im_hi, 3 im_lo.
__device__ __forceinline__ void product(int p, int& qa, int& qb, int& acc, int& neg) {
  acc = p / 6;
  const int part = (p % 6) / 3, t = p % 3;
  const int a_im = part, b_im = acc == 0 ? part : 1 - part;
  qa = 2 * a_im + (t == 2);
  qb = 2 * b_im + (t == 1);
  neg = (acc == 0 && part == 1);
}

// Epilogue scales (power-of-two factors of the FP16 planes; all null for TF32):
// out[r][c] -= acc[r][c] * rowscale[(rowA0 + r) / rs_div] * colscale[rowB0 + c] * (*cscal).
struct TcScales {
  const float* rowscale;
  int rs_div;
  const float* colscale;
  const float* cscal;
  const int* skip;  // nonzero *skip: the launch does nothing (a stopped refinement)
  int upper;        // symmetric update (M == Nn, same origin): only the tiles that are not
                    // strictly below the diagonal (m0 < n0 + BN)
  int ksplit;       // > 1: every tile's K range in ksplit parts on different CTAs, each
                    // reduce-adding its partial product (K / KSTEP divisible by ksplit)
};

// Tile t of a launch: column-major over the mt x nt tiles, or, for an upper launch,
// over the tiles with m0 < n0 + BN only.  There column j holds G (j + 1) row tiles
// (G = BN / TC_BM; the last column may be cut at mt), so the first j columns hold
// S(j) = G j (j + 1) / 2 tiles and t's column is the largest j with S(j) <= t.
template <int BN>
__device__ __forceinline__ int upper_cum(int j) {
  return (BN / 128) * j * (j + 1) / 2;
}
template <int BN>
__device__ __forceinline__ int tile_count(int mt, int nt, int upper) {
  if (!upper) return mt * nt;
  return upper_cum<BN>(nt - 1) + min(mt, (BN / 128) * nt);
}
template <int BN>
__device__ __forceinline__ void tile_coords(int t, int mt, int nt, int upper, int& m0, int& n0) {
  if (!upper) {
    m0 = (t % mt) * 128;
    n0 = (t / mt) * BN;
    return;
  }
  int j = (int)((sqrtf(8.f * (float)t / (float)(BN / 128) + 1.f) - 1.f) * 0.5f);
  j = max(0, min(j, nt - 1));
  while (j > 0 && upper_cum<BN>(j) > t) --j;
  while (j + 1 < nt && upper_cum<BN>(j + 1) <= t) ++j;
  m0 = (t - upper_cum<BN>(j)) * 128;
  n0 = j * BN;
}

// NPROD = 3: the split products hi*hi, hi*lo, lo*hi (12 MMAs per K-step); NPROD = 1:
// hi*hi only (4 MMAs), and only the hi planes are loaded.
template <int BN, int KIND, int NPROD, bool LEAN = false>
__global__ void __launch_bounds__(TC_THREADS, 1)
tc_update_kernel(const __grid_constant__ TcMaps maps, int cx0, int cy0, int M, int Nn, int K,
                 int ax0, int rowA0, int bx0, int rowB0, TcScales sc, int* __restrict__ err) {
  using Cfg = TcCfg<BN, LEAN>;
  static_assert(NPROD == 1 || NPROD == 3, "one or three split products");
  constexpr int KSTEP = KIND == 0 ? 8 : 16;  // K elements per 32-byte operand row
  if (sc.skip && *sc.skip) return;           // before any barrier or TMEM allocation
  constexpr uint32_t B_PLANE_BYTES = Cfg::B_PLANE, STAGE_BYTES = Cfg::STAGE;
  constexpr int NBUF = Cfg::NBUF, NST = Cfg::STAGES;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  unsigned char* stages = smem;
  unsigned char* staging = stages + NST * STAGE_BYTES;  // 2 x 16 KB, 1024-aligned
  uint64_t* bars = reinterpret_cast<uint64_t*>(staging + 2 * STAGING_BYTES);
  // bars[0, NST) full, [NST, 2 NST) empty, [2 NST + 2b] tmem_full of accumulator set b,
  // [2 NST + 2b + 1] its tmem_empty
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * NST + 2 * NBUF);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  volatile int* epi_abort = abort_flag + 1;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int mt = (M + TC_BM - 1) / TC_BM;
  const int nt = (Nn + BN - 1) / BN;
  static_assert(TC_BM == 128 && BN % TC_BM == 0, "tile_coords assumes 128-row tiles");
  const int ntiles = tile_count<BN>(mt, nt, sc.upper);
  const int ksp = sc.ksplit > 1 ? sc.ksplit : 1;
  const int nunits = ntiles * ksp;           // unit u: tile u / ksp, K part u % ksp
  const int ksteps = K / KSTEP / ksp;        // K-steps per unit

  if (threadIdx.x == 0) {
    for (int s = 0; s < NST; ++s) {
      mbar_init(smem_u32(&bars[s]), 1);
      mbar_init(smem_u32(&bars[NST + s]), 1);
    }
    for (int b = 0; b < NBUF; ++b) {
      mbar_init(smem_u32(&bars[2 * NST + 2 * b]), 1);
      mbar_init(smem_u32(&bars[2 * NST + 2 * b + 1]), 4);
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
      for (int u = blockIdx.x; u < nunits && ok; u += gridDim.x) {
        int m0, n0;
        tile_coords<BN>(u / ksp, mt, nt, sc.upper, m0, n0);
        const int kbase = (u % ksp) * ksteps;
        for (int kk = 0; kk < ksteps; ++kk, ++it) {
          const int ks = kbase + kk;
          const uint32_t s = it % NST, ph = (it / NST) & 1;
          if (!mbar_wait(smem_u32(&bars[NST + s]), ph ^ 1, abort_flag)) { ok = false; break; }
          const uint32_t full = smem_u32(&bars[s]);
          mbar_expect_tx(full, NPROD == 3 ? STAGE_BYTES : STAGE_BYTES / 2);
          const uint32_t st = smem_u32(stages + s * STAGE_BYTES);
#pragma unroll
          for (int q = 0; q < 4; q += (NPROD == 3 ? 1 : 2))
            tma_load_2d(st + q * A_PLANE_BYTES, &maps.a[q], ax0 + ks * KSTEP, rowA0 + m0, full);
#pragma unroll
          for (int q = 0; q < 4; q += (NPROD == 3 ? 1 : 2))
            tma_load_2d(st + 4 * A_PLANE_BYTES + q * B_PLANE_BYTES, &maps.b[q], bx0 + ks * KSTEP,
                        rowB0 + n0, full);
        }
      }
      if (!ok) {
        *abort_flag = 1;
        atomicExch(err, 2);
      }
      // drain: the last (up to NST) issued stages must land before exit
      for (uint32_t k = (it > (uint32_t)NST ? it - NST : 0); k < it; ++k) {
        const unsigned long long t0 = gtimer();
        while (!mbar_try(smem_u32(&bars[k % NST]), (k / NST) & 1))
          if (gtimer() - t0 > RMAT_TC_WAIT_NS) break;
      }
    }
  } else if (warp == 1) {
    // ------------------------------- MMA issuer -------------------------------
    if (lane == 0) {
      uint32_t it = 0, tcount = 0;
      bool ok = true;
      uint32_t idesc[2] = {idesc_mma<BN, KIND>(false), idesc_mma<BN, KIND>(true)};
      uint32_t buf = 0, use = 0;
      for (int u = blockIdx.x; u < nunits && ok; u += gridDim.x, ++tcount) {
        buf = tcount % NBUF;
        use = tcount / NBUF;  // earlier units that used this accumulator set
        if (use > 0 &&
            !mbar_wait(smem_u32(&bars[2 * NST + 2 * buf + 1]), (use - 1) & 1, abort_flag)) {
          ok = false;
          break;
        }
        fence_after();
        for (int ks = 0; ks < ksteps; ++ks, ++it) {
          const uint32_t s = it % NST, ph = (it / NST) & 1;
          if (!mbar_wait(smem_u32(&bars[s]), ph, abort_flag)) { ok = false; break; }
          fence_after();
          const uint32_t st = smem_u32(stages + s * STAGE_BYTES);
#pragma unroll
          for (int p = 0; p < 12; ++p) {
            if (NPROD == 1 && p % 3 != 0) continue;  // hi*hi only
            int qa, qb, acc, neg;
            product(p, qa, qb, acc, neg);
            const uint64_t ad = sdesc_sw32(st + qa * A_PLANE_BYTES);
            const uint64_t bd = sdesc_sw32(st + 4 * A_PLANE_BYTES + qb * B_PLANE_BYTES);
            const uint32_t first = (ks == 0) && (p == 0 || p == 6);
            mma_issue<KIND>(tmem + buf * 2 * BN + acc * BN, ad, bd, idesc[neg], first ? 0u : 1u);
          }
          mma_commit(smem_u32(&bars[NST + s]));  // frees the stage once these MMAs have read it
        }
        if (!ok) break;
        mma_commit(smem_u32(&bars[2 * NST + 2 * buf]));  // accumulator set ready for the epilogue
      }
      if (!ok) {
        *abort_flag = 1;
        atomicExch(err, 2);
        // let every MMA issued so far finish before TMEM is released
        buf = tcount % NBUF;
        use = tcount / NBUF;
        mma_commit(smem_u32(&bars[2 * NST + 2 * buf]));
        const unsigned long long t0 = gtimer();
        while (!mbar_try(smem_u32(&bars[2 * NST + 2 * buf]), use & 1))
          if (gtimer() - t0 > RMAT_TC_WAIT_NS) break;
      }
    }
  } else {
    // -------------------------------- epilogue --------------------------------
    // TMEM row -> registers -> (negated) swizzled shared staging tile -> TMA
    // reduce-add into C.  The L2 performs C += (-acc); no load of C sits on this
    // path, and TMEM is handed back to the MMA warp as soon as it has been read.
    const int quad = warp & 3;               // TMEM lane quadrant this warp may access
    const int row = quad * 32 + lane;
    const bool leader = (warp == 2 && lane == 0);
    uint32_t tcount = 0, chunk = 0;
    for (int u = blockIdx.x; u < nunits; u += gridDim.x, ++tcount) {
      int m0, n0;
      tile_coords<BN>(u / ksp, mt, nt, sc.upper, m0, n0);
      const uint32_t buf = tcount % NBUF, use = tcount / NBUF;
      // The four epilogue warps leave together (they share named barriers): each
      // waits (bounded), then one thread snapshots the abort flag for all.
      if (!mbar_wait(smem_u32(&bars[2 * NST + 2 * buf]), use & 1, abort_flag)) {
        *abort_flag = 1;
        atomicExch(err, 2);
      }
      epi_bar();
      if (threadIdx.x == 64) *epi_abort = *abort_flag;
      epi_bar();
      if (*epi_abort) break;
      fence_after();
      const bool rowvalid = (m0 + row) < M;
      float rsc = sc.cscal ? *sc.cscal : 1.f;
      if (sc.rowscale && rowvalid) rsc *= sc.rowscale[(rowA0 + m0 + row) / sc.rs_div];
#pragma unroll 1
      for (int ch = 0; ch < BN / 16; ++ch, ++chunk) {
        float re[16], im[16];
        const uint32_t ta = tmem + buf * 2 * BN + ((uint32_t)(quad * 32) << 16) + ch * 16;
        tmem_ld16(ta, re);
        tmem_ld16(ta + BN, im);
        tmem_wait_ld();
        if (ch == BN / 16 - 1) {             // accumulator set fully read: release it
          fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(smem_u32(&bars[2 * NST + 2 * buf + 1]));
        }
        unsigned char* sbuf = staging + (chunk & 1) * STAGING_BYTES;
        if (leader) bulk_wait_read1();       // the reduce that used this buffer has read it
        epi_bar();
        float4* rowp = reinterpret_cast<float4*>(sbuf + row * 128);
        float cs[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) {
          // columns past Nn inside the output map (a launch narrower than the tile)
          // must add exactly zero
          const int col = n0 + ch * 16 + k;
          cs[k] = col < Nn ? -rsc * (sc.colscale ? sc.colscale[rowB0 + col] : 1.f) : 0.f;
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const float4 v = rowvalid ? make_float4(cs[2 * k] * re[2 * k], cs[2 * k] * im[2 * k],
                                                  cs[2 * k + 1] * re[2 * k + 1],
                                                  cs[2 * k + 1] * im[2 * k + 1])
                                    : make_float4(0.f, 0.f, 0.f, 0.f);
          rowp[k ^ (row & 7)] = v;
        }
        fence_proxy_async_smem();
        epi_bar();
        if (leader) {
          tma_reduce_add_2d(&maps.c, smem_u32(sbuf), 2 * (cx0 + n0 + ch * 16), cy0 + m0);
          bulk_commit();
        }
      }
    }
    if (leader) bulk_wait_all();
  }
  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 1)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
}

// ---------------------------------------------------------------------------
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return nullptr;
    fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

// C viewed as fp32 [rows][2*cols] (interleaved complex), 16 complex columns x 128 rows per box.
int make_out_map(CUtensorMap* m, void* base, int cols, int rows, int ld_complex) {
  EncodeTiledFn enc = encode_fn();
  if (!enc) return RMAT_ECUDA;
  cuuint64_t dims[2] = {(cuuint64_t)2 * cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)ld_complex * 2 * sizeof(float)};
  cuuint32_t box[2] = {32, (cuuint32_t)TC_BM};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, base, dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? RMAT_OK : RMAT_ECUDA;
}

// One operand plane, K-major [rows][row_stride] of fmt 0 (fp32 words holding TF32)
// or fmt 1 (fp16); boxes are 32 bytes of K (8 or 16 elements) by box_rows rows.
int make_plane_map(CUtensorMap* m, void* base, int fmt, int cols, int rows, int row_stride,
                   int box_rows) {
  EncodeTiledFn enc = encode_fn();
  if (!enc) return RMAT_ECUDA;
  const size_t esz = fmt == 1 ? 2 : 4;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)row_stride * esz};
  cuuint32_t box[2] = {(cuuint32_t)(32 / esz), (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(m, fmt == 1 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                   2, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_32B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? RMAT_OK : RMAT_ECUDA;
}

}  // namespace

int tc_make_plane_map_f16(CUtensorMap* m, void* base, int cols, int rows, int row_stride,
                          int box_rows) {
  return make_plane_map(m, base, 1, cols, rows, row_stride, box_rows);
}

namespace {

// Tensor maps of the three operand sources, rebuilt when a buffer or size changes:
//   F  full-size split factor planes, row-major [n][ldf]  (A operand; columns
//      limited to n, so K padding beyond the matrix reads zeros)
//   B  transposed U12 planes [n][256]                      (B operand of the factor update)
//   Y  transposed right-hand-side block planes [nrhs][256] (B operand of the solve updates)
struct TcCache {
  const void* f = nullptr;
  const void* b = nullptr;
  const void* y = nullptr;
  const void* cmat = nullptr;
  const void* bw = nullptr;
  int n = -1, ldf = -1, nrhs = -1, fmt = -1;
  TcMaps upd, sol[2];  // trailing update (BN = 256), solve update (BN = 128) per Y buffer
  TcMaps upd128;       // trailing update with 128-wide tiles (RMAT_PARAM_TC_BN = 128)
  TcMaps u12;          // U12 product: A = the (I - L11^-1) planes, B = upd128's
  const void* mpl = nullptr;
};
bool g_tc_attr[2][2][2][2] = {};

// The cache lives with its context (contexts may run concurrently on separate streams).
TcCache& tc_cache(rmat_ctx c) {
  if (!c->tc) c->tc = new TcCache();
  return *reinterpret_cast<TcCache*>(c->tc);
}

template <int BN, int KIND, int NPROD, bool LEAN = false>
int launch_tc_k(rmat_ctx c, const TcMaps& maps, int cx0, int cy0, int M, int Nn, int K, int ax0,
                int ay0, int bx0, int by0, const TcScales& sc, bool count_as_update) {
  constexpr int KSTEP = KIND == 0 ? 8 : 16;
  if (M <= 0 || Nn <= 0 || K <= 0) return RMAT_OK;
  if (K % KSTEP || ax0 % KSTEP || bx0 % KSTEP) return RMAT_ESTATE;
  constexpr size_t TC_SMEM = TcCfg<BN, LEAN>::SMEM;
  if (!g_tc_attr[BN == 128][KIND][NPROD == 1][LEAN]) {
    RMAT_CU(cudaFuncSetAttribute(tc_update_kernel<BN, KIND, NPROD, LEAN>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TC_SMEM));
    // the whole unified memory as shared memory, so other kernels' CTAs fit beside
    RMAT_CU(cudaFuncSetAttribute(tc_update_kernel<BN, KIND, NPROD, LEAN>,
                                 cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared));
    g_tc_attr[BN == 128][KIND][NPROD == 1][LEAN] = true;
  }
  if (sc.upper && (M != Nn || cx0 != cy0)) return RMAT_ESTATE;
  const int ksp = sc.ksplit > 1 ? sc.ksplit : 1;
  if ((K / KSTEP) % ksp) return RMAT_ESTATE;
  const int mt = ceil_div(M, TC_BM), nt = ceil_div(Nn, BN);
  const int tiles =
      (sc.upper ? (BN / TC_BM) * (nt - 1) * nt / 2 + std::min(mt, (BN / TC_BM) * nt) : mt * nt) *
      ksp;
  // a far-row update on the solves' look-ahead stream leaves SMs to the next step's
  // row update (its split-K units); the next diagonal application runs beside the
  // far update's CTAs (three-stage 128-wide tiles leave it the shared memory); the
  // factorisation's far update leaves the next pair's panels their CTAs (side_free)
  const int free_sms = c->side_free >= 0 ? c->side_free : c->la_free_sms;
  const bool on_side = (c->side && c->stream == c->side) || (c->grp_side && c->stream == c->grp_side);
  const int cap = on_side ? std::max(1, (c->sm_count - free_sms) / std::max(1, c->tc_cap_div))
                          : c->sm_count;
  const int grid = std::min(tiles, cap);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (c->timing && count_as_update) {
    e0 = rmat_event(c);
    e1 = rmat_event(c);
    RMAT_CU(cudaEventRecord(e0, c->stream));
  }
  tc_update_kernel<BN, KIND, NPROD, LEAN><<<grid, TC_THREADS, TC_SMEM, c->stream>>>(
      maps, cx0, cy0, M, Nn, K, ax0, ay0, bx0, by0, sc, c->dstat + ST_TIMEOUT);
  c->launches++;
  RMAT_CU(cudaGetLastError());
  if (count_as_update) {
    if (c->timing) {
      RMAT_CU(cudaEventRecord(e1, c->stream));
      c->tu_events.push_back({e0, e1});
    }
    c->tu_launches++;
    // a symmetric update's algorithmic work: the upper triangle and the lower halves
    // of the 128-row diagonal blocks the next factorisation steps read
    c->tu_flops += sc.upper ? 8.0 * K * (double)M * (M + TC_BM) / 2 : 8.0 * M * (double)Nn * K;
  }
  return RMAT_OK;
}

template <int BN>
int launch_tc(rmat_ctx c, const TcMaps& maps, int cx0, int cy0, int M, int Nn, int K, int ax0,
              int ay0, int bx0, int by0, const TcScales& sc, bool count_as_update) {
  // K beyond the block reads zeros: F columns past n are outside the tensor map and
  // the Y / B planes are zero-filled up to a multiple of 32
  if constexpr (BN == 256) {
    if (c->tc_lean) {  // a far update with look-ahead panels beside it
      if (rmat_plane_fmt(c->precision) == 1) {
        if (count_as_update && rmat_update_products(c->precision) == 1)
          return launch_tc_k<BN, 1, 1, true>(c, maps, cx0, cy0, M, Nn, (int)round_up(K, 16), ax0,
                                             ay0, bx0, by0, sc, count_as_update);
        return launch_tc_k<BN, 1, 3, true>(c, maps, cx0, cy0, M, Nn, (int)round_up(K, 16), ax0, ay0,
                                           bx0, by0, sc, count_as_update);
      }
      return launch_tc_k<BN, 0, 3, true>(c, maps, cx0, cy0, M, Nn, (int)round_up(K, 8), ax0, ay0,
                                         bx0, by0, sc, count_as_update);
    }
  }
  if (rmat_plane_fmt(c->precision) == 1) {
    if (count_as_update && rmat_update_products(c->precision) == 1)  // factor updates only
        return launch_tc_k<BN, 1, 1>(c, maps, cx0, cy0, M, Nn, (int)round_up(K, 16), ax0, ay0, bx0,
                                     by0, sc, count_as_update);
    return launch_tc_k<BN, 1, 3>(c, maps, cx0, cy0, M, Nn, (int)round_up(K, 16), ax0, ay0, bx0, by0,
                                 sc, count_as_update);
  }
  return launch_tc_k<BN, 0, 3>(c, maps, cx0, cy0, M, Nn, (int)round_up(K, 8), ax0, ay0, bx0, by0,
                               sc, count_as_update);
}

}  // namespace

size_t tc_lean_smem() { return TcCfg<256, true>::SMEM; }

int tc_prepare(rmat_ctx c, int n, int nrhs) {
  TcCache& g_tc = tc_cache(c);
  const int ldf = c->ld, fmt = rmat_plane_fmt(c->precision);
  if (g_tc.f == c->Fpl && g_tc.b == c->Bpl && g_tc.y == c->Ypl && g_tc.cmat == c->C &&
      g_tc.bw == c->Bw && g_tc.n == n && g_tc.ldf == ldf && g_tc.nrhs == nrhs && g_tc.fmt == fmt)
    return RMAT_OK;
  if (nrhs % 2) return RMAT_ESTATE;
  const size_t esz = rmat_plane_esz(c->precision);
  const size_t fplane = (size_t)n * ldf * esz, bplane = (size_t)n * RMAT_MAX_NB * esz,
               yplane = (size_t)RMAT_YPL_ROWS * RMAT_MAX_NB * esz;
  char* F = reinterpret_cast<char*>(c->Fpl);
  char* Bp = reinterpret_cast<char*>(c->Bpl);
  char* Y = reinterpret_cast<char*>(c->Ypl);
  for (int q = 0; q < 4; ++q) {
    RMAT_CHECK(make_plane_map(&g_tc.upd.a[q], F + q * fplane, fmt, n, n, ldf, TC_BM));
    RMAT_CHECK(make_plane_map(&g_tc.upd.b[q], Bp + q * bplane, fmt, RMAT_MAX_NB, n, RMAT_MAX_NB,
                              TC_BN));
    g_tc.upd128.a[q] = g_tc.upd.a[q];
    RMAT_CHECK(make_plane_map(&g_tc.upd128.b[q], Bp + q * bplane, fmt, RMAT_MAX_NB, n, RMAT_MAX_NB,
                              128));
    for (int u = 0; u < 2; ++u) {
      g_tc.sol[u].a[q] = g_tc.upd.a[q];
      RMAT_CHECK(make_plane_map(&g_tc.sol[u].b[q], Y + (4 * u + q) * yplane, fmt, RMAT_MAX_NB,
                                std::max(1, nrhs), RMAT_MAX_NB, 128));
    }
  }
  RMAT_CHECK(make_out_map(&g_tc.upd.c, c->C, n, n, c->ld));
  g_tc.upd128.c = g_tc.upd.c;
  RMAT_CHECK(make_out_map(&g_tc.sol[0].c, c->Bw, std::max(2, nrhs), n, std::max(2, nrhs)));
  g_tc.sol[1].c = g_tc.sol[0].c;
  g_tc.f = c->Fpl;
  g_tc.b = c->Bpl;
  g_tc.y = c->Ypl;
  g_tc.cmat = c->C;
  g_tc.bw = c->Bw;
  g_tc.n = n;
  g_tc.ldf = ldf;
  g_tc.nrhs = nrhs;
  g_tc.fmt = fmt;
  g_tc.mpl = nullptr;  // the U12 maps follow the plane format
  return RMAT_OK;
}

// Factor update: C22 -= L21 U12, A = F planes at (x = k0, y = k0+jb), B = U12^T planes.
// upper: C22 is complex symmetric and only its tiles on or above the diagonal are
// kept (the LDL^T factorisation reads the rest as the transpose).
int launch_trailing_tc(rmat_ctx c, float2* A, int ld, int k0, int jb, int n, bool upper) {
  const int rest = n - k0 - jb;
  if (rest <= 0) return RMAT_OK;
  if (reinterpret_cast<void*>(A) != c->C || ld != c->ld) return RMAT_ESTATE;
  RMAT_CHECK(tc_prepare(c, n, c->nrhs + (c->nrhs & 1)));
  TcCache& g_tc = tc_cache(c);
  TcScales sc{nullptr, 1, nullptr, nullptr, nullptr, upper ? 1 : 0};
  if (rmat_plane_fmt(c->precision) == 1) sc.cscal = c->uscale + k0 / jb;  // jb = nb here
  if (c->tc_bn == 128)
    return launch_tc<128>(c, g_tc.upd128, k0 + jb, k0 + jb, rest, rest, jb, k0, k0 + jb, 0, k0 + jb,
                          sc, true);
  return launch_tc<TC_BN>(c, g_tc.upd, k0 + jb, k0 + jb, rest, rest, jb, k0, k0 + jb, 0, k0 + jb,
                          sc, true);
}

int launch_u12_tc(rmat_ctx c, int n, int k0, int jb, int col0, int ncols, const float* minv_scale,
                  const float* b_scale) {
  if (ncols <= 0) return RMAT_OK;
  if (jb > 128 || !c->Mpl) return RMAT_ESTATE;
  RMAT_CHECK(tc_prepare(c, n, c->nrhs + (c->nrhs & 1)));
  TcCache& g_tc = tc_cache(c);
  const int fmt = rmat_plane_fmt(c->precision);
  if (g_tc.mpl != c->Mpl || g_tc.fmt != fmt) {
    const size_t mplane = (size_t)128 * 128 * rmat_plane_esz(c->precision);
    for (int q = 0; q < 4; ++q)
      RMAT_CHECK(make_plane_map(&g_tc.u12.a[q], reinterpret_cast<char*>(c->Mpl) + q * mplane, fmt,
                                128, 128, 128, TC_BM));
    g_tc.mpl = c->Mpl;
  }
  for (int q = 0; q < 4; ++q) g_tc.u12.b[q] = g_tc.upd128.b[q];
  g_tc.u12.c = g_tc.upd.c;
  // one 128-row tile row; no split of K (one reduce-add per element: every bit
  // reproducible)
  TcScales sc{fmt == 1 ? minv_scale : nullptr, 128, nullptr, fmt == 1 ? b_scale : nullptr, nullptr,
              0, 1};
  return launch_tc<128>(c, g_tc.u12, col0, k0, jb, ncols, jb, 0, 0, 0, col0, sc, false);
}

// Rectangular factor update C[rows row0.., cols col0..col0+ncols) -= F B: A = the split
// factor planes at K-columns ax0..ax0+K (rows row0..), B = the U12^T planes rows
// col0.. at K offset 0; uniform inverse scale *cscal (FP16 planes).  upper (row0 ==
// col0, M == ncols): only the tiles on or above the diagonal (symmetric C).
int launch_factor_tc(rmat_ctx c, int n, int row0, int M, int col0, int ncols, int K, int ax0,
                     const float* cscal, bool upper) {
  if (M <= 0 || ncols <= 0) return RMAT_OK;
  RMAT_CHECK(tc_prepare(c, n, c->nrhs + (c->nrhs & 1)));
  TcCache& g_tc = tc_cache(c);
  TcScales sc{nullptr, 1, nullptr, rmat_plane_fmt(c->precision) == 1 ? cscal : nullptr, nullptr,
              upper ? 1 : 0};
  if (c->tc_bn == 128)
    return launch_tc<128>(c, g_tc.upd128, col0, row0, M, ncols, K, ax0, row0, 0, col0, sc, true);
  return launch_tc<TC_BN>(c, g_tc.upd, col0, row0, M, ncols, K, ax0, row0, 0, col0, sc, true);
}

// Solve update: Bsub[M x nrhs] -= F[rows ay0.., cols k0..k0+jb] * Y, Y^T planes in Ypl.
// rowscale (FP16 planes): inverse scale per rs_div rows of F (the U blocks).
// ncols: the current column group's right-hand sides (columns ycol0.. of Bw, rows
// ycol0.. of the Y planes); the tensor maps span all ysolve_nrhs of the solve.
int launch_solve_tc(rmat_ctx c, int row0, int M, int ncols, int k0, int jb, int ay0, int n,
                    const float* rowscale, int rs_div, int ksplit) {
  RMAT_CHECK(tc_prepare(c, n, c->ysolve_nrhs > 0 ? c->ysolve_nrhs : ncols));
  TcCache& g_tc = tc_cache(c);
  TcScales sc{nullptr, 1, nullptr, nullptr, c->skip, 0, ksplit};
  if (rmat_plane_fmt(c->precision) == 1) {
    sc.rowscale = rowscale;
    sc.rs_div = rs_div;
    sc.colscale = rmat_ycs_cur(c) - c->ycol0;  // indexed by the plane row ycol0 + column
  }
  KTimer kt(c, KT_SOLVE_TC);
  RMAT_CHECK(launch_tc<128>(c, g_tc.sol[c->ybuf], c->ycol0, row0, M, ncols, jb, k0, ay0, 0,
                            c->ycol0, sc, false));
  kt.end();
  return RMAT_OK;
}

void tc_release(rmat_ctx c) {
  delete reinterpret_cast<TcCache*>(c->tc);
  c->tc = nullptr;
}
