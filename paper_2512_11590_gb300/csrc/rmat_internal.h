// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <cstddef>
#include <cstdint>
#include <vector>

#include "../../include/rmat.h"

// Maximum CTAs of the cooperative panel kernel (one per SM on GB300: 152).
#define RMAT_MAX_PANEL_CTAS 256
// Largest LU block width supported by the panel/TRSM kernels.
#define RMAT_MAX_NB 256
// Rows of the right-hand-side plane buffer (max nrhs on the tensor solve path).
#define RMAT_YPL_ROWS 1024

struct PanelScratch {
  // barrier counter + candidate slots of the one-barrier-per-column panel
  unsigned int* bar;   // [1]
  void* cval;          // [2][RMAT_MAX_PANEL_CTAS] of T
  int* cidx;           // [2][RMAT_MAX_PANEL_CTAS]
  void* crow;          // [2][RMAT_MAX_PANEL_CTAS][RMAT_MAX_NB] of complex T
  void* trow;          // [2][RMAT_MAX_NB] of complex T
};

// Net row permutation of each LU block (built once per factorisation, reused
// by every solve): rows [nblocks][2*nb] involved rows, idx [nblocks][nb] slot of
// each step's pivot row, src [nblocks][2*nb] net source slot of every involved
// slot, cnt [nblocks] involved-row count.
struct LUPerm {
  int* rows = nullptr;
  int* idx = nullptr;
  int* cnt = nullptr;
  int* src = nullptr;
  size_t cap = 0;  // bytes
};

// Refinement stopping rule at the FP64 floor: u = 2^-53; a residual is at the floor
// when max|r| <= RMAT_FLOOR_CONV u (max|C||X| + max|Phi|) (the floor of a correctly
// rounded solution is ~0.1-0.2 u on the config-3 family; a plain FP64 LU solve sits
// near 1 u).  Once the floor has been seen, one last correction is applied and the
// loop stops without the residual that would only confirm the floor.  A stalled
// refinement counts as converged below RMAT_FLOOR_STALL u.
#define RMAT_U64 1.1102230246251565e-16
#define RMAT_FLOOR_CONV 0.5
#define RMAT_FLOOR_STALL 2.0
static inline int rmat_floor_need(int) { return 1; }

// State of a device-driven refinement loop (graph-capturable solve).
struct IrState {
  double prev, rel;
  int stagn, done, status, iters, floor_hits, final;
};

// One system of a batch's small-system class (batch_small.cu): device pointers.
struct SmallSys {
  int nch, nlag, N, nopen;
  int sys;                      // index in the batch (status, refinement count)
  double hm, a, B, E, phi_max;
  const double2* V;             // cpot(nlag, nch, nch) of the system
  const double* K;              // hm T0 - hm (B/a) f f^T of its mesh, nlag x nlag
  const double* r;              // mesh points
  const double* fa;             // f_i(a)
  const int* l;
  const double* th;
  const double* zz;
  const int* open;
  double2* U;                   // column-major nopen x nopen output (null when nopen = 0)
};
// Per-CTA scratch of the small-system kernel: FP64 X and r (slot doubles2 each) and
// the matching system of collision_cta.cuh.
struct SmallScratch {
  double2* X;
  double2* R;
  size_t slot;
  void* coll;
};

// Device status words written by kernels (read back by the host).
enum { ST_INFO = 0, ST_TIMEOUT = 1, ST_BADARG = 2, ST_CHANFN = 3, ST_LMAX = 4, ST_COUNT = 8 };

struct rmat_ctx_s {
  int device = 0;
  cudaStream_t stream = nullptr;
  int sm_count = 0;
  // parameters
  int nb_param = 0;
  int panel_ctas_param = 0;
  long long spin_limit = 20000000LL;   // ~ seconds of polling
  int timing = 0;
  int smem_optin = 232448;  // cudaDeviceProp::sharedMemPerBlockOptin
  int smem_per_sm = 233472; // cudaDeviceProp::sharedMemPerMultiprocessor
  // device flag read by the refinement-loop kernels: nonzero = this system's
  // device-side refinement has stopped, so the launch returns at once (null: run)
  const int* skip = nullptr;
  int paired = 1;  // complex64 tensor path: two panels per trailing update (RMAT_PARAM_PAIRED)
  bool fpl_final = false;  // F's L parts carry all interchanges; pfwd is their composition
  int fpl_nb = 0;
  void* Bt = nullptr;      size_t Bt_cap = 0;       // gather target of the tensor forward solve
  int equil_param = -1;   // -1: default (on for complex64 paths), 0 off, 1 on
  bool equil = false;     // symmetric diagonal equilibration active for this problem
  // RMAT_PARAM_METHOD: 0 factor M itself, 1 Woodbury-kinetic (factor S = I + (K^-1 (x) I) W)
  int method_param = 0;
  bool woodbury = false;  // the assembled problem's factored matrix is S
  double* Kinv = nullptr;  size_t Kinv_cap = 0;     // K^-1 [nlag*nlag], FP64
  float* Kinv32 = nullptr; size_t Kinv32_cap = 0;   // K^-1 rounded to FP32
  int kinv_nlag = 0;       // mesh size K^-1 was formed for (0: stale)
  void* W32 = nullptr;     size_t W32_cap = 0;      // FP32 copy of Wpt for the S assembly
  void* Bs = nullptr;      size_t Bs_cap = 0;       // reordering scratch of the Woodbury solves
  // R-matrix propagation: a sector system (r1, r2) has right-hand sides
  // [phi_R | phi_L] (nrhs = 2 nch): fa = f_i(r2), faL = f_i(r1)
  bool sector = false;
  double mesh_r1 = -1.0;   // left end of the mesh the tables belong to (-1: regular (0, a))
  double* faL = nullptr;   size_t faL_cap = 0;
  void* prop = nullptr;    size_t prop_cap = 0;     // Rl, the four g blocks, scratch (nch^2 each)
  // sectors s >= 2 solved concurrently on worker contexts (own stream, own host thread)
  int prop_concurrent = 1;                // RMAT_PARAM_PROP_CONCURRENT
  std::vector<rmat_ctx> prop_workers;
  std::vector<cudaStream_t> prop_streams;
  // RMAT_PARAM_REFINE: 0 classical refinement, m > 0 FGMRES-IR with <= m inner steps
  int refine_param = 0;
  long long gm_inner = 0;  // FGMRES inner steps of the last rmat_solve
  void* gm_V = nullptr;     size_t gm_V_cap = 0;     // Krylov basis, (m+1) x N x nrhs FP64
  void* gm_Z = nullptr;     size_t gm_Z_cap = 0;     // preconditioned basis, m x N x nrhs FP64
  void* gm_T = nullptr;     size_t gm_T_cap = 0;     // product scratch, N x nrhs FP64
  void* gm_small = nullptr; size_t gm_small_cap = 0; // reduction partials, H columns, scales

  // problem description
  int kind = 0;          // 0 none, 1 assembled, 2 dense
  int precision = RMAT_C128;
  int N = 0, nrhs = 0, nch = 0, nlag = 0;
  int ld = 0;            // leading dimension (row-major) of the working matrix
  int nb = 0;            // LU block width in use
  double a = 0, hm = 0, bloch_B = 0, E = 0;
  std::vector<int> l;
  std::vector<double> thresh;
  std::vector<double> zz;  // Z1 Z2 e^2 per channel (0 = neutral)
  std::vector<double> K_host;  // hm*T0 - hm*(B/a) f f^T of the current mesh (host)
  std::vector<double> faL_host;  // f_i(r1) of a propagation sector (host)
  std::vector<double> f_a_host;
  double phi_max = 1.0;  // max |Phi| (denominator of the relative residual)

  // device buffers (capacity-managed)
  void* C = nullptr;       size_t C_cap = 0;        // working matrix, complex T, row-major N x ld
  double2* A64 = nullptr;  size_t A64_cap = 0;      // dense loaded system in complex128 (row-major)
  double2* B64 = nullptr;  size_t B64_cap = 0;      // dense loaded right-hand sides (row-major N x nrhs)
  int* ipiv = nullptr;     size_t ipiv_cap = 0;
  LUPerm perm_main, perm_z;                         // main factor / matching-system factor
  LUPerm perm_sub;                                  // 32-column sub-panels of a look-ahead panel
  double* Kmat = nullptr;  size_t Kmat_cap = 0;     // hm*T0 - hm*(B/a) f f^T  [nlag*nlag]
  double* T0 = nullptr;    size_t T0_cap = 0;       // T0 [nlag*nlag]
  double* rmesh = nullptr; size_t rmesh_cap = 0;    // r_i
  double* fa = nullptr;    size_t fa_cap = 0;       // f_i(a)
  int* l_d = nullptr;      size_t l_cap = 0;
  double* th_d = nullptr;  size_t th_cap = 0;
  double* zz_d = nullptr;  size_t zz_cap = 0;
  double2* Wpt = nullptr;  size_t Wpt_cap = 0;      // [nlag][nch][nch] point coupling incl. diagonal
  double2* X = nullptr;    size_t X_cap = 0;        // FP64 solution, row-major N x nrhs
  double2* Rres = nullptr; size_t Rres_cap = 0;     // FP64 residual, row-major N x nrhs
  void* Bw = nullptr;      size_t Bw_cap = 0;       // solve work in the factor precision
  void* Fpl = nullptr;     size_t Fpl_cap = 0;      // full-size split factor planes [4][N][ld] (A operand)
  void* Ypl = nullptr;     size_t Ypl_cap = 0;
  void* Dinv = nullptr;    size_t Dinv_cap = 0;     // inverted diagonal blocks (tensor solve path)
  void* Dinv2 = nullptr;   size_t Dinv2_cap = 0;    // inverses of pairs of 128-row blocks (256 rows)
  void* Pscr = nullptr;    size_t Pscr_cap = 0;     // scratch of their composition
  int inv_pairs = 0;       // pairs with a 256-row inverse (0: 128-row solve steps only)
  bool pairs_off = false;  // 128-row steps although pair inverses exist (refinement fallback)
  int la_free_sms = 16;    // SMs a look-ahead far update leaves to the next step's row update
  int side_free = -1;      // SMs a side-stream tensor update leaves free (-1: la_free_sms)
  bool tc_lean = false;    // 256-wide tensor updates with three stages (look-ahead far update)
  int factor_lookahead = 1;  // RMAT_PARAM_FACTOR_LOOKAHEAD: next pair's panels beside the far update
  int la_panel_ctas = 0;     // RMAT_PARAM_LA_PANEL_CTAS: CTAs of a look-ahead panel (0: all SMs)
  int la_min_rows = 0;       // RMAT_PARAM_LA_MIN_ROWS: far blocks at least this tall look ahead (0: 6144)
  int la_both_rows = 0;      // RMAT_PARAM_LA_BOTH_ROWS: ... with both panels beside the far update (0: 20480)
  int solve_blk = 256;     // RMAT_PARAM_SOLVE_BLOCK: rows per tensor-path solve step (256 or 128)
  int inv_blocks = 0, inv_nb = 0;      // right-hand-side block planes [4][RMAT_YPL_ROWS][256]
  void* Bpl = nullptr;     size_t Bpl_cap = 0;      // tensor B operand planes (U12^T split)
  void* Mpl = nullptr;     size_t Mpl_cap = 0;      // (I - L11^-1) planes, A operand of the U12 product
  int* pfwd = nullptr;     size_t pfwd_cap = 0;     // composed row permutation (tensor forward solve)
  // FP16 planes: per U block max bits and inverse scale 2^e, per right-hand-side
  // column inverse scale of the current solved block
  unsigned* umax = nullptr; size_t umax_cap = 0;
  float* uscale = nullptr; size_t uscale_cap = 0;
  float* ycs = nullptr;    size_t ycs_cap = 0;
  // The solves' Y planes and column scales are double-buffered: block k uses
  // buffer ybuf = k & 1, so block k+1's diagonal application can run while the
  // far-row update of block k (on the side stream) still reads buffer k & 1.
  int ybuf = 0;
  // Column groups of the tensor-path solves: group g owns right-hand-side columns
  // ycol0.. (rows ycol0.. of the Y planes, entries ycol0.. of the column scales) and
  // runs its sweeps on its own pair of streams, concurrently with the other groups
  int ycol0 = 0;
  int ysolve_nrhs = 0;             // right-hand sides of the whole solve (tensor maps)
  int solve_groups = 0;            // RMAT_PARAM_SOLVE_GROUPS (0: auto)
  int tc_cap_div = 1;              // side-stream solve updates share the SMs this many ways
  cudaStream_t grp_main = nullptr, grp_side = nullptr;  // streams of the second group
  cudaEvent_t grp_ev[6] = {};      // its look-ahead events [0..3], fork [4], join [5]
  int solve_lookahead = 1;         // RMAT_PARAM_SOLVE_LOOKAHEAD (2: next rows in the diagonal step)
  cudaStream_t side = nullptr;     // look-ahead stream of the solves
  cudaEvent_t la_ev[4] = {};       // fork / join events of the look-ahead
  double* Dsc = nullptr;   size_t Dsc_cap = 0;      // equilibration scale per row
  std::vector<double> ir_hist;                      // refinement history of the last solve
  double ir_berr = 0.0;  // last max|r| / (max|C||X| + max|Phi|) of the last solve
  double2* Xs = nullptr;   size_t Xs_cap = 0;       // rmat_residual's row-major copy of X
  double2* Rint = nullptr; size_t Rint_cap = 0;     // R-matrix (row-major nch x nch)
  double2* Zbuf = nullptr; size_t Zbuf_cap = 0;     // matching system (nch x nch + nch x nopen)
  int* zpiv = nullptr;     size_t zpiv_cap = 0;
  int* open_d = nullptr;   size_t open_cap = 0;
  unsigned long long* red = nullptr;                // reduction scratch [8]
  PanelScratch ps{};
  void* ps_mem = nullptr;
  int* dstat = nullptr;    // [ST_COUNT]
  int* hstat = nullptr;    // pinned mirror

  bool assembled = false, factored = false, solved = false;
  void* tc = nullptr;      // tensor-map cache of this context (gemm_tc.cu)
  void* oz = nullptr;      // tensor-core FP64 residual state (resid_oz.cu)
  // RMAT_PARAM_RESIDUAL: 0 auto (tensor-core coupling product from nch >= 32),
  // 1 FP64 tensor instruction (mma.m8n8k4.f64), 2 tensor-core digit slices
  int resid_param = 0;
  int tc_bn = 256;         // tile width of the factor's tensor-core updates (RMAT_PARAM_TC_BN)
  int factor_kind = 0;     // RMAT_PARAM_FACTOR: 0 LU with partial pivoting, 1 LDL^T
  int factor_used = 0;     // what rmat_factor runs / last ran (1: LDL^T)
  int resid_comp = -1;     // compensated kinetic sums (RMAT_PARAM_RESID_SUMS; -1 = complex128 only)
  long long wpt_gen = 0;   // bumped whenever the point-coupling table is rewritten
  long long kmat_gen = 0;  // bumped whenever the kinetic matrix is rewritten
  // CUDA graph of one complete solve (both sweeps), captured on first use and replayed
  // by every later solve with the same sizes, buffers and factor layout
  cudaGraphExec_t sg_exec = nullptr;
  std::vector<long long> sg_key;
  long long sg_launches = 0;
  bool borrowed_tables = false;  // mesh/channel tables owned by a batch, not freed here

  // statistics
  long long launches = 0, tu_launches = 0;
  double tu_flops = 0, tu_ms = 0;
  double stage_ms[5] = {-1, -1, -1, -1, -1};
  cudaEvent_t stage_ev[5][2] = {};
  std::vector<cudaEvent_t> ev_pool;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> tu_events;
  // per kernel class (KT_*): event pairs (timing on) and launch counts
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> kt_events[4];
  long long kt_launches[4] = {0, 0, 0, 0};
  size_t ev_next = 0;
};

// --- helpers implemented in api.cu ---------------------------------------
int rmat_grow(rmat_ctx c, void** p, size_t* cap, size_t bytes);
cudaEvent_t rmat_event(rmat_ctx c);

// --- host mesh (mesh.cpp) --------------------------------------------------
int rmat_mesh_host(int nlag, double a, double* x, double* omx, double* lam, double* r,
                   double* f_a, double* T0);

// --- kernel launchers ------------------------------------------------------
// assemble.cu
int launch_assemble(rmat_ctx c, const double2* V, double E);
int launch_point_coupling(rmat_ctx c, const double2* V, double E);
int launch_load_dense(rmat_ctx c, const double2* A, int lda, const double2* B, int ldb);
// lu.cu
template <class T>
int lu_factor_dev(rmat_ctx c, void* A, int n, int ld, int* ipiv, int nb, bool tensor,
                  const LUPerm& pm);
template <class T>
int lu_solve_dev(rmat_ctx c, const void* A, int n, int ld, const LUPerm& pm, int nb,
                 void* B, int ldb, int nrhs, bool tensor = false);
int perm_reserve(rmat_ctx c, LUPerm& pm, int n, int nb);
// gemm_tc.cu
int launch_trailing_tc(rmat_ctx c, float2* A, int ld, int k0, int jb, int n, bool upper = false);
// solve update: rows [row0, row0+M) of the solve buffer Bw (ld = nrhs) -= F(ay0.., k0..k0+jb) * Y
// Cluster size the cluster panel would use for M rows of width jb (0: does not fit).
int panel_cluster_fits(rmat_ctx c, int precision, int M, int jb);
// Woodbury-kinetic form (woodbury.cu)
int woodbury_prepare(rmat_ctx c, const double* K_host);
int launch_schur_assemble(rmat_ctx c);
int launch_kinv_apply(rmat_ctx c);
int launch_radial_to_channel(rmat_ctx c);
// FGMRES-IR (gmres.cu) and the pieces it shares with the classical loop
int launch_apply_resid(rmat_ctx c, const double2* Xin, double2* Rout);
int rmat_solve_system(rmat_ctx c);
int gmres_correction(rmat_ctx c, int m, double tau, int* inner);
// U12 = L11^-1 A12 in place on the tensor cores: C[k0.., col0..] -= Mpl B with the
// (I - L11^-1) planes in c->Mpl and A12^T split in c->Bpl rows col0.. (FP16 planes:
// inverse scales *minv_scale of Mpl and *b_scale of Bpl).
int launch_u12_tc(rmat_ctx c, int n, int k0, int jb, int col0, int ncols, const float* minv_scale,
                  const float* b_scale);
int launch_factor_tc(rmat_ctx c, int n, int row0, int M, int col0, int ncols, int K, int ax0,
                     const float* cscal, bool upper = false);
int launch_solve_tc(rmat_ctx c, int row0, int M, int ncols, int k0, int jb, int ay0, int n,
                    const float* rowscale, int rs_div, int ksplit = 1);
int tc_prepare(rmat_ctx c, int n, int nrhs);
void tc_release(rmat_ctx c);
// lu.cu (SIMT complex GEMM C -= A B, row-major)
int gemm_sub_c128(rmat_ctx c, int M, int N, int K, const double2* A, int lda, const double2* B,
                  int ldb, double2* C, int ldc);
int panel_ctas_for(rmat_ctx c, int M);
// Dynamic shared memory of a three-stage 256-wide tensor update CTA (the look-ahead's
// far part).
size_t tc_lean_smem();
// residual.cu
int launch_residual(rmat_ctx c, double* relres_dev_unused);
int launch_x_out(rmat_ctx c, double2* Xo, int ldx);
int launch_absmax(rmat_ctx c, const double2* v, size_t n);
int launch_update(rmat_ctx c, const IrState* st = nullptr);
int launch_ir_init(rmat_ctx c, IrState* st);
int launch_absprod(rmat_ctx c);
size_t small_coll_scratch_bytes();
size_t small_smem_bytes(int precision, int N, int nch);
int launch_batch_small(cudaStream_t st, int precision, const SmallSys* sys, int nsmall, int* next,
                       int grid, size_t smem, int max_refine, double tol, int* st_all,
                       IrState* ir_all, const SmallScratch& scr);
bool oz_enabled(rmat_ctx c);
int structured_residual(rmat_ctx c, const double2* Xin, double2* Rout, const int* skip);
int launch_to_colmajor(rmat_ctx c, const double2* src, double2* dst, int ld);
int launch_from_colmajor(rmat_ctx c, const double2* src, int ld, double2* dst);
int launch_oz_coupling(rmat_ctx c, const double2* Xin, double2* Rout, const int* skip);
bool oz_kinetic_enabled(rmat_ctx c);
int launch_oz_kinetic(rmat_ctx c, const double2* Xin, double2* Rout, const int* skip);
void oz_release(rmat_ctx c);
int launch_ir_state(rmat_ctx c, double tol, int patience, int last, IrState* st);
// api.cu: solve + refinement enqueued without host synchronisation (fixed step
// budget, device-side stopping rule); X stays in the context's FP64 buffer.
int enqueue_solve_refine(rmat_ctx c, int max_refine, double tol, IrState* st);
int ctx_reserve(rmat_ctx c, bool dense);
int launch_x_from_w(rmat_ctx c);
int launch_w_from_phi(rmat_ctx c);
// collision.cu
int launch_collision(rmat_ctx c, double2* R_dev, double2* U_dev, int nopen);
// U from the R-matrix already in c->Rint (row-major nch x nch), at radius c->a
int launch_u_from_rint(rmat_ctx c, double2* U_dev, int nopen);
// G[ab][al][be] = hm phi_a^T X_b for a, b in {R, L} (sector systems; Rl only for
// the first sector): four row-major nch x nch blocks RR, RL, LR, LL
int launch_sector_g(rmat_ctx c, double2* G);
int launch_prop_step(rmat_ctx c, double2* Rl, double2* G, double2* P);
int launch_prop_finish(rmat_ctx c, const double2* Rl, double2* Rout);
int rmat_sector_mesh_host(int nlag, double r1, double r2, double* r, double* lam, double* fL,
                          double* fR, double* Kf);
size_t collision_workspace_bytes(int nch);
// mesh.cpp: K = hm*T0 - (hm*(B/a)) * (f_i*f_j) in IEEE double, no contraction
void rmat_kinetic_table(int nlag, double hm, double s1, const double* T0, const double* fa, double* K);

// Records the failing call's CUDA error and source location (read back with
// rmat_last_error) before returning RMAT_ECUDA.
void rmat_note_cuda_error(int err, const char* file, int line);

#define RMAT_CU(x)                                        \
  do {                                                    \
    cudaError_t e__ = (x);                                \
    if (e__ != cudaSuccess) {                             \
      rmat_note_cuda_error((int)e__, __FILE__, __LINE__); \
      return RMAT_ECUDA;                                  \
    }                                                     \
  } while (0)

#define RMAT_CHECK(...)                             \
  do {                                              \
    int s__ = (__VA_ARGS__);                        \
    if (s__ != RMAT_OK) return s__;                 \
  } while (0)

// Kernel classes timed separately when timing is on (rmat_get_stats).
enum { KT_PANEL = 0, KT_APPLY_INV = 1, KT_SOLVE_TC = 2, KT_RESID = 3 };

// Brackets the launches of one kernel class with events on the context's stream.
struct KTimer {
  struct rmat_ctx_s* c;
  int k;
  cudaEvent_t e0 = nullptr;
  KTimer(struct rmat_ctx_s* c_, int k_);
  void end();
};

// Tensor-core operand planes: format 0 = TF32 hi/lo held in fp32 words, 1 = FP16 hi/lo.
static inline bool rmat_tensor_prec(int p) {
  return p == RMAT_C64_3XTF32_IR || p == RMAT_C64_3XF16_IR || p == RMAT_C64_1XF16_IR;
}
static inline int rmat_plane_fmt(int p) {
  return (p == RMAT_C64_3XF16_IR || p == RMAT_C64_1XF16_IR) ? 1 : 0;
}
static inline size_t rmat_plane_esz(int p) { return rmat_plane_fmt(p) == 1 ? 2 : 4; }
// split products per real product in the factor's trailing updates (the solves' block
// updates always take three)
static inline int rmat_update_products(int p) { return p == RMAT_C64_1XF16_IR ? 1 : 3; }
// current Y-plane buffer and its column scales
// (rows ycol0.. of the planes: the right-hand-side columns of the current column group)
static inline void* rmat_ypl_cur(rmat_ctx c) {
  return reinterpret_cast<char*>(c->Ypl) +
         ((size_t)c->ybuf * 4 * RMAT_YPL_ROWS + (size_t)c->ycol0) * RMAT_MAX_NB *
             rmat_plane_esz(c->precision);
}
static inline float* rmat_ycs_cur(rmat_ctx c) {
  return c->ycs + (size_t)c->ybuf * RMAT_YPL_ROWS + c->ycol0;
}

static inline int ceil_div(long long a, long long b) { return (int)((a + b - 1) / b); }
static inline long long round_up(long long a, long long b) { return (a + b - 1) / b * b; }
