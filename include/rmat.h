/*
 * rmat.h -- C ABI of the GB300 (sm_103a) Lagrange-Legendre R-matrix library.
 *
 * The library implements the hot path of the R-matrix method as described in
 * J. Lei, "HPRMAT: A high-performance R-matrix solver with GPU acceleration
 * for coupled-channel problems in nuclear physics" (arXiv 2512.11590):
 *
 *   rmat_mesh       Gauss-Legendre mesh on (0,a) and basis values at a (Sec. 2)
 *   rmat_assemble   C = T + L(B) + V - E*I, Eq. (block_structure), and the
 *                   surface right-hand sides of Sec. 3.1 step 2, on the device
 *   rmat_factor     blocked right-looking LU with partial pivoting, M = P L U
 *                   (Sec. 3.1), in complex128 or complex64 (Sec. 3.2, 3.4)
 *   rmat_solve      forward/backward substitution for all nch right-hand sides
 *                   plus iterative refinement with an FP64 residual r = b - M x
 *                   (Sec. 3.2; Sec. 3.4 step 7, here on the device)
 *   rmat_collision  R-matrix contraction (Sec. 3.1 step 4) and the collision
 *                   matrix U from matching at a (Sec. 1; Sec. 4.1)
 *   rmat_load_dense a general dense system M X = B, the analogue of the
 *                   paper's gpu_solve_mixed_(A, B, n, nrhs, ...) entry (Sec. 4.3)
 *
 * Conventions (all entry points):
 *   - Return 0 (RMAT_OK) on success; -i when argument i (1-based) is invalid;
 *     other negative values for CUDA / memory / state errors; positive values
 *     for numerical outcomes (exactly singular pivot, refinement stagnation).
 *   - Device pointers are plain CUDA device addresses owned by the caller; the
 *     library never frees them.  Host pointers are owned by the caller too.
 *   - Complex numbers are interleaved (re, im) pairs: complex128 = 2 doubles.
 *   - Matrices exchanged with the caller are column-major ("Fortran order"),
 *     the paper's layout (Sec. 3.4, Sec. 4.4).
 *   - Work is enqueued on the stream given to rmat_create, in call order.
 *     rmat_factor returns without waiting unless info is requested;
 *     rmat_solve synchronises once per refinement step (its stopping rule is
 *     decided on the host); rmat_collision synchronises before returning.
 *   - There is no CPU fallback: without a usable sm_103 device every entry
 *     point that needs one returns RMAT_ENODEV or RMAT_ECUDA.
 *   - A context is not thread safe; use one context per host thread.
 */
#ifndef RMAT_H_
#define RMAT_H_

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------- */
#define RMAT_OK            0
#define RMAT_ECUDA      (-100)  /* a CUDA runtime/driver call failed            */
#define RMAT_ENOMEM     (-101)  /* device memory for the workspace not available */
#define RMAT_ESTATE     (-102)  /* call out of order (e.g. solve before factor)  */
#define RMAT_ETIMEOUT   (-103)  /* a bounded device-side wait gave up            */
#define RMAT_ENODEV     (-104)  /* no CUDA device of compute capability 10.3     */
#define RMAT_ESINGULAR     1    /* exactly zero pivot; info holds its column     */
#define RMAT_ENOCONV       2    /* refinement stagnated above the FP64 floor     */
#define RMAT_ECHANFN       3    /* a Coulomb/Whittaker function did not converge */

/* ---- precisions --------------------------------------------------------- */
/* complex128 matrix, FP64 LU (panel, TRSM and trailing update on FP64 units). */
#define RMAT_C128            0
/* complex64 matrix and LU; trailing updates on tcgen05 tensor cores as three
 * TF32 products of a hi/lo split (~FP32 accuracy); FP64 residual refinement. */
#define RMAT_C64_3XTF32_IR   1
/* complex64 matrix and LU with FP32 CUDA-core trailing updates; FP64 refinement. */
#define RMAT_C64_SIMT_IR     2
/* complex64 matrix and LU; tensor-core updates as three FP16 products of a hi/lo
 * split (the same 22-bit operand precision as the TF32 split at twice the tensor
 * rate), with power-of-two scaling per U block and per right-hand-side column so
 * every operand stays in FP16 range; FP32 accumulation; FP64 residual refinement. */
#define RMAT_C64_3XF16_IR    3
/* As RMAT_C64_3XF16_IR, but the factor's trailing updates take ONE FP16 product per
 * real product (hi x hi: ~11-bit operands, FP32 accumulation), a third of the
 * tensor work; the factors are then accurate to ~u_16 cond(C) only, so classical
 * refinement converges only for cond(C) u_16 < 1: meant for GMRES-IR
 * (RMAT_PARAM_REFINE > 0), where the factors only precondition.  Solves apply the
 * stored factors with the three-product split. */
#define RMAT_C64_1XF16_IR    4

/* ---- tunable parameters (rmat_set_param) -------------------------------- */
#define RMAT_PARAM_NB          1  /* LU block width (multiple of 32; 0 = default: complex128
                                     32, 64 from N = 2048; complex64 64, 128 from N = 4096) */
#define RMAT_PARAM_PANEL_CTAS  2  /* CTAs of the grid panel (0 = auto: cluster panel
                                     when the rows fit one cluster, else grid) */
#define RMAT_PARAM_SPIN_LIMIT  3  /* polls before a device wait gives up        */
#define RMAT_PARAM_TIMING      4  /* 1 = record per-stage CUDA events           */
/* Symmetric diagonal equilibration of assembled problems: the factor is taken of
 * D C D with D = |diag C|^-1/2 (LAPACK-style scaling; the FP64 residual stays on C).
 * -1 = default (on for the complex64 precisions, off for RMAT_C128), 0 off, 1 on. */
#define RMAT_PARAM_EQUILIBRATE 5
/* Complex64 tensor-core precisions: 1 (default) = two panels share one trailing
 * update of depth 2*nb (half the passes over the trailing matrix), 0 = one update
 * per panel.  Results agree to rounding. */
#define RMAT_PARAM_PAIRED      6
/* Which matrix an assembled problem factors (the paper's Sec. 3.3 Type 3 split
 * M = K_diag + V_coupling, K the real kinetic + Bloch matrix shared by all channels):
 *   0 (default) M itself;
 *   1 Woodbury-kinetic: S = I + (K^-1 (x) I_nch) W in radial-major order
 *     ((i, al) -> i*nch + al), S[(i,al),(j,al')] = delta + Kinv[i][j] W_al,al'(r_j),
 *     W the per-point coupling (potential + centrifugal + threshold - E).  Every
 *     solve maps its right-hand side through K^-1 (FP64 accumulation) and reorders;
 *     the refinement keeps the FP64 residual of M, so X, R and U are those of M
 *     to the same tolerance.  K^-1 is formed once per mesh (host FP64).
 *     Equilibration is not applied to S.  Not used by rmat_load_dense or batches.
 * Takes effect at the next rmat_assemble. */
#define RMAT_PARAM_METHOD      7
/* Refinement of rmat_solve: 0 (default) classical, x += M^-1 r (Sec. 3.2);
 * m = 1..64 GMRES-IR: each correction solves C d = r by flexible GMRES in FP64
 * vectors with the FP64 product of C, right-preconditioned by the factors, with
 * at most m inner steps or until every column's GMRES residual is below 1e-6 of
 * its |r|.  Converges where cond(C) u_factor >= 1 stalls the classical loop.
 * The stopping rule (tol, stagnation, max_refine) counts outer corrections.
 * Not used by batches (their refinement is decided on the device). */
#define RMAT_PARAM_REFINE      8
/* Tensor-path solves: 1 (default) = look-ahead: each step's update of the next
 * step's rows runs first as a tensor-core launch of its own (its K range split over a
 * few CTAs); 2 = look-ahead with that update done inside the step's diagonal-block
 * application instead (the step's solution rows are in that kernel's shared memory,
 * the factor's split planes give the next rows' multipliers; CUDA cores, atomic
 * subtraction), one launch less per step but slower at N = 25600 (13.0 ms per solve
 * against 10.4 ms: the fused part takes ~25 us per step); in both the far rows'
 * update overlaps the next step on a second stream (the concurrent additions make the
 * rounding order, and so the last bits before the FP64 refinement, vary from run to
 * run); 0 = one update per step (every bit reproducible). */
#define RMAT_PARAM_SOLVE_LOOKAHEAD 9
/* rmat_propagate: 1 (default) = when every panel of a sector system fits one
 * thread-block cluster, sectors 2..ns are solved concurrently on worker contexts
 * (each with its own stream and host thread, kept in the context for later calls)
 * while sector 1 runs on the context itself; the propagation steps then run in
 * order.  With RMAT_PARAM_NB = 0 and a default block width too wide for a cluster
 * panel, every sector then uses width 64.  0 = sectors one after the other.
 * Results agree to rounding (identical when the block width is the same). */
#define RMAT_PARAM_PROP_CONCURRENT 10
/* Products of the FP64 refinement residual of assembled problems (Sec. 3.2 with the
 * block structure of Sec. 2): the point couplings (sum over al' of V_al,al'(r_i)
 * X[(al',i),be]) and the kinetic part (sum over j of K_ij X[(al,j),be]).
 * 1 = couplings in FP64 on the FP64 tensor instruction (mma.m8n8k4.f64), kinetic in
 * FP64; 2 = couplings FP64-accurate on the FP16 tensor cores: every row of V_i
 * (diagonal excluded, applied in FP64) and every column of X_i scaled by a power of
 * two and cut into nine signed 6-bit integer digits, the digit products with
 * p + q <= 8 summed exactly in FP32 tensor memory and combined in FP64 (error below
 * 2^-54 of the row and column scales; needs nch <= 2048, else 1), kinetic in FP64;
 * 3 = both products that way (the kinetic one with rows of K and columns of X_al
 * cut the same way; needs nlag <= 2048): faster, but K's rows are dominated by their
 * diagonal, so the cut at 2^-54 of each row's largest entry leaves ~nlag/2 u of
 * |K||X| per row and the refinement stops on a higher floor (about 2e-10 relative
 * residual at N = 25600 instead of 1e-12).  0 (default) auto = 2 when nch >= 32,
 * else 1.  Propagation sectors keep the kinetic part in FP64. */
#define RMAT_PARAM_RESIDUAL 11
/* Tile width (output columns per CTA tile) of the factor's tensor-core trailing
 * updates: 256 (0 = default) or 128 (twice the tiles, two accumulator sets per CTA:
 * better balance on small trailing blocks).  Results agree to rounding. */
#define RMAT_PARAM_TC_BN 12
/* Sums of the kinetic part of the FP64 residual (the dominant terms of C X, whose
 * rounding sets the refinement's floor): 1 = compensated (each product split exactly
 * by FMA, each addition by TwoSum, r rounded once: as if summed in twice the FP64
 * precision), 0 = FP64 sums, -1 (default) = compensated for RMAT_C128 only. */
#define RMAT_PARAM_RESID_SUMS 13
/* Rows per step of the tensor-path triangular solves (block width 128): 256 (0 =
 * default: the inverses of pairs of diagonal blocks are composed once per
 * factorisation, half the dependent steps per sweep) or 128.  Takes effect at the
 * next rmat_factor.  With 256, a classical refinement whose correction fails to
 * halve the residual switches to 128-row steps for the rest of that factorisation
 * (composed inverses of ill-conditioned blocks contract too little) instead of
 * counting a stall. */
#define RMAT_PARAM_SOLVE_BLOCK 14
/* Factorisation of the tensor-core precisions (RMAT_C64_3XTF32_IR, RMAT_C64_3XF16_IR,
 * RMAT_C64_1XF16_IR): 0 (default) = LU with partial pivoting (Sec. 3.1); 1 =
 * complex-symmetric LDL^T without pivoting, C = L D L^T with U = D L^T: each
 * diagonal block is factored alone, the multipliers below it are U12^T D11^-1 (C =
 * C^T for every assembled problem and for a loaded A that is symmetric; a loaded
 * A that is not gives a wrong factor, which the refinement reports as
 * RMAT_ENOCONV), and every trailing update keeps only the tiles on or above the
 * diagonal (half the tensor-core work; no pivot search).  Stable when the diagonal
 * dominates; the largest multiplier is in rmat_get_stats out[24], and a zero pivot
 * gives info > 0 as in LU.  The FP64 refinement is unchanged.  Other precisions,
 * the Woodbury system (RMAT_PARAM_METHOD = 1) and batches always pivot. */
#define RMAT_PARAM_FACTOR 15
/* Pivoted LU of the tensor-core precisions with paired panels (RMAT_PARAM_PAIRED = 1):
 * 1 (default) = look-ahead: while the far block is at least RMAT_PARAM_LA_MIN_ROWS
 * tall, each pair's far update is issued in two parts, the next pair's 2*nb columns
 * first on the context's stream and the rest on a second stream with three pipeline
 * stages (room on every SM for a panel CTA beside it); the next pair's first panel
 * (and, while the far block is at least RMAT_PARAM_LA_BOTH_ROWS tall, its second)
 * then runs beside it on the same SMs as 32-column sub-panels (the interchanges, U12
 * and the CUDA-core update of each sub-panel applied to the block's other columns
 * and to the second panel's columns before the next sub-panel), and the interchanges
 * that reach the far columns and the earlier L columns wait for it.  The pivots are
 * those of partial pivoting (the same columns in the same state); results agree with
 * 0 to rounding.  0 = one far update at a time; 2 = the look-ahead's order of work on
 * one stream (no concurrency: shows what the overlap hides).  LDL^T factorisations do
 * not use it. */
#define RMAT_PARAM_FACTOR_LOOKAHEAD 16
/* CTAs of a look-ahead sub-panel (grid variant; rows in shared memory when they fit):
 * 0 = default (every SM), 1..RMAT_MAX_PANEL_CTAS. */
#define RMAT_PARAM_LA_PANEL_CTAS 17
/* Smallest far block (rows) whose update the look-ahead splits: 0 = default 6144. */
#define RMAT_PARAM_LA_MIN_ROWS 18
/* Tensor-path solves with look-ahead (RMAT_PARAM_SOLVE_LOOKAHEAD = 1): the right-hand
 * sides in column groups whose forward and backward sweeps run concurrently, each on
 * its own pair of streams (the sweeps are chains of dependent steps that leave most
 * of the GPU idle; the columns are independent; two groups need nrhs a multiple of
 * 128 and at least 256).  0 = default (1), 1 = one group, 2 = two groups (measured at
 * N = 25600, 256 right-hand sides: 11.2 ms per solve against 10.4 ms for one group,
 * the groups' diagonal applications and far updates competing for the same SMs).
 * Results agree to rounding. */
#define RMAT_PARAM_SOLVE_GROUPS 19
/* Smallest far block (rows) beside whose far-far update both panels of the next pair
 * run (smaller ones down to RMAT_PARAM_LA_MIN_ROWS: the first panel only): 0 = default
 * 20480. */
#define RMAT_PARAM_LA_BOTH_ROWS 20

typedef struct rmat_ctx_s* rmat_ctx;

/* One coupled-channel problem (Eq. cc_schrodinger of Sec. 2).  N = nch*nlag.
 * Energies are in MeV, lengths in fm, hm = hbar^2/(2 mu) in MeV fm^2.  The
 * unknowns are ordered channel-major: index (alpha, i) -> alpha*nlag + i, the
 * (alpha-1)*nlag + i of the paper's R-matrix formula (Sec. 3.1), 0-based. */
typedef struct {
  int nch;               /* channels, >= 1                                     */
  int nlag;              /* Lagrange-Legendre points per channel, 1..1024      */
  double a;              /* channel radius (fm), > 0                           */
  double hm;             /* hbar^2 / 2mu (MeV fm^2), > 0                       */
  double bloch_B;        /* Bloch boundary constant B of L(B) (0 in the paper) */
  const int* l;          /* host [nch]: orbital momentum of each channel, >= 0 */
  const double* thresh;  /* host [nch]: channel threshold energies (MeV)       */
  int precision;         /* one of the RMAT_C128 / RMAT_C64_* precisions above */
  const double* zz;      /* host [nch] or NULL: Z1 Z2 e^2 of each channel (MeV fm),
                            >= 0 (repulsive); NULL or 0 = neutral channel.  The
                            Coulomb potential itself belongs in V; zz only selects
                            the asymptotic functions (eta_c = zz_c / (2 hm k_c)). */
} rmat_problem;

/* Create a context bound to CUDA device `device` and stream `stream` (a
 * cudaStream_t; NULL = legacy default stream).  The context owns all device
 * workspace (matrix, factors, pivots, refinement buffers), allocated lazily by
 * rmat_assemble/rmat_load_dense and reused while sizes do not grow, the
 * persistent-buffer pattern of the paper's Sec. 3.4 step 1.
 * Errors: -1 ctx NULL; RMAT_ENODEV when the device is not compute
 * capability 10.3; RMAT_ECUDA for other CUDA failures. */
int rmat_create(rmat_ctx* ctx, int device, void* stream);

/* Release the context and its workspace (synchronises its stream). NULL is a no-op. */
int rmat_destroy(rmat_ctx ctx);

/* Set a tunable parameter (RMAT_PARAM_*).  Takes effect at the next call. */
int rmat_set_param(rmat_ctx ctx, int key, long long value);

/* Lagrange-Legendre mesh of Sec. 2, computed on the HOST in IEEE double:
 *   x[i]   zeros of P_nlag(2x-1) on (0,1), ascending, correctly rounded
 *   omx[i] 1 - x[i], correctly rounded
 *   lam[i] Gauss weights on (0,1) (the paper's lambda_i on (0,a) is a*lam[i])
 *   r[i]   a*x[i]
 *   f_a[i] f_i(a) = (-1)^(nlag+i+1) / sqrt(a x_i (1-x_i)) (i 0-based): the
 *          boundary values q2(r_i) of Sec. 3.1 step 2
 *   T0     [nlag*nlag] kinetic+Bloch matrix int_0^a f_i' f_j' dr in fm^-2,
 *          symmetric (Baye's regularised Lagrange-Legendre closed forms)
 * Any output pointer may be NULL.  Needs no GPU.  Errors: -1 nlag out of
 * 1..1024, -2 a <= 0. */
int rmat_mesh(int nlag, double a, double* x, double* omx, double* lam, double* r,
              double* f_a, double* T0);

/* Assemble the internal-region matrix and right-hand sides on the device:
 *   C[(al,i),(al,j)]  = hm*T0[i][j] - hm*(B/a) f_i(a) f_j(a)
 *                       + delta_ij (hm l_al(l_al+1)/r_i^2 + V_alal(r_i) + E_al - E)
 *   C[(al,i),(al',i)] = V_al al'(r_i), al != al';  all other entries 0
 *   Phi[(al,i), be]   = delta_{al be} f_i(a)            (nch right-hand sides)
 * V_dev: device complex128 array cpot(nlag, nch, nch) in Fortran order, i.e.
 *   V_dev[i + nlag*(al + nch*al')] = V_{al al'}(r_i) in MeV, r_i = rmat_mesh's r,
 *   symmetric in (al, al').  Read during this call only.
 * C is stored in the precision's element type; the potential, thresholds and
 * mesh tables are kept for the FP64 residual.  Asynchronous.
 * Errors: -1 ctx, -2 problem fields invalid, -3 E not finite, -4 V_dev NULL,
 * RMAT_ENOMEM when N x N does not fit next to the free device memory. */
int rmat_assemble(rmat_ctx ctx, const rmat_problem* prob, double E, const void* V_dev);

/* Load a general dense system (no R-matrix structure): A_dev complex128 n x n
 * column-major with leading dimension lda >= n, B_dev complex128 n x nrhs
 * column-major with ldb >= n.  Both are copied into the context (converted to
 * the precision's element type); refinement then uses a dense FP64 residual
 * b - A x from the stored complex128 copy of A.  Asynchronous.
 * Errors: -1 ctx, -2 n < 1, -3 nrhs < 1, -4 A_dev, -5 lda, -6 B_dev, -7 ldb,
 * -8 precision; RMAT_ENOMEM. */
int rmat_load_dense(rmat_ctx ctx, int n, int nrhs, const void* A_dev, int lda,
                    const void* B_dev, int ldb, int precision);

/* Factor the assembled/loaded matrix in place: blocked right-looking LU with
 * partial pivoting (pivot = largest |Re|+|Im| in the column, first row on
 * ties).  If info != NULL the call synchronises and stores 0, or k > 0 (1-based
 * column) for the first exactly zero pivot, returning RMAT_ESINGULAR; with
 * info == NULL it returns after enqueueing.
 * Errors: -1 ctx, RMAT_ESTATE (nothing assembled), RMAT_ETIMEOUT, RMAT_ECUDA. */
int rmat_factor(rmat_ctx ctx, int* info);

/* Solve C X = Phi (or A X = B) with the factors, then refine (Sec. 3.2):
 *   loop: r = Phi - C X in FP64 (structured for assembled problems, dense for
 *   loaded ones; RMAT_PARAM_RESIDUAL, RMAT_PARAM_RESID_SUMS); stop with RMAT_OK
 *   when max|r|/max|Phi| < tol; when the normwise backward error
 *   max|r| / (max|C||X| + max|Phi|) is at most u/2 (u = 2^-53; |C||X| of the
 *   first solution, |.| the complex modulus: the FP64 floor, where r is the
 *   rounding of its own evaluation; a correctly rounded solution sits at ~0.1-0.2
 *   u, a plain FP64 LU solve near 1 u) apply one last correction and stop with
 *   RMAT_OK (no residual is formed after it);
 *   stop when the residual fails to drop below half of the previous step's
 *   value (once for the complex64 precisions, twice in a row for RMAT_C128):
 *   RMAT_OK when the backward error is then at most 2u, else RMAT_ENOCONV
 *   (stagnation above the floor, or divergence); stop after max_refine steps
 *   (RMAT_ENOCONV when tol > 0); else solve C d = r with the factors and
 *   X += d (FP64).
 * X_dev: device complex128 N x nrhs column-major, ldx >= N (caller-owned).
 * iters (may be NULL): refinement steps taken.  rel_resid (may be NULL): the
 * last max|r|/max|Phi| measured (0 when max_refine == 0 and tol <= 0, in
 * which case no residual is formed).  Returns RMAT_ENOCONV as above (X is
 * still the best iterate), RMAT_ESINGULAR after a zero pivot.
 * Errors: -1 ctx, -2 X_dev, -3 ldx, -4 max_refine < 0, RMAT_ESTATE. */
int rmat_solve(rmat_ctx ctx, void* X_dev, int ldx, int max_refine, double tol,
               int* iters, double* rel_resid);

/* R-matrix and collision matrix of the last solved assembled problem.
 *   R[al][be] = (hm/a) sum_i f_i(a) X[(al,i), be]    (dimensionless, nch x nch)
 *   k_c = sqrt(|E - E_c| / hm), rho_c = k_c a, eta_c = zz_c / (2 hm k_c);
 *   open channels (E > E_c): I = G - iF, O = G + iF with the Coulomb functions
 *   F_l(eta, rho), G_l(eta, rho) (Sec. 4.1; Riccati-Bessel F_l = rho j_l,
 *   G_l = -rho y_l when eta = 0), by Steed's continued fractions and, inside
 *   the Coulomb turning point, inward Taylor-series integration of G;
 *   closed channels: O = W_{-eta,l+1/2}(2 rho) (for eta = 0 the closed form
 *   e^-rho sum_k (l+k)!/(k!(l-k)!) (2 rho)^-k; for eta > 0 O = 1, O' = W'/W,
 *   which gives the same U), I = 0;
 *   O' -> O' - (B/rho) O, I' -> I' - (B/rho) I;  R~ = a sqrt(k) R sqrt(k);
 *   U = (diag O - R~ diag O')^-1 (diag I - R~ diag I'), open x open block.
 * R_dev: device complex128 nch x nch column-major (may be NULL).
 * U_dev: device complex128 nopen x nopen column-major, open channels in
 * channel order (may be NULL).  nopen: host int (may be NULL).
 * Synchronises.  Errors: -1 ctx, RMAT_ESTATE (no solved assembled problem),
 * RMAT_ESINGULAR (the matching matrix is singular), RMAT_ECHANFN (a channel
 * function did not converge within its iteration bound or overflowed). */
int rmat_collision(rmat_ctx ctx, void* R_dev, void* U_dev, int* nopen);

/* ---- R-matrix propagation over radial sectors --------------------------------
 * The internal region (0, a) cut at 0 = a_0 < a_1 < ... < a_ns = a (the ns sectors
 * of the paper's interface, Sec. 4).  Sector 1 uses rmat_mesh's regularised
 * basis on (0, a_1), its R-matrix in length units Rl = a_1 R(a_1) = hm Phi^T X;
 * sector s >= 2 uses rmat_sector_mesh's basis on (a_{s-1}, a_s), the Bloch
 * operator at both ends, and the blocks g_ab = hm phi_a^T C_s^-1 phi_b (a, b in
 * {L, R}: boundary values at a_{s-1}, a_s) of its Green's function:
 *   Rl <- g_RR - g_RL (Rl + g_LL)^-1 g_LR.
 * Then R = Rl / a and U as rmat_collision at a.  Every sector system is assembled,
 * factored and refined like rmat_assemble/rmat_factor/rmat_solve (the sector
 * systems with the 2 nch right-hand sides [phi_R | phi_L]) in the problem's
 * precision; the propagation step is FP64.
 *
 * rmat_sector_mesh: the non-regularised Lagrange-Legendre mesh of (r1, r2),
 *   f_i(r) = l_i(x) / sqrt(h w_i), x = (r - r1)/h, l_i the Lagrange polynomials
 *   of the Gauss-Legendre nodes of (0, 1) (weights w):  r[i] = r1 + h x_i,
 *   lam[i] = h w_i, fL[i] = f_i(r1), fR[i] = f_i(r2), Kf[i*nlag + j] =
 *   int_{r1}^{r2} f_i' f_j' dr (fm^-2).  Outputs may be NULL.  Needs no GPU.
 *   Errors: -1 nlag outside 2..1024, -2 not 0 <= r1 < r2.
 * rmat_propagate: prob->bloch_B must be 0 (the sector Bloch operators have B = 0);
 *   radii: host [ns+1], radii[0] = 0, increasing; V_dev[s]: device complex128
 *   cpot(nlag, nch, nch) (rmat_assemble's layout) at sector s's mesh points
 *   (rmat_mesh of a_1 for s = 0, rmat_sector_mesh of (a_s, a_{s+1}) after that);
 *   max_refine, tol as rmat_solve for every sector; R_dev (may be NULL), U_dev,
 *   nopen as rmat_collision.  Synchronises.  Returns RMAT_ENOCONV when a sector's
 *   refinement stopped above tol.  Errors: -2 prob invalid or B != 0, -3 ns or
 *   radii invalid, -4 V_dev, -5 max_refine < 0, -6 U_dev NULL with open channels,
 *   RMAT_ESINGULAR, RMAT_ECHANFN, RMAT_ETIMEOUT, RMAT_ENOMEM, RMAT_ECUDA.
 *   Leaves the context without a solved problem (rmat_collision: RMAT_ESTATE). */
int rmat_sector_mesh(int nlag, double r1, double r2, double* r, double* lam, double* fL,
                     double* fR, double* Kf);
int rmat_propagate(rmat_ctx ctx, const rmat_problem* prob, double E, int ns, const double* radii,
                   const void* const* V_dev, int max_refine, double tol, void* R_dev, void* U_dev,
                   int* nopen);

/* Counters and timers of the last factor/solve, for benchmarks:
 *   out[0] N, out[1] nrhs, out[2] LU block width, out[3] panel CTAs,
 *   out[4] kernel launches enqueued since the last rmat_reset_counters,
 *   out[5] trailing-update launches, out[6] trailing-update time (ms, events),
 *   out[7] trailing-update algorithmic flops (8 M N K per launch),
 *   out[8] assemble ms, out[9] factor ms, out[10] first solve ms,
 *   out[11] refinement ms, out[12] collision ms,
 *   out[13] / out[14] panel kernel ms / launches,
 *   out[15] / out[16] solve-path diagonal-block application ms / launches,
 *   out[17] / out[18] solve-path tensor-core block update ms / launches,
 *   out[19] / out[20] FP64 residual ms / launches, out[21] GMRES-IR inner steps of the
 *   last rmat_solve, out[22] the last normwise backward error of the last rmat_solve,
 *   max|r| / (max|C||X| + max|Phi|) (0 when no residual was formed),
 *   out[23] the factorisation of the last rmat_factor (0 LU with partial pivoting,
 *   1 LDL^T), out[24] its largest multiplier max(|Re|, |Im|) of L below the
 *   diagonal blocks (LDL^T only; -1 otherwise)
 *   (timers need RMAT_PARAM_TIMING=1; a time is -1 when it was not timed).
 * n: capacity of out; returns the number of values written (<= 25). */
int rmat_get_stats(rmat_ctx ctx, double* out, int n);
int rmat_reset_counters(rmat_ctx ctx);

/* The FP64 refinement residual of the current system for a caller's X (Sec. 3.2):
 *   R = Phi - C X for an assembled problem (block structure of Sec. 2, the point
 *   couplings as RMAT_PARAM_RESIDUAL selects), R = B - A X for a loaded one.
 * X_dev, R_dev: device complex128 N x nrhs column-major, leading dimensions
 * ldx, ldr >= N (caller-owned; X is read only).  Leaves the factors and the
 * solution untouched.  Synchronises.
 * Errors: -1 ctx, -2 X_dev, -3 ldx, -4 R_dev, -5 ldr, RMAT_ESTATE (nothing
 * assembled or loaded, or a propagation sector). */
int rmat_residual(rmat_ctx ctx, const void* X_dev, int ldx, void* R_dev, int ldr);

/* Refinement history of the last rmat_solve: hist[k] = max|r|/max|Phi| measured
 * before correction k (k = 0 is the residual of the first solve).  Returns the
 * number of entries available (may exceed n; only min(n, count) are written).
 * Errors: -1 ctx, -2 hist NULL with n > 0. */
int rmat_refine_history(rmat_ctx ctx, double* hist, int n);

/* ---- batches of independent systems ------------------------------------------
 * Many energies and partial waves of uneven size (the persistent-buffer energy
 * scan of Sec. 3.4 step 1, generalised).  All systems of a batch share one
 * precision.  The whole batch (assembly, factorisation, refined solve, R and U
 * for every system) is enqueued without host synchronisation and captured into
 * one CUDA graph that later runs replay; refinement uses max_refine steps with
 * the stopping rule of rmat_solve evaluated on the device.  The smallest systems
 * (RMAT_BATCH_SMALL_N) run in one persistent launch, a whole system per thread
 * block.  Systems with N > split_n run one after another with the full-device
 * path; the others are spread over `lanes` concurrent streams, provided their
 * panels fit the shared memory of one thread block cluster (up to 16 CTAs:
 * N <= ~6900 in complex64, ~3400 in complex128), whatever split_n says.
 * Refinement steps after a system has stopped return at once on the device.
 * rmat_batch_tune times candidate plans on the batch itself and keeps the fastest,
 * cached in the JSON-lines file named by the environment variable RMAT_TUNE_CACHE
 * when it is set: coordinate descent over the (lanes, split_n) plan, the
 * small-system class on or off, and the tile shapes (LU block width in lanes and
 * in the serial phase, tensor-update tile width in lanes). */
typedef struct rmat_batch_s* rmat_batch;
#define RMAT_BATCH_LANES   1  /* concurrent streams for small systems (0..16)   */
#define RMAT_BATCH_SPLIT_N 2  /* systems with N <= split_n go to the lanes      */
#define RMAT_BATCH_GRAPH   3  /* 1 = capture and replay a CUDA graph (default)  */
/* Systems with N <= small_n whose complex64 (complex128) matrix fits one thread
 * block's shared memory (N <= 160 (112) at a few channels) run in ONE persistent
 * launch, one system per thread block at a time: assembly, LU with partial
 * pivoting, solves, FP64 refinement, R and U without leaving the SM.  -1 (default)
 * = every system that fits, 0 = off. */
#define RMAT_BATCH_SMALL_N 4
#define RMAT_BATCH_NB_LANE 5    /* LU block width in lanes: 32, 64 (0 = 32 to N 1024, else 64) */
#define RMAT_BATCH_NB_SERIAL 6  /* LU block width of serial systems: 32, 64, 128 (0 = default) */
#define RMAT_BATCH_TC_BN 7      /* tensor-update tile width in lanes: 128 or 256 (0 = 256) */

/* probs[s], E[s], V_dev[s] (device complex128 cpot(nlag,nch,nch) of system s, as
 * in rmat_assemble) for s < nsys; the arrays are copied, V_dev must stay valid
 * while the batch is used.  Reserves all workspace.  Errors: -1 ctx, -2 nsys,
 * -3 a problem invalid or precisions differ, -4 E, -5 V_dev, -6 max_refine,
 * -8 out; RMAT_ENOMEM. */
int rmat_batch_create(rmat_ctx ctx, int nsys, const rmat_problem* probs, const double* E,
                      const void* const* V_dev, int max_refine, double tol, rmat_batch* out);
/* Open channels of every system (host int[nsys]). */
int rmat_batch_nopen(rmat_batch b, int* nopen);
int rmat_batch_set(rmat_batch b, int key, long long value);
/* Choose the plan (lanes, split_n, small-system class, block widths, tile width) by
 * timing candidates with the outputs U_dev; lanes and split_n are returned. */
int rmat_batch_tune(rmat_batch b, void* const* U_dev, int* lanes, int* split_n);
/* Run the batch: U_dev[s] = device complex128 nopen_s x nopen_s column-major
 * collision matrix of system s (may be NULL when nopen_s = 0).  status[s] and
 * iters[s] (host, may be NULL) receive each system's status (as rmat_solve /
 * rmat_collision) and refinement steps.  Synchronises.  Returns the most severe
 * negative status, else RMAT_OK (per-system numerical outcomes in status). */
int rmat_batch_run(rmat_batch b, void* const* U_dev, int* status, int* iters);
/* out[0] systems, out[1] lanes, out[2] split_n, out[3] graph (1 used, -1 capture
 * unavailable, 0 not yet), out[4] kernel launches enqueued so far, out[5] systems in
 * the small-system launch, out[6] small_n, out[7] lane block width, out[8] serial
 * block width (0 = defaults), out[9] tensor-update tile width in lanes. */
int rmat_batch_info(rmat_batch b, long long* out, int n);
int rmat_batch_destroy(rmat_batch b);

/* ---- allocation-free collision step ---------------------------------------
 * The paper has no counterpart of this entry point; it exists for callers that
 * cannot allocate device memory at the point where they need U: code whose
 * device memory is owned by a pool or caching allocator of another framework
 * (a cudaMalloc there fails or fragments the pool), code that must not
 * synchronise the device (cudaMalloc and cudaFree can), and loops with a fixed
 * memory budget.
 *
 * Computes the same R and U as rmat_collision, from a solution X the caller
 * already holds, in one kernel launch on `stream`, allocating nothing.  Its
 * scratch (the nch x nch matching system, channel functions, a status word)
 * is a fixed array in device memory, sized for nch <= RMAT_NOALLOC_MAX_NCH; every
 * GPU that loads the library holds it (about 200 KB) until the process exits.
 *   prob      problem description (nch 1..RMAT_NOALLOC_MAX_NCH; precision ignored)
 *   E         energy (MeV)
 *   f_a_dev   device double[nlag]: f_i(a), as returned by rmat_mesh
 *   X_dev     device complex128 N x nch column-major solution (ld = ldx >= N)
 *   R_dev     device complex128 nch x nch column-major output (may be NULL)
 *   U_dev     device complex128 nopen x nopen column-major output
 *   nopen     host int output (may be NULL)
 * The first call on a device (with that device current) looks up the scratch
 * array's device address and keeps it for the life of the process; make that
 * first call before any stream capture begins, and do not call again after a
 * cudaDeviceReset of that device (the reset may move the array).  All calls share
 * the one scratch array and it keeps the last call's contents (the kernel
 * rewrites everything it reads, and clears its status word, on every call):
 * calls that overlap on the GPU, from any stream or thread, race.  Each call
 * copies the status word to the host and synchronises `stream` before returning.
 * Errors: -1 prob invalid (nch outside 1..RMAT_NOALLOC_MAX_NCH, a, hm, bloch_B or
 * a threshold not finite, ...), -2 E not finite or a channel exactly at
 * threshold, -3 f_a_dev NULL, -4 X_dev NULL, -5 ldx < N, -7 U_dev NULL with open
 * channels, RMAT_ESINGULAR for an exactly singular matching system, RMAT_ECHANFN
 * for a channel function that did not converge, RMAT_ECUDA (rmat_last_error
 * names the failing call). */
#define RMAT_NOALLOC_MAX_NCH 64
int rmat_collision_noalloc(const rmat_problem* prob, double E, const void* f_a_dev,
                           const void* X_dev, int ldx, void* R_dev, void* U_dev, int* nopen,
                           void* stream);

/* Human-readable name of a status code (static storage). */
const char* rmat_status_string(int status);

/* The CUDA runtime error behind the calling thread's most recent RMAT_ECUDA
 * (0 if none yet); writes "file:line cudaErrorName: description" into buf
 * (NUL-terminated, truncated to len bytes; buf may be NULL). */
int rmat_last_error(char* buf, int len);

#ifdef __cplusplus
}
#endif
#endif /* RMAT_H_ */
