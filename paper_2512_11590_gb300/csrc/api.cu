// C ABI entry points (include/rmat.h): context, workspace, orchestration of
// assemble -> factor -> solve/refine -> collision on one stream.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <thread>
#include <vector>

#include "cplx.cuh"
#include "rmat_internal.h"

namespace {

size_t elem_bytes(int precision) { return precision == RMAT_C128 ? 16 : 8; }

int default_nb(int precision, int N) {
  if (precision == RMAT_C128) return N >= 2048 ? 64 : 32;
  return N >= 4096 ? 128 : 64;
}

int clamp_nb(int precision, int nb) { return std::min(nb, precision == RMAT_C128 ? 64 : 128); }

bool valid_precision(int p) {
  return p == RMAT_C128 || p == RMAT_C64_3XTF32_IR || p == RMAT_C64_SIMT_IR ||
         p == RMAT_C64_3XF16_IR || p == RMAT_C64_1XF16_IR;
}

int begin(rmat_ctx c) {
  if (!c) return -1;
  RMAT_CU(cudaSetDevice(c->device));
  return RMAT_OK;
}

int read_status(rmat_ctx c) {
  RMAT_CU(cudaMemcpyAsync(c->hstat, c->dstat, ST_COUNT * sizeof(int), cudaMemcpyDeviceToHost,
                          c->stream));
  RMAT_CU(cudaStreamSynchronize(c->stream));
  return RMAT_OK;
}

double read_red(rmat_ctx c) {
  unsigned long long bits = 0;
  if (cudaMemcpyAsync(c->hstat + ST_COUNT, c->red, sizeof(bits), cudaMemcpyDeviceToHost,
                      c->stream) != cudaSuccess)
    return NAN;
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return NAN;
  std::memcpy(&bits, c->hstat + ST_COUNT, sizeof(bits));
  double v;
  std::memcpy(&v, &bits, sizeof(v));
  return v;
}

// red[0] (max|r|) and red[1] (max|C||X|) in one copy
bool read_red2(rmat_ctx c, double* r0, double* r1) {
  if (cudaMemcpyAsync(c->hstat + ST_COUNT, c->red, 2 * sizeof(unsigned long long),
                      cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
      cudaStreamSynchronize(c->stream) != cudaSuccess)
    return false;
  std::memcpy(r0, c->hstat + ST_COUNT, sizeof(double));
  std::memcpy(r1, c->hstat + ST_COUNT + 2, sizeof(double));
  return true;
}

}  // namespace

// Reserve device memory for the problem; RMAT_ENOMEM when it cannot fit.
int ctx_reserve(rmat_ctx c, bool dense) {
  const size_t N = c->N, ld = c->ld, nrhs = c->nrhs;
  const size_t eb = elem_bytes(c->precision);
  const bool tensor = rmat_tensor_prec(c->precision);
  const size_t pe = rmat_plane_esz(c->precision);
  size_t need = 0;
  auto want = [&](size_t cap, size_t bytes) { need += bytes > cap ? bytes - cap : 0; };
  want(c->C_cap, N * ld * eb);
  want(c->X_cap, N * nrhs * 16);
  want(c->Rres_cap, N * nrhs * 16);
  want(c->Bw_cap, N * nrhs * eb);
  if (tensor) {
    want(c->Fpl_cap, 4 * N * ld * pe);
    want(c->Bpl_cap, 4 * N * RMAT_MAX_NB * pe);
    want(c->Ypl_cap, (size_t)8 * RMAT_YPL_ROWS * RMAT_MAX_NB * pe);
    want(c->Mpl_cap, (size_t)4 * 128 * 128 * pe);
  }
  if (dense) {
    want(c->A64_cap, N * N * 16);
    want(c->B64_cap, N * nrhs * 16);
  }
  size_t free_b = 0, total_b = 0;
  RMAT_CU(cudaMemGetInfo(&free_b, &total_b));
  if (need + (size_t)256 * 1024 * 1024 > free_b) return RMAT_ENOMEM;
  RMAT_CHECK(rmat_grow(c, &c->C, &c->C_cap, N * ld * eb));
  RMAT_CHECK(rmat_grow(c, (void**)&c->X, &c->X_cap, N * nrhs * 16));
  RMAT_CHECK(rmat_grow(c, (void**)&c->Rres, &c->Rres_cap, N * nrhs * 16));
  RMAT_CHECK(rmat_grow(c, &c->Bw, &c->Bw_cap, N * nrhs * eb));
  RMAT_CHECK(rmat_grow(c, (void**)&c->ipiv, &c->ipiv_cap, N * sizeof(int)));
  RMAT_CHECK(perm_reserve(c, c->perm_main, (int)N, c->nb));
  if (tensor) {
    RMAT_CHECK(rmat_grow(c, &c->Fpl, &c->Fpl_cap, 4 * N * ld * pe));
    RMAT_CHECK(rmat_grow(c, &c->Bpl, &c->Bpl_cap, 4 * N * RMAT_MAX_NB * pe));
    RMAT_CHECK(rmat_grow(c, &c->Ypl, &c->Ypl_cap, (size_t)8 * RMAT_YPL_ROWS * RMAT_MAX_NB * pe));
    RMAT_CHECK(rmat_grow(c, &c->Mpl, &c->Mpl_cap, (size_t)4 * 128 * 128 * pe));
    RMAT_CHECK(rmat_grow(c, (void**)&c->pfwd, &c->pfwd_cap, 2 * N * sizeof(int)));
    RMAT_CHECK(rmat_grow(c, &c->Bt, &c->Bt_cap, N * nrhs * eb));
    const size_t nblk = N / 32 + 5;  // per-block scales + the pair slot + two U12 slots + early U12
    RMAT_CHECK(rmat_grow(c, (void**)&c->umax, &c->umax_cap, nblk * sizeof(unsigned)));
    RMAT_CHECK(rmat_grow(c, (void**)&c->uscale, &c->uscale_cap, nblk * sizeof(float)));
    RMAT_CHECK(rmat_grow(c, (void**)&c->ycs, &c->ycs_cap, (size_t)2 * RMAT_YPL_ROWS * sizeof(float)));
    RMAT_CHECK(perm_reserve(c, c->perm_sub, (int)N, 32));  // look-ahead sub-panel row moves
    if (!c->side) {  // look-ahead stream of the tensor-path solves
      RMAT_CU(cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking));
      for (cudaEvent_t& e : c->la_ev) RMAT_CU(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    }
    if (!c->grp_main) {  // the second right-hand-side column group's streams
      RMAT_CU(cudaStreamCreateWithFlags(&c->grp_main, cudaStreamNonBlocking));
      RMAT_CU(cudaStreamCreateWithFlags(&c->grp_side, cudaStreamNonBlocking));
      for (cudaEvent_t& e : c->grp_ev) RMAT_CU(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    }
  }
  if (dense) {
    RMAT_CHECK(rmat_grow(c, (void**)&c->A64, &c->A64_cap, N * N * 16));
    RMAT_CHECK(rmat_grow(c, (void**)&c->B64, &c->B64_cap, N * nrhs * 16));
  }
  return RMAT_OK;
}

namespace {

int reserve(rmat_ctx c, bool dense) { return ctx_reserve(c, dense); }

void record_stage(rmat_ctx c, cudaEvent_t* ev) {
  if (c->timing) {
    *ev = rmat_event(c);
    cudaEventRecord(*ev, c->stream);
  } else {
    *ev = nullptr;
  }
}

double elapsed(cudaEvent_t a, cudaEvent_t b) {
  if (!a || !b) return -1.0;
  float ms = 0.f;
  if (cudaEventSynchronize(b) != cudaSuccess) return -1.0;
  if (cudaEventElapsedTime(&ms, a, b) != cudaSuccess) return -1.0;
  return ms;
}

}  // namespace

namespace {
thread_local int g_last_err = 0;
thread_local char g_last_where[192] = "";
}  // namespace

void rmat_note_cuda_error(int err, const char* file, int line) {
  g_last_err = err;
  const char* base = std::strrchr(file, '/');
  std::snprintf(g_last_where, sizeof(g_last_where), "%s:%d %s: %s", base ? base + 1 : file, line,
                cudaGetErrorName((cudaError_t)err), cudaGetErrorString((cudaError_t)err));
}

int perm_reserve(rmat_ctx c, LUPerm& pm, int n, int nb) {
  const size_t nblk = (size_t)(n + nb - 1) / nb;
  const size_t bytes = nblk * (5 * (size_t)nb + 1) * sizeof(int);
  if (bytes > pm.cap || !pm.rows) {
    void* p = pm.rows;
    size_t cap = pm.cap;
    RMAT_CHECK(rmat_grow(c, &p, &cap, bytes));
    pm.rows = reinterpret_cast<int*>(p);
    pm.cap = cap;
  }
  pm.idx = pm.rows + nblk * 2 * nb;
  pm.src = pm.idx + nblk * nb;
  pm.cnt = pm.src + nblk * 2 * nb;
  return RMAT_OK;
}

int rmat_grow(rmat_ctx c, void** p, size_t* cap, size_t bytes) {
  if (bytes <= *cap && *p) return RMAT_OK;
  if (*p) {
    RMAT_CU(cudaStreamSynchronize(c->stream));
    RMAT_CU(cudaFree(*p));
    *p = nullptr;
    *cap = 0;
  }
  if (bytes == 0) return RMAT_OK;
  if (cudaMalloc(p, bytes) != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return RMAT_ENOMEM;
  }
  *cap = bytes;
  return RMAT_OK;
}

cudaEvent_t rmat_event(rmat_ctx c) {
  if (c->ev_next >= c->ev_pool.size()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    c->ev_pool.push_back(e);
  }
  return c->ev_pool[c->ev_next++];
}

KTimer::KTimer(rmat_ctx c_, int k_) : c(c_), k(k_) {
  if (c->timing) {
    e0 = rmat_event(c);
    if (e0) cudaEventRecord(e0, c->stream);
  }
}

void KTimer::end() {
  c->kt_launches[k]++;
  if (e0) {
    cudaEvent_t e1 = rmat_event(c);
    if (e1) {
      cudaEventRecord(e1, c->stream);
      c->kt_events[k].push_back({e0, e1});
    }
  }
}

extern "C" {

int rmat_last_error(char* buf, int len) {
  if (buf && len > 0) {
    std::strncpy(buf, g_last_where, (size_t)len - 1);
    buf[len - 1] = 0;
  }
  return g_last_err;
}

const char* rmat_status_string(int s) {
  switch (s) {
    case RMAT_OK: return "ok";
    case RMAT_ECUDA: return "CUDA error";
    case RMAT_ENOMEM: return "out of device memory";
    case RMAT_ESTATE: return "call out of order";
    case RMAT_ETIMEOUT: return "bounded device wait timed out";
    case RMAT_ENODEV: return "no compute capability 10.3 device";
    case RMAT_ESINGULAR: return "exactly singular pivot";
    case RMAT_ENOCONV: return "refinement stagnated above tolerance";
    case RMAT_ECHANFN: return "a Coulomb/Whittaker channel function did not converge";
    default: return s < 0 && s > -100 ? "invalid argument" : "unknown status";
  }
}

int rmat_create(rmat_ctx* out, int device, void* stream) {
  if (!out) return -1;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    return RMAT_ENODEV;
  }
  if (device < 0 || device >= ndev) return -2;
  cudaDeviceProp prop;
  RMAT_CU(cudaGetDeviceProperties(&prop, device));
  if (prop.major != 10 || prop.minor != 3) return RMAT_ENODEV;
  RMAT_CU(cudaSetDevice(device));
  rmat_ctx c = new (std::nothrow) rmat_ctx_s();
  if (!c) return RMAT_ENOMEM;
  c->device = device;
  c->stream = reinterpret_cast<cudaStream_t>(stream);
  c->sm_count = prop.multiProcessorCount;
  c->smem_optin = (int)prop.sharedMemPerBlockOptin;
  c->smem_per_sm = (int)prop.sharedMemPerMultiprocessor;
  const size_t cs = sizeof(double2);
  const size_t ps_bytes = 256 + 2 * RMAT_MAX_PANEL_CTAS * sizeof(double) +
                          2 * RMAT_MAX_PANEL_CTAS * sizeof(int) +
                          (size_t)2 * RMAT_MAX_PANEL_CTAS * RMAT_MAX_NB * cs +
                          (size_t)2 * RMAT_MAX_NB * cs + 4 * 256;
  if (cudaMalloc(&c->ps_mem, ps_bytes) != cudaSuccess ||
      cudaMalloc((void**)&c->dstat, ST_COUNT * sizeof(int)) != cudaSuccess ||
      cudaMalloc((void**)&c->red, 8 * sizeof(unsigned long long)) != cudaSuccess ||
      cudaMallocHost((void**)&c->hstat, (ST_COUNT + 8) * sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    rmat_destroy(c);
    return RMAT_ENOMEM;
  }
  char* p = reinterpret_cast<char*>(c->ps_mem);
  c->ps.bar = reinterpret_cast<unsigned*>(p);
  p += 256;
  c->ps.cval = p;
  p += 2 * RMAT_MAX_PANEL_CTAS * sizeof(double);
  c->ps.cidx = reinterpret_cast<int*>(p);
  p += 2 * RMAT_MAX_PANEL_CTAS * sizeof(int);
  p = reinterpret_cast<char*>(round_up(reinterpret_cast<uintptr_t>(p), 256));
  c->ps.crow = p;
  p += (size_t)2 * RMAT_MAX_PANEL_CTAS * RMAT_MAX_NB * cs;
  c->ps.trow = p;
  if (cudaMemset(c->dstat, 0, ST_COUNT * sizeof(int)) != cudaSuccess) {
    rmat_destroy(c);
    return RMAT_ECUDA;
  }
  *out = c;
  return RMAT_OK;
}

int rmat_destroy(rmat_ctx c) {
  if (!c) return RMAT_OK;
  cudaSetDevice(c->device);
  cudaStreamSynchronize(c->stream);
  if (c->sg_exec) cudaGraphExecDestroy(c->sg_exec);
  for (rmat_ctx w : c->prop_workers) rmat_destroy(w);
  for (cudaStream_t s : c->prop_streams)
    if (s) cudaStreamDestroy(s);
  if (c->side) cudaStreamSynchronize(c->side);
  if (c->grp_main) cudaStreamSynchronize(c->grp_main);
  if (c->grp_side) cudaStreamSynchronize(c->grp_side);
  for (cudaEvent_t e : c->la_ev)
    if (e) cudaEventDestroy(e);
  for (cudaEvent_t e : c->grp_ev)
    if (e) cudaEventDestroy(e);
  if (c->side) cudaStreamDestroy(c->side);
  if (c->grp_main) cudaStreamDestroy(c->grp_main);
  if (c->grp_side) cudaStreamDestroy(c->grp_side);
  if (c->borrowed_tables) c->Kmat = c->T0 = c->rmesh = c->fa = nullptr, c->l_d = nullptr,
                          c->th_d = nullptr, c->zz_d = nullptr, c->open_d = nullptr;
  tc_release(c);
  oz_release(c);
  void* bufs[] = {c->C,    c->A64,  c->B64, c->ipiv, c->Kmat, c->T0,  c->rmesh,
                  c->fa,   c->l_d,  c->th_d, c->zz_d, c->Wpt, c->X,  c->Rres, c->Bw,
                  c->Fpl,  c->Bpl, c->Ypl,  c->Rint, c->Zbuf, c->zpiv, c->open_d, c->red,
                  c->ps_mem, c->dstat, c->Dsc, c->perm_main.rows, c->perm_z.rows, c->perm_sub.rows, c->Dinv,
                  c->umax, c->uscale, c->ycs, c->pfwd, c->Bt, c->Kinv, c->Kinv32, c->W32, c->Bs,
                  c->gm_V, c->gm_Z, c->gm_T, c->gm_small, c->faL, c->prop, c->Xs, c->Dinv2,
                  c->Pscr, c->Mpl};
  for (void* b : bufs)
    if (b) cudaFree(b);
  if (c->hstat) cudaFreeHost(c->hstat);
  for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
  delete c;
  return RMAT_OK;
}

int rmat_set_param(rmat_ctx c, int key, long long v) {
  if (!c) return -1;
  switch (key) {
    case RMAT_PARAM_NB:
      if (v < 0 || v > RMAT_MAX_NB || v % 32) return -3;
      c->nb_param = (int)v;
      return RMAT_OK;
    case RMAT_PARAM_PANEL_CTAS:
      if (v < 0 || v > RMAT_MAX_PANEL_CTAS) return -3;
      c->panel_ctas_param = (int)v;
      return RMAT_OK;
    case RMAT_PARAM_SPIN_LIMIT:
      if (v < 1) return -3;
      c->spin_limit = v;
      return RMAT_OK;
    case RMAT_PARAM_TIMING:
      c->timing = v ? 1 : 0;
      return RMAT_OK;
    case RMAT_PARAM_EQUILIBRATE:
      if (v < -1 || v > 1) return -3;
      c->equil_param = (int)v;
      return RMAT_OK;
    case RMAT_PARAM_PAIRED:
      if (v < 0 || v > 1) return -3;
      c->paired = (int)v;
      return RMAT_OK;
    case RMAT_PARAM_METHOD:
      if (v < 0 || v > 1) return -3;
      c->method_param = (int)v;
      return RMAT_OK;
    case RMAT_PARAM_REFINE:
      if (v < 0 || v > 64) return -3;
      c->refine_param = (int)v;
      return RMAT_OK;
    case RMAT_PARAM_SOLVE_LOOKAHEAD:
      if (v < 0 || v > 2) return -3;
      c->solve_lookahead = (int)v;
      return RMAT_OK;
    case RMAT_PARAM_PROP_CONCURRENT:
      if (v < 0 || v > 1) return -3;
      c->prop_concurrent = (int)v;
      return RMAT_OK;
    case RMAT_PARAM_RESIDUAL:
      if (v < 0 || v > 3) return -3;
      c->resid_param = (int)v;
      return RMAT_OK;
    case RMAT_PARAM_TC_BN:
      if (v != 0 && v != 128 && v != 256) return -3;
      c->tc_bn = v == 128 ? 128 : 256;
      return RMAT_OK;
    case RMAT_PARAM_RESID_SUMS:
      if (v < -1 || v > 1) return -3;
      c->resid_comp = (int)v;
      return RMAT_OK;
    case RMAT_PARAM_SOLVE_BLOCK:
      if (v != 0 && v != 128 && v != 256) return -3;
      c->solve_blk = v == 128 ? 128 : 256;
      return RMAT_OK;
    case RMAT_PARAM_FACTOR:
      if (v != 0 && v != 1) return -3;
      c->factor_kind = (int)v;
      return RMAT_OK;
    case RMAT_PARAM_FACTOR_LOOKAHEAD:
      if (v < 0 || v > 2) return -3;
      c->factor_lookahead = (int)v;
      return RMAT_OK;
    case RMAT_PARAM_LA_PANEL_CTAS:
      if (v < 0 || v > RMAT_MAX_PANEL_CTAS) return -3;
      c->la_panel_ctas = (int)v;
      return RMAT_OK;
    case RMAT_PARAM_LA_BOTH_ROWS:
      if (v < 0 || v > (1LL << 30)) return -3;
      c->la_both_rows = (int)v;
      return RMAT_OK;
    case RMAT_PARAM_SOLVE_GROUPS:
      if (v < 0 || v > 2) return -3;
      c->solve_groups = (int)v;
      return RMAT_OK;
    case RMAT_PARAM_LA_MIN_ROWS:
      if (v < 0 || v > (1LL << 30)) return -3;
      c->la_min_rows = (int)v;
      return RMAT_OK;
    default:
      return -2;
  }
}

int rmat_mesh(int nlag, double a, double* x, double* omx, double* lam, double* r, double* f_a,
              double* T0) {
  return rmat_mesh_host(nlag, a, x, omx, lam, r, f_a, T0);
}

// Assembly of the system of the regular mesh on (0, pb->a) (r2 <= 0) or of the
// propagation sector (r1, r2) with right-hand sides [phi_R | phi_L].
static int assemble_impl(rmat_ctx c, const rmat_problem* pb, double E, const void* V_dev,
                         double r1, double r2) {
  const bool sector = r2 > 0.0;
  if (!pb || pb->nch < 1 || pb->nlag < 1 || pb->nlag > 1024 || !(pb->a > 0) || !(pb->hm > 0) ||
      !std::isfinite(pb->bloch_B) || !pb->l || !pb->thresh || !valid_precision(pb->precision))
    return -2;
  if ((long long)pb->nch * pb->nlag > 200000) return -2;
  if (c->method_param == 1 && pb->nch > 65535) return -2;  // one grid z-slice per channel
  for (int k = 0; k < pb->nch; ++k)
    if (pb->l[k] < 0 || pb->l[k] > 64 || !std::isfinite(pb->thresh[k]) ||
        (pb->zz && !(std::isfinite(pb->zz[k]) && pb->zz[k] >= 0.0)))
      return -2;
  if (!std::isfinite(E)) return -3;
  if (!V_dev) return -4;
  const double a_key = sector ? r2 : pb->a, r1_key = sector ? r1 : -1.0;
  const bool mesh_same = c->nlag == pb->nlag && c->a == a_key && c->mesh_r1 == r1_key &&
                         c->hm == pb->hm && c->bloch_B == pb->bloch_B && c->Kmat != nullptr;
  c->kind = 1;
  c->sector = sector;
  c->precision = pb->precision;
  c->nch = pb->nch;
  c->nlag = pb->nlag;
  c->N = pb->nch * pb->nlag;
  c->nrhs = sector ? 2 * pb->nch : pb->nch;
  c->ld = (int)round_up(c->N, 32);
  c->a = a_key;
  c->mesh_r1 = r1_key;
  c->hm = pb->hm;
  c->bloch_B = pb->bloch_B;
  c->E = E;
  c->l.assign(pb->l, pb->l + pb->nch);
  c->thresh.assign(pb->thresh, pb->thresh + pb->nch);
  if (pb->zz) c->zz.assign(pb->zz, pb->zz + pb->nch);
  else c->zz.assign(pb->nch, 0.0);
  c->assembled = c->factored = c->solved = false;
  c->nb = clamp_nb(c->precision, c->nb_param ? c->nb_param : default_nb(c->precision, c->N));
  RMAT_CHECK(reserve(c, false));
  c->woodbury = !sector && c->method_param == 1;
  c->equil = !c->woodbury &&
             (c->equil_param == -1 ? c->precision != RMAT_C128 : c->equil_param == 1);
  if (c->equil) RMAT_CHECK(rmat_grow(c, (void**)&c->Dsc, &c->Dsc_cap, (size_t)c->N * sizeof(double)));
  if (c->woodbury)
    RMAT_CHECK(rmat_grow(c, &c->Bs, &c->Bs_cap,
                         (size_t)c->N * c->nrhs * (c->precision == RMAT_C128 ? 16 : 8)));
  const int nlag = c->nlag, nch = c->nch;
  RMAT_CHECK(rmat_grow(c, (void**)&c->Wpt, &c->Wpt_cap, (size_t)nlag * nch * nch * 16));
  RMAT_CHECK(rmat_grow(c, (void**)&c->l_d, &c->l_cap, nch * sizeof(int)));
  RMAT_CHECK(rmat_grow(c, (void**)&c->th_d, &c->th_cap, nch * sizeof(double)));
  RMAT_CHECK(rmat_grow(c, (void**)&c->zz_d, &c->zz_cap, nch * sizeof(double)));
  RMAT_CHECK(rmat_grow(c, (void**)&c->Rint, &c->Rint_cap, (size_t)nch * nch * 16));
  RMAT_CHECK(rmat_grow(c, (void**)&c->Zbuf, &c->Zbuf_cap, collision_workspace_bytes(nch)));
  RMAT_CHECK(rmat_grow(c, (void**)&c->zpiv, &c->zpiv_cap, nch * sizeof(int)));
  RMAT_CHECK(rmat_grow(c, (void**)&c->open_d, &c->open_cap, nch * sizeof(int)));
  if (!mesh_same) {
    std::vector<double> r(nlag), fa(nlag), T0((size_t)nlag * nlag), K((size_t)nlag * nlag);
    if (sector) {
      // K = hm int f_i' f_j' (Bloch terms at both ends included); fa = f_i(r2), faL = f_i(r1)
      std::vector<double> fL(nlag);
      RMAT_CHECK(rmat_sector_mesh_host(nlag, r1, r2, r.data(), nullptr, fL.data(), fa.data(),
                                       T0.data()));
      rmat_kinetic_table(nlag, c->hm, 0.0, T0.data(), fa.data(), K.data());
      RMAT_CHECK(rmat_grow(c, (void**)&c->faL, &c->faL_cap, nlag * 8));
      RMAT_CU(cudaMemcpy(c->faL, fL.data(), nlag * 8, cudaMemcpyHostToDevice));
      c->faL_host = fL;
    } else {
      RMAT_CHECK(rmat_mesh_host(nlag, c->a, nullptr, nullptr, nullptr, r.data(), fa.data(),
                                T0.data()));
      const double s1 = c->hm * (c->bloch_B / c->a);
      rmat_kinetic_table(nlag, c->hm, s1, T0.data(), fa.data(), K.data());
      c->faL_host.clear();
    }
    RMAT_CHECK(rmat_grow(c, (void**)&c->Kmat, &c->Kmat_cap, K.size() * 8));
    RMAT_CHECK(rmat_grow(c, (void**)&c->T0, &c->T0_cap, T0.size() * 8));
    RMAT_CHECK(rmat_grow(c, (void**)&c->rmesh, &c->rmesh_cap, nlag * 8));
    RMAT_CHECK(rmat_grow(c, (void**)&c->fa, &c->fa_cap, nlag * 8));
    RMAT_CU(cudaMemcpy(c->Kmat, K.data(), K.size() * 8, cudaMemcpyHostToDevice));
    c->kmat_gen++;  // the tensor-core residual's digit planes of K follow
    RMAT_CU(cudaMemcpy(c->T0, T0.data(), T0.size() * 8, cudaMemcpyHostToDevice));
    RMAT_CU(cudaMemcpy(c->rmesh, r.data(), nlag * 8, cudaMemcpyHostToDevice));
    RMAT_CU(cudaMemcpy(c->fa, fa.data(), nlag * 8, cudaMemcpyHostToDevice));
    c->f_a_host = fa;
    c->K_host = K;
    c->kinv_nlag = 0;  // K^-1 belongs to the previous mesh
  }
  if (c->woodbury && c->kinv_nlag != nlag) RMAT_CHECK(woodbury_prepare(c, c->K_host.data()));
  double pm = 0;
  for (double v : c->f_a_host) pm = std::max(pm, std::fabs(v));
  if (sector)
    for (double v : c->faL_host) pm = std::max(pm, std::fabs(v));
  c->phi_max = pm;
  RMAT_CU(cudaMemcpyAsync(c->l_d, c->l.data(), nch * sizeof(int), cudaMemcpyHostToDevice, c->stream));
  RMAT_CU(cudaMemcpyAsync(c->th_d, c->thresh.data(), nch * sizeof(double), cudaMemcpyHostToDevice,
                          c->stream));
  RMAT_CU(cudaMemcpyAsync(c->zz_d, c->zz.data(), nch * sizeof(double), cudaMemcpyHostToDevice,
                          c->stream));
  cudaEvent_t e0, e1;
  record_stage(c, &e0);
  if (c->woodbury) {  // S is built from the per-point table
    RMAT_CHECK(launch_point_coupling(c, reinterpret_cast<const double2*>(V_dev), E));
    RMAT_CHECK(launch_schur_assemble(c));
  } else {
    RMAT_CHECK(launch_assemble(c, reinterpret_cast<const double2*>(V_dev), E));
    RMAT_CHECK(launch_point_coupling(c, reinterpret_cast<const double2*>(V_dev), E));
  }
  record_stage(c, &e1);
  c->stage_ev[0][0] = e0;
  c->stage_ev[0][1] = e1;
  c->assembled = true;
  return RMAT_OK;
}

int rmat_assemble(rmat_ctx c, const rmat_problem* pb, double E, const void* V_dev) {
  RMAT_CHECK(begin(c));
  return assemble_impl(c, pb, E, V_dev, 0.0, -1.0);
}

int rmat_load_dense(rmat_ctx c, int n, int nrhs, const void* A_dev, int lda, const void* B_dev,
                    int ldb, int precision) {
  RMAT_CHECK(begin(c));
  if (n < 1 || n > 200000) return -2;
  if (nrhs < 1) return -3;
  if (!A_dev) return -4;
  if (lda < n) return -5;
  if (!B_dev) return -6;
  if (ldb < n) return -7;
  if (!valid_precision(precision)) return -8;
  c->kind = 2;
  c->equil = false;
  c->precision = precision;
  c->N = n;
  c->nrhs = nrhs;
  c->nch = c->nlag = 0;
  c->ld = (int)round_up(n, 32);
  c->assembled = c->factored = c->solved = false;
  c->nb = clamp_nb(precision, c->nb_param ? c->nb_param : default_nb(precision, n));
  RMAT_CHECK(reserve(c, true));
  RMAT_CHECK(launch_load_dense(c, reinterpret_cast<const double2*>(A_dev), lda,
                               reinterpret_cast<const double2*>(B_dev), ldb));
  RMAT_CHECK(launch_absmax(c, c->B64, (size_t)n * nrhs));
  c->phi_max = read_red(c);
  if (!(c->phi_max > 0)) c->phi_max = 1.0;
  c->assembled = true;
  return RMAT_OK;
}

int rmat_factor(rmat_ctx c, int* info) {
  RMAT_CHECK(begin(c));
  if (!c->assembled) return RMAT_ESTATE;
  RMAT_CU(cudaMemsetAsync(c->dstat, 0, ST_COUNT * sizeof(int), c->stream));
  cudaEvent_t e0, e1;
  record_stage(c, &e0);
  const bool tensor = rmat_tensor_prec(c->precision);
  // LDL^T needs C = C^T: not for the Woodbury system S
  c->factor_used = (tensor && c->factor_kind == 1 && !(c->woodbury && c->kind == 1)) ? 1 : 0;
  int st;
  if (c->precision == RMAT_C128)
    st = lu_factor_dev<double>(c, c->C, c->N, c->ld, c->ipiv, c->nb, false, c->perm_main);
  else
    st = lu_factor_dev<float>(c, c->C, c->N, c->ld, c->ipiv, c->nb, tensor, c->perm_main);
  if (st != RMAT_OK) return st;
  if (c->factor_used)  // the LDL^T multipliers' largest entry, for rmat_get_stats
    RMAT_CU(cudaMemcpyAsync(c->hstat + ST_COUNT + 6, c->dstat + ST_LMAX, sizeof(int),
                            cudaMemcpyDeviceToHost, c->stream));
  record_stage(c, &e1);
  c->factored = true;
  c->solved = false;
  c->stage_ev[1][0] = e0;
  c->stage_ev[1][1] = e1;
  if (info) {
    RMAT_CHECK(read_status(c));
    if (c->hstat[ST_TIMEOUT]) return RMAT_ETIMEOUT;
    *info = c->hstat[ST_INFO];
    if (*info) return RMAT_ESINGULAR;
  }
  return RMAT_OK;
}

static int solve_factors_direct(rmat_ctx c) {
  if (c->precision == RMAT_C128)
    return lu_solve_dev<double>(c, c->C, c->N, c->ld, c->perm_main, c->nb, c->Bw, c->nrhs,
                                c->nrhs);
  return lu_solve_dev<float>(c, c->C, c->N, c->ld, c->perm_main, c->nb, c->Bw, c->nrhs, c->nrhs,
                             rmat_tensor_prec(c->precision));
}

// Tensor-path solves are replayed from a CUDA graph (a solve is ~800 launches at
// N = 25600; replay removes the host launch cost).  Not while the stream is itself
// being captured (batches), on the legacy stream, with per-kernel timing on, or under
// a device-side stop flag.
static int solve_factors(rmat_ctx c) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (!rmat_tensor_prec(c->precision) || c->timing || c->skip || c->stream == nullptr ||
      cudaStreamIsCapturing(c->stream, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
    cudaGetLastError();
    return solve_factors_direct(c);
  }
  const std::vector<long long> key = {
      c->N, c->nb, c->nrhs, c->ld, c->precision, c->inv_blocks, c->inv_nb, c->fpl_final,
      c->fpl_nb, (long long)(uintptr_t)c->Bw, (long long)(uintptr_t)c->Fpl,
      (long long)(uintptr_t)c->Ypl, (long long)(uintptr_t)c->C, (long long)(uintptr_t)c->Dinv,
      (long long)(uintptr_t)c->Bt, (long long)(uintptr_t)c->pfwd,
      (long long)(uintptr_t)c->perm_main.rows, (long long)(uintptr_t)c->stream,
      (long long)(uintptr_t)c->uscale, (long long)(uintptr_t)c->ycs, c->solve_lookahead,
      (long long)(uintptr_t)c->side, c->inv_pairs, (long long)(uintptr_t)c->Dinv2, c->pairs_off,
      c->solve_groups, (long long)(uintptr_t)c->grp_main};
  if (!c->sg_exec || key != c->sg_key) {
    if (c->sg_exec) {
      cudaGraphExecDestroy(c->sg_exec);
      c->sg_exec = nullptr;
    }
    const long long l0 = c->launches;
    RMAT_CU(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeRelaxed));
    const int st = solve_factors_direct(c);
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(c->stream, &g);
    if (st != RMAT_OK || e != cudaSuccess || !g ||
        cudaGraphInstantiate(&c->sg_exec, g, 0) != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();
      c->sg_exec = nullptr;
      c->launches = l0;
      return st != RMAT_OK ? st : solve_factors_direct(c);
    }
    cudaGraphDestroy(g);
    c->sg_key = key;
    c->sg_launches = c->launches - l0;
    c->launches = l0;
  }
  RMAT_CU(cudaGraphLaunch(c->sg_exec, c->stream));
  c->launches += c->sg_launches;
  return RMAT_OK;
}

// One solve of the assembled system with the current factors, in place on Bw.
// Woodbury-kinetic: Bw -> (I (x) K^-1) Bw in radial-major order, the factors
// of S, then back to channel-major.
static int solve_system(rmat_ctx c) {
  if (!(c->woodbury && c->kind == 1)) return solve_factors(c);
  RMAT_CHECK(launch_kinv_apply(c));
  RMAT_CHECK(solve_factors(c));
  return launch_radial_to_channel(c);
}

}  // extern "C"

int rmat_solve_system(rmat_ctx c) { return solve_system(c); }

int enqueue_solve_refine(rmat_ctx c, int max_refine, double tol, IrState* st) {
  RMAT_CHECK(launch_w_from_phi(c));
  RMAT_CHECK(solve_system(c));
  RMAT_CHECK(launch_x_from_w(c));
  RMAT_CHECK(launch_absprod(c));
  RMAT_CHECK(launch_ir_init(c, st));
  const int patience = c->precision == RMAT_C128 ? 2 : 1;
  // once the stopping rule has fired, every later kernel of the loop returns at once
  c->skip = &st->done;
  int rc = RMAT_OK;
  for (int it = 0; it <= max_refine && rc == RMAT_OK; ++it) {
    rc = launch_residual(c, nullptr);
    if (rc == RMAT_OK) rc = launch_ir_state(c, tol, patience, it == max_refine, st);
    if (rc != RMAT_OK || it == max_refine) break;
    rc = solve_system(c);
    if (rc == RMAT_OK) rc = launch_update(c, st);
  }
  c->skip = nullptr;
  return rc;
}

// Whether the tensor-path solves take 256-row steps over composed pair inverses.
static bool pairs_in_use(rmat_ctx c) {
  return c->inv_pairs > 0 && !c->pairs_off && c->refine_param == 0 &&
         rmat_tensor_prec(c->precision);
}

// First solve and refinement of the factored system; X stays in c->X (FP64,
// row-major N x nrhs).  *status: RMAT_OK or RMAT_ENOCONV.
static int solve_refine(rmat_ctx c, int max_refine, double tol, int* iters, double* rel_resid,
                        int* status_out) {
  cudaEvent_t e0, e1, e2;
  record_stage(c, &e0);
  RMAT_CHECK(launch_w_from_phi(c));
  RMAT_CHECK(solve_system(c));
  RMAT_CHECK(launch_x_from_w(c));
  record_stage(c, &e1);
  int it = 0, status = RMAT_OK;
  double rel = 0.0;
  c->ir_hist.clear();
  c->gm_inner = 0;
  if (max_refine > 0 || tol > 0) {
    // |C||X| of the first solution sets the scale of the FP64 floor (X changes
    // only in its last digits after that)
    RMAT_CHECK(launch_absprod(c));
    double prev = INFINITY;
    // complex64 factors: one non-halving step ends the refinement (each extra
    // correction costs a full solve); complex128: two
    const int patience = c->precision == RMAT_C128 ? 2 : 1;
    const int need = rmat_floor_need(c->precision);
    int stagn = 0, floor_hits = 0;
    bool final = false;
    for (;;) {
      RMAT_CHECK(launch_residual(c, nullptr));
      double rmax = NAN, cx = NAN;
      if (!read_red2(c, &rmax, &cx)) return RMAT_ECUDA;
      rel = rmax / c->phi_max;
      const double scale = cx + c->phi_max;  // max|C||X| + max|Phi|
      c->ir_hist.push_back(rel);
      c->ir_berr = rmax / scale;
      floor_hits = rmax <= RMAT_FLOOR_CONV * RMAT_U64 * scale ? floor_hits + 1 : 0;
      if (!std::isfinite(rel)) {
        status = RMAT_ENOCONV;
        break;
      }
      if (rel < tol) break;
      if (it >= max_refine) {
        status = (tol > 0 && rmax > RMAT_FLOOR_STALL * RMAT_U64 * scale) ? RMAT_ENOCONV : RMAT_OK;
        break;
      }
      if (floor_hits >= need) {
        final = true;  // at the FP64 floor: one last correction, no confirming residual
      } else if (rel > 0.5 * prev && pairs_in_use(c)) {
        // the solves' 256-row steps apply composed inverses of pairs of diagonal
        // blocks; on ill-conditioned blocks they contract too little: 128-row steps
        // (the blocks' own inverses) from here on, without counting a stall
        c->pairs_off = true;
      } else if (rel > 0.5 * prev) {  // no longer contracting above the floor (or diverging)
        if (++stagn >= patience) {
          status = rmax <= RMAT_FLOOR_STALL * RMAT_U64 * scale ? RMAT_OK : RMAT_ENOCONV;
          break;
        }
      } else {
        stagn = 0;
      }
      prev = rel;
      if (c->refine_param > 0) {
        int inner = 0;
        RMAT_CHECK(gmres_correction(c, c->refine_param, 1e-6, &inner));
        c->gm_inner += inner;
      } else {
        RMAT_CHECK(solve_system(c));
        RMAT_CHECK(launch_update(c));
      }
      ++it;
      if (final) break;
    }
  }
  record_stage(c, &e2);
  c->stage_ev[2][0] = e0;
  c->stage_ev[2][1] = e1;
  c->stage_ev[3][0] = e1;
  c->stage_ev[3][1] = e2;
  if (iters) *iters = it;
  if (rel_resid) *rel_resid = rel;
  *status_out = status;
  return RMAT_OK;
}

extern "C" {

int rmat_solve(rmat_ctx c, void* X_dev, int ldx, int max_refine, double tol, int* iters,
               double* rel_resid) {
  RMAT_CHECK(begin(c));
  if (!X_dev) return -2;
  if (ldx < c->N) return -3;
  if (max_refine < 0) return -4;
  if (!c->factored) return RMAT_ESTATE;
  if (c->sector) return RMAT_ESTATE;  // a propagation sector's state is internal
  int status = RMAT_OK;
  RMAT_CHECK(solve_refine(c, max_refine, tol, iters, rel_resid, &status));
  RMAT_CHECK(launch_x_out(c, reinterpret_cast<double2*>(X_dev), ldx));
  RMAT_CHECK(read_status(c));
  if (c->hstat[ST_TIMEOUT]) return RMAT_ETIMEOUT;
  if (c->hstat[ST_BADARG]) return RMAT_ESTATE;
  c->solved = true;
  if (c->hstat[ST_INFO]) return RMAT_ESINGULAR;
  return status;
}

int rmat_collision(rmat_ctx c, void* R_dev, void* U_dev, int* nopen) {
  RMAT_CHECK(begin(c));
  if (!c->solved || c->kind != 1) return RMAT_ESTATE;
  std::vector<int> open;
  for (int k = 0; k < c->nch; ++k)
    if (c->E - c->thresh[k] > 0) open.push_back(k);
  const int no = (int)open.size();
  if (nopen) *nopen = no;
  cudaEvent_t e0, e1;
  record_stage(c, &e0);
  if (no > 0)
    RMAT_CU(cudaMemcpyAsync(c->open_d, open.data(), no * sizeof(int), cudaMemcpyHostToDevice,
                            c->stream));
  RMAT_CU(cudaMemsetAsync(c->dstat, 0, ST_COUNT * sizeof(int), c->stream));
  RMAT_CHECK(launch_collision(c, reinterpret_cast<double2*>(R_dev), reinterpret_cast<double2*>(U_dev),
                              no));
  record_stage(c, &e1);
  RMAT_CHECK(read_status(c));
  c->stage_ev[4][0] = e0;
  c->stage_ev[4][1] = e1;
  if (c->hstat[ST_TIMEOUT]) return RMAT_ETIMEOUT;
  if (c->hstat[ST_CHANFN]) return RMAT_ECHANFN;
  if (c->hstat[ST_INFO]) return RMAT_ESINGULAR;
  return RMAT_OK;
}

}  // extern "C"

// One propagation sector (r1, r2) on context w: assemble, factor, solve and refine,
// then its four g blocks into G.  Synchronises w's stream.  *st: RMAT_OK or ENOCONV.
static int sector_pipeline(rmat_ctx w, const rmat_problem* pb, double E, const void* V,
                           double r1, double r2, int max_refine, double tol, double2* G,
                           int* st) {
  RMAT_CHECK(assemble_impl(w, pb, E, V, r1, r2));
  int info = 0;
  RMAT_CHECK(rmat_factor(w, &info));
  int it = 0;
  double rel = 0.0;
  RMAT_CHECK(solve_refine(w, max_refine, tol, &it, &rel, st));
  RMAT_CHECK(launch_sector_g(w, G));
  RMAT_CHECK(read_status(w));
  if (w->hstat[ST_TIMEOUT]) return RMAT_ETIMEOUT;
  if (w->hstat[ST_INFO]) return RMAT_ESINGULAR;
  return RMAT_OK;
}

// Worker contexts for concurrent sectors (created once, kept in c).
static int prop_workers(rmat_ctx c, int n) {
  while ((int)c->prop_workers.size() < n) {
    cudaStream_t s = nullptr;
    RMAT_CU(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    c->prop_streams.push_back(s);
    rmat_ctx w = nullptr;
    RMAT_CHECK(rmat_create(&w, c->device, s));
    c->prop_workers.push_back(w);
  }
  for (int k = 0; k < n; ++k) {  // the caller's settings, without the options that need
    rmat_ctx w = c->prop_workers[k];  // the whole GPU or change the matrix
    w->nb_param = c->nb_param;
    w->spin_limit = c->spin_limit;
    w->equil_param = c->equil_param;
    w->paired = c->paired;
    w->refine_param = c->refine_param;
    w->panel_ctas_param = 0;
    w->method_param = 0;
    w->solve_lookahead = 0;
    w->factor_lookahead = 0;
    w->timing = 0;
  }
  return RMAT_OK;
}

extern "C" {

int rmat_sector_mesh(int nlag, double r1, double r2, double* r, double* lam, double* fL,
                     double* fR, double* Kf) {
  return rmat_sector_mesh_host(nlag, r1, r2, r, lam, fL, fR, Kf);
}

int rmat_propagate(rmat_ctx c, const rmat_problem* pb, double E, int ns, const double* radii,
                   const void* const* V_dev, int max_refine, double tol, void* R_dev, void* U_dev,
                   int* nopen) {
  RMAT_CHECK(begin(c));
  if (!pb || pb->bloch_B != 0.0 || pb->nlag < 2) return -2;
  if (ns < 1 || ns > 4096 || !radii || radii[0] != 0.0) return -3;
  for (int s = 1; s <= ns; ++s)
    if (!(radii[s] > radii[s - 1]) || !std::isfinite(radii[s])) return -3;
  if (!V_dev) return -4;
  for (int s = 0; s < ns; ++s)
    if (!V_dev[s]) return -4;
  if (max_refine < 0) return -5;
  const int nch = pb->nch;
  c->solved = false;
  std::vector<int> open;
  for (int k = 0; k < nch; ++k)
    if (E - pb->thresh[k] > 0) open.push_back(k);
  const int no = (int)open.size();
  if (nopen) *nopen = no;
  if (no > 0 && !U_dev) return -6;
  // With the default block width too wide for a cluster panel, the concurrent
  // mode uses width 64 (as batch lanes do) for every sector, sector 1 included.
  const int Ns = nch * pb->nlag;
  int nbq = clamp_nb(pb->precision, c->nb_param ? c->nb_param : default_nb(pb->precision, Ns));
  bool fits = panel_cluster_fits(c, pb->precision, Ns, nbq) > 0;
  if (!fits && !c->nb_param && nbq > 64 && panel_cluster_fits(c, pb->precision, Ns, 64) > 0) {
    nbq = 64;
    fits = true;
  }
  const bool conc = ns >= 2 && c->prop_concurrent && c->panel_ctas_param <= 0 && fits;
  struct NbRestore {  // the caller's block-width setting comes back on every return
    rmat_ctx c;
    int v;
    ~NbRestore() { c->nb_param = v; }
  } nb_restore{c, c->nb_param};
  if (conc) c->nb_param = nbq;
  // sector 1: the regular mesh on (0, a_1); Rl = a_1 R(a_1) = hm Phi^T X
  rmat_problem p0 = *pb;
  p0.a = radii[1];
  RMAT_CHECK(assemble_impl(c, &p0, E, V_dev[0], 0.0, -1.0));
  const size_t blk = (size_t)nch * nch;
  RMAT_CHECK(rmat_grow(c, &c->prop, &c->prop_cap, 6 * blk * sizeof(double2)));
  double2* Rl = reinterpret_cast<double2*>(c->prop);
  double2* G = Rl + blk;       // RR, RL, LR, LL
  double2* P = G + 4 * blk;
  int status = RMAT_OK, st = RMAT_OK, it = 0;
  double rel = 0.0;
  auto factor_solve = [&]() -> int {
    int info = 0;
    const int fs = rmat_factor(c, &info);
    if (fs != RMAT_OK) return fs;
    RMAT_CHECK(solve_refine(c, max_refine, tol, &it, &rel, &st));
    if (st != RMAT_OK) status = st;
    return RMAT_OK;
  };
  // Sectors are independent systems until the propagation steps.  When every
  // panel of a sector fits one thread-block cluster (no cooperative grid kernel
  // that needs every SM), sectors 2..ns run concurrently on worker contexts, each
  // from its own host thread, while sector 1 runs here.
  std::vector<int> wrc(ns + 1, RMAT_OK), wst(ns + 1, RMAT_OK);
  std::vector<std::thread> threads;
  if (conc) {
    RMAT_CHECK(prop_workers(c, ns - 1));
    for (int s = 2; s <= ns; ++s) {
      rmat_ctx w = c->prop_workers[s - 2];
      int r = rmat_grow(w, &w->prop, &w->prop_cap, 4 * blk * sizeof(double2));
      if (r != RMAT_OK) {
        wrc[s] = r;
        continue;
      }
      threads.emplace_back([&, s, w]() {
        cudaSetDevice(c->device);
        wrc[s] = sector_pipeline(w, pb, E, V_dev[s - 1], radii[s - 1], radii[s], max_refine,
                                 tol, reinterpret_cast<double2*>(w->prop), &wst[s]);
      });
    }
  }
  const int rc1 = factor_solve();
  const int rc2 = rc1 == RMAT_OK ? launch_sector_g(c, Rl) : rc1;
  for (std::thread& t : threads) t.join();
  RMAT_CHECK(rc2);
  for (int s = 2; s <= ns; ++s) {
    double2* Gs = G;
    if (conc) {
      RMAT_CHECK(wrc[s]);
      if (wst[s] != RMAT_OK) status = wst[s];
      Gs = reinterpret_cast<double2*>(c->prop_workers[s - 2]->prop);
    } else {
      RMAT_CHECK(assemble_impl(c, pb, E, V_dev[s - 1], radii[s - 1], radii[s]));
      RMAT_CHECK(factor_solve());
      RMAT_CHECK(launch_sector_g(c, G));
    }
    // Rl <- g_RR - g_RL (Rl + g_LL)^-1 g_LR  (FP64 LU of the nch x nch matrix)
    RMAT_CHECK(launch_prop_step(c, Rl, Gs, P));
  }
  // R(a) = Rl / a and U at a = a_ns
  c->a = radii[ns];
  RMAT_CHECK(launch_prop_finish(c, Rl, reinterpret_cast<double2*>(R_dev)));
  if (no > 0)
    RMAT_CU(cudaMemcpyAsync(c->open_d, open.data(), no * sizeof(int), cudaMemcpyHostToDevice,
                            c->stream));
  RMAT_CHECK(launch_u_from_rint(c, reinterpret_cast<double2*>(U_dev), no));
  RMAT_CHECK(read_status(c));
  if (c->hstat[ST_TIMEOUT]) return RMAT_ETIMEOUT;
  if (c->hstat[ST_CHANFN]) return RMAT_ECHANFN;
  if (c->hstat[ST_INFO]) return RMAT_ESINGULAR;
  return status;
}

static float lmax_bits(int b) {
  float f;
  std::memcpy(&f, &b, sizeof(f));
  return f;
}

int rmat_get_stats(rmat_ctx c, double* out, int n) {
  if (!c) return -1;
  if (!out || n < 0) return -2;
  auto sum = [](const std::vector<std::pair<cudaEvent_t, cudaEvent_t>>& evs) {
    if (evs.empty()) return -1.0;
    double t = 0;
    for (auto& pr : evs) {
      const double ms = elapsed(pr.first, pr.second);
      if (ms < 0) return -1.0;
      t += ms;
    }
    return t;
  };
  for (int k = 0; k < 5; ++k)
    c->stage_ms[k] = elapsed(c->stage_ev[k][0], c->stage_ev[k][1]);
  const double v[25] = {(double)c->N, (double)c->nrhs, (double)c->nb,
                        (double)panel_ctas_for(c, c->N > 0 ? c->N : 1), (double)c->launches,
                        (double)c->tu_launches, sum(c->tu_events), c->tu_flops, c->stage_ms[0],
                        c->stage_ms[1], c->stage_ms[2], c->stage_ms[3], c->stage_ms[4],
                        sum(c->kt_events[KT_PANEL]), (double)c->kt_launches[KT_PANEL],
                        sum(c->kt_events[KT_APPLY_INV]), (double)c->kt_launches[KT_APPLY_INV],
                        sum(c->kt_events[KT_SOLVE_TC]), (double)c->kt_launches[KT_SOLVE_TC],
                        sum(c->kt_events[KT_RESID]), (double)c->kt_launches[KT_RESID],
                        (double)c->gm_inner, c->ir_berr, (double)c->factor_used,
                        c->factor_used ? (double)lmax_bits(c->hstat[ST_COUNT + 6]) : -1.0};
  const int m = n < 25 ? n : 25;
  for (int k = 0; k < m; ++k) out[k] = v[k];
  return m;
}

int rmat_residual(rmat_ctx c, const void* X_dev, int ldx, void* R_dev, int ldr) {
  RMAT_CHECK(begin(c));
  if (!X_dev) return -2;
  if (ldx < c->N) return -3;
  if (!R_dev) return -4;
  if (ldr < c->N) return -5;
  if (!c->assembled || c->sector) return RMAT_ESTATE;
  RMAT_CHECK(rmat_grow(c, (void**)&c->Xs, &c->Xs_cap, (size_t)c->N * c->nrhs * 16));
  RMAT_CHECK(launch_from_colmajor(c, reinterpret_cast<const double2*>(X_dev), ldx, c->Xs));
  RMAT_CHECK(launch_apply_resid(c, c->Xs, c->Rres));
  RMAT_CHECK(launch_to_colmajor(c, c->Rres, reinterpret_cast<double2*>(R_dev), ldr));
  RMAT_CU(cudaStreamSynchronize(c->stream));
  return RMAT_OK;
}

int rmat_refine_history(rmat_ctx c, double* hist, int n) {
  if (!c) return -1;
  if (!hist && n > 0) return -2;
  const int cnt = (int)c->ir_hist.size();
  for (int k = 0; k < std::min(n, cnt); ++k) hist[k] = c->ir_hist[k];
  return cnt;
}

int rmat_reset_counters(rmat_ctx c) {
  if (!c) return -1;
  c->launches = c->tu_launches = 0;
  c->tu_flops = 0;
  c->tu_events.clear();
  for (int k = 0; k < 4; ++k) {
    c->kt_events[k].clear();
    c->kt_launches[k] = 0;
  }
  c->ev_next = 0;
  for (double& s : c->stage_ms) s = -1;
  for (auto& pr : c->stage_ev) pr[0] = pr[1] = nullptr;
  return RMAT_OK;
}

}  // extern "C"
