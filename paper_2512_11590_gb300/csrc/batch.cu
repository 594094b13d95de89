// a11: batched driver for many independent coupled-channel systems of uneven size
// (energies and partial waves of a scan, the paper's persistent-buffer energy scan
// of Sec. 3.4 step 1 generalised to a batch).
//
// Execution plan (everything enqueued without host synchronisation, so the whole
// batch is captured into one CUDA graph and replayed):
//   * systems larger than `split_n` run one after another on the caller's stream
//     with the full-device path (cooperative panels across all SMs, tcgen05
//     updates); they are the bulk of the flops;
//   * the other systems are spread over `lanes` concurrent streams (longest job
//     first onto the least-loaded lane), each with cluster panels (one thread
//     block cluster, distributed shared memory), so no kernel of a lane waits for
//     CTAs outside its own cluster and lanes share the GPU with the large systems
//     without any grid-wide co-residency requirement;
//   * refinement runs a fixed step budget with the stopping rule evaluated on the
//     device (converged systems skip their updates);
//   * per-system statuses and refinement counts are read once at the end.
// The split and the lane count come from rmat_batch_tune, which times candidate
// plans on the batch itself and caches the winner in the JSON file named by
// RMAT_TUNE_CACHE.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <new>
#include <sstream>
#include <string>
#include <vector>

#include "cplx.cuh"
#include "rmat_internal.h"

namespace {

struct BatchSys {
  int nch, nlag, N, nopen;
  double a, hm, B, E;
  const double2* V;
  int mesh;
  size_t off_l, off_open;
  int lane;  // -1 small-system kernel, 0 serial phase on the caller's stream, >= 1 lane
  double cost;
};

struct MeshTab {
  int nlag;
  double a, hm, B;
  double* K = nullptr;
  double* r = nullptr;
  double* fa = nullptr;
  double phi_max = 1.0;
};

constexpr int MAX_LANES = 16;

}  // namespace

struct rmat_batch_s {
  rmat_ctx parent = nullptr;
  int precision = RMAT_C64_3XTF32_IR;
  std::vector<BatchSys> sys;
  std::vector<MeshTab> meshes;
  int* l_all = nullptr;
  double* th_all = nullptr;
  double* zz_all = nullptr;
  int* open_all = nullptr;
  IrState* ir = nullptr;
  int* st_dev = nullptr;
  int* st_host = nullptr;
  IrState* ir_host = nullptr;
  rmat_ctx lane_ctx[MAX_LANES + 1] = {};
  cudaStream_t lane_stream[MAX_LANES + 1] = {};
  cudaEvent_t fork = nullptr, join[MAX_LANES + 1] = {};
  int max_refine = 30;
  double tol = 1e-13;
  int lanes = 8;
  int split_n = 8192;
  bool use_graph = true;
  bool planned = false, warm = false;
  cudaGraphExec_t gexec = nullptr;
  std::vector<void*> graph_U;
  int graph_ok = 0;
  // small-system class: one persistent launch (batch_small.cu)
  int small_n = -1;                 // N limit of the class (-1: the largest that fits, 0: off)
  int nb_lane = 0, nb_serial = 0;   // LU block widths (0: the size-class defaults)
  int tc_bn_lane = 256;             // tensor-update tile width of lane systems
  std::vector<int> small_idx;       // systems of the class, largest first
  SmallSys* small_dev = nullptr;    size_t small_dev_cap = 0;
  std::vector<SmallSys> small_host;
  std::vector<void*> small_U;       // U pointers the device descriptors hold
  bool small_dirty = true;          // descriptors changed on the host since the last copy
  int* small_next = nullptr;
  SmallScratch small_scr{};
  size_t small_scr_cap[3] = {0, 0, 0};
  size_t small_smem = 0;
  int small_grid = 0;
};

namespace {

// LU block width of a system: in a lane 32 up to N = 1024 and 64 above (its panel
// runs as one thread block cluster), the single-system default otherwise; the
// autotuner may set either class (RMAT_BATCH_NB_LANE / RMAT_BATCH_NB_SERIAL).
int sys_nb(rmat_batch b, const BatchSys& y) {
  if (y.lane > 0) return b->nb_lane > 0 ? b->nb_lane : (y.N <= 1024 ? 32 : 64);
  const int cap = b->precision == RMAT_C128 ? 64 : 128;
  if (b->nb_serial > 0) return std::min(b->nb_serial, cap);
  if (b->precision == RMAT_C128) return y.N >= 2048 ? 64 : 32;
  return y.N >= 4096 ? 128 : 64;
}

// Whether a system goes to the small-system kernel: its matrix, right-hand sides and
// pivots fit one thread block's shared memory and its N is within the class limit.
bool small_fits(rmat_batch b, const BatchSys& y) {
  if (b->small_n == 0 || y.nch > RMAT_NOALLOC_MAX_NCH) return false;
  if (b->small_n > 0 && y.N > b->small_n) return false;
  return small_smem_bytes(b->precision, y.N, y.nch) + 4096 <= (size_t)b->parent->smem_optin;
}

template <class T>
int enqueue_system(rmat_batch b, int s, void* U) {
  BatchSys& y = b->sys[s];
  const MeshTab& m = b->meshes[y.mesh];
  rmat_ctx c = b->lane_ctx[y.lane];
  c->kind = 1;
  c->precision = b->precision;
  c->nch = y.nch;
  c->nlag = y.nlag;
  c->N = y.N;
  c->nrhs = y.nch;
  c->ld = (int)round_up(y.N, 32);
  c->a = y.a;
  c->hm = y.hm;
  c->bloch_B = y.B;
  c->E = y.E;
  c->nb = sys_nb(b, y);
  c->panel_ctas_param = 0;
  c->Kmat = m.K;
  c->rmesh = m.r;
  c->fa = m.fa;
  c->phi_max = m.phi_max;
  c->l_d = b->l_all + y.off_l;
  c->th_d = b->th_all + y.off_l;
  c->zz_d = b->zz_all + y.off_l;
  c->open_d = b->open_all + y.off_open;
  c->borrowed_tables = true;
  c->woodbury = false;      // batches factor M itself
  c->solve_lookahead = 0;   // lanes are their own concurrency
  c->factor_lookahead = 0;
  c->tc_bn = y.lane > 0 ? b->tc_bn_lane : 256;
  c->equil = c->equil_param == -1 ? b->precision != RMAT_C128 : c->equil_param == 1;
  RMAT_CHECK(perm_reserve(c, c->perm_main, y.N, c->nb));  // lay out, no growth (plan sized it)
  RMAT_CU(cudaMemsetAsync(c->dstat, 0, ST_COUNT * sizeof(int), c->stream));
  RMAT_CHECK(launch_assemble(c, y.V, y.E));
  RMAT_CHECK(launch_point_coupling(c, y.V, y.E));
  RMAT_CHECK(lu_factor_dev<T>(c, c->C, c->N, c->ld, c->ipiv, c->nb,
                              rmat_tensor_prec(b->precision), c->perm_main));
  RMAT_CHECK(enqueue_solve_refine(c, b->max_refine, b->tol, b->ir + s));
  RMAT_CHECK(launch_collision(c, nullptr, reinterpret_cast<double2*>(U), y.nopen));
  RMAT_CU(cudaMemcpyAsync(b->st_dev + (size_t)s * ST_COUNT, c->dstat, ST_COUNT * sizeof(int),
                          cudaMemcpyDeviceToDevice, c->stream));
  return RMAT_OK;
}

int enqueue_all(rmat_batch b, void* const* U) {
  cudaStream_t main = b->lane_stream[0];
  RMAT_CU(cudaEventRecord(b->fork, main));
  for (int l = 1; l <= b->lanes; ++l) RMAT_CU(cudaStreamWaitEvent(b->lane_stream[l], b->fork, 0));
  // the small-system class: one persistent launch, concurrent with the lanes
  RMAT_CHECK(launch_batch_small(main, b->precision, b->small_dev, (int)b->small_idx.size(),
                                b->small_next, b->small_grid, b->small_smem, b->max_refine, b->tol,
                                b->st_dev, b->ir, b->small_scr));
  if (!b->small_idx.empty()) b->lane_ctx[0]->launches++;
  for (size_t s = 0; s < b->sys.size(); ++s) {
    if (b->sys[s].lane < 0) continue;
    if (b->precision == RMAT_C128)
      RMAT_CHECK(enqueue_system<double>(b, (int)s, U[s]));
    else
      RMAT_CHECK(enqueue_system<float>(b, (int)s, U[s]));
  }
  for (int l = 1; l <= b->lanes; ++l) {
    RMAT_CU(cudaEventRecord(b->join[l], b->lane_stream[l]));
    RMAT_CU(cudaStreamWaitEvent(main, b->join[l], 0));
  }
  return RMAT_OK;
}

// A lane takes a system whose panels fit one thread block cluster's shared memory
// (the cluster panel), so no kernel of a lane waits on CTAs it cannot see.
bool lane_fits(rmat_batch b, const BatchSys& y) {
  BatchSys t = y;
  t.lane = 1;
  return panel_cluster_fits(b->parent, b->precision, y.N, sys_nb(b, t)) > 0;
}

// Device descriptors and per-CTA scratch of the small-system class.
int plan_small(rmat_batch b) {
  rmat_ctx c = b->parent;
  const int n = (int)b->small_idx.size();
  b->small_host.assign(n, SmallSys{});
  b->small_U.assign(n, nullptr);
  b->small_dirty = true;
  if (n == 0) return RMAT_OK;
  size_t slot = 0;
  int maxN = 0, maxc = 0;
  for (int k = 0; k < n; ++k) {
    const BatchSys& y = b->sys[b->small_idx[k]];
    const MeshTab& m = b->meshes[y.mesh];
    SmallSys& d = b->small_host[k];
    d.nch = y.nch;
    d.nlag = y.nlag;
    d.N = y.N;
    d.nopen = y.nopen;
    d.sys = b->small_idx[k];
    d.hm = y.hm;
    d.a = y.a;
    d.B = y.B;
    d.E = y.E;
    d.phi_max = m.phi_max;
    d.V = y.V;
    d.K = m.K;
    d.r = m.r;
    d.fa = m.fa;
    d.l = b->l_all + y.off_l;
    d.th = b->th_all + y.off_l;
    d.zz = b->zz_all + y.off_l;
    d.open = b->open_all + y.off_open;
    d.U = nullptr;
    slot = std::max(slot, (size_t)y.N * y.nch);
    maxN = std::max(maxN, y.N);
    maxc = std::max(maxc, y.nch);
  }
  b->small_grid = std::min(n, c->sm_count);
  b->small_smem = 0;
  for (int k = 0; k < n; ++k)
    b->small_smem = std::max(b->small_smem, small_smem_bytes(b->precision, b->small_host[k].N,
                                                             b->small_host[k].nch));
  const size_t xb = (size_t)b->small_grid * slot * sizeof(double2);
  const size_t cb = (size_t)b->small_grid * small_coll_scratch_bytes();
  RMAT_CHECK(rmat_grow(c, (void**)&b->small_scr.X, &b->small_scr_cap[0], xb));
  RMAT_CHECK(rmat_grow(c, (void**)&b->small_scr.R, &b->small_scr_cap[1], xb));
  RMAT_CHECK(rmat_grow(c, &b->small_scr.coll, &b->small_scr_cap[2], cb));
  b->small_scr.slot = slot;
  RMAT_CHECK(rmat_grow(c, (void**)&b->small_dev, &b->small_dev_cap, (size_t)n * sizeof(SmallSys)));
  if (!b->small_next) RMAT_CU(cudaMalloc((void**)&b->small_next, sizeof(int)));
  return RMAT_OK;
}

// The descriptors carry the U pointers of the run: rewritten (outside any capture)
// whenever they change.
int small_prepare(rmat_batch b, void* const* U) {
  const int n = (int)b->small_idx.size();
  if (n == 0) return RMAT_OK;
  bool same = !b->small_dirty;
  for (int k = 0; k < n; ++k)
    if (b->small_U[k] != U[b->small_idx[k]]) same = false;
  if (same) return RMAT_OK;
  for (int k = 0; k < n; ++k) {
    b->small_U[k] = U[b->small_idx[k]];
    b->small_host[k].U = reinterpret_cast<double2*>(b->small_U[k]);
  }
  RMAT_CU(cudaMemcpy(b->small_dev, b->small_host.data(), n * sizeof(SmallSys),
                     cudaMemcpyHostToDevice));
  b->small_dirty = false;
  return RMAT_OK;
}

// Assign systems to the serial phase or to lanes (longest first onto the least
// loaded lane) and size every lane context for its largest system.
int plan(rmat_batch b) {
  if (b->gexec) {
    cudaGraphExecDestroy(b->gexec);
    b->gexec = nullptr;
  }
  std::vector<int> order(b->sys.size());
  for (size_t s = 0; s < order.size(); ++s) order[s] = (int)s;
  std::sort(order.begin(), order.end(),
            [&](int x, int y) { return b->sys[x].cost > b->sys[y].cost; });
  std::vector<double> load(b->lanes + 1, 0.0);
  b->small_idx.clear();
  for (int s : order) {
    BatchSys& y = b->sys[s];
    if (small_fits(b, y)) {  // whole hot path in one CTA's shared memory
      y.lane = -1;
      b->small_idx.push_back(s);
      continue;
    }
    // lanes hold systems whose panels fit one cluster
    if (y.N > b->split_n || b->lanes == 0 || !lane_fits(b, y)) {
      y.lane = 0;
    } else {
      int best = 1;
      for (int l = 2; l <= b->lanes; ++l)
        if (load[l] < load[best]) best = l;
      y.lane = best;
      load[best] += y.cost;
    }
  }
  for (int l = 0; l <= b->lanes; ++l) {
    rmat_ctx c = b->lane_ctx[l];
    int maxN = 0, maxc = 0, maxlag = 0;
    for (const BatchSys& y : b->sys)
      if (y.lane == l) {
        maxN = std::max(maxN, y.N);
        maxc = std::max(maxc, y.nch);
        maxlag = std::max(maxlag, y.nlag);
      }
    if (maxN == 0) continue;
    c->precision = b->precision;
    c->N = maxN;
    c->ld = (int)round_up(maxN, 32);
    c->nrhs = maxc;
    c->kind = 1;
    c->nb = 64;
    RMAT_CHECK(ctx_reserve(c, false));
    for (const BatchSys& y : b->sys)
      if (y.lane == l) RMAT_CHECK(perm_reserve(c, c->perm_main, y.N, sys_nb(b, y)));
    RMAT_CHECK(perm_reserve(c, c->perm_z, maxc, 32));
    RMAT_CHECK(rmat_grow(c, (void**)&c->Wpt, &c->Wpt_cap, (size_t)maxlag * maxc * maxc * 16));
    RMAT_CHECK(rmat_grow(c, (void**)&c->Rint, &c->Rint_cap, (size_t)maxc * maxc * 16));
    RMAT_CHECK(rmat_grow(c, (void**)&c->Zbuf, &c->Zbuf_cap, collision_workspace_bytes(maxc)));
    RMAT_CHECK(rmat_grow(c, (void**)&c->zpiv, &c->zpiv_cap, maxc * sizeof(int)));
    RMAT_CHECK(rmat_grow(c, (void**)&c->Dsc, &c->Dsc_cap, (size_t)maxN * sizeof(double)));
  }
  RMAT_CHECK(plan_small(b));
  b->planned = true;
  b->warm = false;
  b->graph_ok = 0;
  return RMAT_OK;
}

int run_once(rmat_batch b, void* const* U, bool allow_graph) {
  cudaStream_t main = b->lane_stream[0];
  RMAT_CHECK(small_prepare(b, U));
  if (!b->warm) {  // first pass outside capture: grows lazy buffers, sets kernel attributes
    RMAT_CHECK(enqueue_all(b, U));
    RMAT_CU(cudaStreamSynchronize(main));
    b->warm = true;
    return RMAT_OK;
  }
  const bool same_U = b->gexec && b->graph_U.size() == b->sys.size() &&
                      std::equal(b->graph_U.begin(), b->graph_U.end(), U);
  if (allow_graph && b->use_graph && b->graph_ok >= 0 && !same_U) {
    if (b->gexec) {
      cudaGraphExecDestroy(b->gexec);
      b->gexec = nullptr;
    }
    cudaGraph_t g = nullptr;
    // the legacy default stream cannot be captured: run without a graph there
    if (main == nullptr) {
      b->graph_ok = -1;
    } else if (cudaStreamBeginCapture(main, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
      cudaGetLastError();
      b->graph_ok = -1;
    } else {
      const int st = enqueue_all(b, U);
      const cudaError_t e = cudaStreamEndCapture(main, &g);
      if (st == RMAT_OK && e == cudaSuccess && g &&
          cudaGraphInstantiate(&b->gexec, g, 0) == cudaSuccess) {
        b->graph_U.assign(U, U + b->sys.size());
        b->graph_ok = 1;
      } else {
        b->gexec = nullptr;
        b->graph_ok = -1;  // capture unsupported here: fall back to direct launches
      }
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();
    }
  }
  if (allow_graph && b->gexec) {
    RMAT_CU(cudaGraphLaunch(b->gexec, main));
    return RMAT_OK;
  }
  return enqueue_all(b, U);
}

double time_run(rmat_batch b, void* const* U) {
  cudaStream_t main = b->lane_stream[0];
  if (run_once(b, U, false) != RMAT_OK) return INFINITY;  // warm-up
  if (cudaStreamSynchronize(main) != cudaSuccess) return INFINITY;
  const auto t0 = std::chrono::steady_clock::now();
  if (run_once(b, U, false) != RMAT_OK) return INFINITY;
  if (cudaStreamSynchronize(main) != cudaSuccess) return INFINITY;
  return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

std::string tune_key(rmat_batch b) {
  std::ostringstream k;
  long long h = 1469598103934665603LL;
  for (const BatchSys& y : b->sys) h = (h ^ (long long)y.N) * 1099511628211LL;
  k << "v2_prec" << b->precision << "_n" << b->sys.size() << "_h" << (unsigned long long)h;
  return k.str();
}

// The tuned knobs of a batch plan.
struct Knobs {
  int lanes, split, small_n, nb_lane, nb_serial, tc_bn;
};

void apply_knobs(rmat_batch b, const Knobs& k) {
  b->lanes = k.lanes;
  b->split_n = k.split;
  b->small_n = k.small_n;
  b->nb_lane = k.nb_lane;
  b->nb_serial = k.nb_serial;
  b->tc_bn_lane = k.tc_bn;
}

bool cache_lookup(const std::string& key, Knobs* k) {
  const char* path = std::getenv("RMAT_TUNE_CACHE");
  if (!path) return false;
  std::ifstream f(path);
  std::string line;
  while (std::getline(f, line)) {
    const size_t p = line.find("\"" + key + "\"");
    if (p == std::string::npos) continue;
    Knobs t{};
    if (std::sscanf(line.c_str() + line.find(':', p) + 1,
                    " {\"lanes\": %d, \"split_n\": %d, \"small_n\": %d, \"nb_lane\": %d, "
                    "\"nb_serial\": %d, \"tc_bn\": %d",
                    &t.lanes, &t.split, &t.small_n, &t.nb_lane, &t.nb_serial, &t.tc_bn) == 6) {
      *k = t;
      return true;
    }
  }
  return false;
}

void cache_store(const std::string& key, const Knobs& k, double secs) {
  const char* path = std::getenv("RMAT_TUNE_CACHE");
  if (!path) return;
  std::ofstream f(path, std::ios::app);
  f << "{\"" << key << "\": {\"lanes\": " << k.lanes << ", \"split_n\": " << k.split
    << ", \"small_n\": " << k.small_n << ", \"nb_lane\": " << k.nb_lane
    << ", \"nb_serial\": " << k.nb_serial << ", \"tc_bn\": " << k.tc_bn
    << ", \"seconds\": " << secs << "}}\n";
}

}  // namespace

extern "C" {

int rmat_batch_create(rmat_ctx ctx, int nsys, const rmat_problem* probs, const double* E,
                      const void* const* V_dev, int max_refine, double tol, rmat_batch* out) {
  if (!ctx) return -1;
  if (nsys < 1) return -2;
  if (!probs) return -3;
  if (!E) return -4;
  if (!V_dev) return -5;
  if (max_refine < 0) return -6;
  if (!out) return -8;
  *out = nullptr;
  RMAT_CU(cudaSetDevice(ctx->device));
  const int prec = probs[0].precision;
  for (int s = 0; s < nsys; ++s) {
    const rmat_problem& p = probs[s];
    if (p.nch < 1 || p.nlag < 1 || p.nlag > 1024 || !(p.a > 0) || !(p.hm > 0) || !p.l ||
        !p.thresh || p.precision != prec || (long long)p.nch * p.nlag > 200000 ||
        !std::isfinite(E[s]) || !V_dev[s])
      return -3;
    for (int k = 0; k < p.nch; ++k)
      if (p.zz && !(std::isfinite(p.zz[k]) && p.zz[k] >= 0.0)) return -3;
    if (prec != RMAT_C128 && prec != RMAT_C64_3XTF32_IR && prec != RMAT_C64_SIMT_IR &&
        prec != RMAT_C64_3XF16_IR && prec != RMAT_C64_1XF16_IR)
      return -3;
  }
  rmat_batch b = new (std::nothrow) rmat_batch_s();
  if (!b) return RMAT_ENOMEM;
  b->parent = ctx;
  b->precision = prec;
  b->max_refine = max_refine;
  b->tol = tol;
  std::vector<int> l_h, open_h;
  std::vector<double> th_h, zz_h;
  for (int s = 0; s < nsys; ++s) {
    const rmat_problem& p = probs[s];
    BatchSys y{};
    y.nch = p.nch;
    y.nlag = p.nlag;
    y.N = p.nch * p.nlag;
    y.a = p.a;
    y.hm = p.hm;
    y.B = p.bloch_B;
    y.E = E[s];
    y.V = reinterpret_cast<const double2*>(V_dev[s]);
    y.cost = std::pow((double)y.N, 3.0);
    y.off_l = l_h.size();
    y.off_open = open_h.size();
    for (int k = 0; k < p.nch; ++k) {
      l_h.push_back(p.l[k]);
      th_h.push_back(p.thresh[k]);
      zz_h.push_back(p.zz ? p.zz[k] : 0.0);
      if (E[s] - p.thresh[k] > 0) open_h.push_back(k);
    }
    y.nopen = (int)(open_h.size() - y.off_open);
    int m = -1;
    for (size_t q = 0; q < b->meshes.size(); ++q)
      if (b->meshes[q].nlag == p.nlag && b->meshes[q].a == p.a && b->meshes[q].hm == p.hm &&
          b->meshes[q].B == p.bloch_B)
        m = (int)q;
    if (m < 0) {
      MeshTab t;
      t.nlag = p.nlag;
      t.a = p.a;
      t.hm = p.hm;
      t.B = p.bloch_B;
      std::vector<double> r(p.nlag), fa(p.nlag), T0((size_t)p.nlag * p.nlag), K(T0.size());
      rmat_mesh_host(p.nlag, p.a, nullptr, nullptr, nullptr, r.data(), fa.data(), T0.data());
      rmat_kinetic_table(p.nlag, p.hm, p.hm * (p.bloch_B / p.a), T0.data(), fa.data(), K.data());
      double pm = 0;
      for (double v : fa) pm = std::max(pm, std::fabs(v));
      t.phi_max = pm;
      if (cudaMalloc(&t.K, K.size() * 8) != cudaSuccess ||
          cudaMalloc(&t.r, r.size() * 8) != cudaSuccess ||
          cudaMalloc(&t.fa, fa.size() * 8) != cudaSuccess) {
        b->meshes.push_back(t);
        rmat_batch_destroy(b);
        return RMAT_ENOMEM;
      }
      cudaMemcpy(t.K, K.data(), K.size() * 8, cudaMemcpyHostToDevice);
      cudaMemcpy(t.r, r.data(), r.size() * 8, cudaMemcpyHostToDevice);
      cudaMemcpy(t.fa, fa.data(), fa.size() * 8, cudaMemcpyHostToDevice);
      b->meshes.push_back(t);
      m = (int)b->meshes.size() - 1;
    }
    y.mesh = m;
    b->sys.push_back(y);
  }
  const size_t nl = l_h.size(), no = std::max<size_t>(1, open_h.size());
  if (cudaMalloc(&b->l_all, nl * sizeof(int)) != cudaSuccess ||
      cudaMalloc(&b->th_all, nl * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&b->zz_all, nl * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&b->open_all, no * sizeof(int)) != cudaSuccess ||
      cudaMalloc(&b->ir, nsys * sizeof(IrState)) != cudaSuccess ||
      cudaMalloc(&b->st_dev, (size_t)nsys * ST_COUNT * sizeof(int)) != cudaSuccess ||
      cudaMallocHost(&b->st_host, (size_t)nsys * ST_COUNT * sizeof(int)) != cudaSuccess ||
      cudaMallocHost(&b->ir_host, nsys * sizeof(IrState)) != cudaSuccess) {
    cudaGetLastError();
    rmat_batch_destroy(b);
    return RMAT_ENOMEM;
  }
  cudaMemcpy(b->l_all, l_h.data(), nl * sizeof(int), cudaMemcpyHostToDevice);
  cudaMemcpy(b->th_all, th_h.data(), nl * sizeof(double), cudaMemcpyHostToDevice);
  cudaMemcpy(b->zz_all, zz_h.data(), nl * sizeof(double), cudaMemcpyHostToDevice);
  if (!open_h.empty())
    cudaMemcpy(b->open_all, open_h.data(), open_h.size() * sizeof(int), cudaMemcpyHostToDevice);
  b->lane_stream[0] = ctx->stream;
  for (int l = 0; l <= MAX_LANES; ++l) {
    if (l > 0 && cudaStreamCreateWithFlags(&b->lane_stream[l], cudaStreamNonBlocking) != cudaSuccess) {
      rmat_batch_destroy(b);
      return RMAT_ECUDA;
    }
    int st = rmat_create(&b->lane_ctx[l], ctx->device, b->lane_stream[l]);
    if (st != RMAT_OK) {
      rmat_batch_destroy(b);
      return st;
    }
    b->lane_ctx[l]->spin_limit = ctx->spin_limit;
    cudaEventCreateWithFlags(&b->join[l], cudaEventDisableTiming);
  }
  cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
  int st = plan(b);
  if (st != RMAT_OK) {
    rmat_batch_destroy(b);
    return st;
  }
  *out = b;
  return RMAT_OK;
}

int rmat_batch_nopen(rmat_batch b, int* nopen) {
  if (!b) return -1;
  if (!nopen) return -2;
  for (size_t s = 0; s < b->sys.size(); ++s) nopen[s] = b->sys[s].nopen;
  return RMAT_OK;
}

int rmat_batch_set(rmat_batch b, int key, long long v) {
  if (!b) return -1;
  switch (key) {
    case RMAT_BATCH_LANES:
      if (v < 0 || v > MAX_LANES) return -3;
      b->lanes = (int)v;
      break;
    case RMAT_BATCH_SPLIT_N:
      if (v < 0) return -3;
      b->split_n = (int)v;
      break;
    case RMAT_BATCH_GRAPH:
      b->use_graph = v != 0;
      return RMAT_OK;
    case RMAT_BATCH_SMALL_N:
      if (v < -1 || v > 100000) return -3;
      b->small_n = (int)v;
      break;
    case RMAT_BATCH_NB_LANE:
      if (v != 0 && v != 32 && v != 64) return -3;
      b->nb_lane = (int)v;
      break;
    case RMAT_BATCH_NB_SERIAL:
      if (v != 0 && v != 32 && v != 64 && v != 128) return -3;
      b->nb_serial = (int)v;
      break;
    case RMAT_BATCH_TC_BN:
      if (v != 0 && v != 128 && v != 256) return -3;
      b->tc_bn_lane = v == 128 ? 128 : 256;
      break;
    default:
      return -2;
  }
  RMAT_CU(cudaStreamSynchronize(b->lane_stream[0]));
  return plan(b);
}

int rmat_batch_tune(rmat_batch b, void* const* U_dev, int* lanes, int* split_n) {
  if (!b) return -1;
  if (!U_dev) return -2;
  const std::string key = tune_key(b);
  Knobs best{b->lanes, b->split_n, b->small_n, b->nb_lane, b->nb_serial, b->tc_bn_lane};
  if (!cache_lookup(key, &best)) {
    // coordinate descent, each candidate plan timed on the batch itself: first the
    // lane / split plan, then the small-system class, then the LU block widths (the
    // tile shapes of the panels, U12 solves and tensor-core updates) of the lanes and
    // of the serial systems
    double tbest = INFINITY;
    auto trial = [&](const Knobs& k) -> int {
      apply_knobs(b, k);
      RMAT_CHECK(plan(b));
      const double t = time_run(b, U_dev);
      if (t < tbest) {
        tbest = t;
        best = k;
      }
      return RMAT_OK;
    };
    const int cand[][2] = {{0, 0}, {8, 1024}, {8, 8192}, {16, 1024}, {16, 8192}};
    for (const auto& cd : cand) RMAT_CHECK(trial({cd[0], cd[1], -1, 0, 0, 256}));
    {
      Knobs k = best;
      k.small_n = 0;
      RMAT_CHECK(trial(k));
    }
    {
      const Knobs base = best;
      for (int nb : {32, 64}) {
        Knobs k = base;
        k.nb_lane = nb;
        RMAT_CHECK(trial(k));
      }
    }
    if (rmat_tensor_prec(b->precision) && best.lanes > 0) {
      Knobs k = best;
      k.tc_bn = 128;
      RMAT_CHECK(trial(k));
    }
    {
      const Knobs base = best;
      for (int nb : {32, 64, 128})
        if (!(b->precision == RMAT_C128 && nb == 128)) {
          Knobs k = base;
          k.nb_serial = nb;
          RMAT_CHECK(trial(k));
        }
    }
    cache_store(key, best, tbest);
  }
  apply_knobs(b, best);
  RMAT_CHECK(plan(b));
  if (lanes) *lanes = best.lanes;
  if (split_n) *split_n = best.split;
  return RMAT_OK;
}

int rmat_batch_run(rmat_batch b, void* const* U_dev, int* status, int* iters) {
  if (!b) return -1;
  if (!U_dev) return -2;
  for (size_t s = 0; s < b->sys.size(); ++s)
    if (b->sys[s].nopen > 0 && !U_dev[s]) return -2;
  RMAT_CU(cudaSetDevice(b->parent->device));
  if (!b->planned) RMAT_CHECK(plan(b));
  if (!b->warm) RMAT_CHECK(run_once(b, U_dev, true));  // warm-up pass (buffers, attributes)
  RMAT_CHECK(run_once(b, U_dev, true));
  cudaStream_t main = b->lane_stream[0];
  const size_t n = b->sys.size();
  RMAT_CU(cudaMemcpyAsync(b->st_host, b->st_dev, n * ST_COUNT * sizeof(int), cudaMemcpyDeviceToHost,
                          main));
  RMAT_CU(cudaMemcpyAsync(b->ir_host, b->ir, n * sizeof(IrState), cudaMemcpyDeviceToHost, main));
  RMAT_CU(cudaStreamSynchronize(main));
  int worst = RMAT_OK;
  for (size_t s = 0; s < n; ++s) {
    const int* w = b->st_host + s * ST_COUNT;
    int st = b->ir_host[s].status;
    if (w[ST_INFO]) st = RMAT_ESINGULAR;
    if (w[ST_CHANFN]) st = RMAT_ECHANFN;
    if (w[ST_BADARG]) st = RMAT_ESTATE;
    if (w[ST_TIMEOUT]) st = RMAT_ETIMEOUT;
    if (status) status[s] = st;
    if (iters) iters[s] = b->ir_host[s].iters;
    if (st < 0) worst = st;
  }
  return worst;
}

int rmat_batch_info(rmat_batch b, long long* out, int n) {
  if (!b) return -1;
  if (!out || n < 0) return -2;
  long long launches = 0;
  for (int l = 0; l <= MAX_LANES; ++l)
    if (b->lane_ctx[l]) launches += b->lane_ctx[l]->launches;
  const long long v[10] = {(long long)b->sys.size(), b->lanes, b->split_n, b->graph_ok, launches,
                           (long long)b->small_idx.size(), b->small_n, b->nb_lane, b->nb_serial,
                           b->tc_bn_lane};
  const int m = std::min(n, 10);
  for (int k = 0; k < m; ++k) out[k] = v[k];
  return m;
}

int rmat_batch_destroy(rmat_batch b) {
  if (!b) return RMAT_OK;
  if (b->lane_stream[0]) cudaStreamSynchronize(b->lane_stream[0]);
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  for (int l = 0; l <= MAX_LANES; ++l) {
    if (b->lane_ctx[l]) rmat_destroy(b->lane_ctx[l]);
    if (l > 0 && b->lane_stream[l]) cudaStreamDestroy(b->lane_stream[l]);
    if (b->join[l]) cudaEventDestroy(b->join[l]);
  }
  if (b->fork) cudaEventDestroy(b->fork);
  for (MeshTab& t : b->meshes) {
    cudaFree(t.K);
    cudaFree(t.r);
    cudaFree(t.fa);
  }
  cudaFree(b->small_dev);
  cudaFree(b->small_next);
  cudaFree(b->small_scr.X);
  cudaFree(b->small_scr.R);
  cudaFree(b->small_scr.coll);
  cudaFree(b->l_all);
  cudaFree(b->th_all);
  cudaFree(b->zz_all);
  cudaFree(b->open_all);
  cudaFree(b->ir);
  cudaFree(b->st_dev);
  if (b->st_host) cudaFreeHost(b->st_host);
  if (b->ir_host) cudaFreeHost(b->ir_host);
  delete b;
  return RMAT_OK;
}

}  // extern "C"
