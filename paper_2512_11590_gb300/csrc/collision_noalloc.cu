// rmat_collision_noalloc: the R-matrix and collision matrix of a solved system in
// ONE kernel launch that allocates nothing.
//
// Some callers cannot allocate device memory when they need U: code running
// under a memory pool or caching allocator that owns the whole device (so a
// cudaMalloc would fail or fragment it), code that must not synchronise the
// device (cudaMalloc/cudaFree can), and real-time loops with a fixed memory
// budget.  This entry point takes the solution X and the boundary values f_i(a)
// from the caller, writes R and U into caller buffers, and keeps its scratch
// (the nch x nch matching system, channel functions, status word) in the
// file-scope device array below, of fixed size for nch <= RMAT_NOALLOC_MAX_NCH.
//
// It computes the same quantities as rmat_collision (see include/rmat.h):
//   R = (hm/a) Phi^T X;  R~ = a sqrt(k) R sqrt(k);
//   U = (diag O - R~ diag O')^-1 (diag I - R~ diag I'), open x open block,
// but in a single CTA: R contraction, channel functions, the matching system,
// Gaussian elimination with partial pivoting (largest |Re|+|Im|, first row on
// ties) carrying the right-hand sides, and back substitution.
#include <atomic>
#include <cmath>
#include <cstring>

#include "collision_cta.cuh"

namespace {

// Scratch shared by every call on this device (contents persist between calls).
static __device__ __align__(256) unsigned char g_noalloc_scratch[sizeof(NoallocScratch)];

__global__ void __launch_bounds__(NA_THREADS)
collision_noalloc_kernel(const NoallocParams p, const double* __restrict__ fa,
                         const double2* __restrict__ X, double2* __restrict__ Rout,
                         double2* __restrict__ Uout, NoallocScratch* __restrict__ S) {
  matching_cta(p, fa, X, 1, (size_t)p.ldx, Rout, Uout, S);  // X column-major, ld = ldx
}

// Device address of the scratch array, looked up once per device (the first call
// with that device current).  A cudaDeviceReset reloads the module and may move
// the array: the cached address then no longer belongs to it.
std::atomic<void*> g_scratch_ptr[64];

}  // namespace

extern "C" int rmat_collision_noalloc(const rmat_problem* prob, double E, const void* f_a_dev,
                                      const void* X_dev, int ldx, void* R_dev, void* U_dev,
                                      int* nopen, void* stream) {
  if (!prob || prob->nch < 1 || prob->nch > RMAT_NOALLOC_MAX_NCH || prob->nlag < 1 ||
      !(prob->a > 0) || !(prob->hm > 0) || !std::isfinite(prob->a) || !std::isfinite(prob->hm) ||
      !std::isfinite(prob->bloch_B) || !prob->l || !prob->thresh)
    return -1;
  for (int c = 0; c < prob->nch; ++c)
    if (!std::isfinite(prob->thresh[c]) ||
        (prob->zz && !(std::isfinite(prob->zz[c]) && prob->zz[c] >= 0.0)))
      return -1;
  if (!std::isfinite(E)) return -2;
  if (!f_a_dev) return -3;
  if (!X_dev) return -4;
  if (ldx < prob->nch * prob->nlag) return -5;
  NoallocParams p;
  std::memset(&p, 0, sizeof(p));
  p.nch = prob->nch;
  p.nlag = prob->nlag;
  p.ldx = ldx;
  p.a = prob->a;
  p.hm = prob->hm;
  p.B = prob->bloch_B;
  p.E = E;
  int no = 0;
  for (int c = 0; c < prob->nch; ++c) {
    if (prob->l[c] < 0 || prob->l[c] > 64) return -1;
    p.l[c] = prob->l[c];
    p.thresh[c] = prob->thresh[c];
    p.zz[c] = prob->zz ? prob->zz[c] : 0.0;
    if (E - prob->thresh[c] == 0.0) return -2;  // a channel exactly at threshold
    if (E - prob->thresh[c] > 0) p.open[no++] = c;
  }
  p.nopen = no;
  if (nopen) *nopen = no;
  if (no > 0 && !U_dev) return -7;
  int dev = 0;
  RMAT_CU(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return RMAT_ECUDA;
  void* ptr = g_scratch_ptr[dev].load();
  if (!ptr) {
    // first call on this device: resolve the scratch array's device address
    // (the host-side symbol is only a stand-in and must not reach a kernel)
    RMAT_CU(cudaGetSymbolAddress(&ptr, g_noalloc_scratch));
    if (!ptr) return RMAT_ECUDA;
    g_scratch_ptr[dev].store(ptr);
  }
  NoallocScratch* S = reinterpret_cast<NoallocScratch*>(ptr);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  cudaGetLastError();  // an earlier, unrelated launch error must not be reported as ours
  collision_noalloc_kernel<<<1, NA_THREADS, 0, st>>>(
      p, reinterpret_cast<const double*>(f_a_dev), reinterpret_cast<const double2*>(X_dev),
      reinterpret_cast<double2*>(R_dev), reinterpret_cast<double2*>(U_dev), S);
  RMAT_CU(cudaGetLastError());
  int status = 0;
  RMAT_CU(cudaMemcpyAsync(&status, &S->status, sizeof(int), cudaMemcpyDeviceToHost, st));
  RMAT_CU(cudaStreamSynchronize(st));
  if (status < 0) return RMAT_ECHANFN;
  return status ? RMAT_ESINGULAR : RMAT_OK;
}
