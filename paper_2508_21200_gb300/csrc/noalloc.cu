// Observables without any device allocation.
//
// Some callers cannot allocate device memory: hosts that hand all device memory to their own
// allocator (a framework's caching pool, a fixed memory budget), and monitoring loops where an
// allocation's latency or the heap fragmentation it causes is not acceptable.
// lrei_observables_noalloc computes the same observables as lrei_observables, without a
// context, taking every input explicitly.  Its per-CTA partial sums and small results live in
// one file-scope device array (g_noalloc_scratch, about 3.8 MB), which every GPU that loads
// this library's device code holds until the process exits.
#include "lrei.h"
#include "common.cuh"
#include "tsk.cuh"

#include <cmath>
#include <cstring>

namespace lrei {
void launch_obs_final(const double *red, int r, const double *lam, double *out, cudaStream_t st);
int launch_obs_capped(bool fp64, const ModelArgs &M, const void *V, long long N, int r, double *partial,
                      int max_grid, cudaStream_t st);
}  // namespace lrei

using namespace lrei;

namespace {
constexpr int NA_MAX_R = LREI_NOALLOC_MAX_R;
constexpr int NA_PARTS = 152;                               // partial sums (CTAs) at most
constexpr size_t NA_ENT = 6ull * NA_MAX_R * NA_MAX_R * 2;    // doubles per partial (6 r x r Grams)
// partials + 16 reduction slices + reduced Grams + spectrum + outputs
constexpr size_t NA_DOUBLES = (NA_PARTS + 16) * NA_ENT + NA_ENT + 64 + 64;

static __device__ __align__(256) double g_noalloc_scratch[NA_DOUBLES];

// Device address of the scratch array on the current device.  Host code cannot use the symbol
// itself (in host code it names a host-side stand-in, not device memory), so every call looks
// the address up with the device current: the lookup allocates nothing, and a cached address
// could dangle after the caller resets the device or its primary context is recreated.
double *scratch_for_current_device(int *code) {
  void *p = nullptr;
  if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
    *code = LREI_ERR_CUDA;
    return nullptr;
  }
  *code = LREI_OK;
  return reinterpret_cast<double *>(p);
}
}  // namespace

extern "C" int lrei_observables_noalloc(int n, const lrei_bonds *J, const double B[3], const void *V_dev, int r,
                                        int dtype, const double *Lambda_host, void *cuda_stream, lrei_obs *out) {
  if (!V_dev || !Lambda_host || !out) return LREI_ERR_ARG;
  if (n < 1 || n > MAX_SPINS || r < 1 || r > NA_MAX_R || (long long)r > (1LL << n)) return LREI_ERR_ARG;
  if (dtype != LREI_C128 && dtype != LREI_C64) return LREI_ERR_ARG;
  ModelArgs M;
  const int mrc = build_model_args(n, J, B, &M);
  if (mrc != LREI_OK) return mrc;
  int code = LREI_OK;
  double *base = scratch_for_current_device(&code);
  if (!base) return code;
  double *partial = base;
  double *red = base + (NA_PARTS + 16) * NA_ENT;
  double *lam = red + NA_ENT;
  double *res = lam + 64;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);
  const long long N = 1LL << n;
  // Every region read below is first written by this call, so nothing needs clearing.
  if (cudaMemcpyAsync(lam, Lambda_host, r * sizeof(double), cudaMemcpyHostToDevice, st) != cudaSuccess)
    return LREI_ERR_CUDA;
  const int grid = launch_obs_capped(dtype == LREI_C128, M, V_dev, N, r, partial, NA_PARTS, st);
  launch_reduce(partial, grid, 6 * r * r * 2, red, st);
  launch_obs_final(red, r, lam, res, st);
  double h[9];
  if (cudaMemcpyAsync(h, res, 9 * sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess) return LREI_ERR_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return LREI_ERR_CUDA;
  if (cudaGetLastError() != cudaSuccess) return LREI_ERR_CUDA;
  std::memset(out, 0, sizeof(*out));
  out->energy = h[0];
  out->mx = h[1];
  out->my = h[2];
  out->mz = h[3];
  out->purity = h[4];
  out->trace = h[5];
  out->orth_err = h[6];
  out->herm_err = h[7];
  out->comm_norm = h[8];
  out->r = r;
  for (int i = 0; i < r; ++i) out->lambda0[i] = Lambda_host[i];
  return LREI_OK;
}
