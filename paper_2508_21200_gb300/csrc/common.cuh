// Shared device/host definitions of the LREI GB300 library.
//
// Complex numbers are interleaved (re, im) pairs; the storage type T of the
// N-length (bulk) data is double (complex128) or float (complex64).  Small
// r x r / k x k matrices are always complex double, column-major.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>
#include <cstddef>

namespace lrei {

template <typename T>
struct alignas(2 * sizeof(T)) cx {
  T re, im;
};
using zd = cx<double>;

template <typename T> __host__ __device__ __forceinline__ cx<T> mk(T a, T b) { cx<T> z; z.re = a; z.im = b; return z; }
template <typename T> __host__ __device__ __forceinline__ cx<T> operator+(cx<T> a, cx<T> b) { return mk<T>(a.re + b.re, a.im + b.im); }
template <typename T> __host__ __device__ __forceinline__ cx<T> operator-(cx<T> a, cx<T> b) { return mk<T>(a.re - b.re, a.im - b.im); }
template <typename T> __host__ __device__ __forceinline__ cx<T> operator*(cx<T> a, cx<T> b) {
  return mk<T>(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
template <typename T> __host__ __device__ __forceinline__ cx<T> operator*(T s, cx<T> a) { return mk<T>(s * a.re, s * a.im); }
template <typename T> __host__ __device__ __forceinline__ cx<T> conj(cx<T> a) { return mk<T>(a.re, -a.im); }
// conj(a) * b
template <typename T> __host__ __device__ __forceinline__ cx<T> cmulc(cx<T> a, cx<T> b) {
  return mk<T>(a.re * b.re + a.im * b.im, a.re * b.im - a.im * b.re);
}
// acc += a * b
template <typename T> __host__ __device__ __forceinline__ void fma_(cx<T> &acc, cx<T> a, cx<T> b) {
  acc.re = fma(a.re, b.re, fma(-a.im, b.im, acc.re));
  acc.im = fma(a.re, b.im, fma(a.im, b.re, acc.im));
}
// acc += conj(a) * b
template <typename T> __host__ __device__ __forceinline__ void fmac_(cx<T> &acc, cx<T> a, cx<T> b) {
  acc.re = fma(a.re, b.re, fma(a.im, b.im, acc.re));
  acc.im = fma(a.re, b.im, fma(-a.im, b.re, acc.im));
}
template <typename T> __host__ __device__ __forceinline__ T norm2(cx<T> a) { return a.re * a.re + a.im * a.im; }
template <typename T, typename U> __host__ __device__ __forceinline__ cx<T> cvt(cx<U> a) { return mk<T>((T)a.re, (T)a.im); }

constexpr int MAX_BONDS = 64;
constexpr int MAX_SPINS = 26;
constexpr int MAX_R = 32;
constexpr int MAXB = 12;          // most N x r blocks one tall-skinny kernel reads

// The spin Hamiltonian of eq. H1 in the form the kernels use.  Per bond (i, j): the two bit
// positions (bi of site i, bj of site j), the pair-flip amplitude jxy, the S^zS^z coefficient jz
// and the z component dz of the Dzyaloshinskii-Moriya vector: the bond's flip part is
// (jxy + i dz) S^+_i S^-_j + (jxy - i dz) S^-_i S^+_j, so row b of H V takes the partner
// b ^ mask with amplitude jxy + i dz when site i is up in b (bit 0) and jxy - i dz when it is
// down.  diag(b) = c0 - sum_{antiparallel bonds} jz + bz (n/2 - popcount(b)), c0 = sum jz / 2.
// A transverse field (bx, by) flips one spin: row b takes b ^ 2^q with amplitude
// (bx - i by)/2 when bit q of b is 0 and (bx + i by)/2 when it is 1.  cplx != 0 when any dz,
// bx or by is nonzero (complex amplitudes or one-bit partners).
struct ModelArgs {
  int n;
  int nb;
  int cplx;
  double c0;
  double bz;
  double bx, by;
  uint32_t mask[MAX_BONDS];
  uint8_t bi[MAX_BONDS];
  uint8_t bj[MAX_BONDS];
  double jxy[MAX_BONDS];
  double jz[MAX_BONDS];
  double dz[MAX_BONDS];
};

// Device status word bits (written by kernels, read by the host after a step).
enum : int {
  ST_NONFINITE = 1,
  ST_EIG_NOCONV = 2,
  ST_RANK = 4,
  ST_TIMEOUT = 8,
  ST_TRACE = 16,
  ST_EIG_RESID = 32,
};

}  // namespace lrei

#define LREI_CUDA_TRY(expr)                                   \
  do {                                                        \
    cudaError_t _e = (expr);                                  \
    if (_e != cudaSuccess) return ::lrei::cuda_fail(_e, #expr); \
  } while (0)

namespace lrei {
int cuda_fail(cudaError_t e, const char *what);
// Validates n, the bonds (an lrei_bonds, may be NULL) and the field by the argument rules of
// lrei_create and fills M.
// Returns LREI_OK or the lrei_status code.
int build_model_args(int n, const void *bonds, const double B[3], ModelArgs *M);
// Kernels launched (or recorded into a graph) by this library's wrappers in this process.
long long launch_counter();
void count_launch(int n = 1);
}
