// Tall-skinny (N-length) kernels of the LREI hot path.
//
//  * The per-row matrix-free H.V gather (hv_group; paper Sec. 3.3 "sparsity of H",
//    Hamiltonian eq. H1), used inside the fused passes and as the fallback of the
//    full-row H.V kernel of hv.cu for rows that are not a multiple of 16 bytes:
//    a thread owns CPT consecutive columns of one row; partner rows are read
//    through the read-only cache (rows of one N x r block are contiguous).
//  * Fused tile passes (apply / extend / combine, see tsk.cuh) compute the
//    tall-skinny products Q^*S, S^*S, S A + Q C of the block-Krylov partial
//    eigendecomposition (Sec. 3.7, eq. g-func replaced by an exact block
//    Rayleigh-Ritz on the Krylov space of H) with per-CTA partial Grams.
//  * Observable Grams V^*AV for A in {H, (HV)^*(HV), I, M_x, M_y, M_z}
//    (Sec. 3.6 eq. measuerA).
// Gram accumulation: per tile in the storage precision, then into per-CTA
// accumulators that are FP64 (complex128 path) or compensated FP32 pairs
// (complex64 path, TwoSum), written out as FP64 partials.
#include "tsk.cuh"

#include <cstdlib>

namespace lrei {

// ---------------------------------------------------------------- loads
__device__ __forceinline__ cx<float> ldg1(const cx<float> *p) {
  float2 v = __ldg(reinterpret_cast<const float2 *>(p));
  return mk<float>(v.x, v.y);
}
__device__ __forceinline__ cx<double> ldg1(const cx<double> *p) {
  double2 v = __ldg(reinterpret_cast<const double2 *>(p));
  return mk<double>(v.x, v.y);
}

// Load CPT consecutive complex values (p aligned to CPT * sizeof(cx<T>) when CPT > 1).
template <typename T, int CPT> struct Group {
  __device__ __forceinline__ static void load(const cx<T> *p, cx<T> (&v)[CPT]) {
#pragma unroll
    for (int c = 0; c < CPT; ++c) v[c] = ldg1(p + c);
  }
};
template <> struct Group<float, 4> {
  __device__ __forceinline__ static void load(const cx<float> *p, cx<float> (&v)[4]) {
    float4 a = __ldg(reinterpret_cast<const float4 *>(p));
    float4 b = __ldg(reinterpret_cast<const float4 *>(p) + 1);
    v[0] = mk<float>(a.x, a.y); v[1] = mk<float>(a.z, a.w);
    v[2] = mk<float>(b.x, b.y); v[3] = mk<float>(b.z, b.w);
  }
};
template <> struct Group<float, 2> {
  __device__ __forceinline__ static void load(const cx<float> *p, cx<float> (&v)[2]) {
    float4 a = __ldg(reinterpret_cast<const float4 *>(p));
    v[0] = mk<float>(a.x, a.y); v[1] = mk<float>(a.z, a.w);
  }
};

// Row b, columns [c0, c0 + CPT) of H X.
template <typename T, int CPT>
__device__ __forceinline__ void hv_group(const ModelArgs &M, const cx<T> *__restrict__ X, int r, uint32_t b,
                                         int c0, cx<T> (&out)[CPT]) {
  T diag = (T)(M.c0 + M.bz * (0.5 * M.n - (double)__popc(b)));
  cx<T> acc[CPT];
#pragma unroll
  for (int c = 0; c < CPT; ++c) acc[c] = mk<T>(0, 0);
  if (!M.cplx) {
    for (int k = 0; k < M.nb; ++k) {
      if (((b >> M.bi[k]) ^ (b >> M.bj[k])) & 1u) {
        diag -= (T)M.jz[k];
        const T j = (T)M.jxy[k];
        cx<T> v[CPT];
        Group<T, CPT>::load(X + (size_t)(b ^ M.mask[k]) * r + c0, v);
#pragma unroll
        for (int c = 0; c < CPT; ++c) {
          acc[c].re = fma(j, v[c].re, acc[c].re);
          acc[c].im = fma(j, v[c].im, acc[c].im);
        }
      }
    }
  } else {
    // complex amplitudes: jxy + i dz when site i is up in b, jxy - i dz when it is down
    for (int k = 0; k < M.nb; ++k) {
      if (((b >> M.bi[k]) ^ (b >> M.bj[k])) & 1u) {
        diag -= (T)M.jz[k];
        const cx<T> a = mk<T>((T)M.jxy[k], (T)(((b >> M.bi[k]) & 1u) ? -M.dz[k] : M.dz[k]));
        cx<T> v[CPT];
        Group<T, CPT>::load(X + (size_t)(b ^ M.mask[k]) * r + c0, v);
#pragma unroll
        for (int c = 0; c < CPT; ++c) fma_(acc[c], a, v[c]);
      }
    }
    // one-bit flips of the transverse field: (bx -+ i by)/2 for bit q of b equal to 0 / 1
    if (M.bx != 0.0 || M.by != 0.0)
      for (int q = 0; q < M.n; ++q) {
        const cx<T> a = mk<T>((T)(0.5 * M.bx), (T)(((b >> q) & 1u) ? 0.5 * M.by : -0.5 * M.by));
        cx<T> v[CPT];
        Group<T, CPT>::load(X + (size_t)(b ^ (1u << q)) * r + c0, v);
#pragma unroll
        for (int c = 0; c < CPT; ++c) fma_(acc[c], a, v[c]);
      }
  }
  cx<T> v[CPT];
  Group<T, CPT>::load(X + (size_t)b * r + c0, v);
#pragma unroll
  for (int c = 0; c < CPT; ++c) {
    out[c].re = fma(diag, v[c].re, acc[c].re);
    out[c].im = fma(diag, v[c].im, acc[c].im);
  }
}

template <typename T, int CPT>
__global__ void __launch_bounds__(256) hv_kernel(const __grid_constant__ ModelArgs M, const cx<T> *__restrict__ X,
                                                 cx<T> *__restrict__ Y, long long N, int r) {
  const int gpr = r / CPT;
  const long long total = N * gpr;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const uint32_t b = (uint32_t)(e / gpr);
    const int c0 = (int)(e % gpr) * CPT;
    cx<T> o[CPT];
    hv_group<T, CPT>(M, X, r, b, c0, o);
    cx<T> *y = Y + (size_t)b * r + c0;
#pragma unroll
    for (int c = 0; c < CPT; ++c) y[c] = o[c];
  }
}

// ------------------------------------------------------ accumulation
// Error-free sum: s + e == a + b exactly (Knuth TwoSum).
__device__ __forceinline__ void two_sum_acc(float &hi, float &lo, float b) {
  float s = hi + b;
  float bp = s - hi;
  float err = (hi - (s - bp)) + (b - bp);
  hi = s;
  lo += err;
}

template <typename T> struct Acc;
template <> struct Acc<double> {
  __device__ __forceinline__ static void add(double *acc, int e, cx<double> s) {
    acc[2 * e] += s.re;
    acc[2 * e + 1] += s.im;
  }
  __device__ __forceinline__ static cx<double> get(const double *acc, int e) { return mk<double>(acc[2 * e], acc[2 * e + 1]); }
};
template <> struct Acc<float> {
  __device__ __forceinline__ static void add(double *accd, int e, cx<float> s) {
    float *acc = reinterpret_cast<float *>(accd);
    two_sum_acc(acc[4 * e], acc[4 * e + 1], s.re);
    two_sum_acc(acc[4 * e + 2], acc[4 * e + 3], s.im);
  }
  __device__ __forceinline__ static cx<double> get(const double *accd, int e) {
    const float *acc = reinterpret_cast<const float *>(accd);
    return mk<double>((double)acc[4 * e] + (double)acc[4 * e + 1], (double)acc[4 * e + 2] + (double)acc[4 * e + 3]);
  }
};

// ------------------------------------------------------ fused tile pass
constexpr int TS_THREADS = 256;


template <typename T>
struct TSLayout {
  int tr;          // tile rows
  size_t bytes;    // dynamic shared memory
  bool coef_smem;  // coefficients staged in shared memory
};

template <typename T>
__host__ __device__ inline size_t ts_bytes(int nq, int gram_left, int r, int tr, bool coef_smem, int mode) {
  size_t cxs = sizeof(cx<T>);
  size_t tiles = ((size_t)nq * tr * r + 2 * (size_t)tr * r) * cxs;
  size_t coef = (coef_smem && mode != 0) ? (size_t)(nq + 1) * r * r * cxs : 0;
  size_t acc = (size_t)(gram_left + 1) * r * r * 16;
  return tiles + coef + acc;
}

template <typename T, int CPT>
__global__ void __launch_bounds__(TS_THREADS) ts_kernel(const __grid_constant__ ModelArgs M,
                                                       const __grid_constant__ TSArgs a, int tr, int coef_smem,
                                                       const cx<T> *__restrict__ coefg) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int r = a.r, nq = a.nq, gl = a.gram_left;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int ldc = (nq + 1) * r;          // coefficient rows: [coefQ (nq*r); coefS (r)]
  const int ldg_ = (gl + 1) * r;         // Gram rows
  const int nent = ldg_ * r;
  cx<T> *qs = reinterpret_cast<cx<T> *>(smem);
  cx<T> *gs = qs + (size_t)nq * tr * r;
  cx<T> *ns = gs + (size_t)tr * r;
  cx<T> *csm = ns + (size_t)tr * r;
  const bool use_coef = a.mode != 0;
  double *acc = reinterpret_cast<double *>(csm + ((coef_smem && use_coef) ? (size_t)ldc * r : 0));
  const cx<T> *cs = (coef_smem && use_coef) ? csm : coefg;

  if (coef_smem && use_coef) {
    for (int e = tid; e < ldc * r; e += nt) csm[e] = coefg[e];
  }
  for (int e = tid; e < nent * 2; e += nt) acc[e] = 0.0;
  __syncthreads();

  const long long ntiles = (a.N + tr - 1) / tr;
  const int gpr = r / CPT;
  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const long long row0 = tile * tr;
    const int rows = (int)((a.N - row0) < tr ? (a.N - row0) : tr);
    // S tile
    if (a.mode != 2) {
      const cx<T> *src = reinterpret_cast<const cx<T> *>(a.src);
      for (int e = tid; e < tr * gpr; e += nt) {
        const int lr = e / gpr, c0 = (e % gpr) * CPT;
        cx<T> v[CPT];
        if (lr < rows) {
          if (a.apply_h) {
            hv_group<T, CPT>(M, src, r, (uint32_t)(row0 + lr), c0, v);
          } else {
            Group<T, CPT>::load(src + (size_t)(row0 + lr) * r + c0, v);
          }
        } else {
#pragma unroll
          for (int c = 0; c < CPT; ++c) v[c] = mk<T>(0, 0);
        }
#pragma unroll
        for (int c = 0; c < CPT; ++c) gs[lr * r + c0 + c] = v[c];
      }
    }
    // Q tiles: the tile of block m is a contiguous run of rows*r complex values
    for (int m = 0; m < nq; ++m) {
      const cx<T> *qm = reinterpret_cast<const cx<T> *>(a.q[m]) + (size_t)row0 * r;
      cx<T> *dst = qs + (size_t)m * tr * r;
      for (int e = tid; e < tr * r; e += nt) dst[e] = (e < rows * r) ? ldg1(qm + e) : mk<T>(0, 0);
    }
    __syncthreads();
    const cx<T> *G = gs;
    if (a.mode != 0) {
      cx<T> *out = reinterpret_cast<cx<T> *>(a.out);
      for (int e = tid; e < tr * r; e += nt) {
        const int lr = e / r, j = e % r;
        cx<T> s = mk<T>(0, 0);
        const cx<T> *cj = cs + (size_t)j * ldc;
        if (a.mode == 1) {
          for (int i = 0; i < r; ++i) fma_(s, gs[lr * r + i], cj[nq * r + i]);
        }
        for (int m = 0; m < nq; ++m) {
          const cx<T> *qrow = qs + (size_t)m * tr * r + lr * r;
          const cx<T> *cm = cj + m * r;
          for (int i = 0; i < r; ++i) fma_(s, qrow[i], cm[i]);
        }
        if (lr >= rows || row0 + lr < a.zero_rows) s = mk<T>(0, 0);
        ns[e] = s;
        if (lr < rows && out) out[(size_t)(row0 + lr) * r + j] = s;
      }
      __syncthreads();
      G = ns;
    } else if (a.out) {
      cx<T> *out = reinterpret_cast<cx<T> *>(a.out);
      for (int e = tid; e < rows * r; e += nt) out[(size_t)row0 * r + e] = gs[e];
    }
    // Gram partial of this tile
    for (int e = tid; e < nent; e += nt) {
      const int j = e / ldg_, row = e % ldg_, m = row / r, i = row % r;
      const cx<T> *L = (m < gl) ? qs + (size_t)m * tr * r : G;
      cx<T> s = mk<T>(0, 0);
      for (int lr = 0; lr < tr; ++lr) fmac_(s, L[lr * r + i], G[lr * r + j]);
      Acc<T>::add(acc, e, s);
    }
    __syncthreads();
  }
  double *outp = a.partial + (size_t)blockIdx.x * nent * 2;
  for (int e = tid; e < nent; e += nt) {
    cx<double> v = Acc<T>::get(acc, e);
    outp[2 * e] = v.re;
    outp[2 * e + 1] = v.im;
  }
}

// ------------------------------------------------ fused tile pass, register-blocked
// Same contract as ts_kernel.  Shared tiles use a padded row stride RS (complex elements) so
// that rows of a tile fall in different banks.  The Gram is computed by MI x MJ register
// micro-tiles (rows (m, i) of [q_0..q_{gl-1}, G], columns j), split over `nph` phases of the
// tile rows; per-thread partials are flushed every FLUSH tiles into per-thread accumulators
// in shared memory (compensated FP32 pairs or FP64), then reduced over phases at the end.
// The new tile is a small GEMM [q_0..q_{nq-1}, S] (tr x (nq+1) rp) x coef ((nq+1) rp x rp),
// one row x 4 columns per thread.
template <typename T> struct TS2 {
  static constexpr int MI = sizeof(T) == 4 ? 4 : 2;
  static constexpr int MJ = 4;
  static constexpr int PAD = sizeof(T) == 4 ? 2 : 1;     // row padding (complex elements)
  static constexpr int STAG = sizeof(T) == 4 ? 8 : 4;    // block base stagger (64 bytes)
  static constexpr int FLUSH = sizeof(T) == 4 ? 2 : 1 << 30;
};

__host__ __device__ inline int ts2_rp(int r) { return (r + 3) & ~3; }

// Gram work split: NMT micro-tiles, nph (power of two) phases per micro-tile; the phases of one
// micro-tile are consecutive lanes of one warp, so their partials are combined by shuffles.
__host__ __device__ inline int ts2_nph(int nmt) {
  int p = 1;
  while (p < 16 && nmt * p * 2 <= TS_THREADS) p *= 2;
  return p;
}

template <typename T>
__host__ __device__ inline size_t ts2_bytes(int nq, int gl, int r, int tr, int mode, int mt) {
  const int rp = ts2_rp(r), RS = rp + TS2<T>::PAD;
  const size_t bstride = (size_t)tr * RS + TS2<T>::STAG;
  size_t b = ((size_t)(nq + 2) * bstride) * sizeof(cx<T>);
  if (mode != 0) b += (size_t)(nq + 1) * rp * rp * sizeof(cx<T>);
  const int nmt = (gl + 1) * rp / TS2<T>::MI * (rp / TS2<T>::MJ);
  b += (size_t)nmt * TS2<T>::MI * TS2<T>::MJ * 16;   // one accumulator set per micro-tile
  (void)mt;
  return b;
}

template <typename T, int CPT, int MT>
__global__ void __launch_bounds__(TS_THREADS) ts2_kernel(const __grid_constant__ ModelArgs M,
                                                        const __grid_constant__ TSArgs a, int tr,
                                                        const cx<T> *__restrict__ coefg) {
  constexpr int MI = TS2<T>::MI, MJ = TS2<T>::MJ;
  extern __shared__ __align__(16) unsigned char smem[];
  const int r = a.r, nq = a.nq, gl = a.gram_left;
  const int rp = ts2_rp(r), RS = rp + TS2<T>::PAD;
  const size_t BS = (size_t)tr * RS + TS2<T>::STAG;     // staggered block stride
  const int tid = threadIdx.x, lane = tid & 31;
  cx<T> *qs = reinterpret_cast<cx<T> *>(smem);
  cx<T> *gs = qs + (size_t)nq * BS;
  cx<T> *ns = gs + BS;
  cx<T> *cs = ns + BS;
  const int ncoef = (a.mode != 0) ? (nq + 1) * rp * rp : 0;
  double *slots = reinterpret_cast<double *>(cs + ncoef);   // [NMT][MI*MJ] x 16 bytes

  const int nI = (gl + 1) * rp / MI, nJ = rp / MJ, NMT = nI * nJ;
  for (int e = tid; e < ncoef; e += TS_THREADS) cs[e] = coefg[e];
  for (int e = tid; e < NMT * MI * MJ * 2; e += TS_THREADS) slots[e] = 0.0;

  // Gram micro-tile assignment: MT == 1 -> micro-tile tid / nph, phase tid % nph (lanes);
  // MT == 2 -> micro-tiles tid and tid + 256, one phase.
  const int nph = (MT == 1) ? ts2_nph(NMT) : 1;
  const int ph = (MT == 1) ? (tid % nph) : 0;
  int mts[MT];
  bool mval[MT];
#pragma unroll
  for (int u = 0; u < MT; ++u) {
    mts[u] = (MT == 1) ? tid / nph : tid + u * TS_THREADS;
    mval[u] = mts[u] < NMT;
  }
  cx<T> acc[MT][MI][MJ];
#pragma unroll
  for (int u = 0; u < MT; ++u)
#pragma unroll
    for (int x = 0; x < MI; ++x)
#pragma unroll
      for (int y = 0; y < MJ; ++y) acc[u][x][y] = mk<T>(0, 0);
  __syncthreads();

  auto flush = [&]() {
#pragma unroll
    for (int u = 0; u < MT; ++u)
#pragma unroll
      for (int x = 0; x < MI; ++x)
#pragma unroll
        for (int y = 0; y < MJ; ++y) {
          cx<T> v = acc[u][x][y];
          for (int o = nph >> 1; o > 0; o >>= 1) {   // combine the phases of this micro-tile
            v.re += __shfl_down_sync(0xffffffffu, v.re, o, nph);
            v.im += __shfl_down_sync(0xffffffffu, v.im, o, nph);
          }
          if (ph == 0 && mval[u]) Acc<T>::add(slots, mts[u] * MI * MJ + x * MJ + y, v);
          acc[u][x][y] = mk<T>(0, 0);
        }
  };

  const long long ntiles = (a.N + tr - 1) / tr;
  const int gpr = r / CPT;
  int since_flush = 0;
  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const long long row0 = tile * tr;
    const int rows = (int)((a.N - row0) < tr ? (a.N - row0) : tr);
    // S tile
    if (a.mode != 2) {
      const cx<T> *src = reinterpret_cast<const cx<T> *>(a.src);
      for (int e = tid; e < tr * gpr; e += TS_THREADS) {
        const int lr = e / gpr, c0 = (e % gpr) * CPT;
        cx<T> v[CPT];
        if (lr < rows) {
          if (a.apply_h) hv_group<T, CPT>(M, src, r, (uint32_t)(row0 + lr), c0, v);
          else Group<T, CPT>::load(src + (size_t)(row0 + lr) * r + c0, v);
        } else {
#pragma unroll
          for (int c = 0; c < CPT; ++c) v[c] = mk<T>(0, 0);
        }
#pragma unroll
        for (int c = 0; c < CPT; ++c) gs[lr * RS + c0 + c] = v[c];
      }
      if (rp > r)
        for (int e = tid; e < tr * (rp - r); e += TS_THREADS) gs[(e / (rp - r)) * RS + r + e % (rp - r)] = mk<T>(0, 0);
    }
    // Q tiles (rows of one block are contiguous in global memory)
    for (int m = 0; m < nq; ++m) {
      const cx<T> *qm = reinterpret_cast<const cx<T> *>(a.q[m]) + (size_t)row0 * r;
      cx<T> *dst = qs + (size_t)m * BS;
      if (rp == r && (r % 2 == 0) && sizeof(T) == 4) {
        // 16-byte vectors: two complex64 per load
        const int hr = r / 2;
        for (int e = tid; e < tr * hr; e += TS_THREADS) {
          const int lr = e / hr, c = (e % hr) * 2;
          float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
          if (lr < rows) v = __ldg(reinterpret_cast<const float4 *>(qm + (size_t)lr * r + c));
          cx<T> *d = dst + lr * RS + c;
          d[0] = mk<T>((T)v.x, (T)v.y);
          d[1] = mk<T>((T)v.z, (T)v.w);
        }
      } else {
        for (int e = tid; e < tr * rp; e += TS_THREADS) {
          const int lr = e / rp, c = e % rp;
          dst[lr * RS + c] = (lr < rows && c < r) ? ldg1(qm + (size_t)lr * r + c) : mk<T>(0, 0);
        }
      }
    }
    __syncthreads();
    const cx<T> *G = gs;
    if (a.mode != 0) {
      cx<T> *out = reinterpret_cast<cx<T> *>(a.out);
      const int ngrp = rp / 4;
      for (int e = tid; e < tr * ngrp; e += TS_THREADS) {
        const int lr = e / ngrp, j0 = (e % ngrp) * 4;
        cx<T> o[4];
#pragma unroll
        for (int y = 0; y < 4; ++y) o[y] = mk<T>(0, 0);
        const int mlast = (a.mode == 1) ? nq : nq - 1;
        for (int m = 0; m <= mlast; ++m) {
          const cx<T> *X = (m < nq) ? qs + (size_t)m * BS + lr * RS : gs + lr * RS;
          const cx<T> *C = cs + (size_t)m * rp * rp + j0;
          for (int i = 0; i < r; ++i) {
            const cx<T> x = X[i];
            const cx<T> *ci = C + i * rp;
#pragma unroll
            for (int y = 0; y < 4; ++y) fma_(o[y], x, ci[y]);
          }
        }
#pragma unroll
        for (int y = 0; y < 4; ++y) {
          const int j = j0 + y;
          const cx<T> v = (lr < rows && j < r && row0 + lr >= a.zero_rows) ? o[y] : mk<T>(0, 0);
          ns[lr * RS + j] = v;
          if (lr < rows && j < r && out) out[(size_t)(row0 + lr) * r + j] = v;
        }
      }
      __syncthreads();
      G = ns;
    } else if (a.out) {
      cx<T> *out = reinterpret_cast<cx<T> *>(a.out);
      for (int e = tid; e < rows * r; e += TS_THREADS) out[(size_t)row0 * r + e] = gs[(e / r) * RS + e % r];
    }
    // Gram micro-tiles
#pragma unroll
    for (int u = 0; u < MT; ++u) {
      if (!mval[u]) continue;
      const int I = mts[u] / nJ, J = mts[u] % nJ;
      const int i0 = I * MI, m = i0 / rp, ii0 = i0 % rp, j0 = J * MJ;
      const cx<T> *L = (m < gl) ? qs + (size_t)m * BS : G;
      for (int lr = ph; lr < tr; lr += nph) {
        cx<T> lv[MI], gv[MJ];
#pragma unroll
        for (int x = 0; x < MI; ++x) lv[x] = L[lr * RS + ii0 + x];
#pragma unroll
        for (int y = 0; y < MJ; ++y) gv[y] = G[lr * RS + j0 + y];
#pragma unroll
        for (int x = 0; x < MI; ++x)
#pragma unroll
          for (int y = 0; y < MJ; ++y) fmac_(acc[u][x][y], lv[x], gv[y]);
      }
    }
    if (++since_flush >= TS2<T>::FLUSH) {
      since_flush = 0;
      flush();
    }
    __syncthreads();
  }
  flush();
  __syncthreads();
  // write the CTA partial in the column-major ((gl+1) r) x r layout
  const int ldg_ = (gl + 1) * r, nent = ldg_ * r;
  double *outp = a.partial + (size_t)blockIdx.x * nent * 2;
  for (int e = tid; e < nent; e += TS_THREADS) {
    const int j = e / ldg_, row = e % ldg_, m = row / r, i = row % r;
    const int ic = m * rp + i;
    const int I = ic / MI, x = ic % MI, J = j / MJ, y = j % MJ;
    const cx<double> sum = Acc<T>::get(slots, (I * nJ + J) * MI * MJ + x * MJ + y);
    outp[2 * e] = sum.re;
    outp[2 * e + 1] = sum.im;
  }
  (void)lane;
}

// ------------------------------------------- fused tile pass, pipelined (complex64 bulk)
// Same contract as ts_kernel for T = float, split H.V (apply_h == 0) and r in {8, 16, 32}.
// Each CTA walks its tiles of TR rows with the next tile's blocks already in flight: cp.async
// copies the rows of every input block into the other half of a double buffer (padded rows,
// RS = r + 2 complex, so that rows of one column fall in different banks) while the current
// tile is computed.  Gram work split: a micro-tile is column c of every Gram block against 4
// consecutive G columns (g x 4 complex accumulators); NPH lanes of one warp take interleaved
// rows of the same micro-tile and are combined by shuffles at each flush, every FLUSHT tiles
// (at r = 16: 16 tiles, 128 rows per lane in plain FP32), into compensated FP32 pairs (TwoSum)
// in shared memory.  Lane = phase * TPW + micro-tile, so
// the G loads of a quarter-warp are one row (distinct 16-byte columns) and the block loads of
// a half-warp are two rows of two columns: no bank conflicts at r = 16.
template <int R, int TR, int GMAX, int MINB = (TR <= 32 ? 2 : 1)>
__global__ void __launch_bounds__(256, MINB) ts3_kernel(const __grid_constant__ TSArgs a,
                                                       const cx<float> *__restrict__ coefg) {
  constexpr int RS = R + 2;
  constexpr int MTS = R * R / 4;
  constexpr int NPH = 256 / MTS;
  constexpr int TPW = 32 / NPH;
  constexpr int CH = R / 2;                 // 16-byte chunks per row
  // GMAX: Gram blocks this instance handles (gl + 1 <= GMAX).  Flush period and row-loop unroll
  // measured at n = 20, r = 16 (16 tiles and 8 / 4 for g = 2 / 5: 7-9% faster than 8 tiles and
  // 2); the other widths keep the previous 8 and 2
  constexpr int FLUSHT = R == 16 ? 16 : 8;
  constexpr int UNR = R == 16 ? (GMAX <= 2 ? 8 : 4) : 2;
  constexpr int PU = R == 16 ? 16 : 4;      // projection: inputs per block unrolled (measured, r = 16)
  static_assert(NPH >= 1 && NPH <= 32 && (32 % NPH) == 0 && (RS * 8) % 16 == 0, "r in {8, 16, 32}");
  extern __shared__ __align__(16) unsigned char smem3[];
  const int nq = a.nq, gl = a.gram_left, mode = a.mode;
  const int nb = nq + (mode != 2 ? 1 : 0);
  const int g = gl + 1;
  const int bstride = TR * RS;
  cx<float> *buf = reinterpret_cast<cx<float> *>(smem3);       // [2][nb][TR][RS]
  cx<float> *ns = buf + 2 * nb * bstride;                       // [TR][RS] new tile
  cx<float> *cs = ns + bstride;                                 // [(nq+1) R][R] coefficients
  float *slots = reinterpret_cast<float *>(cs + (mode != 0 ? (nq + 1) * R * R : 0));   // [g R][R][4]
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int ph = lane / TPW;
  const int mt = warp * TPW + lane % TPW;
  const int c = mt / (R / 4), j0 = (mt % (R / 4)) * 4;
  const long long N = a.N;
  const long long ntiles = (N + TR - 1) / TR;

  if (mode != 0)
    for (int e = tid; e < (nq + 1) * R * R; e += 256) cs[e] = coefg[e];
  for (int e = tid; e < g * R * R * 4; e += 256) slots[e] = 0.f;

  auto prefetch = [&](long long tile, int sb) {
    const long long row0 = tile * TR;
    for (int m = 0; m < nb; ++m) {
      const cx<float> *base = reinterpret_cast<const cx<float> *>(m < nq ? a.q[m] : a.src);
      cx<float> *dst = buf + (size_t)(sb * nb + m) * bstride;
      for (int e = tid; e < TR * CH; e += 256) {
        const int lr = e / CH, ch = e % CH;
        const bool ok = row0 + lr < N;
        const cx<float> *gp = ok ? base + (size_t)(row0 + lr) * R + ch * 2 : base;
        const uint32_t sa = (uint32_t)__cvta_generic_to_shared(dst + lr * RS + ch * 2);
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(sa), "l"(gp), "r"(ok ? 16 : 0));
      }
    }
  };

  cx<float> acc[GMAX][4];
#pragma unroll
  for (int m = 0; m < GMAX; ++m)
#pragma unroll
    for (int y = 0; y < 4; ++y) acc[m][y] = mk<float>(0.f, 0.f);

  auto flush = [&]() {
#pragma unroll
    for (int m = 0; m < GMAX; ++m) {
      if (m < g) {
#pragma unroll
        for (int y = 0; y < 4; ++y) {
          float re = acc[m][y].re, im = acc[m][y].im;
#pragma unroll
          for (int o = TPW; o < 32; o <<= 1) {
            re += __shfl_xor_sync(0xffffffffu, re, o);
            im += __shfl_xor_sync(0xffffffffu, im, o);
          }
          if (ph == 0) {
            float *s = slots + ((size_t)(m * R + c) * R + j0 + y) * 4;
            two_sum_acc(s[0], s[1], re);
            two_sum_acc(s[2], s[3], im);
          }
          acc[m][y] = mk<float>(0.f, 0.f);
        }
      }
    }
  };

  long long tile = blockIdx.x;
  int sb = 0;
  if (tile < ntiles) prefetch(tile, 0);
  asm volatile("cp.async.commit_group;\n" ::);
  int since = 0;
  for (; tile < ntiles; tile += gridDim.x) {
    const long long nxt = tile + gridDim.x;
    if (nxt < ntiles) prefetch(nxt, sb ^ 1);
    asm volatile("cp.async.commit_group;\n" ::);
    asm volatile("cp.async.wait_group 1;\n" ::);
    __syncthreads();
    const cx<float> *B0 = buf + (size_t)sb * nb * bstride;
    const long long row0 = tile * TR;
    const int rows = (int)((N - row0) < TR ? (N - row0) : TR);
    const cx<float> *G;
    if (mode != 0) {
      const int mlast = (mode == 1) ? nq : nq - 1;
      cx<float> *out = reinterpret_cast<cx<float> *>(a.out);
      for (int e = tid; e < TR * (R / 4); e += 256) {
        const int lr = e / (R / 4), q0 = (e % (R / 4)) * 4;
        cx<float> o[4];
#pragma unroll
        for (int y = 0; y < 4; ++y) o[y] = mk<float>(0.f, 0.f);
        for (int m = 0; m <= mlast; ++m) {
          const cx<float> *X = B0 + (size_t)m * bstride + lr * RS;
          const cx<float> *C = cs + (size_t)m * R * R + q0;
#pragma unroll PU
          for (int i = 0; i < R; ++i) {
            const cx<float> x = X[i];
            const float4 c01 = *reinterpret_cast<const float4 *>(C + i * R);
            const float4 c23 = *reinterpret_cast<const float4 *>(C + i * R + 2);
            fma_(o[0], x, mk<float>(c01.x, c01.y));
            fma_(o[1], x, mk<float>(c01.z, c01.w));
            fma_(o[2], x, mk<float>(c23.x, c23.y));
            fma_(o[3], x, mk<float>(c23.z, c23.w));
          }
        }
        const bool valid = lr < rows && row0 + lr >= a.zero_rows;
#pragma unroll
        for (int y = 0; y < 4; ++y)
          if (!valid) o[y] = mk<float>(0.f, 0.f);
        float4 *nd = reinterpret_cast<float4 *>(ns + lr * RS + q0);
        nd[0] = make_float4(o[0].re, o[0].im, o[1].re, o[1].im);
        nd[1] = make_float4(o[2].re, o[2].im, o[3].re, o[3].im);
        if (out && lr < rows) {
          float4 *od = reinterpret_cast<float4 *>(out + (size_t)(row0 + lr) * R + q0);
          od[0] = nd[0];
          od[1] = nd[1];
        }
      }
      __syncthreads();
      G = ns;
    } else {
      G = B0 + (size_t)nq * bstride;
    }
#pragma unroll UNR
    for (int lr = ph; lr < TR; lr += NPH) {
      const float4 ga = *reinterpret_cast<const float4 *>(G + lr * RS + j0);
      const float4 gb = *reinterpret_cast<const float4 *>(G + lr * RS + j0 + 2);
      const cx<float> gv0 = mk<float>(ga.x, ga.y), gv1 = mk<float>(ga.z, ga.w);
      const cx<float> gv2 = mk<float>(gb.x, gb.y), gv3 = mk<float>(gb.z, gb.w);
#pragma unroll
      for (int m = 0; m < GMAX; ++m) {
        if (m < g) {
          const cx<float> *L = (m < gl) ? B0 + (size_t)m * bstride : G;
          const cx<float> lv = L[lr * RS + c];
          fmac_(acc[m][0], lv, gv0);
          fmac_(acc[m][1], lv, gv1);
          fmac_(acc[m][2], lv, gv2);
          fmac_(acc[m][3], lv, gv3);
        }
      }
    }
    if (++since >= FLUSHT) {
      since = 0;
      flush();
    }
    __syncthreads();
    sb ^= 1;
  }
  asm volatile("cp.async.wait_group 0;\n" ::);
  flush();
  __syncthreads();
  const int ldg_ = g * R, nent = ldg_ * R;
  double *outp = a.partial + (size_t)blockIdx.x * nent * 2;
  for (int e = tid; e < nent; e += 256) {
    const int j = e / ldg_, row = e % ldg_;
    const float *s = slots + ((size_t)row * R + j) * 4;
    outp[2 * e] = (double)s[0] + (double)s[1];
    outp[2 * e + 1] = (double)s[2] + (double)s[3];
  }
}

template <int R, int TR>
__host__ inline size_t ts3_bytes(int nq, int gl, int mode) {
  const int nb = nq + (mode != 2 ? 1 : 0);
  const size_t bstride = (size_t)TR * (R + 2) * sizeof(cx<float>);
  size_t b = (2 * (size_t)nb + 1) * bstride;
  if (mode != 0) b += (size_t)(nq + 1) * R * R * sizeof(cx<float>);
  b += (size_t)(gl + 1) * R * R * 16;
  return b;
}

// Coefficients in the padded row-major layout of ts2_kernel: row m*rp + i, column j.
template <typename T>
__global__ void coef_convert2_kernel(const zd *coefQ, const zd *coefS, int nq, int r, int mode, cx<T> *out) {
  const int rp = ts2_rp(r);
  const int rows = (nq + 1) * rp;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < rows * rp; e += gridDim.x * blockDim.x) {
    const int row = e / rp, j = e % rp, m = row / rp, i = row % rp;
    zd v = mk<double>(0, 0);
    if (i < r && j < r) {
      if (m < nq) v = coefQ ? coefQ[(size_t)j * nq * r + m * r + i] : mk<double>(0, 0);
      else if (mode == 1 && coefS) v = coefS[(size_t)j * r + i];
    }
    out[e] = mk<T>((T)v.re, (T)v.im);
  }
}

template <typename T>
__global__ void coef_convert_kernel(const zd *coefQ, const zd *coefS, int nq, int r, int mode, cx<T> *out) {
  const int ldc = (nq + 1) * r;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < ldc * r; e += gridDim.x * blockDim.x) {
    const int j = e / ldc, row = e % ldc;
    zd v;
    if (row < nq * r) {
      v = coefQ ? coefQ[(size_t)j * nq * r + row] : mk<double>(0, 0);
    } else {
      const int i = row - nq * r;
      v = (mode == 1 && coefS) ? coefS[(size_t)j * r + i] : mk<double>(0, 0);
    }
    out[e] = mk<T>((T)v.re, (T)v.im);
  }
}

__global__ void reduce_kernel(const double *__restrict__ part, int nparts, int len, double *__restrict__ out) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < len; e += gridDim.x * blockDim.x) {
    double s[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    int p = 0;
    for (; p + 8 <= nparts; p += 8)
#pragma unroll
      for (int u = 0; u < 8; ++u) s[u] += part[(size_t)(p + u) * len + e];
    for (; p < nparts; ++p) s[0] += part[(size_t)p * len + e];
    out[e] = ((s[0] + s[1]) + (s[2] + s[3])) + ((s[4] + s[5]) + (s[6] + s[7]));
  }
}

int ts_max_grid(int nsm) { return 2 * nsm; }
size_t ts_partial_doubles(int gram_left, int r) { return (size_t)(gram_left + 1) * r * r * 2; }

template <typename T>
static int launch_ts_v1(const ModelArgs &M, const TSArgs &a, int nsm, cudaStream_t st) {
  const int r = a.r;
  // choose tile rows / coefficient placement so the CTA fits in shared memory
  const size_t budget = 200 * 1024;
  int tr = 64;
  bool coef_smem = true;
  while (tr > 4 && ts_bytes<T>(a.nq, a.gram_left, r, tr, coef_smem, a.mode) > budget) tr /= 2;
  if (ts_bytes<T>(a.nq, a.gram_left, r, tr, coef_smem, a.mode) > budget) {
    coef_smem = false;
    tr = 64;
    while (tr > 1 && ts_bytes<T>(a.nq, a.gram_left, r, tr, coef_smem, a.mode) > budget) tr /= 2;
  }
  const size_t bytes = ts_bytes<T>(a.nq, a.gram_left, r, tr, coef_smem, a.mode);
  if (bytes > budget) return -1;
  cx<T> *coefg = nullptr;
  if (a.mode != 0) {
    if (!a.coef_scratch) return -1;
    coefg = reinterpret_cast<cx<T> *>(a.coef_scratch);
    ::lrei::count_launch(); coef_convert_kernel<T><<<8, 256, 0, st>>>(a.coefQ, a.coefS, a.nq, r, a.mode, coefg);
  }
  const long long ntiles = (a.N + tr - 1) / tr;
  int grid = (int)(ntiles < (long long)ts_max_grid(nsm) ? ntiles : ts_max_grid(nsm));
  if (grid < 1) grid = 1;
  // pick the widest column group the row length and alignment allow
  const int cpt_max = sizeof(T) == 4 ? 4 : 2;
  int cpt = 1;
  if (r % cpt_max == 0) cpt = cpt_max;
  else if (r % 2 == 0) cpt = 2;
  auto go = [&](auto kern) { ::lrei::count_launch(); kern<<<grid, TS_THREADS, bytes, st>>>(M, a, tr, coef_smem ? 1 : 0, coefg); };
  if (cpt == 4) go(ts_kernel<T, (sizeof(T) == 4 ? 4 : 2)>);
  else if (cpt == 2) go(ts_kernel<T, 2>);
  else go(ts_kernel<T, 1>);
  return grid;
}


// Shared memory of the pipelined pass for the given arguments, or 0 if it does not apply.
static size_t ts3_plan(const TSArgs &a, int *tr) {
  if (a.apply_h) return 0;
  if (a.mode == 0 && a.out) return 0;
  const int r = a.r, nq = a.nq, gl = a.gram_left, mode = a.mode;
  const int nb = nq + (mode != 2 ? 1 : 0);
  if (nb < 1 || nb > 8 || gl + 1 > 8 || gl > nq || (mode == 2 && nq < 1)) return 0;
  auto al = [](const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; };
  for (int m = 0; m < nq; ++m)
    if (!al(a.q[m])) return 0;
  if (mode != 2 && !al(a.src)) return 0;
  if (a.out && !al(a.out)) return 0;
  size_t b = 0;
  if (r == 16) {
    *tr = 32;
    b = ts3_bytes<16, 32>(nq, gl, mode);
  } else if (r == 8) {
    *tr = 64;
    b = ts3_bytes<8, 64>(nq, gl, mode);
  } else if (r == 32) {
    *tr = 32;
    b = ts3_bytes<32, 32>(nq, gl, mode);
  } else {
    return 0;
  }
  return b <= 227 * 1024 ? b : 0;
}

static int launch_ts3(const TSArgs &a, int nsm, cudaStream_t st, size_t bytes, int tr) {
  const cx<float> *coefg = nullptr;
  if (a.mode != 0) {
    if (!a.coef_scratch) return -1;
    coefg = reinterpret_cast<const cx<float> *>(a.coef_scratch);
    ::lrei::count_launch();
    coef_convert2_kernel<float><<<8, 256, 0, st>>>(a.coefQ, a.coefS, a.nq, a.r, a.mode,
                                                  reinterpret_cast<cx<float> *>(a.coef_scratch));
  }
  // persistent, each CTA walking tiles blockIdx.x, + gridDim.x, ...: one CTA per SM at 64-row
  // tiles, two at 32-row tiles (at most 128 registers per thread and 110 KB of shared memory)
  const long long ntiles = (a.N + tr - 1) / tr;
  const long long cap = (tr <= 32 && bytes <= 110 * 1024) ? 2LL * nsm : (long long)nsm;
  int grid = (int)(ntiles < cap ? ntiles : cap);
  if (grid < 1) grid = 1;
  ::lrei::count_launch();
  const int g = a.gram_left + 1;
  if (a.r == 16) {
    if (g <= 2) ts3_kernel<16, 32, 2><<<grid, 256, bytes, st>>>(a, coefg);
    else if (g <= 3) ts3_kernel<16, 32, 3><<<grid, 256, bytes, st>>>(a, coefg);
    else if (g <= 4) ts3_kernel<16, 32, 4><<<grid, 256, bytes, st>>>(a, coefg);
    else if (g <= 5) ts3_kernel<16, 32, 5><<<grid, 256, bytes, st>>>(a, coefg);
    else ts3_kernel<16, 32, 8><<<grid, 256, bytes, st>>>(a, coefg);
  } else if (a.r == 8) {
    ts3_kernel<8, 64, 8><<<grid, 256, bytes, st>>>(a, coefg);
  } else {
    ts3_kernel<32, 32, 8><<<grid, 256, bytes, st>>>(a, coefg);
  }
  return grid;
}

template <typename T>
static int launch_ts_t(const ModelArgs &M, const TSArgs &a, int nsm, cudaStream_t st) {
  if (sizeof(T) == 4) {
    int tr3 = 0;
    const size_t b3 = ts3_plan(a, &tr3);
    if (b3) return launch_ts3(a, nsm, st, b3, tr3);
  }
  const int r = a.r, rp = ts2_rp(r);
  const int NMT = (a.gram_left + 1) * rp / TS2<T>::MI * (rp / TS2<T>::MJ);
  const int mt = NMT <= TS_THREADS ? 1 : (NMT <= 2 * TS_THREADS ? 2 : 0);
  const size_t budget = 200 * 1024;
  int tr = 64;
  if (mt > 0)
    while (tr > 8 && ts2_bytes<T>(a.nq, a.gram_left, r, tr, a.mode, mt) > budget) tr /= 2;
  if (mt == 0 || ts2_bytes<T>(a.nq, a.gram_left, r, tr, a.mode, mt) > budget)
    return launch_ts_v1<T>(M, a, nsm, st);
  const size_t bytes = ts2_bytes<T>(a.nq, a.gram_left, r, tr, a.mode, mt);
  cx<T> *coefg = nullptr;
  if (a.mode != 0) {
    if (!a.coef_scratch) return -1;
    coefg = reinterpret_cast<cx<T> *>(a.coef_scratch);
    ::lrei::count_launch();
    coef_convert2_kernel<T><<<8, 256, 0, st>>>(a.coefQ, a.coefS, a.nq, r, a.mode, coefg);
  }
  const long long ntiles = (a.N + tr - 1) / tr;
  int grid = (int)(ntiles < (long long)ts_max_grid(nsm) ? ntiles : ts_max_grid(nsm));
  if (grid < 1) grid = 1;
  const int cpt_max = sizeof(T) == 4 ? 4 : 2;
  int cpt = 1;
  if (r % cpt_max == 0) cpt = cpt_max;
  else if (r % 2 == 0) cpt = 2;
  auto go = [&](auto kern) { ::lrei::count_launch(); kern<<<grid, TS_THREADS, bytes, st>>>(M, a, tr, coefg); };
  if (mt == 1) {
    if (cpt == cpt_max && cpt_max == 4) go(ts2_kernel<T, (sizeof(T) == 4 ? 4 : 2), 1>);
    else if (cpt == 2) go(ts2_kernel<T, 2, 1>);
    else go(ts2_kernel<T, 1, 1>);
  } else {
    if (cpt == cpt_max && cpt_max == 4) go(ts2_kernel<T, (sizeof(T) == 4 ? 4 : 2), 2>);
    else if (cpt == 2) go(ts2_kernel<T, 2, 2>);
    else go(ts2_kernel<T, 1, 2>);
  }
  return grid;
}

int launch_ts(bool fp64, const ModelArgs &M, const TSArgs &a, int nsm, cudaStream_t st) {
  if (a.nq > MAXB || a.gram_left > a.nq || a.r < 1 || a.r > MAX_R) return -1;
  return fp64 ? launch_ts_t<double>(M, a, nsm, st) : launch_ts_t<float>(M, a, nsm, st);
}

// Two-stage deterministic reduction: CTAs (entry chunk, part slice) sum a fixed slice of parts,
// then one pass sums the slices in order.
__global__ void reduce_slices_kernel(const double *__restrict__ part, int nparts, int len, int nslice,
                                     double *__restrict__ tmp) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  const int sl = blockIdx.y;
  if (e >= len) return;
  const int per = (nparts + nslice - 1) / nslice;
  const int p0 = sl * per, p1 = min(nparts, p0 + per);
  double s[4] = {0, 0, 0, 0};
  int p = p0;
  for (; p + 4 <= p1; p += 4)
#pragma unroll
    for (int u = 0; u < 4; ++u) s[u] += part[(size_t)(p + u) * len + e];
  for (; p < p1; ++p) s[0] += part[(size_t)p * len + e];
  tmp[(size_t)sl * len + e] = (s[0] + s[1]) + (s[2] + s[3]);
}

void launch_reduce(const double *partial, int nparts, int len_doubles, double *out, cudaStream_t st) {
  const int nslice = nparts >= 64 ? 16 : 1;
  if (nslice == 1) {
    int blocks = (len_doubles + 255) / 256;
    ::lrei::count_launch();
    reduce_kernel<<<blocks, 256, 0, st>>>(partial, nparts, len_doubles, out);
    return;
  }
  // the slices live after the partials of the largest grid (ts_max_grid(nsm) parts), which the
  // caller sized with room for nslice extra rows
  double *tmp = const_cast<double *>(partial) + (size_t)nparts * len_doubles;
  dim3 g((len_doubles + 127) / 128, nslice);
  ::lrei::count_launch(2);
  reduce_slices_kernel<<<g, 128, 0, st>>>(partial, nparts, len_doubles, nslice, tmp);
  reduce_kernel<<<(len_doubles + 255) / 256, 256, 0, st>>>(tmp, nslice, len_doubles, out);
}

void launch_hv(bool fp64, const ModelArgs &M, const void *X, void *Y, long long N, int r, int nsm, cudaStream_t st,
               int *status) {
  if (launch_hv_tiled(fp64, M, X, Y, N, r, nsm, st, status)) return;
  // rows that are not a multiple of 16 bytes, or fewer than 16 rows: the per-row gather
  auto grid_for = [&](int cpt) {
    long long total = N * (r / cpt);
    long long g = (total + 255) / 256;
    long long cap = (long long)nsm * 16;
    return (int)(g < cap ? g : cap);
  };
  if (fp64) {
    using T = double;
    if (r % 2 == 0) { ::lrei::count_launch(); hv_kernel<T, 2><<<grid_for(2), 256, 0, st>>>(M, (const cx<T> *)X, (cx<T> *)Y, N, r); }
    else { ::lrei::count_launch(); hv_kernel<T, 1><<<grid_for(1), 256, 0, st>>>(M, (const cx<T> *)X, (cx<T> *)Y, N, r); }
  } else {
    using T = float;
    if (r % 4 == 0) { ::lrei::count_launch(); hv_kernel<T, 4><<<grid_for(4), 256, 0, st>>>(M, (const cx<T> *)X, (cx<T> *)Y, N, r); }
    else if (r % 2 == 0) { ::lrei::count_launch(); hv_kernel<T, 2><<<grid_for(2), 256, 0, st>>>(M, (const cx<T> *)X, (cx<T> *)Y, N, r); }
    else { ::lrei::count_launch(); hv_kernel<T, 1><<<grid_for(1), 256, 0, st>>>(M, (const cx<T> *)X, (cx<T> *)Y, N, r); }
  }
}

// ------------------------------------------------------ observables
// Row b of M_x V and M_y V: (1/n) sum over spins q of (1/2) V[b ^ 2^q] and
// (1/2)(bit_q(b) ? +i : -i) V[b ^ 2^q] (sigma_y with bit 0 = spin up).
constexpr int OBS_BLOCKS = 6;

template <typename T>
__global__ void __launch_bounds__(256) obs_kernel(const __grid_constant__ ModelArgs M, const cx<T> *__restrict__ V, long long N, int r,
                                                  int tr, double *partial) {
  extern __shared__ __align__(16) unsigned char smem[];
  cx<T> *vs = reinterpret_cast<cx<T> *>(smem);   // tr x r
  cx<T> *ss = vs + (size_t)tr * r;                // H V
  cx<T> *xs = ss + (size_t)tr * r;                // Mx V
  cx<T> *ys = xs + (size_t)tr * r;                // My V
  cx<T> *zs = ys + (size_t)tr * r;                // Mz V
  double *acc = reinterpret_cast<double *>(zs + (size_t)tr * r);
  const int tid = threadIdx.x, nt = blockDim.x;
  const int nent = OBS_BLOCKS * r * r;
  for (int e = tid; e < nent * 2; e += nt) acc[e] = 0.0;
  __syncthreads();
  const T inv_n = (T)(1.0 / M.n);
  const long long ntiles = (N + tr - 1) / tr;
  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const long long row0 = tile * tr;
    const int rows = (int)((N - row0) < tr ? (N - row0) : tr);
    for (int e = tid; e < tr * r; e += nt) {
      const int lr = e / r, c = e % r;
      cx<T> v = mk<T>(0, 0), s = v, x = v, y = v, z = v;
      if (lr < rows) {
        const uint32_t b = (uint32_t)(row0 + lr);
        cx<T> o[1];
        hv_group<T, 1>(M, V, r, b, c, o);
        s = o[0];
        v = ldg1(V + (size_t)b * r + c);
        for (int q = 0; q < M.n; ++q) {
          const cx<T> p = ldg1(V + (size_t)(b ^ (1u << q)) * r + c);
          x = x + p;
          // (sigma_y)_{0,1} = -i, (sigma_y)_{1,0} = +i
          if ((b >> q) & 1u) y = y + mk<T>(-p.im, p.re);
          else y = y + mk<T>(p.im, -p.re);
        }
        x = ((T)0.5 * inv_n) * x;
        y = ((T)0.5 * inv_n) * y;
        z = ((T)((0.5 * M.n - (double)__popc(b)) / M.n)) * v;
      }
      vs[e] = v; ss[e] = s; xs[e] = x; ys[e] = y; zs[e] = z;
    }
    __syncthreads();
    for (int e = tid; e < nent; e += nt) {
      const int blk = e / (r * r), j = (e / r) % r, i = e % r;
      const cx<T> *L = (blk == 1) ? ss : vs;
      const cx<T> *R = blk == 0 ? ss : blk == 1 ? ss : blk == 2 ? vs : blk == 3 ? xs : blk == 4 ? ys : zs;
      cx<T> s = mk<T>(0, 0);
      for (int lr = 0; lr < tr; ++lr) fmac_(s, L[lr * r + i], R[lr * r + j]);
      Acc<T>::add(acc, e, s);
    }
    __syncthreads();
  }
  double *outp = partial + (size_t)blockIdx.x * nent * 2;
  for (int e = tid; e < nent; e += nt) {
    cx<double> v = Acc<T>::get(acc, e);
    outp[2 * e] = v.re;
    outp[2 * e + 1] = v.im;
  }
}

int launch_obs(bool fp64, const ModelArgs &M, const void *V, long long N, int r, double *partial, int nsm,
               cudaStream_t st) {
  const int tr = 16;
  const long long ntiles = (N + tr - 1) / tr;
  int grid = (int)(ntiles < (long long)ts_max_grid(nsm) ? ntiles : ts_max_grid(nsm));
  if (grid < 1) grid = 1;
  const size_t nent = (size_t)OBS_BLOCKS * r * r;
  if (fp64) {
    size_t bytes = 5 * (size_t)tr * r * sizeof(cx<double>) + nent * 16;
    ::lrei::count_launch(); obs_kernel<double><<<grid, 256, bytes, st>>>(M, (const cx<double> *)V, N, r, tr, partial);
  } else {
    size_t bytes = 5 * (size_t)tr * r * sizeof(cx<float>) + nent * 16;
    ::lrei::count_launch(); obs_kernel<float><<<grid, 256, bytes, st>>>(M, (const cx<float> *)V, N, r, tr, partial);
  }
  return grid;
}


// Same pass with the number of partial sums capped (used by the allocation-free observables).
int launch_obs_capped(bool fp64, const ModelArgs &M, const void *V, long long N, int r, double *partial,
                      int max_grid, cudaStream_t st) {
  const int tr = 16;
  const long long ntiles = (N + tr - 1) / tr;
  int grid = (int)(ntiles < (long long)max_grid ? ntiles : max_grid);
  if (grid < 1) grid = 1;
  const size_t nent = (size_t)OBS_BLOCKS * r * r;
  if (fp64) {
    size_t bytes = 5 * (size_t)tr * r * sizeof(cx<double>) + nent * 16;
    ::lrei::count_launch(); obs_kernel<double><<<grid, 256, bytes, st>>>(M, (const cx<double> *)V, N, r, tr, partial);
  } else {
    size_t bytes = 5 * (size_t)tr * r * sizeof(cx<float>) + nent * 16;
    ::lrei::count_launch(); obs_kernel<float><<<grid, 256, bytes, st>>>(M, (const cx<float> *)V, N, r, tr, partial);
  }
  return grid;
}


// ------------------------------------------------------ conversion / checks
template <typename S, typename D>
__global__ void convert_kernel(const cx<S> *src, int ld, cx<D> *dst, long long N, int r) {
  const long long total = N * r;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long b = e / r;
    const int c = (int)(e % r);
    const cx<S> v = src[b * ld + c];
    dst[e] = mk<D>((D)v.re, (D)v.im);
  }
}

void launch_convert(const void *src, int src_c64, int ld, void *dst, int dst_fp64, long long N, int r,
                    cudaStream_t st) {
  long long total = N * r;
  int grid = (int)((total + 255) / 256 < 4096 ? (total + 255) / 256 : 4096);
  if (grid < 1) grid = 1;
  if (src_c64) {
    if (dst_fp64) { ::lrei::count_launch(); convert_kernel<float, double><<<grid, 256, 0, st>>>((const cx<float> *)src, ld, (cx<double> *)dst, N, r); }
    else { ::lrei::count_launch(); convert_kernel<float, float><<<grid, 256, 0, st>>>((const cx<float> *)src, ld, (cx<float> *)dst, N, r); }
  } else {
    if (dst_fp64) { ::lrei::count_launch(); convert_kernel<double, double><<<grid, 256, 0, st>>>((const cx<double> *)src, ld, (cx<double> *)dst, N, r); }
    else { ::lrei::count_launch(); convert_kernel<double, float><<<grid, 256, 0, st>>>((const cx<double> *)src, ld, (cx<float> *)dst, N, r); }
  }
}

template <typename T>
__global__ void finite_kernel(const T *x, long long n, int *status) {
  bool bad = false;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
    if (!isfinite(x[e])) bad = true;
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(status, ST_NONFINITE);
}

void launch_check_finite(bool fp64, const void *X, long long N, int r, int *status, cudaStream_t st) {
  long long n = N * r * 2;
  int grid = (int)((n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024);
  if (grid < 1) grid = 1;
  if (fp64) { ::lrei::count_launch(); finite_kernel<double><<<grid, 256, 0, st>>>((const double *)X, n, status); }
  else { ::lrei::count_launch(); finite_kernel<float><<<grid, 256, 0, st>>>((const float *)X, n, status); }
}

}  // namespace lrei

namespace lrei {
// Raise the dynamic shared-memory limit of every tile kernel once (outside any stream capture).
int ts_init() {
  if (hv_tiled_init()) return -1;
  const int lim = 210 * 1024;
  cudaError_t e = cudaSuccess;
  auto set = [&](const void *f) {
    cudaError_t x = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    if (x != cudaSuccess) e = x;
  };
  auto set3 = [&](const void *f) {
    cudaError_t x = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    if (x != cudaSuccess) e = x;
  };
  set3((const void *)ts3_kernel<16, 32, 2>);
  set3((const void *)ts3_kernel<16, 32, 3>);
  set3((const void *)ts3_kernel<16, 32, 4>);
  set3((const void *)ts3_kernel<16, 32, 5>);
  set3((const void *)ts3_kernel<16, 32, 8>);
  set3((const void *)ts3_kernel<8, 64, 8>);
  set3((const void *)ts3_kernel<32, 32, 8>);
  set((const void *)ts_kernel<double, 2>);
  set((const void *)ts_kernel<double, 1>);
  set((const void *)ts_kernel<float, 4>);
  set((const void *)ts_kernel<float, 2>);
  set((const void *)ts_kernel<float, 1>);
  set((const void *)ts2_kernel<double, 2, 1>);
  set((const void *)ts2_kernel<double, 1, 1>);
  set((const void *)ts2_kernel<double, 2, 2>);
  set((const void *)ts2_kernel<double, 1, 2>);
  set((const void *)ts2_kernel<float, 4, 1>);
  set((const void *)ts2_kernel<float, 2, 1>);
  set((const void *)ts2_kernel<float, 1, 1>);
  set((const void *)ts2_kernel<float, 4, 2>);
  set((const void *)ts2_kernel<float, 2, 2>);
  set((const void *)ts2_kernel<float, 1, 2>);
  set((const void *)obs_kernel<double>);
  set((const void *)obs_kernel<float>);
  return e == cudaSuccess ? 0 : -1;
}
}  // namespace lrei
