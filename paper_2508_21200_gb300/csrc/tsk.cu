// Tall-skinny (N-length) kernels of the LREI hot path.
//
//  * Matrix-free H.V (paper Sec. 3.3: "sparsity of H"; Hamiltonian eq. H1):
//    row b of Y = H V is diag(b) V[b] + sum over bonds whose two spins are
//    antiparallel in b of jxy * V[b ^ mask], with mask the two bonds' bits.
//    A thread owns CPT consecutive columns of one row; partner rows are read
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

namespace lrei {

// ---------------------------------------------------------------- loads
template <typename T> struct VecT;
template <> struct VecT<float> { using v2 = float2; using v4 = float4; };
template <> struct VecT<double> { using v2 = double2; using v4 = double4; };

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
        if (lr >= rows) s = mk<T>(0, 0);
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
    double s = 0.0;
    for (int p = 0; p < nparts; ++p) s += part[(size_t)p * len + e];
    out[e] = s;
  }
}

int ts_max_grid(int nsm) { return 2 * nsm; }
size_t ts_partial_doubles(int gram_left, int r) { return (size_t)(gram_left + 1) * r * r * 2; }

template <typename T>
static int launch_ts_t(const ModelArgs &M, const TSArgs &a, int nsm, cudaStream_t st) {
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
    coef_convert_kernel<T><<<8, 256, 0, st>>>(a.coefQ, a.coefS, a.nq, r, a.mode, coefg);
  }
  const long long ntiles = (a.N + tr - 1) / tr;
  int grid = (int)(ntiles < (long long)ts_max_grid(nsm) ? ntiles : ts_max_grid(nsm));
  if (grid < 1) grid = 1;
  // pick the widest column group the row length and alignment allow
  const int cpt_max = sizeof(T) == 4 ? 4 : 2;
  int cpt = 1;
  if (r % cpt_max == 0) cpt = cpt_max;
  else if (r % 2 == 0) cpt = 2;
  auto go = [&](auto kern) { kern<<<grid, TS_THREADS, bytes, st>>>(M, a, tr, coef_smem ? 1 : 0, coefg); };
  if (cpt == 4) go(ts_kernel<T, (sizeof(T) == 4 ? 4 : 2)>);
  else if (cpt == 2) go(ts_kernel<T, 2>);
  else go(ts_kernel<T, 1>);
  return grid;
}

int launch_ts(bool fp64, const ModelArgs &M, const TSArgs &a, int nsm, cudaStream_t st) {
  if (a.nq > MAXB || a.gram_left > a.nq || a.r < 1 || a.r > MAX_R) return -1;
  return fp64 ? launch_ts_t<double>(M, a, nsm, st) : launch_ts_t<float>(M, a, nsm, st);
}

void launch_reduce(const double *partial, int nparts, int len_doubles, double *out, cudaStream_t st) {
  int blocks = (len_doubles + 255) / 256;
  if (blocks > 1024) blocks = 1024;
  reduce_kernel<<<blocks, 256, 0, st>>>(partial, nparts, len_doubles, out);
}

void launch_hv(bool fp64, const ModelArgs &M, const void *X, void *Y, long long N, int r, int nsm, cudaStream_t st) {
  auto grid_for = [&](int cpt) {
    long long total = N * (r / cpt);
    long long g = (total + 255) / 256;
    long long cap = (long long)nsm * 16;
    return (int)(g < cap ? g : cap);
  };
  if (fp64) {
    using T = double;
    if (r % 2 == 0) hv_kernel<T, 2><<<grid_for(2), 256, 0, st>>>(M, (const cx<T> *)X, (cx<T> *)Y, N, r);
    else hv_kernel<T, 1><<<grid_for(1), 256, 0, st>>>(M, (const cx<T> *)X, (cx<T> *)Y, N, r);
  } else {
    using T = float;
    if (r % 4 == 0) hv_kernel<T, 4><<<grid_for(4), 256, 0, st>>>(M, (const cx<T> *)X, (cx<T> *)Y, N, r);
    else if (r % 2 == 0) hv_kernel<T, 2><<<grid_for(2), 256, 0, st>>>(M, (const cx<T> *)X, (cx<T> *)Y, N, r);
    else hv_kernel<T, 1><<<grid_for(1), 256, 0, st>>>(M, (const cx<T> *)X, (cx<T> *)Y, N, r);
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
    obs_kernel<double><<<grid, 256, bytes, st>>>(M, (const cx<double> *)V, N, r, tr, partial);
  } else {
    size_t bytes = 5 * (size_t)tr * r * sizeof(cx<float>) + nent * 16;
    obs_kernel<float><<<grid, 256, bytes, st>>>(M, (const cx<float> *)V, N, r, tr, partial);
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
    if (dst_fp64) convert_kernel<float, double><<<grid, 256, 0, st>>>((const cx<float> *)src, ld, (cx<double> *)dst, N, r);
    else convert_kernel<float, float><<<grid, 256, 0, st>>>((const cx<float> *)src, ld, (cx<float> *)dst, N, r);
  } else {
    if (dst_fp64) convert_kernel<double, double><<<grid, 256, 0, st>>>((const cx<double> *)src, ld, (cx<double> *)dst, N, r);
    else convert_kernel<double, float><<<grid, 256, 0, st>>>((const cx<double> *)src, ld, (cx<float> *)dst, N, r);
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
  if (fp64) finite_kernel<double><<<grid, 256, 0, st>>>((const double *)X, n, status);
  else finite_kernel<float><<<grid, 256, 0, st>>>((const float *)X, n, status);
}

}  // namespace lrei

namespace lrei {
// Raise the dynamic shared-memory limit of every tile kernel once (outside any stream capture).
int ts_init() {
  const int lim = 210 * 1024;
  cudaError_t e = cudaSuccess;
  auto set = [&](const void *f) {
    cudaError_t x = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    if (x != cudaSuccess) e = x;
  };
  set((const void *)ts_kernel<double, 2>);
  set((const void *)ts_kernel<double, 1>);
  set((const void *)ts_kernel<float, 4>);
  set((const void *)ts_kernel<float, 2>);
  set((const void *)ts_kernel<float, 1>);
  set((const void *)obs_kernel<double>);
  set((const void *)obs_kernel<float>);
  return e == cudaSuccess ? 0 : -1;
}
}  // namespace lrei
