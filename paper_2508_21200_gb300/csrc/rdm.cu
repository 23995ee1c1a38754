// Two-spin reduced density matrices R_kl and their entanglement measures (paper Sec. 3.6: the
// partial trace of rho over every spin but k and l, measured from the low-rank factor; the
// concurrence of Wootters (1998) and the negativity of Vidal and Werner (2002) from the 4 x 4).
//
// With rho = Vb Lambda Vb^* (Vb the orthonormalised factor), the rows of the N x r factor fall
// into N/4 groups of four that differ only in the bits of sites k and l; group g with the two
// bits set to s = (s_k, s_l) is row b_s(g), and
//     R[s, s'] = sum_g sum_c lambda_c Vb[b_s(g), c] conj(Vb[b_s'(g), c]),
// the index of R being 2 s_k + s_l (site k the first factor, 0 = spin up).  One pass per pair
// over the factor computes the ten entries s <= s'; each thread owns one column c of a group
// (threads of consecutive columns read consecutive words of a row) and keeps running sums,
// compensated (TwoSum) in the complex64 path, combined per CTA and written as FP64 partials.
// A one-thread-per-pair FP64 kernel then sums the partials in a fixed order, applies the Werner
// weight p (R -> p I/4 + (1 - p) R) and evaluates the two measures by 4 x 4 Jacobi.
#include "common.cuh"

namespace lrei {

namespace {

__device__ __forceinline__ void two_sum(float &hi, float &lo, float b) {
  const float s = hi + b, bp = s - hi;
  lo += (hi - (s - bp)) + (b - bp);
  hi = s;
}

template <typename T> struct RAcc;
template <> struct RAcc<double> {
  double v[20];
  __device__ void zero() {
#pragma unroll
    for (int i = 0; i < 20; ++i) v[i] = 0.0;
  }
  __device__ void add(int i, double x) { v[i] += x; }
  __device__ double get(int i) const { return v[i]; }
};
template <> struct RAcc<float> {
  float v[20], e[20];
  __device__ void zero() {
#pragma unroll
    for (int i = 0; i < 20; ++i) v[i] = e[i] = 0.f;
  }
  __device__ void add(int i, float x) { two_sum(v[i], e[i], x); }
  __device__ double get(int i) const { return (double)v[i] + (double)e[i]; }
};

__device__ __forceinline__ uint32_t insert_zero(uint32_t x, int pos) {
  const uint32_t low = x & ((1u << pos) - 1u);
  return low | ((x >> pos) << (pos + 1));
}

}  // namespace

// pairs: 2 ints per pair, the bit positions of sites k and l in the basis index.
// partial: [npairs][gridDim.x][20] doubles (entries (s, s') with s <= s' in row order, re/im).
template <typename T>
__global__ void __launch_bounds__(256) rdm_kernel(const cx<T> *__restrict__ V, long long N, int r,
                                                  const double *__restrict__ lam, const int *__restrict__ pairs,
                                                  double *__restrict__ partial) {
  __shared__ double red[8][20];
  const int p = blockIdx.y;
  const int bk = pairs[2 * p], bl = pairs[2 * p + 1];
  const int lo = bk < bl ? bk : bl, hi = bk < bl ? bl : bk;
  const int tid = threadIdx.x;
  const int gpb = 256 / r;                              // groups per CTA pass (one thread per column)
  const int c = tid % r, gl = tid / r;
  const long long ngroups = N >> 2;
  const T lc = (T)lam[c < r ? c : 0];
  RAcc<T> acc;
  acc.zero();
  if (gl < gpb) {
    for (long long g = (long long)blockIdx.x * gpb + gl; g < ngroups; g += (long long)gridDim.x * gpb) {
      const uint32_t b0 = insert_zero(insert_zero((uint32_t)g, lo), hi);
      cx<T> v[4];
#pragma unroll
      for (int s = 0; s < 4; ++s) {
        const uint32_t b = b0 | ((uint32_t)(s >> 1) << bk) | ((uint32_t)(s & 1) << bl);
        v[s] = V[(size_t)b * r + c];
      }
      int e = 0;
#pragma unroll
      for (int s = 0; s < 4; ++s)
#pragma unroll
        for (int t = s; t < 4; ++t) {
          // lambda_c v_s conj(v_t)
          const T re = v[s].re * v[t].re + v[s].im * v[t].im;
          const T im = v[s].im * v[t].re - v[s].re * v[t].im;
          acc.add(2 * e, lc * re);
          acc.add(2 * e + 1, lc * im);
          ++e;
        }
    }
  }
  // combine the CTA's threads: warp shuffles, then the warps in a fixed order
  const int lane = tid & 31, wp = tid >> 5;
#pragma unroll
  for (int i = 0; i < 20; ++i) {
    double x = acc.get(i);
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (lane == 0) red[wp][i] = x;
  }
  __syncthreads();
  if (tid < 20) {
    double s = 0.0;
    for (int w = 0; w < 8; ++w) s += red[w][tid];
    partial[((size_t)p * gridDim.x + blockIdx.x) * 20 + tid] = s;
  }
}

namespace {
// Eigenvalues (decreasing) and eigenvectors (columns of U, 4 x 4 column-major) of a Hermitian 4 x 4
// matrix A (column-major, overwritten) by cyclic complex Jacobi in FP64.
__device__ void herm4_eig(zd *A, zd *U, double *w) {
  for (int i = 0; i < 16; ++i) U[i] = mk<double>((i % 5) == 0 ? 1.0 : 0.0, 0.0);
  for (int sweep = 0; sweep < 30; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int i = 0; i < 16; ++i) {
      tot += norm2(A[i]);
      if (i % 5) off += norm2(A[i]);
    }
    if (off <= 1e-32 * tot || off == 0.0) break;
    for (int p = 0; p < 3; ++p)
      for (int q = p + 1; q < 4; ++q) {
        const zd apq = A[q * 4 + p];
        const double ab = sqrt(norm2(apq));
        if (ab == 0.0) continue;
        const double app = A[p * 4 + p].re, aqq = A[q * 4 + q].re;
        // rotate so that the (p, q) entry vanishes: phase e = apq / |apq|
        const double theta = 0.5 * (aqq - app) / ab;
        const double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
        const double cs = 1.0 / sqrt(t * t + 1.0), sn = t * cs;
        const zd e = mk<double>(apq.re / ab, apq.im / ab);
        // columns: A <- A G with G = [[c, s e], [-s conj(e), c]] on (p, q)
        for (int i = 0; i < 4; ++i) {
          const zd aip = A[p * 4 + i], aiq = A[q * 4 + i];
          A[p * 4 + i] = cs * aip - sn * (aiq * conj(e));
          A[q * 4 + i] = cs * aiq + sn * (aip * e);
          const zd uip = U[p * 4 + i], uiq = U[q * 4 + i];
          U[p * 4 + i] = cs * uip - sn * (uiq * conj(e));
          U[q * 4 + i] = cs * uiq + sn * (uip * e);
        }
        // rows: A <- G^H A
        for (int j = 0; j < 4; ++j) {
          const zd apj = A[j * 4 + p], aqj = A[j * 4 + q];
          A[j * 4 + p] = cs * apj - sn * (aqj * e);
          A[j * 4 + q] = cs * aqj + sn * (apj * conj(e));
        }
      }
  }
  for (int i = 0; i < 4; ++i) w[i] = A[i * 4 + i].re;
  // sort decreasing (with the vectors)
  for (int i = 0; i < 4; ++i)
    for (int j = i + 1; j < 4; ++j)
      if (w[j] > w[i]) {
        const double tw = w[i]; w[i] = w[j]; w[j] = tw;
        for (int m = 0; m < 4; ++m) { const zd tu = U[i * 4 + m]; U[i * 4 + m] = U[j * 4 + m]; U[j * 4 + m] = tu; }
      }
}
}  // namespace

// One thread per pair: R from the partials, the Werner map, concurrence and negativity.
// out: [npairs][32 + 2] doubles: R (4 x 4 complex, column-major), concurrence, negativity.
__global__ void rdm_final_kernel(const double *__restrict__ partial, int nparts, int npairs, double p_werner,
                                 double *__restrict__ out) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= npairs) return;
  double s[20];
  for (int i = 0; i < 20; ++i) s[i] = 0.0;
  for (int b = 0; b < nparts; ++b)
    for (int i = 0; i < 20; ++i) s[i] += partial[((size_t)q * nparts + b) * 20 + i];
  zd R[16];
  int e = 0;
  for (int a = 0; a < 4; ++a)
    for (int t = a; t < 4; ++t) {
      const zd v = mk<double>(s[2 * e], s[2 * e + 1]);
      R[t * 4 + a] = v;            // (a, t)
      R[a * 4 + t] = conj(v);      // (t, a)
      ++e;
    }
  const double qw = 1.0 - p_werner;
  for (int i = 0; i < 16; ++i) R[i] = qw * R[i];
  for (int i = 0; i < 4; ++i) R[i * 5].re += 0.25 * p_werner;
  double *o = out + (size_t)q * 34;
  for (int i = 0; i < 16; ++i) {
    o[2 * i] = R[i].re;
    o[2 * i + 1] = R[i].im;
  }
  // concurrence: C = max(0, s1 - s2 - s3 - s4), s_i the decreasing square roots of the eigenvalues
  // of R Rt, Rt = (Y x Y) conj(R) (Y x Y), which are those of the Hermitian sqrt(R) Rt sqrt(R)
  zd A[16], U[16], S[16], Rt[16], Tm[16];
  double w[4];
  for (int i = 0; i < 16; ++i) A[i] = R[i];
  herm4_eig(A, U, w);
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) {
      zd v = mk<double>(0, 0);
      for (int m = 0; m < 4; ++m) v = v + sqrt(fmax(w[m], 0.0)) * (U[m * 4 + i] * conj(U[m * 4 + j]));
      S[j * 4 + i] = v;
    }
  // (Y x Y)_{ab} = -1 for (a, b) in {(0,3), (3,0)}, +1 for {(1,2), (2,1)}, 0 otherwise
  const int yy_col[4] = {3, 2, 1, 0};
  const double yy_val[4] = {-1.0, 1.0, 1.0, -1.0};
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) {
      // Rt_ij = sum yy_i,a conj(R_ab) yy_b,j with a = yy_col[i], b = yy_col[j]
      Rt[j * 4 + i] = (yy_val[i] * yy_val[j]) * conj(R[yy_col[j] * 4 + yy_col[i]]);
    }
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) {
      zd v = mk<double>(0, 0);
      for (int m = 0; m < 4; ++m) v = v + Rt[m * 4 + i] * S[j * 4 + m];
      Tm[j * 4 + i] = v;   // Rt S
    }
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) {
      zd v = mk<double>(0, 0);
      for (int m = 0; m < 4; ++m) v = v + S[m * 4 + i] * Tm[j * 4 + m];
      A[j * 4 + i] = v;    // S Rt S
    }
  for (int i = 0; i < 4; ++i)
    for (int j = i + 1; j < 4; ++j) {
      const zd h = mk<double>(0.5 * (A[j * 4 + i].re + A[i * 4 + j].re), 0.5 * (A[j * 4 + i].im - A[i * 4 + j].im));
      A[j * 4 + i] = h;
      A[i * 4 + j] = conj(h);
    }
  for (int i = 0; i < 4; ++i) A[i * 5].im = 0.0;
  herm4_eig(A, U, w);
  const double c = sqrt(fmax(w[0], 0.0)) - sqrt(fmax(w[1], 0.0)) - sqrt(fmax(w[2], 0.0)) - sqrt(fmax(w[3], 0.0));
  o[32] = fmax(0.0, c);
  // negativity: minus the sum of the negative eigenvalues of the partial transpose on spin l:
  // T[(a0 a1), (b0 b1)] = R[(a0 b1), (b0 a1)]
  for (int a0 = 0; a0 < 2; ++a0)
    for (int a1 = 0; a1 < 2; ++a1)
      for (int b0 = 0; b0 < 2; ++b0)
        for (int b1 = 0; b1 < 2; ++b1) A[(2 * b0 + b1) * 4 + (2 * a0 + a1)] = R[(2 * b0 + a1) * 4 + (2 * a0 + b1)];
  herm4_eig(A, U, w);
  double neg = 0.0;
  for (int i = 0; i < 4; ++i)
    if (w[i] < 0.0) neg -= w[i];
  o[33] = neg;
}

int launch_rdm(bool fp64, const void *V, long long N, int r, const double *lam, const int *pairs, int npairs,
               double *partial, int ncta, cudaStream_t st) {
  if (npairs <= 0 || r < 1 || r > 256 || N < 4) return -1;
  dim3 grid(ncta, npairs);
  ::lrei::count_launch();
  if (fp64) rdm_kernel<double><<<grid, 256, 0, st>>>((const cx<double> *)V, N, r, lam, pairs, partial);
  else rdm_kernel<float><<<grid, 256, 0, st>>>((const cx<float> *)V, N, r, lam, pairs, partial);
  return 0;
}

void launch_rdm_final(const double *partial, int nparts, int npairs, double p_werner, double *out, cudaStream_t st) {
  ::lrei::count_launch();
  rdm_final_kernel<<<(npairs + 63) / 64, 64, 0, st>>>(partial, nparts, npairs, p_werner, out);
}

}  // namespace lrei
