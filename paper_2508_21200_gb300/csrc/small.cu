// Small dense complex linear algebra for the r x r / k x k part of the LREI step.
//
// These solves are FP64 in every precision mode.  GB300 executes FP64 at a
// small fraction of its FP32 rate per SM, so every kernel here spreads its
// FP64 work over many small CTAs (a warp per output entry or per column)
// instead of running on one SM.  The one exception is the cyclic Jacobi
// eigensolver, which runs in one CTA: the k x k eigenproblem of each stage
// is solved in FP32 and then corrected to FP64 accuracy on its top-r
// invariant subspace (sm_eig_topr), so only r x r Jacobi runs in FP64.
#include "small.cuh"

#include <cstdlib>

namespace lrei {

// [0] FP32 Jacobi calls, [1] FP32 sweeps, [2] FP64 Jacobi calls, [3] FP64 sweeps (diagnostics)
__device__ unsigned long long g_jacobi_counters[4];

__device__ __forceinline__ zd zdiv_real(zd a, double d) { return mk<double>(a.re / d, a.im / d); }
__device__ __forceinline__ zd zdiv(zd a, zd d) {
  const double n = d.re * d.re + d.im * d.im;
  return mk<double>((a.re * d.re + a.im * d.im) / n, (a.im * d.re - a.re * d.im) / n);
}
__device__ __forceinline__ zd warp_sum(zd v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    v.re += __shfl_xor_sync(0xffffffffu, v.re, o);
    v.im += __shfl_xor_sync(0xffffffffu, v.im, o);
  }
  return v;
}

// ------------------------------------------------------------------ GEMM
__device__ __forceinline__ zd opget(char op, const zd *A, int ld, int i, int p) {
  return op == 'N' ? A[(size_t)p * ld + i] : conj(A[(size_t)i * ld + p]);
}

__global__ void gemm_thread_kernel(char opA, char opB, int M, int N, int K, zd alpha, const zd *__restrict__ A, int lda,
                                   const zd *__restrict__ B, int ldb, zd beta, zd *__restrict__ C, int ldc) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= M * N) return;
  const int i = e % M, j = e / M;
  zd s = mk<double>(0, 0);
  for (int p = 0; p < K; ++p) fma_(s, opget(opA, A, lda, i, p), opget(opB, B, ldb, p, j));
  zd c = alpha * s;
  if (beta.re != 0.0 || beta.im != 0.0) c = c + beta * C[(size_t)j * ldc + i];
  C[(size_t)j * ldc + i] = c;
}

__global__ void gemm_warp_kernel(char opA, char opB, int M, int N, int K, zd alpha, const zd *__restrict__ A, int lda,
                                 const zd *__restrict__ B, int ldb, zd beta, zd *__restrict__ C, int ldc) {
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (w >= M * N) return;
  const int i = w % M, j = w / M;
  zd s = mk<double>(0, 0);
  for (int p = lane; p < K; p += 32) fma_(s, opget(opA, A, lda, i, p), opget(opB, B, ldb, p, j));
  s = warp_sum(s);
  if (lane == 0) {
    zd c = alpha * s;
    if (beta.re != 0.0 || beta.im != 0.0) c = c + beta * C[(size_t)j * ldc + i];
    C[(size_t)j * ldc + i] = c;
  }
}

void sm_gemm(char opA, char opB, int M, int N, int K, zd alpha, const zd *A, int lda, const zd *B, int ldb, zd beta,
             zd *C, int ldc, cudaStream_t st) {
  if (M <= 0 || N <= 0) return;
  if (K >= 48) {
    const long long threads = (long long)M * N * 32;
    ::lrei::count_launch(); gemm_warp_kernel<<<(int)((threads + 127) / 128), 128, 0, st>>>(opA, opB, M, N, K, alpha, A, lda, B, ldb, beta, C,
                                                                    ldc);
  } else {
    ::lrei::count_launch(); gemm_thread_kernel<<<(M * N + 63) / 64, 64, 0, st>>>(opA, opB, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc);
  }
}

// ------------------------------------------------------- triangular solves
// Triangular solves, one warp per right-hand side, four warps per CTA sharing one copy of the
// triangle in shared memory.  Right-looking: x_j = b_j / d_j is broadcast from shared memory and
// every lane updates the rows it owns, so the loop has no reductions and no divisions (the
// reciprocal diagonal is precomputed).  Up to k = 90 the triangle is staged in shared memory
// (column j of T holds the multipliers of x_j); larger k reads it from global memory.
constexpr int TRSV_SMEM_K = 90;
__global__ void __launch_bounds__(128) trsv_kernel(char op, const zd *__restrict__ L, int ldl, int k,
                                                   zd *__restrict__ B, int ldb, int ncols) {
  extern __shared__ zd trsv_sm[];
  const bool staged = k <= TRSV_SMEM_K;
  zd *Ts = trsv_sm;                                  // k x k: Ts[j*k + i] = multiplier of x_j in row i
  zd *xs = staged ? trsv_sm + (size_t)k * k : trsv_sm;    // 4 warps x k
  double *rd = reinterpret_cast<double *>(xs + 4 * k);   // k reciprocal diagonal entries
  const int t = threadIdx.x, lane = t & 31, wp = t >> 5;
  for (int i = t; i < k; i += blockDim.x) {
    const double d = L[(size_t)i * ldl + i].re;
    rd[i] = d != 0.0 ? 1.0 / d : 0.0;
  }
  if (staged) {
    for (int e = t; e < k * k; e += blockDim.x) {
      const int i = e % k, j = e / k;
      zd v = mk<double>(0, 0);
      if (op == 'N') { if (i > j) v = L[(size_t)j * ldl + i]; }          // L(i, j)
      else { if (i < j) v = conj(L[(size_t)i * ldl + j]); }               // (L^H)(i, j) = conj(L(j, i))
      Ts[e] = v;
    }
  }
  const int col = blockIdx.x * 4 + wp;
  zd *x = xs + wp * k;
  zd *bcol = B + (size_t)col * ldb;
  if (col < ncols)
    for (int i = lane; i < k; i += 32) x[i] = bcol[i];
  __syncthreads();
  if (col < ncols) {
    auto mult = [&](int i, int j) -> zd {
      if (staged) return Ts[(size_t)j * k + i];
      return op == 'N' ? L[(size_t)j * ldl + i] : conj(L[(size_t)i * ldl + j]);
    };
    if (op == 'N') {
      for (int j = 0; j < k; ++j) {
        __syncwarp();
        const zd xj = mk<double>(x[j].re * rd[j], x[j].im * rd[j]);
        __syncwarp();
        if (lane == 0) x[j] = xj;
        for (int i = j + 1 + lane; i < k; i += 32) x[i] = x[i] - mult(i, j) * xj;
      }
    } else {
      for (int j = k - 1; j >= 0; --j) {
        __syncwarp();
        const zd xj = mk<double>(x[j].re * rd[j], x[j].im * rd[j]);
        __syncwarp();
        if (lane == 0) x[j] = xj;
        for (int i = lane; i < j; i += 32) x[i] = x[i] - mult(i, j) * xj;
      }
    }
    __syncwarp();
    for (int i = lane; i < k; i += 32) bcol[i] = x[i];
  }
}

void sm_trsv(char op, const zd *L, int ldl, int k, zd *B, int ldb, int ncols, cudaStream_t st) {
  if (ncols <= 0 || k <= 0) return;
  const size_t bytes = ((k <= TRSV_SMEM_K ? (size_t)k * k : 0) + 4 * (size_t)k) * sizeof(zd) + (size_t)k * 8;
  ::lrei::count_launch();
  trsv_kernel<<<(ncols + 3) / 4, 128, bytes, st>>>(op, L, ldl, k, B, ldb, ncols);
}

// X <- X (L^H)^{-1}: the inverse (L^H)^{-1} is formed by triangular solves on the identity and
// applied with one GEMM, so no FP64 dependency chain runs per row.  Needs a k x k scratch and a
// copy of X (both from the caller's workspace).
void sm_rtrsm_lh_ws(zd *X, int ldx, int nrows, const zd *L, int ldl, int k, zd *inv, zd *xcopy, cudaStream_t st) {
  if (nrows <= 0) return;
  sm_set_identity(inv, k, k, k, st);
  sm_trsv('C', L, ldl, k, inv, k, k, st);                 // inv = (L^H)^{-1}
  sm_copy(X, ldx, nrows, k, xcopy, nrows, st);
  sm_gemm('N', 'N', nrows, k, k, mk<double>(1, 0), xcopy, nrows, inv, k, mk<double>(0, 0), X, ldx, st);
}

// ------------------------------------------------------------- Cholesky
// Right-looking Cholesky A = L L^H of a Hermitian k x k matrix (k <= 64) in one CTA: after each
// pivot the trailing matrix gets a rank-one update, one element per thread, so the dependency
// chain is k steps of one fused multiply-add (FP64 latency, not dot products, sets the time).
// Column j is dead when its pivot is below tol times a reference: the j-th diagonal entry of
// `ref` when given (the squared norm of the raw column), else the largest diagonal entry of A.
// A dead column gets L[j][j] = 1 and a zero sub-column (and, with zero_row, a zero row).
__global__ void chol_kernel(const zd *__restrict__ A, int lda, int k, zd *__restrict__ Lout, int ldl, double tol,
                            int zero_row, int *dead, int *status, int flag_rank, const zd *__restrict__ ref, int ldref) {
  extern __shared__ zd Ls[];   // k x k, ld = k (lower part used)
  __shared__ double maxdiag, piv;
  __shared__ int isdead, ndead;
  const int t = threadIdx.x, nt = blockDim.x;
  for (int e = t; e < k * k; e += nt) {
    const int i = e % k, j = e / k;
    Ls[e] = (i >= j) ? A[(size_t)j * lda + i] : mk<double>(0, 0);
  }
  if (t < 32) {
    double m = 0.0;
    for (int i = t; i < k; i += 32) m = fmax(m, A[(size_t)i * lda + i].re);
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (t == 0) { maxdiag = m; ndead = 0; }
  }
  __syncthreads();
  for (int j = 0; j < k; ++j) {
    if (t == 0) {
      piv = Ls[j * k + j].re;
      const double refj = ref ? ref[(size_t)j * ldref + j].re : maxdiag;
      isdead = !(piv > tol * refj) || !isfinite(piv) || !(refj > 0.0);
      if (isdead) ndead++;
      if (dead) dead[j] = isdead;
    }
    __syncthreads();
    const double d = isdead ? 1.0 : sqrt(piv);
    const double inv = 1.0 / d;
    for (int i = j + t; i < k; i += nt) {
      if (isdead) Ls[j * k + i] = (i == j) ? mk<double>(1, 0) : mk<double>(0, 0);
      else Ls[j * k + i] = (i == j) ? mk<double>(d, 0) : mk<double>(Ls[j * k + i].re * inv, Ls[j * k + i].im * inv);
    }
    if (isdead && zero_row)
      for (int m = t; m < j; m += nt) Ls[m * k + j] = mk<double>(0, 0);
    __syncthreads();
    if (!isdead) {
      // trailing update: A[i][c] -= L[i][j] conj(L[c][j]) for j < c <= i
      const int nrem = k - j - 1;
      for (int e = t; e < nrem * nrem; e += nt) {
        const int i = j + 1 + e % nrem, cc = j + 1 + e / nrem;
        if (i >= cc) Ls[cc * k + i] = Ls[cc * k + i] - Ls[j * k + i] * conj(Ls[j * k + cc]);
      }
    }
    __syncthreads();
  }
  for (int e = t; e < k * k; e += nt) {
    const int i = e % k, j = e / k;
    Lout[(size_t)j * ldl + i] = (i >= j) ? Ls[e] : mk<double>(0, 0);
  }
  if (t == 0 && ndead > 0 && flag_rank && status) atomicOr(status, ST_RANK);
}

void sm_chol(const zd *A, int lda, int k, zd *L, int ldl, double tol, int zero_row, int *dead, int *status,
             int flag_rank, cudaStream_t st, const zd *ref, int ldref) {
  ::lrei::count_launch();
  chol_kernel<<<1, 256, (size_t)k * k * sizeof(zd), st>>>(A, lda, k, L, ldl, tol, zero_row, dead, status, flag_rank,
                                                          ref, ldref);
}

// --------------------------------------------------------------- Jacobi
template <typename T>
struct Rot {
  T c;
  cx<T> s;
  int p, q;
};

// One CTA.  A (k x k Hermitian, FP64 input) -> eigenpairs in working precision T.
template <typename T, int NT>
__global__ void __launch_bounds__(NT) jacobi_kernel(const zd *__restrict__ Ain, int lda, int k, zd *__restrict__ Uout,
                                                     int ldu, double *__restrict__ wout, cx<T> *Ug, int max_sweeps,
                                                     double tol, int *status, cx<float> *__restrict__ Uf, int nout) {
  extern __shared__ __align__(16) unsigned char sm[];
  const int kp = k + (k & 1);
  const int np = kp / 2;
  cx<T> *A = reinterpret_cast<cx<T> *>(sm);
  Rot<T> *rot = reinterpret_cast<Rot<T> *>(A + (size_t)kp * kp);
  cx<T> *U = Ug ? Ug : reinterpret_cast<cx<T> *>(rot + np);
  __shared__ double red[32];
  __shared__ int done;
  const int t = threadIdx.x, nt = blockDim.x;
  for (int e = t; e < kp * kp; e += nt) {
    const int i = e % kp, j = e / kp;
    if (i < k && j < k) {
      zd v = Ain[(size_t)j * lda + i];
      A[e] = mk<T>((T)v.re, (T)v.im);
    } else {
      A[e] = mk<T>(0, 0);
    }
    U[e] = mk<T>(i == j ? 1 : 0, 0);
  }
  __syncthreads();
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    // convergence test: off-diagonal vs total Frobenius norm (summed in T per thread: the FP32
    // solver's test needs no FP64 arithmetic, which is slow on this part)
    T offt = 0, tott = 0;
    for (int e = t; e < kp * kp; e += nt) {
      const int i = e % kp, j = e / kp;
      const T v = norm2(A[e]);
      tott += v;
      if (i != j) offt += v;
    }
    double off = (double)offt, tot = (double)tott;
    for (int o = 16; o > 0; o >>= 1) {
      off += __shfl_xor_sync(0xffffffffu, off, o);
      tot += __shfl_xor_sync(0xffffffffu, tot, o);
    }
    if ((t & 31) == 0) red[t >> 5] = off;
    __syncthreads();
    if (t == 0) {
      double s = 0.0;
      for (int w = 0; w < (nt + 31) / 32; ++w) s += red[w];
      off = s;
    }
    __syncthreads();
    if ((t & 31) == 0) red[t >> 5] = tot;
    __syncthreads();
    if (t == 0) {
      double s = 0.0;
      for (int w = 0; w < (nt + 31) / 32; ++w) s += red[w];
      done = (off <= tol * tol * s) || !(s == s);
    }
    __syncthreads();
    if (done) break;
    for (int round = 0; round < kp - 1; ++round) {
      for (int pi = t; pi < np; pi += nt) {
        // circle-method tournament: position 0 fixed, positions 1..kp-1 rotate
        auto player = [&](int pos) { return pos == 0 ? 0 : 1 + ((pos - 1 + round) % (kp - 1)); };
        int p = player(pi), q = player(kp - 1 - pi);
        if (p > q) { const int tmp = p; p = q; q = tmp; }
        const cx<T> b = A[(size_t)q * kp + p];
        const T ab = sqrt(b.re * b.re + b.im * b.im);
        const T a = A[(size_t)p * kp + p].re, d = A[(size_t)q * kp + q].re;
        Rot<T> R;
        R.p = p;
        R.q = q;
        const T small = (sizeof(T) == 4) ? (T)1e-30 : (T)1e-280;
        if (ab <= small) {
          R.c = 1;
          R.s = mk<T>(0, 0);
        } else {
          const T tau = (d - a) / (2 * ab);
          T tt;
          if (fabs((double)tau) > ((sizeof(T) == 4) ? 1e7 : 1e150)) tt = (T)0.5 / tau;
          else tt = (tau >= 0 ? (T)1 : (T)-1) / (fabs(tau) + sqrt((T)1 + tau * tau));
          const T c = (T)1 / sqrt((T)1 + tt * tt);
          R.c = c;
          R.s = mk<T>(tt * c * b.re / ab, tt * c * b.im / ab);
        }
        rot[pi] = R;
      }
      __syncthreads();
      // A <- J^H A J on 2x2 blocks (pairs a, b): every element is read and written once;
      // U <- U J on the pairs' columns.  J = [[c, s], [-conj(s), c]] on (p, q).
      for (int e = t; e < np * np + np * kp; e += nt) {
        if (e < np * np) {
          const Rot<T> Ra = rot[e % np], Rb = rot[e / np];
          cx<T> *a0 = A + (size_t)Rb.p * kp, *a1 = A + (size_t)Rb.q * kp;
          const cx<T> x00 = a0[Ra.p], x10 = a0[Ra.q], x01 = a1[Ra.p], x11 = a1[Ra.q];
          // Y = X J_b
          const cx<T> y00 = Rb.c * x00 - conj(Rb.s) * x01, y01 = Rb.s * x00 + Rb.c * x01;
          const cx<T> y10 = Rb.c * x10 - conj(Rb.s) * x11, y11 = Rb.s * x10 + Rb.c * x11;
          // X' = J_a^H Y
          a0[Ra.p] = Ra.c * y00 - Ra.s * y10;
          a1[Ra.p] = Ra.c * y01 - Ra.s * y11;
          a0[Ra.q] = conj(Ra.s) * y00 + Ra.c * y10;
          a1[Ra.q] = conj(Ra.s) * y01 + Ra.c * y11;
        } else {
          const int f = e - np * np;
          const Rot<T> R = rot[f / kp];
          const int i = f % kp;
          if (R.s.re == 0 && R.s.im == 0) continue;
          cx<T> *up = U + (size_t)R.p * kp, *uq = U + (size_t)R.q * kp;
          const cx<T> ux = up[i], uy = uq[i];
          up[i] = R.c * ux - conj(R.s) * uy;
          uq[i] = R.s * ux + R.c * uy;
        }
      }
      __syncthreads();
    }
    if (sweep == max_sweeps - 1 && t == 0 && status) atomicOr(status, ST_EIG_NOCONV);
    if (t == 0) atomicAdd(&g_jacobi_counters[sizeof(T) == 4 ? 1 : 3], 1ull);
  }
  if (t == 0) atomicAdd(&g_jacobi_counters[sizeof(T) == 4 ? 0 : 2], 1ull);
  // sort eigenvalues decreasing (ties by index) and write out
  for (int i = t; i < k; i += nt) {
    const T wi = A[(size_t)i * kp + i].re;
    int rank = 0;
    for (int j = 0; j < k; ++j) {
      const T wj = A[(size_t)j * kp + j].re;
      rank += (wj > wi) || (wj == wi && j < i);
    }
    wout[rank] = (double)wi;
    if (rank < nout)
      for (int row = 0; row < k; ++row) {
        const cx<T> u = U[(size_t)i * kp + row];
        Uout[(size_t)rank * ldu + row] = mk<double>((double)u.re, (double)u.im);
      }
    if (Uf)
      for (int row = 0; row < k; ++row) {
        const cx<T> u = U[(size_t)i * kp + row];
        Uf[(size_t)rank * k + row] = mk<float>((float)u.re, (float)u.im);
      }
  }
}

template <typename T>
static size_t jacobi_smem(int k, bool u_in_smem) {
  const int kp = k + (k & 1);
  return (size_t)kp * kp * sizeof(cx<T>) * (u_in_smem ? 2 : 1) + (size_t)(kp / 2) * sizeof(Rot<T>) + 64;
}

size_t sm_jacobi_scratch_bytes(int k) {
  const int kp = k + (k & 1);
  return (size_t)kp * kp * sizeof(cx<double>);
}

void sm_jacobi(bool fp64, const zd *A, int lda, int k, zd *U, int ldu, double *w, void *scratch, int max_sweeps,
               double tol, int *status, cudaStream_t st, void *Uf32, int nout) {
  const size_t lim = 200 * 1024;
  if (nout < 0 || nout > k) nout = k;
  if (fp64) {
    const bool in_smem = jacobi_smem<double>(k, true) <= lim;
    const size_t bytes = jacobi_smem<double>(k, in_smem);
    ::lrei::count_launch(); jacobi_kernel<double, 512><<<1, 512, bytes, st>>>(A, lda, k, U, ldu, w, in_smem ? nullptr : (cx<double> *)scratch,
                                                 max_sweeps, tol, status, reinterpret_cast<cx<float> *>(Uf32), nout);
  } else {
    const bool in_smem = jacobi_smem<float>(k, true) <= lim;
    const size_t bytes = jacobi_smem<float>(k, in_smem);
    ::lrei::count_launch();
    jacobi_kernel<float, 1024><<<1, 1024, bytes, st>>>(A, lda, k, U, ldu, w, in_smem ? nullptr : (cx<float> *)scratch,
                                                       max_sweeps, tol, status, reinterpret_cast<cx<float> *>(Uf32), nout);
  }
}

// ------------------------------------------------------------ top-r eig
// Block-Newton correction of the top-r invariant subspace (one column per CTA):
// X_ij = (Ur^H R)_ij / (d_j - w_{r+i}), with R = M E - E (E^H M E) the residual of the current
// basis E, d_j = (E^H M E)_jj its Rayleigh quotients, and Ur, w_{r+i} the FP32 eigenpairs of the
// other k - r eigenvalues.  Because the correction is driven by the residual (which vanishes
// exactly on the invariant subspace), repeated passes converge to FP64 accuracy even though Ur
// is only FP32-accurate.
// One CTA per column j of E; every step below is local to that column once W1 = M E is known:
//   a = E^H W1[:, j],  R = W1[:, j] - E a                  (FP64: the residual is a small difference)
//   X_i = (Ur^H R)_i / (a_j - w_{r+i}),  D = Ur X           (FP32: only the correction's leading digits
//   Enew[:, j] = E[:, j] + D - E (E^H D)                      matter; Ur is FP32-accurate anyway)
// Ur is read from the FP32 eigenvectors (k x k, ld k, column r + i).  E is read by all CTAs, so the
// result goes to a separate array.  FP64 work is kept to the residual: on this part FP64
// (including conversions) runs at 1/58 of the FP32 rate.
__global__ void __launch_bounds__(256) newton_chain_kernel(const zd *__restrict__ W1, int ldw, const zd *__restrict__ E,
                                                           int lde, const cx<float> *__restrict__ Uf,
                                                           const double *__restrict__ w, int k, int r,
                                                           zd *__restrict__ Enew, int ldn) {
  extern __shared__ __align__(16) unsigned char nsm[];
  zd *w1 = reinterpret_cast<zd *>(nsm);                    // k
  zd *av = w1 + k;                                          // r
  cx<float> *rf = reinterpret_cast<cx<float> *>(av + r);    // k: residual (FP32)
  cx<float> *x = rf + k;                                    // k - r
  cx<float> *d2 = x + k;                                    // k
  cx<float> *ef = d2 + k;                                   // k x r: E in FP32 (for the projection)
  cx<float> *g1 = ef + (size_t)k * r;                       // r
  const int j = blockIdx.x, t = threadIdx.x, lane = t & 31, wp = t >> 5, nw = blockDim.x >> 5;
  for (int p = t; p < k; p += blockDim.x) w1[p] = W1[(size_t)j * ldw + p];
  __syncthreads();
  for (int i = wp; i < r; i += nw) {          // a = E^H w1
    zd s = mk<double>(0, 0);
    for (int p = lane; p < k; p += 32) fmac_(s, E[(size_t)i * lde + p], w1[p]);
    s = warp_sum(s);
    if (lane == 0) av[i] = s;
  }
  __syncthreads();
  for (int p = t; p < k; p += blockDim.x) {   // R = w1 - E a; E to FP32 for the projection below
    zd s = w1[p];
    for (int i = 0; i < r; ++i) {
      const zd e = E[(size_t)i * lde + p];
      s = s - e * av[i];
      ef[(size_t)i * k + p] = cvt<float>(e);
    }
    rf[p] = cvt<float>(s);
  }
  __syncthreads();
  const double dj = av[j].re;
  for (int i = wp; i < k - r; i += nw) {      // X = (Ur^H R) ./ (d_j - w)
    cx<float> s = mk<float>(0.f, 0.f);
    const cx<float> *u = Uf + (size_t)(r + i) * k;
    for (int p = lane; p < k; p += 32) fmac_(s, u[p], rf[p]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      s.re += __shfl_xor_sync(0xffffffffu, s.re, o);
      s.im += __shfl_xor_sync(0xffffffffu, s.im, o);
    }
    if (lane == 0) {
      const float den = (float)(dj - w[r + i]);
      x[i] = (fabsf(den) > 1e-30f) ? mk<float>(s.re / den, s.im / den) : mk<float>(0.f, 0.f);
    }
  }
  __syncthreads();
  for (int p = t; p < k; p += blockDim.x) {   // D = Ur X
    cx<float> s = mk<float>(0.f, 0.f);
#pragma unroll 8
    for (int i = 0; i < k - r; ++i) fma_(s, Uf[(size_t)(r + i) * k + p], x[i]);
    d2[p] = s;
  }
  __syncthreads();
  for (int i = wp; i < r; i += nw) {          // g = E^H D
    cx<float> s = mk<float>(0.f, 0.f);
    for (int p = lane; p < k; p += 32) fmac_(s, ef[(size_t)i * k + p], d2[p]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      s.re += __shfl_xor_sync(0xffffffffu, s.re, o);
      s.im += __shfl_xor_sync(0xffffffffu, s.im, o);
    }
    if (lane == 0) g1[i] = s;
  }
  __syncthreads();
  for (int p = t; p < k; p += blockDim.x) {   // Enew = E + D - E g
    cx<float> s = d2[p];
    for (int i = 0; i < r; ++i) s = s - ef[(size_t)i * k + p] * g1[i];
    const zd e = E[(size_t)j * lde + p];
    Enew[(size_t)j * ldn + p] = mk<double>(e.re + (double)s.re, e.im + (double)s.im);
  }
}

size_t newton_chain_smem(int k, int r) {
  return (size_t)(k + r) * sizeof(zd) + (size_t)(3 * k + (size_t)k * r + r) * sizeof(cx<float>) + 64;
}

// T = (15/8) I - (5/4) G + (3/8) G^2 for G = E^H E = I + d: then E T = E (E^H E)^{-1/2} + O(d^3),
// the orthonormal polar factor of E (same span).  One CTA per column j; the sum over m of
// (G^2)_{ij} is split over the CTA's threads and combined in shared memory.
__global__ void __launch_bounds__(256) polar_t_kernel(const zd *__restrict__ G, int ldg, int r, zd *__restrict__ T,
                                                      int ldt) {
  __shared__ zd part[256];
  const int j = blockIdx.x, t = threadIdx.x;
  const int i = t % r, q = t / r, nq = blockDim.x / r;
  zd s = mk<double>(0, 0);
  if (q < nq)
    for (int m = q; m < r; m += nq) fma_(s, G[(size_t)m * ldg + i], G[(size_t)j * ldg + m]);
  part[t] = s;
  __syncthreads();
  if (t < r) {
    zd g2 = mk<double>(0, 0);
    for (int u = 0; u < nq; ++u) g2 = g2 + part[u * r + t];
    const zd gij = G[(size_t)j * ldg + t];
    zd v = mk<double>(-1.25 * gij.re + 0.375 * g2.re, -1.25 * gij.im + 0.375 * g2.im);
    if (t == j) v.re += 1.875;
    T[(size_t)j * ldt + t] = v;
  }
}

// Residual check ||M Y - Y diag(mu)||_max <= tol * max|mu|, else flag.
__global__ void eig_check_kernel(const zd *__restrict__ MY, int ldmy, const zd *__restrict__ Y, int ldy,
                                 const double *__restrict__ mu, int k, int r, double tol, int *status) {
  __shared__ double red[8];
  double m = 0.0, mm = 0.0;
  for (int e = threadIdx.x; e < k * r; e += blockDim.x) {
    const int i = e % k, j = e / k;
    const zd a = MY[(size_t)j * ldmy + i], y = Y[(size_t)j * ldy + i];
    const double rr = a.re - mu[j] * y.re, ri = a.im - mu[j] * y.im;
    m = fmax(m, sqrt(rr * rr + ri * ri));
    if (!isfinite(a.re) || !isfinite(a.im)) m = 1e300;
  }
  for (int j = threadIdx.x; j < r; j += blockDim.x) mm = fmax(mm, fabs(mu[j]));
  for (int o = 16; o > 0; o >>= 1) {
    m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    mm = fmax(mm, __shfl_xor_sync(0xffffffffu, mm, o));
  }
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0;
    for (int i = 0; i < (int)(blockDim.x + 31) / 32; ++i) a = fmax(a, red[i]);
    if (!(a <= tol * fmax(mm, 1e-300))) atomicOr(status, ST_EIG_RESID);
  }
}

size_t sm_eig_ws_bytes(int kmax, int rmax) {
  size_t z = sizeof(zd);
  size_t b = 0;
  b += (size_t)kmax * 8;             // w
  b += 4 * (size_t)kmax * rmax * z;  // W1, A21, E1, W2
  b += 4 * (size_t)rmax * rmax * z;  // G1, L1, Ar, Wr
  b += sm_jacobi_scratch_bytes(kmax);
  b += (size_t)rmax * rmax * z + (size_t)kmax * rmax * z;
  b += (size_t)kmax * kmax * sizeof(cx<float>) + 256;   // FP32 eigenvectors
  return b + 4096;
}

void sm_eig_topr(const zd *M, int ldm, int k, int r, zd *Y, int ldy, double *mu, void *ws, int *status,
                 cudaStream_t st, int max_sweeps) {
  unsigned char *p = reinterpret_cast<unsigned char *>(ws);
  auto take = [&](size_t bytes) { unsigned char *q = p; p += (bytes + 255) & ~(size_t)255; return q; };
  double *w = (double *)take((size_t)k * 8);
  zd *W1 = (zd *)take((size_t)k * r * sizeof(zd));
  zd *A21 = (zd *)take((size_t)k * r * sizeof(zd));
  zd *E1 = (zd *)take((size_t)k * r * sizeof(zd));
  zd *W2 = (zd *)take((size_t)k * r * sizeof(zd));
  zd *G1 = (zd *)take((size_t)r * r * sizeof(zd));
  zd *L1 = (zd *)take((size_t)r * r * sizeof(zd));
  zd *Ar = (zd *)take((size_t)r * r * sizeof(zd));
  zd *Wr = (zd *)take((size_t)r * r * sizeof(zd));
  void *jscratch = take(sm_jacobi_scratch_bytes(k));
  zd *Inv = (zd *)take((size_t)r * r * sizeof(zd));
  zd *Xc = (zd *)take((size_t)k * r * sizeof(zd));
  cx<float> *U32 = (cx<float> *)take((size_t)k * k * sizeof(cx<float>));
  const zd one = mk<double>(1, 0), zero = mk<double>(0, 0);
  (void)Inv; (void)Xc; (void)A21; (void)L1;
  // 1. FP32 eigendecomposition of the whole k x k matrix: all eigenvectors in FP32 (U32), the
  //    top r also in FP64 (E1), eigenvalues in FP64 (w)
  sm_jacobi(false, M, ldm, k, E1, k, w, jscratch, 12, 1e-5, nullptr, st, U32, r);
  // 2.-3. block-Newton corrections of the top-r invariant subspace, each followed by the polar
  // re-orthonormalisation E <- E T, T = (E^H E)^{-1/2} to third order (multi-CTA FP64 gemms)
  const int passes = (k > r) ? 4 : 1;
  for (int it = 0; it < passes; ++it) {
    zd *Ecur = E1;
    if (k > r) {
      sm_gemm('N', 'N', k, r, k, one, M, ldm, E1, k, zero, W1, k, st);           // W1 = M E
      ::lrei::count_launch();
      newton_chain_kernel<<<r, 256, newton_chain_smem(k, r), st>>>(W1, k, E1, k, U32, w, k, r, W2, k);
      Ecur = W2;
    }
    sm_gemm('C', 'N', r, r, k, one, Ecur, k, Ecur, k, zero, G1, r, st);         // G = E^H E
    ::lrei::count_launch();
    polar_t_kernel<<<r, 256, 0, st>>>(G1, r, r, Ar, r);                        // T
    sm_gemm('N', 'N', k, r, r, one, Ecur, k, Ar, r, zero, (Ecur == E1) ? W2 : E1, k, st);
    if (Ecur == E1) sm_copy(W2, k, k, r, E1, k, st);
  }
  // 4. Rayleigh-Ritz on span(E1) in FP64
  sm_gemm('N', 'N', k, r, k, one, M, ldm, E1, k, zero, W2, k, st);
  sm_gemm('C', 'N', r, r, k, one, E1, k, W2, k, zero, Ar, r, st);
  sm_hermitize(Ar, r, r, st);
  sm_jacobi(true, Ar, r, r, Wr, r, mu, jscratch, max_sweeps, 1e-14, status, st);
  sm_gemm('N', 'N', k, r, r, one, E1, k, Wr, r, zero, Y, ldy, st);
  // 5. residual check of the returned pairs
  sm_gemm('N', 'N', k, r, k, one, M, ldm, Y, ldy, zero, W1, k, st);
  ::lrei::count_launch(); eig_check_kernel<<<1, 256, 0, st>>>(W1, k, Y, ldy, mu, k, r, 1e-9, status);
}

// ------------------------------------------------------------ elementwise
__global__ void copy_kernel(const zd *A, int lda, int M, int N, zd *B, int ldb, int mode) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < M * N; e += gridDim.x * blockDim.x) {
    const int i = e % M, j = e / M;
    if (mode == 0) B[(size_t)j * ldb + i] = A[(size_t)j * lda + i];
    else if (mode == 1) B[(size_t)i * ldb + j] = conj(A[(size_t)j * lda + i]);   // B = A^H (N x M)
    else if (mode == 2) B[(size_t)j * ldb + i] = mk<double>(0, 0);
    else B[(size_t)j * ldb + i] = mk<double>(i == j ? 1 : 0, 0);
  }
}
static int grid_for(long long n) { long long g = (n + 255) / 256; return (int)(g < 1 ? 1 : (g > 1024 ? 1024 : g)); }
void sm_copy(const zd *A, int lda, int M, int N, zd *B, int ldb, cudaStream_t st) {
  ::lrei::count_launch(); copy_kernel<<<grid_for((long long)M * N), 256, 0, st>>>(A, lda, M, N, B, ldb, 0);
}
void sm_conj_transpose(const zd *A, int lda, int M, int N, zd *B, int ldb, cudaStream_t st) {
  ::lrei::count_launch(); copy_kernel<<<grid_for((long long)M * N), 256, 0, st>>>(A, lda, M, N, B, ldb, 1);
}
void sm_zero(zd *A, int lda, int M, int N, cudaStream_t st) {
  ::lrei::count_launch(); copy_kernel<<<grid_for((long long)M * N), 256, 0, st>>>(nullptr, 0, M, N, A, lda, 2);
}
void sm_set_identity(zd *A, int lda, int M, int N, cudaStream_t st) {
  ::lrei::count_launch(); copy_kernel<<<grid_for((long long)M * N), 256, 0, st>>>(nullptr, 0, M, N, A, lda, 3);
}

__global__ void hermitize_kernel(zd *A, int lda, int k) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < k * k; e += gridDim.x * blockDim.x) {
    const int i = e % k, j = e / k;
    if (i > j) continue;
    const zd a = A[(size_t)j * lda + i], b = A[(size_t)i * lda + j];
    const zd h = mk<double>(0.5 * (a.re + b.re), 0.5 * (a.im - b.im));
    A[(size_t)j * lda + i] = h;
    A[(size_t)i * lda + j] = conj(h);
    if (i == j) A[(size_t)j * lda + i] = mk<double>(h.re, 0);
  }
}
void sm_hermitize(zd *A, int lda, int k, cudaStream_t st) { ::lrei::count_launch(); hermitize_kernel<<<grid_for((long long)k * k), 256, 0, st>>>(A, lda, k); }

__global__ void scale_kernel(zd *A, int lda, int M, int N, double s) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < M * N; e += gridDim.x * blockDim.x) {
    const int i = e % M, j = e / M;
    A[(size_t)j * lda + i] = s * A[(size_t)j * lda + i];
  }
}
void sm_scale_cols(zd *A, int lda, int M, int N, double s, cudaStream_t st) {
  ::lrei::count_launch(); scale_kernel<<<grid_for((long long)M * N), 256, 0, st>>>(A, lda, M, N, s);
}

// Columns k..k+r-1 of the Hermitian Gram G from the measured block R ((k + r) x r) and their
// mirror rows.  Inside the new r x r diagonal block only R's upper triangle is used (the lower one
// is its conjugate), so every entry of G has exactly one writer: R's two triangles differ in the
// last bit, and two threads storing both into one entry would make the result depend on which
// store lands last.
__global__ void store_gram_cols_kernel(const zd *R, int ldr, int k, int r, zd *G, int ldg) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < (k + r) * r; e += gridDim.x * blockDim.x) {
    const int i = e % (k + r), j = e / (k + r);
    if (i > k + j) continue;   // below the diagonal of the new block: written as the mirror of (k + j, i)
    const zd v = R[(size_t)j * ldr + i];
    if (i == k + j) {
      G[(size_t)(k + j) * ldg + i] = mk<double>(v.re, 0);
    } else {
      G[(size_t)(k + j) * ldg + i] = v;
      G[(size_t)i * ldg + (k + j)] = conj(v);
    }
  }
}
void sm_store_gram_cols(const zd *R, int ldr, int k, int r, zd *G, int ldg, cudaStream_t st) {
  ::lrei::count_launch(); store_gram_cols_kernel<<<grid_for((long long)(k + r) * r), 256, 0, st>>>(R, ldr, k, r, G, ldg);
}

}  // namespace lrei

namespace lrei {
int sm_init() {
  const int lim = 210 * 1024;
  cudaFuncSetAttribute(trsv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  cudaError_t a = cudaFuncSetAttribute(jacobi_kernel<double, 512>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  cudaError_t b = cudaFuncSetAttribute(jacobi_kernel<float, 1024>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  cudaError_t c = cudaFuncSetAttribute(newton_chain_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  return (a == cudaSuccess && b == cudaSuccess && c == cudaSuccess) ? 0 : -1;
}
}  // namespace lrei

namespace lrei {
int sm_read_counters(unsigned long long *out) {
  return cudaMemcpyFromSymbol(out, g_jacobi_counters, sizeof(unsigned long long) * 4) == cudaSuccess ? 0 : -1;
}
}  // namespace lrei
