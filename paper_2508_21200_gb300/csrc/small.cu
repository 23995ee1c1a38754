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

namespace lrei {

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
    gemm_warp_kernel<<<(int)((threads + 127) / 128), 128, 0, st>>>(opA, opB, M, N, K, alpha, A, lda, B, ldb, beta, C,
                                                                    ldc);
  } else {
    gemm_thread_kernel<<<(M * N + 63) / 64, 64, 0, st>>>(opA, opB, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc);
  }
}

// ------------------------------------------------------- triangular solves
__global__ void trsv_kernel(char op, const zd *__restrict__ L, int ldl, int k, zd *__restrict__ B, int ldb) {
  extern __shared__ zd xs[];
  zd *x = B + (size_t)blockIdx.x * ldb;
  const int lane = threadIdx.x;
  for (int i = lane; i < k; i += 32) xs[i] = x[i];
  __syncwarp();
  if (op == 'N') {
    for (int i = 0; i < k; ++i) {
      zd s = mk<double>(0, 0);
      for (int m = lane; m < i; m += 32) fma_(s, L[(size_t)m * ldl + i], xs[m]);
      s = warp_sum(s);
      if (lane == 0) {
        const zd d = L[(size_t)i * ldl + i];
        xs[i] = (d.re == 0.0 && d.im == 0.0) ? mk<double>(0, 0) : zdiv(xs[i] - s, d);
      }
      __syncwarp();
    }
  } else {
    for (int i = k - 1; i >= 0; --i) {
      zd s = mk<double>(0, 0);
      for (int m = i + 1 + lane; m < k; m += 32) fmac_(s, L[(size_t)i * ldl + m], xs[m]);
      s = warp_sum(s);
      if (lane == 0) {
        const zd d = conj(L[(size_t)i * ldl + i]);
        xs[i] = (d.re == 0.0 && d.im == 0.0) ? mk<double>(0, 0) : zdiv(xs[i] - s, d);
      }
      __syncwarp();
    }
  }
  for (int i = lane; i < k; i += 32) x[i] = xs[i];
}

void sm_trsv(char op, const zd *L, int ldl, int k, zd *B, int ldb, int ncols, cudaStream_t st) {
  if (ncols <= 0 || k <= 0) return;
  trsv_kernel<<<ncols, 32, k * sizeof(zd), st>>>(op, L, ldl, k, B, ldb);
}

// X <- X (L^H)^{-1}: row y solves y L^H = x, i.e. y_j = (x_j - sum_{m<j} y_m conj(L[j][m])) / L[j][j].
__global__ void rtrsm_lh_kernel(zd *X, int ldx, int nrows, const zd *__restrict__ L, int ldl, int k) {
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= nrows) return;
  for (int j = 0; j < k; ++j) {
    zd s = X[(size_t)j * ldx + row];
    for (int m = 0; m < j; ++m) {
      const zd l = conj(L[(size_t)m * ldl + j]);
      const zd y = X[(size_t)m * ldx + row];
      s = s - y * l;
    }
    const zd d = conj(L[(size_t)j * ldl + j]);
    X[(size_t)j * ldx + row] = (d.re == 0.0 && d.im == 0.0) ? mk<double>(0, 0) : zdiv(s, d);
  }
}

void sm_rtrsm_lh(zd *X, int ldx, int nrows, const zd *L, int ldl, int k, cudaStream_t st) {
  if (nrows <= 0) return;
  rtrsm_lh_kernel<<<(nrows + 63) / 64, 64, 0, st>>>(X, ldx, nrows, L, ldl, k);
}

// ------------------------------------------------------------- Cholesky
__global__ void chol_kernel(const zd *__restrict__ A, int lda, int k, zd *__restrict__ Lout, int ldl, double tol,
                            int zero_row, int *dead, int *status, int flag_rank) {
  extern __shared__ zd Ls[];   // k x k, ld = k
  __shared__ double maxdiag;
  __shared__ int ndead;
  const int t = threadIdx.x;
  for (int e = t; e < k * k; e += blockDim.x) {
    const int i = e % k, j = e / k;
    Ls[e] = (i >= j) ? A[(size_t)j * lda + i] : mk<double>(0, 0);
  }
  if (t == 0) {
    double m = 0.0;
    for (int i = 0; i < k; ++i) m = fmax(m, A[(size_t)i * lda + i].re);
    maxdiag = m;
    ndead = 0;
  }
  __syncthreads();
  for (int j = 0; j < k; ++j) {
    // v_i = A[i][j] - sum_{m<j} L[i][m] conj(L[j][m]) for i >= j
    zd v = mk<double>(0, 0);
    const int i = j + t;
    if (i < k) {
      v = Ls[j * k + i];
      for (int m = 0; m < j; ++m) v = v - Ls[m * k + i] * conj(Ls[m * k + j]);
    }
    __syncthreads();
    __shared__ double piv;
    __shared__ int isdead;
    if (t == 0) {
      piv = v.re;
      isdead = !(piv > tol * maxdiag) || !isfinite(piv) || maxdiag <= 0.0;
      if (isdead) ndead++;
    }
    __syncthreads();
    if (i < k) {
      if (isdead) {
        Ls[j * k + i] = (i == j) ? mk<double>(1, 0) : mk<double>(0, 0);
      } else {
        const double d = sqrt(piv);
        Ls[j * k + i] = (i == j) ? mk<double>(d, 0) : zdiv_real(v, d);
      }
    }
    if (isdead && zero_row && t < j) Ls[t * k + j] = mk<double>(0, 0);
    if (dead && t == 0) dead[j] = isdead;
    __syncthreads();
  }
  for (int e = t; e < k * k; e += blockDim.x) {
    const int i = e % k, j = e / k;
    Lout[(size_t)j * ldl + i] = Ls[e];
  }
  if (t == 0 && ndead > 0 && flag_rank && status) atomicOr(status, ST_RANK);
}

void sm_chol(const zd *A, int lda, int k, zd *L, int ldl, double tol, int zero_row, int *dead, int *status,
             int flag_rank, cudaStream_t st) {
  chol_kernel<<<1, 64, (size_t)k * k * sizeof(zd), st>>>(A, lda, k, L, ldl, tol, zero_row, dead, status, flag_rank);
}

// --------------------------------------------------------------- Jacobi
template <typename T>
struct Rot {
  T c;
  cx<T> s;
  int p, q;
};

// One CTA.  A (k x k Hermitian, FP64 input) -> eigenpairs in working precision T.
template <typename T>
__global__ void __launch_bounds__(512) jacobi_kernel(const zd *__restrict__ Ain, int lda, int k, zd *__restrict__ Uout,
                                                     int ldu, double *__restrict__ wout, cx<T> *Ug, int max_sweeps,
                                                     double tol, int *status) {
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
    // convergence test: off-diagonal vs total Frobenius norm
    double off = 0.0, tot = 0.0;
    for (int e = t; e < kp * kp; e += nt) {
      const int i = e % kp, j = e / kp;
      const double v = (double)norm2(A[e]);
      tot += v;
      if (i != j) off += v;
    }
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
      // A <- A J and U <- U J (columns p, q), J = [[c, s], [-conj(s), c]]
      for (int e = t; e < np * kp; e += nt) {
        const Rot<T> R = rot[e / kp];
        const int i = e % kp;
        if (R.s.re == 0 && R.s.im == 0) continue;
        cx<T> *cp = A + (size_t)R.p * kp, *cq = A + (size_t)R.q * kp;
        const cx<T> x = cp[i], y = cq[i];
        cp[i] = R.c * x - conj(R.s) * y;
        cq[i] = R.s * x + R.c * y;
        cx<T> *up = U + (size_t)R.p * kp, *uq = U + (size_t)R.q * kp;
        const cx<T> ux = up[i], uy = uq[i];
        up[i] = R.c * ux - conj(R.s) * uy;
        uq[i] = R.s * ux + R.c * uy;
      }
      __syncthreads();
      // A <- J^H A (rows p, q)
      for (int e = t; e < np * kp; e += nt) {
        const Rot<T> R = rot[e / kp];
        const int i = e % kp;
        if (R.s.re == 0 && R.s.im == 0) continue;
        const cx<T> x = A[(size_t)i * kp + R.p], y = A[(size_t)i * kp + R.q];
        A[(size_t)i * kp + R.p] = R.c * x - R.s * y;
        A[(size_t)i * kp + R.q] = conj(R.s) * x + R.c * y;
      }
      __syncthreads();
    }
    if (sweep == max_sweeps - 1 && t == 0 && status) atomicOr(status, ST_EIG_NOCONV);
  }
  // sort eigenvalues decreasing (ties by index) and write out
  for (int i = t; i < k; i += nt) {
    const T wi = A[(size_t)i * kp + i].re;
    int rank = 0;
    for (int j = 0; j < k; ++j) {
      const T wj = A[(size_t)j * kp + j].re;
      rank += (wj > wi) || (wj == wi && j < i);
    }
    wout[rank] = (double)wi;
    for (int row = 0; row < k; ++row) {
      const cx<T> u = U[(size_t)i * kp + row];
      Uout[(size_t)rank * ldu + row] = mk<double>((double)u.re, (double)u.im);
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
               double tol, int *status, cudaStream_t st) {
  const size_t lim = 200 * 1024;
  if (fp64) {
    const bool in_smem = jacobi_smem<double>(k, true) <= lim;
    const size_t bytes = jacobi_smem<double>(k, in_smem);
    jacobi_kernel<double><<<1, 512, bytes, st>>>(A, lda, k, U, ldu, w, in_smem ? nullptr : (cx<double> *)scratch,
                                                 max_sweeps, tol, status);
  } else {
    const bool in_smem = jacobi_smem<float>(k, true) <= lim;
    const size_t bytes = jacobi_smem<float>(k, in_smem);
    jacobi_kernel<float><<<1, 512, bytes, st>>>(A, lda, k, U, ldu, w, in_smem ? nullptr : (cx<float> *)scratch,
                                                max_sweeps, tol, status);
  }
}

// ------------------------------------------------------------ top-r eig
// Block-Newton correction of the top-r invariant subspace (one column per CTA):
// X_ij = (Ur^H R)_ij / (d_j - w_{r+i}), with R = M E - E (E^H M E) the residual of the current
// basis E, d_j = (E^H M E)_jj its Rayleigh quotients, and Ur, w_{r+i} the FP32 eigenpairs of the
// other k - r eigenvalues.  Because the correction is driven by the residual (which vanishes
// exactly on the invariant subspace), repeated passes converge to FP64 accuracy even though Ur
// is only FP32-accurate.
__global__ void newton_scale_kernel(zd *__restrict__ A21, int lda21, const zd *__restrict__ A11, int r,
                                    const double *__restrict__ w, int k) {
  const int j = blockIdx.x;
  const double d = A11[(size_t)j * r + j].re;
  for (int i = threadIdx.x; i < k - r; i += blockDim.x) {
    const double den = d - w[r + i];
    const zd a = A21[(size_t)j * lda21 + i];
    A21[(size_t)j * lda21 + i] = (fabs(den) > 1e-300) ? mk<double>(a.re / den, a.im / den) : mk<double>(0, 0);
  }
}

__global__ void add_kernel(zd *__restrict__ E, int lde, const zd *__restrict__ D, int ldd, int k, int r) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < k * r; e += gridDim.x * blockDim.x) {
    const int i = e % k, j = e / k;
    E[(size_t)j * lde + i] = E[(size_t)j * lde + i] + D[(size_t)j * ldd + i];
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
  b += (size_t)kmax * kmax * z;      // U
  b += (size_t)kmax * 8;             // w
  b += 4 * (size_t)kmax * rmax * z;  // W1, A21, E1, W2
  b += 4 * (size_t)rmax * rmax * z;  // G1, L1, Ar, Wr
  b += sm_jacobi_scratch_bytes(kmax);
  return b + 1024;
}

void sm_eig_topr(const zd *M, int ldm, int k, int r, zd *Y, int ldy, double *mu, void *ws, int *status,
                 cudaStream_t st) {
  unsigned char *p = reinterpret_cast<unsigned char *>(ws);
  auto take = [&](size_t bytes) { unsigned char *q = p; p += (bytes + 255) & ~(size_t)255; return q; };
  zd *U = (zd *)take((size_t)k * k * sizeof(zd));
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
  const zd one = mk<double>(1, 0), zero = mk<double>(0, 0);
  // 1. FP32 eigendecomposition of the whole k x k matrix
  sm_jacobi(false, M, ldm, k, U, k, w, jscratch, 20, 1e-6, nullptr, st);
  // 2.-3. block-Newton corrections of the top-r invariant subspace, each followed by an
  // FP64 Cholesky-QR re-orthonormalisation of E1
  sm_copy(U, k, k, r, E1, k, st);
  const zd mone = mk<double>(-1, 0);
  const int passes = (k > r) ? 3 : 1;
  for (int it = 0; it < passes; ++it) {
    if (k > r) {
      sm_gemm('N', 'N', k, r, k, one, M, ldm, E1, k, zero, W1, k, st);           // W1 = M E
      sm_gemm('C', 'N', r, r, k, one, E1, k, W1, k, zero, Ar, r, st);            // A11 = E^H M E
      sm_gemm('N', 'N', k, r, r, mone, E1, k, Ar, r, one, W1, k, st);           // R = M E - E A11
      sm_gemm('C', 'N', k - r, r, k, one, U + (size_t)r * k, k, W1, k, zero, A21, k, st);   // Ur^H R
      newton_scale_kernel<<<r, 64, 0, st>>>(A21, k, Ar, r, w, k);               // X
      sm_gemm('N', 'N', k, r, k - r, one, U + (size_t)r * k, k, A21, k, zero, W2, k, st);    // D = Ur X
      sm_gemm('C', 'N', r, r, k, one, E1, k, W2, k, zero, G1, r, st);            // E^H D
      sm_gemm('N', 'N', k, r, r, mone, E1, k, G1, r, one, W2, k, st);           // D -= E (E^H D)
      add_kernel<<<8, 256, 0, st>>>(E1, k, W2, k, k, r);                        // E += D
    }
    sm_gemm('C', 'N', r, r, k, one, E1, k, E1, k, zero, G1, r, st);
    sm_chol(G1, r, r, L1, r, 0.0, 0, nullptr, nullptr, 0, st);
    sm_rtrsm_lh(E1, k, k, L1, r, r, st);
  }
  // 4. Rayleigh-Ritz on span(E1) in FP64
  sm_gemm('N', 'N', k, r, k, one, M, ldm, E1, k, zero, W2, k, st);
  sm_gemm('C', 'N', r, r, k, one, E1, k, W2, k, zero, Ar, r, st);
  sm_hermitize(Ar, r, r, st);
  sm_jacobi(true, Ar, r, r, Wr, r, mu, jscratch, 30, 1e-14, status, st);
  sm_gemm('N', 'N', k, r, r, one, E1, k, Wr, r, zero, Y, ldy, st);
  // 5. residual check of the returned pairs
  sm_gemm('N', 'N', k, r, k, one, M, ldm, Y, ldy, zero, W1, k, st);
  eig_check_kernel<<<1, 256, 0, st>>>(W1, k, Y, ldy, mu, k, r, 1e-9, status);
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
  copy_kernel<<<grid_for((long long)M * N), 256, 0, st>>>(A, lda, M, N, B, ldb, 0);
}
void sm_conj_transpose(const zd *A, int lda, int M, int N, zd *B, int ldb, cudaStream_t st) {
  copy_kernel<<<grid_for((long long)M * N), 256, 0, st>>>(A, lda, M, N, B, ldb, 1);
}
void sm_zero(zd *A, int lda, int M, int N, cudaStream_t st) {
  copy_kernel<<<grid_for((long long)M * N), 256, 0, st>>>(nullptr, 0, M, N, A, lda, 2);
}
void sm_set_identity(zd *A, int lda, int M, int N, cudaStream_t st) {
  copy_kernel<<<grid_for((long long)M * N), 256, 0, st>>>(nullptr, 0, M, N, A, lda, 3);
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
void sm_hermitize(zd *A, int lda, int k, cudaStream_t st) { hermitize_kernel<<<grid_for((long long)k * k), 256, 0, st>>>(A, lda, k); }

__global__ void scale_kernel(zd *A, int lda, int M, int N, double s) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < M * N; e += gridDim.x * blockDim.x) {
    const int i = e % M, j = e / M;
    A[(size_t)j * lda + i] = s * A[(size_t)j * lda + i];
  }
}
void sm_scale_cols(zd *A, int lda, int M, int N, double s, cudaStream_t st) {
  scale_kernel<<<grid_for((long long)M * N), 256, 0, st>>>(A, lda, M, N, s);
}

__global__ void store_gram_cols_kernel(const zd *R, int ldr, int k, int r, zd *G, int ldg) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < (k + r) * r; e += gridDim.x * blockDim.x) {
    const int i = e % (k + r), j = e / (k + r);
    const zd v = R[(size_t)j * ldr + i];
    G[(size_t)(k + j) * ldg + i] = v;
    G[(size_t)i * ldg + (k + j)] = conj(v);
    if (i == k + j) G[(size_t)(k + j) * ldg + i] = mk<double>(v.re, 0);
  }
}
void sm_store_gram_cols(const zd *R, int ldr, int k, int r, zd *G, int ldg, cudaStream_t st) {
  store_gram_cols_kernel<<<grid_for((long long)(k + r) * r), 256, 0, st>>>(R, ldr, k, r, G, ldg);
}

}  // namespace lrei

namespace lrei {
int sm_init() {
  const int lim = 210 * 1024;
  cudaError_t a = cudaFuncSetAttribute(jacobi_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  cudaError_t b = cudaFuncSetAttribute(jacobi_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  return (a == cudaSuccess && b == cudaSuccess) ? 0 : -1;
}
}  // namespace lrei
