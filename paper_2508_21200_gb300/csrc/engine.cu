// LREI step engine and C ABI (include/lrei.h).
//
// One RK_s step (paper Sec. 3.7, eqs. rk:sstageform, K-expand, rho-expand)
// is computed exactly as the paper's scheme, but organised for the GPU:
//
//  * Every stage matrix K_{j+1} = K_1 + h sum_l a_{j+1,l} (Z_l V_l^* + V_l W_l^*)
//    has its range inside span{V_1, W_1, ..., W_j}, and since W_l lies in
//    span{V_l, H V_l} and V_l in range(K_l), that span is the block Krylov
//    space K_{j+1}(H, V_1).  The engine therefore builds one block-Krylov
//    basis Q = [Q_0 = V_1, Q_1, ..., Q_s] per step (one H application and two
//    tall-skinny passes per block, measured Gram Gamma = Q^*Q) and evaluates
//    every stage -- G_j = V_j^* H V_j, the X blocks of eqs. X-blocks-sol /
//    X-blocks-sol-qLL, W_j, Z_j, the stage matrix and its partial
//    eigendecomposition -- in the (s+1) r dimensional coordinates of Q.
//  * The partial eigendecomposition of each K_{j+1} (the paper's IRLM on
//    g(x), eq. g-func) is an exact Rayleigh-Ritz on that space, so the result
//    equals the projected EI scheme up to rounding.
//  * The complement product W = V^ X12^* (Sec. 3.4-3.5) is applied in
//    coordinates as (I - V V^*) H V diag(conj c), which equals the Householder
//    form for any orthonormal complement.
//  * The new factor V_{k+1} = Q Y is formed in one pass at the end of the step.
// All small algebra is FP64; the N-length passes run in the context's
// precision.  A whole step is captured once in a CUDA graph and replayed.
#include "lrei.h"
#include "common.cuh"
#include "small.cuh"
#include "tsk.cuh"

#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

namespace lrei {

int cuda_fail(cudaError_t e, const char *what) {
  (void)what;
  if (e == cudaErrorMemoryAllocation) return LREI_ERR_OOM;
  return LREI_ERR_CUDA;
}

struct Tableau {
  int s;
  double a[4][4];
  double b[4];
};
// Butcher tableaus: forward Euler, the paper's RK2 example (a21 = 1, b = 1/2, 1/2),
// Kutta's third-order method, classic RK4.
static const Tableau kRK[4] = {
    {1, {{0}}, {1.0}},
    {2, {{0, 0}, {1.0, 0}}, {0.5, 0.5}},
    {3, {{0, 0, 0}, {0.5, 0, 0}, {-1.0, 2.0, 0}}, {1.0 / 6, 4.0 / 6, 1.0 / 6}},
    {4, {{0, 0, 0, 0}, {0.5, 0, 0, 0}, {0, 0.5, 0, 0}, {0, 0, 1.0, 0}}, {1.0 / 6, 2.0 / 6, 2.0 / 6, 1.0 / 6}},
};

// Adams-Bashforth weights b_1..b_m (most recent first).  The 2-step weights are
// (3/2, -1/2); the printed -3/2 would not be consistent (weights must sum to 1).
static const double kAB[3][4] = {
    {1.5, -0.5, 0, 0},
    {23.0 / 12, -16.0 / 12, 5.0 / 12, 0},
    {55.0 / 24, -59.0 / 24, 37.0 / 24, -9.0 / 24},
};

// ----------------------------------------------------------- stage kernels
// Column j of the X11 block, the complement coefficient c_j, and the W, Z
// coordinates of one stage (eqs. X-blocks-sol and X-blocks-sol-qLL, hbar = 1):
//   q-LLG: X11_ij = i (l_i - l_j) G_ij / (1 - i kappa (l_i - l_j)),  c_i = i l_i / (1 - i kappa l_i)
//   q-LL:  X11_ij = (i (l_i - l_j) - kappa (l_i - l_j)^2) G_ij,       c_i = (i - kappa l_i) l_i
//   W = (H V - V G) diag(conj c),  Z = V X11 + W.
__device__ __forceinline__ zd x11_factor(double li, double lj, double kappa, int model) {
  const double d = li - lj;
  if (model == LREI_QLLG) {
    // i d / (1 - i kappa d) = i d (1 + i kappa d) / (1 + kappa^2 d^2)
    const double den = 1.0 + kappa * kappa * d * d;
    return mk<double>(-kappa * d * d / den, d / den);
  }
  return mk<double>(-kappa * d * d, d);
}
__device__ __forceinline__ zd c_factor(double l, double kappa, int model) {
  if (model == LREI_QLLG) {
    const double den = 1.0 + kappa * kappa * l * l;
    return mk<double>(-kappa * l * l / den, l / den);
  }
  return mk<double>(-kappa * l * l, l);
}

__global__ void stage_xwz_kernel(const zd *__restrict__ G, int r, const double *__restrict__ lam, double kappa,
                                 int model, const zd *__restrict__ Y, const zd *__restrict__ T, int K, int ld,
                                 zd *__restrict__ X11, zd *__restrict__ Z, zd *__restrict__ W, zd *__restrict__ Gh) {
  const int j = blockIdx.x;
  extern __shared__ zd sh[];
  zd *gcol = sh;        // hermitised column j of G
  zd *xcol = sh + r;    // column j of X11
  for (int i = threadIdx.x; i < r; i += blockDim.x) {
    const zd a = G[(size_t)j * r + i], b = G[(size_t)i * r + j];
    zd g = mk<double>(0.5 * (a.re + b.re), 0.5 * (a.im - b.im));
    if (i == j) g.im = 0.0;
    gcol[i] = g;
    xcol[i] = x11_factor(lam[i], lam[j], kappa, model) * g;
    X11[(size_t)j * r + i] = xcol[i];
    if (Gh) Gh[(size_t)j * r + i] = g;
  }
  __syncthreads();
  const zd cc = conj(c_factor(lam[j], kappa, model));
  for (int row = threadIdx.x; row < K; row += blockDim.x) {
    zd yg = mk<double>(0, 0), yx = mk<double>(0, 0);
    for (int i = 0; i < r; ++i) {
      const zd y = Y[(size_t)i * ld + row];
      fma_(yg, y, gcol[i]);
      fma_(yx, y, xcol[i]);
    }
    const zd w = (T[(size_t)j * ld + row] - yg) * cc;
    W[(size_t)j * ld + row] = w;
    Z[(size_t)j * ld + row] = yx + w;
  }
}

struct StageCoefs {
  int nterms;
  double c[4];
};

// Factor matrices of a stage matrix: M = sum_b U_b V_b^H with
//   U = [Y_0 Lambda_0 | h c_0 Z_0 | h c_0 Y_0 | h c_1 Z_1 | h c_1 Y_1 | ...]
//   V = [Y_0          | Y_0       | W_0       | Y_1       | W_1       | ...]
// i.e. K_1 + h sum_l c_l (Z_l V_l^* + V_l W_l^*) in the Krylov coordinates (eqs. K-expand, rho-expand).
struct StagePtrs {
  const zd *y[5];
  const zd *z[4];
  const zd *w[4];
};
__global__ void stage_factors_kernel(StagePtrs P, StageCoefs C, const double *__restrict__ lam,
                                     const double *__restrict__ dt, int r, int K, int ld, zd *__restrict__ U,
                                     zd *__restrict__ V) {
  const int nb = 1 + 2 * C.nterms;
  const double h = *dt;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nb * r * K; e += gridDim.x * blockDim.x) {
    const int row = e % K, col = e / K, blk = col / r, j = col % r;
    zd u, v;
    if (blk == 0) {
      const zd y = P.y[0][(size_t)j * ld + row];
      u = lam[j] * y;
      v = y;
    } else {
      const int l = (blk - 1) / 2;
      const double a = h * C.c[l];
      if ((blk - 1) % 2 == 0) {
        u = a * P.z[l][(size_t)j * ld + row];
        v = P.y[l][(size_t)j * ld + row];
      } else {
        u = a * P.y[l][(size_t)j * ld + row];
        v = P.w[l][(size_t)j * ld + row];
      }
    }
    U[(size_t)col * ld + row] = u;
    V[(size_t)col * ld + row] = v;
  }
}

// Rc = Lr^H with the rows of dead residual columns zeroed, written into Chat.
__global__ void store_rc_kernel(const zd *__restrict__ Lr, int r, const int *__restrict__ dead, zd *__restrict__ dst,
                                int ld) {
  for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
    const int i = e % r, j = e / r;
    zd v = (i <= j) ? conj(Lr[(size_t)i * r + j]) : mk<double>(0, 0);
    if (dead[i]) v = mk<double>(0, 0);
    dst[(size_t)j * ld + i] = v;
  }
}

// New rows k..k+r-1 of the Cholesky factor of Gamma: [Bs^H | L22], dead rows decoupled.
__global__ void store_lrows_kernel(const zd *__restrict__ Bs, int ldb, const zd *__restrict__ L22, int r, int k,
                                   const int *__restrict__ dead, zd *__restrict__ L, int ldl) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < r * (k + r); e += gridDim.x * blockDim.x) {
    const int j = e % r, m = e / r;   // row k + j, column m
    zd v;
    if (m < k) v = dead[j] ? mk<double>(0, 0) : conj(Bs[(size_t)j * ldb + m]);
    else v = L22[(size_t)(m - k) * r + j];
    L[(size_t)m * ldl + (k + j)] = v;
  }
}

__global__ void check_small_kernel(const double *mu, int r, const zd *G, int ldg, int *status) {
  bool bad = false;
  for (int i = threadIdx.x; i < r; i += blockDim.x) bad |= !isfinite(mu[i]);
  for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
    const zd v = G[(size_t)(e / r) * ldg + (e % r)];
    bad |= !isfinite(v.re) || !isfinite(v.im);
  }
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(status, ST_NONFINITE);
}

// Diagonal matrix of conj(c) (for the explicit right-hand side) and -G diag(conj c).
__global__ void rhs_coef_kernel(const zd *__restrict__ G, int r, const double *__restrict__ lam, double kappa,
                                int model, zd *__restrict__ Dc, zd *__restrict__ Gc, zd *__restrict__ X11) {
  for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
    const int i = e % r, j = e / r;
    const zd a = G[(size_t)j * r + i], b = G[(size_t)i * r + j];
    zd g = mk<double>(0.5 * (a.re + b.re), 0.5 * (a.im - b.im));
    const zd cc = conj(c_factor(lam[j], kappa, model));
    Dc[e] = (i == j) ? cc : mk<double>(0, 0);
    Gc[e] = mk<double>(-1, 0) * (g * cc);
    X11[e] = x11_factor(lam[i], lam[j], kappa, model) * g;
  }
}

// B = L^H diag(lam) L (r x r) for set_state.
__global__ void lhl_kernel(const zd *__restrict__ L, int r, const double *__restrict__ lam, zd *__restrict__ B) {
  for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
    const int i = e % r, j = e / r;
    zd s = mk<double>(0, 0);
    for (int m = 0; m < r; ++m) {
      // (L^H)_{im} = conj(L_{mi}), L_{mj}
      const zd a = conj(L[(size_t)i * r + m]);
      fma_(s, a, lam[m] * L[(size_t)j * r + m]);
    }
    B[e] = s;
  }
}

// Observables from the Gram blocks of the observable pass.
__global__ void obs_final_kernel(const double *__restrict__ red, int r, const double *__restrict__ lam,
                                 double *__restrict__ out) {
  // blocks: 0 V^*HV, 1 (HV)^*(HV), 2 V^*V, 3 V^*MxV, 4 V^*MyV, 5 V^*MzV
  extern __shared__ zd s[];
  zd *Gm = s, *X = s + r * r;  // Gamma copy then L, X = L^{-1}
  const zd *B = reinterpret_cast<const zd *>(red);
  const int t = threadIdx.x;
  for (int e = t; e < r * r; e += blockDim.x) Gm[e] = B[2 * r * r + e];
  __syncthreads();
  if (t == 0) {
    // in-place Cholesky of Gamma (lower), then X = L^{-1}
    for (int j = 0; j < r; ++j) {
      double d = Gm[j * r + j].re;
      for (int m = 0; m < j; ++m) d -= norm2(Gm[m * r + j]);
      d = sqrt(fmax(d, 1e-300));
      Gm[j * r + j] = mk<double>(d, 0);
      for (int i = j + 1; i < r; ++i) {
        zd v = Gm[j * r + i];
        for (int m = 0; m < j; ++m) v = v - Gm[m * r + i] * conj(Gm[m * r + j]);
        Gm[j * r + i] = mk<double>(v.re / d, v.im / d);
      }
    }
    for (int j = 0; j < r; ++j)
      for (int i = 0; i < r; ++i) {
        if (i < j) { X[j * r + i] = mk<double>(0, 0); continue; }
        zd v = mk<double>(i == j ? 1.0 : 0.0, 0);
        for (int m = j; m < i; ++m) v = v - Gm[m * r + i] * X[j * r + m];
        const double d = Gm[i * r + i].re;
        X[j * r + i] = mk<double>(v.re / d, v.im / d);
      }
  }
  __syncthreads();
  if (t == 0) {
    double acc[6] = {0, 0, 0, 0, 0, 0};
    // Abar = X A X^H, trace with Lambda: sum_i lam_i sum_{m,n} X_im A_mn conj(X_in)
    const int which[5] = {0, 1, 3, 4, 5};
    for (int w = 0; w < 5; ++w) {
      const zd *A = B + which[w] * r * r;
      double tr = 0.0;
      for (int i = 0; i < r; ++i) {
        const double li = (w == 1) ? lam[i] * lam[i] : lam[i];
        zd sacc = mk<double>(0, 0);
        for (int m = 0; m < r; ++m)
          for (int n = 0; n < r; ++n) sacc = sacc + X[m * r + i] * A[n * r + m] * conj(X[n * r + i]);
        tr += li * sacc.re;
      }
      acc[w] = tr;
    }
    // Tr(Lambda Gbar Lambda Gbar)
    double tgg = 0.0;
    for (int i = 0; i < r; ++i)
      for (int j = 0; j < r; ++j) {
        zd g = mk<double>(0, 0);
        for (int m = 0; m < r; ++m)
          for (int n = 0; n < r; ++n) g = g + X[m * r + i] * B[n * r + m] * conj(X[n * r + j]);
        tgg += lam[i] * lam[j] * norm2(g);
      }
    const zd *Gam = B + 2 * r * r;
    double trace = 0.0, purity = 0.0, orth = 0.0;
    for (int i = 0; i < r; ++i) {
      trace += lam[i] * Gam[i * r + i].re;
      for (int j = 0; j < r; ++j) {
        purity += lam[i] * lam[j] * norm2(Gam[j * r + i]);
        const zd d = Gam[j * r + i] - mk<double>(i == j ? 1.0 : 0.0, 0);
        orth = fmax(orth, sqrt(norm2(d)));
      }
    }
    double herm = 0.0, gmax = 0.0;
    for (int i = 0; i < r; ++i)
      for (int j = 0; j < r; ++j) {
        const zd a = B[j * r + i], b = B[i * r + j];
        herm = fmax(herm, sqrt(norm2(a - conj(b))));
        gmax = fmax(gmax, sqrt(norm2(a)));
      }
    out[0] = acc[0];                                // energy
    out[1] = acc[2];                                // mx
    out[2] = acc[3];                                // my
    out[3] = acc[4];                                // mz
    out[4] = purity;
    out[5] = trace;
    out[6] = orth;
    out[7] = gmax > 0 ? herm / gmax : 0.0;
    out[8] = sqrt(fmax(0.0, 2.0 * acc[1] - 2.0 * tgg));   // ||[rho, H]||_F
  }
}

}  // namespace lrei

using namespace lrei;

struct lrei_ctx {
  int dev = 0, nsm = 0;
  int n = 0;
  long long N = 0;
  int r_max = 0, r = 0;
  int model = 0, prec = 0;
  double kappa = 0.0;
  bool fp64 = true;
  size_t elem = 16;
  cudaStream_t user = nullptr, st = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  ModelArgs M;
  int KM = 0;   // leading dimension / capacity of the small k x k arrays
  // N x r blocks
  void *V = nullptr;
  void *blk[MAXB] = {};
  int nblk = 0;
  // device workspace
  double *partial = nullptr;
  double *red = nullptr;
  void *coef_scratch = nullptr;
  zd *Gam = nullptr, *L = nullptr, *Chat = nullptr, *Tbar = nullptr, *Xh = nullptr, *Cc = nullptr, *GR = nullptr,
     *Lr = nullptr, *Ainv = nullptr, *coefQ = nullptr, *Bs = nullptr, *Dm = nullptr, *L22 = nullptr, *Mm = nullptr,
     *Uf = nullptr, *Vf = nullptr, *Yc = nullptr, *ts = nullptr, *G = nullptr, *X11 = nullptr, *Gh = nullptr;
  zd *ys[5] = {}, *zs[4] = {}, *wsv[4] = {};
  zd *yfin = nullptr;
  double *lam0_dev = nullptr, *mu_dev = nullptr, *dt_dev = nullptr, *obs_dev = nullptr;
  int *status_dev = nullptr, *dead_dev = nullptr;
  void *eig_ws = nullptr;
  int *status_host = nullptr;
  double *obs_host = nullptr;
  std::vector<double> lam0;
  double t = 0.0;
  double dt_cur = 0.0;
  bool has_state = false;
  // graph cache for one step of a given scheme
  cudaGraphExec_t gexec = nullptr;
  int g_scheme = -1, g_r = -1;
  long long g_nodes = 0;
  long long launches = 0;
  int last_status = 0;
  // allocation list
  std::vector<void *> allocs;
};

namespace {

int dalloc(lrei_ctx *c, void **p, size_t bytes) {
  cudaError_t e = cudaMalloc(p, bytes ? bytes : 16);
  if (e != cudaSuccess) return LREI_ERR_OOM;
  c->allocs.push_back(*p);
  cudaMemset(*p, 0, bytes ? bytes : 16);
  return LREI_OK;
}
template <typename P>
int dalloc_t(lrei_ctx *c, P **p, size_t bytes) {
  void *q = nullptr;
  int rc = dalloc(c, &q, bytes);
  *p = reinterpret_cast<P *>(q);
  return rc;
}

int status_to_code(int st) {
  if (st & ST_NONFINITE) return LREI_ERR_NONFINITE;
  if (st & ST_TIMEOUT) return LREI_ERR_TIMEOUT;
  if (st & ST_RANK) return LREI_ERR_RANK;
  if (st & (ST_EIG_NOCONV | ST_EIG_RESID)) return LREI_ERR_EIG_NOCONV;
  if (st & ST_TRACE) return LREI_ERR_TRACE;
  return LREI_OK;
}

// Order the internal stream after the caller's stream, and back.
void enter(lrei_ctx *c) {
  cudaEventRecord(c->ev_in, c->user);
  cudaStreamWaitEvent(c->st, c->ev_in, 0);
}
void leave(lrei_ctx *c) {
  cudaEventRecord(c->ev_out, c->st);
  cudaStreamWaitEvent(c->user, c->ev_out, 0);
}

const zd ONE = {1.0, 0.0}, ZERO = {0.0, 0.0}, MONE = {-1.0, 0.0};

double tol_rc(const lrei_ctx *c) { return c->fp64 ? 1e-24 : 1e-12; }
const double TOL_GAM = 1e-6;

// One tall-skinny pass + deterministic reduction of its Gram into c->red.
int ts_pass(lrei_ctx *c, TSArgs a) {
  a.N = c->N;
  a.r = c->r;
  a.partial = c->partial;
  a.coef_scratch = c->coef_scratch;
  int g = launch_ts(c->fp64, c->M, a, c->nsm, c->st);
  if (g < 0) return LREI_ERR_ARG;
  launch_reduce(c->partial, g, (int)ts_partial_doubles(a.gram_left, c->r), c->red, c->st);
  return LREI_OK;
}

void *qblock(lrei_ctx *c, int m) { return m == 0 ? c->V : c->blk[m - 1]; }

// Gamma[0:r,0:r] <- red (V^*V), L[0:r,0:r] <- chol.
void set_gamma00(lrei_ctx *c) {
  const int r = c->r, KM = c->KM;
  sm_copy(reinterpret_cast<zd *>(c->red), r, r, r, c->Gam, KM, c->st);
  sm_hermitize(c->Gam, KM, r, c->st);
  sm_chol(c->Gam, KM, r, c->L22, r, TOL_GAM, 1, c->dead_dev, c->status_dev, 1, c->st);
  sm_copy(c->L22, r, r, r, c->L, KM, c->st);
}

// Enqueue one RK step (scheme 0..3) on c->st.  Precondition: Gam/L leading r x r hold V^*V.
int enqueue_rk_step(lrei_ctx *c, int scheme) {
  const Tableau &tb = kRK[scheme];
  const int s = tb.s, r = c->r, KM = c->KM, K = (s + 1) * r, sr = s * r;
  cudaStream_t st = c->st;
  zd *red = reinterpret_cast<zd *>(c->red);
  for (int l = 0; l < s; ++l) {
    const int k = (l + 1) * r, ldr = (l + 2) * r;
    // pass A: S = H Q_l, P = [Q_0..Q_l]^* S, S^*S
    TSArgs a{};
    a.nq = l + 1;
    a.gram_left = l + 1;
    for (int m = 0; m <= l; ++m) a.q[m] = qblock(c, m);
    a.src = qblock(c, l);
    a.apply_h = 1;
    a.mode = 0;
    int rc = ts_pass(c, a);
    if (rc) return rc;
    // C = Gamma^{-1} P
    sm_copy(red, ldr, k, r, c->Cc, KM, st);
    sm_trsv('N', c->L, KM, k, c->Cc, KM, r, st);
    sm_trsv('C', c->L, KM, k, c->Cc, KM, r, st);
    // GR = S^*S - P^* C (Gram of the projected residual)
    sm_copy(red + k, ldr, r, r, c->GR, r, st);
    sm_gemm('C', 'N', r, r, k, MONE, red, ldr, c->Cc, KM, ONE, c->GR, r, st);
    sm_hermitize(c->GR, r, r, st);
    sm_chol(c->GR, r, r, c->Lr, r, tol_rc(c), 0, c->dead_dev, c->status_dev, 0, st);
    // A = (Lr^H)^{-1}; coefQ = -C A; Chat column block l = [C; Lr^H]
    sm_set_identity(c->Ainv, r, r, r, st);
    sm_trsv('C', c->Lr, r, r, c->Ainv, r, r, st);
    sm_gemm('N', 'N', k, r, r, MONE, c->Cc, KM, c->Ainv, r, ZERO, c->coefQ, k, st);
    sm_copy(c->Cc, KM, k, r, c->Chat + (size_t)l * r * KM, KM, st);
    store_rc_kernel<<<1, 256, 0, st>>>(c->Lr, r, c->dead_dev, c->Chat + (size_t)l * r * KM + k, KM);
    // pass B: Q_{l+1} = S A - Q C A, Gram column [Q_0..Q_l, Q_{l+1}]^* Q_{l+1}
    TSArgs b = a;
    b.mode = 1;
    b.coefS = c->Ainv;
    b.coefQ = c->coefQ;
    b.out = qblock(c, l + 1);
    rc = ts_pass(c, b);
    if (rc) return rc;
    sm_store_gram_cols(red, ldr, k, r, c->Gam, KM, st);
    // extend the Cholesky factor of Gamma
    sm_copy(c->Gam + (size_t)k * KM, KM, k, r, c->Bs, KM, st);
    sm_trsv('N', c->L, KM, k, c->Bs, KM, r, st);
    sm_copy(c->Gam + (size_t)k * KM + k, KM, r, r, c->Dm, r, st);
    sm_gemm('C', 'N', r, r, k, MONE, c->Bs, KM, c->Bs, KM, ONE, c->Dm, r, st);
    sm_hermitize(c->Dm, r, r, st);
    sm_chol(c->Dm, r, r, c->L22, r, TOL_GAM, 1, c->dead_dev, c->status_dev, 0, st);
    store_lrows_kernel<<<8, 256, 0, st>>>(c->Bs, KM, c->L22, r, k, c->dead_dev, c->L, KM);
  }
  // Tbar = L^H Chat L_s^{-H}: H Qbar_{0..s-1} = Qbar Tbar in the orthonormal frame Qbar = Q L^{-H}
  sm_conj_transpose(c->Chat, KM, K, sr, c->Xh, KM, st);
  sm_trsv('N', c->L, KM, sr, c->Xh, KM, K, st);
  sm_gemm('C', 'C', K, sr, K, ONE, c->L, KM, c->Xh, KM, ZERO, c->Tbar, KM, st);
  sm_hermitize(c->Tbar, KM, sr, st);
  // stages
  sm_zero(c->ys[0], KM, K, r, st);
  sm_set_identity(c->ys[0], KM, r, r, st);
  StagePtrs P{};
  for (int j = 0; j < s; ++j) {
    sm_gemm('N', 'N', K, r, sr, ONE, c->Tbar, KM, c->ys[j], KM, ZERO, c->ts, KM, st);
    sm_gemm('C', 'N', r, r, sr, ONE, c->ys[j], KM, c->ts, KM, ZERO, c->G, r, st);
    stage_xwz_kernel<<<r, 128, 2 * r * sizeof(zd), st>>>(c->G, r, c->lam0_dev, c->kappa, c->model, c->ys[j], c->ts, K,
                                                         KM, c->X11, c->zs[j], c->wsv[j], j == 0 ? c->Gh : nullptr);
    StageCoefs C{};
    C.nterms = j + 1;
    const bool last = (j + 1 == s);
    for (int l = 0; l <= j; ++l) C.c[l] = last ? tb.b[l] : tb.a[j + 1][l];
    for (int l = 0; l <= j; ++l) {
      P.y[l] = c->ys[l];
      P.z[l] = c->zs[l];
      P.w[l] = c->wsv[l];
    }
    const int nf = r * (1 + 2 * (j + 1));
    const int kk = last ? K : (j + 2) * r;
    stage_factors_kernel<<<64, 256, 0, st>>>(P, C, c->lam0_dev, c->dt_dev, r, K, KM, c->Uf, c->Vf);
    sm_gemm('N', 'C', kk, kk, nf, ONE, c->Uf, KM, c->Vf, KM, ZERO, c->Mm, KM, st);
    sm_hermitize(c->Mm, KM, kk, st);
    zd *dst = last ? c->yfin : c->ys[j + 1];
    sm_zero(dst, KM, K, r, st);
    sm_eig_topr(c->Mm, KM, kk, r, dst, KM, c->mu_dev, c->eig_ws, c->status_dev, st);
  }
  // V_{k+1} = Qbar Yfin = Q (L^{-H} Yfin), formed in place over Q_0 = V
  sm_copy(c->yfin, KM, K, r, c->Yc, KM, st);
  sm_trsv('C', c->L, KM, K, c->Yc, KM, r, st);
  sm_copy(c->Yc, KM, K, r, c->coefQ, K, st);
  TSArgs cmb{};
  cmb.nq = s + 1;
  cmb.gram_left = 0;
  for (int m = 0; m <= s; ++m) cmb.q[m] = qblock(c, m);
  cmb.coefQ = c->coefQ;
  cmb.mode = 2;
  cmb.out = c->V;
  int rc = ts_pass(c, cmb);
  if (rc) return rc;
  set_gamma00(c);
  check_small_kernel<<<1, 256, 0, st>>>(c->mu_dev, r, c->Gam, KM, c->status_dev);
  return LREI_OK;
}

int count_kernel_nodes(cudaGraph_t g) {
  size_t n = 0;
  cudaGraphGetNodes(g, nullptr, &n);
  std::vector<cudaGraphNode_t> nodes(n);
  cudaGraphGetNodes(g, nodes.data(), &n);
  int k = 0;
  for (size_t i = 0; i < n; ++i) {
    cudaGraphNodeType t;
    cudaGraphNodeGetType(nodes[i], &t);
    if (t == cudaGraphNodeTypeKernel) ++k;
  }
  return k;
}

int build_graph(lrei_ctx *c, int scheme) {
  if (c->gexec && c->g_scheme == scheme && c->g_r == c->r) return LREI_OK;
  if (c->gexec) {
    cudaGraphExecDestroy(c->gexec);
    c->gexec = nullptr;
  }
  cudaGraph_t g = nullptr;
  LREI_CUDA_TRY(cudaStreamBeginCapture(c->st, cudaStreamCaptureModeThreadLocal));
  int rc = enqueue_rk_step(c, scheme);
  cudaError_t e = cudaStreamEndCapture(c->st, &g);
  if (rc) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  if (e != cudaSuccess) return cuda_fail(e, "capture");
  c->g_nodes = count_kernel_nodes(g);
  e = cudaGraphInstantiate(&c->gexec, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return cuda_fail(e, "instantiate");
  c->g_scheme = scheme;
  c->g_r = c->r;
  return LREI_OK;
}

int read_status(lrei_ctx *c) {
  LREI_CUDA_TRY(cudaMemcpyAsync(c->status_host, c->status_dev, sizeof(int), cudaMemcpyDeviceToHost, c->st));
  LREI_CUDA_TRY(cudaStreamSynchronize(c->st));
  int s = *c->status_host;
  c->last_status = s;
  LREI_CUDA_TRY(cudaMemsetAsync(c->status_dev, 0, sizeof(int), c->st));
  return s;
}

}  // namespace

extern "C" {

const char *lrei_error_string(int code) {
  switch (code) {
    case LREI_OK: return "ok";
    case LREI_ERR_ARG: return "invalid argument";
    case LREI_ERR_UNSUPPORTED: return "unsupported physics in this build (transverse field)";
    case LREI_ERR_NONFINITE: return "non-finite value in input or state";
    case LREI_ERR_TRACE: return "spectrum must be >= 0 and sum to 1";
    case LREI_ERR_RANK: return "rank-deficient factor";
    case LREI_ERR_EIG_NOCONV: return "small eigensolver did not converge";
    case LREI_ERR_OOM: return "device allocation failed";
    case LREI_ERR_CUDA: return "CUDA runtime error";
    case LREI_ERR_STATE: return "call out of order";
    case LREI_ERR_TIMEOUT: return "bounded device wait ran out";
    default: return "unknown error";
  }
}

int lrei_create(int n, const lrei_bonds *J, const double B[3], double lambda, lrei_model model,
                lrei_precision prec, int r_max, void *cuda_stream, lrei_ctx **out) {
  if (!out) return LREI_ERR_ARG;
  *out = nullptr;
  if (n < 1 || n > MAX_SPINS || r_max < 1 || r_max > MAX_R || !(lambda >= 0.0) || !std::isfinite(lambda))
    return LREI_ERR_ARG;
  if (model != LREI_QLL && model != LREI_QLLG) return LREI_ERR_ARG;
  if (prec != LREI_FP64 && prec != LREI_MIXED_C64) return LREI_ERR_ARG;
  if ((long long)r_max > (1LL << n)) return LREI_ERR_ARG;
  double Bv[3] = {0, 0, 0};
  if (B) for (int i = 0; i < 3; ++i) Bv[i] = B[i];
  for (int i = 0; i < 3; ++i)
    if (!std::isfinite(Bv[i])) return LREI_ERR_NONFINITE;
  if (Bv[0] != 0.0 || Bv[1] != 0.0) return LREI_ERR_UNSUPPORTED;
  const int nb = J ? J->nbonds : 0;
  if (nb < 0 || nb > MAX_BONDS) return LREI_ERR_ARG;
  if (nb > 0 && (!J->site_i || !J->site_j || !J->jxy || !J->jz)) return LREI_ERR_ARG;
  lrei_ctx *c = new (std::nothrow) lrei_ctx();
  if (!c) return LREI_ERR_OOM;
  std::memset(&c->M, 0, sizeof(c->M));
  c->M.n = n;
  c->M.nb = nb;
  c->M.bz = Bv[2];
  double c0 = 0.0;
  for (int b = 0; b < nb; ++b) {
    const int i = J->site_i[b], j = J->site_j[b];
    if (i < 0 || i >= n || j < 0 || j >= n || i == j || !std::isfinite(J->jxy[b]) || !std::isfinite(J->jz[b])) {
      delete c;
      return LREI_ERR_ARG;
    }
    // site i is bit n-1-i of the basis index (site 0 = most significant bit)
    c->M.bi[b] = (uint8_t)(n - 1 - i);
    c->M.bj[b] = (uint8_t)(n - 1 - j);
    c->M.mask[b] = (1u << (n - 1 - i)) | (1u << (n - 1 - j));
    c->M.jxy[b] = J->jxy[b];
    c->M.jz[b] = J->jz[b];
    c0 += 0.5 * J->jz[b];
  }
  c->M.c0 = c0;
  c->n = n;
  c->N = 1LL << n;
  c->r_max = r_max;
  c->model = model;
  c->prec = prec;
  c->kappa = lambda;
  c->fp64 = (prec == LREI_FP64);
  c->elem = c->fp64 ? 16 : 8;
  c->user = reinterpret_cast<cudaStream_t>(cuda_stream);
  int rc = LREI_OK;
  auto fail = [&](int code) {
    lrei_destroy(c);
    return code;
  };
  if (cudaGetDevice(&c->dev) != cudaSuccess) return fail(LREI_ERR_CUDA);
  cudaDeviceGetAttribute(&c->nsm, cudaDevAttrMultiProcessorCount, c->dev);
  if (cudaStreamCreateWithFlags(&c->st, cudaStreamNonBlocking) != cudaSuccess) return fail(LREI_ERR_CUDA);
  cudaEventCreateWithFlags(&c->ev_in, cudaEventDisableTiming);
  cudaEventCreateWithFlags(&c->ev_out, cudaEventDisableTiming);
  if (ts_init() || sm_init()) return fail(LREI_ERR_CUDA);
  const size_t blk_bytes = (size_t)c->N * r_max * c->elem;
  c->nblk = 4;
  if ((rc = dalloc(c, &c->V, blk_bytes))) return fail(rc);
  for (int i = 0; i < c->nblk; ++i)
    if ((rc = dalloc(c, &c->blk[i], blk_bytes))) return fail(rc);
  c->KM = 5 * r_max;
  const int KM = c->KM, R = r_max;
  const size_t zs = sizeof(zd);
  if ((rc = dalloc_t(c, &c->partial, (size_t)ts_max_grid(c->nsm) * (MAXB + 1) * R * R * 2 * sizeof(double)))) return fail(rc);
  if ((rc = dalloc_t(c, &c->red, (size_t)(MAXB + 1) * R * R * 2 * sizeof(double)))) return fail(rc);
  if ((rc = dalloc(c, &c->coef_scratch, (size_t)(MAXB + 1) * R * R * zs))) return fail(rc);
  zd **kk[] = {&c->Gam, &c->L, &c->Chat, &c->Tbar, &c->Xh, &c->Mm};
  for (auto p : kk)
    if ((rc = dalloc_t(c, p, (size_t)KM * KM * zs))) return fail(rc);
  zd **kr[] = {&c->Cc, &c->coefQ, &c->Bs, &c->Yc, &c->ts, &c->yfin};
  for (auto p : kr)
    if ((rc = dalloc_t(c, p, (size_t)KM * R * zs))) return fail(rc);
  for (int i = 0; i < 5; ++i)
    if ((rc = dalloc_t(c, &c->ys[i], (size_t)KM * R * zs))) return fail(rc);
  for (int i = 0; i < 4; ++i) {
    if ((rc = dalloc_t(c, &c->zs[i], (size_t)KM * R * zs))) return fail(rc);
    if ((rc = dalloc_t(c, &c->wsv[i], (size_t)KM * R * zs))) return fail(rc);
  }
  if ((rc = dalloc_t(c, &c->Uf, (size_t)KM * 9 * R * zs))) return fail(rc);
  if ((rc = dalloc_t(c, &c->Vf, (size_t)KM * 9 * R * zs))) return fail(rc);
  zd **rr[] = {&c->GR, &c->Lr, &c->Ainv, &c->Dm, &c->L22, &c->G, &c->X11, &c->Gh};
  for (auto p : rr)
    if ((rc = dalloc_t(c, p, (size_t)R * R * zs))) return fail(rc);
  if ((rc = dalloc_t(c, &c->lam0_dev, R * sizeof(double)))) return fail(rc);
  if ((rc = dalloc_t(c, &c->mu_dev, R * sizeof(double)))) return fail(rc);
  if ((rc = dalloc_t(c, &c->dt_dev, sizeof(double)))) return fail(rc);
  if ((rc = dalloc_t(c, &c->obs_dev, 16 * sizeof(double)))) return fail(rc);
  if ((rc = dalloc_t(c, &c->status_dev, sizeof(int)))) return fail(rc);
  if ((rc = dalloc_t(c, &c->dead_dev, R * sizeof(int)))) return fail(rc);
  if ((rc = dalloc(c, &c->eig_ws, sm_eig_ws_bytes(KM, R)))) return fail(rc);
  if (cudaMallocHost(&c->status_host, sizeof(int)) != cudaSuccess) return fail(LREI_ERR_OOM);
  if (cudaMallocHost(&c->obs_host, 16 * sizeof(double)) != cudaSuccess) return fail(LREI_ERR_OOM);
  if (cudaDeviceSynchronize() != cudaSuccess) return fail(LREI_ERR_CUDA);
  *out = c;
  return LREI_OK;
}

int lrei_destroy(lrei_ctx *c) {
  if (!c) return LREI_OK;
  if (c->st) cudaStreamSynchronize(c->st);
  if (c->gexec) cudaGraphExecDestroy(c->gexec);
  for (void *p : c->allocs) cudaFree(p);
  if (c->status_host) cudaFreeHost(c->status_host);
  if (c->obs_host) cudaFreeHost(c->obs_host);
  if (c->ev_in) cudaEventDestroy(c->ev_in);
  if (c->ev_out) cudaEventDestroy(c->ev_out);
  if (c->st) cudaStreamDestroy(c->st);
  delete c;
  return LREI_OK;
}

int lrei_set_state(lrei_ctx *c, const void *V_dev, int r, int ld, int dtype, const double *Lambda_host) {
  if (!c || !V_dev || !Lambda_host) return LREI_ERR_ARG;
  if (r < 1 || r > c->r_max || ld < r || (dtype != LREI_C128 && dtype != LREI_C64)) return LREI_ERR_ARG;
  double sum = 0.0;
  for (int i = 0; i < r; ++i) {
    if (!std::isfinite(Lambda_host[i])) return LREI_ERR_NONFINITE;
    if (Lambda_host[i] < 0.0) return LREI_ERR_TRACE;
    sum += Lambda_host[i];
  }
  if (std::fabs(sum - 1.0) > 1e-12) return LREI_ERR_TRACE;
  enter(c);
  c->r = r;
  c->has_state = false;
  const int KM = c->KM;
  std::vector<double> lam_in(Lambda_host, Lambda_host + r);
  LREI_CUDA_TRY(cudaMemsetAsync(c->status_dev, 0, sizeof(int), c->st));
  LREI_CUDA_TRY(cudaMemsetAsync(c->L, 0, (size_t)KM * KM * sizeof(zd), c->st));
  LREI_CUDA_TRY(cudaMemsetAsync(c->Gam, 0, (size_t)KM * KM * sizeof(zd), c->st));
  launch_convert(V_dev, dtype == LREI_C64, ld, c->V, c->fp64, c->N, r, c->st);
  launch_check_finite(c->fp64, c->V, c->N, r, c->status_dev, c->st);
  // R^H R = V^*V (Cholesky), rho_0 = Q (R Lambda R^H) Q^*, Q = V R^{-1}
  TSArgs a{};
  a.nq = 0;
  a.gram_left = 0;
  a.src = c->V;
  a.apply_h = 0;
  a.mode = 0;
  int rc = ts_pass(c, a);
  if (rc) { leave(c); return rc; }
  zd *red = reinterpret_cast<zd *>(c->red);
  sm_hermitize(red, r, r, c->st);
  sm_chol(red, r, r, c->L22, r, 1e-24, 1, c->dead_dev, c->status_dev, 1, c->st);
  LREI_CUDA_TRY(cudaMemcpyAsync(c->lam0_dev, lam_in.data(), r * sizeof(double), cudaMemcpyHostToDevice, c->st));
  lhl_kernel<<<1, 256, 0, c->st>>>(c->L22, r, c->lam0_dev, c->Dm);
  sm_jacobi(true, c->Dm, r, r, c->Lr, r, c->mu_dev, c->eig_ws, 60, 1e-15, c->status_dev, c->st);
  // coefficients R^{-1} E = L^{-H} E
  sm_copy(c->Lr, r, r, r, c->coefQ, r, c->st);
  sm_trsv('C', c->L22, r, r, c->coefQ, r, r, c->st);
  TSArgs cmb{};
  cmb.nq = 1;
  cmb.gram_left = 0;
  cmb.q[0] = c->V;
  cmb.coefQ = c->coefQ;
  cmb.mode = 2;
  cmb.out = c->V;
  rc = ts_pass(c, cmb);
  if (rc) { leave(c); return rc; }
  set_gamma00(c);
  LREI_CUDA_TRY(cudaMemcpyAsync(c->lam0_dev, c->mu_dev, r * sizeof(double), cudaMemcpyDeviceToDevice, c->st));
  c->lam0.assign(r, 0.0);
  LREI_CUDA_TRY(cudaMemcpyAsync(c->lam0.data(), c->mu_dev, r * sizeof(double), cudaMemcpyDeviceToHost, c->st));
  const int s = read_status(c);
  leave(c);
  if (s) return status_to_code(s);
  for (int i = 0; i < r; ++i) {
    if (!std::isfinite(c->lam0[i])) return LREI_ERR_NONFINITE;
    if (c->lam0[i] < -1e-12) return LREI_ERR_TRACE;
    if (c->lam0[i] < 0.0) c->lam0[i] = 0.0;
  }
  cudaMemcpy(c->lam0_dev, c->lam0.data(), r * sizeof(double), cudaMemcpyHostToDevice);
  c->t = 0.0;
  c->has_state = true;
  return LREI_OK;
}

int lrei_get_state(lrei_ctx *c, void *V_dev_out, double *Lambda_host_out, double *t_out) {
  if (!c) return LREI_ERR_ARG;
  if (!c->has_state) return LREI_ERR_STATE;
  enter(c);
  if (V_dev_out)
    LREI_CUDA_TRY(cudaMemcpyAsync(V_dev_out, c->V, (size_t)c->N * c->r * c->elem, cudaMemcpyDeviceToDevice, c->st));
  leave(c);
  LREI_CUDA_TRY(cudaStreamSynchronize(c->st));
  if (Lambda_host_out) std::memcpy(Lambda_host_out, c->lam0.data(), c->r * sizeof(double));
  if (t_out) *t_out = c->t;
  return LREI_OK;
}

int lrei_step(lrei_ctx *c, double dt, lrei_scheme scheme, int nsteps) {
  if (!c) return LREI_ERR_ARG;
  if (!c->has_state) return LREI_ERR_STATE;
  if (!std::isfinite(dt) || nsteps < 0) return LREI_ERR_ARG;
  if (scheme < LREI_RK1 || scheme > LREI_AB4) return LREI_ERR_ARG;
  if (scheme > LREI_RK4) return LREI_ERR_UNSUPPORTED;
  if (nsteps == 0) return LREI_OK;
  enter(c);
  if (dt != c->dt_cur) {
    LREI_CUDA_TRY(cudaMemcpyAsync(c->dt_dev, &dt, sizeof(double), cudaMemcpyHostToDevice, c->st));
    LREI_CUDA_TRY(cudaStreamSynchronize(c->st));
    c->dt_cur = dt;
  }
  int rc = build_graph(c, (int)scheme);
  if (rc) { leave(c); return rc; }
  for (int i = 0; i < nsteps; ++i) {
    LREI_CUDA_TRY(cudaGraphLaunch(c->gexec, c->st));
    c->launches += c->g_nodes;
  }
  const int s = read_status(c);
  leave(c);
  c->t += dt * nsteps;
  return status_to_code(s);
}

int lrei_step_adaptive(lrei_ctx *c, double t_end, double tol, int controller) {
  (void)t_end; (void)tol; (void)controller;
  if (!c) return LREI_ERR_ARG;
  return LREI_ERR_UNSUPPORTED;
}

int lrei_observables(lrei_ctx *c, lrei_obs *out) {
  if (!c || !out) return LREI_ERR_ARG;
  if (!c->has_state) return LREI_ERR_STATE;
  const int r = c->r;
  enter(c);
  int g = launch_obs(c->fp64, c->M, c->V, c->N, r, c->partial, c->nsm, c->st);
  launch_reduce(c->partial, g, 6 * r * r * 2, c->red, c->st);
  obs_final_kernel<<<1, 32, 2 * r * r * sizeof(zd), c->st>>>(c->red, r, c->lam0_dev, c->obs_dev);
  LREI_CUDA_TRY(cudaMemcpyAsync(c->obs_host, c->obs_dev, 9 * sizeof(double), cudaMemcpyDeviceToHost, c->st));
  std::vector<double> mu(r);
  LREI_CUDA_TRY(cudaMemcpyAsync(mu.data(), c->mu_dev, r * sizeof(double), cudaMemcpyDeviceToHost, c->st));
  leave(c);
  LREI_CUDA_TRY(cudaStreamSynchronize(c->st));
  c->launches += 3;
  std::memset(out, 0, sizeof(*out));
  out->t = c->t;
  out->energy = c->obs_host[0];
  out->mx = c->obs_host[1];
  out->my = c->obs_host[2];
  out->mz = c->obs_host[3];
  out->purity = c->obs_host[4];
  out->trace = c->obs_host[5];
  out->orth_err = c->obs_host[6];
  out->herm_err = c->obs_host[7];
  out->comm_norm = c->obs_host[8];
  out->r = r;
  for (int i = 0; i < r && i < 64; ++i) {
    out->ritz[i] = mu[i];
    out->lambda0[i] = c->lam0[i];
  }
  return LREI_OK;
}

int lrei_apply_h(lrei_ctx *c, const void *V_dev, void *Y_dev, int r) {
  if (!c || !V_dev || !Y_dev || V_dev == Y_dev || r < 1 || r > MAX_R) return LREI_ERR_ARG;
  enter(c);
  launch_hv(c->fp64, c->M, V_dev, Y_dev, c->N, r, c->nsm, c->st);
  leave(c);
  c->launches += 1;
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? LREI_OK : cuda_fail(e, "apply_h");
}

int lrei_rhs(lrei_ctx *c, void *Z_dev, void *W_dev, double *G_host, int complement) {
  if (!c || !Z_dev || !W_dev) return LREI_ERR_ARG;
  if (!c->has_state) return LREI_ERR_STATE;
  if (complement != 0) return LREI_ERR_UNSUPPORTED;
  const int r = c->r;
  enter(c);
  // pass 1: Y = H V written to W, G = V^* Y
  TSArgs a{};
  a.nq = 1;
  a.gram_left = 1;
  a.q[0] = c->V;
  a.src = c->V;
  a.apply_h = 1;
  a.mode = 0;
  a.out = W_dev;
  int rc = ts_pass(c, a);
  if (rc) { leave(c); return rc; }
  zd *red = reinterpret_cast<zd *>(c->red);
  sm_copy(red, 2 * r, r, r, c->G, r, c->st);
  rhs_coef_kernel<<<1, 256, 0, c->st>>>(c->G, r, c->lam0_dev, c->kappa, c->model, c->Dm, c->GR, c->X11);
  // pass 2: W = Y diag(conj c) - V (G diag(conj c))   (in place over Y: row-local)
  TSArgs b{};
  b.nq = 1;
  b.gram_left = 0;
  b.q[0] = c->V;
  b.src = W_dev;
  b.apply_h = 0;
  b.mode = 1;
  b.coefS = c->Dm;
  b.coefQ = c->GR;
  b.out = W_dev;
  if ((rc = ts_pass(c, b))) { leave(c); return rc; }
  // pass 3: Z = V X11 + W
  sm_set_identity(c->Ainv, r, r, r, c->st);
  TSArgs z = b;
  z.src = W_dev;
  z.coefS = c->Ainv;
  z.coefQ = c->X11;
  z.out = Z_dev;
  if ((rc = ts_pass(c, z))) { leave(c); return rc; }
  if (G_host) {
    sm_hermitize(c->G, r, r, c->st);
    LREI_CUDA_TRY(cudaMemcpyAsync(G_host, c->G, (size_t)r * r * sizeof(zd), cudaMemcpyDeviceToHost, c->st));
  }
  leave(c);
  LREI_CUDA_TRY(cudaStreamSynchronize(c->st));
  c->launches += 12;
  return LREI_OK;
}

int lrei_last_status(lrei_ctx *c) { return c ? c->last_status : 0; }

long long lrei_kernel_launches(lrei_ctx *c) {
  if (!c) return 0;
  long long n = c->launches;
  c->launches = 0;
  return n;
}

}  // extern "C"
