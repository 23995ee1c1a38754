// Small dense complex linear algebra on the device (r x r and k x k, k <= 5 r).
// All matrices are complex double, column-major: element (i, j) at A[j * ld + i].
// FP64 work is spread over many small CTAs (GB300's FP64 rate per SM is low).
#pragma once
#include "common.cuh"

namespace lrei {

int sm_init();   // raise shared-memory limits once, outside any stream capture

// C = alpha * op(A) * op(B) + beta * C, op in {'N', 'C'} ('C' = conjugate transpose).
void sm_gemm(char opA, char opB, int M, int N, int K, zd alpha, const zd *A, int lda, const zd *B, int ldb, zd beta,
             zd *C, int ldc, cudaStream_t st);

// For each of ncols columns of B (in place): solve L x = b (op 'N') or L^H x = b (op 'C'),
// L lower triangular k x k.  A zero diagonal entry gives x_i = 0.
void sm_trsv(char op, const zd *L, int ldl, int k, zd *B, int ldb, int ncols, cudaStream_t st);

// Rows of X (nrows x k): X <- X (L^H)^{-1}, L lower triangular k x k.
void sm_rtrsm_lh(zd *X, int ldx, int nrows, const zd *L, int ldl, int k, cudaStream_t st);
// Same through an explicit inverse and one GEMM; inv: k x k scratch, xcopy: nrows x k scratch.
void sm_rtrsm_lh_ws(zd *X, int ldx, int nrows, const zd *L, int ldl, int k, zd *inv, zd *xcopy, cudaStream_t st);

// Cholesky A = L L^H of a Hermitian k x k matrix (k <= 64), one CTA.  A pivot below
// tol * max_i A_ii marks column j dead: L[j][j] = 1 and the rest of column j zero; with
// zero_row also row j of L (left of the diagonal) is zeroed.  dead (k ints) may be NULL.
// Nonzero status bit ST_RANK is set when any column is dead and flag_rank is 1.
void sm_chol(const zd *A, int lda, int k, zd *L, int ldl, double tol, int zero_row, int *dead, int *status,
             int flag_rank, cudaStream_t st, const zd *ref = nullptr, int ldref = 0);

// Hermitian eigendecomposition by cyclic Jacobi in working precision T (float or double),
// one CTA.  Eigenvalues w sorted decreasing (ties by index), eigenvectors U (k x k, FP64).
void sm_jacobi(bool fp64, const zd *A, int lda, int k, zd *U, int ldu, double *w, void *scratch, int max_sweeps,
               double tol, int *status, cudaStream_t st, void *Uf32 = nullptr, int nout = -1);
size_t sm_jacobi_scratch_bytes(int k);

// Top-r eigenpairs of the Hermitian k x k matrix M to FP64 accuracy: FP32 Jacobi, one
// block-Newton correction of the top-r invariant subspace, FP64 Rayleigh-Ritz on it
// (FP64 Jacobi of the r x r projection, at most max_sweeps sweeps; more sets ST_EIG_NOCONV).  Y (k x r, ld ldy) gets the eigenvectors,
// mu the eigenvalues, both sorted decreasing.  ws: see sm_eig_ws_bytes.
void sm_eig_topr(const zd *M, int ldm, int k, int r, zd *Y, int ldy, double *mu, void *ws, int *status,
                 cudaStream_t st, int max_sweeps = 30);
size_t sm_eig_ws_bytes(int kmax, int rmax);

// Elementwise helpers
void sm_copy(const zd *A, int lda, int M, int N, zd *B, int ldb, cudaStream_t st);
void sm_conj_transpose(const zd *A, int lda, int M, int N, zd *B, int ldb, cudaStream_t st);   // B = A^H
void sm_zero(zd *A, int lda, int M, int N, cudaStream_t st);
void sm_set_identity(zd *A, int lda, int M, int N, cudaStream_t st);                         // A = [I; 0]
void sm_hermitize(zd *A, int lda, int k, cudaStream_t st);                                  // A <- (A + A^H)/2
void sm_scale_cols(zd *A, int lda, int M, int N, double s, cudaStream_t st);
// Write the Hermitian Gram column block: G[0:k+r, k:k+r] = R and G[k:k+r, 0:k+r] = R^H.
void sm_store_gram_cols(const zd *R, int ldr, int k, int r, zd *G, int ldg, cudaStream_t st);

}  // namespace lrei
