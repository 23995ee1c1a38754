// Tall-skinny (N-length) kernels: launch interface.
#pragma once
#include "common.cuh"

namespace lrei {

// One fused pass over N rows, tiled by `tr` rows per CTA iteration.
//  mode 0 (apply):   S = (apply_h ? H src : src); optionally write S to out;
//                    Gram = [q_0 .. q_{gram_left-1}, S]^* S
//  mode 1 (extend):  S as above; new = S coefS + sum_m q_m coefQ_m; write new;
//                    Gram = [q_0 .. q_{gram_left-1}, new]^* new
//  mode 2 (combine): new = sum_m q_m coefQ_m; write new; Gram = [q_0..q_{gram_left-1}, new]^* new
// coefQ is (nq*r) x r column-major (ld = nq*r), coefS r x r column-major, both complex double.
// The per-CTA Gram partials ((gram_left+1)*r x r complex, column-major) go to
// partial[blockIdx.x]; reduce_partials() sums them in a fixed order.
struct TSArgs {
  long long N;
  int r;
  int nq;
  int gram_left;
  const void *q[MAXB];
  const void *src;
  int apply_h;
  const zd *coefS;
  const zd *coefQ;
  void *out;
  double *partial;
  int mode;
  void *coef_scratch;   // device, >= (MAXB+1)*MAX_R*MAX_R*16 bytes (converted coefficients)
  long long zero_rows;  // modes 1, 2: rows < zero_rows of the new block are set to zero
};

// Returns the grid size used (number of partials written), or -1 on error.
int launch_ts(bool fp64, const ModelArgs &M, const TSArgs &a, int nsm, cudaStream_t st);
int ts_max_grid(int nsm);
int ts_init();
size_t ts_partial_doubles(int gram_left, int r);   // per CTA

void launch_reduce(const double *partial, int nparts, int len_doubles, double *out, cudaStream_t st);

// Y = H X (standalone matrix-free action), X, Y: N x r row-major of the given precision.
void launch_hv(bool fp64, const ModelArgs &M, const void *X, void *Y, long long N, int r, int nsm, cudaStream_t st,
               int *status = nullptr);

// Full-row matrix-free H.V (hv.cu): returns false when the layout does not apply.
// tile_bits > 0 overrides the tile size (rows = 2^tile_bits), else about 32 KB per tile.
bool launch_hv_tiled(bool fp64, const ModelArgs &M, const void *X, void *Y, long long N, int r, int nsm, cudaStream_t st,
                int *status, int tile_bits = 0);
int hv_tiled_init();
// Y = M_z X (which = 0) or Y = (M_x + i M_y) X (which = 1) on full rows (hv.cu); false when the
// layout does not apply.
bool launch_magnetization(bool fp64, int which, int n, const void *X, void *Y, long long N, int r, int nsm,
                          cudaStream_t st, int *status);


// Observable Grams of V (N x r): blocks (column-major r x r each, complex double):
//   0: V^*HV  1: (HV)^*(HV)  2: V^*V  3: V^* Mx V  4: V^* My V  5: V^* Mz V
int launch_obs(bool fp64, const ModelArgs &M, const void *V, long long N, int r, double *partial, int nsm,
               cudaStream_t st);

// Convert / copy an N x r factor with row stride ld (dtype c128 or c64) into the internal
// contiguous layout of the given precision.
void launch_convert(const void *src, int src_c64, int ld, void *dst, int dst_fp64, long long N, int r,
                    cudaStream_t st);

// Checks every element of an N x r block for NaN/Inf; ORs ST_NONFINITE into *status.
void launch_check_finite(bool fp64, const void *X, long long N, int r, int *status, cudaStream_t st);

}  // namespace lrei
