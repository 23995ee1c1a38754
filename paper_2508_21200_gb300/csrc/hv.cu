// Matrix-free H.V for full rows of the N x r factor (paper Sec. 3.3, "sparsity of H";
// Hamiltonian of eq. H1 with exchange bonds and a Zeeman field along z).
//
// Row b of Y = H V is
//     d(b) V[b] + sum over bonds (i, j) whose spins are antiparallel in b of jxy_ij V[b ^ m_ij],
//     d(b) = c0 - sum_{antiparallel bonds} jz + bz (n/2 - popcount(b)),
// with m_ij the two bits of the bond.  All coefficients are real, so every 16-byte word of a
// row (two complex64 or one complex128) is updated independently.
//
// Work decomposition.  A CTA owns tiles of TR = 2^tb consecutive rows (about 32 KB), one tile
// at a time, and its threads own 16-byte words of rows (ch = row bytes / 16 threads per row,
// each thread the same word of RPT rows of the tile).
// Bonds fall into three classes relative to the tile bits:
//  * in-tile (both bits below tb): the partner row is in the same tile.  The tile is copied
//    into shared memory by the tensor-memory accelerator (bulk copy, mbarrier completion), and
//    which in-tile bonds are active on row lr depends only on lr, so a per-CTA table holds the
//    active set (a bitmask) and its diagonal contribution for every lr;
//  * outside (both bits at or above tb): active for every row of a tile or for none, with the
//    partner rows forming the tile t0 ^ m.  Per tile, the active ones and their diagonal
//    contribution are listed once; the thread then goes bond by bond, loading the partner words
//    of all its RPT rows as one group of independent 16-byte loads (read-only path, not
//    allocated in L1) before adding them, two bonds per iteration, so up to 2 RPT L2 requests
//    are in flight per thread;
//  * straddling (one bit on each side): activity per row from one low bit and one tile bit;
//    the partner row is loaded from global memory like an outside bond's.
// The own tile is single- or double-buffered (a template parameter; the library runs several
// single-buffered CTAs per SM, which overlap each other's copies).  Every wait on a copy is bounded; a wait that runs out sets ST_TIMEOUT, the tile
// is skipped, and before the kernel exits thread 0 waits (again bounded) for every copy it
// issued, so no copy is left in flight into released shared memory.
#include "common.cuh"

#include <cstring>

namespace lrei {

namespace {

template <typename T> struct W16;
template <> struct W16<float> { using V = float4; };
template <> struct W16<double> { using V = double2; };

__device__ __forceinline__ float4 ld_stream(const float4 *p) {
  float4 v;
  asm("ld.global.nc.L1::no_allocate.v4.f32 {%0, %1, %2, %3}, [%4];"
      : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "l"(p));
  return v;
}
__device__ __forceinline__ double2 ld_stream(const double2 *p) {
  double2 v;
  asm("ld.global.nc.L1::no_allocate.v2.f64 {%0, %1}, [%2];" : "=d"(v.x), "=d"(v.y) : "l"(p));
  return v;
}
__device__ __forceinline__ void axpy(float4 &a, float s, const float4 &p) {
  a.x = fmaf(s, p.x, a.x); a.y = fmaf(s, p.y, a.y); a.z = fmaf(s, p.z, a.z); a.w = fmaf(s, p.w, a.w);
}
__device__ __forceinline__ void axpy(double2 &a, double s, const double2 &p) {
  a.x = fma(s, p.x, a.x); a.y = fma(s, p.y, a.y);
}
// a += (sr + i si) p for the complex numbers of a 16-byte word
__device__ __forceinline__ void caxpy(float4 &a, float sr, float si, const float4 &p) {
  a.x = fmaf(sr, p.x, fmaf(-si, p.y, a.x)); a.y = fmaf(sr, p.y, fmaf(si, p.x, a.y));
  a.z = fmaf(sr, p.z, fmaf(-si, p.w, a.z)); a.w = fmaf(sr, p.w, fmaf(si, p.z, a.w));
}
__device__ __forceinline__ void caxpy(double2 &a, double sr, double si, const double2 &p) {
  a.x = fma(sr, p.x, fma(-si, p.y, a.x)); a.y = fma(sr, p.y, fma(si, p.x, a.y));
}
__device__ __forceinline__ float4 zero16(float4 *) { return make_float4(0.f, 0.f, 0.f, 0.f); }
__device__ __forceinline__ double2 zero16(double2 *) { return make_double2(0.0, 0.0); }

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Bounded wait for phase `parity` of an mbarrier: 2^22 polls with back-off (a few hundred ms).
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  for (int it = 0; it < (1 << 22); ++it) {
    uint32_t done;
    asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
                 : "=r"(done) : "r"(bar), "r"(parity) : "memory");
    if (done) return true;
    if (it > 32) __nanosleep(64);
  }
  return false;
}

}  // namespace

// Terms of the model sorted into the three classes for one tile size (built on the host).  A term
// is a bond (two bits: active on rows where they differ, diagonal share -jz when active) or a
// one-bit flip of the transverse field (always active).  Its amplitude depends on one bit of the
// output row, the selector: a0 when it is 0, a1 when it is 1 (a bond's selector is the bit of its
// site i, a one-bit term's its own bit; with real amplitudes a0 = a1).
constexpr int HV_MAX_TERMS = MAX_BONDS + MAX_SPINS;
struct HvPlan {
  long long N;
  int n, tb, ch;
  int nI, nS, nF;
  double c0, bz;
  // class order: in-tile [0, nI), straddling [nI, nI + nS), outside [nI + nS, nI + nS + nF)
  uint32_t mask[HV_MAX_TERMS];
  uint8_t bi[HV_MAX_TERMS], bj[HV_MAX_TERMS];   // low and high bit (equal for a one-bit term)
  uint8_t sb[HV_MAX_TERMS];                     // selector bit
  uint8_t two[HV_MAX_TERMS];                    // 1: bond, 0: one-bit term
  double jz[HV_MAX_TERMS];
  double a0r[HV_MAX_TERMS], a0i[HV_MAX_TERMS], a1r[HV_MAX_TERMS], a1i[HV_MAX_TERMS];
};

// RPT: rows per thread and tile (tile bytes / 16 / 256 threads; 8 for the 32 KB tiles of the
// launcher).  CPLX: complex amplitudes or one-bit terms present.  ROWMAJOR: each thread takes its
// rows one at a time and issues the outside partner loads of a row LIF at a time; otherwise it
// goes term by term over all its rows (RPT loads per term).  MINB: CTAs per SM to fit.
template <typename T, int NBUF, int RPT, bool CPLX, bool ROWMAJOR, int LIF, int MINB>
__global__ void __launch_bounds__(256, MINB) hv6_kernel(const __grid_constant__ HvPlan P,
                                                  const typename W16<T>::V *__restrict__ X,
                                                  typename W16<T>::V *__restrict__ Y, int *status) {
  using V = typename W16<T>::V;
  extern __shared__ __align__(128) unsigned char hv6_smem[];
  const int tb = P.tb, ch = P.ch;
  const uint32_t TR = 1u << tb;
  V *buf = reinterpret_cast<V *>(hv6_smem);                                           // [NBUF][TR][ch]
  unsigned long long *rmask = reinterpret_cast<unsigned long long *>(buf + (size_t)NBUF * TR * ch);   // [TR]
  T *rdiag = reinterpret_cast<T *>(rmask + TR);                                        // [TR]
  __shared__ __align__(8) unsigned long long bar[NBUF];
  __shared__ uint32_t imask[64], smask[HV_MAX_TERMS], fmask[HV_MAX_TERMS];
  __shared__ T i0r[64], i0i[64], i1r[64], i1i[64];                    // in-tile amplitudes
  __shared__ T s0r[HV_MAX_TERMS], s0i[HV_MAX_TERMS], s1r[HV_MAX_TERMS], s1i[HV_MAX_TERMS], sjz[HV_MAX_TERMS];
  __shared__ T fr[HV_MAX_TERMS], fi[HV_MAX_TERMS];                    // outside amplitudes on this tile
  __shared__ uint8_t isb[64], slo[HV_MAX_TERMS], ssb[HV_MAX_TERMS], sselin[HV_MAX_TERMS];
  __shared__ unsigned long long sflip, ssel;
  __shared__ T dconst;
  __shared__ int nfa;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int rp = nt / ch;                    // rows per pass
  const int slot = tid / ch, c = tid - slot * ch;
  const long long ntiles = P.N >> tb;
  const int nI = P.nI, nS = P.nS, nF = P.nF;

  // per-CTA tables: in-tile terms' active set and diagonal share for every row of a tile
  for (uint32_t lr = tid; lr < TR; lr += nt) {
    unsigned long long m = 0;
    double d = -P.bz * (double)__popc(lr);
    for (int k = 0; k < nI; ++k)
      if (!P.two[k] || (((lr >> P.bi[k]) ^ (lr >> P.bj[k])) & 1u)) {
        m |= 1ull << k;
        if (P.two[k]) d -= P.jz[k];
      }
    rmask[lr] = m;
    rdiag[lr] = (T)d;
  }
  for (int k = tid; k < nI; k += nt) {
    imask[k] = P.mask[k];
    i0r[k] = (T)P.a0r[k]; i0i[k] = (T)P.a0i[k]; i1r[k] = (T)P.a1r[k]; i1i[k] = (T)P.a1i[k];
    isb[k] = P.sb[k];
  }
  for (int k = tid; k < nS; k += nt) {
    const int q = nI + k;
    smask[k] = P.mask[q];
    s0r[k] = (T)P.a0r[q]; s0i[k] = (T)P.a0i[q]; s1r[k] = (T)P.a1r[q]; s1i[k] = (T)P.a1i[q];
    sjz[k] = (T)P.jz[q];
    slo[k] = P.bi[q];
    ssb[k] = P.sb[q];
    sselin[k] = P.sb[q] < tb ? 1 : 0;   // selector inside the tile (from the row) or a tile bit
  }
  if (tid == 0) {
    for (int i = 0; i < NBUF; ++i) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&bar[i])));
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncthreads();

  const uint32_t tile_bytes = TR * (uint32_t)ch * 16u;
  auto issue = [&](int b, long long tile) {   // thread 0 only
    const uint32_t ba = smem_u32(&bar[b]);
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(ba), "r"(tile_bytes) : "memory");
    const char *src = reinterpret_cast<const char *>(X) + (size_t)tile * tile_bytes;
    const uint32_t dst = smem_u32(buf + (size_t)b * TR * ch);
    for (uint32_t off = 0; off < tile_bytes; off += 16384u) {
      const uint32_t sz = (tile_bytes - off) < 16384u ? (tile_bytes - off) : 16384u;
      asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(dst + off),
                   "l"(src + off), "r"(sz), "r"(ba)
                   : "memory");
    }
  };

  int issued[NBUF], waited[NBUF];   // copies issued into / completions consumed from each buffer (thread 0)
#pragma unroll
  for (int i = 0; i < NBUF; ++i) issued[i] = waited[i] = 0;
  bool ok = true;
  int it = 0;
  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
    const int b = it % NBUF;
    const uint32_t t0 = (uint32_t)(tile << tb);
    if (tid == 0) {
      // the buffers written here were last read in an earlier iteration, which ended with a barrier
      asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
      if (it == 0) { issue(0, tile); ++issued[0]; }
      if (NBUF == 1 && it > 0) { issue(0, tile); ++issued[0]; }
      if (NBUF > 1 && tile + gridDim.x < ntiles) {
        const int nb = (it + 1) % NBUF;
        issue(nb, tile + gridDim.x);
        ++issued[nb];
      }
      // outside terms active on this tile with their amplitudes, the tile part of the diagonal,
      // the straddling bonds' tile bits
      double d = P.c0 + P.bz * (0.5 * P.n - (double)__popc(t0));
      int m = 0;
      for (int k = nI + nS; k < nI + nS + nF; ++k)
        if (!P.two[k] || (((t0 >> P.bi[k]) ^ (t0 >> P.bj[k])) & 1u)) {
          const bool s1 = (t0 >> P.sb[k]) & 1u;
          fmask[m] = P.mask[k];
          fr[m] = (T)(s1 ? P.a1r[k] : P.a0r[k]);
          fi[m] = (T)(s1 ? P.a1i[k] : P.a0i[k]);
          ++m;
          if (P.two[k]) d -= P.jz[k];
        }
      nfa = m;
      dconst = (T)d;
      unsigned long long f = 0, g = 0;
      for (int k = 0; k < nS; ++k) {
        if ((t0 >> P.bj[nI + k]) & 1u) f |= 1ull << k;
        if ((t0 >> P.sb[nI + k]) & 1u) g |= 1ull << k;
      }
      sflip = f;
      ssel = g;
    }
    __syncthreads();
    const bool got = mbar_wait(smem_u32(&bar[b]), (uint32_t)((it / NBUF) & 1));
    if (tid == 0 && got) ++waited[b];
    if (!__syncthreads_and(got)) {   // a copy did not arrive in time: every thread leaves the loop
      ok = false;
      break;
    }
    if (ROWMAJOR && slot < rp) {
      const V *own = buf + (size_t)b * TR * ch;
      const int nf = nfa;
      const T dc = dconst;
      const unsigned long long sf = sflip, sg = ssel;
      for (uint32_t lr = slot; lr < TR; lr += rp) {
        const uint32_t row = t0 + lr;
        T d = dc + rdiag[lr];
        V acc = zero16((V *)nullptr);
        // outside terms: LIF partner loads at a time, then their sums
        for (int f0 = 0; f0 < nf; f0 += LIF) {
          V p[LIF];
#pragma unroll
          for (int u = 0; u < LIF; ++u)
            if (f0 + u < nf) p[u] = ld_stream(X + (size_t)(row ^ fmask[f0 + u]) * ch + c);
#pragma unroll
          for (int u = 0; u < LIF; ++u)
            if (f0 + u < nf) {
              if constexpr (CPLX) caxpy(acc, fr[f0 + u], fi[f0 + u], p[u]);
              else axpy(acc, fr[f0 + u], p[u]);
            }
        }
        for (int k = 0; k < nS; ++k)
          if (((lr >> slo[k]) ^ (uint32_t)(sf >> k)) & 1u) {
            d -= sjz[k];
            const V pv = ld_stream(X + (size_t)(row ^ smask[k]) * ch + c);
            if constexpr (CPLX) {
              const bool s1 = sselin[k] ? ((lr >> ssb[k]) & 1u) : ((sg >> k) & 1u);
              caxpy(acc, s1 ? s1r[k] : s0r[k], s1 ? s1i[k] : s0i[k], pv);
            } else {
              axpy(acc, s0r[k], pv);
            }
          }
        unsigned long long am = rmask[lr];
        while (am) {
          const int k = __ffsll((long long)am) - 1;
          am &= am - 1;
          const V pv = own[(size_t)(lr ^ imask[k]) * ch + c];
          if constexpr (CPLX) {
            const bool s1 = (lr >> isb[k]) & 1u;
            caxpy(acc, s1 ? i1r[k] : i0r[k], s1 ? i1i[k] : i0i[k], pv);
          } else {
            axpy(acc, i0r[k], pv);
          }
        }
        axpy(acc, d, own[(size_t)lr * ch + c]);
        __stcs(Y + (size_t)row * ch + c, acc);   // streaming: keep V, not Y, in L2
      }
    }
    if (!ROWMAJOR && slot < rp) {
      const V *own = buf + (size_t)b * TR * ch;
      const int nf = nfa;
      const T dc = dconst;
      const unsigned long long sf = sflip, sg = ssel;
      // rows of this thread in the tile: lr_i = slot + i rp, i < RPT
      V acc[RPT];
#pragma unroll
      for (int i = 0; i < RPT; ++i) acc[i] = zero16((V *)nullptr);
      // outside terms, term by term: the partner rows of all the thread's rows are one group of
      // independent loads (two terms per iteration: up to 2 RPT loads in flight per thread)
      const size_t step = (size_t)rp * ch;
#pragma unroll 2
      for (int f = 0; f < nf; ++f) {
        // partner of row t0 + lr is (t0 + lr) ^ m = (t0 ^ m) + lr (m has no bits below tb): the
        // partner tile starts at row t0 ^ m, which is below N
        const V *xp = X + ((size_t)(t0 ^ fmask[f]) + (size_t)slot) * ch + c;
        const T ar = fr[f], ai = fi[f];
        V p[RPT];
#pragma unroll
        for (int i = 0; i < RPT; ++i)
          if (slot + i * rp < (int)TR) p[i] = ld_stream(xp + i * step);
#pragma unroll
        for (int i = 0; i < RPT; ++i)
          if (slot + i * rp < (int)TR) {
            if constexpr (CPLX) caxpy(acc[i], ar, ai, p[i]);
            else axpy(acc[i], ar, p[i]);
          }
      }
#pragma unroll
      for (int i = 0; i < RPT; ++i) {
        const uint32_t lr = (uint32_t)(slot + i * rp);
        if (lr >= TR) continue;
        const uint32_t row = t0 + lr;
        T d = dc + rdiag[lr];
        // straddling bonds: active when the row's low bit differs from the tile's high bit
        for (int k = 0; k < nS; ++k)
          if (((lr >> slo[k]) ^ (uint32_t)(sf >> k)) & 1u) {
            d -= sjz[k];
            const V pv = ld_stream(X + (size_t)(row ^ smask[k]) * ch + c);
            if constexpr (CPLX) {
              const bool s1 = sselin[k] ? ((lr >> ssb[k]) & 1u) : ((sg >> k) & 1u);
              caxpy(acc[i], s1 ? s1r[k] : s0r[k], s1 ? s1i[k] : s0i[k], pv);
            } else {
              axpy(acc[i], s0r[k], pv);
            }
          }
        // in-tile terms from shared memory
        unsigned long long am = rmask[lr];
        while (am) {
          const int k = __ffsll((long long)am) - 1;
          am &= am - 1;
          const V pv = own[(size_t)(lr ^ imask[k]) * ch + c];
          if constexpr (CPLX) {
            const bool s1 = (lr >> isb[k]) & 1u;
            caxpy(acc[i], s1 ? i1r[k] : i0r[k], s1 ? i1i[k] : i0i[k], pv);
          } else {
            axpy(acc[i], i0r[k], pv);
          }
        }
        axpy(acc[i], d, own[(size_t)lr * ch + c]);
        __stcs(Y + (size_t)row * ch + c, acc[i]);
      }
    }
    __syncthreads();   // buffer b and the per-tile lists are free again
  }
  // drain: no copy may still be in flight when the CTA releases its shared memory
  if (tid == 0) {
    for (int i = 0; i < NBUF; ++i)
      while (waited[i] < issued[i]) {
        const bool got = mbar_wait(smem_u32(&bar[i]), (uint32_t)(waited[i] & 1));
        ++waited[i];
        ok = ok && got;
      }
  }
  if (!ok && status) atomicOr(status, ST_TIMEOUT);
}

// ---------------------------------------------------------------- launcher
constexpr int HV6_RPT = 8;   // rows per thread and tile at the launcher's tile sizes (see hv6_tile_bits)
// the configuration the library launches (measured best of row/term order, 1-2 own-tile buffers,
// 4-8 loads in flight and 2-6 CTAs per SM at n = 18 and 20): row-major, one own-tile buffer per
// CTA (the 5 CTAs of an SM overlap each other's copies), 6 outside partner loads in flight per
// thread, 5 CTAs per SM
constexpr int HV6_NBUF = 1, HV6_LIF = 6, HV6_MINB = 5;
constexpr bool HV6_ROWMAJOR = true;

template <typename T, bool CPLX>
constexpr auto hv6_product = hv6_kernel<T, HV6_NBUF, HV6_RPT, CPLX, HV6_ROWMAJOR, HV6_LIF, HV6_MINB>;

template <typename T>
size_t hv6_smem_bytes(int tb, int ch, int nbuf) {
  const size_t TR = (size_t)1 << tb;
  return (size_t)nbuf * TR * ch * 16 + TR * (8 + sizeof(T));
}

namespace {
int g_hv6_occ[2][2] = {{0, 0}, {0, 0}};   // [fp64][cplx]: CTAs per SM of the product kernel
}  // namespace

// Tile bits for a row of `rowb` bytes: about 32 KB of rows per tile, at most all N rows.
static int hv6_tile_bits(int n, size_t rowb) {
  int tb = 0;
  while (((size_t)2 << tb) * rowb <= 32768) ++tb;
  return tb < n ? tb : n;
}

int hv6_init() {
  const int lim = 200 * 1024;
  cudaError_t e = cudaSuccess;
  auto set = [&](const void *f) {
    const cudaError_t x = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    if (x != cudaSuccess) e = x;
  };
  set((const void *)hv6_product<float, false>);
  set((const void *)hv6_product<double, false>);
  set((const void *)hv6_product<float, true>);
  set((const void *)hv6_product<double, true>);
  if (e != cudaSuccess) return -1;
  // occupancy at the standard tile size (32 KB per tile buffer)
  int o = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, hv6_product<float, false>, 256, hv6_smem_bytes<float>(8, 8, HV6_NBUF));
  g_hv6_occ[0][0] = o > 0 ? o : 1;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, hv6_product<float, true>, 256, hv6_smem_bytes<float>(8, 8, HV6_NBUF));
  g_hv6_occ[0][1] = o > 0 ? o : 1;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, hv6_product<double, false>, 256, hv6_smem_bytes<double>(7, 16, HV6_NBUF));
  g_hv6_occ[1][0] = o > 0 ? o : 1;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, hv6_product<double, true>, 256, hv6_smem_bytes<double>(7, 16, HV6_NBUF));
  g_hv6_occ[1][1] = o > 0 ? o : 1;
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// The terms of the model sorted for a tile size (tile_bits > 0 overrides the 32 KB default).
// Returns false when hv6 does not apply: row bytes not a multiple of 16, fewer than 16 rows per
// tile, or more than 64 terms inside a tile.
bool hv6_plan(bool fp64, const ModelArgs &M, long long N, int r, int tile_bits, HvPlan *Pout) {
  const size_t rowb = (size_t)r * (fp64 ? 16 : 8);
  if (rowb % 16 != 0 || rowb / 16 > 256) return false;
  int tb = tile_bits > 0 ? (tile_bits < M.n ? tile_bits : M.n) : hv6_tile_bits(M.n, rowb);
  const int rp = 256 / (int)(rowb / 16);
  while (tb > 0 && (((1 << tb) + rp - 1) / rp) > HV6_RPT) --tb;   // every row of a tile has a thread
  if (tb < 4 || M.nb > MAX_BONDS) return false;
  // the terms: the bonds, then (with a transverse field) one one-bit flip per spin
  const bool field = M.cplx && (M.bx != 0.0 || M.by != 0.0);
  const int nterm = M.nb + (field ? M.n : 0);
  HvPlan &P = *Pout;
  std::memset(&P, 0, sizeof(P));
  P.N = N;
  P.n = M.n;
  P.tb = tb;
  P.ch = (int)(rowb / 16);
  P.c0 = M.c0;
  P.bz = M.bz;
  int cnt[3] = {0, 0, 0};
  int cls[HV_MAX_TERMS];
  auto term_mask = [&](int k) -> uint32_t { return k < M.nb ? M.mask[k] : (1u << (k - M.nb)); };
  for (int k = 0; k < nterm; ++k) {
    const uint32_t m = term_mask(k), lo = m & ((1u << tb) - 1u), hi = m >> tb;
    cls[k] = hi == 0 ? 0 : (lo == 0 ? 2 : 1);
    ++cnt[cls[k]];
  }
  if (cnt[0] > 64) return false;   // the per-row active set is a 64-bit mask
  P.nI = cnt[0];
  P.nS = cnt[1];
  P.nF = cnt[2];
  int pos[3] = {0, cnt[0], cnt[0] + cnt[1]};
  for (int k = 0; k < nterm; ++k) {
    const int q = pos[cls[k]]++;
    P.mask[q] = term_mask(k);
    if (k < M.nb) {
      uint8_t a = M.bi[k], b = M.bj[k];
      if (a > b) { const uint8_t t = a; a = b; b = t; }
      P.bi[q] = a;   // lower bit (inside the tile for a straddling bond)
      P.bj[q] = b;
      P.sb[q] = M.bi[k];   // site i's bit selects jxy + i dz (bit 0) or jxy - i dz (bit 1)
      P.two[q] = 1;
      P.jz[q] = M.jz[k];
      P.a0r[q] = M.jxy[k];
      P.a1r[q] = M.jxy[k];
      P.a0i[q] = M.cplx ? M.dz[k] : 0.0;
      P.a1i[q] = M.cplx ? -M.dz[k] : 0.0;
    } else {
      const uint8_t bit = (uint8_t)(k - M.nb);
      P.bi[q] = P.bj[q] = P.sb[q] = bit;
      P.two[q] = 0;
      P.a0r[q] = P.a1r[q] = 0.5 * M.bx;
      P.a0i[q] = -0.5 * M.by;
      P.a1i[q] = 0.5 * M.by;
    }
  }
  return true;
}

// Returns true when the launch was made; false when the caller must use another kernel.
bool launch_hv6(bool fp64, const ModelArgs &M, const void *X, void *Y, long long N, int r, int nsm, cudaStream_t st,
                int *status, int tile_bits) {
  if ((reinterpret_cast<uintptr_t>(X) & 15) || (reinterpret_cast<uintptr_t>(Y) & 15) || X == Y) return false;
  HvPlan P;
  if (!hv6_plan(fp64, M, N, r, tile_bits, &P)) return false;
  const size_t smem = fp64 ? hv6_smem_bytes<double>(P.tb, P.ch, HV6_NBUF) : hv6_smem_bytes<float>(P.tb, P.ch, HV6_NBUF);
  if (smem > 200 * 1024) return false;
  const int occ = g_hv6_occ[fp64 ? 1 : 0][M.cplx ? 1 : 0];
  const long long ntiles = N >> P.tb;
  const long long cap = (long long)(occ > 0 ? occ : 1) * nsm;
  const int grid = (int)(ntiles < cap ? ntiles : cap);
  ::lrei::count_launch();
  if (fp64) {
    auto kern = M.cplx ? hv6_product<double, true> : hv6_product<double, false>;
    kern<<<grid, 256, smem, st>>>(P, reinterpret_cast<const double2 *>(X), reinterpret_cast<double2 *>(Y), status);
  } else {
    auto kern = M.cplx ? hv6_product<float, true> : hv6_product<float, false>;
    kern<<<grid, 256, smem, st>>>(P, reinterpret_cast<const float4 *>(X), reinterpret_cast<float4 *>(Y), status);
  }
  return true;
}

}  // namespace lrei
