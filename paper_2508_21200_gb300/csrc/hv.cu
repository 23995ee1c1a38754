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
// at a time; thread (slot, c) of its 8 consumer warps owns 16-byte word c of rows slot + i rp
// (ch = row bytes / 16 words per row, rp = 256 / ch rows per pass).  Terms fall into three
// classes relative to the tile bits:
//  * in-tile (both bits below tb): the partner row is in the same tile; which in-tile terms
//    are active on row lr depends only on lr, so a per-CTA table holds the active set (a
//    bitmask) and its diagonal share for every lr;
//  * outside (both bits at or above tb): active for every row of a tile or for none, with the
//    partner rows forming the whole tile t0 ^ m;
//  * straddling (one bit on each side): active on the rows whose low bit differs from the
//    tile's high bit; their partners fill half of tile t0 ^ m (a contiguous half when the low
//    bit is the top row bit).
// The own tile and every partner tile needed by the tile are brought into shared memory by
// bulk copies (hv7_kernel below), so the bytes in flight are bounded by shared memory rather
// than by registers.  Every wait on a copy is bounded; see the kernel's comment for the error
// path.
#include "common.cuh"

#include <cstring>

namespace lrei {

namespace {

template <typename T> struct W16;
template <> struct W16<float> { using V = float4; };
template <> struct W16<double> { using V = double2; };

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

// ------------------------------------------------------- hv7: partner tiles by bulk copy
// The rows of an outside term's partners form one whole tile (t0 ^ m), and those of a straddling
// bond half of one (the rows whose low bit equals the tile's high bit).  hv7 brings every partner
// tile into shared memory with bulk copies instead of per-thread loads, so the bytes in flight
// are bounded by shared memory rather than by registers: a ring of NB tile buffers, filled by one
// producer warp (one elected lane issues the copies; a full barrier per buffer counts the bytes)
// and drained by 8 consumer warps (an empty barrier per buffer counts the warps that are done).
// Per tile the chunks are the own tile, then each straddling bond's half or whole partner tile,
// then each outside term active on the tile; the consumers keep the tile's output words in
// registers across its chunks and store them once.  Every wait is bounded: a consumer or the
// producer that gives up sets ST_TIMEOUT and a shared abort flag that ends everyone's loop, and
// the producer waits (bounded) for each buffer's last copy before the CTA exits.
template <typename T, int NB, int RPT, bool CPLX, int MINB, int SUSP = 0, int NCW = 8>
__global__ void __launch_bounds__(NCW * 32 + 32, MINB) hv7_kernel(const __grid_constant__ HvPlan P,
                                                  const typename W16<T>::V *__restrict__ X,
                                                  typename W16<T>::V *__restrict__ Y, int *status) {
  using V = typename W16<T>::V;
  extern __shared__ __align__(128) unsigned char hv7_smem[];
  const int tb = P.tb, ch = P.ch;
  const uint32_t TR = 1u << tb;
  V *buf = reinterpret_cast<V *>(hv7_smem);                                                   // [NB][TR][ch]
  unsigned long long *rmask = reinterpret_cast<unsigned long long *>(buf + (size_t)NB * TR * ch);   // [TR]
  T *rdiag = reinterpret_cast<T *>(rmask + TR);                                                // [TR]
  __shared__ __align__(8) unsigned long long full[NB], empty[NB];
  __shared__ volatile int abort_flag;
  __shared__ uint32_t imask[64];
  __shared__ T i0r[64], i0i[64], i1r[64], i1i[64];
  __shared__ uint8_t isb[64];
  __shared__ uint32_t shi[HV_MAX_TERMS];   // straddling: partner tile offset (mask >> tb)
  __shared__ uint8_t slo[HV_MAX_TERMS], shb[HV_MAX_TERMS], ssb[HV_MAX_TERMS], ssel_in[HV_MAX_TERMS];
  __shared__ T sjz[HV_MAX_TERMS], s0r[HV_MAX_TERMS], s0i[HV_MAX_TERMS], s1r[HV_MAX_TERMS], s1i[HV_MAX_TERMS];
  __shared__ uint32_t fhi[HV_MAX_TERMS];   // outside: partner tile offset (mask >> tb)
  __shared__ uint8_t fbi[HV_MAX_TERMS], fbj[HV_MAX_TERMS], ftwo[HV_MAX_TERMS], fsb[HV_MAX_TERMS];
  __shared__ T f0r[HV_MAX_TERMS], f0i[HV_MAX_TERMS], f1r[HV_MAX_TERMS], f1i[HV_MAX_TERMS];
  const int tid = threadIdx.x;
  const long long ntiles = P.N >> tb;
  const int nI = P.nI, nS = P.nS, nF = P.nF;
  const uint32_t TB = TR * (uint32_t)ch * 16u;   // tile bytes

  for (uint32_t lr = tid; lr < TR; lr += blockDim.x) {
    unsigned long long m = 0;
    double d = -P.bz * (double)__popc(lr);
    for (int k = 0; k < nI; ++k)
      if (!P.two[k] || (((lr >> P.bi[k]) ^ (lr >> P.bj[k])) & 1u)) {
        if (P.two[k]) d -= P.jz[k];
        // a term whose amplitude on this row is zero keeps its diagonal share but reads no partner
        const bool s1 = (lr >> P.sb[k]) & 1u;
        if (s1 ? (P.a1r[k] != 0.0 || P.a1i[k] != 0.0) : (P.a0r[k] != 0.0 || P.a0i[k] != 0.0)) m |= 1ull << k;
      }
    rmask[lr] = m;
    rdiag[lr] = (T)d;
  }
  for (int k = tid; k < nI; k += blockDim.x) {
    imask[k] = P.mask[k];
    i0r[k] = (T)P.a0r[k]; i0i[k] = (T)P.a0i[k]; i1r[k] = (T)P.a1r[k]; i1i[k] = (T)P.a1i[k];
    isb[k] = P.sb[k];
  }
  for (int k = tid; k < nS; k += blockDim.x) {
    const int q = nI + k;
    shi[k] = P.mask[q] >> tb;
    slo[k] = P.bi[q];
    shb[k] = P.bj[q];
    ssb[k] = P.sb[q];
    ssel_in[k] = P.sb[q] < tb ? 1 : 0;
    sjz[k] = (T)P.jz[q];
    s0r[k] = (T)P.a0r[q]; s0i[k] = (T)P.a0i[q]; s1r[k] = (T)P.a1r[q]; s1i[k] = (T)P.a1i[q];
  }
  for (int k = tid; k < nF; k += blockDim.x) {
    const int q = nI + nS + k;
    fhi[k] = P.mask[q] >> tb;
    fbi[k] = P.bi[q];
    fbj[k] = P.bj[q];
    ftwo[k] = P.two[q];
    fsb[k] = P.sb[q];
    f0r[k] = (T)P.a0r[q]; f0i[k] = (T)P.a0i[q]; f1r[k] = (T)P.a1r[q]; f1i[k] = (T)P.a1i[q];
  }
  if (tid == 0) {
    abort_flag = 0;
    for (int i = 0; i < NB; ++i) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&full[i])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(&empty[i])), "r"(NCW));
    }
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncthreads();

  // a straddling bond copies the half of its partner tile that holds the partners (rows whose
  // bit slo equals the tile's bit) when slo is the top row bit, else the whole tile
  auto half_of = [&](int s) { return (int)slo[s] == tb - 1; };
  auto outside_active = [&](int f, uint32_t t0) {   // the term acts on the tile (diagonal share)
    return !ftwo[f] || (((t0 >> fbi[f]) ^ (t0 >> fbj[f])) & 1u);
  };
  auto outside_load = [&](int f, uint32_t t0) {     // ... and its amplitude there is nonzero
    if (!outside_active(f, t0)) return false;
    const bool s1 = (t0 >> fsb[f]) & 1u;
    return s1 ? (f1r[f] != (T)0 || f1i[f] != (T)0) : (f0r[f] != (T)0 || f0i[f] != (T)0);
  };
  // bounded wait that also gives up once another warp has aborted
  auto wait_bar = [&](unsigned long long *bar, uint32_t parity) -> bool {
    const uint32_t a = smem_u32(bar);
    for (int it = 0; it < (SUSP ? (1 << 16) : (1 << 22)); ++it) {
      uint32_t done;
      if constexpr (SUSP > 0) {
        // the waiting thread may be suspended for up to SUSP ns instead of spinning on issue slots
        asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\nselp.u32 %0, 1, 0, p;\n}\n"
                     : "=r"(done) : "r"(a), "r"(parity), "r"((uint32_t)SUSP) : "memory");
      } else {
        asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
                     : "=r"(done) : "r"(a), "r"(parity) : "memory");
      }
      if (done) return true;
      if (abort_flag) return false;
      if (!SUSP && it > 32) __nanosleep(64);
    }
    return false;
  };

  if (tid >= NCW * 32) {
    // ---- producer warp: lane 0 issues every copy of the CTA's chunk sequence
    if (tid != NCW * 32) return;
    int last_u[NB];
#pragma unroll
    for (int i = 0; i < NB; ++i) last_u[i] = -1;
    bool ok = true;
    long long k = 0;
    auto issue = [&](long long ptile, uint32_t off, uint32_t bytes) -> bool {
      const int b = (int)(k % NB);
      const int u = (int)(k / NB);
      if (u > 0 && !wait_bar(&empty[b], (uint32_t)((u - 1) & 1))) return false;
      asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
      const uint32_t fb = smem_u32(&full[b]);
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(fb), "r"(bytes) : "memory");
      const char *src = reinterpret_cast<const char *>(X) + (size_t)ptile * TB + off;
      const uint32_t dst = smem_u32(buf + (size_t)b * TR * ch);
      for (uint32_t o = 0; o < bytes; o += 16384u) {
        const uint32_t sz = (bytes - o) < 16384u ? (bytes - o) : 16384u;
        asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(dst + o),
                     "l"(src + o), "r"(sz), "r"(fb)
                     : "memory");
      }
      last_u[b] = u;
      ++k;
      return true;
    };
    for (long long tile = blockIdx.x; ok && tile < ntiles; tile += gridDim.x) {
      const uint32_t t0 = (uint32_t)(tile << tb);
      ok = issue(tile, 0, TB);
      for (int s = 0; ok && s < nS; ++s) {
        const uint32_t tbit = (t0 >> shb[s]) & 1u;
        const bool h = half_of(s);
        ok = issue(tile ^ (long long)shi[s], h ? (tbit ? TB / 2 : 0u) : 0u, h ? TB / 2 : TB);
      }
      for (int f = 0; ok && f < nF; ++f)
        if (outside_load(f, t0)) ok = issue(tile ^ (long long)fhi[f], 0, TB);
    }
    if (!ok) abort_flag = 1;
    // drain: every buffer's last copy has landed before the CTA releases its shared memory
    for (int b = 0; b < NB; ++b)
      if (last_u[b] >= 0) {
        const uint32_t a = smem_u32(&full[b]);
        bool got = false;
        for (int it = 0; it < (1 << 22) && !got; ++it) {
          uint32_t done;
          asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
                       : "=r"(done) : "r"(a), "r"((uint32_t)(last_u[b] & 1)) : "memory");
          got = done != 0;
          if (!got && it > 32) __nanosleep(64);
        }
        ok = ok && got;
      }
    if (!ok && status) atomicOr(status, ST_TIMEOUT);
    return;
  }

  // ---- consumer warps: thread (slot, c) owns word c of rows slot + i rp of every tile
  const int rp = NCW * 32 / ch;
  const int slot = tid / ch, c = tid - slot * ch;
  const bool active_thread = slot < rp;
  const int lane = tid & 31;
  bool ok = true;
  long long k = 0;
  auto take = [&]() -> const V * {   // wait for chunk k; returns its buffer (null for the whole warp on a timeout)
    const int b = (int)(k % NB);
    const bool got = wait_bar(&full[b], (uint32_t)((k / NB) & 1));
    if (!__all_sync(0xffffffffu, got)) return nullptr;
    return buf + (size_t)b * TR * ch;
  };
  auto release = [&]() {
    __syncwarp();
    if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_u32(&empty[k % NB])) : "memory");
    ++k;
  };
  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const uint32_t t0 = (uint32_t)(tile << tb);
    // tile-level parts: the diagonal's constant and outside shares, the straddling bonds' tile bits
    double dcd = P.c0 + P.bz * (0.5 * P.n - (double)__popc(t0));
    for (int f = 0; f < nF; ++f)
      if (ftwo[f] && outside_active(f, t0)) dcd -= P.jz[nI + nS + f];
    const T dc = (T)dcd;
    unsigned long long sf = 0, sg = 0;
    for (int s = 0; s < nS; ++s) {
      sf |= (unsigned long long)((t0 >> shb[s]) & 1u) << s;
      sg |= (unsigned long long)((t0 >> ssb[s]) & 1u) << s;
    }
    V acc[RPT];
    // own tile: diagonal and in-tile terms
    const V *own = take();
    if (!own) { ok = false; break; }
    if (active_thread) {
#pragma unroll
      for (int i = 0; i < RPT; ++i) {
        const uint32_t lr = (uint32_t)(slot + i * rp);
        acc[i] = zero16((V *)nullptr);
        if (lr >= TR) continue;
        T d = dc + rdiag[lr];
        for (int s = 0; s < nS; ++s)
          if (((lr >> slo[s]) ^ (uint32_t)(sf >> s)) & 1u) d -= sjz[s];
        V a = zero16((V *)nullptr);
        axpy(a, d, own[(size_t)lr * ch + c]);
        unsigned long long am = rmask[lr];
        while (am) {
          const int q = __ffsll((long long)am) - 1;
          am &= am - 1;
          const V pv = own[(size_t)(lr ^ imask[q]) * ch + c];
          if constexpr (CPLX) {
            const bool s1 = (lr >> isb[q]) & 1u;
            caxpy(a, s1 ? i1r[q] : i0r[q], s1 ? i1i[q] : i0i[q], pv);
          } else {
            axpy(a, i0r[q], pv);
          }
        }
        acc[i] = a;
      }
    }
    release();
    // straddling bonds: active on the rows whose bit slo differs from the tile's bit
    for (int s = 0; s < nS; ++s) {
      const V *pb = take();
      if (!pb) { ok = false; break; }
      if (active_thread) {
        const uint32_t tbit = (uint32_t)(sf >> s) & 1u, lo = slo[s];
        const uint32_t base = (lo == (uint32_t)(tb - 1) && tbit) ? TR / 2 : 0u;
        const bool selin = ssel_in[s];
        const bool sgt = (sg >> s) & 1u;
#pragma unroll
        for (int i = 0; i < RPT; ++i) {
          const uint32_t lr = (uint32_t)(slot + i * rp);
          if (lr >= TR || !(((lr >> lo) ^ tbit) & 1u)) continue;
          const V pv = pb[(size_t)((lr ^ (1u << lo)) - base) * ch + c];
          if constexpr (CPLX) {
            const bool s1 = selin ? ((lr >> ssb[s]) & 1u) : sgt;
            caxpy(acc[i], s1 ? s1r[s] : s0r[s], s1 ? s1i[s] : s0i[s], pv);
          } else {
            axpy(acc[i], s0r[s], pv);
          }
        }
      }
      release();
    }
    if (!ok) break;
    // outside terms active on this tile: the whole partner tile, one amplitude
    for (int f = 0; f < nF; ++f) {
      if (!outside_load(f, t0)) continue;
      const V *pb = take();
      if (!pb) { ok = false; break; }
      if (active_thread) {
        const bool s1 = (t0 >> fsb[f]) & 1u;
        const T ar = s1 ? f1r[f] : f0r[f], ai = s1 ? f1i[f] : f0i[f];
#pragma unroll
        for (int i = 0; i < RPT; ++i) {
          const uint32_t lr = (uint32_t)(slot + i * rp);
          if (lr >= TR) continue;
          if constexpr (CPLX) caxpy(acc[i], ar, ai, pb[(size_t)lr * ch + c]);
          else axpy(acc[i], ar, pb[(size_t)lr * ch + c]);
        }
      }
      release();
    }
    if (!ok) break;
    if (active_thread) {
#pragma unroll
      for (int i = 0; i < RPT; ++i) {
        const uint32_t lr = (uint32_t)(slot + i * rp);
        if (lr < TR) __stcs(Y + (size_t)(t0 + lr) * ch + c, acc[i]);
      }
    }
  }
  if (!ok) {
    abort_flag = 1;
    if (status && lane == 0) atomicOr(status, ST_TIMEOUT);
  }
}

template <typename T>
size_t hv7_smem_bytes(int tb, int ch, int nb) {
  const size_t TR = (size_t)1 << tb;
  return (size_t)nb * TR * ch * 16 + TR * (8 + sizeof(T));
}

// ---------------------------------------------------------------- launcher
constexpr int HV_RPT = 8;   // rows per thread and tile at the launcher's tile sizes (see hv_tile_bits)
// the configuration the library launches (measured best of 1-6 tile buffers and 1-6 CTAs per SM,
// 16 and 32 KB tiles, at n = 14..20 in both precisions): 32 KB tiles, two buffers per CTA, three
// CTAs per SM, waits that suspend the thread for up to 2 us per poll
constexpr int HV_NB = 2, HV_MINB = 3, HV_SUSP = 2000;

template <typename T, bool CPLX>
constexpr auto hv_product = hv7_kernel<T, HV_NB, HV_RPT, CPLX, HV_MINB, HV_SUSP>;

namespace {
int g_hv_occ[2][2] = {{0, 0}, {0, 0}};   // [fp64][cplx]: CTAs per SM of the product kernel
}  // namespace

// Tile bits for a row of `rowb` bytes: about 32 KB of rows per tile, at most all N rows.
static int hv_tile_bits(int n, size_t rowb) {
  int tb = 0;
  while (((size_t)2 << tb) * rowb <= 32768) ++tb;
  return tb < n ? tb : n;
}

int hv_tiled_init() {
  const int lim = 200 * 1024;
  cudaError_t e = cudaSuccess;
  auto set = [&](const void *f) {
    const cudaError_t x = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    if (x != cudaSuccess) e = x;
  };
  set((const void *)hv_product<float, false>);
  set((const void *)hv_product<double, false>);
  set((const void *)hv_product<float, true>);
  set((const void *)hv_product<double, true>);
  if (e != cudaSuccess) return -1;
  // occupancy at the standard tile size (32 KB per tile buffer)
  int o = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, hv_product<float, false>, 288, hv7_smem_bytes<float>(8, 8, HV_NB));
  g_hv_occ[0][0] = o > 0 ? o : 1;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, hv_product<float, true>, 288, hv7_smem_bytes<float>(8, 8, HV_NB));
  g_hv_occ[0][1] = o > 0 ? o : 1;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, hv_product<double, false>, 288, hv7_smem_bytes<double>(7, 16, HV_NB));
  g_hv_occ[1][0] = o > 0 ? o : 1;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, hv_product<double, true>, 288, hv7_smem_bytes<double>(7, 16, HV_NB));
  g_hv_occ[1][1] = o > 0 ? o : 1;
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// The terms of the model sorted for a tile size (tile_bits > 0 overrides the 32 KB default).
// Returns false when the tiled kernel does not apply: row bytes not a multiple of 16, fewer than 16 rows per
// tile, or more than 64 terms inside a tile.
bool hv_plan(bool fp64, const ModelArgs &M, long long N, int r, int tile_bits, HvPlan *Pout) {
  const size_t rowb = (size_t)r * (fp64 ? 16 : 8);
  if (rowb % 16 != 0 || rowb / 16 > 256) return false;
  int tb = tile_bits > 0 ? (tile_bits < M.n ? tile_bits : M.n) : hv_tile_bits(M.n, rowb);
  const int rp = 256 / (int)(rowb / 16);
  while (tb > 0 && (((1 << tb) + rp - 1) / rp) > HV_RPT) --tb;   // every row of a tile has a thread
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

// One launch of the product kernel for a built plan (cplx: complex or row-dependent amplitudes).
static bool launch_hv_plan(bool fp64, bool cplx, const HvPlan &P, const void *X, void *Y, int nsm, cudaStream_t st,
                           int *status) {
  if ((reinterpret_cast<uintptr_t>(X) & 15) || (reinterpret_cast<uintptr_t>(Y) & 15) || X == Y) return false;
  const size_t smem = fp64 ? hv7_smem_bytes<double>(P.tb, P.ch, HV_NB) : hv7_smem_bytes<float>(P.tb, P.ch, HV_NB);
  if (smem > 200 * 1024) return false;
  const int occ = g_hv_occ[fp64 ? 1 : 0][cplx ? 1 : 0];
  const long long ntiles = P.N >> P.tb;
  const long long cap = (long long)(occ > 0 ? occ : 1) * nsm;
  const int grid = (int)(ntiles < cap ? ntiles : cap);
  ::lrei::count_launch();
  if (fp64) {
    auto kern = cplx ? hv_product<double, true> : hv_product<double, false>;
    kern<<<grid, 288, smem, st>>>(P, reinterpret_cast<const double2 *>(X), reinterpret_cast<double2 *>(Y), status);
  } else {
    auto kern = cplx ? hv_product<float, true> : hv_product<float, false>;
    kern<<<grid, 288, smem, st>>>(P, reinterpret_cast<const float4 *>(X), reinterpret_cast<float4 *>(Y), status);
  }
  return true;
}

// Returns true when the launch was made; false when the caller must use another kernel.
bool launch_hv_tiled(bool fp64, const ModelArgs &M, const void *X, void *Y, long long N, int r, int nsm,
                     cudaStream_t st, int *status, int tile_bits) {
  HvPlan P;
  if (!hv_plan(fp64, M, N, r, tile_bits, &P)) return false;
  return launch_hv_plan(fp64, M.cplx != 0, P, X, Y, nsm, st, status);
}

// The magnetisation operators on full rows (Sec. 3.6, the expectation values of eq. spin_op):
// which = 0: Y = M_z X, M_z = (1/n) sum_i S^z_i, a diagonal (n/2 - popcount(b)) / n;
// which = 1: Y = (M_x + i M_y) X = (1/n) sum_i S^+_i X, the raising operator of each site, which
//   maps a row b with bit i = 0 (spin up) to the partner b ^ 2^i and rows with bit i = 1 to zero.
// Both M_x and M_y Grams follow from the one Gram C = X^*(M_x + i M_y)X: X^*M_xX = (C + C^*)/2 and
// X^*M_yX = (C - C^*)/(2i), the two operators being Hermitian.
bool launch_magnetization(bool fp64, int which, int n, const void *X, void *Y, long long N, int r, int nsm,
                          cudaStream_t st, int *status) {
  ModelArgs M;
  std::memset(&M, 0, sizeof(M));
  M.n = n;
  if (which == 0) {
    M.bz = 1.0 / n;
  } else {
    M.cplx = 1;
    M.bx = 1.0;   // gives one one-bit term per site; the amplitudes are set below
  }
  HvPlan P;
  if (!hv_plan(fp64, M, N, r, 0, &P)) return false;
  if (which == 1) {
    const int nt = P.nI + P.nS + P.nF;
    for (int k = 0; k < nt; ++k) {
      P.a0r[k] = 1.0 / n;   // output row with the bit up: the partner's amplitude
      P.a0i[k] = 0.0;
      P.a1r[k] = 0.0;
      P.a1i[k] = 0.0;
    }
  }
  return launch_hv_plan(fp64, which == 1, P, X, Y, nsm, st, status);
}

}  // namespace lrei
