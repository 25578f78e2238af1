// Grid-sum contractions of Eq. (1) on the 5th-generation tensor cores (tcgen05, sm_103a).
//
//   part[chunk][m][n] = sum_{r in chunk} X_m(r) Y_n(r),  X_m = F[i1(m)] F[i2(m)],  Y_n = Y[n]
//
// The pair products X (phi_i phi_a for the exchange element, phi_a phi_b for the direct element) are
// formed by the producer warps from FP32 orbitals and never stored in global memory. Both operands
// are split into BF16 high and low parts (x = hi + lo) and three MMAs per K slice accumulate
// hi*hi + hi*lo + lo*hi in FP32 in tensor memory (relative error ~1e-5 of each product instead of
// BF16's 4e-3). One CTA owns a 128 x NT output tile (NT <= 256, multiple of 16) and a chunk of grid
// points; stages of 64 points are double-buffered in shared memory in the canonical K-major layout
// without swizzle (8-row x 16-byte core matrices: K-adjacent core matrices 128 B apart, row groups
// 1024 B apart). Thread 0 issues the MMAs and commits them to one mbarrier per stage; every wait on
// an mbarrier is bounded and sets *err on timeout. Partials (FP64) are reduced by the caller.
#include <cuda.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <mutex>

#include "bounds.cuh"
#include "kernels.h"
#include "tma.cuh"

namespace sbse {

constexpr int kUmM = 128;     // rows per tile (UMMA M)
constexpr int kUmBK = 64;     // grid points per stage
constexpr int kUmThreads = 128;  // the cleaning update
constexpr int kPgThreads = 256;  // the grid-sum GEMM: eight producer warps keep more loads in flight
constexpr int kUmStages = 2;
constexpr unsigned kWaitLimit = 1u << 26;

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// shared memory matrix descriptor: start >> 4 [0,14), LBO >> 4 [16,30), SBO >> 4 [32,46),
// version 1 [46,48), base offset 0, layout SWIZZLE_NONE (0) [61,64)
__device__ __forceinline__ uint64_t make_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// instruction descriptor, kind::f16: D F32 (bits 4-5 = 1), A BF16 (bits 7-9 = 1), B BF16
// (bits 10-12 = 1), both K-major, N >> 3 at bit 17, M >> 4 at bit 24
__host__ __device__ constexpr uint32_t make_idesc(int m, int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
      "l"(ad), "l"(bd), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t mbar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(mbar), "r"(parity)
      : "memory");
  return ok != 0;
}

// bounded wait; false on timeout
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
  for (unsigned i = 0; i < kWaitLimit; ++i)
    if (mbar_try_wait(mbar, parity)) return true;
  return false;
}

// bytes of one stage: A hi/lo (128 rows) + B hi/lo (NT rows), BF16, 64 points
__host__ __device__ constexpr size_t umma_stage_bytes(int nt) {
  return (size_t)2 * (kUmM + nt) * kUmBK * 2;
}

// offset (bytes) of element (row, k) of a R x 64 BF16 tile in the canonical no-swizzle K-major layout
__device__ __forceinline__ uint32_t canon_off(int row, int kc) {
  return (uint32_t)(((row >> 3) * 8 + kc) * 128 + (row & 7) * 16);
}

__device__ __forceinline__ void split8(const float *x, uint4 *hi, uint4 *lo) {
  __nv_bfloat162 h[4], l[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const __nv_bfloat16 h0 = __float2bfloat16_rn(x[2 * i]), h1 = __float2bfloat16_rn(x[2 * i + 1]);
    const __nv_bfloat16 l0 = __float2bfloat16_rn(x[2 * i] - __bfloat162float(h0));
    const __nv_bfloat16 l1 = __float2bfloat16_rn(x[2 * i + 1] - __bfloat162float(h1));
    h[i] = __halves2bfloat162(h0, h1);
    l[i] = __halves2bfloat162(l0, l1);
  }
  *hi = *reinterpret_cast<uint4 *>(h);
  *lo = *reinterpret_cast<uint4 *>(l);
}

// A-operand modes: pair products X_m = F[xi[m].x] F[xi[m].y], or the real / imaginary parts of
// complex rows (row m = 2c + h of the interleaved complex array F, c < M / 2)
enum UmmaAMode { UA_PRODUCT = 0, UA_COMPLEX = 1 };

// Producer: fill one stage. A unit = 8 rows x 32 points (4 core matrices along K); lane l covers
// row (l & 7) of the group and core matrix kq = l >> 3, i.e. 8 consecutive points of one row. Each
// warp loads kUB units before converting and storing any of them, so that several global loads per
// lane are in flight.
constexpr int kUB = 6;

template <int AMODE>
__device__ __forceinline__ void load_unit(int u, int units_a, const float *F, const int2 *xi, int M, int m0,
                                          const float *Y, int Nn, int n0, long long ng, long long k0,
                                          long long kend, bool vec_ok, float *x) {
  const int lane = threadIdx.x & 31;
  const int rr = lane & 7, kq = lane >> 3;
  const bool isA = u < units_a;
  const int uu = isA ? u : u - units_a;
  const int row = (uu >> 1) * 8 + rr;
  const int kc = (uu & 1) * 4 + kq;  // core matrix index along K (0..7)
  const long long kb = k0 + kc * 8;
#pragma unroll
  for (int j = 0; j < 8; ++j) x[j] = 0.f;
  const bool full = vec_ok && kb + 8 <= kend;
  if (isA && AMODE == UA_COMPLEX) {
    const int m = m0 + row;
    if (m < M) {
      const float *f = F + 2 * ((long long)(m >> 1) * ng + kb) + (m & 1);
      if (full) {
        const float4 c0 = *reinterpret_cast<const float4 *>(f - (m & 1));
        const float4 c1 = *reinterpret_cast<const float4 *>(f - (m & 1) + 4);
        const float4 c2 = *reinterpret_cast<const float4 *>(f - (m & 1) + 8);
        const float4 c3 = *reinterpret_cast<const float4 *>(f - (m & 1) + 12);
        if (m & 1) {
          x[0] = c0.y; x[1] = c0.w; x[2] = c1.y; x[3] = c1.w; x[4] = c2.y; x[5] = c2.w; x[6] = c3.y; x[7] = c3.w;
        } else {
          x[0] = c0.x; x[1] = c0.z; x[2] = c1.x; x[3] = c1.z; x[4] = c2.x; x[5] = c2.z; x[6] = c3.x; x[7] = c3.z;
        }
      } else {
#pragma unroll
        for (int j = 0; j < 8; ++j) x[j] = (kb + j < kend) ? f[2 * j] : 0.f;
      }
    }
  } else if (isA) {
    const int m = m0 + row;
    if (m < M) {
      const int2 q = xi[m];
      (void)SBSE_IDX(kb, ng);
      const float *f1 = F + (long long)q.x * ng + kb, *f2 = F + (long long)q.y * ng + kb;
      if (full) {
        const float4 a0 = *reinterpret_cast<const float4 *>(f1), a1 = *reinterpret_cast<const float4 *>(f1 + 4);
        const float4 b0 = *reinterpret_cast<const float4 *>(f2), b1 = *reinterpret_cast<const float4 *>(f2 + 4);
        x[0] = a0.x * b0.x; x[1] = a0.y * b0.y; x[2] = a0.z * b0.z; x[3] = a0.w * b0.w;
        x[4] = a1.x * b1.x; x[5] = a1.y * b1.y; x[6] = a1.z * b1.z; x[7] = a1.w * b1.w;
      } else {
#pragma unroll
        for (int j = 0; j < 8; ++j) x[j] = (kb + j < kend) ? f1[j] * f2[j] : 0.f;
      }
    }
  } else {
    const int n = n0 + row;
    if (n < Nn) {
      const float *y = Y + (long long)n * ng + kb;
      if (full) {
        const float4 a0 = *reinterpret_cast<const float4 *>(y), a1 = *reinterpret_cast<const float4 *>(y + 4);
        x[0] = a0.x; x[1] = a0.y; x[2] = a0.z; x[3] = a0.w;
        x[4] = a1.x; x[5] = a1.y; x[6] = a1.z; x[7] = a1.w;
      } else {
#pragma unroll
        for (int j = 0; j < 8; ++j) x[j] = (kb + j < kend) ? y[j] : 0.f;
      }
    }
  }
}

template <int AMODE, int NTHR>
__device__ __forceinline__ void produce_stage(uint8_t *st, int nt, const float *F, const int2 *xi, int M,
                                              int m0, const float *Y, int Nn, int n0, long long ng,
                                              long long k0, long long kend) {
  uint8_t *a_hi = st;
  uint8_t *a_lo = a_hi + kUmM * kUmBK * 2;
  uint8_t *b_hi = a_lo + kUmM * kUmBK * 2;
  uint8_t *b_lo = b_hi + nt * kUmBK * 2;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int rr = lane & 7, kq = lane >> 3;
  const int units_a = (kUmM / 8) * 2, units_b = (nt / 8) * 2, total = units_a + units_b;
  const bool vec_ok = (ng & 3) == 0;  // 16-byte aligned rows
  constexpr int W = NTHR / 32;
  for (int u0 = warp; u0 < total; u0 += W * kUB) {
    float x[kUB][8];
#pragma unroll
    for (int i = 0; i < kUB; ++i)
      if (u0 + i * W < total)
        load_unit<AMODE>(u0 + i * W, units_a, F, xi, M, m0, Y, Nn, n0, ng, k0, kend, vec_ok, x[i]);
#pragma unroll
    for (int i = 0; i < kUB; ++i) {
      const int u = u0 + i * W;
      if (u >= total) break;
      const bool isA = u < units_a;
      const int uu = isA ? u : u - units_a;
      const int row = (uu >> 1) * 8 + rr;
      const int kc = (uu & 1) * 4 + kq;
      uint4 hi, lo;
      split8(x[i], &hi, &lo);
      const uint32_t off = canon_off(row, kc);
      *reinterpret_cast<uint4 *>((isA ? a_hi : b_hi) + off) = hi;
      *reinterpret_cast<uint4 *>((isA ? a_lo : b_lo) + off) = lo;
    }
  }
}

template <int AMODE>
__global__ void __launch_bounds__(kPgThreads)
    k_umma_prod_gemm(const float *F, const int2 *xi, int M, const float *Y, int Nn, int nt, long long ng,
                     long long kchunk, double *part, int *err) {
  extern __shared__ __align__(128) uint8_t smem[];
  __shared__ __align__(8) uint64_t mbar[kUmStages];
  __shared__ uint32_t tmem_slot;
  const int m0 = blockIdx.y * kUmM, n0 = blockIdx.z * nt;
  const long long kbeg = (long long)blockIdx.x * kchunk;
  const long long kend = (kbeg + kchunk < ng) ? kbeg + kchunk : ng;
  const int n_iter = (int)((kend - kbeg + kUmBK - 1) / kUmBK);
  const size_t stage_bytes = umma_stage_bytes(nt);
  int ncols = 32;
  while (ncols < nt) ncols <<= 1;
  const int warp = threadIdx.x >> 5;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(ncols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (threadIdx.x == 0) {
    for (int s = 0; s < kUmStages; ++s)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[s])));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_slot;
  const uint32_t idesc = make_idesc(kUmM, nt);
  bool ok = true;
  for (int it = 0; it < n_iter; ++it) {
    const int s = it & 1;
    bool w = true;
    if (it >= kUmStages) w = mbar_wait(smem_u32(&mbar[s]), (uint32_t)((it / kUmStages - 1) & 1));
    if (!__syncthreads_and(w)) {  // uniform decision: every thread leaves the loop together
      ok = false;
      break;
    }
    uint8_t *st = smem + s * stage_bytes;
    produce_stage<AMODE, kPgThreads>(st, nt, F, xi, M, m0, Y, Nn, n0, ng, kbeg + (long long)it * kUmBK, kend);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (threadIdx.x == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;");
      const uint32_t a_hi = smem_u32(st), a_lo = a_hi + kUmM * kUmBK * 2;
      const uint32_t b_hi = a_lo + kUmM * kUmBK * 2, b_lo = b_hi + nt * kUmBK * 2;
#pragma unroll
      for (int t = 0; t < kUmBK / 16; ++t) {
        const uint32_t o = t * 256;  // two core matrices (16 points) per MMA along K
        const uint64_t dah = make_desc(a_hi + o, 128, 1024), dal = make_desc(a_lo + o, 128, 1024);
        const uint64_t dbh = make_desc(b_hi + o, 128, 1024), dbl = make_desc(b_lo + o, 128, 1024);
        mma_bf16(tmem, dah, dbh, idesc, (it > 0 || t > 0) ? 1u : 0u);
        mma_bf16(tmem, dah, dbl, idesc, 1u);
        mma_bf16(tmem, dal, dbh, idesc, 1u);
      }
      mma_commit(smem_u32(&mbar[s]));
    }
  }
  // all committed MMAs done (commits complete in order: the last one covers the rest)
  if (ok && n_iter > 0) {
    const int last = n_iter - 1;
    ok = __syncthreads_and(mbar_wait(smem_u32(&mbar[last & 1]), (uint32_t)((last / kUmStages) & 1)));
  }
  if (!ok) {
    if (threadIdx.x == 0) atomicExch(err, 1);
    // give in-flight MMAs a further bounded chance to finish before the accumulator is freed
    for (int s = 0; s < kUmStages; ++s) {
      const int cnt = (n_iter - s + kUmStages - 1) / kUmStages;
      if (cnt > 0) mbar_wait(smem_u32(&mbar[s]), (uint32_t)((cnt - 1) & 1));
    }
  }
  asm volatile("tcgen05.fence::after_thread_sync;");
  // epilogue: warp w reads the tensor-memory lanes of its quarter (w % 4) and half of the columns
  const int quarter = warp & 3, chalf = warp >> 2;
  const int c_lo = chalf == 0 ? 0 : ((nt / 16 + 1) / 2) * 16, c_hi = chalf == 0 ? ((nt / 16 + 1) / 2) * 16 : nt;
  if (ok && n_iter > 0) {
    const int lane = threadIdx.x & 31;
    const int m = m0 + quarter * 32 + lane;
    for (int c = c_lo; c < c_hi; c += 16) {
      uint32_t r[16];
      const uint32_t taddr = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)c;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
            "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (m < M) {
        double *o = part + ((long long)blockIdx.x * M + m) * Nn;
#pragma unroll
        for (int j = 0; j < 16; ++j)
          if (n0 + c + j < Nn) o[n0 + c + j] = (double)__uint_as_float(r[j]);
      }
    }
  } else if (n_iter == 0) {
    const int lane = threadIdx.x & 31;
    const int m = m0 + quarter * 32 + lane;
    if (m < M)
      for (int c = c_lo; c < c_hi && n0 + c < Nn; ++c) part[((long long)blockIdx.x * M + m) * Nn + n0 + c] = 0.0;
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols));
}

// ---- cleaning projection update on the tensor cores ------------------------------------------
// d_c(r) -= sum_s O[c][s] phi_s(r) (Eq. 15) as D[m][r] = sum_s O[m][s] phi_s(r) with m = 2c + h the
// real / imaginary row of column c; A = O (128 rows per tile), B = phi^T (256 grid points per tile),
// K = the occupied states in chunks of 32. Both operands are split into BF16 high / low parts and
// laid out in the canonical K-major tiles once (B once per propagation, A once per cleaning), so a
// CTA only issues two bulk copies (TMA) per K chunk and then the MMAs; one thread keeps two chunks
// in flight (the copies of the next chunk land while the MMAs of the current one run). The
// epilogue subtracts D
// from d in place (coalesced through shared memory) and writes per-tile partial sums of
// 2 Re(conj(eta0) d) and |d|^2 per column for the renormalisation.
constexpr int kCuN = 256;
constexpr int kUdBK = 32;                          // occupied states per operand chunk of the update
constexpr int kUdStages = 2;                       // operand chunks in flight per CTA
constexpr unsigned kCanA = 2u * kUmM * kUdBK * 2;  // bytes of one A chunk (hi, lo): 16 KB
constexpr unsigned kCanB = 2u * kCuN * kUdBK * 2;  // bytes of one B chunk (hi, lo): 32 KB

// offset of element (row, core matrix kc) of an R x kUdBK BF16 tile, canonical K-major, no swizzle:
// K-adjacent core matrices 128 B apart, 8-row groups kUdBK / 8 x 128 B apart
__device__ __forceinline__ uint32_t canon_ud_off(int row, int kc) {
  return (uint32_t)(((row >> 3) * (kUdBK / 8) + kc) * 128 + (row & 7) * 16);
}

// canonical BF16 hi / lo tiles: out[tile][chunk] = hi (R x 64) then lo (R x 64); element (row, k)
// of a tile is src(tile R + row, chunk 64 + k), zero outside the source. Thread per (row, group of
// 8 k); consecutive threads take consecutive rows.
struct SrcRowsF64 {  // O[m][s], row-major FP64
  const double *p;
  long long rows;
  int K;
  __device__ float operator()(long long r, int k) const { return (r < rows && k < K) ? (float)p[r * K + k] : 0.f; }
};
struct SrcColsF32 {  // phi^T: element (r, s) = phi[s][r]
  const float *p;
  long long rows;
  int K;
  __device__ float operator()(long long r, int k) const { return (r < rows && k < K) ? p[(long long)k * rows + r] : 0.f; }
};

template <int R, class Src>
__global__ void k_canon_tiles(Src src, long long n_tiles, int n_kc, uint8_t *out) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  constexpr int G = kUdBK / 8;  // groups of 8 K values per chunk
  const long long per_chunk = (long long)R * G, per_tile = per_chunk * n_kc;
  if (t >= n_tiles * per_tile) return;
  const long long tile = t / per_tile;
  const long long rem = t - tile * per_tile;
  const int kc = (int)(rem / per_chunk);
  const int rem2 = (int)(rem - (long long)kc * per_chunk);
  const int g = rem2 / R, row = rem2 - g * R;
  float x[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) x[j] = src(tile * R + row, kc * kUdBK + g * 8 + j);
  uint4 hi, lo;
  split8(x, &hi, &lo);
  uint8_t *base = out + (tile * n_kc + kc) * (2ll * R * kUdBK * 2);
  const uint32_t off = canon_ud_off(row, g);
  *reinterpret_cast<uint4 *>(base + off) = hi;
  *reinterpret_cast<uint4 *>(base + (size_t)R * kUdBK * 2 + off) = lo;
}

__global__ void __launch_bounds__(kUmThreads)
    k_umma_clean_update(const uint8_t *o_can, int M, const uint8_t *phi_can, int n_kc, long long ng, float *d,
                        const float *a, int L, double *npart, int *err) {
  extern __shared__ __align__(128) uint8_t smem[];
  __shared__ __align__(8) uint64_t full[kUdStages], done[kUdStages];
  __shared__ uint32_t tmem_slot;
  __shared__ int fail;
  // stage s: A chunk (hi, lo) then B chunk (hi, lo), as laid out by k_canon_tiles
  auto stage = [&](int s) { return smem + (size_t)s * (kCanA + kCanB); };
  // row tile fastest: the CTAs that read one tile of phi operands run together (L2 reuse)
  const int mt = blockIdx.x;
  const long long tile = blockIdx.y;
  const int m0 = mt * kUmM;
  const long long r0 = tile * kCuN;
  const int n_cols = M / 2;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(kCuN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (threadIdx.x == 0) {
    for (int s = 0; s < kUdStages; ++s) {
      tma_bar_init(&full[s], 1);
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&done[s])));
    }
    fail = 0;
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_slot;
  const uint32_t idesc = make_idesc(kUmM, kCuN);
  if (threadIdx.x == 0) {
    // One thread drives a ring of kUdStages operand chunks: the copies of chunk it + kUdStages are
    // issued as soon as the MMAs of chunk it have read its stage, so copies and MMAs overlap.
    auto load = [&](int it) {
      const int s = it % kUdStages;
      (void)SBSE_IDX((long long)mt * n_kc + it, (long long)gridDim.x * n_kc);
      (void)SBSE_IDX(tile * n_kc + it, (long long)((ng + kCuN - 1) / kCuN) * n_kc);
      tma_bar_expect(&full[s], kCanA + kCanB);
      tma_load_1d(stage(s), o_can + ((size_t)mt * n_kc + it) * kCanA, kCanA, &full[s]);
      tma_load_1d(stage(s) + kCanA, phi_can + ((size_t)tile * n_kc + it) * kCanB, kCanB, &full[s]);
    };
    int loaded = 0, committed = 0;
    for (; loaded < n_kc && loaded < kUdStages; ++loaded) load(loaded);
    bool ok = true;
    for (int it = 0; it < n_kc && ok; ++it) {
      const int s = it % kUdStages;
      if (!mbar_wait(smem_u32(&full[s]), (uint32_t)((it / kUdStages) & 1))) {
        ok = false;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;");
      const uint32_t ah = smem_u32(stage(s)), al = ah + kUmM * kUdBK * 2;
      const uint32_t bh = ah + kCanA, bl = bh + kCuN * kUdBK * 2;
#pragma unroll
      for (int t = 0; t < kUdBK / 16; ++t) {
        const uint32_t o = t * 256;  // two core matrices (16 states) per MMA along K
        const uint64_t dah = make_desc(ah + o, 128, kUdBK / 8 * 128), dal = make_desc(al + o, 128, kUdBK / 8 * 128);
        const uint64_t dbh = make_desc(bh + o, 128, kUdBK / 8 * 128), dbl = make_desc(bl + o, 128, kUdBK / 8 * 128);
        mma_bf16(tmem, dah, dbh, idesc, (it > 0 || t > 0) ? 1u : 0u);
        mma_bf16(tmem, dah, dbl, idesc, 1u);
        mma_bf16(tmem, dal, dbh, idesc, 1u);
      }
      mma_commit(smem_u32(&done[s]));
      ++committed;
      if (loaded < n_kc) {  // the stage is refilled once its MMAs are done with it
        if (!mbar_wait(smem_u32(&done[s]), (uint32_t)((it / kUdStages) & 1))) {
          ok = false;
          break;
        }
        load(loaded++);
      }
    }
    // every MMA done (commits complete in order: the last one covers the rest)
    if (ok && committed > 0)
      ok = mbar_wait(smem_u32(&done[(committed - 1) % kUdStages]), (uint32_t)(((committed - 1) / kUdStages) & 1));
    if (!ok) {
      fail = 1;
      atomicExch(err, 1);
      // copies and MMAs still in flight must land before shared and tensor memory are released
      for (int it = committed; it < loaded; ++it)
        mbar_wait(smem_u32(&full[it % kUdStages]), (uint32_t)((it / kUdStages) & 1));
      if (committed > 0)
        mbar_wait(smem_u32(&done[(committed - 1) % kUdStages]), (uint32_t)(((committed - 1) / kUdStages) & 1));
    }
  }
  __syncthreads();
  const bool ok = fail == 0;
  asm volatile("tcgen05.fence::after_thread_sync;");
  // Epilogue, in two halves of 128 grid points: the accumulator rows (m = 2c + h) are staged in the
  // (now free) operand shared memory with a padded stride, then every warp updates whole complex
  // columns with coalesced float2 accesses and reduces their norm sums.
  constexpr int kHalf = 128, kLd = kHalf + 1;
  float *Dsm = reinterpret_cast<float *>(smem);  // kUmM x kLd floats (66 KB) inside the operand buffer
  // per-tile sums stay in FP32 (256 points): a warp-wide FP64 instruction occupies this GPU's narrow
  // FP64 pipe for many cycles even with one active lane
  __shared__ float colsum[kUmM / 2][2];
  for (int i = threadIdx.x; i < kUmM; i += blockDim.x) colsum[i >> 1][i & 1] = 0.f;
  const int c0 = m0 / 2;
  for (int half = 0; half < kCuN / kHalf && ok; ++half) {
    __syncthreads();
    for (int cc = 0; cc < kHalf; cc += 16) {
      uint32_t rr[16];
      const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(half * kHalf + cc);
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
          : "=r"(rr[0]), "=r"(rr[1]), "=r"(rr[2]), "=r"(rr[3]), "=r"(rr[4]), "=r"(rr[5]), "=r"(rr[6]), "=r"(rr[7]),
            "=r"(rr[8]), "=r"(rr[9]), "=r"(rr[10]), "=r"(rr[11]), "=r"(rr[12]), "=r"(rr[13]), "=r"(rr[14]), "=r"(rr[15])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      float *row = Dsm + (warp * 32 + lane) * kLd + cc;
#pragma unroll
      for (int j = 0; j < 16; ++j) row[j] = __uint_as_float(rr[j]);
    }
    __syncthreads();
    // each warp updates CB complex columns at a time, with all their loads issued together
    constexpr int CB = 4, PP = kHalf / 32;
    for (int cb = warp * CB; cb < kUmM / 2; cb += CB * (kUmThreads / 32)) {
      float2 dv[CB][PP], av[CB][PP];
#pragma unroll
      for (int i = 0; i < CB; ++i) {
        const int c = c0 + cb + i;
        const float2 *dc = reinterpret_cast<const float2 *>(d) + (long long)c * ng;
        const float2 *ac = reinterpret_cast<const float2 *>(a) + (long long)(c % L) * ng;
#pragma unroll
        for (int j = 0; j < PP; ++j) {
          const long long r = r0 + half * kHalf + lane + 32 * j;
          const bool in = c < n_cols && r < ng;
          dv[i][j] = in ? dc[r] : make_float2(0.f, 0.f);
          av[i][j] = in ? ac[r] : make_float2(0.f, 0.f);
        }
      }
#pragma unroll
      for (int i = 0; i < CB; ++i) {
        const int cl = cb + i, c = c0 + cl;
        float2 *dc = reinterpret_cast<float2 *>(d) + (long long)c * ng;
        // FP32 sums over the points of the tile; FP64 from the per-tile partials on
        float v1 = 0.f, v2 = 0.f;
#pragma unroll
        for (int j = 0; j < PP; ++j) {
          const int p = lane + 32 * j;
          const long long r = r0 + half * kHalf + p;
          if (c < n_cols && r < ng) {
            float2 x = dv[i][j];
            x.x -= Dsm[(2 * cl) * kLd + p];
            x.y -= Dsm[(2 * cl + 1) * kLd + p];
            dc[r] = x;
            v1 += 2.f * (av[i][j].x * x.x + av[i][j].y * x.y);
            v2 += x.x * x.x + x.y * x.y;
          }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          v1 += __shfl_xor_sync(0xffffffffu, v1, o);
          v2 += __shfl_xor_sync(0xffffffffu, v2, o);
        }
        if (lane == 0) {
          colsum[cl][0] += v1;
          colsum[cl][1] += v2;
        }
      }
    }
  }
  __syncthreads();
  for (int cl = threadIdx.x; cl < kUmM / 2; cl += blockDim.x) {
    const int c = c0 + cl;
    if (ok && c < n_cols) {
      npart[(tile * n_cols + c) * 2 + 0] = (double)colsum[cl][0];
      npart[(tile * n_cols + c) * 2 + 1] = (double)colsum[cl][1];
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kCuN));
}

// grid-point tiles of the tensor-core cleaning update (rows of its norm partials)
long long umma_clean_update_tiles(long long ng) { return (ng + kCuN - 1) / kCuN; }

static int kchunks(int n_occ) { return (n_occ + kUdBK - 1) / kUdBK; }

size_t umma_update_phi_bytes(long long ng, int n_occ) {
  return (size_t)umma_clean_update_tiles(ng) * kchunks(n_occ) * kCanB;
}
size_t umma_update_o_bytes(int n_cols, int n_occ) {
  return (size_t)((2 * n_cols + kUmM - 1) / kUmM) * kchunks(n_occ) * kCanA;
}

void umma_prepare_update_phi(const float *phi, int n_occ, long long ng, uint8_t *phi_can, cudaStream_t s) {
  const long long tiles = umma_clean_update_tiles(ng);
  const long long threads = tiles * kchunks(n_occ) * kCuN * (kUdBK / 8);
  k_canon_tiles<kCuN, SrcColsF32><<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(
      SrcColsF32{phi, ng, n_occ}, tiles, kchunks(n_occ), phi_can);
  count_launch(1);
}

void launch_umma_clean_update(const double *ov, int n_cols, const uint8_t *phi_can, int n_occ, long long ng,
                              float *d_interleaved, const float *a_interleaved, int L, double *npart,
                              uint8_t *o_can, int *err, cudaStream_t s) {
  const int M = 2 * n_cols;
  const long long m_tiles = (M + kUmM - 1) / kUmM;
  const long long threads = m_tiles * kchunks(n_occ) * kUmM * (kUdBK / 8);
  k_canon_tiles<kUmM, SrcRowsF64><<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(
      SrcRowsF64{ov, M, n_occ}, m_tiles, kchunks(n_occ), o_can);
  const size_t smem = (size_t)kUdStages * (kCanA + kCanB);
  raise_smem_limit((const void *)k_umma_clean_update, smem);
  dim3 grid((unsigned)m_tiles, (unsigned)umma_clean_update_tiles(ng));
  k_umma_clean_update<<<grid, kUmThreads, smem, s>>>(o_can, M, phi_can, kchunks(n_occ), ng, d_interleaved,
                                                     a_interleaved, L, npart, err);
  count_launch(2);
}

// tile width for Nn output columns: multiple of 16, at most 256
static int umma_nt(int Nn) {
  int nt = ((Nn + 15) / 16) * 16;
  return nt > 256 ? 256 : nt;
}

static long long umma_kchunk(long long ng, int tiles) {
  // about two CTAs per SM across all tiles, whole stages per chunk
  long long target = 304 / (tiles > 0 ? tiles : 1);
  if (target < 1) target = 1;
  long long c = (ng + target - 1) / target;
  c = ((c + kUmBK - 1) / kUmBK) * kUmBK;
  return c < kUmBK ? kUmBK : c;
}

size_t umma_prod_gemm_work_bytes(int M, int Nn, long long ng) {
  const int nt = umma_nt(Nn);
  const int tiles = ((M + kUmM - 1) / kUmM) * ((Nn + nt - 1) / nt);
  const long long kc = umma_kchunk(ng, tiles);
  const long long chunks = (ng + kc - 1) / kc;
  return (size_t)(chunks * M * Nn) * sizeof(double);
}

template <int AMODE>
static int launch_umma(const float *F, const int2 *xi, int M, const float *Y, int Nn, long long ng,
                       double scale, double *out, double *work, int *err, cudaStream_t s) {
  const int nt = umma_nt(Nn);
  const int tiles = ((M + kUmM - 1) / kUmM) * ((Nn + nt - 1) / nt);
  const long long kc = umma_kchunk(ng, tiles);
  const long long chunks = (ng + kc - 1) / kc;
  const size_t smem = kUmStages * umma_stage_bytes(nt);
  raise_smem_limit((const void *)k_umma_prod_gemm<AMODE>, smem);
  dim3 grid((unsigned)chunks, (M + kUmM - 1) / kUmM, (Nn + nt - 1) / nt);
  k_umma_prod_gemm<AMODE><<<grid, kPgThreads, smem, s>>>(F, xi, M, Y, Nn, nt, ng, kc, work, err);
  count_launch(1);
  launch_reduce_cols(work, (int)chunks, M * Nn, scale, out, s);
  return 0;
}

int launch_umma_prod_gemm(const float *F, const int2 *xi, int M, const float *Y, int Nn, long long ng,
                          double scale, double *out, double *work, int *err, cudaStream_t s) {
  return launch_umma<UA_PRODUCT>(F, xi, M, Y, Nn, ng, scale, out, work, err, s);
}

// cleaning overlaps of Eq. (15): out[2c + h][s] = scale sum_r (Re, Im)_h d_c(r) phi_s(r)
int launch_umma_clean_overlap(const float *d_interleaved, int n_cols, const float *phi, int n_occ,
                              long long ng, double scale, double *out, double *work, int *err,
                              cudaStream_t s) {
  return launch_umma<UA_COMPLEX>(d_interleaved, nullptr, 2 * n_cols, phi, n_occ, ng, scale, out, work,
                                 err, s);
}


// ---- cleaning overlaps, streamed form ----------------------------------------------------------
// ov[2c + h][s] = sum_r (Re, Im)_h d_c(r) phi_s(r) (Eq. 15) with the grid points as the contraction
// index. One CTA owns 64 complex columns of d (128 accumulator rows: real and imaginary part of each
// column) times every occupied state (up to 512 accumulator columns in tensor memory), over a chunk
// of grid points. Warp roles:
//   warp 4     bulk copies: the raw interleaved FP32 d rows of a 32-point stage (two tiled
//              tensor copies of 64 rows x 128 B, 128-byte swizzle, zero fill outside d) and the
//              stage's slab of pre-split phi tiles (one copy), on one mbarrier;
//   warps 0-3  split the raw stage into BF16 hi / lo rows 2c, 2c + 1 of the A tile (shared memory
//              to shared memory), then, after the last stage, read the accumulator (one TMEM lane
//              quarter each) and write the FP64 partials of the chunk;
//   warp 5     allocates tensor memory and issues the MMAs (hi*hi + hi*lo + lo*hi per 16 points,
//              N split into pieces of at most 256), committing each stage to its `empty` barrier.
// A ring of S stages keeps copies, splits and MMAs of successive stages in flight together. Every
// wait is bounded; a role that gives up raises a shared abort flag (the others then stop waiting)
// and *err, and the copies and MMAs already issued are waited for before memory is released.
constexpr int kOvKS = 32;                           // grid points per stage
constexpr int kOvCols = kUmM / 2;                   // complex columns of d per CTA
constexpr unsigned kOvRawHalf = kOvCols * 128;      // one tensor-copy box: 64 rows x 16 points
constexpr unsigned kOvRaw = 2 * kOvRawHalf;         // 16384 (1024-byte aligned: the swizzle atom)
constexpr unsigned kOvA = 2u * kUmM * kOvKS * 2;    // hi + lo A tile: 16384
constexpr int kOvThreads = 192;
constexpr int kOvMaxStages = 8;
constexpr size_t kOvSmemBudget = 200u * 1024u;
constexpr unsigned kOvAlign = 1024;                 // dynamic shared memory is aligned up to this

__host__ __device__ constexpr unsigned ov_b_bytes(int nb) { return 2u * (unsigned)nb * kOvKS * 2; }
__host__ __device__ constexpr unsigned ov_stage_bytes(int nb) { return kOvRaw + kOvA + ov_b_bytes(nb); }

// offset of element (row, core matrix kc) in an R x 32 BF16 tile, canonical K-major, no swizzle:
// K-adjacent core matrices 128 B apart, 8-row groups 512 B apart
__device__ __forceinline__ uint32_t canon32_off(int row, int kc) {
  return (uint32_t)(((row >> 3) * (kOvKS / 8) + kc) * 128 + (row & 7) * 16);
}

// accumulator rows (padded occupied count) of the streamed overlaps: a multiple of 16
static int ov_rows(int n_occ) { return ((n_occ + 15) / 16) * 16; }

// phi as the B operand of the streamed overlaps: per 32-point stage a slab of hi then lo tiles of
// ov_rows(n_occ) rows (zero beyond n_occ and beyond the last grid point)
size_t umma_ov_phi_bytes(long long ng, int n_occ) {
  return (size_t)((ng + kOvKS - 1) / kOvKS) * ov_b_bytes(ov_rows(n_occ));
}

__global__ void k_ov_phi_tiles(const float *phi, int n_occ, int nb, long long ng, long long n_ks, uint8_t *out) {
  // thread per (row, stage, group of 8 points); groups fastest, so a warp reads a row contiguously
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long per_row = n_ks * (kOvKS / 8);
  if (t >= (long long)nb * per_row) return;
  const int row = (int)(t / per_row);
  const long long rem = t - (long long)row * per_row;
  const long long ks = rem / (kOvKS / 8);
  const int g = (int)(rem - ks * (kOvKS / 8));
  const long long p0 = ks * kOvKS + g * 8;
  float x[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) x[j] = (row < n_occ && p0 + j < ng) ? phi[(long long)row * ng + p0 + j] : 0.f;
  uint4 hi, lo;
  split8(x, &hi, &lo);
  uint8_t *slab = out + (size_t)ks * ov_b_bytes(nb);
  const uint32_t off = canon32_off(row, g);
  *reinterpret_cast<uint4 *>(slab + off) = hi;
  *reinterpret_cast<uint4 *>(slab + (size_t)nb * kOvKS * 2 + off) = lo;
}

void umma_prepare_ov_phi(const float *phi, int n_occ, long long ng, uint8_t *out, cudaStream_t s) {
  const int nb = ov_rows(n_occ);
  const long long n_ks = (ng + kOvKS - 1) / kOvKS;
  const long long threads = (long long)nb * n_ks * (kOvKS / 8);
  k_ov_phi_tiles<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(phi, n_occ, nb, ng, n_ks, out);
  count_launch(1);
}

// bounded wait that also gives up when another role has raised the abort flag
__device__ __forceinline__ bool ov_wait(uint64_t *bar, uint32_t parity, volatile int *abort_flag) {
  const uint32_t a = smem_u32(bar);
  for (unsigned i = 0; i < kWaitLimit; ++i) {
    if (mbar_try_wait(a, parity)) return true;
    if ((i & 255u) == 255u && *abort_flag) return false;
  }
  return false;
}

__device__ __forceinline__ void ov_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// byte offset of the 16-byte chunk j of row r in a 128-byte-swizzled box of 128-byte rows
__device__ __forceinline__ uint32_t swz128(int r, int j) { return (uint32_t)(r * 128 + ((j ^ (r & 7)) << 4)); }

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          smem_u32(dst)),
      "l"((uint64_t)(uintptr_t)map), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

__global__ void __launch_bounds__(kOvThreads, 1)
    k_umma_clean_ov(const __grid_constant__ CUtensorMap dmap, int n_cols, const uint8_t *phi_t, int nb, int n_occ,
                    long long ng, long long kchunk, int S, double *part, int *err) {
  extern __shared__ __align__(128) uint8_t smem_raw[];
  uint8_t *smem = smem_raw + ((kOvAlign - (smem_u32(smem_raw) & (kOvAlign - 1))) & (kOvAlign - 1));
  __shared__ __align__(8) uint64_t full[kOvMaxStages], conv[kOvMaxStages], empty[kOvMaxStages], accb;
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;
  volatile int *abort_v = &abort_flag;
  uint8_t *raw = smem;
  uint8_t *atile = raw + (size_t)S * kOvRaw;
  uint8_t *btile = atile + (size_t)S * kOvA;
  const unsigned bbytes = ov_b_bytes(nb);
  const int M = 2 * n_cols;
  const int mt = blockIdx.x;  // m tile fastest: the CTAs that share a chunk's phi slabs run together
  const int c0 = mt * kOvCols;
  const int ncols_t = min(kOvCols, n_cols - c0);
  const long long kbeg = (long long)blockIdx.y * kchunk;
  const long long kend = min(kbeg + kchunk, ng);
  const int n_iter = kend > kbeg ? (int)((kend - kbeg + kOvKS - 1) / kOvKS) : 0;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int tcols = 32;
  while (tcols < nb) tcols <<= 1;
  if (warp == 5) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(tcols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&full[s])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 4;" ::"r"(smem_u32(&conv[s])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&empty[s])));
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&accb)));
    asm volatile("fence.mbarrier_init.release.cluster;");
    abort_flag = 0;
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_slot;

  int issued = 0;  // bulk-copy stages issued (warp 4)
  if (warp == 4) {
    // ---- bulk copies
    for (int it = 0; it < n_iter; ++it) {
      const int s = it % S;
      bool ok = true;
      if (it >= S) ok = ov_wait(&empty[s], (uint32_t)((it / S - 1) & 1), abort_v);
      if (!__all_sync(0xffffffffu, ok)) {
        if (lane == 0) { *abort_v = 1; atomicExch(err, 1); }
        break;
      }
      const long long k0 = kbeg + (long long)it * kOvKS;
      (void)SBSE_IDX(k0, ng);
      (void)SBSE_IDX(c0, n_cols);
      (void)SBSE_IDX(k0 / kOvKS, (ng + kOvKS - 1) / kOvKS);
      if (lane == 0) {
        // d viewed as n_cols rows of 2 ng floats: boxes of 64 rows x 32 floats at float x = 2 k0
        // (+ 32), a multiple of 64 (16-byte rule); rows past n_cols and points past ng read as zero
        tma_bar_expect(&full[s], kOvRaw + bbytes);
        tma_load_2d(raw + (size_t)s * kOvRaw, &dmap, (int)(2 * k0), c0, &full[s]);
        tma_load_2d(raw + (size_t)s * kOvRaw + kOvRawHalf, &dmap, (int)(2 * k0 + 32), c0, &full[s]);
        tma_load_1d(btile + (size_t)s * bbytes, phi_t + (size_t)(k0 / kOvKS) * bbytes, bbytes, &full[s]);
      }
      __syncwarp();
      ++issued;
    }
  } else if (warp == 5) {
    // ---- MMA issue
    if (lane == 0) {
      for (int it = 0; it < n_iter; ++it) {
        const int s = it % S;
        if (!ov_wait(&conv[s], (uint32_t)((it / S) & 1), abort_v)) {
          *abort_v = 1;
          atomicExch(err, 1);
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;");
        const uint32_t ah = smem_u32(atile + (size_t)s * kOvA), al = ah + kUmM * kOvKS * 2;
        const uint32_t bh = smem_u32(btile + (size_t)s * bbytes), bl = bh + (uint32_t)nb * kOvKS * 2;
#pragma unroll
        for (int t = 0; t < kOvKS / 16; ++t) {
          const uint32_t o = t * 256;
          const uint64_t dah = make_desc(ah + o, 128, 512), dal = make_desc(al + o, 128, 512);
          const uint32_t acc = (it > 0 || t > 0) ? 1u : 0u;
          for (int n0 = 0; n0 < nb; n0 += 256) {
            const int nn = min(256, nb - n0);
            const uint32_t idesc = make_idesc(kUmM, nn);
            const uint32_t boff = (uint32_t)(n0 / 8) * 512u + o;
            const uint64_t dbh = make_desc(bh + boff, 128, 512), dbl = make_desc(bl + boff, 128, 512);
            mma_bf16(tmem + (uint32_t)n0, dah, dbh, idesc, acc);
            mma_bf16(tmem + (uint32_t)n0, dah, dbl, idesc, 1u);
            mma_bf16(tmem + (uint32_t)n0, dal, dbh, idesc, 1u);
          }
        }
        mma_commit(smem_u32(&empty[s]));
      }
      mma_commit(smem_u32(&accb));  // arrives once every MMA issued above has completed
    }
  } else {
    // ---- split the raw stage into the A tile (warps 0-3, 128 threads)
    const int t = threadIdx.x;
    for (int it = 0; it < n_iter; ++it) {
      const int s = it % S;
      const bool ok = ov_wait(&full[s], (uint32_t)((it / S) & 1), abort_v);
      if (!__all_sync(0xffffffffu, ok)) {
        if (lane == 0) { *abort_v = 1; atomicExch(err, 1); }
        break;
      }
      const long long k0 = kbeg + (long long)it * kOvKS;
      const int npts = (int)min((long long)kOvKS, kend - k0);
      const uint8_t *rs = raw + (size_t)s * kOvRaw;
      uint8_t *ahi = atile + (size_t)s * kOvA, *alo = ahi + kUmM * kOvKS * 2;
#pragma unroll
      for (int pass = 0; pass < 2; ++pass) {
        // points 8g .. 8g + 7 of column col: box g / 2, 16-byte chunks 4 (g % 2) + q of row col
        // (consecutive lanes take consecutive rows, whose swizzled chunks fall in distinct banks)
        const int col = t & (kOvCols - 1), g = (t >> 6) + 2 * pass;
        const uint8_t *box = rs + (g >> 1) * kOvRawHalf;
        float re[8], im[8];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const float4 v = *reinterpret_cast<const float4 *>(box + swz128(col, 4 * (g & 1) + q));
          re[2 * q] = v.x; im[2 * q] = v.y; re[2 * q + 1] = v.z; im[2 * q + 1] = v.w;
        }
        if (g * 8 + 8 > npts) {  // the chunk ends inside this stage: points past it belong to no one here
#pragma unroll
          for (int j = 0; j < 8; ++j)
            if (g * 8 + j >= npts) re[j] = im[j] = 0.f;
        }
        uint4 hi, lo;
        split8(re, &hi, &lo);
        *reinterpret_cast<uint4 *>(ahi + canon32_off(2 * col, g)) = hi;
        *reinterpret_cast<uint4 *>(alo + canon32_off(2 * col, g)) = lo;
        split8(im, &hi, &lo);
        *reinterpret_cast<uint4 *>(ahi + canon32_off(2 * col + 1, g)) = hi;
        *reinterpret_cast<uint4 *>(alo + canon32_off(2 * col + 1, g)) = lo;
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // generic writes -> tensor core reads
      __syncwarp();
      if (lane == 0) ov_arrive(&conv[s]);
    }
    // ---- epilogue: accumulator lane quarter `warp`, FP64 partials of this chunk
    bool ok = n_iter > 0 && __all_sync(0xffffffffu, ov_wait(&accb, 0u, abort_v)) && !*abort_v;
    asm volatile("tcgen05.fence::after_thread_sync;");
    const int m = mt * kUmM + warp * 32 + lane;
    double *o = part + ((long long)blockIdx.y * M + m) * n_occ;
    if (ok) {
      for (int c = 0; c < nb; c += 16) {
        uint32_t r[16];
        const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c;
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
            : "r"(taddr));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (m < M) {
#pragma unroll
          for (int j = 0; j < 16; ++j)
            if (c + j < n_occ) o[c + j] = (double)__uint_as_float(r[j]);
        }
      }
    } else if (n_iter == 0 && m < M) {
      for (int c = 0; c < n_occ; ++c) o[c] = 0.0;
    }
  }
  __syncthreads();
  if (*abort_v) {
    // an abandoned pipeline: every issued copy has landed and every issued MMA has completed
    // before shared and tensor memory are released (bounded waits again)
    if (warp == 4 && lane == 0)
      for (int s = 0; s < S && s < issued; ++s) {
        const int last = issued - 1 - ((issued - 1 - s) % S);  // last iteration that used slot s
        mbar_wait(smem_u32(&full[s]), (uint32_t)((last / S) & 1));
      }
    if (warp == 5 && lane == 0) mbar_wait(smem_u32(&accb), 0u);
    __syncthreads();
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 5) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tcols));
}

// grid of the streamed overlaps: (m tiles, chunks); about one CTA per SM, whole stages per chunk
static void ov_grid(int n_cols, long long ng, int *m_tiles, long long *kc, long long *chunks) {
  *m_tiles = (n_cols + kOvCols - 1) / kOvCols;
  long long target = 152 / *m_tiles;
  if (target < 1) target = 1;
  long long c = (ng + target - 1) / target;
  c = ((c + kOvKS - 1) / kOvKS) * kOvKS;
  *kc = c;
  *chunks = (ng + c - 1) / c;
}

static int ov_stages(int nb) {
  int s = (int)((kOvSmemBudget - kOvAlign) / ov_stage_bytes(nb));
  return s > kOvMaxStages ? kOvMaxStages : s;
}

// the driver's tensor-map encoder, looked up once through the runtime
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
static EncodeTiledFn encode_tiled() {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
  });
  return fn;
}

bool make_tensor_map_f32(CUtensorMap *map, const void *base, int rank, const uint64_t *dims,
                         const uint64_t *strides_bytes, const uint32_t *box, bool swizzle128) {
  EncodeTiledFn enc = encode_tiled();
  if (!enc || rank < 1 || rank > 5) return false;
  cuuint64_t d[5], st[4];
  cuuint32_t b[5], e[5];
  for (int i = 0; i < rank; ++i) {
    d[i] = dims[i];
    b[i] = box[i];
    e[i] = 1;
    if (i + 1 < rank) st[i] = strides_bytes[i];
  }
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, (cuuint32_t)rank, const_cast<void *>(base), d, st, b, e,
             CU_TENSOR_MAP_INTERLEAVE_NONE, swizzle128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE,
             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool umma_clean_ov_supported(int n_occ, long long ng) {
  const int nb = ov_rows(n_occ);
  // rows of 2 ng floats: a 16-byte multiple stride; 2 ng < 2^32 for the tensor-copy coordinates
  return nb <= 512 && (ng % 2) == 0 && 2 * ng < (1ll << 31) && ov_stages(nb) >= 2 && encode_tiled() != nullptr;
}

size_t umma_clean_ov_work_bytes(int n_cols, int n_occ, long long ng) {
  int mt;
  long long kc, chunks;
  ov_grid(n_cols, ng, &mt, &kc, &chunks);
  return (size_t)(chunks * 2 * n_cols * n_occ) * sizeof(double);
}

int launch_umma_clean_ov(const float *d_interleaved, int n_cols, const uint8_t *phi_t, int n_occ, long long ng,
                         double scale, double *out, double *work, int *err, cudaStream_t s) {
  const int nb = ov_rows(n_occ);
  const int S = ov_stages(nb);
  int mt;
  long long kc, chunks;
  ov_grid(n_cols, ng, &mt, &kc, &chunks);
  const size_t smem = (size_t)S * ov_stage_bytes(nb) + kOvAlign;
  CUtensorMap dmap;
  const uint64_t dims[2] = {(uint64_t)(2 * ng), (uint64_t)n_cols};
  const uint64_t strides[1] = {(uint64_t)(2 * ng * sizeof(float))};
  const uint32_t box[2] = {32u, (uint32_t)kOvCols};
  if (!make_tensor_map_f32(&dmap, d_interleaved, 2, dims, strides, box, true)) return -1;
  raise_smem_limit((const void *)k_umma_clean_ov, smem);
  dim3 grid((unsigned)mt, (unsigned)chunks);
  k_umma_clean_ov<<<grid, kOvThreads, smem, s>>>(dmap, n_cols, phi_t, nb, n_occ, ng, kc, S, work, err);
  count_launch(1);
  launch_reduce_cols(work, (int)chunks, 2 * n_cols * n_occ, scale, out, s);
  return 0;
}

}  // namespace sbse
