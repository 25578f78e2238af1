// Three-pass 3D FFT round trip for the grid edges N = 80 and 96 (FP32): the split-operator step
// of Eq. (10), the Poisson solves of Eq. (11) / q_ij and the exchange potentials of Eq. (1) on the
// paper-scale grids (the 520-electron system of Sec. III sits on ~0.85M points, 96^3 here).
//
// A pencil of N points is too long for one thread's registers next to the epilogue's state, so it
// is split over a lane pair (l, l ^ 16) of one warp: N = 2H, each lane holds H points, transforms
// them with the register FFT of length H, and one radix-2 butterfly across the pair (operands
// swapped by warp shuffles) completes the transform. Forward transforms take the pencil
// interleaved (lane s holds x[2m + s]) and return it in two quarter blocks (decimation in time);
// inverse transforms take the blocks and return the interleaved order (decimation in frequency),
// so no pass needs a reordering step. A warp transforms 16 pencils; 16 consecutive lanes always
// touch 16 consecutive grid points or rows of a padded shared-memory tile (conflict-free, 128-byte
// global segments).
//
// The split-operator step (Eq. 10) takes two sweeps over the orbitals: the kinetic propagator is
// the product of three one-dimensional operators (one per axis), so
//   plane kinetic : one z-plane per block (2N threads): fused pre-operation (potential phase), the
//                   x and then the y operator (forward FFT, exp(-i dt k^2 / 2) / N, inverse FFT)
//   z kinetic     : 16 columns per warp: the z operator, and for the pair batch the induced density
//                   of the pair's L orbitals (Eq. 11)
// The Poisson solves (4 pi / |G|^2 does not factor over the axes) keep the 3D round trip:
//   plane forward : pre-operation (packing), x FFTs in the padded tile, y FFTs stored to global
//   z columns     : forward z FFT, 4 pi / |G|^2 with 1/N^3, inverse z FFT
//   plane inverse : y then x inverse FFTs, then the unpacking with the damped time-integral
//                   accumulation of Eq. (13) and E - 1 of the next step
// Blocks are ordered plane-major (plane outer, item inner), so the tables read beside the orbitals
// (eta0 of each stochastic orbital, the potential phases, E - 1 of each pair) are the same z-slice
// for consecutive blocks and stay in L2 even when the whole table set does not fit there.
#include <math.h>

#include <type_traits>

#include "fft_reg.cuh"
#include "kernels.h"
#include "bounds.cuh"
#include "passes.cuh"
#include "tma.cuh"

namespace sbse {

namespace {

__constant__ float2 c_tws[kRegTotal];

struct TwS {
  __device__ __forceinline__ static float2 get(int i) { return c_tws[i]; }
};

constexpr unsigned kFull = 0xffffffffu;

// exp(SIGN 2 pi i k / N)
template <int N, int SIGN> __device__ __forceinline__ float2 tw_full(int k) {
  float2 w = TwS::get(reg_offset(N) + k);
  if (SIGN > 0) w.y = -w.y;
  return w;
}

__device__ __forceinline__ float2 shfl_pair(float2 v) {
  return make_float2(__shfl_xor_sync(kFull, v.x, 16), __shfl_xor_sync(kFull, v.y, 16));
}

// Decimation in time across the lane pair. On entry lane s of the pair holds x[2m + s], m < H;
// on return it holds X[s Q + j] in v[j] and X[H + s Q + j] in v[Q + j] (j < Q = H / 2), where
// X[k] = sum_n x[n] exp(SIGN 2 pi i n k / N): X[k] = E[k] + W^k O[k], X[k + H] = E[k] - W^k O[k]
// with E, O the H-point transforms of the even and odd samples.
template <int N, int SIGN> __device__ __forceinline__ void fft2_dit(float2 (&v)[N / 2], int s) {
  constexpr int H = N / 2, Q = H / 2;
  fft_reg<float, H, SIGN, TwS>(v);
#pragma unroll
  for (int j = 0; j < Q; ++j) {
    // lane 0 keeps E[j] and needs O[j]; lane 1 keeps O[Q + j] and needs E[Q + j]
    const float2 rcv = shfl_pair(s ? v[j] : v[Q + j]);
    const float2 e = s ? rcv : v[j];
    const float2 o = s ? v[Q + j] : rcv;
    float2 t = cmul(o, tw_full<N, SIGN>(j));
    if (s) t = cmul_si(t, SIGN);  // W^Q = exp(SIGN i pi / 2) = SIGN i
    v[j] = cadd(e, t);
    v[Q + j] = csub(e, t);
  }
}

// Decimation in frequency across the lane pair: the inverse of the layout change above. On entry
// lane s holds X[s Q + j] in v[j] and X[H + s Q + j] in v[Q + j]; on return it holds x[2m + s] in
// v[m], x[n] = sum_k X[k] exp(SIGN 2 pi i n k / N). The even outputs are the H-point transform of
// a_k = X[k] + X[k + H], the odd ones that of b_k = (X[k] - X[k + H]) W^k; lane 0 gathers every
// a_k and lane 1 every b_k.
template <int N, int SIGN> __device__ __forceinline__ void fft2_dif(float2 (&v)[N / 2], int s) {
  constexpr int H = N / 2, Q = H / 2;
#pragma unroll
  for (int j = 0; j < Q; ++j) {
    const float2 a = cadd(v[j], v[Q + j]);
    float2 b = cmul(csub(v[j], v[Q + j]), tw_full<N, SIGN>(j));
    if (s) b = cmul_si(b, SIGN);
    const float2 rcv = shfl_pair(s ? a : b);
    v[j] = s ? rcv : a;
    v[Q + j] = s ? b : rcv;
  }
  fft_reg<float, H, SIGN, TwS>(v);
}

// the padded plane tile; the density pass adds the pair's density accumulator (N^2 floats)
// One-dimensional kinetic operator F^-1 diag(K / N) F on the pencil held by a lane pair, without
// leaving registers: on entry lane s holds x[2m + s], on return y[2m + s] (y = F^-1 K F x / N). Each
// lane takes the half-length transform of its samples (E for the even ones, O for the odd ones),
// receives the other lane's, forms E Kp + O M1 (lane 0: even outputs) or O Kp + E M2 (lane 1: odd
// outputs), and transforms back. tab = [Kp | M1 | M2], N/2 entries each (see set_kinetic).
template <int N>
__device__ __forceinline__ void kin_roundtrip(float2 (&v)[N / 2], int s, const float2 *tab) {
  constexpr int H = N / 2;
  fft_reg<float, H, -1, TwS>(v);
  const float2 *mt = tab + (s ? 2 * H : H);
#pragma unroll
  for (int k = 0; k < H; ++k) {
    const float2 o = shfl_pair(v[k]);
    const float2 kp = tab[k], mk = mt[k];
    v[k] = cmac2(v[k], kp, o, mk);
  }
  fft_reg<float, H, +1, TwS>(v);
}

template <int N> constexpr size_t split_smem() { return (size_t)N * (N + 1) * sizeof(float2); }
template <int N> constexpr size_t split_density_smem() { return split_smem<N>() + (size_t)N * N * sizeof(float); }

// ------------------------------------------------------------------------------------------
// The pre-operation of a forward plane pass into the padded tile. Thread t of the 2N covers the
// points t + k 2N (k < N / 2) of the plane, i.e. row t / N + 2k, column t % N.
template <int N, bool PAIR>
__device__ __forceinline__ void preop_plane(const GView<float> &g, const XfwdArgs<float> &a, long long item,
                                            long long off, float2 *S) {
  using C = float2;
  constexpr int LD = N + 1, NT = 2 * N, KP = N / 2, UB = 8;
  const PreopItem<float> it = preop_item<float>(g, a, item);
  (void)SBSE_IDX(item, a.n_items);
  (void)SBSE_IDX(off + threadIdx.x + (long long)(KP - 1) * NT, g.ng);  // the largest point this thread reads
  if constexpr (PAIR) (void)SBSE_IDX(item / a.L, a.n_items / a.L);     // the pair of E - 1
  const int y0 = threadIdx.x / N;
  C *srow = S + y0 * LD + (threadIdx.x - y0 * N);
  if constexpr (PAIR) {
    const C *dp = it.in + off + threadIdx.x, *ap = it.a + off + threadIdx.x, *pp = it.pv + off + threadIdx.x;
    const C *ep = it.em1 ? it.em1 + off + threadIdx.x : nullptr;
    // the deferred renormalisation is pending only in the step after a cleaning (cm1 != 0, the same
    // for the whole block): the other steps skip its arithmetic (d is then unchanged by it)
    auto sweep = [&](auto renorm) {
      constexpr bool RN = decltype(renorm)::value;
#pragma unroll 1
      for (int k0 = 0; k0 < KP; k0 += UB) {
        C dv[UB], av[UB], pv[UB], ev[UB];
#pragma unroll
        for (int k = 0; k < UB; ++k) {
          if (k0 + k < KP) {
            const int l = (k0 + k) * NT;
            dv[k] = dp[l];
            av[k] = ap[l];
            pv[k] = pp[l];
            ev[k] = ep ? ep[l] : C{0.f, 0.f};
          }
        }
#pragma unroll
        for (int k = 0; k < UB; ++k)
          if (k0 + k < KP)
            srow[2 * (k0 + k) * LD] =
                pair_phase<float>(pv[k], ev[k], av[k], RN ? renorm_value<float>(dv[k], av[k], it.cm1) : dv[k]);
      }
    };
    if (it.cm1 != 0.f)
      sweep(std::true_type{});
    else
      sweep(std::false_type{});
  } else {
    auto run = [&](auto f) {
#pragma unroll 1
      for (int k0 = 0; k0 < KP; k0 += UB) {
        C v[UB];
#pragma unroll
        for (int k = 0; k < UB; ++k)
          if (k0 + k < KP) v[k] = f(off + threadIdx.x + (k0 + k) * NT);
#pragma unroll
        for (int k = 0; k < UB; ++k)
          if (k0 + k < KP) srow[2 * (k0 + k) * LD] = v[k];
      }
    };
    if (it.mode == XF_PHASE_A) {
      run([&](long long i) { return cmul(it.pv[i], it.in[i]); });
    } else if (it.mode == XF_PACK_DN) {
      if (it.r1)
        run([&](long long i) { return C{it.r0[i], it.r1[i]}; });
      else
        run([&](long long i) { return C{it.r0[i], 0.f}; });
    } else if (it.mode == XF_PACK_PROD) {
      if (it.r2)
        run([&](long long i) { return C{it.r0[i] * it.r1[i], it.r2[i] * it.r3[i]}; });
      else
        run([&](long long i) { return C{it.r0[i] * it.r1[i], 0.f}; });
    } else {
      run([&](long long i) { return preop_at<float>(g, it, i); });
    }
  }
}

// ------------------------------------------------------------------------------------------
// plane forward pass of the three-pass round trip (Poisson packing of densities and pair
// products): block = (plane z, item), 2N threads; x FFTs in the tile, y FFTs stored to global

template <int N>
__global__ void __launch_bounds__(2 * N, N == 96 ? 2 : 3) k_plane_fwd2(GView<float> g, XfwdArgs<float> a, int n_items) {
  using C = float2;
  constexpr int LD = N + 1, NN = N * N, H = N / 2, Q = H / 2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C *S = reinterpret_cast<C *>(smem_raw);
  const int z = (int)(blockIdx.x / (unsigned)n_items);
  const long long item = (long long)blockIdx.x - (long long)z * n_items;
  const long long off = (long long)z * NN;
  preop_plane<N, false>(g, a, item, off, S);
  __syncthreads();
  const int lane = threadIdx.x & 31, s = lane >> 4, p = (threadIdx.x >> 5) * 16 + (lane & 15);
  {  // x transforms, pencil p = row p of the tile, in place
    C v[H];
    C *row = S + p * LD;
#pragma unroll
    for (int m = 0; m < H; ++m) v[m] = row[2 * m + s];
    fft2_dit<N, -1>(v, s);
    __syncwarp();
#pragma unroll
    for (int j = 0; j < Q; ++j) {
      row[s * Q + j] = v[j];
      row[H + s * Q + j] = v[Q + j];
    }
  }
  __syncthreads();
  {  // y transforms, pencil p = column p, stored to global
    C v[H];
    const C *col = S + p;
#pragma unroll
    for (int m = 0; m < H; ++m) v[m] = col[(2 * m + s) * LD];
    fft2_dit<N, -1>(v, s);
    (void)SBSE_IDX(off + p + (long long)(N - 1) * N, g.ng);
    C *out = a.out + item * g.ng + off + p;
#pragma unroll
    for (int j = 0; j < Q; ++j) {
      out[(s * Q + j) * N] = v[j];
      out[(H + s * Q + j) * N] = v[Q + j];
    }
  }
}

// ------------------------------------------------------------------------------------------
// First sweep of the two-sweep split-operator step. The kinetic propagator of Eq. (10) is
// exp(-i dt |G|^2 / 2) = prod_axes exp(-i dt k_a^2 / 2), so in real space it is the product of three
// one-dimensional operators F_a^-1 K_a F_a, one per axis, which commute. This pass applies the
// potential phase (the pre-operation) and the x and y operators to one z-plane held in shared
// memory (kin_roundtrip along each axis); the second sweep applies the z operator. One HBM round trip per sweep: two per step instead of the three of a 3D FFT round trip.

template <int N, bool PAIR>
__global__ void __launch_bounds__(2 * N, N == 96 ? 2 : 3) k_plane_kin2(GView<float> g, XfwdArgs<float> a, int n_items) {
  using C = float2;
  constexpr int LD = N + 1, NN = N * N, H = N / 2, Q = H / 2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C *S = reinterpret_cast<C *>(smem_raw);
  const int z = (int)(blockIdx.x / (unsigned)n_items);
  const long long item = (long long)blockIdx.x - (long long)z * n_items;
  const long long off = (long long)z * NN;
  __shared__ C tab[3 * H];
  for (int i = threadIdx.x; i < 3 * H; i += blockDim.x) tab[i] = g.kin[N + i];
  preop_plane<N, PAIR>(g, a, item, off, S);
  __syncthreads();
  const int lane = threadIdx.x & 31, s = lane >> 4, p = (threadIdx.x >> 5) * 16 + (lane & 15);
  {  // x operator on row p, in place
    C v[H];
    C *row = S + p * LD;
#pragma unroll
    for (int m = 0; m < H; ++m) v[m] = row[2 * m + s];
    kin_roundtrip<N>(v, s, tab);
    __syncwarp();
#pragma unroll
    for (int m = 0; m < H; ++m) row[2 * m + s] = v[m];
  }
  __syncthreads();
  {  // y operator on column p, stored to global
    C v[H];
    const C *col = S + p;
#pragma unroll
    for (int m = 0; m < H; ++m) v[m] = col[(2 * m + s) * LD];
    kin_roundtrip<N>(v, s, tab);
    (void)SBSE_IDX(off + p + (long long)(N - 1) * N, g.ng);
    C *out = a.out + item * g.ng + off + p;
#pragma unroll
    for (int m = 0; m < H; ++m) out[(2 * m + s) * N] = v[m];
  }
}

// Second sweep: the z operator on 64 columns of one item (PLAIN) or of each of the L orbitals of a
// pair (DENS), which also sums the pair's induced density 2 sum_l (2 Re(conj(eta0_l) d_l) +
// |d_l|^2) (Eq. 11) in shared memory and writes it.
constexpr int kZDPitch = 80;  // density rows of 64 columns padded so the two half-warps miss each other's banks

template <int N, bool DENS>
__global__ void __launch_bounds__(128, 3) k_zkin2(GView<float> g, float2 *data, const float2 *a_next, float *dens,
                                                  int n_units, int L) {
  using C = float2;
  constexpr int NN = N * N, H = N / 2, UB = 16;
  __shared__ float D[DENS ? N * kZDPitch : 1];
  __shared__ C tab[3 * H];
  for (int i = threadIdx.x; i < 3 * H; i += blockDim.x) tab[i] = g.kin[N + i];
  __syncthreads();
  const int cs = (int)(blockIdx.x / (unsigned)n_units);
  const int unit = (int)blockIdx.x - cs * n_units;
  const int lane = threadIdx.x & 31, s = lane >> 4, cw = (threadIdx.x >> 5) * 16 + (lane & 15);
  const int rem = cs * 64 + cw;
  const int n_orb = DENS ? L : 1;
  (void)SBSE_IDX(rem, NN);
  for (int ell = 0; ell < n_orb; ++ell) {
    const long long item = DENS ? (long long)unit * L + ell : unit;
    (void)SBSE_IDX(item, (long long)n_units * n_orb);
    C *base = data + item * g.ng + rem;
    C v[H];
#pragma unroll
    for (int m = 0; m < H; ++m) v[m] = base[(long long)(2 * m + s) * NN];
    kin_roundtrip<N>(v, s, tab);
#pragma unroll
    for (int m = 0; m < H; ++m) base[(long long)(2 * m + s) * NN] = v[m];
    if constexpr (DENS) {
      const C *ab = a_next + (long long)ell * g.ng + rem;
#pragma unroll
      for (int m0 = 0; m0 < H; m0 += UB) {
        C a0[UB];
#pragma unroll
        for (int k = 0; k < UB; ++k)
          if (m0 + k < H) a0[k] = ab[(long long)(2 * (m0 + k) + s) * NN];
#pragma unroll
        for (int k = 0; k < UB; ++k) {
          if (m0 + k < H) {
            const C dv = v[m0 + k];
            const float t = 2.f * (2.f * (a0[k].x * dv.x + a0[k].y * dv.y) + dv.x * dv.x + dv.y * dv.y);
            float &acc = D[(2 * (m0 + k) + s) * kZDPitch + cw];
            acc = ell ? acc + t : t;
          }
        }
        // keep the loads of the next batch below this one (hoisting them all costs registers)
        asm volatile("" ::: "memory");
      }
    }
  }
  if constexpr (DENS) {
    float *db = dens + (long long)unit * g.ng + rem;
#pragma unroll 8
    for (int m = 0; m < H; ++m) db[(long long)(2 * m + s) * NN] = D[(2 * m + s) * kZDPitch + cw];
  }
}

// The same sweep for the pair batch with the columns of the next orbital staged in shared memory
// by one bulk tensor copy (N z-rows x ZT_CW columns) while the current orbital is transformed, so
// the column loads no longer stall the warps. ZT_CW = 32 columns (two warps) per block keep the
// stage (24 KB at N = 96) and the density rows small enough for five blocks per SM.
constexpr int kZtCw = 32;
constexpr int kZtPitch = kZtCw + 16;  // density rows: the two half-warps' rows fall on different banks

// dynamic shared memory of the staged z sweep: the stage and the density rows, plus the slack that
// lets the kernel start the stage on a 128-byte boundary (the alignment a tensor copy's shared
// destination needs; the dynamic region itself follows the static variables)
constexpr unsigned kZtAlign = 128;
template <int N> constexpr size_t ztma_smem() {
  return (size_t)N * kZtCw * sizeof(float2) + (size_t)N * kZtPitch * sizeof(float) + kZtAlign;
}

__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, int x, int y, int z, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(
          tma_smem_addr(dst)),
      "l"((uint64_t)(uintptr_t)map), "r"(x), "r"(y), "r"(z), "r"(tma_smem_addr(bar))
      : "memory");
}

template <int N>
__global__ void __launch_bounds__(2 * kZtCw, 5)
    k_zkin2_tma(const __grid_constant__ CUtensorMap dmap, GView<float> g, float2 *data, const float2 *a_next,
                float *dens, int n_units, int L, int *err) {
  using C = float2;
  constexpr int NN = N * N, H = N / 2, UB = 48;
  constexpr unsigned kStage = (unsigned)N * kZtCw * sizeof(C);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned char *smem = smem_raw + ((kZtAlign - (tma_smem_addr(smem_raw) & (kZtAlign - 1))) & (kZtAlign - 1));
  C *St = reinterpret_cast<C *>(smem);                    // [z][column], 128-byte aligned
  float *D = reinterpret_cast<float *>(smem + kStage);    // [z][kZtPitch]
  __shared__ C tab[3 * H];
  __shared__ __align__(8) uint64_t bar;
  const int cs = (int)(blockIdx.x / (unsigned)n_units);
  const int unit = (int)blockIdx.x - cs * n_units;
  const long long item0 = (long long)unit * L;
  if (tma_smem_addr(St) & (kZtAlign - 1)) {  // never expected: report instead of issuing the copy
    if (threadIdx.x == 0) atomicExch(err, 1);
    return;
  }
  if (threadIdx.x == 0) {
    tma_bar_init(&bar, 1);
    tma_bar_expect(&bar, kStage);
    tma_load_3d(St, &dmap, 2 * cs * kZtCw, 0, (int)item0, &bar);
  }
  for (int i = threadIdx.x; i < 3 * H; i += blockDim.x) tab[i] = g.kin[N + i];
  __syncthreads();
  const int lane = threadIdx.x & 31, s = lane >> 4, cw = (threadIdx.x >> 5) * 16 + (lane & 15);
  const int rem = cs * kZtCw + cw;
  (void)SBSE_IDX(rem, NN);
  (void)SBSE_IDX(item0 + L - 1, (long long)n_units * L);
  int failed = -1;  // the orbital whose copy did not land in time
  for (int ell = 0; ell < L; ++ell) {
    if (!__syncthreads_and(tma_bar_wait(&bar, (unsigned)(ell & 1)))) {
      failed = ell;
      break;
    }
    C v[H];
#pragma unroll
    for (int m = 0; m < H; ++m) v[m] = St[(2 * m + s) * kZtCw + cw];
    __syncthreads();  // every thread holds its columns: the stage can take the next orbital
    if (threadIdx.x == 0 && ell + 1 < L) {
      tma_fence_proxy();
      tma_bar_expect(&bar, kStage);
      tma_load_3d(St, &dmap, 2 * cs * kZtCw, 0, (int)(item0 + ell + 1), &bar);
    }
    kin_roundtrip<N>(v, s, tab);
    C *base = data + (item0 + ell) * g.ng + rem;
#pragma unroll
    for (int m = 0; m < H; ++m) base[(long long)(2 * m + s) * NN] = v[m];
    const C *ab = a_next + (long long)ell * g.ng + rem;
#pragma unroll
    for (int m0 = 0; m0 < H; m0 += UB) {
      C a0[UB];
#pragma unroll
      for (int k = 0; k < UB; ++k)
        if (m0 + k < H) a0[k] = ab[(long long)(2 * (m0 + k) + s) * NN];
#pragma unroll
      for (int k = 0; k < UB; ++k) {
        if (m0 + k < H) {
          const C dv = v[m0 + k];
          const float t = 2.f * (2.f * (a0[k].x * dv.x + a0[k].y * dv.y) + dv.x * dv.x + dv.y * dv.y);
          float &acc = D[(2 * (m0 + k) + s) * kZtPitch + cw];
          acc = ell ? acc + t : t;
        }
      }
      asm volatile("" ::: "memory");
    }
  }
  if (failed >= 0) {
    if (threadIdx.x == 0) {
      atomicExch(err, 1);
      tma_bar_wait(&bar, (unsigned)(failed & 1));  // the copy still in flight: a bounded chance to land
    }
    __syncthreads();
    return;
  }
  __syncthreads();
  float *db = dens + (long long)unit * g.ng + rem;
#pragma unroll 8
  for (int m = 0; m < H; ++m) db[(long long)(2 * m + s) * NN] = D[(2 * m + s) * kZtPitch + cw];
}

// ------------------------------------------------------------------------------------------
// z columns: 64 columns per block of 128 threads (NN is a multiple of 64 for N = 80, 96)

template <int N>
__global__ void __launch_bounds__(128, 4) k_zcol2(GView<float> g, float2 *data, int mult, int n_items) {
  using C = float2;
  constexpr int NN = N * N, H = N / 2, Q = H / 2;
  const int lane = threadIdx.x & 31, s = lane >> 4;
  const long long c = (long long)blockIdx.x * 64 + (threadIdx.x >> 5) * 16 + (lane & 15);
  const long long item = c / NN;
  const int rem = (int)(c - item * NN), y = rem / N, x = rem - y * N;
  (void)SBSE_IDX(item, n_items);
  C *base = data + item * g.ng + rem;
  C v[H];
#pragma unroll
  for (int m = 0; m < H; ++m) v[m] = base[(long long)(2 * m + s) * NN];
  fft2_dit<N, -1>(v, s);
  const float inv_ng = 1.f / (float)(N * N * N);
  if (mult == Z_KINETIC) {
    const C mxy = cscale(cmul(g.kin[x], g.kin[y]), inv_ng);
#pragma unroll
    for (int j = 0; j < Q; ++j) {
      v[j] = cmul(v[j], cmul(mxy, g.kin[s * Q + j]));
      v[Q + j] = cmul(v[Q + j], cmul(mxy, g.kin[H + s * Q + j]));
    }
  } else {
    const float gxy = g.k2[x] + g.k2[y];
#pragma unroll
    for (int j = 0; j < Q; ++j) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const float G2 = gxy + g.k2[h * H + s * Q + j];
        const float f = mult == Z_HALF_G2 ? 0.5f * G2 * inv_ng : (G2 > 0.f ? float(4.0 * M_PI) * inv_ng / G2 : 0.f);
        v[h * Q + j] = cscale(v[h * Q + j], f);
      }
    }
  }
  fft2_dif<N, +1>(v, s);
#pragma unroll
  for (int m = 0; m < H; ++m) base[(long long)(2 * m + s) * NN] = v[m];
}

// ------------------------------------------------------------------------------------------
// plane inverse pass of the Poisson round trip: block = (plane z, packed slot). y then x inverse
// FFTs of the plane, then the epilogue: the two real potentials of the slot, u, the damped time
// integral of Eq. (13) and E - 1 for the next step.

template <int N>
__global__ void __launch_bounds__(2 * N, N == 96 ? 2 : 3) k_plane_inv2(GView<float> g, float2 *data, float *u_out,
                                                                       float *acc, float2 *em1_out, int n_units,
                                                                       PoissonOut po) {
  using C = float2;
  constexpr int LD = N + 1, NN = N * N, NT = 2 * N, H = N / 2, Q = H / 2, KP = NN / NT;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C *S = reinterpret_cast<C *>(smem_raw);
  const int z = (int)(blockIdx.x / (unsigned)n_units);
  const long long item = (long long)blockIdx.x - (long long)z * n_units;
  const long long off = (long long)z * NN;
  const int lane = threadIdx.x & 31, s = lane >> 4, p = (threadIdx.x >> 5) * 16 + (lane & 15);
  (void)SBSE_IDX(off + p + (long long)(N - 1) * N, g.ng);
  (void)SBSE_IDX(2 * item + 1, 2ll * n_units);  // the slot's two densities
  {  // y inverse FFTs from global (frequency blocks) into the tile (interleaved rows)
    C v[H];
    const C *col = data + item * g.ng + off + p;
#pragma unroll
    for (int j = 0; j < Q; ++j) {
      v[j] = col[(s * Q + j) * N];
      v[Q + j] = col[(H + s * Q + j) * N];
    }
    fft2_dif<N, +1>(v, s);
#pragma unroll
    for (int m = 0; m < H; ++m) S[(2 * m + s) * LD + p] = v[m];
  }
  __syncthreads();
  {  // x inverse FFTs in the tile
    C v[H];
    C *row = S + p * LD;
#pragma unroll
    for (int j = 0; j < Q; ++j) {
      v[j] = row[s * Q + j];
      v[Q + j] = row[H + s * Q + j];
    }
    fft2_dif<N, +1>(v, s);
    __syncwarp();
#pragma unroll
    for (int m = 0; m < H; ++m) row[2 * m + s] = v[m];
  }
  __syncthreads();
  const float coef = (float)po.coef, tau = (float)po.tau_next;
  const bool keep = po.keep != 0.0;
  const int n_h = (2 * item + 1 < po.n_out) ? 2 : 1;
  const int y0 = threadIdx.x / N;
  const C *srow = S + y0 * LD + (threadIdx.x - y0 * N);
  constexpr int UB = 8;
#pragma unroll 1
  for (int k0 = 0; k0 < KP; k0 += UB) {
    C v[UB];
    float old[UB][2];
#pragma unroll
    for (int k = 0; k < UB; ++k) {
      if (k0 + k >= KP) break;
      const int l = threadIdx.x + (k0 + k) * NT;
      v[k] = srow[2 * (k0 + k) * LD];
#pragma unroll
      for (int h = 0; h < 2; ++h)
        old[k][h] = (acc && keep && h < n_h) ? acc[(2 * item + h) * g.ng + off + l] : 0.f;
    }
#pragma unroll
    for (int k = 0; k < UB; ++k) {
      if (k0 + k >= KP) break;
      const int l = threadIdx.x + (k0 + k) * NT;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        if (h >= n_h) break;
        const float val = h ? v[k].y : v[k].x;
        const long long o = (2 * item + h) * g.ng + off + l;
        if (u_out) u_out[o] = val;
        if (acc) acc[o] = old[k][h] + coef * val;
        if (em1_out) em1_out[o] = phase_em1<float>(val, tau);
      }
    }
  }
}

template <int N> void set_split_attrs() {
  const int sm = (int)split_smem<N>();
  cudaFuncSetAttribute(k_plane_fwd2<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  cudaFuncSetAttribute(k_plane_kin2<N, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  cudaFuncSetAttribute(k_plane_kin2<N, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  cudaFuncSetAttribute(k_plane_inv2<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
}

template <int N> void fwd2(const GridTables<float> &g, const XfwdArgs<float> &a, cudaStream_t s) {
  k_plane_fwd2<N><<<(unsigned)a.n_items * N, 2 * N, split_smem<N>(), s>>>(view(g), a, a.n_items);
}

template <int N> void kin2(const GridTables<float> &g, const XfwdArgs<float> &a, cudaStream_t s) {
  const unsigned blocks = (unsigned)a.n_items * N;
  if (a.mode == XF_PHASE_PAIR)
    k_plane_kin2<N, true><<<blocks, 2 * N, split_smem<N>(), s>>>(view(g), a, a.n_items);
  else
    k_plane_kin2<N, false><<<blocks, 2 * N, split_smem<N>(), s>>>(view(g), a, a.n_items);
}

template <int N> void zcol2(const GridTables<float> &g, float2 *d, int n_items, int mult, cudaStream_t s) {
  static_assert((N * N) % 64 == 0, "z pass blocks hold 64 whole columns");
  const unsigned blocks = (unsigned)((long long)n_items * N * N / 64);
  k_zcol2<N><<<blocks, 128, 0, s>>>(view(g), d, mult, n_items);
}

template <int N>
void zkin2(const GridTables<float> &g, float2 *d, int n_items, const float2 *a_next, int L, float *dens,
           cudaStream_t s, int *err) {
  const int units = dens ? n_items / L : n_items;
  if (dens && err) {
    // d as n_items orbitals x N z-planes x 2 N^2 floats; boxes of 2 ZT_CW floats x N planes x 1
    CUtensorMap map;
    const uint64_t dims[3] = {(uint64_t)2 * N * N, (uint64_t)N, (uint64_t)n_items};
    const uint64_t strides[2] = {(uint64_t)N * N * sizeof(float2), (uint64_t)g.ng * sizeof(float2)};
    const uint32_t box[3] = {2u * kZtCw, (uint32_t)N, 1u};
    if (make_tensor_map_f32(&map, d, 3, dims, strides, box, false)) {
      raise_smem_limit((const void *)k_zkin2_tma<N>, ztma_smem<N>());
      const unsigned blocks = (unsigned)units * (N * N / kZtCw);
      k_zkin2_tma<N><<<blocks, 2 * kZtCw, ztma_smem<N>(), s>>>(map, view(g), d, a_next, dens, units, L, err);
      return;
    }
  }
  const unsigned blocks = (unsigned)units * (N * N / 64);
  if (dens)
    k_zkin2<N, true><<<blocks, 128, 0, s>>>(view(g), d, a_next, dens, units, L);
  else
    k_zkin2<N, false><<<blocks, 128, 0, s>>>(view(g), d, nullptr, nullptr, units, 1);
}

template <int N>
void inv2(const GridTables<float> &g, float2 *d, int n_units, float *u_out, float *acc, float2 *em1_out,
          const PoissonOut &po, cudaStream_t s) {
  k_plane_inv2<N><<<(unsigned)n_units * N, 2 * N, split_smem<N>(), s>>>(view(g), d, u_out, acc, em1_out, n_units,
                                                                      po);
}

}  // namespace

bool split_size(int N) { return N == 80 || N == 96; }

int upload_split_twiddles() {
  float2 hf[kRegTotal];
  for (int s = 0; s < kRegCount; ++s) {
    const int N = kRegSizes[s], off = reg_offset(N);
    for (int k = 0; k < N; ++k) {
      const double a = -2.0 * M_PI * (double)k / (double)N;
      hf[off + k] = make_float2((float)cos(a), (float)sin(a));
    }
  }
  return cudaMemcpyToSymbol(c_tws, hf, sizeof(hf)) == cudaSuccess ? 0 : -1;
}

void init_split_kernels() {
  set_split_attrs<80>();
  set_split_attrs<96>();
}

void launch_plane_fwd2(const GridTables<float> &g, const XfwdArgs<float> &a, cudaStream_t s) {
  if (g.N == 80) fwd2<80>(g, a, s);
  else if (g.N == 96) fwd2<96>(g, a, s);
}

void launch_zcol2(const GridTables<float> &g, float2 *d, int n_items, int mult, cudaStream_t s) {
  if (g.N == 80) zcol2<80>(g, d, n_items, mult, s);
  else if (g.N == 96) zcol2<96>(g, d, n_items, mult, s);
}

void launch_plane_inv2_poisson(const GridTables<float> &g, float2 *d, int n_slots, const PoissonOut &po,
                               float *u_out, float *acc, float2 *em1_out, cudaStream_t s) {
  if (g.N == 80) inv2<80>(g, d, n_slots, u_out, acc, em1_out, po, s);
  else if (g.N == 96) inv2<96>(g, d, n_slots, u_out, acc, em1_out, po, s);
}

void launch_plane_kin2(const GridTables<float> &g, const XfwdArgs<float> &a, cudaStream_t s) {
  if (g.N == 80) kin2<80>(g, a, s);
  else if (g.N == 96) kin2<96>(g, a, s);
}

void launch_zkin2(const GridTables<float> &g, float2 *d, int n_items, const float2 *a_next, int L, float *dens,
                  cudaStream_t s, int *err) {
  if (g.N == 80) zkin2<80>(g, d, n_items, a_next, L, dens, s, err);
  else if (g.N == 96) zkin2<96>(g, d, n_items, a_next, L, dens, s, err);
}

}  // namespace sbse
