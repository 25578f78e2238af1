// Three-pass 3D FFT round trip with compile-time N and register-resident pencils, used by the
// split-operator step of Eq. (10), the Poisson solves of Eq. (11) / q_ij and the exchange
// potentials of Eq. (1):
//   plane forward  : coalesced load of PPB z-planes with the fused pre-operation into shared
//                    memory (rows padded to N + 1), x FFT (thread per row), y FFT (thread per
//                    column), coalesced store
//   z column       : thread per (x, y) column, coalesced across x: forward z FFT, multiplier
//                    (kinetic propagator exp(-i |G|^2 dt / 2) or 4 pi / |G|^2, with 1/N^3),
//                    inverse z FFT, store
//   plane inverse  : y and x inverse FFTs, then the fused epilogue: plain store, store plus the
//                    induced density of all L orbitals of a pair (Eq. 11), or the Poisson
//                    unpacking with the damped time-integral accumulation of Eq. (13)
// Each element crosses HBM three times per round trip instead of five for the generic passes.
#include <math.h>

#include "fft_reg.cuh"
#include "bounds.cuh"
#include "kernels.h"
#include "passes.cuh"
#include "tma.cuh"

namespace sbse {

__constant__ float2 c_twf[kRegTotal];
__constant__ double2 c_twd[kRegTotal];

template <> struct TwTab<float> {
  __device__ __forceinline__ static float2 get(int i) { return c_twf[i]; }
};
template <> struct TwTab<double> {
  __device__ __forceinline__ static double2 get(int i) { return c_twd[i]; }
};

int upload_reg_twiddles() {
  float2 hf[kRegTotal];
  double2 hd[kRegTotal];
  for (int s = 0; s < kRegCount; ++s) {
    const int N = kRegSizes[s], off = reg_offset(N);
    for (int k = 0; k < N; ++k) {
      const double a = -2.0 * M_PI * (double)k / (double)N;
      hd[off + k] = make_double2(cos(a), sin(a));
      hf[off + k] = make_float2((float)cos(a), (float)sin(a));
    }
  }
  if (cudaMemcpyToSymbol(c_twf, hf, sizeof(hf)) != cudaSuccess) return -1;
  if (cudaMemcpyToSymbol(c_twd, hd, sizeof(hd)) != cudaSuccess) return -1;
  return 0;
}

// Loads of data that other blocks of the same launch may have written (persistent step kernel)
// bypass L1, which is not coherent across SMs.
template <bool COH, typename C> __device__ __forceinline__ C ldv(const C *p) {
  if constexpr (COH) return __ldcg(p);
  else return *p;
}

// planes per block: the largest divisor of N with <= 256 threads and <= 96 KB of shared memory
constexpr int plane_ppb(int N, int csize) {
  int best = 1;
  for (int d = 1; d <= N; ++d)
    if (N % d == 0 && d * N <= 256 && (long long)d * N * (N + 1) * csize <= 96 * 1024) best = d;
  return best;
}

template <typename T, int N> constexpr int kPPB = plane_ppb(N, (int)sizeof(C2<T>));
template <typename T, int N> constexpr size_t plane_smem() {
  return (size_t)kPPB<T, N> * N * (N + 1) * sizeof(C2<T>);
}

// ------------------------------------------------------------------------------------------

// forward x and y FFTs of the PPB planes starting at plane offset `off` (= z0 N^2) of `item`, with
// the fused pre-operation; S is the block's shared tile
template <typename T, int N, bool PAIR, int PPB = kPPB<T, N>>
__device__ __forceinline__ void fwd_planes(const GView<T> &g, const XfwdArgs<T> &a, long long item,
                                           long long off, C2<T> *S) {
  using C = C2<T>;
  constexpr int LD = N + 1, NN = N * N, NT = PPB * N;
  const PreopItem<T> it = preop_item<T>(g, a, item);
  if constexpr (PAIR) {
    // the hot pre-operation of the pair batch: loads of 8 points are issued before any is used;
    // the batch loop stays rolled (the unrolled one stalled on instruction fetch: 162 -> 156 us)
    constexpr int UB = 8;
    const C *dp = it.in + off, *ap = it.a + off, *pp = it.pv + off;
    const C *ep = it.em1 ? it.em1 + off : nullptr;
#pragma unroll 1
    for (int k0 = 0; k0 < N; k0 += UB) {
      C dv[UB], av[UB], pv[UB], ev[UB];
#pragma unroll
      for (int k = 0; k < UB; ++k) {
        if (k0 + k < N) {
          const int l = threadIdx.x + (k0 + k) * NT;
          dv[k] = dp[l];
          av[k] = ap[l];
          pv[k] = pp[l];
          ev[k] = ep ? ep[l] : C{T(0), T(0)};
        }
      }
#pragma unroll
      for (int k = 0; k < UB; ++k) {
        if (k0 + k < N) {
          const int l = threadIdx.x + (k0 + k) * NT;
          const int pl = l / NN, rem = l - pl * NN, y = rem / N, x = rem - y * N;
          S[(pl * N + y) * LD + x] = pair_phase<T>(pv[k], ev[k], av[k], renorm_value<T>(dv[k], av[k], it.cm1));
        }
      }
    }
  } else {
    // the other pre-operations, with the mode resolved outside the point loop so that each batch
    // of UB points issues all its loads before the first shared-memory store
    constexpr int UB = 8;
    auto run = [&](auto f) {
      // the batch loop is not unrolled: five variants of fully unrolled point loops overflowed the
      // instruction cache (no-instruction stalls)
#pragma unroll 1
      for (int k0 = 0; k0 < N; k0 += UB) {
        C v[UB];
#pragma unroll
        for (int k = 0; k < UB; ++k)
          if (k0 + k < N) v[k] = f(off + threadIdx.x + (k0 + k) * NT);
#pragma unroll
        for (int k = 0; k < UB; ++k) {
          if (k0 + k < N) {
            const int l = threadIdx.x + (k0 + k) * NT;
            const int pl = l / NN, rem = l - pl * NN, y = rem / N, x = rem - y * N;
            S[(pl * N + y) * LD + x] = v[k];
          }
        }
      }
    };
    if (it.mode == XF_PHASE_A) {
      run([&](long long i) { return cmul(it.pv[i], it.in[i]); });
    } else if (it.mode == XF_PACK_DN) {
      if (it.r1)
        run([&](long long i) { return C{it.r0[i], it.r1[i]}; });
      else
        run([&](long long i) { return C{it.r0[i], T(0)}; });
    } else if (it.mode == XF_PACK_PROD) {
      if (it.r2)
        run([&](long long i) { return C{it.r0[i] * it.r1[i], it.r2[i] * it.r3[i]}; });
      else
        run([&](long long i) { return C{it.r0[i] * it.r1[i], T(0)}; });
    } else {
      run([&](long long i) { return preop_at<T>(g, it, i); });
    }
  }
  __syncthreads();
  const int pl = threadIdx.x / N, q = threadIdx.x - pl * N;
  {
    C v[N];
    C *row = S + (pl * N + q) * LD;
#pragma unroll
    for (int x = 0; x < N; ++x) v[x] = row[x];
    fft_reg<T, N, -1>(v);
#pragma unroll
    for (int x = 0; x < N; ++x) row[x] = v[x];
  }
  __syncthreads();
  {
    C v[N];
    const C *col = S + pl * N * LD + q;
#pragma unroll
    for (int y = 0; y < N; ++y) v[y] = col[y * LD];
    fft_reg<T, N, -1>(v);
    C *out = a.out + item * g.ng + off + pl * NN + q;
#pragma unroll
    for (int y = 0; y < N; ++y) out[y * N] = v[y];
  }
}

// planes per block of the forward pass: the FP32 pair batch takes half the planes of the other
// passes (smaller blocks: five resident per SM instead of two, 15 warps instead of 12, to hide
// the L2 latency of its pre-operation's table loads)
template <typename T, int N, bool PAIR> constexpr int fwd_ppb() {
  return (PAIR && sizeof(T) == 4 && kPPB<T, N> % 2 == 0) ? kPPB<T, N> / 2 : kPPB<T, N>;
}
template <typename T, int N, bool PAIR> constexpr size_t fwd_smem() {
  return (size_t)fwd_ppb<T, N, PAIR>() * N * (N + 1) * sizeof(C2<T>);
}

template <typename T, int N, bool PAIR>
__global__ void __launch_bounds__(fwd_ppb<T, N, PAIR>() * N)
    k_plane_fwd(GView<T> g, XfwdArgs<T> a, long long planes_total) {
  constexpr int PPB = fwd_ppb<T, N, PAIR>(), NN = N * N;
  extern __shared__ unsigned char smem_raw[];
  // PPB divides N: the block's planes z0 .. z0 + PPB - 1 are contiguous inside one item
  const long long p0 = (long long)blockIdx.x * PPB;
  const long long item = p0 / N;
  (void)SBSE_IDX(p0 + PPB - 1, planes_total);
  (void)SBSE_IDX(item, a.n_items);
  fwd_planes<T, N, PAIR, PPB>(g, a, item, (p0 - item * N) * NN, reinterpret_cast<C2<T> *>(smem_raw));
}

// one (x, y) column of one item: forward z FFT, multiplier, inverse z FFT (thread per column)
template <typename T, int N, bool COH>
__device__ __forceinline__ void zcol_column(const GView<T> &g, C2<T> *data, long long item, int rem,
                                            int mult) {
  using C = C2<T>;
  constexpr int NN = N * N;
  const int y = rem / N, x = rem - y * N;
  C *base = data + item * g.ng + rem;
  C v[N];
#pragma unroll
  for (int z = 0; z < N; ++z) v[z] = ldv<COH>(base + (long long)z * NN);
  fft_reg<T, N, -1>(v);
  const T inv_ng = T(1) / T(N * N * N);
  if (mult == Z_KINETIC) {
    const C mxy = cscale(cmul(g.kin[x], g.kin[y]), inv_ng);
#pragma unroll
    for (int z = 0; z < N; ++z) v[z] = cmul(v[z], cmul(mxy, g.kin[z]));
  } else if (mult == Z_HALF_G2) {
    const T gxy = g.k2[x] + g.k2[y];
#pragma unroll
    for (int z = 0; z < N; ++z) v[z] = cscale(v[z], T(0.5) * (gxy + g.k2[z]) * inv_ng);
  } else {
    const T gxy = g.k2[x] + g.k2[y];
#pragma unroll
    for (int z = 0; z < N; ++z) {
      const T G2 = gxy + g.k2[z];
      v[z] = cscale(v[z], G2 > T(0) ? T(4.0 * M_PI) * inv_ng / G2 : T(0));
    }
  }
  fft_reg<T, N, +1>(v);
#pragma unroll
  for (int z = 0; z < N; ++z) base[(long long)z * NN] = v[z];
}

template <typename T, int N>
__global__ void __launch_bounds__(128) k_zcol(GView<T> g, C2<T> *data, long long cols_total, int mult) {
  constexpr int NN = N * N;
  const long long c = (long long)blockIdx.x * 128 + threadIdx.x;
  if (c >= cols_total) return;
  const long long item = c / NN;
  zcol_column<T, N, false>(g, data, item, (int)(c - item * NN), mult);
}

enum PlaneInvMode { PI_PLAIN = 0, PI_DENSITY = 1, PI_POISSON = 2 };

struct PlaneInvArgs {
  long long planes_total;  // PLAIN, POISSON: planes of all items
  int L;                   // DENSITY: orbitals per pair
  PoissonOut po;           // POISSON
};

// y then x inverse transforms of PPB planes held in shared memory
template <typename T, int N, bool COH = false>
__device__ __forceinline__ void plane_inverse(C2<T> *S, const C2<T> *src_item_plane0, int pl, int q) {
  using C = C2<T>;
  constexpr int LD = N + 1, NN = N * N;
  {
    C v[N];
    const C *col = src_item_plane0 + (long long)pl * NN + q;
#pragma unroll
    for (int y = 0; y < N; ++y) v[y] = ldv<COH>(col + y * N);
    fft_reg<T, N, +1>(v);
    C *dst = S + pl * N * LD + q;
#pragma unroll
    for (int y = 0; y < N; ++y) dst[y * LD] = v[y];
  }
  __syncthreads();
  {
    C v[N];
    C *row = S + (pl * N + q) * LD;
#pragma unroll
    for (int x = 0; x < N; ++x) v[x] = row[x];
    fft_reg<T, N, +1>(v);
#pragma unroll
    for (int x = 0; x < N; ++x) row[x] = v[x];
  }
  __syncthreads();
}

// y, x inverse FFTs of the planes z0 .. z0 + PPB - 1 of the L orbitals of `pair`, storing each and
// accumulating the induced density 2 sum_l (2 Re(conj(eta0_l) d_l) + |d_l|^2) (Eq. 11)
template <typename T, int N, bool COH>
__device__ __forceinline__ void inv_density_planes(const GView<T> &g, C2<T> *data, const C2<T> *a_next,
                                                   T *dens, int pair, int L, int z0, C2<T> *S) {
  using C = C2<T>;
  constexpr int PPB = kPPB<T, N>, LD = N + 1, NN = N * N, NT = PPB * N;
  const int pl = threadIdx.x / N, q = threadIdx.x - pl * N;
  T accd[N];
#pragma unroll
  for (int k = 0; k < N; ++k) accd[k] = T(0);
  for (int ell = 0; ell < L; ++ell) {
    const long long item = (long long)pair * L + ell;
    (void)SBSE_IDX((long long)z0 * NN + NN * PPB - 1, g.ng);  // the block's planes inside the item
    C *base = data + item * g.ng + (long long)z0 * NN;
    plane_inverse<T, N, COH>(S, base, pl, q);
    const C *ab = a_next + (long long)ell * g.ng + (long long)z0 * NN;
#pragma unroll
    for (int k = 0; k < N; ++k) {
      const int l = threadIdx.x + k * NT;
      const int p = l / NN, rem = l - p * NN, y = rem / N, x = rem - y * N;
      const C dv = S[(p * N + y) * LD + x];
      base[l] = dv;
      const C a0 = ldv<COH>(ab + l);
      accd[k] += T(2) * (T(2) * (a0.x * dv.x + a0.y * dv.y) + dv.x * dv.x + dv.y * dv.y);
    }
    __syncthreads();
  }
  T *db = dens + (long long)pair * g.ng + (long long)z0 * NN;
#pragma unroll
  for (int k = 0; k < N; ++k) db[threadIdx.x + k * NT] = accd[k];
}

// y, x inverse FFTs of the PPB planes at plane offset `off` of `item`, stored back in place
template <typename T, int N, bool COH>
__device__ __forceinline__ void inv_plain_planes(const GView<T> &g, C2<T> *data, long long item,
                                                 long long off, C2<T> *S) {
  using C = C2<T>;
  constexpr int PPB = kPPB<T, N>, LD = N + 1, NN = N * N, NT = PPB * N;
  const int pl = threadIdx.x / N, q = threadIdx.x - pl * N;
  C *base = data + item * g.ng + off;
  plane_inverse<T, N, COH>(S, base, pl, q);
#pragma unroll 4
  for (int k = 0; k < N; ++k) {
    const int l = threadIdx.x + k * NT;
    const int p = l / NN, rem = l - p * NN, y = rem / N, x = rem - y * N;
    base[l] = S[(p * N + y) * LD + x];
  }
}

template <typename T, int N, int MODE>
__global__ void __launch_bounds__(kPPB<T, N> * N)
    k_plane_inv(GView<T> g, C2<T> *data, const C2<T> *a_next, T *dens, T *u_out, T *acc,
                C2<T> *em1_out, PlaneInvArgs pa) {
  using C = C2<T>;
  constexpr int PPB = kPPB<T, N>, LD = N + 1, NN = N * N, NT = PPB * N;
  extern __shared__ unsigned char smem_raw[];
  C *S = reinterpret_cast<C *>(smem_raw);
  const int pl = threadIdx.x / N, q = threadIdx.x - pl * N;
  if (MODE == PI_DENSITY) {
    // blockIdx.y = pair, blockIdx.x = group of PPB planes of each of its L orbitals
    inv_density_planes<T, N, false>(g, data, a_next, dens, blockIdx.y, pa.L, blockIdx.x * PPB, S);
    return;
  }
  const long long p0 = (long long)blockIdx.x * PPB;  // PPB divides N: all planes of one item
  const long long item = p0 / N;
  const long long off = (p0 - item * N) * NN;
  if (MODE == PI_PLAIN) {
    inv_plain_planes<T, N, false>(g, data, item, off, S);
    return;
  }
  C *base = data + item * g.ng + off;
  plane_inverse<T, N>(S, base, pl, q);
  // Poisson epilogue: unpack the two real potentials of the item, store u, accumulate the damped
  // time integral and store E - 1; the accumulator loads of a batch are issued together
  const T coef = (T)pa.po.coef, tau = (T)pa.po.tau_next;
  const bool keep = pa.po.keep != 0.0;
  const int n_h = (2 * item + 1 < pa.po.n_out) ? 2 : 1;
  constexpr int UB = 8;
#pragma unroll 1  // code size: the unrolled epilogue missed the instruction cache
  for (int k0 = 0; k0 < N; k0 += UB) {
    C v[UB];
    T old[UB][2];
#pragma unroll
    for (int k = 0; k < UB; ++k) {
      if (k0 + k >= N) break;
      const int l = threadIdx.x + (k0 + k) * NT;
      const int p = l / NN, rem = l - p * NN, y = rem / N, x = rem - y * N;
      v[k] = S[(p * N + y) * LD + x];
#pragma unroll
      for (int h = 0; h < 2; ++h)
        old[k][h] = (acc && keep && h < n_h) ? acc[(2 * item + h) * g.ng + off + l] : T(0);
    }
#pragma unroll
    for (int k = 0; k < UB; ++k) {
      if (k0 + k >= N) break;
      const int l = threadIdx.x + (k0 + k) * NT;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        if (h >= n_h) break;
        const T val = h ? v[k].y : v[k].x;
        const long long o = (2 * item + h) * g.ng + off + l;
        if (u_out) u_out[o] = val;
        if (acc) acc[o] = old[k][h] + coef * val;
        if (em1_out) em1_out[o] = phase_em1<T>(val, tau);
      }
    }
  }
}

// ------------------------------------------------------------------------------------------
// Inverse plane pass of the pair batch with the induced density, streamed by bulk copies (TMA):
// a persistent block walks its (pair, plane group) units and, inside each, the L orbitals; the PPB
// contiguous planes of the next orbital (and of eta0 at the same planes) are copied into shared
// memory while the current ones are transformed, so no thread waits on a global load. Per chunk:
// y inverse FFTs read the staged planes (thread per column, conflict-free) into the padded work
// tile, which frees the staging buffer for the next chunk's copy; x inverse FFTs in the work tile;
// the epilogue stores the orbital and accumulates the density from the staged eta0.

// planes per chunk: largest divisor of N with <= 128 threads and <= 112 KB of shared memory
// (two blocks per SM)
constexpr int tma_inv_ppb(int N) {
  int best = 0;
  for (int d = 1; d <= N; ++d)
    if (N % d == 0 && d * N <= 128 && (long long)d * N * N * 16 + (long long)d * N * (N + 1) * 8 <= 112 * 1024)
      best = d;
  return best;
}
template <int N> constexpr size_t tma_inv_smem() {
  return (size_t)tma_inv_ppb(N) * N * N * 16 + (size_t)tma_inv_ppb(N) * N * (N + 1) * 8;
}
// grids streamed this way (even N: every chunk offset is a multiple of 16 bytes)
constexpr bool tma_inv_size(int N) { return N == 32 || N == 40 || N == 48 || N == 64; }

template <int N>
__global__ void __launch_bounds__(tma_inv_ppb(N) * N)
    k_plane_inv_density_tma(GView<float> g, float2 *data, const float2 *a_next, float *dens, int L,
                            int n_pairs, int *err) {
  using C = float2;
  constexpr int PPB = tma_inv_ppb(N), NN = N * N, LD = N + 1, NT = PPB * N, G = N / PPB;
  constexpr unsigned kChunk = PPB * NN * sizeof(C);
  extern __shared__ __align__(128) unsigned char smem_raw[];
  C *Sd = reinterpret_cast<C *>(smem_raw);  // staged orbital planes (dense)
  C *Sa = Sd + PPB * NN;                     // staged eta0 planes (dense)
  C *W = Sa + PPB * NN;                      // work tile, rows padded to N + 1
  __shared__ __align__(8) uint64_t bar_d, bar_a;
  const long long units = (long long)n_pairs * G;
  long long u = blockIdx.x;
  if (u >= units) return;
  const int pl = threadIdx.x / N, q = threadIdx.x - pl * N;
  auto src_d = [&](long long uu, int e) {
    return data + ((uu / G) * L + e) * g.ng + (uu % G) * (long long)(PPB * NN);
  };
  auto src_a = [&](long long uu, int e) { return a_next + (long long)e * g.ng + (uu % G) * (long long)(PPB * NN); };
  if (threadIdx.x == 0) {
    tma_bar_init(&bar_d, 1);
    tma_bar_init(&bar_a, 1);
    tma_bar_expect(&bar_d, kChunk);
    tma_load_1d(Sd, src_d(u, 0), kChunk, &bar_d);
    tma_bar_expect(&bar_a, kChunk);
    tma_load_1d(Sa, src_a(u, 0), kChunk, &bar_a);
  }
  __syncthreads();
  unsigned ph_d = 0, ph_a = 0;
  bool pend_d = true, pend_a = true, ok = true;
  int ell = 0;
  float accd[N];
#pragma unroll
  for (int k = 0; k < N; ++k) accd[k] = 0.f;
  while (true) {
    long long un = u;
    int en = ell + 1;
    if (en == L) {
      en = 0;
      un += gridDim.x;
    }
    const bool has_next = un < units;
    // y inverse FFTs from the staged planes into the work tile
    if (!__syncthreads_and(tma_bar_wait(&bar_d, ph_d))) {
      ok = false;
      break;
    }
    ph_d ^= 1u;
    pend_d = false;
    {
      C v[N];
#pragma unroll
      for (int y = 0; y < N; ++y) v[y] = Sd[pl * NN + y * N + q];
      fft_reg<float, N, +1>(v);
#pragma unroll
      for (int y = 0; y < N; ++y) W[(pl * N + y) * LD + q] = v[y];
    }
    __syncthreads();
    if (threadIdx.x == 0 && has_next) {
      tma_fence_proxy();
      tma_bar_expect(&bar_d, kChunk);
      tma_load_1d(Sd, src_d(un, en), kChunk, &bar_d);
    }
    pend_d = has_next;
    {
      C v[N];
      C *row = W + (pl * N + q) * LD;
#pragma unroll
      for (int x = 0; x < N; ++x) v[x] = row[x];
      fft_reg<float, N, +1>(v);
#pragma unroll
      for (int x = 0; x < N; ++x) row[x] = v[x];
    }
    if (!__syncthreads_and(tma_bar_wait(&bar_a, ph_a))) {
      ok = false;
      break;
    }
    ph_a ^= 1u;
    pend_a = false;
    const long long pair = u / G, off = (u % G) * (long long)(PPB * NN);
    C *base = data + (pair * L + ell) * g.ng + off;
#pragma unroll
    for (int k = 0; k < N; ++k) {
      const int l = threadIdx.x + k * NT;
      const int p = l / NN, rem = l - p * NN, y = rem / N, x = rem - y * N;
      const C dv = W[(p * N + y) * LD + x];
      base[l] = dv;
      const C a0 = Sa[l];
      accd[k] += 2.f * (2.f * (a0.x * dv.x + a0.y * dv.y) + dv.x * dv.x + dv.y * dv.y);
    }
    __syncthreads();
    if (threadIdx.x == 0 && has_next) {
      tma_fence_proxy();
      tma_bar_expect(&bar_a, kChunk);
      tma_load_1d(Sa, src_a(un, en), kChunk, &bar_a);
    }
    pend_a = has_next;
    if (ell == L - 1) {
      float *db = dens + pair * g.ng + off;
#pragma unroll
      for (int k = 0; k < N; ++k) {
        db[threadIdx.x + k * NT] = accd[k];
        accd[k] = 0.f;
      }
    }
    if (!has_next) break;
    u = un;
    ell = en;
  }
  if (!ok) {
    if (threadIdx.x == 0) atomicExch(err, 1);
    // copies still in flight must land before the block's shared memory is released
    if (pend_d) tma_bar_wait(&bar_d, ph_d);
    if (pend_a) tma_bar_wait(&bar_a, ph_a);
  }
}

// z-column pass streamed by bulk copies: a persistent block walks (item, slab of Y rows) units;
// the slab's N z-rows (Y N contiguous points each) are copied into shared memory, every thread takes
// its column (conflict-free across x) into registers, the buffer is refilled with the next unit,
// and the forward z FFT, the multiplier and the inverse z FFT run while the copies are in flight.
constexpr int tma_z_rows(int N) {
  int best = 0;
  for (int y = 1; y <= N; ++y)
    if (N % y == 0 && y * N <= 256 && (long long)y * N * N * 8 <= 80 * 1024) best = y;
  return best;
}

template <int N>
__global__ void __launch_bounds__(tma_z_rows(N) * N)
    k_zcol_tma(GView<float> g, float2 *data, long long n_items, int mult, int *err) {
  using C = float2;
  constexpr int Y = tma_z_rows(N), NN = N * N, G = N / Y;
  constexpr unsigned kRow = Y * N * sizeof(C);
  extern __shared__ __align__(128) unsigned char smem_raw[];
  C *S = reinterpret_cast<C *>(smem_raw);  // [z][y][x] of the slab
  __shared__ __align__(8) uint64_t bar;
  const long long units = n_items * G;
  long long u = blockIdx.x;
  if (u >= units) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int yy = threadIdx.x / N, x = threadIdx.x - yy * N;
  auto issue = [&](long long uu) {  // warp 0: one arrival with the byte count, then N row copies
    const C *src = data + (uu / G) * g.ng + (uu % G) * (long long)(Y * N);
    if (lane == 0) tma_bar_expect(&bar, kRow * N);
    __syncwarp();
    for (int z = lane; z < N; z += 32) tma_load_1d(S + z * Y * N, src + (long long)z * NN, kRow, &bar);
  };
  if (threadIdx.x == 0) tma_bar_init(&bar, 1);
  __syncthreads();
  if (warp == 0) issue(u);
  unsigned ph = 0;
  bool pend = true, ok = true;
  const float inv_ng = 1.f / (float)(N * N * N);
  while (true) {
    const long long un = u + gridDim.x;
    const bool has_next = un < units;
    if (!__syncthreads_and(tma_bar_wait(&bar, ph))) {
      ok = false;
      break;
    }
    ph ^= 1u;
    pend = false;
    C v[N];
#pragma unroll
    for (int z = 0; z < N; ++z) v[z] = S[(z * Y + yy) * N + x];
    __syncthreads();
    if (warp == 0 && has_next) {
      tma_fence_proxy();
      issue(un);
    }
    pend = has_next;
    const int y = (int)(u % G) * Y + yy;
    fft_reg<float, N, -1>(v);
    if (mult == Z_KINETIC) {
      const C mxy = cscale(cmul(g.kin[x], g.kin[y]), inv_ng);
#pragma unroll
      for (int z = 0; z < N; ++z) v[z] = cmul(v[z], cmul(mxy, g.kin[z]));
    } else {
      const float gxy = g.k2[x] + g.k2[y];
#pragma unroll
      for (int z = 0; z < N; ++z) {
        const float G2 = gxy + g.k2[z];
        v[z] = cscale(v[z], G2 > 0.f ? float(4.0 * M_PI) * inv_ng / G2 : 0.f);
      }
    }
    fft_reg<float, N, +1>(v);
    C *base = data + (u / G) * g.ng + (long long)y * N + x;
#pragma unroll
    for (int z = 0; z < N; ++z) base[(long long)z * NN] = v[z];
    if (!has_next) break;
    u = un;
  }
  if (!ok) {
    if (threadIdx.x == 0) atomicExch(err, 1);
    if (pend) tma_bar_wait(&bar, ph);
  }
}

// resident blocks per SM times SMs of the current device for a kernel and launch shape (0 if the
// query fails)
template <typename K> static long long resident_slots(K kernel, int threads, size_t smem) {
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return (long long)per_sm * sms;
}

template <int N>
static bool zcol_tma(const GridTables<float> &g, float2 *d, int n_items, int mult, int *err, cudaStream_t s) {
  if constexpr (tma_inv_size(N)) {
    constexpr int Y = tma_z_rows(N);
    constexpr size_t sm = (size_t)Y * N * N * sizeof(float2);
    const long long units = (long long)n_items * (N / Y);
    // resident blocks of the whole GPU; function-local static: initialised once, thread-safe
    static const long long slots = resident_slots(k_zcol_tma<N>, Y * N, sm);
    if (slots < 1 || units < 1) return false;
    const long long grid = units < slots ? units : slots;
    k_zcol_tma<N><<<(unsigned)grid, Y * N, sm, s>>>(view(g), d, n_items, mult, err);
    return true;
  }
  return false;
}

template <int N>
static bool inv_density_tma(const GridTables<float> &g, float2 *d, int n_items, const float2 *a_next, int L,
                            float *dens, int *err, cudaStream_t s) {
  if constexpr (tma_inv_size(N)) {
    constexpr int PPB = tma_inv_ppb(N);
    const long long units = (long long)(n_items / L) * (N / PPB);
    static const long long slots = resident_slots(k_plane_inv_density_tma<N>, PPB * N, tma_inv_smem<N>());
    if (slots < 1 || units < 1) return false;
    const long long grid = units < slots ? units : slots;
    k_plane_inv_density_tma<N><<<(unsigned)grid, PPB * N, tma_inv_smem<N>(), s>>>(view(g), d, a_next, dens, L,
                                                                                  n_items / L, err);
    return true;
  }
  return false;
}

// ------------------------------------------------------------------------------------------
// Persistent split-operator step: one launch advances the eta0 set and every pair's L orbitals by
// one step of Eq. (10) and writes each pair's induced density. Blocks claim tiles from a host-built
// queue; a tile waits (bounded) for the tiles it reads, whose queue positions are always earlier,
// so every awaited tile is held by a running block and the launch cannot deadlock. The queue
// pipelines pairs (forward tiles of pair j, z tiles of pair j-1, inverse tiles of pair j-2) so that
// the orbitals in flight stay in L2 between the three passes.

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// bounded wait for *p >= target (`limit` polls ~100 ns apart; the default 2^23 is about a second);
// false on timeout
__device__ __forceinline__ bool wait_geq(const unsigned *p, unsigned target, unsigned limit) {
  for (unsigned i = 0; i < limit; ++i) {
    if (ld_acquire(p) >= target) return true;
    __nanosleep(100);
  }
  return false;
}

template <typename T, int N>
__global__ void __launch_bounds__(kPPB<T, N> * N)
    k_step_persistent(GView<T> g, XfwdArgs<T> fa, XfwdArgs<T> fp, C2<T> *a_next, C2<T> *d, T *dens,
                      int L, StepQueue q) {
  using C = C2<T>;
  constexpr int PPB = kPPB<T, N>, NN = N * N, G = N / PPB, NT = PPB * N;
  extern __shared__ unsigned char smem_raw[];
  C *S = reinterpret_cast<C *>(smem_raw);
  __shared__ int4 cur;
  __shared__ int go;
  const unsigned tgt = (q.epoch + 1) * (unsigned)G;
  for (;;) {
    if (threadIdx.x == 0) {
      const unsigned i = atomicAdd(q.claim, 1u) - q.claim_base;
      const int4 it = (i < (unsigned)q.n_items) ? q.items[i] : make_int4(-1, 0, 0, 0);
      bool ok = true;
      if (it.x == SI_A_Z) {
        ok = wait_geq(q.a_fwd + it.y, tgt, q.wait_limit);
      } else if (it.x == SI_A_INV) {
        ok = wait_geq(q.a_z + it.y, tgt, q.wait_limit);
      } else if (it.x == SI_P_Z) {
        ok = wait_geq(q.p_fwd + it.y, tgt, q.wait_limit);
      } else if (it.x == SI_P_INV) {
        ok = wait_geq(q.a_inv, (q.epoch + 1) * (unsigned)(L * G), q.wait_limit);
        for (int l = 0; l < L && ok; ++l) ok = wait_geq(q.p_z + it.y * L + l, tgt, q.wait_limit);
      }
      if (!ok) atomicExch(q.err, 1);
      __threadfence();
      cur = it;
      go = ok ? 1 : 0;
    }
    __syncthreads();
    const int4 it = cur;
    if (it.x < 0) break;
    if (go) {
      switch (it.x) {
        case SI_A_FWD: fwd_planes<T, N, false>(g, fa, it.y, (long long)it.z * PPB * NN, S); break;
        case SI_P_FWD: fwd_planes<T, N, true>(g, fp, it.y, (long long)it.z * PPB * NN, S); break;
        case SI_A_Z: zcol_column<T, N, true>(g, a_next, it.y, it.z * NT + threadIdx.x, Z_KINETIC); break;
        case SI_P_Z: zcol_column<T, N, true>(g, d, it.y, it.z * NT + threadIdx.x, Z_KINETIC); break;
        case SI_A_INV: inv_plain_planes<T, N, true>(g, a_next, it.y, (long long)it.z * PPB * NN, S); break;
        case SI_P_INV: inv_density_planes<T, N, true>(g, d, a_next, dens, it.y, L, it.z * PPB, S); break;
        default: break;
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      unsigned *c = nullptr;
      if (it.x == SI_A_FWD) c = q.a_fwd + it.y;
      else if (it.x == SI_A_Z) c = q.a_z + it.y;
      else if (it.x == SI_A_INV) c = q.a_inv;
      else if (it.x == SI_P_FWD) c = q.p_fwd + it.y;
      else if (it.x == SI_P_Z) c = q.p_z + it.y;
      if (c) atomicAdd(c, 1u);
    }
  }
}

// ------------------------------------------------------------------------------------------
// dispatch over the compile-time sizes

template <typename T, int N> static void set_attrs() {
  const int sm = (int)plane_smem<T, N>();
  cudaFuncSetAttribute(k_step_persistent<T, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  cudaFuncSetAttribute(k_plane_fwd<T, N, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)fwd_smem<T, N, true>());
  cudaFuncSetAttribute(k_plane_fwd<T, N, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  cudaFuncSetAttribute(k_plane_inv<T, N, PI_PLAIN>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  cudaFuncSetAttribute(k_plane_inv<T, N, PI_DENSITY>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  cudaFuncSetAttribute(k_plane_inv<T, N, PI_POISSON>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  if constexpr (sizeof(T) == 4 && tma_inv_size(N)) {
    cudaFuncSetAttribute(k_plane_inv_density_tma<N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)tma_inv_smem<N>());
    cudaFuncSetAttribute(k_zcol_tma<N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)(tma_z_rows(N) * N * N * sizeof(float2)));
  }
}

template <typename T> struct FastOps {
  template <int N>
  static void step(const GridTables<T> &g, const XfwdArgs<T> &fa, const XfwdArgs<T> &fp, C2<T> *a_next,
                   C2<T> *d, T *dens, int L, const StepQueue &q, int grid, cudaStream_t s) {
    if constexpr (!(sizeof(T) == 8 && N > 48)) {
      k_step_persistent<T, N><<<grid, kPPB<T, N> * N, plane_smem<T, N>(), s>>>(view(g), fa, fp, a_next, d,
                                                                              dens, L, q);
    }
  }
  template <int N> static int resident_blocks() {
    if constexpr (!(sizeof(T) == 8 && N > 48)) {
      int per_sm = 0, dev = 0, sms = 0;
      cudaGetDevice(&dev);
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_step_persistent<T, N>, kPPB<T, N> * N,
                                                    plane_smem<T, N>());
      return per_sm * sms;
    }
    return 0;
  }
  template <int N> static int tiles_per_orbital() { return N / kPPB<T, N>; }
  template <int N> static void fwd(const GridTables<T> &g, const XfwdArgs<T> &a, cudaStream_t s) {
    if constexpr (!(sizeof(T) == 8 && N > 48)) {
      const long long planes = (long long)a.n_items * N;
      if (a.mode == XF_PHASE_PAIR) {
        constexpr int P2 = fwd_ppb<T, N, true>();
        k_plane_fwd<T, N, true><<<(unsigned)(planes / P2), P2 * N, fwd_smem<T, N, true>(), s>>>(view(g), a,
                                                                                              planes);
      } else {
        k_plane_fwd<T, N, false><<<(unsigned)(planes / kPPB<T, N>), kPPB<T, N> * N, plane_smem<T, N>(), s>>>(
            view(g), a, planes);
      }
    }
  }
  template <int N> static void z(const GridTables<T> &g, C2<T> *d, int n_items, int mult, cudaStream_t s) {
    if constexpr (!(sizeof(T) == 8 && N > 48)) {
      const long long cols = (long long)n_items * N * N;
      k_zcol<T, N><<<(unsigned)((cols + 127) / 128), 128, 0, s>>>(view(g), d, cols, mult);
    }
  }
  template <int N>
  static void inv(const GridTables<T> &g, C2<T> *d, int n_items, const C2<T> *a_next, int L, T *dens,
                  T *u_out, T *acc, C2<T> *em1_out, const PoissonOut &po, int mode, cudaStream_t s) {
    if constexpr (!(sizeof(T) == 8 && N > 48)) {
      PlaneInvArgs pa{(long long)n_items * N, L, po};
      const size_t sm = plane_smem<T, N>();
      constexpr int NT = kPPB<T, N> * N;
      if (mode == PI_DENSITY) {
        dim3 grid(N / kPPB<T, N>, n_items / L);
        k_plane_inv<T, N, PI_DENSITY><<<grid, NT, sm, s>>>(view(g), d, a_next, dens, nullptr, nullptr,
                                                            nullptr, pa);
      } else if (mode == PI_PLAIN) {
        k_plane_inv<T, N, PI_PLAIN><<<(unsigned)(pa.planes_total / kPPB<T, N>), NT, sm, s>>>(
            view(g), d, nullptr, nullptr, nullptr, nullptr, nullptr, pa);
      } else {
        k_plane_inv<T, N, PI_POISSON><<<(unsigned)(pa.planes_total / kPPB<T, N>), NT, sm, s>>>(
            view(g), d, nullptr, nullptr, u_out, acc, em1_out, pa);
      }
  }
  }
};

#define SBSE_FAST_SWITCH(N, CALL)      \
  switch (N) {                         \
    case 8: CALL(8); break;            \
    case 10: CALL(10); break;          \
    case 12: CALL(12); break;          \
    case 16: CALL(16); break;          \
    case 20: CALL(20); break;          \
    case 24: CALL(24); break;          \
    case 32: CALL(32); break;          \
    case 40: CALL(40); break;          \
    case 48: CALL(48); break;          \
    case 64: CALL(64); break;          \
    default: break;                    \
  }

template <typename T>
void launch_step_persistent(const GridTables<T> &g, const XfwdArgs<T> &fa, const XfwdArgs<T> &fp,
                            C2<T> *a_next, C2<T> *d, T *dens, int L, const StepQueue &q, int grid,
                            cudaStream_t s) {
#define SBSE_CALL(n) FastOps<T>::template step<n>(g, fa, fp, a_next, d, dens, L, q, grid, s)
  SBSE_FAST_SWITCH(g.N, SBSE_CALL)
#undef SBSE_CALL
  count_launch(1);
}

template <typename T> int step_resident_blocks(int N) {
  int r = 0;
#define SBSE_CALL(n) r = FastOps<T>::template resident_blocks<n>()
  SBSE_FAST_SWITCH(N, SBSE_CALL)
#undef SBSE_CALL
  return r;
}

template <typename T> int step_tiles_per_orbital(int N) {
  int r = 0;
#define SBSE_CALL(n) r = FastOps<T>::template tiles_per_orbital<n>()
  SBSE_FAST_SWITCH(N, SBSE_CALL)
#undef SBSE_CALL
  return r;
}

template <typename T> bool fast_supported(int N) {
  // FP64 pencils of 64 would not fit in the register file; 80 and 96 take the FP32 lane-pair
  // passes of fft_split.cu
  if (split_size(N)) return sizeof(T) == 4;
  for (int i = 0; i < kRegCount; ++i)
    if (kRegSizes[i] == N) return !(sizeof(T) == 8 && N > 48);
  return false;
}

template <typename T> void init_fast_kernels() {
#define SBSE_ATTR(n) set_attrs<T, n>()
  SBSE_ATTR(8); SBSE_ATTR(10); SBSE_ATTR(12); SBSE_ATTR(16); SBSE_ATTR(20);
  SBSE_ATTR(24); SBSE_ATTR(32); SBSE_ATTR(40); SBSE_ATTR(48);
  if constexpr (sizeof(T) == 4) set_attrs<T, 64>();
#undef SBSE_ATTR
}

template <typename T> void launch_plane_fwd(const GridTables<T> &g, const XfwdArgs<T> &a, cudaStream_t s) {
  if constexpr (sizeof(T) == 4) {
    if (split_size(g.N)) {
      launch_plane_fwd2(g, a, s);
      count_launch(1);
      return;
    }
  }
#define SBSE_CALL(n) FastOps<T>::template fwd<n>(g, a, s)
  SBSE_FAST_SWITCH(g.N, SBSE_CALL)
#undef SBSE_CALL
  count_launch(1);
}

template <typename T>
void launch_zcol(const GridTables<T> &g, C2<T> *d, int n_items, int mult, cudaStream_t s, int *tma_err) {
  if constexpr (sizeof(T) == 4) {
    if (split_size(g.N)) {
      launch_zcol2(g, d, n_items, mult, s);
      count_launch(1);
      return;
    }
    if (tma_err) {
      bool done = false;
#define SBSE_CALL(n) done = zcol_tma<n>(g, d, n_items, mult, tma_err, s)
      SBSE_FAST_SWITCH(g.N, SBSE_CALL)
#undef SBSE_CALL
      if (done) {
        count_launch(1);
        return;
      }
    }
  }
#define SBSE_CALL(n) FastOps<T>::template z<n>(g, d, n_items, mult, s)
  SBSE_FAST_SWITCH(g.N, SBSE_CALL)
#undef SBSE_CALL
  count_launch(1);
}

template <typename T>
void launch_plane_inv_orb(const GridTables<T> &g, C2<T> *d, int n_items, const C2<T> *a_next, int L,
                          T *dens, cudaStream_t s, int *tma_err) {
  if constexpr (sizeof(T) == 4) {
    if (dens && tma_err) {
      bool done = false;
#define SBSE_CALL(n) done = inv_density_tma<n>(g, d, n_items, a_next, L, dens, tma_err, s)
      SBSE_FAST_SWITCH(g.N, SBSE_CALL)
#undef SBSE_CALL
      if (done) {
        count_launch(1);
        return;
      }
    }
  }
  const int mode = dens ? PI_DENSITY : PI_PLAIN;
  const PoissonOut po{0, 0.0, 0.0, 0.0};
#define SBSE_CALL(n) FastOps<T>::template inv<n>(g, d, n_items, a_next, L, dens, nullptr, nullptr, nullptr, po, mode, s)
  SBSE_FAST_SWITCH(g.N, SBSE_CALL)
#undef SBSE_CALL
  count_launch(1);
}

template <typename T>
void launch_plane_inv_poisson(const GridTables<T> &g, C2<T> *d, int n_slots, const PoissonOut &po,
                              T *u_out, T *acc, C2<T> *em1_out, cudaStream_t s) {
  if constexpr (sizeof(T) == 4) {
    if (split_size(g.N)) {
      launch_plane_inv2_poisson(g, d, n_slots, po, u_out, acc, em1_out, s);
      count_launch(1);
      return;
    }
  }
#define SBSE_CALL(n) FastOps<T>::template inv<n>(g, d, n_slots, nullptr, 1, nullptr, u_out, acc, em1_out, po, PI_POISSON, s)
  SBSE_FAST_SWITCH(g.N, SBSE_CALL)
#undef SBSE_CALL
  count_launch(1);
}

#define SBSE_FAST_INST(T)                                                                           \
  template void launch_step_persistent<T>(const GridTables<T> &, const XfwdArgs<T> &,              \
                                          const XfwdArgs<T> &, C2<T> *, C2<T> *, T *, int,         \
                                          const StepQueue &, int, cudaStream_t);                   \
  template int step_resident_blocks<T>(int);                                                       \
  template int step_tiles_per_orbital<T>(int);                                                     \
  template bool fast_supported<T>(int);                                                            \
  template void init_fast_kernels<T>();                                                            \
  template void launch_plane_fwd<T>(const GridTables<T> &, const XfwdArgs<T> &, cudaStream_t);     \
  template void launch_zcol<T>(const GridTables<T> &, C2<T> *, int, int, cudaStream_t, int *);     \
  template void launch_plane_inv_orb<T>(const GridTables<T> &, C2<T> *, int, const C2<T> *, int,   \
                                        T *, cudaStream_t, int *);                                 \
  template void launch_plane_inv_poisson<T>(const GridTables<T> &, C2<T> *, int, const PoissonOut &, \
                                            T *, T *, C2<T> *, cudaStream_t);

SBSE_FAST_INST(float)
SBSE_FAST_INST(double)

}  // namespace sbse
