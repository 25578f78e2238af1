// Device kernels of the stochastic-TDH action of W (Sec. II.B, Eqs. 10-15).
//
// A 3D FFT of an item (one complex field of N^3 points, x fastest) is three batched pencil
// passes over shared-memory tiles of 32 pencils: x (rows), y and z (columns of 32 consecutive
// x values, coalesced). Element-wise work is fused into the passes that touch the data anyway:
//   x forward  <- potential phase of the split-operator step (Eq. 10) or Poisson packing
//   z          <- forward FFT, kinetic phase (or 4 pi / G^2) and 1/N^3, inverse FFT in one pass
//   x inverse  -> induced density (Eq. 11) of all L orbitals of a pair, or the Poisson unpacking
//                 with the damped time-integral accumulation of Eq. (13)
#include <math.h>

#include "gemm_nt.cuh"
#include <algorithm>

#include "kernels.h"
#include "passes.cuh"

namespace sbse {

constexpr int kTP = 32;        // pencils per tile
constexpr int kThreads = 256;  // threads per FFT block
constexpr int kMaxPerThread = (kTP * kMaxN + kThreads - 1) / kThreads;

template <typename T> static size_t fft_smem(int N, int tp) {
  return (size_t)(N + 2 * N * (tp + 1)) * sizeof(C2<T>);
}

template <typename T> __device__ __forceinline__ void load_twiddles(C2<T> *tw_s, const C2<T> *tw, int N) {
  for (int i = threadIdx.x; i < N; i += blockDim.x) tw_s[i] = tw[i];
}

// ------------------------------------------------------------------------------------------
// x forward pass with fused pre-operation

template <typename T>
__global__ void __launch_bounds__(kThreads) k_xfwd(GView<T> g, XfwdArgs<T> a, long long rows_total) {
  using C = C2<T>;
  extern __shared__ unsigned char smem_raw[];
  const int N = g.N, ld = kTP + 1;
  C *tw = reinterpret_cast<C *>(smem_raw);
  C *A = tw + N;
  C *B = A + N * ld;
  load_twiddles<T>(tw, g.tw, N);
  const long long N2 = (long long)N * N;
  const long long row0 = (long long)blockIdx.x * kTP;
  for (int l = threadIdx.x; l < kTP * N; l += blockDim.x) {
    const int p = l / N, e = l - p * N;
    const long long row = row0 + p;
    C v = C{T(0), T(0)};
    if (row < rows_total) {
      const long long item = row / N2;
      const long long idx = (row - item * N2) * N + e;
      const long long gi = row * N + e;
      v = preop_value<T>(g, a, item, idx, gi);
    }
    A[e * ld + p] = v;
  }
  __syncthreads();
  C *R = fft_tile<T>(A, B, tw, g.plan, kTP, ld, -1);
  for (int l = threadIdx.x; l < kTP * N; l += blockDim.x) {
    const int p = l / N, e = l - p * N;
    const long long row = row0 + p;
    if (row < rows_total) a.out[row * N + e] = R[e * ld + p];
  }
}

template <typename T> void launch_xfwd(const GridTables<T> &g, const XfwdArgs<T> &a, cudaStream_t s) {
  const long long rows = (long long)a.n_items * g.N * g.N;
  const long long blocks = (rows + kTP - 1) / kTP;
  k_xfwd<T><<<(unsigned)blocks, kThreads, fft_smem<T>(g.N, kTP), s>>>(view(g), a, rows);
  count_launch(1);
}

// ------------------------------------------------------------------------------------------
// y pass (forward or inverse), in place

template <typename T>
__global__ void __launch_bounds__(kThreads) k_ypass(GView<T> g, C2<T> *data, int sign) {
  using C = C2<T>;
  extern __shared__ unsigned char smem_raw[];
  const int N = g.N, tp = N < kTP ? N : kTP, ld = tp + 1;
  C *tw = reinterpret_cast<C *>(smem_raw);
  C *A = tw + N;
  C *B = A + N * ld;
  load_twiddles<T>(tw, g.tw, N);
  const int x0 = blockIdx.x * tp;
  const int xt = (N - x0) < tp ? (N - x0) : tp;
  C *base = data + (long long)blockIdx.z * g.ng + (long long)blockIdx.y * N * N + x0;
  for (int l = threadIdx.x; l < tp * N; l += blockDim.x) {
    const int e = l / tp, p = l - e * tp;
    A[e * ld + p] = (p < xt) ? base[(long long)e * N + p] : C{T(0), T(0)};
  }
  __syncthreads();
  C *R = fft_tile<T>(A, B, tw, g.plan, tp, ld, sign);
  for (int l = threadIdx.x; l < tp * N; l += blockDim.x) {
    const int e = l / tp, p = l - e * tp;
    if (p < xt) base[(long long)e * N + p] = R[e * ld + p];
  }
}

template <typename T>
void launch_ypass(const GridTables<T> &g, C2<T> *data, int n_items, int sign, cudaStream_t s) {
  const int tp = g.N < kTP ? g.N : kTP;
  dim3 grid((g.N + tp - 1) / tp, g.N, n_items);
  k_ypass<T><<<grid, kThreads, fft_smem<T>(g.N, tp), s>>>(view(g), data, sign);
  count_launch(1);
}

// ------------------------------------------------------------------------------------------
// z pass: forward FFT, multiply by the kinetic propagator (or the Coulomb kernel) and 1/N^3,
// inverse FFT. The x and y passes before it have already transformed the other two axes.

template <typename T>
__global__ void __launch_bounds__(kThreads) k_zpass(GView<T> g, C2<T> *data, int mult) {
  using C = C2<T>;
  extern __shared__ unsigned char smem_raw[];
  const int N = g.N, tp = N < kTP ? N : kTP, ld = tp + 1;
  C *tw = reinterpret_cast<C *>(smem_raw);
  C *A = tw + N;
  C *B = A + N * ld;
  load_twiddles<T>(tw, g.tw, N);
  const int x0 = blockIdx.x * tp;
  const int xt = (N - x0) < tp ? (N - x0) : tp;
  const int y = blockIdx.y;
  const long long N2 = (long long)N * N;
  C *base = data + (long long)blockIdx.z * g.ng + (long long)y * N + x0;
  for (int l = threadIdx.x; l < tp * N; l += blockDim.x) {
    const int e = l / tp, p = l - e * tp;
    A[e * ld + p] = (p < xt) ? base[(long long)e * N2 + p] : C{T(0), T(0)};
  }
  __syncthreads();
  C *R = fft_tile<T>(A, B, tw, g.plan, tp, ld, -1);
  C *S = (R == A) ? B : A;
  const T inv_ng = T(1) / T(g.ng);
  for (int l = threadIdx.x; l < tp * N; l += blockDim.x) {
    const int e = l / tp, p = l - e * tp;
    const int kx = x0 + (p < xt ? p : 0);
    C v = R[e * ld + p];
    if (mult == Z_KINETIC) {
      C m = cmul(cmul(g.kin[kx], g.kin[y]), g.kin[e]);
      v = cscale(cmul(v, m), inv_ng);
    } else {
      const T G2 = g.k2[kx] + g.k2[y] + g.k2[e];
      const T f = mult == Z_HALF_G2 ? T(0.5) * G2 * inv_ng : (G2 > T(0) ? T(4.0 * M_PI) / G2 * inv_ng : T(0));
      v = cscale(v, f);
    }
    R[e * ld + p] = v;
  }
  __syncthreads();
  C *R2 = fft_tile<T>(R, S, tw, g.plan, tp, ld, +1);
  for (int l = threadIdx.x; l < tp * N; l += blockDim.x) {
    const int e = l / tp, p = l - e * tp;
    if (p < xt) base[(long long)e * N2 + p] = R2[e * ld + p];
  }
}

template <typename T>
void launch_zpass(const GridTables<T> &g, C2<T> *data, int n_items, int mult, cudaStream_t s) {
  const int tp = g.N < kTP ? g.N : kTP;
  dim3 grid((g.N + tp - 1) / tp, g.N, n_items);
  k_zpass<T><<<grid, kThreads, fft_smem<T>(g.N, tp), s>>>(view(g), data, mult);
  count_launch(1);
}

// ------------------------------------------------------------------------------------------
// x inverse pass of orbitals, optionally with the induced density of each pair:
// delta n = 2 sum_l (2 Re(conj(eta0_l) d_l) + |d_l|^2)  (n = 2 sum |eta|^2, Eq. 11)

template <typename T>
__global__ void __launch_bounds__(kThreads)
    k_xinv_orb(GView<T> g, C2<T> *data, long long rows_total, const C2<T> *a_next, int L, T *dens) {
  using C = C2<T>;
  extern __shared__ unsigned char smem_raw[];
  const int N = g.N, ld = kTP + 1;
  C *tw = reinterpret_cast<C *>(smem_raw);
  C *A = tw + N;
  C *B = A + N * ld;
  load_twiddles<T>(tw, g.tw, N);
  const long long N2 = (long long)N * N;
  if (dens == nullptr) {
    const long long row0 = (long long)blockIdx.x * kTP;
    for (int l = threadIdx.x; l < kTP * N; l += blockDim.x) {
      const int p = l / N, e = l - p * N;
      const long long row = row0 + p;
      A[e * ld + p] = row < rows_total ? data[row * N + e] : C{T(0), T(0)};
    }
    __syncthreads();
    C *R = fft_tile<T>(A, B, tw, g.plan, kTP, ld, +1);
    for (int l = threadIdx.x; l < kTP * N; l += blockDim.x) {
      const int p = l / N, e = l - p * N;
      const long long row = row0 + p;
      if (row < rows_total) data[row * N + e] = R[e * ld + p];
    }
    return;
  }
  // density mode: blockIdx.y = pair, blockIdx.x = tile of rows inside one orbital
  const int pair = blockIdx.y;
  const long long rr0 = (long long)blockIdx.x * kTP;
  T acc[kMaxPerThread];
#pragma unroll
  for (int k = 0; k < kMaxPerThread; ++k) acc[k] = T(0);
  for (int ell = 0; ell < L; ++ell) {
    C *item = data + ((long long)pair * L + ell) * g.ng;
    const C *av = a_next + (long long)ell * g.ng;
    for (int l = threadIdx.x; l < kTP * N; l += blockDim.x) {
      const int p = l / N, e = l - p * N;
      const long long rr = rr0 + p;
      A[e * ld + p] = rr < N2 ? item[rr * N + e] : C{T(0), T(0)};
    }
    __syncthreads();
    C *R = fft_tile<T>(A, B, tw, g.plan, kTP, ld, +1);
    int k = 0;
    for (int l = threadIdx.x; l < kTP * N; l += blockDim.x, ++k) {
      const int p = l / N, e = l - p * N;
      const long long rr = rr0 + p;
      if (rr < N2) {
        const C d = R[e * ld + p];
        item[rr * N + e] = d;
        const C a0 = av[rr * N + e];
        acc[k] += T(2) * (T(2) * (a0.x * d.x + a0.y * d.y) + d.x * d.x + d.y * d.y);
      }
    }
    __syncthreads();
  }
  int k = 0;
  for (int l = threadIdx.x; l < kTP * N; l += blockDim.x, ++k) {
    const int p = l / N, e = l - p * N;
    const long long rr = rr0 + p;
    if (rr < N2) dens[(long long)pair * g.ng + rr * N + e] = acc[k];
  }
}

template <typename T>
void launch_xinv_orb(const GridTables<T> &g, C2<T> *data, int n_items, const C2<T> *a_next, int L,
                     T *dens, cudaStream_t s) {
  const size_t sm = fft_smem<T>(g.N, kTP);
  if (dens == nullptr) {
    const long long rows = (long long)n_items * g.N * g.N;
    k_xinv_orb<T><<<(unsigned)((rows + kTP - 1) / kTP), kThreads, sm, s>>>(view(g), data, rows,
                                                                            nullptr, 1, nullptr);
  } else {
    const long long tiles = ((long long)g.N * g.N + kTP - 1) / kTP;
    dim3 grid((unsigned)tiles, n_items / L);
    k_xinv_orb<T><<<grid, kThreads, sm, s>>>(view(g), data, 0, a_next, L, dens);
  }
  count_launch(1);
}

// ------------------------------------------------------------------------------------------
// x inverse pass of packed Poisson slots, unpacking two real potentials per slot and
// accumulating the damped time integral of Eq. (13) in FP64.

template <typename T>
__global__ void __launch_bounds__(kThreads)
    k_xinv_poisson(GView<T> g, const C2<T> *data, long long rows_total, PoissonOut po, T *u_out,
                   T *acc, C2<T> *em1_out) {
  using C = C2<T>;
  extern __shared__ unsigned char smem_raw[];
  const int N = g.N, ld = kTP + 1;
  C *tw = reinterpret_cast<C *>(smem_raw);
  C *A = tw + N;
  C *B = A + N * ld;
  load_twiddles<T>(tw, g.tw, N);
  const long long N2 = (long long)N * N;
  const long long row0 = (long long)blockIdx.x * kTP;
  for (int l = threadIdx.x; l < kTP * N; l += blockDim.x) {
    const int p = l / N, e = l - p * N;
    const long long row = row0 + p;
    A[e * ld + p] = row < rows_total ? data[row * N + e] : C{T(0), T(0)};
  }
  __syncthreads();
  C *R = fft_tile<T>(A, B, tw, g.plan, kTP, ld, +1);
  for (int l = threadIdx.x; l < kTP * N; l += blockDim.x) {
    const int p = l / N, e = l - p * N;
    const long long row = row0 + p;
    if (row >= rows_total) continue;
    const long long slot = row / N2;
    const long long idx = (row - slot * N2) * N + e;
    const C v = R[e * ld + p];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const long long k = 2 * slot + h;
      if (k >= po.n_out) break;
      const T val = h ? v.y : v.x;
      if (u_out) u_out[k * g.ng + idx] = val;
      if (acc) {
        T *w = acc + k * g.ng + idx;
        *w = (po.keep != 0.0) ? (*w) + (T)po.coef * val : (T)po.coef * val;
      }
      if (em1_out) em1_out[k * g.ng + idx] = phase_em1<T>(val, (T)po.tau_next);
    }
  }
}

template <typename T>
void launch_xinv_poisson(const GridTables<T> &g, C2<T> *data, int n_slots, const PoissonOut &po,
                         T *u_out, T *acc, C2<T> *em1_out, cudaStream_t s) {
  const long long rows = (long long)n_slots * g.N * g.N;
  k_xinv_poisson<T><<<(unsigned)((rows + kTP - 1) / kTP), kThreads, fft_smem<T>(g.N, kTP), s>>>(
      view(g), data, rows, po, u_out, acc, em1_out);
  count_launch(1);
}

// ------------------------------------------------------------------------------------------
// initial stochastic orbitals eta_l = L^-1/2 sum_s c[l][s] phi_s (Eq. 14), FP64 sums, and the
// per-block partial sums of |eta_l|^2 for N0_l.

template <typename T>
__global__ void k_init_a(long long ng, const double *phi, int n_occ, const double *coeff, int L,
                         C2<T> *a, double *part) {
  __shared__ double red[256];
  const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const double inv = 1.0 / sqrt((double)L);
  for (int ell = 0; ell < L; ++ell) {
    double s = 0.0;
    if (r < ng)
      for (int q = 0; q < n_occ; ++q) s += coeff[(long long)ell * n_occ + q] * phi[(long long)q * ng + r];
    s *= inv;
    if (r < ng) a[(long long)ell * ng + r] = C2<T>{(T)s, T(0)};
    red[threadIdx.x] = (r < ng) ? s * s : 0.0;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
      if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
      __syncthreads();
    }
    if (threadIdx.x == 0) part[(long long)blockIdx.x * L + ell] = red[0];
    __syncthreads();
  }
}

template <typename T>
void launch_init_a(const GridTables<T> &g, const double *phi, int n_occ, const double *coeff, int L,
                   C2<T> *a, double *part, int *n_part, cudaStream_t s) {
  const int blocks = (int)((g.ng + 255) / 256);
  k_init_a<T><<<blocks, 256, 0, s>>>(g.ng, phi, n_occ, coeff, L, a, part);
  *n_part = blocks;
  count_launch(1);
}

// out[c] = scale * sum_{row < rows} part[row][c]  (fixed order: deterministic). A block owns 8
// adjacent columns; its 32 row groups read rows g, g + 32, ... (8 consecutive doubles per row and
// group: 64-byte segments) and are combined by a fixed tree in shared memory.
constexpr int kRcCols = 8, kRcGroups = 32;
__global__ void __launch_bounds__(kRcCols * kRcGroups)
    k_reduce_cols(const double *part, int rows, int cols, double scale, double *out) {
  __shared__ double red[kRcGroups][kRcCols];
  const int cx = threadIdx.x % kRcCols, g = threadIdx.x / kRcCols;
  const int c = blockIdx.x * kRcCols + cx;
  double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
  if (c < cols) {
    int r = g;
    for (; r + 3 * kRcGroups < rows; r += 4 * kRcGroups) {
      s0 += part[(long long)r * cols + c];
      s1 += part[(long long)(r + kRcGroups) * cols + c];
      s2 += part[(long long)(r + 2 * kRcGroups) * cols + c];
      s3 += part[(long long)(r + 3 * kRcGroups) * cols + c];
    }
    for (; r < rows; r += kRcGroups) s0 += part[(long long)r * cols + c];
  }
  red[g][cx] = (s0 + s1) + (s2 + s3);
  __syncthreads();
  for (int w = kRcGroups / 2; w > 0; w >>= 1) {
    if (g < w) red[g][cx] += red[g + w][cx];
    __syncthreads();
  }
  if (g == 0 && c < cols) out[c] = scale * red[0][cx];
}

void launch_reduce_cols(const double *part, int rows, int cols, double scale, double *out,
                        cudaStream_t s) {
  if (cols > 0) k_reduce_cols<<<(cols + kRcCols - 1) / kRcCols, kRcCols * kRcGroups, 0, s>>>(part, rows, cols, scale, out);
  count_launch(1);
}

// ------------------------------------------------------------------------------------------
// kick (Sec. II.B): d_l = (exp(-i alpha q) - 1) eta0_l = -2i sin(alpha q/2) exp(-i alpha q/2) eta0_l

template <typename T>
__global__ void k_kick(long long ng, const double *q, int P, const C2<T> *a, int L, double alpha,
                       C2<T> *d) {
  const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int pair = blockIdx.y;
  if (r >= ng) return;
  double s, c;
  sincos(0.5 * alpha * q[(long long)pair * ng + r], &s, &c);
  const C2<T> f = C2<T>{(T)(-2.0 * s * s), (T)(-2.0 * s * c)};
  for (int ell = 0; ell < L; ++ell)
    d[((long long)pair * L + ell) * ng + r] = cmul(f, a[(long long)ell * ng + r]);
}

template <typename T>
void launch_kick(const GridTables<T> &g, const double *q, int P, const C2<T> *a, int L, double alpha,
                 C2<T> *d, cudaStream_t s) {
  dim3 grid((unsigned)((g.ng + 255) / 256), P);
  k_kick<T><<<grid, 256, 0, s>>>(g.ng, q, P, a, L, alpha, d);
  count_launch(1);
}

// ------------------------------------------------------------------------------------------
// pending half potential step on (eta0, d) before cleaning (same rule as the x-forward pass)

// the pending half step of the potential before a cleaning, on the difference form:
// d <- P [(E - 1) a + E d], a <- P a, with the tables P = exp(-i V_loc dt/2) and E - 1 of each pair
// at tau = dt/2 (written by the preceding Poisson epilogue; null without feedback)
template <typename T>
__global__ void k_half_phase(long long ng, C2<T> *a, C2<T> *d, const C2<T> *pv, const C2<T> *em1, int P,
                             int L) {
  using C = C2<T>;
  const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int ell = blockIdx.y;
  if (r >= ng) return;
  const C av = a[(long long)ell * ng + r];
  const C p = pv[r];
  for (int pair = 0; pair < P; ++pair) {
    const C em = em1 ? em1[(long long)pair * ng + r] : C{T(0), T(0)};
    C *dp = d + ((long long)pair * L + ell) * ng + r;
    *dp = pair_phase<T>(p, em, av, *dp);
  }
  a[(long long)ell * ng + r] = cmul(p, av);
}

template <typename T>
void launch_half_phase(const GridTables<T> &g, C2<T> *a, C2<T> *d, const C2<T> *em1, int P, int L,
                       cudaStream_t s) {
  dim3 grid((unsigned)((g.ng + 255) / 256), L);
  k_half_phase<T><<<grid, 256, 0, s>>>(g.ng, a, d, g.pv_half, em1, P, L);
  count_launch(1);
}

// ------------------------------------------------------------------------------------------
// cleaning, Eq. (15): d_c <- d_c - sum_{s < N_occ} phi_s <phi_s|d_c>, then renormalisation of
// eta^alpha = eta0 + d to its initial norm N0: d <- c d + (c - 1) eta0, c = (1 + x)^-1/2,
// x = (2 Re<eta0|d> + |d|^2) / N0, c - 1 = -x / (sqrt(1+x) (1 + sqrt(1+x))).

// c - 1 per column from the reduced sums (FP64, one thread per column)
__global__ void k_cm1(int n_cols, int L, const double *sums /* [c][2], times dV */, const double *n0,
                      double *cm1) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n_cols) return;
  const double x = (sums[2 * c] + sums[2 * c + 1]) / n0[c % L];
  const double sq = sqrt(1.0 + x);
  cm1[c] = -x / (sq * (1.0 + sq));
}


// induced densities (Eq. 11) of the cleaned and rescaled orbitals, the rescaling d <- c d + (c-1) eta0
// being applied in registers only (the next forward pre-operation applies it to d itself): block =
// 256 points of one pair; c - 1 of the pair's L orbitals is converted to T once per block (a
// per-point FP64 -> FP32 conversion would load the narrow FP64 pipe)
template <typename T>
__global__ void k_density_renormed(long long ng, const C2<T> *d, const C2<T> *a, int L, const double *cm1v,
                                   T *dens) {
  extern __shared__ unsigned char sm_raw[];
  T *cm1s = reinterpret_cast<T *>(sm_raw);
  const int pair = blockIdx.y;
  for (int l = threadIdx.x; l < L; l += blockDim.x) cm1s[l] = (T)cm1v[(long long)pair * L + l];
  __syncthreads();
  const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= ng) return;
  T acc = T(0);
  for (int ell = 0; ell < L; ++ell) {
    const C2<T> a0 = a[(long long)ell * ng + r];
    const C2<T> dv = renorm_value<T>(d[((long long)pair * L + ell) * ng + r], a0, cm1s[ell]);
    acc += T(2) * (T(2) * (a0.x * dv.x + a0.y * dv.y) + dv.x * dv.x + dv.y * dv.y);
  }
  dens[(long long)pair * ng + r] = acc;
}

// Overlaps of the complex columns d_c with the occupied orbitals, split over chunks of grid
// points: part[chunk][c][s] = sum_{r in chunk} (Re d_c(r), Im d_c(r)) phi_s(r). Tile of 64
// columns x 64 states, 16 points per stage, 4 x 4 complex outputs per thread.
constexpr int kOvC = 64, kOvS = 64, kOvK = 16;

template <typename T>
__global__ void __launch_bounds__(256)
    k_clean_overlap(const C2<T> *d, const T *phi, int n_cols, int n_occ, long long ng,
                    long long kchunk, double *part) {
  __shared__ __align__(16) T Dre[kOvK][kOvC + 4];
  __shared__ __align__(16) T Dim[kOvK][kOvC + 4];
  __shared__ __align__(16) T Ph[kOvK][kOvS + 4];
  const int c0 = blockIdx.y * kOvC, s0 = blockIdx.z * kOvS;
  const long long kbeg = (long long)blockIdx.x * kchunk;
  const long long kend = (kbeg + kchunk < ng) ? kbeg + kchunk : ng;
  const int tc = threadIdx.x % 16, ts = threadIdx.x / 16;
  T are[4][4], aim[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) are[i][j] = aim[i][j] = T(0);
  for (long long k0 = kbeg; k0 < kend; k0 += kOvK) {
#pragma unroll
    for (int it = 0; it < 4; ++it) {
      const int l = threadIdx.x + it * 256;
      const int cc = l / kOvK, kk = l % kOvK;
      const long long k = k0 + kk;
      const int c = c0 + cc, s = s0 + cc;
      C2<T> v = C2<T>{T(0), T(0)};
      if (c < n_cols && k < kend) v = d[(long long)c * ng + k];
      Dre[kk][cc] = v.x;
      Dim[kk][cc] = v.y;
      Ph[kk][cc] = (s < n_occ && k < kend) ? phi[(long long)s * ng + k] : T(0);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kOvK; ++kk) {
      T xr[4], xi[4], p[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        xr[i] = Dre[kk][tc * 4 + i];
        xi[i] = Dim[kk][tc * 4 + i];
        p[i] = Ph[kk][ts * 4 + i];
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          are[i][j] += xr[i] * p[j];
          aim[i][j] += xi[i] * p[j];
        }
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int c = c0 + tc * 4 + i;
    if (c >= n_cols) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int s = s0 + ts * 4 + j;
      if (s >= n_occ) continue;
      double *o = part + ((long long)blockIdx.x * 2 * n_cols + 2 * c) * n_occ + s;
      o[0] = (double)are[i][j];
      o[n_occ] = (double)aim[i][j];
    }
  }
}

// d_c(r) -= sum_s O[c][s] phi_s(r) on 128 points per block, all columns in groups of 32 (4 points
// x 4 columns per thread), plus per-block partial sums of 2 Re(conj(eta0) d) and |d|^2 per column.
constexpr int kUpPts = 128, kUpCols = 32, kUpS = 64;

template <typename T>
__global__ void __launch_bounds__(256)
    k_clean_update2(long long ng, const T *phi, int n_occ, const double *ov /* [2c+h][s], x dV */,
                    C2<T> *d, const C2<T> *a, int n_cols, int L, double *npart) {
  using C = C2<T>;
  __shared__ __align__(16) T Ph[kUpS][kUpPts];
  __shared__ __align__(16) C Os[kUpCols][kUpS + 1];
  const int tp = threadIdx.x % 32, tcg = threadIdx.x / 32;
  const long long r0 = (long long)blockIdx.x * kUpPts;
  const bool one_tile = n_occ <= kUpS;
  auto load_phi = [&](int st0) {
    for (int l = threadIdx.x; l < kUpS * kUpPts; l += 256) {
      const int ss = l / kUpPts, pp = l % kUpPts;
      const int s = st0 + ss;
      const long long r = r0 + pp;
      Ph[ss][pp] = (s < n_occ && r < ng) ? phi[(long long)s * ng + r] : T(0);
    }
  };
  if (one_tile) load_phi(0);
  for (int cg0 = 0; cg0 < n_cols; cg0 += kUpCols) {
    C acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = C{T(0), T(0)};
    for (int st0 = 0; st0 < n_occ; st0 += kUpS) {
      __syncthreads();
      if (!one_tile) load_phi(st0);
      for (int l = threadIdx.x; l < kUpCols * kUpS; l += 256) {
        const int cc = l / kUpS, ss = l % kUpS;
        const int c = cg0 + cc, s = st0 + ss;
        C v = C{T(0), T(0)};
        if (c < n_cols && s < n_occ) {
          const double *o = ov + (long long)(2 * c) * n_occ + s;
          v = C{(T)o[0], (T)o[n_occ]};
        }
        Os[cc][ss] = v;
      }
      __syncthreads();
      // the tiles are zero-padded beyond n_occ, so the full (unrolled) tile can be swept
#pragma unroll 16
      for (int ss = 0; ss < kUpS; ++ss) {
        T p[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) p[j] = Ph[ss][tp * 4 + j];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const C o = Os[tcg * 4 + i][ss];
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            acc[i][j].x += o.x * p[j];
            acc[i][j].y += o.y * p[j];
          }
        }
      }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int c = cg0 + tcg * 4 + i;
      // sums in T over the block's 128 points (FP64 per-point work would saturate this GPU's
      // narrow FP64 pipe); FP64 from the per-tile partials on
      T v1 = T(0), v2 = T(0);
      if (c < n_cols) {
        C *dp = d + (long long)c * ng + r0 + tp * 4;
        const C *ap = a + (long long)(c % L) * ng + r0 + tp * 4;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          if (r0 + tp * 4 + j < ng) {
            C dv = dp[j];
            dv.x -= acc[i][j].x;
            dv.y -= acc[i][j].y;
            dp[j] = dv;
            const C a0 = ap[j];
            v1 += T(2) * (a0.x * dv.x + a0.y * dv.y);
            v2 += dv.x * dv.x + dv.y * dv.y;
          }
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        v1 += __shfl_xor_sync(0xffffffffu, v1, o);
        v2 += __shfl_xor_sync(0xffffffffu, v2, o);
      }
      if (tp == 0 && c < n_cols) {
        npart[((long long)blockIdx.x * n_cols + c) * 2 + 0] = (double)v1;
        npart[((long long)blockIdx.x * n_cols + c) * 2 + 1] = (double)v2;
      }
    }
  }
}

template <typename T> size_t clean_work_bytes(long long ng, int n_occ, int P, int L) {
  const long long n_cols = (long long)P * L;
  const long long kc = gemm_kchunk(ng);
  const long long chunks = (ng + kc - 1) / kc;
  const long long ptb = (ng + kUpPts - 1) / kUpPts;
  size_t b = 0;
  const size_t tc_part = std::max(umma_prod_gemm_work_bytes((int)(2 * n_cols), n_occ, ng),
                                  umma_clean_ov_work_bytes((int)n_cols, n_occ, ng));
  const size_t simt_part = (size_t)(chunks * n_cols * n_occ * 2) * sizeof(double);
  b += simt_part > tc_part ? simt_part : tc_part;                 // overlap partials
  b += (size_t)(n_cols * n_occ * 2) * sizeof(double);           // overlaps
  b += (size_t)(ptb * n_cols * 2) * sizeof(double);             // norm partials
  b += (size_t)(n_cols * 2) * sizeof(double);                   // norm sums
  b += (size_t)n_cols * sizeof(double);                         // c - 1 per column
  b = (b + 127) / 128 * 128;
  if (sizeof(T) == 4) b += umma_update_o_bytes((int)n_cols, n_occ);  // overlaps as operand tiles
  return b;
}

template <typename T>
const double *launch_clean(const GridTables<T> &g, const T *phi_occ, int n_occ, const C2<T> *a, C2<T> *d,
                           int P, int L, const double *n0, double dV, double *work, size_t work_bytes,
                           bool use_tc, const uint8_t *phi_can, int *err, cudaStream_t s, T *dens,
                           const uint8_t *phi_ov) {
  (void)work_bytes;
  const int n_cols = P * L;
  const long long kc = gemm_kchunk(g.ng);
  const long long chunks = (g.ng + kc - 1) / kc;
  const long long ptb = (g.ng + kUpPts - 1) / kUpPts;
  double *part = work;
  const size_t tc_part = std::max(umma_prod_gemm_work_bytes(2 * n_cols, n_occ, g.ng),
                                  umma_clean_ov_work_bytes(n_cols, n_occ, g.ng)) / sizeof(double);
  const size_t simt_part = (size_t)(chunks * n_cols * n_occ * 2);
  double *ov = part + (simt_part > tc_part ? simt_part : tc_part);
  double *npart = ov + (long long)n_cols * n_occ * 2;
  double *sums = npart + ptb * n_cols * 2;
  double *cm1 = sums + (long long)n_cols * 2;
  if (phi_ov && sizeof(T) == sizeof(float) &&
      launch_umma_clean_ov(reinterpret_cast<const float *>(d), n_cols, phi_ov, n_occ, g.ng, dV, ov, part, err,
                           s) == 0) {
  } else if (use_tc && sizeof(T) == sizeof(float)) {
    launch_umma_clean_overlap(reinterpret_cast<const float *>(d), n_cols,
                              reinterpret_cast<const float *>(phi_occ), n_occ, g.ng, dV, ov, part, err, s);
  } else {
    dim3 grid((unsigned)chunks, (n_cols + kOvC - 1) / kOvC, (n_occ + kOvS - 1) / kOvS);
    k_clean_overlap<T><<<grid, 256, 0, s>>>(d, phi_occ, n_cols, n_occ, g.ng, kc, part);
    count_launch(1);
    launch_reduce_cols(part, (int)chunks, n_cols * n_occ * 2, dV, ov, s);
  }
  if (phi_can && sizeof(T) == sizeof(float)) {
    size_t o_off = (size_t)((cm1 + n_cols) - work) * sizeof(double);
    o_off = (o_off + 127) / 128 * 128;
    uint8_t *o_can = reinterpret_cast<uint8_t *>(work) + o_off;
    launch_umma_clean_update(ov, n_cols, phi_can, n_occ, g.ng, reinterpret_cast<float *>(d),
                             reinterpret_cast<const float *>(a), L, npart, o_can, err, s);
    launch_reduce_cols(npart, (int)umma_clean_update_tiles(g.ng), n_cols * 2, dV, sums, s);
  } else {
    k_clean_update2<T><<<(unsigned)ptb, 256, 0, s>>>(g.ng, phi_occ, n_occ, ov, d, a, n_cols, L, npart);
    launch_reduce_cols(npart, (int)ptb, n_cols * 2, dV, sums, s);
  }
  k_cm1<<<(n_cols + 127) / 128, 128, 0, s>>>(n_cols, L, sums, n0, cm1);
  dim3 g3((unsigned)((g.ng + 255) / 256), P);
  k_density_renormed<T><<<g3, 256, (size_t)L * sizeof(T), s>>>(g.ng, d, a, L, cm1, dens);
  count_launch(3);
  return cm1;
}

// ------------------------------------------------------------------------------------------

// out = exp(-i V_loc tau) per grid point
// (computed in FP64 from the FP64 potential, then rounded to T)
template <typename T> __global__ void k_phase_table(const double *v, long long ng, double tau, C2<T> *out) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < ng) {
    const double2 e = expmi<double>(v[i] * tau);
    out[i] = C2<T>{(T)e.x, (T)e.y};
  }
}
template <typename T>
void launch_phase_table(const double *v64, long long ng, double tau, C2<T> *out, cudaStream_t s) {
  k_phase_table<T><<<(unsigned)((ng + 255) / 256), 256, 0, s>>>(v64, ng, tau, out);
  count_launch(1);
}

// acc64 += acc; acc = 0  (FP32 partial sums of the time integral folded into the FP64 W)
template <typename T> __global__ void k_flush_acc(double *acc64, T *acc, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    acc64[i] += (double)acc[i];
    acc[i] = T(0);
  }
}
template <typename T> void launch_flush_acc(double *acc64, T *acc, long long n, cudaStream_t s) {
  if (n > 0) k_flush_acc<T><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(acc64, acc, n);
  count_launch(1);
}

template <typename T> __global__ void k_convert(const double *src, T *dst, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = (T)src[i];
}
template <typename T> void launch_convert(const double *src, T *dst, long long n, cudaStream_t s) {
  if (n > 0) k_convert<T><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(src, dst, n);
  count_launch(1);
}

__global__ void k_scan_nonfinite(const double *x, long long n, int *flag) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    if (!isfinite(x[i])) atomicExch(flag, 1);
}
int scan_nonfinite(const double *x, long long n, int *flag_dev, cudaStream_t s) {
  int h = 0;
  cudaMemsetAsync(flag_dev, 0, sizeof(int), s);
  k_scan_nonfinite<<<1024, 256, 0, s>>>(x, n, flag_dev);
  count_launch(1);
  cudaMemcpyAsync(&h, flag_dev, sizeof(int), cudaMemcpyDeviceToHost, s);
  cudaStreamSynchronize(s);
  return h;
}

// one-time opt-in to large dynamic shared memory for the FFT passes
template <typename T> static void set_smem_attrs() {
  const int mx = (int)fft_smem<T>(kMaxN, kTP);
  cudaFuncSetAttribute(k_xfwd<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  cudaFuncSetAttribute(k_ypass<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  cudaFuncSetAttribute(k_zpass<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  cudaFuncSetAttribute(k_xinv_orb<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  cudaFuncSetAttribute(k_xinv_poisson<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
}
void init_fft_kernels() {
  set_smem_attrs<float>();
  set_smem_attrs<double>();
}

#define SBSE_INST(T)                                                                               \
  template void launch_xfwd<T>(const GridTables<T> &, const XfwdArgs<T> &, cudaStream_t);          \
  template void launch_ypass<T>(const GridTables<T> &, C2<T> *, int, int, cudaStream_t);           \
  template void launch_zpass<T>(const GridTables<T> &, C2<T> *, int, int, cudaStream_t);           \
  template void launch_xinv_orb<T>(const GridTables<T> &, C2<T> *, int, const C2<T> *, int, T *,   \
                                   cudaStream_t);                                                  \
  template void launch_xinv_poisson<T>(const GridTables<T> &, C2<T> *, int, const PoissonOut &,    \
                                       T *, T *, C2<T> *, cudaStream_t);                           \
  template void launch_phase_table<T>(const double *, long long, double, C2<T> *, cudaStream_t);  \
  template void launch_flush_acc<T>(double *, T *, long long, cudaStream_t);                       \
  template void launch_init_a<T>(const GridTables<T> &, const double *, int, const double *, int,  \
                                 C2<T> *, double *, int *, cudaStream_t);                          \
  template void launch_kick<T>(const GridTables<T> &, const double *, int, const C2<T> *, int,     \
                               double, C2<T> *, cudaStream_t);                                     \
  template void launch_half_phase<T>(const GridTables<T> &, C2<T> *, C2<T> *, const C2<T> *, int, int, \
                                     cudaStream_t);                                              \
  template const double *launch_clean<T>(const GridTables<T> &, const T *, int, const C2<T> *,      \
                                         C2<T> *, int, int, const double *, double, double *, size_t, \
                                         bool, const uint8_t *, int *, cudaStream_t, T *, const uint8_t *); \
  template size_t clean_work_bytes<T>(long long, int, int, int);                                   \
  template void launch_convert<T>(const double *, T *, long long, cudaStream_t);

SBSE_INST(float)
SBSE_INST(double)

}  // namespace sbse
