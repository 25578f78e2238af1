// Absorption spectrum of the exciton matrix A by a Chebyshev expansion (Sec. II.C, electron-hole
// basis: the paragraph after Eq. 18): sigma(omega) = omega <f0| delta_s(A - omega) |f0> with the
// dipole start vector f0_ia = <phi_a| x |phi_i>, so that only the residues R_n = <f0|T_n(A~)|f0> of
// repeated applications of the scaled A are needed.
//
//   dipoles   : one block per (i, a), FP64 grid sum with x measured from the box centre
//   scaling   : Gershgorin bounds [lo, hi] of A, A~ = (A - c) / w, c = (lo + hi) / 2,
//               w = 1.01 (hi - lo) / 2
//   recursion : v_0 = f0, v_1 = A~ f0, v_{n+1} = 2 A~ v_n - v_{n-1} (one launch per term, a warp
//               per row of A); f0_r v_n[r] is stored per row and term and reduced in a fixed order
//   spectrum  : with K = n_terms Chebyshev-Gauss nodes x_k = cos(pi (k + 1/2) / K),
//               D_k = sum_n (2 - delta_n0) R_n T_n(x_k) and
//               sigma(omega) = omega / K sum_k G_s(c + w x_k - omega) D_k, G_s a normalised Gaussian.
// Everything is FP64 (A is FP64 in both precision modes).
#include <math.h>

#include "kernels.h"

namespace sbse {

namespace {

constexpr int kSpT = 256;

__device__ __forceinline__ double block_sum_fixed(double v, double *red) {
  red[threadIdx.x] = v;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  const double s = red[0];
  __syncthreads();
  return s;
}

// f0[i n_c + a] = dV sum_r phi_c[a](r) x(r) phi_o[i](r)
__global__ void __launch_bounds__(kSpT)
    k_dipole(const double *phi_o, const double *phi_c, int n_c, int N, double h, double box, int axis, double dV,
             double *f0) {
  __shared__ double red[kSpT];
  const int i = blockIdx.x / n_c, a = blockIdx.x - i * n_c;
  const long long ng = (long long)N * N * N;
  const double *pi = phi_o + (long long)i * ng, *pa = phi_c + (long long)a * ng;
  double s = 0.0;
  for (long long r = threadIdx.x; r < ng; r += kSpT) {
    const long long idx = axis == 0 ? r % N : (axis == 1 ? (r / N) % N : r / ((long long)N * N));
    s += pi[r] * pa[r] * (h * (double)idx - 0.5 * box);
  }
  s = block_sum_fixed(s, red);
  if (threadIdx.x == 0) f0[blockIdx.x] = s * dV;
}

// cw = {c, w} from the Gershgorin discs of the rows of A; R_0 term and v_0 = f0
__global__ void __launch_bounds__(kSpT)
    k_cheb_init(const double *A, int n, const double *f0, double *cw, double *v0, double *prod, int n_terms) {
  __shared__ double red[kSpT];
  double lo = INFINITY, hi = -INFINITY;
  for (int r = threadIdx.x; r < n; r += kSpT) {
    double rad = 0.0;
    for (int j = 0; j < n; ++j)
      if (j != r) rad += fabs(A[(long long)r * n + j]);
    const double d = A[(long long)r * n + r];
    lo = fmin(lo, d - rad);
    hi = fmax(hi, d + rad);
    v0[r] = f0[r];
    prod[(long long)r * n_terms] = f0[r] * f0[r];
  }
  red[threadIdx.x] = lo;
  __syncthreads();
  for (int w = kSpT / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] = fmin(red[threadIdx.x], red[threadIdx.x + w]);
    __syncthreads();
  }
  const double glo = red[0];
  __syncthreads();
  red[threadIdx.x] = hi;
  __syncthreads();
  for (int w = kSpT / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + w]);
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    cw[0] = 0.5 * (glo + red[0]);
    cw[1] = 1.01 * 0.5 * (red[0] - glo);
  }
}

// v_next = A~ v_cur (first term) or 2 A~ v_cur - v_prev; prod[r][term] = f0_r v_next[r]
__global__ void __launch_bounds__(kSpT)
    k_cheb_step(const double *A, int n, const double *cw, const double *f0, const double *v_prev,
                const double *v_cur, double *v_next, double *prod, int n_terms, int term) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int r = blockIdx.x * (kSpT / 32) + warp;
  if (r >= n) return;
  const double *row = A + (long long)r * n;
  double s = 0.0;
  for (int j = lane; j < n; j += 32) s += row[j] * v_cur[j];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) {
    const double at = (s - cw[0] * v_cur[r]) / cw[1];
    const double v = term == 1 ? at : 2.0 * at - v_prev[r];
    v_next[r] = v;
    prod[(long long)r * n_terms + term] = f0[r] * v;
  }
}

// D_k = sum_n (2 - delta_n0) R_n T_n(x_k), T_n(x_k) = cos(pi n (k + 1/2) / K)
__global__ void k_cheb_density(const double *R, int K, double *D) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= K) return;
  const double t = ((double)k + 0.5) / (double)K;
  double s = R[0];
  for (int n = 1; n < K; ++n) s += 2.0 * R[n] * cospi((double)n * t);
  D[k] = s;
}

// sigma_j = omega_j / K sum_k G_s(c + w x_k - omega_j) D_k
__global__ void k_sigma(const double *D, int K, const double *cw, const double *omega, int n_omega, double s,
                        double *sigma) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n_omega) return;
  const double c = cw[0], w = cw[1], om = omega[j];
  const double norm = 1.0 / (s * sqrt(2.0 * M_PI));
  double acc = 0.0;
  for (int k = 0; k < K; ++k) {
    const double e = (c + w * cospi(((double)k + 0.5) / (double)K) - om) / s;
    acc += exp(-0.5 * e * e) * D[k];
  }
  sigma[j] = om * norm * acc / (double)K;
}

}  // namespace

size_t spectrum_work_bytes(int n, int n_terms, int n_omega) {
  // f0, cw, three vectors, prod (n x n_terms), R, D, omega, sigma
  return sizeof(double) * ((size_t)n + 2 + 3 * (size_t)n + (size_t)n * n_terms + 2 * (size_t)n_terms +
                           2 * (size_t)n_omega);
}

SpectrumBufs spectrum_bufs(double *work, int n, int n_terms, int n_omega) {
  SpectrumBufs b{};
  b.f0 = work;
  b.cw = b.f0 + n;
  b.v[0] = b.cw + 2;
  b.v[1] = b.v[0] + n;
  b.v[2] = b.v[1] + n;
  b.prod = b.v[2] + n;
  b.R = b.prod + (size_t)n * n_terms;
  b.D = b.R + n_terms;
  b.omega = b.D + n_terms;
  b.sigma = b.omega + n_omega;
  return b;
}

void launch_sigma_from_residues(const double *R, int K, const double *cw, const double *omega, int n_omega,
                                double s, double *D, double *sigma, cudaStream_t st) {
  k_cheb_density<<<(K + 127) / 128, 128, 0, st>>>(R, K, D);
  k_sigma<<<(n_omega + 127) / 128, 128, 0, st>>>(D, K, cw, omega, n_omega, s, sigma);
  count_launch(2);
}

void launch_absorption(const SpectrumBufs &b, const double *phi_o, const double *phi_c, int n_o, int n_c, int N,
                       double h, double box, double dV, const double *A, int axis, int n_terms, double s,
                       int n_omega, cudaStream_t st) {
  const int n = n_o * n_c;
  k_dipole<<<n, kSpT, 0, st>>>(phi_o, phi_c, n_c, N, h, box, axis, dV, b.f0);
  k_cheb_init<<<1, kSpT, 0, st>>>(A, n, b.f0, b.cw, b.v[0], b.prod, n_terms);
  count_launch(2);
  const unsigned row_blocks = (unsigned)((n + kSpT / 32 - 1) / (kSpT / 32));
  for (int t = 1; t < n_terms; ++t) {  // v_t from v_{t-1} (and v_{t-2}), rotating three buffers
    const double *prev = t >= 2 ? b.v[(t - 2) % 3] : nullptr;
    k_cheb_step<<<row_blocks, kSpT, 0, st>>>(A, n, b.cw, b.f0, prev, b.v[(t - 1) % 3], b.v[t % 3], b.prod,
                                             n_terms, t);
  }
  count_launch(n_terms - 1);
  launch_reduce_cols(b.prod, n, n_terms, 1.0, b.R, st);
  k_cheb_density<<<(n_terms + 127) / 128, 128, 0, st>>>(b.R, n_terms, b.D);
  k_sigma<<<(n_omega + 127) / 128, 128, 0, st>>>(b.D, n_terms, b.cw, b.omega, n_omega, s, b.sigma);
  count_launch(2);
}

}  // namespace sbse
