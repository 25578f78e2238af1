// Localized occupied window (Forward perspective of the paper: localized occupied orbitals reduce the
// number of (i, j) pairs whose W_ij is needed): the device parts of the Gamma-point localization and
// of the pair screening. The Jacobi sweeps themselves run on the host (n_o x n_o matrices).
//   k_phase_fields : cos, sin of 2 pi x_alpha / L on the grid, alpha = x, y, z (6 fields)
//   (the spread matrices Z_alpha,ij = dV sum_r phi_i phi_j e^{i 2 pi x_alpha / L} are a pair-product
//    grid sum, launch_prod_gemm against those six fields)
//   k_rotate_rows  : phi'_k = sum_i U_ik phi_i for the n_o window rows (into a separate buffer)
//   k_pair_norms   : sum_r (phi_i phi_j)^2 per pair, block partials
#include <math.h>

#include "kernels.h"

namespace sbse {

namespace {

__global__ void k_phase_fields(int N, double *out) {
  const long long ng = (long long)N * N * N;
  for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < ng; r += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(r % N), y = (int)((r / N) % N), z = (int)(r / ((long long)N * N));
    const int idx[3] = {x, y, z};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      double s, c;
      sincospi(2.0 * (double)idx[a] / (double)N, &s, &c);
      out[(2 * a) * ng + r] = c;
      out[(2 * a + 1) * ng + r] = s;
    }
  }
}

// out[k] = sum_i U_ik phi[base + i] for k < n (rows of ng points); U row-major n x n
__global__ void k_rotate_rows(const double *phi, int base, int n, const double *U, long long ng, double *out) {
  extern __shared__ double Us[];
  for (int i = threadIdx.x; i < n * n; i += blockDim.x) Us[i] = U[i];
  __syncthreads();
  double v[32];
  for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < ng; r += (long long)gridDim.x * blockDim.x) {
    for (int c0 = 0; c0 < n; c0 += 32) {
      const int cn = n - c0 < 32 ? n - c0 : 32;
#pragma unroll
      for (int k = 0; k < 32; ++k) v[k] = 0.0;
      for (int i = 0; i < n; ++i) {
        const double p = phi[(long long)(base + i) * ng + r];
#pragma unroll
        for (int k = 0; k < 32; ++k)
          if (k < cn) v[k] += Us[i * n + c0 + k] * p;
      }
#pragma unroll
      for (int k = 0; k < 32; ++k)
        if (k < cn) out[(long long)(c0 + k) * ng + r] = v[k];
    }
  }
}

constexpr int kPnBlocks = 128;

__global__ void k_pair_norms(const double *phi, const int2 *pairs, long long ng, double *part) {
  __shared__ double red[256];
  const int2 q = pairs[blockIdx.y];
  const double *a = phi + (long long)q.x * ng, *b = phi + (long long)q.y * ng;
  double s = 0.0;
  for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < ng; r += (long long)gridDim.x * blockDim.x) {
    const double p = a[r] * b[r];
    s += p * p;
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[(long long)blockIdx.x * gridDim.y + blockIdx.y] = red[0];
}

}  // namespace

void launch_phase_fields(int N, double *out, cudaStream_t s) {
  k_phase_fields<<<1024, 256, 0, s>>>(N, out);
  count_launch(1);
}

void launch_rotate_rows(const double *phi, int base, int n, const double *U, long long ng, double *out,
                        cudaStream_t s) {
  k_rotate_rows<<<1024, 128, (size_t)n * n * sizeof(double), s>>>(phi, base, n, U, ng, out);
  count_launch(1);
}

size_t pair_norms_work_doubles(int n_pairs) { return (size_t)kPnBlocks * n_pairs; }

void launch_pair_norms(const double *phi, const int2 *pairs, int n_pairs, long long ng, double scale,
                       double *work, double *out, cudaStream_t s) {
  k_pair_norms<<<dim3(kPnBlocks, n_pairs), 256, 0, s>>>(phi, pairs, ng, work);
  count_launch(1);
  launch_reduce_cols(work, kPnBlocks, n_pairs, scale, out, s);
}

}  // namespace sbse
