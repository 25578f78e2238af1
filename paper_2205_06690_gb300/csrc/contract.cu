// Grid-sum contractions of Eq. (1) and the assembly of the Tamm-Dancoff matrix A.
//   exchange (ia|jb) = dV sum_r [phi_i phi_a](r) [v phi_j phi_b](r)
//   direct   (phi_a phi_b|W|phi_i phi_j) = dV sum_r [phi_a phi_b](r) W_ij(r)
// Both are "pair product x field" GEMMs over the grid: the pair products are formed while the
// tile is loaded and never stored.
#include "gemm_nt.cuh"
#include "kernels.h"

namespace sbse {

template <typename T> struct LoadProduct {  // X_m(r) = F[xi[m].x](r) * F[xi[m].y](r)
  const T *F;
  const int2 *xi;
  long long ng;
  __device__ T operator()(int m, long long k) const {
    const int2 q = xi[m];
    return F[(long long)q.x * ng + k] * F[(long long)q.y * ng + k];
  }
};
template <typename T> struct LoadField {
  const T *Y;
  long long ng;
  __device__ T operator()(int n, long long k) const { return Y[(long long)n * ng + k]; }
};

template <typename T> size_t prod_gemm_work_bytes(int M, int Nn, long long ng) {
  const long long kc = gemm_kchunk(ng);
  const long long chunks = (ng + kc - 1) / kc;
  return (size_t)(chunks * M * Nn) * sizeof(double);
}

template <typename T>
void launch_prod_gemm(const T *F, const int2 *xi, int M, const T *Y, int Nn, long long ng,
                      double scale, double *out, double *work, size_t work_bytes, cudaStream_t s) {
  (void)work_bytes;
  const long long kc = gemm_kchunk(ng);
  const long long chunks = (ng + kc - 1) / kc;
  dim3 grid((unsigned)chunks, (M + kGemmBM - 1) / kGemmBM, (Nn + kGemmBN - 1) / kGemmBN);
  k_gemm_nt_part<T><<<grid, kGemmThreads, 0, s>>>(M, Nn, ng, kc, LoadProduct<T>{F, xi, ng},
                                                   LoadField<T>{Y, ng}, work);
  count_launch(1);
  launch_reduce_cols(work, (int)chunks, M * Nn, scale, out, s);
}

// A[ia][jb] = delta (eps_a - eps_i + Delta) + 2 K[ia][jb] - Dab[a * n_c + b][p(i, j)], with
// p(i, j) the index of the pair (min(i,j), max(i,j)) in the order (0,0), (0,1), .., (1,1), ..
// and W_ji = W_ij, so for i > j the direct element is Dab[b * n_c + a][p(j, i)].
// K or Dab may be null (term switched off). With fock_o (a rotated occupied window, Forward
// perspective) the diagonal term is delta_ab (eps_a delta_ij - F_ij) + Delta delta_ij delta_ab.
__global__ void k_assemble_A(const double *eps_o, const double *eps_c, int n_o, int n_c,
                             double scissor, const double *K, const double *Dab, int P, double *A,
                             const double *fock_o) {
  const int n = n_o * n_c;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)n * n) return;
  const int row = (int)(idx / n), col = (int)(idx % n);
  const int i = row / n_c, a = row % n_c, j = col / n_c, b = col % n_c;
  double v;
  if (fock_o)
    v = (a == b ? ((i == j ? eps_c[a] + scissor : 0.0) - fock_o[i * n_o + j]) : 0.0);
  else
    v = (row == col) ? (eps_c[a] - eps_o[i] + scissor) : 0.0;
  if (K) v += 2.0 * K[idx];
  if (Dab) {
    const int lo = i < j ? i : j, hi = i < j ? j : i;
    const int p = lo * n_o - lo * (lo - 1) / 2 + (hi - lo);
    const int ab = (i <= j) ? a * n_c + b : b * n_c + a;
    v -= Dab[(long long)ab * P + p];
  }
  A[idx] = v;
}

void launch_assemble_A(const double *eps_o, const double *eps_c, int n_o, int n_c, double scissor,
                       const double *K, const double *Dab, int P, double *A, cudaStream_t s,
                       const double *fock_o) {
  const long long n2 = (long long)(n_o * n_c) * (n_o * n_c);
  k_assemble_A<<<(unsigned)((n2 + 255) / 256), 256, 0, s>>>(eps_o, eps_c, n_o, n_c, scissor, K, Dab,
                                                           P, A, fock_o);
  count_launch(1);
}

template size_t prod_gemm_work_bytes<float>(int, int, long long);
template size_t prod_gemm_work_bytes<double>(int, int, long long);
template void launch_prod_gemm<float>(const float *, const int2 *, int, const float *, int, long long,
                                      double, double *, double *, size_t, cudaStream_t);
template void launch_prod_gemm<double>(const double *, const int2 *, int, const double *, int,
                                       long long, double, double *, double *, size_t, cudaStream_t);

}  // namespace sbse
