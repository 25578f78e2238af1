// Split-K "NT" GEMM over grid points: part[chunk][m][n] = sum_{k in chunk} A(m, k) B(n, k).
// Both operands are indexed (row, grid point) and read through functors, so pair products and
// complex columns are formed while loading instead of being materialised. Used for the cleaning
// overlaps of Eq. (15) and the grid-sum contractions of the exchange and direct elements of Eq. (1).
// Chunks are accumulated in T and written as FP64 partials; a fixed-order column reduction
// (launch_reduce_cols) finishes the sum, so results are deterministic.
#pragma once

#include "common.cuh"

namespace sbse {

constexpr int kGemmBM = 64, kGemmBN = 64, kGemmBK = 16, kGemmThreads = 256;

template <typename T, class LA, class LB>
__global__ void __launch_bounds__(kGemmThreads)
    k_gemm_nt_part(int M, int Nn, long long K, long long kchunk, LA la, LB lb, double *part) {
  __shared__ T As[kGemmBK][kGemmBM + 4];
  __shared__ T Bs[kGemmBK][kGemmBN + 4];
  const int m0 = blockIdx.y * kGemmBM, n0 = blockIdx.z * kGemmBN;
  const long long kbeg = (long long)blockIdx.x * kchunk;
  const long long kend = (kbeg + kchunk < K) ? kbeg + kchunk : K;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  T acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = T(0);
  for (long long k0 = kbeg; k0 < kend; k0 += kGemmBK) {
    for (int l = threadIdx.x; l < kGemmBM * kGemmBK; l += kGemmThreads) {
      const int mm = l / kGemmBK, kk = l % kGemmBK;
      const long long k = k0 + kk;
      const int m = m0 + mm;
      As[kk][mm] = (m < M && k < kend) ? la(m, k) : T(0);
    }
    for (int l = threadIdx.x; l < kGemmBN * kGemmBK; l += kGemmThreads) {
      const int nn = l / kGemmBK, kk = l % kGemmBK;
      const long long k = k0 + kk;
      const int n = n0 + nn;
      Bs[kk][nn] = (n < Nn && k < kend) ? lb(n, k) : T(0);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kGemmBK; ++kk) {
      T a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] += a[i] * b[j];
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int m = m0 + ty * 4 + i;
    if (m >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int n = n0 + tx * 4 + j;
      if (n < Nn) part[((long long)blockIdx.x * M + m) * Nn + n] = (double)acc[i][j];
    }
  }
}

// Number of K chunks used for a GEMM with K grid points (at most 65535, at least 1).
inline long long gemm_kchunk(long long K) {
  long long c = 4096;
  while ((K + c - 1) / c > 2048) c *= 2;
  return c;
}

}  // namespace sbse
