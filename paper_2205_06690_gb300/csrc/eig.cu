// Lowest eigenvalues of the real symmetric Tamm-Dancoff matrix A (Eq. 1), in FP64 on the device:
// Householder reduction to tridiagonal form (one block, matrix in global memory / L2) followed by
// Sturm-sequence bisection, one thread per requested eigenvalue.
#include <math.h>

#include "kernels.h"

namespace sbse {

constexpr int kEigThreads = 1024;

__device__ double block_sum(double v, double *red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x < 32) {
    s = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) red[32] = s;
  }
  __syncthreads();
  return red[32];
}

// A (n x n, row-major, overwritten) -> diagonal dg[n] and off-diagonal of[n-1].
// H = I - beta v v^T maps A[k+1:, k] onto alpha e_1; the trailing block becomes
// A' - v w^T - w v^T with p = beta A' v, K = beta v.p / 2, w = p - K v.
__global__ void __launch_bounds__(kEigThreads) k_tridiag(double *A, int n, double *dg, double *of) {
  extern __shared__ double sm[];
  double *v = sm;
  double *p = v + n;
  double *red = p + n;  // 33 doubles
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  for (int k = 0; k + 2 < n; ++k) {
    const int m = n - k - 1;
    const int o = k + 1;
    double ss = 0.0;
    for (int i = tid; i < m; i += blockDim.x) {
      const double x = A[(long long)(o + i) * n + k];
      v[i] = x;
      ss += x * x;
    }
    const double sigma = block_sum(ss, red);
    const double x0 = v[0];
    if (sigma - x0 * x0 <= 0.0) {  // column already reduced
      if (tid == 0) {
        dg[k] = A[(long long)k * n + k];
        of[k] = x0;
      }
      __syncthreads();
      continue;
    }
    const double alpha = (x0 >= 0.0) ? -sqrt(sigma) : sqrt(sigma);
    const double beta = 1.0 / (sigma - x0 * alpha);  // 2 / |v|^2
    __syncthreads();
    if (tid == 0) v[0] = x0 - alpha;
    __syncthreads();
    // p = beta A' v, one warp per row (coalesced across the row)
    for (int i = warp; i < m; i += nw) {
      const double *row = A + (long long)(o + i) * n + o;
      double s = 0.0;
      for (int j = lane; j < m; j += 32) s += row[j] * v[j];
      for (int q = 16; q > 0; q >>= 1) s += __shfl_xor_sync(0xffffffffu, s, q);
      if (lane == 0) p[i] = beta * s;
    }
    __syncthreads();
    double vp = 0.0;
    for (int i = tid; i < m; i += blockDim.x) vp += v[i] * p[i];
    const double K = 0.5 * beta * block_sum(vp, red);
    for (int i = tid; i < m; i += blockDim.x) p[i] -= K * v[i];  // p <- w
    __syncthreads();
    const long long mm = (long long)m * m;
    for (long long l = tid; l < mm; l += blockDim.x) {
      const int i = (int)(l / m), j = (int)(l - (long long)i * m);
      A[(long long)(o + i) * n + o + j] -= v[i] * p[j] + p[i] * v[j];
    }
    if (tid == 0) {
      dg[k] = A[(long long)k * n + k];
      of[k] = alpha;
    }
    __syncthreads();
  }
  if (tid == 0) {
    if (n >= 2) {
      dg[n - 2] = A[(long long)(n - 2) * n + n - 2];
      of[n - 2] = A[(long long)(n - 1) * n + n - 2];
    }
    dg[n - 1] = A[(long long)(n - 1) * n + n - 1];
  }
}

// number of eigenvalues of the tridiagonal (dg, of) below x (Sturm count by LDL^T pivots)
__device__ int sturm_count(const double *dg, const double *of, int n, double x, double tiny) {
  int c = 0;
  double q = dg[0] - x;
  if (q == 0.0) q = -tiny;
  if (q < 0.0) ++c;
  for (int i = 1; i < n; ++i) {
    q = dg[i] - x - of[i - 1] * of[i - 1] / q;
    if (q == 0.0) q = -tiny;
    if (q < 0.0) ++c;
  }
  return c;
}

__global__ void k_bisect(const double *dg, const double *of, int n, int k, double *ev) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= k) return;
  double lo = dg[0], hi = dg[0], nrm = 0.0;
  for (int i = 0; i < n; ++i) {
    const double r = (i > 0 ? fabs(of[i - 1]) : 0.0) + (i < n - 1 ? fabs(of[i]) : 0.0);
    lo = fmin(lo, dg[i] - r);
    hi = fmax(hi, dg[i] + r);
    nrm = fmax(nrm, fabs(dg[i]) + r);
  }
  const double tiny = 1e-300 + 1e-30 * nrm * 2.2e-16;
  lo -= 1e-12 * (nrm + 1.0);
  hi += 1e-12 * (nrm + 1.0);
  // find x with count(x) <= j < count(x') ... the (j+1)-th smallest eigenvalue
  for (int it = 0; it < 200; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (mid <= lo || mid >= hi) break;
    if (sturm_count(dg, of, n, mid, tiny) > j)
      hi = mid;
    else
      lo = mid;
  }
  ev[j] = 0.5 * (lo + hi);
}

size_t eig_work_bytes(int n) { return (size_t)n * n * sizeof(double) + 2 * (size_t)n * sizeof(double); }

// A (device, n x n) is copied into work and reduced there; the lowest k eigenvalues go to evals_dev.
int launch_eig_lowest(double *A, int n, int k, double *evals_dev, double *work, cudaStream_t s) {
  double *Aw = work;
  double *dg = Aw + (long long)n * n;
  double *of = dg + n;
  cudaMemcpyAsync(Aw, A, (size_t)n * n * sizeof(double), cudaMemcpyDeviceToDevice, s);
  const size_t sm = (2 * (size_t)n + 33) * sizeof(double);
  if (sm > 48 * 1024) cudaFuncSetAttribute(k_tridiag, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (n >= 3) {
    k_tridiag<<<1, kEigThreads, sm, s>>>(Aw, n, dg, of);
    count_launch(1);
  } else {
    // n <= 2: the matrix is already tridiagonal
    cudaMemcpyAsync(dg, Aw, sizeof(double), cudaMemcpyDeviceToDevice, s);
    if (n == 2) {
      cudaMemcpyAsync(dg + 1, Aw + 3, sizeof(double), cudaMemcpyDeviceToDevice, s);
      cudaMemcpyAsync(of, Aw + 2, sizeof(double), cudaMemcpyDeviceToDevice, s);
    }
  }
  k_bisect<<<(k + 127) / 128, 128, 0, s>>>(dg, of, n, k, evals_dev);
  count_launch(1);
  return 0;
}

}  // namespace sbse
