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
// INSMEM: the matrix is first copied to shared memory (small n), otherwise it stays in global
// memory (L2-resident for the sizes of A).
// refl != null: the Householder vector of step k is stored in row k of refl (entries k+1 .. n-1)
// and its beta in betas[k] (0 where the step is the identity), for the back-transformation of
// eigenvectors.
template <bool INSMEM>
__global__ void __launch_bounds__(kEigThreads)
    k_tridiag(double *Ag, int n, double *dg, double *of, double *refl, double *betas) {
  extern __shared__ double sm[];
  double *v = sm;
  double *p = v + n;
  double *red = p + n;  // 33 doubles
  double *A = Ag;
  if (INSMEM) {
    A = red + 34;
    for (long long l = threadIdx.x; l < (long long)n * n; l += blockDim.x) A[l] = Ag[l];
    __syncthreads();
  }
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
        if (betas) betas[k] = 0.0;
      }
      __syncthreads();
      continue;
    }
    const double alpha = (x0 >= 0.0) ? -sqrt(sigma) : sqrt(sigma);
    const double beta = 1.0 / (sigma - x0 * alpha);  // 2 / |v|^2
    __syncthreads();
    if (tid == 0) v[0] = x0 - alpha;
    __syncthreads();
    if (refl) {
      for (int i = tid; i < m; i += blockDim.x) refl[(long long)k * n + o + i] = v[i];
      if (tid == 0) betas[k] = beta;
    }
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

// (j+1)-th smallest eigenvalue by multisection: one warp per eigenvalue, each lane counts the
// eigenvalues below one of 32 interior points of the bracket, which shrinks 33-fold per round.
__global__ void k_bisect(const double *dg, const double *of, int n, int k, double *ev) {
  const int lane = threadIdx.x & 31;
  const int j = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
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
  for (int it = 0; it < 64; ++it) {
    const double w = (hi - lo) / 33.0;
    const double x = lo + (lane + 1) * w;
    const bool below = (x > lo && x < hi) ? (sturm_count(dg, of, n, x, tiny) <= j) : (x <= lo);
    const unsigned bal = __ballot_sync(0xffffffffu, below);
    const int m = __popc(bal);  // lanes 0..m-1 have at most j eigenvalues below their point
    const double nlo = (m == 0) ? lo : lo + m * w;
    const double nhi = (m == 32) ? hi : lo + (m + 1) * w;
    if (!(nhi - nlo < hi - lo)) break;  // no further progress in floating point
    lo = nlo;
    hi = nhi;
  }
  if (lane == 0) ev[j] = 0.5 * (lo + hi);
}

size_t eig_work_bytes(int n) { return (size_t)n * n * sizeof(double) + 2 * (size_t)n * sizeof(double); }

// A (device, n x n) is copied into work and reduced there; the lowest k eigenvalues go to evals_dev.
int launch_eig_lowest(double *A, int n, int k, double *evals_dev, double *work, cudaStream_t s) {
  double *Aw = work;
  double *dg = Aw + (long long)n * n;
  double *of = dg + n;
  cudaMemcpyAsync(Aw, A, (size_t)n * n * sizeof(double), cudaMemcpyDeviceToDevice, s);
  const size_t sm = (2 * (size_t)n + 34) * sizeof(double);
  const size_t sm_full = sm + (size_t)n * n * sizeof(double);
  if (n >= 3) {
    if (sm_full <= 200 * 1024) {
      raise_smem_limit((const void *)k_tridiag<true>, sm_full);
      k_tridiag<true><<<1, kEigThreads, sm_full, s>>>(Aw, n, dg, of, nullptr, nullptr);
    } else {
      if (sm > 48 * 1024)
        raise_smem_limit((const void *)k_tridiag<false>, sm);
      k_tridiag<false><<<1, kEigThreads, sm, s>>>(Aw, n, dg, of, nullptr, nullptr);
    }
    count_launch(1);
  } else {
    // n <= 2: the matrix is already tridiagonal
    cudaMemcpyAsync(dg, Aw, sizeof(double), cudaMemcpyDeviceToDevice, s);
    if (n == 2) {
      cudaMemcpyAsync(dg + 1, Aw + 3, sizeof(double), cudaMemcpyDeviceToDevice, s);
      cudaMemcpyAsync(of, Aw + 2, sizeof(double), cudaMemcpyDeviceToDevice, s);
    }
  }
  k_bisect<<<(k + 7) / 8, 256, 0, s>>>(dg, of, n, k, evals_dev);
  count_launch(1);
  return 0;
}

// ---- eigenvectors: inverse iteration on the tridiagonal T, then x = Q y with the stored reflectors

// (T - lam I) = P L U by Gaussian elimination with partial pivoting (row interchanges between
// neighbours); U has the diagonal d, first and second superdiagonals e, f; mult and piv record
// the elimination for the right-hand sides. tiny replaces exact zero pivots.
__device__ void tri_factor(const double *dg, const double *of, int n, double lam, double tiny, double *d,
                           double *e, double *f, double *mult, unsigned char *piv) {
  double b = dg[0] - lam, c = n > 1 ? of[0] : 0.0;
  for (int i = 0; i + 1 < n; ++i) {
    const double a = of[i], bn = dg[i + 1] - lam, cn = (i + 2 < n) ? of[i + 1] : 0.0;
    if (fabs(b) >= fabs(a)) {
      if (b == 0.0) b = tiny;
      const double m = a / b;
      piv[i] = 0;
      d[i] = b;
      e[i] = c;
      f[i] = 0.0;
      mult[i] = m;
      b = bn - m * c;
      c = cn;
    } else {
      const double m = b / a;
      piv[i] = 1;
      d[i] = a;
      e[i] = bn;
      f[i] = cn;
      mult[i] = m;
      b = c - m * bn;
      c = -m * cn;
    }
  }
  d[n - 1] = (b == 0.0) ? tiny : b;
}

// r <- (T - lam I)^-1 r with the factors of tri_factor
__device__ void tri_solve(int n, const double *d, const double *e, const double *f, const double *mult,
                          const unsigned char *piv, double *r) {
  for (int i = 0; i + 1 < n; ++i) {
    if (piv[i]) {
      const double t = r[i];
      r[i] = r[i + 1];
      r[i + 1] = t;
    }
    r[i + 1] -= mult[i] * r[i];
  }
  r[n - 1] /= d[n - 1];
  if (n >= 2) r[n - 2] = (r[n - 2] - e[n - 2] * r[n - 1]) / d[n - 2];
  for (int i = n - 3; i >= 0; --i) r[i] = (r[i] - e[i] * r[i + 1] - f[i] * r[i + 2]) / d[i];
}

// eigenvectors Y[j][.] of T for the ascending eigenvalues ev[j], j < k (one block): three inverse
// iterations each from a fixed start vector; a vector whose eigenvalue is within 1e-3 |T| of an
// earlier one is orthogonalised against that cluster after every iteration.
__global__ void __launch_bounds__(256)
    k_tri_vectors(const double *dg, const double *of, int n, int k, const double *ev, double *Y,
                  double *fac /* 4 n doubles + n bytes */) {
  __shared__ double red[33];
  double *d = fac, *e = d + n, *f = e + n, *mult = f + n;
  unsigned char *piv = reinterpret_cast<unsigned char *>(mult + n);
  double nrm = 0.0;
  for (int i = 0; i < n; ++i)
    nrm = fmax(nrm, fabs(dg[i]) + (i > 0 ? fabs(of[i - 1]) : 0.0) + (i + 1 < n ? fabs(of[i]) : 0.0));
  const double tiny = 2.2e-16 * (nrm + 1e-300);
  for (int j = 0; j < k; ++j) {
    double *y = Y + (long long)j * n;
    if (threadIdx.x == 0) tri_factor(dg, of, n, ev[j], tiny, d, e, f, mult, piv);
    for (int i = threadIdx.x; i < n; i += blockDim.x) y[i] = 1.0 + 0.5 * sin(1.0 + i);  // fixed start
    __syncthreads();
    for (int it = 0; it < 3; ++it) {
      if (threadIdx.x == 0) tri_solve(n, d, e, f, mult, piv, y);
      __syncthreads();
      for (int q = j - 1; q >= 0 && ev[j] - ev[q] < 1e-3 * nrm; --q) {  // cluster: Gram-Schmidt
        const double *yq = Y + (long long)q * n;
        double s = 0.0;
        for (int i = threadIdx.x; i < n; i += blockDim.x) s += yq[i] * y[i];
        s = block_sum(s, red);
        for (int i = threadIdx.x; i < n; i += blockDim.x) y[i] -= s * yq[i];
        __syncthreads();
      }
      double s = 0.0;
      for (int i = threadIdx.x; i < n; i += blockDim.x) s += y[i] * y[i];
      const double inv = 1.0 / sqrt(block_sum(s, red));
      for (int i = threadIdx.x; i < n; i += blockDim.x) y[i] *= inv;
      __syncthreads();
    }
  }
}

// x_j = H_0 H_1 ... H_{n-3} y_j (one block per eigenvector), sign fixed so that the component of
// largest magnitude is positive; X row-major n x k
__global__ void __launch_bounds__(256)
    k_tri_backtransform(const double *refl, const double *betas, int n, int k, const double *Y, double *X) {
  extern __shared__ double sy[];
  __shared__ double red[33];
  const int j = blockIdx.x;
  for (int i = threadIdx.x; i < n; i += blockDim.x) sy[i] = Y[(long long)j * n + i];
  __syncthreads();
  for (int kk = n - 3; kk >= 0; --kk) {
    const double beta = betas[kk];
    if (beta == 0.0) continue;
    const double *v = refl + (long long)kk * n;
    double s = 0.0;
    for (int i = kk + 1 + threadIdx.x; i < n; i += blockDim.x) s += v[i] * sy[i];
    s = beta * block_sum(s, red);
    for (int i = kk + 1 + threadIdx.x; i < n; i += blockDim.x) sy[i] -= s * v[i];
    __syncthreads();
  }
  // sign: the largest-magnitude component positive (first index on ties)
  double best = -1.0;
  int arg = n;
  for (int i = threadIdx.x; i < n; i += blockDim.x)
    if (fabs(sy[i]) > best) {
      best = fabs(sy[i]);
      arg = i;
    }
  __shared__ double bv[256];
  __shared__ int bi[256];
  bv[threadIdx.x] = best;
  bi[threadIdx.x] = arg;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) {
      const double o = bv[threadIdx.x + w];
      const int oi = bi[threadIdx.x + w];
      if (o > bv[threadIdx.x] || (o == bv[threadIdx.x] && oi < bi[threadIdx.x])) {
        bv[threadIdx.x] = o;
        bi[threadIdx.x] = oi;
      }
    }
    __syncthreads();
  }
  const double sg = (bi[0] < n && sy[bi[0]] < 0.0) ? -1.0 : 1.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) X[(long long)i * k + j] = sg * sy[i];
}

size_t eig_vectors_work_bytes(int n, int k) {
  return eig_work_bytes(n) + ((size_t)n * n + n + (size_t)k * n + 4 * (size_t)n) * sizeof(double) + n + 16;
}

// lowest k eigenvalues and their eigenvectors (row-major n x k, device) of A (device, n x n)
int launch_eig_vectors(const double *A, int n, int k, double *evals_dev, double *evecs_dev, double *work,
                       cudaStream_t s) {
  double *Aw = work;
  double *dg = Aw + (long long)n * n;
  double *of = dg + n;
  double *refl = of + n;
  double *betas = refl + (long long)n * n;
  double *Y = betas + n;
  double *fac = Y + (long long)k * n;
  cudaMemcpyAsync(Aw, A, (size_t)n * n * sizeof(double), cudaMemcpyDeviceToDevice, s);
  cudaMemsetAsync(betas, 0, (size_t)n * sizeof(double), s);
  const size_t sm = (2 * (size_t)n + 34) * sizeof(double);
  const size_t sm_full = sm + (size_t)n * n * sizeof(double);
  if (n >= 3) {
    if (sm_full <= 200 * 1024) {
      raise_smem_limit((const void *)k_tridiag<true>, sm_full);
      k_tridiag<true><<<1, kEigThreads, sm_full, s>>>(Aw, n, dg, of, refl, betas);
    } else {
      if (sm > 48 * 1024)
        raise_smem_limit((const void *)k_tridiag<false>, sm);
      k_tridiag<false><<<1, kEigThreads, sm, s>>>(Aw, n, dg, of, refl, betas);
    }
    count_launch(1);
  } else {
    cudaMemcpyAsync(dg, Aw, sizeof(double), cudaMemcpyDeviceToDevice, s);
    if (n == 2) {
      cudaMemcpyAsync(dg + 1, Aw + 3, sizeof(double), cudaMemcpyDeviceToDevice, s);
      cudaMemcpyAsync(of, Aw + 2, sizeof(double), cudaMemcpyDeviceToDevice, s);
    }
  }
  k_bisect<<<(k + 7) / 8, 256, 0, s>>>(dg, of, n, k, evals_dev);
  k_tri_vectors<<<1, 256, 0, s>>>(dg, of, n, k, evals_dev, Y, fac);
  k_tri_backtransform<<<k, 256, (size_t)n * sizeof(double), s>>>(refl, betas, n, k, Y, evecs_dev);
  count_launch(3);
  return 0;
}

}  // namespace sbse
