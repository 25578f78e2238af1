// Finite-box correction W(k -> 0) = eps_eff^-1 v_bndry of Sec. III (the paragraph before the
// algorithm summary): the average Kohn-Sham potential on the box boundary of a run, and the fit of
// eps_eff^-1 that makes the exciton spectra of runs in several box sizes overlap.
//
// Readings: the model's Kohn-Sham potential is V_loc - mean(V_loc) + v n0 with n0 = 2 sum_s |phi_s|^2
// over the occupied states (spin factor of Eq. 11) and v the periodic Coulomb operator with G = 0
// dropped (the zero-average convention of a periodic calculation); the boundary of the periodic box
// is the set of grid points with ix = 0, iy = 0 or iz = 0; "overlap" is least squares (see
// fit_inverse_dielectric below).
#include "kernels.h"

namespace sbse {

namespace {

constexpr int kFbBlocks = 256, kFbThreads = 256;

// n0(r) = 2 sum_s phi_s(r)^2, FP64
__global__ void k_ground_density(const double *phi, int n_occ, long long ng, double *n0) {
  for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < ng; r += (long long)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int s = 0; s < n_occ; ++s) {
      const double p = phi[(long long)s * ng + r];
      acc += p * p;
    }
    n0[r] = 2.0 * acc;
  }
}

// per-block partial sums: part[b][0] = sum over all points of v, part[b][1] = sum over the boundary
// points of v + u (fixed block count and order: the result does not depend on scheduling)
__global__ void k_box_sums(const double *v, const double *u, int N, double *part) {
  __shared__ double red[2][kFbThreads];
  const long long ng = (long long)N * N * N;
  const long long nb = 3LL * N * N - 3LL * N + 1;
  double s_all = 0.0, s_bnd = 0.0;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < ng; r += stride) s_all += v[r];
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < nb; t += stride) {
    // boundary point t: first the plane z = 0 (N^2), then y = 0 with z > 0 (N (N - 1)), then x = 0
    // with y, z > 0 ((N - 1)^2)
    long long x, y, z;
    const long long NN = (long long)N * N;
    if (t < NN) {
      z = 0; y = t / N; x = t % N;
    } else if (t < NN + (long long)N * (N - 1)) {
      const long long q = t - NN;
      y = 0; z = 1 + q / N; x = q % N;
    } else {
      const long long q = t - NN - (long long)N * (N - 1);
      x = 0; z = 1 + q / (N - 1); y = 1 + q % (N - 1);
    }
    const long long r = (z * N + y) * N + x;
    s_bnd += v[r] + u[r];
  }
  red[0][threadIdx.x] = s_all;
  red[1][threadIdx.x] = s_bnd;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      red[0][threadIdx.x] += red[0][threadIdx.x + w];
      red[1][threadIdx.x] += red[1][threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[blockIdx.x * 2] = red[0][0];
    part[blockIdx.x * 2 + 1] = red[1][0];
  }
}

}  // namespace

size_t boundary_work_doubles(long long ng) { return (size_t)ng + 2 * kFbBlocks + 2; }

void launch_ground_density(const double *phi, int n_occ, long long ng, double *n0, cudaStream_t s) {
  k_ground_density<<<kFbBlocks * 4, kFbThreads, 0, s>>>(phi, n_occ, ng, n0);
  count_launch(1);
}

void launch_box_sums(const double *v, const double *u, int N, double *work, double *sums, cudaStream_t s) {
  k_box_sums<<<kFbBlocks, kFbThreads, 0, s>>>(v, u, N, work);
  launch_reduce_cols(work, kFbBlocks, 2, 1.0, sums, s);
  count_launch(1);
}

}  // namespace sbse
