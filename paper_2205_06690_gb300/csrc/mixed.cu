// Mixed hole-grid representation of the BSE operator (Sec. II.C, "Mixed Representation Iterative
// Solution"): A = Q A-bar acting on f_j(r), one grid function per occupied window state j,
//   (A-bar f)_j = (H0 + Delta - eps_j) f_j + dv phi_j - sum_i f_i W_ij,  dv = v dn,
//   dn = 2 sum_i phi_i f_i,
// Q = 1 - sum_{s <= N_occ} |phi_s><phi_s| (or the projector onto the n_c conduction states, the
// electron-hole-basis variant), and the Chebyshev recursion for the absorption spectrum. FP64.
// The kinetic part -1/2 Laplacian and dv come from the library's Poisson round trip (packed real
// fields) with the multipliers |G|^2 / 2 and 4 pi / |G|^2; this file holds the pointwise kernels,
// the projection and the reductions.
#include "gemm_nt.cuh"
#include "kernels.h"

namespace sbse {

namespace {

constexpr int kMxT = 256;

__global__ void k_exciton_density(const double *phi_o, const double *f, int n_o, long long ng, double *dn) {
  for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < ng; r += (long long)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int i = 0; i < n_o; ++i) s += phi_o[(long long)i * ng + r] * f[(long long)i * ng + r];
    dn[r] = 2.0 * s;
  }
}

// out_j = tf_j + (v + scissor - eps_j - shift) f_j + dv phi_j - sum_i f_i W_ij (W in canonical slots)
__global__ void k_abar(const double *tf, const double *f, const double *v, const double *eps_o, double scissor,
                       double shift, const double *dv, const double *phi_o, const double *W, int n_o, long long ng,
                       double *out) {
  const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y;
  if (r >= ng) return;
  const long long o = (long long)j * ng + r;
  double acc = tf[o] + (v[r] + scissor - eps_o[j] - shift) * f[o] + dv[r] * phi_o[o];
  for (int i = 0; i < n_o; ++i) {
    const int lo = i < j ? i : j, hi = i < j ? j : i;
    const int p = lo * n_o - lo * (lo - 1) / 2 + (hi - lo);
    acc -= f[(long long)i * ng + r] * W[(long long)p * ng + r];
  }
  out[o] = acc;
}

// keep == 0: out_j -= sum_s ov[j][s] basis_s; keep == 1: out_j = sum_s ov[j][s] basis_s
__global__ void k_project_apply(double *out, const double *ov, const double *basis, int n_b, long long ng, int keep) {
  const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y;
  if (r >= ng) return;
  double s = 0.0;
  for (int b = 0; b < n_b; ++b) s += ov[(long long)j * n_b + b] * basis[(long long)b * ng + r];
  const long long o = (long long)j * ng + r;
  out[o] = keep ? s : out[o] - s;
}

// out_j = x phi_j, x measured from the box centre along `axis`
__global__ void k_coord_times(const double *phi_o, long long ng, int N, double h, double box, int axis, double *out) {
  const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y;
  if (r >= ng) return;
  const long long idx = axis == 0 ? r % N : (axis == 1 ? (r / N) % N : r / ((long long)N * N));
  out[(long long)j * ng + r] = (h * (double)idx - 0.5 * box) * phi_o[(long long)j * ng + r];
}

// y = a x + b y (elementwise)
__global__ void k_axpby(double a, const double *x, double b, double *y, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = a * x[i] + b * y[i];
}

// per-block partial sums of x . y in a fixed order
constexpr int kDotBlocks = 256;
__global__ void k_dot_part(const double *x, const double *y, long long n, double *part) {
  __shared__ double red[kMxT];
  double s = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    s += x[i] * y[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

struct Rows {
  const double *p;
  long long ng;
  __device__ double operator()(int m, long long k) const { return p[(long long)m * ng + k]; }
};

}  // namespace

void launch_exciton_density(const double *phi_o, const double *f, int n_o, long long ng, double *dn, cudaStream_t s) {
  k_exciton_density<<<1024, kMxT, 0, s>>>(phi_o, f, n_o, ng, dn);
  count_launch(1);
}

void launch_abar(const double *tf, const double *f, const double *v, const double *eps_o, double scissor, double shift,
                 const double *dv, const double *phi_o, const double *W, int n_o, long long ng, double *out,
                 cudaStream_t s) {
  dim3 grid((unsigned)((ng + kMxT - 1) / kMxT), n_o);
  k_abar<<<grid, kMxT, 0, s>>>(tf, f, v, eps_o, scissor, shift, dv, phi_o, W, n_o, ng, out);
  count_launch(1);
}

size_t project_work_doubles(int n_o, int n_b, long long ng) {
  const long long kc = gemm_kchunk(ng);
  return (size_t)((ng + kc - 1) / kc) * n_o * n_b + (size_t)n_o * n_b;
}

void launch_project(double *out, int n_o, const double *basis, int n_b, long long ng, double dV, int keep,
                    double *work, cudaStream_t s) {
  const long long kc = gemm_kchunk(ng);
  const long long chunks = (ng + kc - 1) / kc;
  double *ov = work + chunks * n_o * n_b;
  dim3 g1((unsigned)chunks, (n_o + kGemmBM - 1) / kGemmBM, (n_b + kGemmBN - 1) / kGemmBN);
  k_gemm_nt_part<double><<<g1, kGemmThreads, 0, s>>>(n_o, n_b, ng, kc, Rows{out, ng}, Rows{basis, ng}, work);
  count_launch(1);
  launch_reduce_cols(work, (int)chunks, n_o * n_b, dV, ov, s);
  dim3 g2((unsigned)((ng + kMxT - 1) / kMxT), n_o);
  k_project_apply<<<g2, kMxT, 0, s>>>(out, ov, basis, n_b, ng, keep);
  count_launch(1);
}

void launch_coord_times(const double *phi_o, int n_o, int N, double h, double box, int axis, double *out,
                        cudaStream_t s) {
  const long long ng = (long long)N * N * N;
  dim3 grid((unsigned)((ng + kMxT - 1) / kMxT), n_o);
  k_coord_times<<<grid, kMxT, 0, s>>>(phi_o, ng, N, h, box, axis, out);
  count_launch(1);
}

void launch_axpby(double a, const double *x, double b, double *y, long long n, cudaStream_t s) {
  k_axpby<<<1024, kMxT, 0, s>>>(a, x, b, y, n);
  count_launch(1);
}

size_t dot_work_doubles() { return kDotBlocks; }

void launch_dot(const double *x, const double *y, long long n, double scale, double *work, double *out,
                cudaStream_t s) {
  k_dot_part<<<kDotBlocks, kMxT, 0, s>>>(x, y, n, work);
  count_launch(1);
  launch_reduce_cols(work, kDotBlocks, 1, scale, out, s);
}

}  // namespace sbse
