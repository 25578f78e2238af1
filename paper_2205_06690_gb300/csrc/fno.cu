// Fourier-neural-operator surrogate of the screened potential (the learned part of the workload;
// the paper itself has none). Inputs (rho_ij, V_loc) on the N^3 grid -> lift to C channels ->
// n_layers x [ U = K(V) + W V + b, V' = GELU(U) (no activation after the last layer) ] ->
// projection to one channel. K(V) = irfftn(R . rfftn(V) on the kept modes kx in [0, m),
// ky, kz in [0, m) U [N-m, N)). Weights used by the kernels are BF16 (spectral R and pointwise W),
// all sums are FP32; FP32 master weights and Adam moments are kept for training.
//
// Layout: activations [b][c][z][y][x] (x fastest); spectra [b][c][kz][ky][kx] (2m x 2m x m);
// spectral weights [kz][ky][kx][ci][co] complex.
#include <cuda_bf16.h>
#include <math.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "gemm_nt.cuh"
#include "kernels.h"
#include "sbse.h"

namespace sbse {
void set_thread_error(const std::string &msg);
struct CtxView {
  int N, n_occ, n_o, device;
  long long ng;
  const float *phi32;
  const double *v64;
  double *W;
  cudaStream_t stream;
};
int ctx_view(sbse_ctx *ctx, CtxView *v);
int ctx_pair_slot(sbse_ctx *ctx, int i, int j);
void ctx_mark_pair(sbse_ctx *ctx, int slot);
void ctx_set_error(sbse_ctx *ctx, const std::string &m);
bool ctx_have_pair(sbse_ctx *ctx, int slot);
int ctx_device(sbse_ctx *ctx, int *device);
}

using namespace sbse;

namespace {

constexpr int kT = 256;

__device__ __forceinline__ float gelu_f(float x) { return 0.5f * x * (1.f + erff(x * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad_f(float x) {
  return 0.5f * (1.f + erff(x * 0.70710678118654752f)) + x * expf(-0.5f * x * x) * 0.39894228040143268f;
}

// FFT index kept at position j of a full axis: 0..m-1, N-m..N-1
__device__ __forceinline__ int kept(int j, int m, int N) { return j < m ? j : N - 2 * m + j; }

// ---- truncated transforms ----------------------------------------------------------------------

// forward along x, real -> complex: out[row][kx] = sum_x in[row][x] e^{-2 pi i kx x / N}, kx < m
__global__ void k_dft_x(const float *in, float2 *out, long long rows, int N, int m, const float2 *tw) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= rows * m) return;
  const long long row = t / m;
  const int kx = (int)(t - row * m);
  const float *v = in + row * N;
  float re = 0.f, im = 0.f;
  for (int x = 0; x < N; ++x) {
    const float2 w = tw[(kx * x) % N];
    re += v[x] * w.x;
    im += v[x] * w.y;
  }
  out[t] = make_float2(re, im);
}

// along a middle axis of length n_in -> n_out, complex:
//   out[o][j][i] = sum_s in[o][s][i] * exp(sign 2 pi i f(j, s) / N)
// forward (inv = 0): s over N points, j over the 2m kept indices, f = kept(j) s
// inverse (inv = 1): s over the 2m kept indices, j over N points, f = kept(s) j
__global__ void k_dft_mid(const float2 *in, float2 *out, long long n_outer, int n_in, int n_out, int inner,
                          int N, int m, int inv, int sign, const float2 *tw) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long tot = n_outer * n_out * inner;
  if (t >= tot) return;
  const int i = (int)(t % inner);
  const long long r = t / inner;
  const int j = (int)(r % n_out);
  const long long o = r / n_out;
  const float2 *src = in + o * n_in * inner + i;
  float re = 0.f, im = 0.f;
  for (int s = 0; s < n_in; ++s) {
    const int f = inv ? kept(s, m, N) * j : kept(j, m, N) * s;
    float2 w = tw[((f % N) + N) % N];
    if (sign > 0) w.y = -w.y;
    const float2 a = src[(long long)s * inner];
    re += a.x * w.x - a.y * w.y;
    im += a.x * w.y + a.y * w.x;
  }
  out[t] = make_float2(re, im);
}

// inverse along x, complex m modes -> real: out[row][x] = scale sum_kx c_kx Re(in[row][kx] e^{+2 pi i kx x/N})
// with c_0 = 1 and c_kx = (hermitian ? 2 : 1) for kx > 0
__global__ void k_idft_x(const float2 *in, float *out, long long rows, int N, int m, int hermitian,
                         float scale, const float2 *tw) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= rows * N) return;
  const long long row = t / N;
  const int x = (int)(t - row * N);
  const float2 *a = in + row * m;
  float s = 0.f;
  for (int kx = 0; kx < m; ++kx) {
    const float2 w = tw[(kx * x) % N];  // e^{-i theta}; e^{+i theta} = conj
    const float c = (kx == 0 || !hermitian) ? 1.f : 2.f;
    s += c * (a[kx].x * w.x + a[kx].y * w.y);
  }
  out[t] = scale * s;
}

// G[b][co][mode] = sum_ci F[b][ci][mode] R[mode][ci][co]       (transpose = 0)
// dF[b][ci][mode] = sum_co conj(R[mode][ci][co]) dG[b][co][mode] (transpose = 1)
// with an optional per-kx factor on the input modes (kxscale[mode % m], null = 1)
__global__ void k_fno_mix(const float2 *in, const __nv_bfloat162 *R, float2 *out, int B, int C, int modes,
                          int m, int transpose, const float *kxscale) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)B * C * modes) return;
  const int mode = (int)(t % modes);
  const long long r = t / modes;
  const int c = (int)(r % C);
  const int b = (int)(r / C);
  const float ks = kxscale ? kxscale[mode % m] : 1.f;
  float re = 0.f, im = 0.f;
  for (int k = 0; k < C; ++k) {
    const float2 x = in[((long long)b * C + k) * modes + mode];
    const float2 w = transpose ? __bfloat1622float2(R[((long long)mode * C + c) * C + k])
                               : __bfloat1622float2(R[((long long)mode * C + k) * C + c]);
    if (transpose) {  // conj(w) x
      re += w.x * x.x + w.y * x.y;
      im += w.x * x.y - w.y * x.x;
    } else {
      re += x.x * w.x - x.y * w.y;
      im += x.x * w.y + x.y * w.x;
    }
  }
  out[t] = make_float2(ks * re, ks * im);
}

// dR[mode][ci][co] = sum_b conj(F[b][ci][mode]) dG[b][co][mode]  (written as float2 pairs)
__global__ void k_fno_dR(const float2 *F, const float2 *dG, float2 *dR, int B, int C, int modes) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)modes * C * C) return;
  const int co = (int)(t % C);
  const long long r = t / C;
  const int ci = (int)(r % C);
  const int mode = (int)(r / C);
  float re = 0.f, im = 0.f;
  for (int b = 0; b < B; ++b) {
    const float2 f = F[((long long)b * C + ci) * modes + mode];
    const float2 g = dG[((long long)b * C + co) * modes + mode];
    re += f.x * g.x + f.y * g.y;
    im += f.x * g.y - f.y * g.x;
  }
  dR[t] = make_float2(re, im);
}

// ---- pointwise parts ---------------------------------------------------------------------------

// V0[b][c][r] = sum_i Wl[c][i] x[b][i][r] + bl[c]
__global__ void k_fno_lift(const float *x, const float *Wl, const float *bl, float *V0, int B, int C,
                           long long ng) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)B * ng) return;
  const int b = (int)(t / ng);
  const long long r = t - (long long)b * ng;
  const float x0 = x[((long long)b * 2) * ng + r], x1 = x[((long long)b * 2 + 1) * ng + r];
  for (int c = 0; c < C; ++c) V0[((long long)b * C + c) * ng + r] = Wl[2 * c] * x0 + Wl[2 * c + 1] * x1 + bl[c];
}

// U[b][co][r] = S[b][co][r] + sum_ci W[co][ci] V[b][ci][r] + bias[co]; Vn = GELU(U) or U
__global__ void k_fno_pointwise(const float *S, const float *V, const __nv_bfloat16 *W, const float *bias,
                                float *U, float *Vn, int B, int C, long long ng, int act) {
  extern __shared__ float ws[];
  for (int i = threadIdx.x; i < C * C; i += blockDim.x) ws[i] = __bfloat162float(W[i]);
  __syncthreads();
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)B * ng) return;
  const int b = (int)(t / ng);
  const long long r = t - (long long)b * ng;
  float v[64];
  for (int ci = 0; ci < C; ++ci) v[ci] = V[((long long)b * C + ci) * ng + r];
  for (int co = 0; co < C; ++co) {
    float s = bias[co] + S[((long long)b * C + co) * ng + r];
    for (int ci = 0; ci < C; ++ci) s += ws[co * C + ci] * v[ci];
    const long long o = ((long long)b * C + co) * ng + r;
    U[o] = s;
    Vn[o] = act ? gelu_f(s) : s;
  }
}

// y[b][r] = sum_c w[c] V[b][c][r] + bias
__global__ void k_fno_project(const float *V, const float *w, const float *bias, float *y, int B, int C,
                              long long ng) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)B * ng) return;
  const int b = (int)(t / ng);
  const long long r = t - (long long)b * ng;
  float s = *bias;
  for (int c = 0; c < C; ++c) s += w[c] * V[((long long)b * C + c) * ng + r];
  y[t] = s;
}

// dV[b][c][r] = w[c] dy[b][r]
__global__ void k_fno_project_back(const float *dy, const float *w, float *dV, int B, int C, long long ng) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)B * C * ng) return;
  const long long r = t % ng;
  const long long bc = t / ng;
  const int c = (int)(bc % C);
  const int b = (int)(bc / C);
  dV[t] = w[c] * dy[(long long)b * ng + r];
}

// dU = dVn * GELU'(U) (or dVn), in place into dU
__global__ void k_fno_act_back(const float *dVn, const float *U, float *dU, long long n, int act) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  dU[t] = act ? dVn[t] * gelu_grad_f(U[t]) : dVn[t];
}

// dV[b][ci][r] = sum_co W[co][ci] dU[b][co][r] + dVspec[b][ci][r]
__global__ void k_fno_pointwise_back(const float *dU, const __nv_bfloat16 *W, const float *dVspec, float *dV,
                                     int B, int C, long long ng) {
  extern __shared__ float ws[];
  for (int i = threadIdx.x; i < C * C; i += blockDim.x) ws[i] = __bfloat162float(W[i]);
  __syncthreads();
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)B * ng) return;
  const int b = (int)(t / ng);
  const long long r = t - (long long)b * ng;
  float g[64];
  for (int co = 0; co < C; ++co) g[co] = dU[((long long)b * C + co) * ng + r];
  for (int ci = 0; ci < C; ++ci) {
    float s = dVspec[((long long)b * C + ci) * ng + r];
    for (int co = 0; co < C; ++co) s += ws[co * C + ci] * g[co];
    dV[((long long)b * C + ci) * ng + r] = s;
  }
}

// loss = 0.5 sum (y - t)^2 / count, dy = (y - t) / count; per-block partial losses (FP64)
__global__ void k_fno_mse(const float *y, const float *tg, float *dy, long long n, float inv_count, double *part) {
  __shared__ double red[kT];
  double s = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float d = y[i] - tg[i];
    dy[i] = d * inv_count;
    s += 0.5 * (double)d * d * inv_count;
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

// Adam: m = b1 m + (1-b1) g; v = b2 v + (1-b2) g^2; p -= lr mhat / (sqrt(vhat) + eps)
__global__ void k_adam(float *p, const float *g, float *mo, float *ve, long long n, float lr, float b1,
                       float b2, float c1, float c2, float eps) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float m = b1 * mo[i] + (1.f - b1) * gi;
  const float v = b2 * ve[i] + (1.f - b2) * gi * gi;
  mo[i] = m;
  ve[i] = v;
  p[i] -= lr * (m / c1) / (sqrtf(v / c2) + eps);
}

__global__ void k_to_bf16(const float *src, __nv_bfloat16 *dst, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = __float2bfloat16_rn(src[i]);
}

__global__ void k_d2f(const double *src, float *dst, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = (float)src[i];
}

// loaders for the split-K weight-gradient sums over (b, r): K index k = b * ng + r
struct LoadChan {  // X(row = c, k) = A[b][c][r]
  const float *A;
  int C;
  long long ng;
  __device__ float operator()(int c, long long k) const {
    const long long b = k / ng;
    return A[(b * C + c) * ng + (k - b * ng)];
  }
};
struct LoadOne {
  __device__ float operator()(int, long long) const { return 1.f; }
};

inline unsigned nblk(long long n) { return (unsigned)((n + kT - 1) / kT); }

// surrogate inputs of pairs (i, j): x[k][0] = phi_i phi_j / s_rho, x[k][1] = V_loc / s_v (FP32)
__global__ void k_pair_inputs(const float *phi, const double *v, const int2 *st, int n, long long ng,
                              float inv_rho, float inv_v, float *x) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)n * ng) return;
  const int k = (int)(t / ng);
  const long long r = t - (long long)k * ng;
  const int2 s = st[k];
  x[((long long)k * 2) * ng + r] = phi[(long long)s.x * ng + r] * phi[(long long)s.y * ng + r] * inv_rho;
  x[((long long)k * 2 + 1) * ng + r] = (float)v[r] * inv_v;
}

// W slot = s_w * y (FP32 network output -> FP64 screened potential)
__global__ void k_store_w(const float *y, double *W, long long ng, double s_w) {
  const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (r < ng) W[r] = s_w * (double)y[r];
}

// W slot += scale * y (FP32 field added to the FP64 screened potential)
__global__ void k_add_w(const float *y, double *W, long long ng, double scale) {
  const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (r < ng) W[r] += scale * (double)y[r];
}

// periodic trilinear resampling of `count` fields from an ns^3 grid onto an nd^3 grid of the same
// box (point i of the new grid sits at i ns / nd in old grid units; weights from the exact rational
// position)
__global__ void k_resample(const float *src, int ns, float *dst, int nd, long long total) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= total) return;
  const long long nd3 = (long long)nd * nd * nd, ns3 = (long long)ns * ns * ns;
  const long long fld = t / nd3;
  long long r = t - fld * nd3;
  const int ix = (int)(r % nd);
  r /= nd;
  const int iy = (int)(r % nd), iz = (int)(r / nd);
  int i0[3], i1[3];
  float w1[3];
  const int id[3] = {ix, iy, iz};
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const long long p = (long long)id[a] * ns;
    i0[a] = (int)(p / nd);
    w1[a] = (float)(p - (long long)i0[a] * nd) / (float)nd;
    i1[a] = i0[a] + 1 == ns ? 0 : i0[a] + 1;
  }
  const float *s = src + fld * ns3;
  auto at = [&](int x, int y, int z) { return s[((long long)z * ns + y) * ns + x]; };
  float acc = 0.f;
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const int bx = c & 1, by = (c >> 1) & 1, bz = c >> 2;
    const float w = (bx ? w1[0] : 1.f - w1[0]) * (by ? w1[1] : 1.f - w1[1]) * (bz ? w1[2] : 1.f - w1[2]);
    if (w != 0.f) acc += w * at(bx ? i1[0] : i0[0], by ? i1[1] : i0[1], bz ? i1[2] : i0[2]);
  }
  dst[t] = acc;
}

// a[i] *= s[i % m]: the per-kx factor c_kx / N^3 of the spectral gradient (kx is the fastest mode index)
__global__ void k_fno_scale_kx(float2 *a, long long n, int m, const float *s) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float f = s[i % m];
  a[i].x *= f;
  a[i].y *= f;
}


}  // namespace

// ================================================================================================

struct sbse_fno {
  int device = 0;
  int N = 0, C = 0, m = 0, L = 0, maxB = 0;
  long long ng = 0;
  int modes = 0;  // 4 m^3
  cudaStream_t stream = nullptr;
  std::string err;
  // parameters: FP32 master, gradient, Adam moments; BF16 copies of spectral and pointwise weights
  long long n_par = 0;
  float *par = nullptr, *grad = nullptr, *mom = nullptr, *vel = nullptr;
  __nv_bfloat16 *par16 = nullptr;
  long long off_lw = 0, off_lb = 0, off_pw = 0, off_pb = 0;
  std::vector<long long> off_spec, off_w, off_b;
  long long adam_t = 0;
  // tables and activations
  float2 *tw = nullptr;
  float *kx_herm = nullptr;  // c_kx / N^3
  float *V = nullptr, *U = nullptr, *S = nullptr, *T1 = nullptr, *dV = nullptr, *dU = nullptr;
  float2 *F = nullptr, *C1 = nullptr, *C2b = nullptr, *G = nullptr;
  float *y = nullptr, *dy = nullptr;
  double *red = nullptr, *gpart = nullptr, *gout = nullptr;
  size_t gpart_cap = 0;
};

namespace {

int fno_fail(sbse_fno *f, int code, const std::string &m) {
  f->err = m;
  return code;
}

#define FCK(call)                                                                          \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess) return fno_fail(f, SBSE_ERR_CUDA, std::string(#call) + ": " +   \
                                                                 cudaGetErrorString(e_));  \
  } while (0)

template <typename X> int falloc(sbse_fno *f, X **p, size_t bytes) {
  *p = nullptr;
  if (cudaMalloc((void **)p, bytes) != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return fno_fail(f, SBSE_ERR_OOM, "FNO device allocation failed");
  }
  return SBSE_OK;
}

// spectral transform of `rows` real rows grouped as [bc][z][y][x] -> F[bc][kz][ky][kx]
void fwd_spectrum(sbse_fno *f, const float *in, float2 *out, long long bc) {
  const int N = f->N, m = f->m;
  const long long rows = bc * N * N;
  k_dft_x<<<nblk(rows * m), kT, 0, f->stream>>>(in, f->C1, rows, N, m, f->tw);  // [bc][z][y][kx]
  // y: [bc*N (z)][N (y)][m] -> [bc*N][2m][m]
  k_dft_mid<<<nblk(bc * N * 2 * m * m), kT, 0, f->stream>>>(f->C1, f->C2b, bc * N, N, 2 * m, m, N, m, 0, -1, f->tw);
  // z: [bc][N (z)][2m*m] -> [bc][2m][2m*m]
  k_dft_mid<<<nblk(bc * 2 * m * 2 * m * m), kT, 0, f->stream>>>(f->C2b, out, bc, N, 2 * m, 2 * m * m, N, m, 0, -1,
                                                               f->tw);
  count_launch(3);
}

// inverse of the kept modes: in[bc][kz][ky][kx] -> real out[bc][z][y][x]
void inv_spectrum(sbse_fno *f, const float2 *in, float *out, long long bc, int hermitian, float scale) {
  const int N = f->N, m = f->m;
  k_dft_mid<<<nblk(bc * N * 2 * m * m), kT, 0, f->stream>>>(in, f->C2b, bc, 2 * m, N, 2 * m * m, N, m, 1, +1, f->tw);
  k_dft_mid<<<nblk(bc * N * N * m), kT, 0, f->stream>>>(f->C2b, f->C1, bc * N, 2 * m, N, m, N, m, 1, +1, f->tw);
  k_idft_x<<<nblk(bc * N * N * N), kT, 0, f->stream>>>(f->C1, out, bc * N * N, N, m, hermitian, scale, f->tw);
  count_launch(3);
}

float *Vl(sbse_fno *f, int l, int B) { return f->V + (long long)l * B * f->C * f->ng; }
float *Ul(sbse_fno *f, int l, int B) { return f->U + (long long)l * B * f->C * f->ng; }
float2 *Fl(sbse_fno *f, int l, int B) { return f->F + (long long)l * B * f->C * f->modes; }

void forward_impl(sbse_fno *f, int B, const float *x) {
  const int C = f->C;
  const long long ng = f->ng;
  const float *par = f->par;
  k_fno_lift<<<nblk(B * ng), kT, 0, f->stream>>>(x, par + f->off_lw, par + f->off_lb, Vl(f, 0, B), B, C, ng);
  count_launch(1);
  const __nv_bfloat162 *R16;
  for (int l = 0; l < f->L; ++l) {
    fwd_spectrum(f, Vl(f, l, B), Fl(f, l, B), (long long)B * C);
    R16 = reinterpret_cast<const __nv_bfloat162 *>(f->par16 + f->off_spec[l]);
    k_fno_mix<<<nblk((long long)B * C * f->modes), kT, 0, f->stream>>>(Fl(f, l, B), R16, f->G, B, C, f->modes, f->m,
                                                                       0, nullptr);
    count_launch(1);
    inv_spectrum(f, f->G, f->S, (long long)B * C, 1, 1.f / (float)(ng));
    k_fno_pointwise<<<nblk(B * ng), kT, C * C * sizeof(float), f->stream>>>(
        f->S, Vl(f, l, B), f->par16 + f->off_w[l], par + f->off_b[l], Ul(f, l, B), Vl(f, l + 1, B), B, C, ng,
        l < f->L - 1 ? 1 : 0);
    count_launch(1);
  }
  k_fno_project<<<nblk(B * ng), kT, 0, f->stream>>>(Vl(f, f->L, B), par + f->off_pw, par + f->off_pb, f->y, B,
                                                    C, ng);
  count_launch(1);
}

// weight gradient: out[M][Nn] = sum_{b,r} A[b][row][r] Bm[b][col][r]  (Bm = null: ones)
int wgrad(sbse_fno *f, const float *A, int M, const float *Bm, int Nn, int B, float *out) {
  const long long K = (long long)B * f->ng;
  const long long kc = gemm_kchunk(K);
  const long long chunks = (K + kc - 1) / kc;
  const size_t need = (size_t)chunks * M * Nn * sizeof(double);
  if (need > f->gpart_cap) {
    if (f->gpart) cudaFree(f->gpart);
    f->gpart = nullptr;
    f->gpart_cap = 0;
    int rc = falloc(f, &f->gpart, need);
    if (rc) return rc;
    f->gpart_cap = need;
  }
  dim3 grid((unsigned)chunks, (M + kGemmBM - 1) / kGemmBM, (Nn + kGemmBN - 1) / kGemmBN);
  if (Bm)
    k_gemm_nt_part<float><<<grid, kGemmThreads, 0, f->stream>>>(M, Nn, K, kc, LoadChan{A, M, f->ng},
                                                                LoadChan{Bm, Nn, f->ng}, f->gpart);
  else
    k_gemm_nt_part<float><<<grid, kGemmThreads, 0, f->stream>>>(M, Nn, K, kc, LoadChan{A, M, f->ng}, LoadOne{},
                                                                f->gpart);
  count_launch(1);
  launch_reduce_cols(f->gpart, (int)chunks, M * Nn, 1.0, f->gout, f->stream);
  k_d2f<<<nblk((long long)M * Nn), kT, 0, f->stream>>>(f->gout, out, (long long)M * Nn);
  count_launch(1);
  return SBSE_OK;
}

// backward from dL/dy (in f->dy); fills f->grad (and dL/dx into dx when given)
int backward_impl(sbse_fno *f, int B, const float *x) {
  const int C = f->C, L = f->L;
  const long long ng = f->ng, n_act = (long long)B * C * ng;
  int rc;
  // projection
  if ((rc = wgrad(f, Vl(f, L, B), C, f->dy, 1, B, f->grad + f->off_pw))) return rc;
  if ((rc = wgrad(f, f->dy, 1, nullptr, 1, B, f->grad + f->off_pb))) return rc;
  k_fno_project_back<<<nblk(n_act), kT, 0, f->stream>>>(f->dy, f->par + f->off_pw, f->dV, B, C, ng);
  count_launch(1);
  for (int l = L - 1; l >= 0; --l) {
    k_fno_act_back<<<nblk(n_act), kT, 0, f->stream>>>(f->dV, Ul(f, l, B), f->dU, n_act, l < L - 1 ? 1 : 0);
    count_launch(1);
    if ((rc = wgrad(f, f->dU, C, Vl(f, l, B), C, B, f->grad + f->off_w[l]))) return rc;
    if ((rc = wgrad(f, f->dU, C, nullptr, 1, B, f->grad + f->off_b[l]))) return rc;
    // spectral: dG = c_kx / N^3 rfft(dU) on the kept modes (scaled inside the mix kernel input)
    fwd_spectrum(f, f->dU, f->G, (long long)B * C);
    {  // dG *= c_kx / N^3
      const long long n = (long long)B * C * f->modes;
      k_fno_scale_kx<<<nblk(n), kT, 0, f->stream>>>(f->G, n, f->m, f->kx_herm);
      count_launch(1);
    }
    // dR[mode][ci][co] = sum_b conj(F[b][ci]) dG[b][co]
    k_fno_dR<<<nblk((long long)f->modes * C * C), kT, 0, f->stream>>>(Fl(f, l, B), f->G,
                                                                      reinterpret_cast<float2 *>(f->grad + f->off_spec[l]),
                                                                      B, C, f->modes);
    count_launch(1);
    const __nv_bfloat162 *R16 = reinterpret_cast<const __nv_bfloat162 *>(f->par16 + f->off_spec[l]);
    k_fno_mix<<<nblk((long long)B * C * f->modes), kT, 0, f->stream>>>(f->G, R16, reinterpret_cast<float2 *>(f->T1),
                                                                       B, C, f->modes, f->m, 1, nullptr);
    count_launch(1);
    // dV_spec = Re sum_k dF_k e^{+i k.r} (no Hermitian doubling, no 1/N^3)
    inv_spectrum(f, reinterpret_cast<float2 *>(f->T1), f->S, (long long)B * C, 0, 1.f);
    k_fno_pointwise_back<<<nblk(B * ng), kT, C * C * sizeof(float), f->stream>>>(
        f->dU, f->par16 + f->off_w[l], f->S, f->dV, B, C, ng);
    count_launch(1);
  }
  if ((rc = wgrad(f, f->dV, C, x, 2, B, f->grad + f->off_lw))) return rc;
  if ((rc = wgrad(f, f->dV, C, nullptr, 1, B, f->grad + f->off_lb))) return rc;
  return SBSE_OK;
}

void refresh_bf16(sbse_fno *f) {
  k_to_bf16<<<nblk(f->n_par), kT, 0, f->stream>>>(f->par, f->par16, f->n_par);
  count_launch(1);
}

}  // namespace

// ================================================================================================
extern "C" {

int sbse_fno_create(sbse_fno **out, int device, int n, int width, int modes, int layers, int max_batch) {
  if (!out) return SBSE_ERR_INVALID_ARG;
  *out = nullptr;
  if (n < 4 || width < 1 || width > 64 || modes < 1 || 2 * modes > n || layers < 1 || max_batch < 1) {
    sbse::set_thread_error("FNO: need n >= 4, 1 <= width <= 64, 1 <= 2 modes <= n, layers >= 1, batch >= 1");
    return SBSE_ERR_INVALID_ARG;
  }
  sbse_fno *f = new sbse_fno();
  f->device = device;
  f->N = n;
  f->C = width;
  f->m = modes;
  f->L = layers;
  f->maxB = max_batch;
  f->ng = (long long)n * n * n;
  f->modes = 4 * modes * modes * modes;
  if (cudaSetDevice(device) != cudaSuccess || cudaStreamCreateWithFlags(&f->stream, cudaStreamNonBlocking) != cudaSuccess) {
    sbse::set_thread_error("FNO: CUDA setup failed");
    delete f;
    return SBSE_ERR_CUDA;
  }
  // parameter layout
  long long o = 0;
  f->off_lw = o;
  o += 2LL * width;
  f->off_lb = o;
  o += width;
  for (int l = 0; l < layers; ++l) {
    f->off_spec.push_back(o);
    o += 2LL * f->modes * width * width;
    f->off_w.push_back(o);
    o += (long long)width * width;
    f->off_b.push_back(o);
    o += width;
  }
  f->off_pw = o;
  o += width;
  f->off_pb = o;
  o += 1;
  f->n_par = o;
  const long long B = max_batch, act = B * width * f->ng;
  int rc = 0;
  rc = rc ? rc : falloc(f, &f->par, f->n_par * sizeof(float));
  rc = rc ? rc : falloc(f, &f->grad, f->n_par * sizeof(float));
  rc = rc ? rc : falloc(f, &f->mom, f->n_par * sizeof(float));
  rc = rc ? rc : falloc(f, &f->vel, f->n_par * sizeof(float));
  rc = rc ? rc : falloc(f, &f->par16, f->n_par * sizeof(__nv_bfloat16));
  rc = rc ? rc : falloc(f, &f->tw, n * sizeof(float2));
  rc = rc ? rc : falloc(f, &f->kx_herm, modes * sizeof(float));
  rc = rc ? rc : falloc(f, &f->V, (layers + 1) * act * sizeof(float));
  rc = rc ? rc : falloc(f, &f->U, layers * act * sizeof(float));
  rc = rc ? rc : falloc(f, &f->S, act * sizeof(float));
  rc = rc ? rc : falloc(f, &f->T1, act * sizeof(float));
  rc = rc ? rc : falloc(f, &f->dV, act * sizeof(float));
  rc = rc ? rc : falloc(f, &f->dU, act * sizeof(float));
  rc = rc ? rc : falloc(f, &f->F, (size_t)layers * B * width * f->modes * sizeof(float2));
  rc = rc ? rc : falloc(f, &f->G, (size_t)B * width * f->modes * sizeof(float2));
  rc = rc ? rc : falloc(f, &f->C1, (size_t)B * width * n * n * modes * sizeof(float2) + 64);
  rc = rc ? rc : falloc(f, &f->C2b, (size_t)B * width * n * 2 * modes * modes * sizeof(float2) + 64);
  rc = rc ? rc : falloc(f, &f->y, B * f->ng * sizeof(float));
  rc = rc ? rc : falloc(f, &f->dy, B * f->ng * sizeof(float));
  rc = rc ? rc : falloc(f, &f->red, 4096 * sizeof(double));
  rc = rc ? rc : falloc(f, &f->gout, ((size_t)width * width + 64) * sizeof(double));
  if (rc) {
    sbse::set_thread_error(f->err);
    sbse_fno_destroy(f);
    return rc;
  }
  std::vector<float2> tw(n);
  for (int k = 0; k < n; ++k) {
    const double a = -2.0 * M_PI * k / n;
    tw[k] = make_float2((float)cos(a), (float)sin(a));
  }
  std::vector<float> kh(modes);
  for (int k = 0; k < modes; ++k) kh[k] = (k == 0 ? 1.f : 2.f) / (float)f->ng;
  cudaMemcpy(f->tw, tw.data(), n * sizeof(float2), cudaMemcpyHostToDevice);
  cudaMemcpy(f->kx_herm, kh.data(), modes * sizeof(float), cudaMemcpyHostToDevice);
  cudaMemset(f->par, 0, f->n_par * sizeof(float));
  cudaMemset(f->mom, 0, f->n_par * sizeof(float));
  cudaMemset(f->vel, 0, f->n_par * sizeof(float));
  *out = f;
  return SBSE_OK;
}

void sbse_fno_destroy(sbse_fno *f) {
  if (!f) return;
  cudaSetDevice(f->device);
  if (f->stream) cudaStreamSynchronize(f->stream);
  void *ptrs[] = {f->par, f->grad, f->mom, f->vel, f->par16, f->tw, f->kx_herm, f->V, f->U, f->S, f->T1, f->dV,
                  f->dU, f->F, f->G, f->C1, f->C2b, f->y, f->dy, f->red, f->gpart, f->gout};
  for (void *p : ptrs)
    if (p) cudaFree(p);
  if (f->stream) cudaStreamDestroy(f->stream);
  delete f;
}

const char *sbse_fno_last_error(const sbse_fno *f) { return f ? f->err.c_str() : ""; }

long long sbse_fno_num_params(const sbse_fno *f) { return f ? f->n_par : 0; }

int sbse_fno_set_params(sbse_fno *f, const float *host) {
  if (!f || !host) return SBSE_ERR_INVALID_ARG;
  FCK(cudaSetDevice(f->device));
  FCK(cudaMemcpyAsync(f->par, host, f->n_par * sizeof(float), cudaMemcpyHostToDevice, f->stream));
  refresh_bf16(f);
  FCK(cudaStreamSynchronize(f->stream));
  f->adam_t = 0;
  FCK(cudaMemset(f->mom, 0, f->n_par * sizeof(float)));
  FCK(cudaMemset(f->vel, 0, f->n_par * sizeof(float)));
  return SBSE_OK;
}

int sbse_fno_get_params(sbse_fno *f, float *host, float *grad_host) {
  if (!f || (!host && !grad_host)) return SBSE_ERR_INVALID_ARG;
  FCK(cudaSetDevice(f->device));
  if (host) FCK(cudaMemcpy(host, f->par, f->n_par * sizeof(float), cudaMemcpyDeviceToHost));
  if (grad_host) FCK(cudaMemcpy(grad_host, f->grad, f->n_par * sizeof(float), cudaMemcpyDeviceToHost));
  return SBSE_OK;
}

int sbse_fno_forward(sbse_fno *f, int batch, const float *x_dev, float *y_dev) {
  if (!f || !x_dev || !y_dev || batch < 1 || batch > f->maxB) return SBSE_ERR_INVALID_ARG;
  FCK(cudaSetDevice(f->device));
  forward_impl(f, batch, x_dev);
  FCK(cudaMemcpyAsync(y_dev, f->y, (size_t)batch * f->ng * sizeof(float), cudaMemcpyDeviceToDevice, f->stream));
  FCK(cudaGetLastError());
  FCK(cudaStreamSynchronize(f->stream));
  return SBSE_OK;
}

int sbse_fno_gradients(sbse_fno *f, int batch, const float *x_dev, const float *dy_dev) {
  if (!f || !x_dev || !dy_dev || batch < 1 || batch > f->maxB) return SBSE_ERR_INVALID_ARG;
  FCK(cudaSetDevice(f->device));
  forward_impl(f, batch, x_dev);
  FCK(cudaMemcpyAsync(f->dy, dy_dev, (size_t)batch * f->ng * sizeof(float), cudaMemcpyDeviceToDevice, f->stream));
  int rc = backward_impl(f, batch, x_dev);
  if (rc) return rc;
  FCK(cudaGetLastError());
  FCK(cudaStreamSynchronize(f->stream));
  return SBSE_OK;
}

int sbse_fno_train_step(sbse_fno *f, int batch, const float *x_dev, const float *t_dev, float lr, double *loss) {
  if (!f || !x_dev || !t_dev || batch < 1 || batch > f->maxB || !(lr > 0.f)) return SBSE_ERR_INVALID_ARG;
  FCK(cudaSetDevice(f->device));
  forward_impl(f, batch, x_dev);
  const long long n = (long long)batch * f->ng;
  const int blocks = 1024;
  k_fno_mse<<<blocks, kT, 0, f->stream>>>(f->y, t_dev, f->dy, n, 1.f / (float)n, f->red);
  count_launch(1);
  int rc = backward_impl(f, batch, x_dev);
  if (rc) return rc;
  f->adam_t += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - powf(b1, (float)f->adam_t), c2 = 1.f - powf(b2, (float)f->adam_t);
  k_adam<<<nblk(f->n_par), kT, 0, f->stream>>>(f->par, f->grad, f->mom, f->vel, f->n_par, lr, b1, b2, c1, c2, 1e-8f);
  count_launch(1);
  refresh_bf16(f);
  if (loss) {
    std::vector<double> h(blocks);
    FCK(cudaMemcpyAsync(h.data(), f->red, blocks * sizeof(double), cudaMemcpyDeviceToHost, f->stream));
    FCK(cudaStreamSynchronize(f->stream));
    double s = 0.0;
    for (double v : h) s += v;
    *loss = s;
  }
  FCK(cudaGetLastError());
  FCK(cudaStreamSynchronize(f->stream));
  return SBSE_OK;
}

int sbse_fno_pair_inputs(sbse_ctx *ctx, int n_pairs, const int *pi, const int *pj, double s_rho, double s_v,
                         float *x_dev) {
  sbse::CtxView cv;
  if (sbse::ctx_view(ctx, &cv) != SBSE_OK) return SBSE_ERR_NOT_READY;
  if (!pi || !pj || !x_dev || n_pairs < 1 || !(s_rho > 0) || !(s_v > 0)) return SBSE_ERR_INVALID_ARG;
  std::vector<int2> st(n_pairs);
  const int base = cv.n_occ - cv.n_o;
  for (int k = 0; k < n_pairs; ++k) {
    if (pi[k] < 0 || pj[k] < pi[k] || pj[k] >= cv.n_o) return SBSE_ERR_INVALID_ARG;
    st[k] = make_int2(base + pi[k], base + pj[k]);
  }
  int2 *sd = nullptr;
  if (cudaSetDevice(cv.device) != cudaSuccess || cudaMallocAsync((void **)&sd, n_pairs * sizeof(int2), cv.stream) != cudaSuccess)
    return SBSE_ERR_CUDA;
  cudaMemcpyAsync(sd, st.data(), n_pairs * sizeof(int2), cudaMemcpyHostToDevice, cv.stream);
  k_pair_inputs<<<nblk((long long)n_pairs * cv.ng), kT, 0, cv.stream>>>(cv.phi32, cv.v64, sd, n_pairs, cv.ng,
                                                                        (float)(1.0 / s_rho), (float)(1.0 / s_v),
                                                                        x_dev);
  count_launch(1);
  cudaFreeAsync(sd, cv.stream);
  const cudaError_t e = cudaStreamSynchronize(cv.stream);
  return e == cudaSuccess ? SBSE_OK : SBSE_ERR_CUDA;
}

int sbse_surrogate_W(sbse_ctx *ctx, sbse_fno *f, int n_pairs, const int *pi, const int *pj, double s_rho,
                     double s_v, double s_w) {
  sbse::CtxView cv;
  if (sbse::ctx_view(ctx, &cv) != SBSE_OK) return SBSE_ERR_NOT_READY;
  if (!f || !pi || !pj || n_pairs < 1) return SBSE_ERR_INVALID_ARG;
  if (f->N != cv.N) {
    sbse::ctx_set_error(ctx, "surrogate grid differs from the context grid");
    return SBSE_ERR_SHAPE;
  }
  FCK(cudaSetDevice(f->device));
  float *x = nullptr, *y = nullptr;
  const int bmax = f->maxB;
  FCK(cudaMallocAsync((void **)&x, (size_t)bmax * 2 * f->ng * sizeof(float), f->stream));
  FCK(cudaMallocAsync((void **)&y, (size_t)bmax * f->ng * sizeof(float), f->stream));
  FCK(cudaStreamSynchronize(f->stream));
  int rc = SBSE_OK;
  for (int k0 = 0; k0 < n_pairs && rc == SBSE_OK; k0 += bmax) {
    const int nb = (n_pairs - k0) < bmax ? (n_pairs - k0) : bmax;
    rc = sbse_fno_pair_inputs(ctx, nb, pi + k0, pj + k0, s_rho, s_v, x);
    if (rc) break;
    forward_impl(f, nb, x);
    for (int k = 0; k < nb; ++k) {
      const int slot = sbse::ctx_pair_slot(ctx, pi[k0 + k], pj[k0 + k]);
      k_store_w<<<nblk(f->ng), kT, 0, f->stream>>>(f->y + (long long)k * f->ng, cv.W + (long long)slot * f->ng,
                                                  f->ng, s_w);
      count_launch(1);
      sbse::ctx_mark_pair(ctx, slot);
    }
    if (cudaStreamSynchronize(f->stream) != cudaSuccess) rc = SBSE_ERR_CUDA;
  }
  cudaFreeAsync(x, f->stream);
  cudaFreeAsync(y, f->stream);
  cudaStreamSynchronize(f->stream);
  return rc;
}

int sbse_add_W(sbse_ctx *ctx, int n_pairs, const int *pi, const int *pj, const float *y_dev, double scale) {
  sbse::CtxView cv;
  if (sbse::ctx_view(ctx, &cv) != SBSE_OK) return SBSE_ERR_NOT_READY;
  if (!pi || !pj || !y_dev || n_pairs < 1 || !isfinite(scale)) return SBSE_ERR_INVALID_ARG;
  std::vector<int> slots(n_pairs);
  for (int k = 0; k < n_pairs; ++k) {
    if (pi[k] < 0 || pj[k] < pi[k] || pj[k] >= cv.n_o) return SBSE_ERR_INVALID_ARG;
    slots[k] = sbse::ctx_pair_slot(ctx, pi[k], pj[k]);
    if (!sbse::ctx_have_pair(ctx, slots[k])) {
      sbse::ctx_set_error(ctx, "sbse_add_W: W of a pair is not available (sbse_bare_W or sbse_apply_W first)");
      return SBSE_ERR_NOT_READY;
    }
  }
  if (cudaSetDevice(cv.device) != cudaSuccess) return SBSE_ERR_CUDA;
  for (int k = 0; k < n_pairs; ++k) {
    k_add_w<<<nblk(cv.ng), kT, 0, cv.stream>>>(y_dev + (long long)k * cv.ng, cv.W + (long long)slots[k] * cv.ng,
                                               cv.ng, scale);
    count_launch(1);
    sbse::ctx_mark_pair(ctx, slots[k]);
  }
  return cudaStreamSynchronize(cv.stream) == cudaSuccess ? SBSE_OK : SBSE_ERR_CUDA;
}

int sbse_resample(sbse_ctx *ctx, int count, int n_src, const float *src_dev, int n_dst, float *dst_dev) {
  if (!ctx || count < 1 || n_src < 1 || n_dst < 1 || !src_dev || !dst_dev || src_dev == dst_dev)
    return SBSE_ERR_INVALID_ARG;
  int device = 0;
  cudaStream_t st = nullptr;
  if (sbse_get_stream(ctx, (void **)&st) != SBSE_OK || sbse::ctx_device(ctx, &device) != SBSE_OK)
    return SBSE_ERR_INVALID_ARG;
  if (cudaSetDevice(device) != cudaSuccess) return SBSE_ERR_CUDA;
  const long long total = (long long)count * n_dst * n_dst * n_dst;
  k_resample<<<nblk(total), kT, 0, st>>>(src_dev, n_src, dst_dev, n_dst, total);
  count_launch(1);
  return cudaStreamSynchronize(st) == cudaSuccess ? SBSE_OK : SBSE_ERR_CUDA;
}

}  // extern "C"
