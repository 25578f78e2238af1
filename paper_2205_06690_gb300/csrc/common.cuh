// Shared device helpers of the sbse library: complex arithmetic, FFT plans and the in-shared-memory
// Stockham FFT used by every grid pass.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace sbse {

template <typename T> struct Vec2;
template <> struct Vec2<float> { using type = float2; };
template <> struct Vec2<double> { using type = double2; };
template <typename T> using C2 = typename Vec2<T>::type;

template <typename C> __device__ __forceinline__ C cadd(C a, C b) { return C{a.x + b.x, a.y + b.y}; }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { return C{a.x - b.x, a.y - b.y}; }
// FP32 complex sums as one packed two-lane instruction (add / sub .f32x2, sm_100 and later): the
// same IEEE round-to-nearest results as two scalar instructions, half the issue slots
#if defined(__CUDA_ARCH__) && __CUDA_ARCH__ >= 1000
__device__ __forceinline__ float2 cadd(float2 a, float2 b) {
  float2 r;
  asm("{\n\t.reg .b64 pa, pb, pr;\n\tmov.b64 pa, {%2, %3};\n\tmov.b64 pb, {%4, %5};\n\t"
      "add.rn.f32x2 pr, pa, pb;\n\tmov.b64 {%0, %1}, pr;\n\t}"
      : "=f"(r.x), "=f"(r.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return r;
}
__device__ __forceinline__ float2 csub(float2 a, float2 b) {
  float2 r;
  asm("{\n\t.reg .b64 pa, pb, pr;\n\tmov.b64 pa, {%2, %3};\n\tmov.b64 pb, {%4, %5};\n\t"
      "sub.rn.f32x2 pr, pa, pb;\n\tmov.b64 {%0, %1}, pr;\n\t}"
      : "=f"(r.x), "=f"(r.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return r;
}
#endif
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
  return C{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
// a b + c e as fused multiply-adds (four per component), for sums of two complex products
template <typename C> __device__ __forceinline__ C cmac2(C a, C b, C c, C e) {
  return C{fma(a.x, b.x, fma(-a.y, b.y, fma(c.x, e.x, -c.y * e.y))),
           fma(a.x, b.y, fma(a.y, b.x, fma(c.x, e.y, c.y * e.x)))};
}
template <typename C> __device__ __forceinline__ C cconj(C a) { return C{a.x, -a.y}; }
// s * i * a for s = +-1
template <typename C> __device__ __forceinline__ C cmul_si(C a, int s) {
  return s > 0 ? C{-a.y, a.x} : C{a.y, -a.x};
}
template <typename C, typename T> __device__ __forceinline__ C cscale(C a, T s) { return C{a.x * s, a.y * s}; }

__device__ __forceinline__ void sincos_t(float x, float *s, float *c) { sincosf(x, s, c); }
__device__ __forceinline__ void sincos_t(double x, double *s, double *c) { sincos(x, s, c); }

// Largest supported grid edge. Every FFT runs on one pencil held in shared memory.
constexpr int kMaxN = 128;
constexpr int kMaxStages = 8;

// Mixed-radix plan N = prod radix[k], radices in {4, 2, 3, 5}, applied in order.
struct FftPlan {
  int n;
  int nst;
  int radix[kMaxStages];
};

// Batched in-shared-memory Stockham FFT over TP pencils of length N.
// Layout: element e of pencil p at buf[e * ld + p]. Ping-pongs between A and B; returns the
// buffer that holds the result. tw[k] = exp(-2 pi i k / N) (computed on the host in FP64).
// sign = -1: forward (exp(-2 pi i ...)), +1: inverse, unnormalised.
// All threads of the block must call it; it ends with __syncthreads().
template <typename T>
__device__ C2<T> *fft_tile(C2<T> *A, C2<T> *B, const C2<T> *tw, const FftPlan &pl, int TP, int ld,
                           int sign) {
  using C = C2<T>;
  const int N = pl.n;
  int Ns = 1;
  for (int st = 0; st < pl.nst; ++st) {
    const int R = pl.radix[st];
    const int nb = N / R;
    const int tot = nb * TP;
    const int tstride = N / (Ns * R);
    for (int b = threadIdx.x; b < tot; b += blockDim.x) {
      const int p = b % TP;
      const int j = b / TP;
      const int jm = j % Ns;
      C v[5];
#pragma unroll
      for (int r = 0; r < 5; ++r)
        if (r < R) v[r] = A[(j + r * nb) * ld + p];
      if (jm != 0) {
        const int ts = jm * tstride;
#pragma unroll
        for (int r = 1; r < 5; ++r)
          if (r < R) {
            C w = tw[(r * ts) % N];
            if (sign > 0) w = cconj(w);
            v[r] = cmul(v[r], w);
          }
      }
      C o[5];
      if (R == 4) {
        C s02 = cadd(v[0], v[2]), d02 = csub(v[0], v[2]);
        C s13 = cadd(v[1], v[3]), d13 = cmul_si(csub(v[1], v[3]), sign);
        o[0] = cadd(s02, s13);
        o[2] = csub(s02, s13);
        o[1] = cadd(d02, d13);
        o[3] = csub(d02, d13);
      } else if (R == 2) {
        o[0] = cadd(v[0], v[1]);
        o[1] = csub(v[0], v[1]);
      } else if (R == 3) {
        // X1,2 = x0 - (x1 + x2)/2 +- s i sin(2 pi/3) (x1 - x2); sin(2 pi / 3) = -Im tw[N/3]
        const T s3 = -tw[N / 3].y;
        C t = cadd(v[1], v[2]);
        C m = C{v[0].x - T(0.5) * t.x, v[0].y - T(0.5) * t.y};
        C d = cmul_si(cscale(csub(v[1], v[2]), s3), sign);
        o[0] = cadd(v[0], t);
        o[1] = cadd(m, d);
        o[2] = csub(m, d);
      } else {  // R == 5, constants cos/sin(2 pi k / 5) from the twiddle table
        const T c1 = tw[N / 5].x, s1 = -tw[N / 5].y;
        const T c2 = tw[2 * (N / 5)].x, s2 = -tw[2 * (N / 5)].y;
        C a1 = cadd(v[1], v[4]), a2 = cadd(v[2], v[3]);
        C b1 = csub(v[1], v[4]), b2 = csub(v[2], v[3]);
        C r1 = C{v[0].x + c1 * a1.x + c2 * a2.x, v[0].y + c1 * a1.y + c2 * a2.y};
        C r2 = C{v[0].x + c2 * a1.x + c1 * a2.x, v[0].y + c2 * a1.y + c1 * a2.y};
        C i1 = cmul_si(C{s1 * b1.x + s2 * b2.x, s1 * b1.y + s2 * b2.y}, sign);
        C i2 = cmul_si(C{s2 * b1.x - s1 * b2.x, s2 * b1.y - s1 * b2.y}, sign);
        o[0] = C{v[0].x + a1.x + a2.x, v[0].y + a1.y + a2.y};
        o[1] = cadd(r1, i1);
        o[4] = csub(r1, i1);
        o[2] = cadd(r2, i2);
        o[3] = csub(r2, i2);
      }
      const int idxD = (j / Ns) * Ns * R + jm;
#pragma unroll
      for (int r = 0; r < 5; ++r)
        if (r < R) B[(idxD + r * Ns) * ld + p] = o[r];
    }
    __syncthreads();
    C *t = A;
    A = B;
    B = t;
    Ns *= R;
  }
  return A;
}

}  // namespace sbse
