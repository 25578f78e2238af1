// Register-resident FFT of one pencil of compile-time length N (one thread per pencil).
// Mixed-radix Stockham stages (radices 4, then 2, 3, 5) fully unrolled, so every index and every
// twiddle index is a compile-time constant; the twiddles exp(-2 pi i k / N) are read from a
// __constant__ table that the host fills from FP64 cos/sin. The table is reached through a
// provider type TW (static get(i) returning entry i of the layout below), so that every
// translation unit can keep its own copy of the table.
#pragma once

#include "common.cuh"

namespace sbse {

// Sizes with a register FFT, and the offset of each size's twiddle table.
constexpr int kRegSizes[] = {8, 10, 12, 16, 20, 24, 32, 40, 48, 64, 80, 96};
constexpr int kRegCount = sizeof(kRegSizes) / sizeof(int);
constexpr int reg_offset(int N) {
  int o = 0;
  for (int i = 0; i < kRegCount; ++i) {
    if (kRegSizes[i] == N) return o;
    o += kRegSizes[i];
  }
  return -1;
}
constexpr int kRegTotal = reg_offset(96) + 96;

constexpr int stage_radix(int N, int st) {
  int m = N, s = 0;
  while (m % 4 == 0) {
    if (s == st) return 4;
    m /= 4;
    ++s;
  }
  while (m % 2 == 0) {
    if (s == st) return 2;
    m /= 2;
    ++s;
  }
  while (m % 3 == 0) {
    if (s == st) return 3;
    m /= 3;
    ++s;
  }
  while (m % 5 == 0) {
    if (s == st) return 5;
    m /= 5;
    ++s;
  }
  return 0;
}

template <typename T> struct TwTab;

template <typename T, int R, int SIGN, typename TW = TwTab<T>>
__device__ __forceinline__ void dft_small(C2<T> (&x)[R], int off, int N) {
  using C = C2<T>;
  if constexpr (R == 2) {
    C a = cadd(x[0], x[1]);
    x[1] = csub(x[0], x[1]);
    x[0] = a;
  } else if constexpr (R == 4) {
    C s02 = cadd(x[0], x[2]), d02 = csub(x[0], x[2]);
    C s13 = cadd(x[1], x[3]), d13 = cmul_si(csub(x[1], x[3]), SIGN);
    x[0] = cadd(s02, s13);
    x[2] = csub(s02, s13);
    x[1] = cadd(d02, d13);
    x[3] = csub(d02, d13);
  } else if constexpr (R == 3) {
    const T s3 = -TW::get(off + N / 3).y;
    C t = cadd(x[1], x[2]);
    C m = C{x[0].x - T(0.5) * t.x, x[0].y - T(0.5) * t.y};
    C d = cmul_si(cscale(csub(x[1], x[2]), s3), SIGN);
    x[0] = cadd(x[0], t);
    x[1] = cadd(m, d);
    x[2] = csub(m, d);
  } else {  // R == 5
    const C w1 = TW::get(off + N / 5), w2 = TW::get(off + 2 * (N / 5));
    const T c1 = w1.x, s1 = -w1.y, c2 = w2.x, s2 = -w2.y;
    C a1 = cadd(x[1], x[4]), a2 = cadd(x[2], x[3]);
    C b1 = csub(x[1], x[4]), b2 = csub(x[2], x[3]);
    C r1 = C{x[0].x + c1 * a1.x + c2 * a2.x, x[0].y + c1 * a1.y + c2 * a2.y};
    C r2 = C{x[0].x + c2 * a1.x + c1 * a2.x, x[0].y + c2 * a1.y + c1 * a2.y};
    C i1 = cmul_si(C{s1 * b1.x + s2 * b2.x, s1 * b1.y + s2 * b2.y}, SIGN);
    C i2 = cmul_si(C{s2 * b1.x - s1 * b2.x, s2 * b1.y - s1 * b2.y}, SIGN);
    x[0] = C{x[0].x + a1.x + a2.x, x[0].y + a1.y + a2.y};
    x[1] = cadd(r1, i1);
    x[4] = csub(r1, i1);
    x[2] = cadd(r2, i2);
    x[3] = csub(r2, i2);
  }
}

template <typename T, int N, int SIGN, int ST, int NS, typename TW> struct RegStage {
  __device__ __forceinline__ static void run(C2<T> (&v)[N]) {
    constexpr int R = stage_radix(N, ST);
    if constexpr (R != 0) {
      constexpr int nb = N / R;
      constexpr int off = reg_offset(N);
      constexpr int tstride = N / (NS * R);
      C2<T> w[N];
#pragma unroll
      for (int j = 0; j < nb; ++j) {
        const int jm = j % NS;
        C2<T> x[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
          x[r] = v[j + r * nb];
          if (r > 0 && jm != 0) {
            C2<T> t = TW::get(off + (r * jm * tstride) % N);
            if (SIGN > 0) t.y = -t.y;
            x[r] = cmul(x[r], t);
          }
        }
        dft_small<T, R, SIGN, TW>(x, off, N);
        const int idxD = (j / NS) * NS * R + jm;
#pragma unroll
        for (int r = 0; r < R; ++r) w[idxD + r * NS] = x[r];
      }
#pragma unroll
      for (int i = 0; i < N; ++i) v[i] = w[i];
      RegStage<T, N, SIGN, ST + 1, NS * R, TW>::run(v);
    }
  }
};

// In-register FFT of v (natural order in, natural order out). SIGN = -1 forward, +1 inverse
// (unnormalised).
template <typename T, int N, int SIGN, typename TW = TwTab<T>>
__device__ __forceinline__ void fft_reg(C2<T> (&v)[N]) {
  RegStage<T, N, SIGN, 0, 1, TW>::run(v);
}

}  // namespace sbse
