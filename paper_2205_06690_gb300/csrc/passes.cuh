// Pieces shared by the two families of grid passes (generic shared-memory Stockham passes and the
// compile-time-N register passes): device view of the grid tables and the fused pre-operation of
// the forward pass.
#pragma once

#include "kernels.h"

namespace sbse {

template <typename T> struct GView {
  int N;
  long long ng;
  FftPlan plan;
  const C2<T> *tw;
  const C2<T> *kin;
  const T *k2;
  const T *v_loc;
};

template <typename T> static GView<T> view(const GridTables<T> &g) {
  return GView<T>{g.N, g.ng, g.plan, g.tw, g.kin, g.k2, g.v_loc};
}

// E - 1 = exp(-i u tau) - 1 = -2i sin(u tau/2) exp(-i u tau/2) = (-2 s^2, -2 s c), without the
// cancellation of 1 - cos(u tau) (u tau is O(alpha))
template <typename T> __device__ __forceinline__ C2<T> phase_em1(T u, T tau) {
  T s, c;
  sincos_t(T(0.5) * u * tau, &s, &c);
  return C2<T>{T(-2) * s * s, T(-2) * s * c};
}

// exp(-i x) as a complex number
template <typename T> __device__ __forceinline__ C2<T> expmi(T x) {
  T s, c;
  sincos_t(x, &s, &c);
  return C2<T>{c, -s};
}

// Value entering the forward transform at grid point idx of one item:
//  XF_PHASE_A    P a                                  with P = exp(-i V tau) (precomputed table)
//  XF_PHASE_PAIR P [(E - 1) a + E d]                  with E - 1 = exp(-i u tau) - 1 precomputed per
//                pair by the Poisson epilogue (E = 1 without feedback): the potential part of the
//                split-operator step of Eq. (10) on the difference d = eta^alpha - eta0
//  XF_PACK_DN    dn[2 item] + i dn[2 item + 1]        (two real densities per complex transform)
//  XF_PACK_PROD  phi_i1 phi_j1 + i phi_i2 phi_j2      (pair products, for q_ij and (ia|jb))
// The per-item pointers are resolved once (preop_item) and then indexed per point (preop_at).
template <typename T> struct PreopItem {
  int mode;
  const C2<T> *in;   // PHASE_A, PHASE_PAIR
  const C2<T> *a;    // PHASE_PAIR: eta0 of the same stochastic orbital
  const C2<T> *em1;  // PHASE_PAIR: E - 1 of the pair (null: no feedback)
  T cm1;             // PHASE_PAIR: c - 1 of a deferred renormalisation (0: none)
  const C2<T> *pv;   // PHASE_A, PHASE_PAIR
  const T *r0, *r1, *r2, *r3;  // PACK_DN: r0 (re), r1 (im or null); PACK_PROD: r0 r1 (re), r2 r3 (im)
};

template <typename T>
__device__ __forceinline__ PreopItem<T> preop_item(const GView<T> &g, const XfwdArgs<T> &a, long long item) {
  PreopItem<T> it{};
  it.mode = a.mode;
  it.pv = a.pv;
  if (a.mode == XF_PHASE_A) {
    it.in = a.in + item * g.ng;
  } else if (a.mode == XF_PHASE_PAIR) {
    const int itm = (int)item;
    const int pair = itm / a.L, ell = itm - pair * a.L;
    it.in = a.in + item * g.ng;
    it.a = a.a + (long long)ell * g.ng;
    it.em1 = a.em1 ? a.em1 + (long long)pair * g.ng : nullptr;
    it.cm1 = a.cm1 ? (T)a.cm1[item] : T(0);
  } else if (a.mode == XF_PACK_DN) {
    it.r0 = a.dn + 2 * item * g.ng;
    it.r1 = (2 * item + 1 < a.n_dn) ? a.dn + (2 * item + 1) * g.ng : nullptr;
  } else {
    const int4 q = a.prod[item];
    it.r0 = a.orb + (long long)q.x * g.ng;
    it.r1 = a.orb + (long long)q.y * g.ng;
    it.r2 = q.z >= 0 ? a.orb + (long long)q.z * g.ng : nullptr;
    it.r3 = q.z >= 0 ? a.orb + (long long)q.w * g.ng : nullptr;
  }
  return it;
}

// deferred renormalisation of a cleaning (Eq. 15 reading): d <- c d + (c - 1) eta0, cm1 = c - 1
template <typename T> __device__ __forceinline__ C2<T> renorm_value(C2<T> dv, C2<T> av, T cm1) {
  return C2<T>{(T(1) + cm1) * dv.x + cm1 * av.x, (T(1) + cm1) * dv.y + cm1 * av.y};
}

template <typename T>
__device__ __forceinline__ C2<T> pair_phase(C2<T> pv, C2<T> em1, C2<T> av, C2<T> dv) {
  const C2<T> E = C2<T>{T(1) + em1.x, em1.y};
  return cmul(pv, cmac2(em1, av, E, dv));
}

template <typename T>
__device__ __forceinline__ C2<T> preop_at(const GView<T> &g, const PreopItem<T> &it, long long idx) {
  using C = C2<T>;
  if (it.mode == XF_PHASE_A) return cmul(it.pv[idx], it.in[idx]);
  if (it.mode == XF_PHASE_PAIR) {
    const C av = it.a[idx];
    return pair_phase<T>(it.pv[idx], it.em1 ? it.em1[idx] : C{T(0), T(0)}, av,
                         renorm_value<T>(it.in[idx], av, it.cm1));
  }
  if (it.mode == XF_PACK_DN) return C{it.r0[idx], it.r1 ? it.r1[idx] : T(0)};
  return C{it.r0[idx] * it.r1[idx], it.r2 ? it.r2[idx] * it.r3[idx] : T(0)};
}

template <typename T>
__device__ __forceinline__ C2<T> preop_value(const GView<T> &g, const XfwdArgs<T> &a, long long item,
                                             long long idx, long long gi) {
  (void)gi;
  return preop_at<T>(g, preop_item<T>(g, a, item), idx);
}

}  // namespace sbse
