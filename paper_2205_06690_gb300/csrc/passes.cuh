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

// exp(-i x) as a complex number
template <typename T> __device__ __forceinline__ C2<T> expmi(T x) {
  T s, c;
  sincos_t(x, &s, &c);
  return C2<T>{c, -s};
}

// Value entering the forward transform at grid point idx of item `item` (gi = item * ng + idx):
//  XF_PHASE_A    P a                                  with P = exp(-i V tau)
//  XF_PHASE_PAIR P [(E - 1) a + E d]                  with E = exp(-i u tau) (u = 0 without feedback),
//                E - 1 = -2i sin(u tau/2) exp(-i u tau/2): the potential part of the split-operator
//                step of Eq. (10) on the difference d = eta^alpha - eta0 of one stochastic orbital
//  XF_PACK_DN    dn[2 item] + i dn[2 item + 1]        (two real densities per complex transform)
//  XF_PACK_PROD  phi_i1 phi_j1 + i phi_i2 phi_j2      (pair products, for q_ij and (ia|jb))
template <typename T>
__device__ __forceinline__ C2<T> preop_value(const GView<T> &g, const XfwdArgs<T> &a, long long item,
                                             long long idx, long long gi) {
  using C = C2<T>;
  if (a.mode == XF_PHASE_A) return cmul(expmi<T>(g.v_loc[idx] * a.tau), a.in[gi]);
  if (a.mode == XF_PHASE_PAIR) {
    const int pair = (int)(item / a.L), ell = (int)(item - (long long)pair * a.L);
    const C av = a.a[(long long)ell * g.ng + idx];
    const C dv = a.in[gi];
    const T uu = a.feedback ? a.u[(long long)pair * g.ng + idx] : T(0);
    T s, c;
    sincos_t(T(0.5) * uu * a.tau, &s, &c);
    const C em1 = C{T(-2) * s * s, T(-2) * s * c};
    const C E = C{T(1) + em1.x, em1.y};
    return cmul(expmi<T>(g.v_loc[idx] * a.tau), cadd(cmul(em1, av), cmul(E, dv)));
  }
  if (a.mode == XF_PACK_DN) {
    const long long k0 = 2 * item, k1 = 2 * item + 1;
    return C{a.dn[k0 * g.ng + idx], (k1 < a.n_dn) ? a.dn[k1 * g.ng + idx] : T(0)};
  }
  const int4 q = a.prod[item];
  return C{a.orb[(long long)q.x * g.ng + idx] * a.orb[(long long)q.y * g.ng + idx],
           (q.z >= 0) ? a.orb[(long long)q.z * g.ng + idx] * a.orb[(long long)q.w * g.ng + idx] : T(0)};
}

}  // namespace sbse
