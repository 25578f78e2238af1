// Data structures shared by the host launchers and the FFT pass kernels: the device tables of a
// grid, the pre-operation arguments of a forward pass, the Poisson epilogue outputs, the z-pass
// multipliers and the tile queue of the persistent step kernel.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace sbse {

// Device tables of one grid, in working precision T.
template <typename T> struct GridTables {
  int N = 0;
  long long ng = 0;
  FftPlan plan{};
  C2<T> *tw = nullptr;      // exp(-2 pi i k / N), k < N
  C2<T> *kin = nullptr;     // exp(-i k_m^2 dt / 2) per axis index m (rebuilt per dt); for even N
                            // followed by the lane-pair round-trip multipliers Kp, M1, M2 (N/2 each)
  T *k2 = nullptr;          // k_m^2 per axis index m
  T *v_loc = nullptr;       // V_loc(r), ng
  C2<T> *pv_dt = nullptr;   // exp(-i V_loc dt), ng (rebuilt per dt)
  C2<T> *pv_half = nullptr; // exp(-i V_loc dt / 2), ng
};

enum XfwdMode { XF_PHASE_A = 0, XF_PHASE_PAIR = 1, XF_PACK_DN = 2, XF_PACK_PROD = 3 };

template <typename T> struct XfwdArgs {
  int mode;
  int n_items;           // orbitals (A: L, PAIR: P*L) or Poisson slots
  const C2<T> *in;       // A: a_cur; PAIR: d (in place)
  C2<T> *out;            // A: a_next; PAIR: d; PACK: packed work buffer
  const C2<T> *a;        // PAIR: a_cur
  const C2<T> *pv;       // A, PAIR: exp(-i V_loc tau) per grid point (tau = dt or dt/2)
  const C2<T> *em1;      // PAIR: exp(-i u tau) - 1 per pair (ng each); null -> u ignored
  const double *cm1;     // PAIR: c - 1 per orbital of a renormalisation still to apply (null: none)
  int L;                 // PAIR: orbitals per pair
  const T *dn;           // PACK_DN: density per pair; slot s packs 2s (re) and 2s+1 (im)
  int n_dn;              // PACK_DN: number of densities
  const T *orb;          // PACK_PROD: orbital rows (ng each)
  const int4 *prod;      // PACK_PROD: per slot (i1, j1, i2, j2); i2 < 0 -> imaginary part 0
};

// Poisson epilogue outputs of slot pair k: u_out[k] = u, acc[k] (+)= coef u, and, when em1_out is
// not null, em1_out[k] = exp(-i u tau_next) - 1 = -2i sin(u tau_next/2) exp(-i u tau_next/2), the
// potential factor of the next split-operator step.
struct PoissonOut {
  int n_out;
  double coef, keep;
  double tau_next;
};

// multiplier of the z pass: kinetic propagator, Coulomb kernel 4 pi / |G|^2 (G = 0 dropped), or the
// kinetic energy |G|^2 / 2 (the spectral -1/2 Laplacian); each with the 1/N^3 of the round trip
enum ZMult { Z_KINETIC = 0, Z_POISSON = 1, Z_HALF_G2 = 2 };

// tile queue and completion counters of the persistent split-operator step (fft_fast.cu)
enum StepItemKind { SI_A_FWD = 0, SI_A_Z = 1, SI_A_INV = 2, SI_P_FWD = 3, SI_P_Z = 4, SI_P_INV = 5 };
struct StepQueue {
  const int4 *items;    // {kind, orbital (or pair for SI_P_INV), tile, 0}, dependency-ordered
  int n_items;
  unsigned *claim;      // claim counter, monotonic over the launches of one sbse_apply_W
  unsigned claim_base;  // its value when this launch starts
  unsigned *a_fwd, *a_z;  // per eta0 orbital
  unsigned *a_inv;        // all eta0 inverse tiles
  unsigned *p_fwd, *p_z;  // per pair orbital
  unsigned epoch;         // launch index: completion targets are (epoch + 1) x tiles
  int *err;               // set when a bounded wait times out
  unsigned wait_limit;    // iterations of each bounded wait (about 100 ns each)
};

}  // namespace sbse
