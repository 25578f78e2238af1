// Host-side interface between the translation units of the sbse library (not part of the C ABI).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"
#include "tables.cuh"

namespace sbse {

// Number of kernel launches issued by the library in this process (sbse_api.cu).
void count_launch(int n);
// raise (never lower) a kernel's dynamic shared memory limit to `bytes`, thread-safe
void raise_smem_limit(const void *fn, size_t bytes);
// tiled tensor map of an FP32 array for bulk tensor copies (dims / box innermost first, strides in
// bytes of the rank - 1 outer dimensions; zero fill outside the array); false if the driver's
// encoder is unavailable or rejects the layout
bool make_tensor_map_f32(CUtensorMap *map, const void *base, int rank, const uint64_t *dims,
                         const uint64_t *strides_bytes, const uint32_t *box, bool swizzle128);

// ---- register-pencil three-pass round trip (fft_fast.cu), for the sizes fast_supported<T>(N)
int upload_reg_twiddles();
// ---- lane-pair split-pencil passes for the grid edges 80 and 96, FP32 (fft_split.cu); the
// launchers of fft_fast.cu route those sizes here
bool split_size(int N);
int upload_split_twiddles();
void init_split_kernels();
template <typename T> bool fast_supported(int N);
template <typename T> void init_fast_kernels();

// ---- FFT passes (tdh_kernels.cu). Items are contiguous arrays of ng complex values.
template <typename T> void launch_xfwd(const GridTables<T> &g, const XfwdArgs<T> &a, cudaStream_t s);
template <typename T> void launch_plane_fwd(const GridTables<T> &g, const XfwdArgs<T> &a, cudaStream_t s);
// tma_err != null (FP32, N in 32 / 40 / 48 / 64): the bulk-copy streamed column kernel
template <typename T> void launch_zcol(const GridTables<T> &g, C2<T> *d, int n_items, int mult, cudaStream_t s,
                                       int *tma_err = nullptr);
// tma_err != null (FP32, density epilogue, N in 32 / 40 / 48 / 64): the bulk-copy streamed kernel,
// which sets *tma_err if one of its bounded waits runs out
template <typename T> void launch_plane_inv_orb(const GridTables<T> &g, C2<T> *d, int n_items,
                                                const C2<T> *a_next, int L, T *dens, cudaStream_t s,
                                                int *tma_err = nullptr);
template <typename T> void launch_plane_inv_poisson(const GridTables<T> &g, C2<T> *d, int n_slots,
                                                    const PoissonOut &po, T *u_out, T *acc,
                                                    C2<T> *em1_out, cudaStream_t s);
// split sizes (fft_split.cu): the Poisson round trip (packing modes of XfwdArgs, Z_POISSON)
void launch_plane_fwd2(const GridTables<float> &g, const XfwdArgs<float> &a, cudaStream_t s);
void launch_zcol2(const GridTables<float> &g, float2 *d, int n_items, int mult, cudaStream_t s);
void launch_plane_inv2_poisson(const GridTables<float> &g, float2 *d, int n_slots, const PoissonOut &po,
                               float *u_out, float *acc, float2 *em1_out, cudaStream_t s);
// split sizes: the two sweeps of a split-operator step of the orbitals (XF_PHASE_A / XF_PHASE_PAIR
// pre-operation + x and y kinetic operators; z kinetic operator + the pairs' induced density when
// dens != null, L orbitals per pair)
void launch_plane_kin2(const GridTables<float> &g, const XfwdArgs<float> &a, cudaStream_t s);
// err != null: the pair batch's sweep (dens != null) stages each orbital's columns by bulk tensor
// copies while the one before is transformed (bounded waits; *err set if one runs out)
void launch_zkin2(const GridTables<float> &g, float2 *d, int n_items, const float2 *a_next, int L, float *dens,
                  cudaStream_t s, int *err = nullptr);
// out = exp(-i V_loc tau), computed in FP64 from the FP64 potential v64
template <typename T> void launch_phase_table(const double *v64, long long ng, double tau, C2<T> *out,
                                              cudaStream_t s);
template <typename T> void launch_ypass(const GridTables<T> &g, C2<T> *data, int n_items, int sign,
                                        cudaStream_t s);
template <typename T> void launch_zpass(const GridTables<T> &g, C2<T> *data, int n_items, int mult,
                                        cudaStream_t s);
// inverse x pass of orbitals; with dens != nullptr, items are grouped L per pair and the induced
// density 2 sum_l (2 Re(conj(a_l) d_l) + |d_l|^2) of each pair is written to dens[pair].
template <typename T> void launch_xinv_orb(const GridTables<T> &g, C2<T> *data, int n_items,
                                           const C2<T> *a_next, int L, T *dens, cudaStream_t s);
// inverse x pass of packed Poisson slots: potential of density 2s (re) / 2s+1 (im) ->
// u_out[k] (if non-null) and acc[k] = acc[k] + coef * value, or coef * value when keep == 0
// (if acc non-null), k < n_out.
template <typename T> void launch_xinv_poisson(const GridTables<T> &g, C2<T> *data, int n_slots,
                                               const PoissonOut &po, T *u_out, T *acc,
                                               C2<T> *em1_out, cudaStream_t s);
// acc64 += acc, acc = 0
template <typename T> void launch_flush_acc(double *acc64, T *acc, long long n, cudaStream_t s);

// ---- persistent split-operator step (fft_fast.cu; its tile queue StepQueue is in tables.cuh)
template <typename T>
void launch_step_persistent(const GridTables<T> &g, const XfwdArgs<T> &fa, const XfwdArgs<T> &fp,
                            C2<T> *a_next, C2<T> *d, T *dens, int L, const StepQueue &q, int grid,
                            cudaStream_t s);
template <typename T> int step_resident_blocks(int N);
template <typename T> int step_tiles_per_orbital(int N);

// ---- elementwise and reduction kernels (tdh_kernels.cu)
template <typename T> void launch_init_a(const GridTables<T> &g, const double *phi, int n_occ,
                                         const double *coeff, int L, C2<T> *a, double *part,
                                         int *n_part, cudaStream_t s);
void launch_reduce_cols(const double *part, int rows, int cols, double scale, double *out,
                        cudaStream_t s);
template <typename T> void launch_kick(const GridTables<T> &g, const double *q, int P, const C2<T> *a,
                                       int L, double alpha, C2<T> *d, cudaStream_t s);
// pending half potential step before a cleaning: P = exp(-i V_loc dt/2) from the grid tables, E - 1
// per pair (tau = dt/2) from em1 (null: no feedback)
template <typename T> void launch_half_phase(const GridTables<T> &g, C2<T> *a, C2<T> *d, const C2<T> *em1,
                                             int P, int L, cudaStream_t s);
// cleaning of Eq. (15): overlaps O[c][s] = dV sum_r phi_s d_c (c < P*L complex columns)
// use_tc (FP32 only): overlaps on the tensor cores; *err set on a timed-out tensor-core wait;
// dens != null: the renormalisation also writes the induced density of each pair (Eq. 11)
// phi_can != null (FP32 only): the projection update on the tensor cores from pre-split orbitals;
// phi_ov != null (FP32 only): the overlaps by the streamed tensor-core kernel from pre-split orbitals.
// Returns c - 1 per orbital (device, P L values inside work); d is left unscaled: the next forward
// pre-operation applies d <- c d + (c - 1) eta0 (XfwdArgs::cm1), and dens (P n_g) receives the
// induced densities of the rescaled orbitals.
template <typename T> const double *launch_clean(const GridTables<T> &g, const T *phi_occ, int n_occ,
                                                 const C2<T> *a, C2<T> *d, int P, int L, const double *n0,
                                                 double dV, double *work, size_t work_bytes, bool use_tc,
                                                 const uint8_t *phi_can, int *err, cudaStream_t s, T *dens,
                                                 const uint8_t *phi_ov = nullptr);
template <typename T> size_t clean_work_bytes(long long ng, int n_occ, int P, int L);
// d64 -> T conversion and FP64 -> T copies
template <typename T> void launch_convert(const double *src, T *dst, long long n, cudaStream_t s);
int scan_nonfinite(const double *x, long long n, int *flag_dev, cudaStream_t s);

// ---- contractions (contract.cu)
// out[m][n] = scale * sum_r X_m(r) Y_n(r), X_m = F[xi[m].x](r) * F[xi[m].y](r), Y_n = Y[n] row
template <typename T> void launch_prod_gemm(const T *F, const int2 *xi, int M, const T *Y, int Nn,
                                            long long ng, double scale, double *out, double *work,
                                            size_t work_bytes, cudaStream_t s);
template <typename T> size_t prod_gemm_work_bytes(int M, int Nn, long long ng);
// fock_o (n_o x n_o, may be null): the occupied block of H0 in a rotated window, replacing eps_o
void launch_assemble_A(const double *eps_o, const double *eps_c, int n_o, int n_c, double scissor,
                       const double *K, const double *Dab, int P, double *A, cudaStream_t s,
                       const double *fock_o = nullptr);

// tensor-core (tcgen05, BF16 split, FP32 accumulate) version of launch_prod_gemm for FP32 inputs;
// *err (device int) is set when a bounded wait on the tensor cores times out
int launch_umma_prod_gemm(const float *F, const int2 *xi, int M, const float *Y, int Nn, long long ng,
                          double scale, double *out, double *work, int *err, cudaStream_t s);
size_t umma_prod_gemm_work_bytes(int M, int Nn, long long ng);
// cleaning overlaps on the tensor cores: out[2c + h][s] = scale sum_r (Re, Im)_h d_c phi_s
int launch_umma_clean_overlap(const float *d_interleaved, int n_cols, const float *phi, int n_occ,
                              long long ng, double scale, double *out, double *work, int *err,
                              cudaStream_t s);

// cleaning overlaps, streamed form (warp-specialised: bulk copies of raw d rows and of pre-split phi
// slabs, BF16 split in shared memory, tcgen05 MMAs over a ring of stages): same result layout as
// launch_umma_clean_overlap. phi_t holds phi as pre-split B tiles (umma_prepare_ov_phi, once per
// propagation). Usable when umma_clean_ov_supported (n_occ <= 512, even point count).
int launch_umma_clean_ov(const float *d_interleaved, int n_cols, const uint8_t *phi_t, int n_occ, long long ng,
                         double scale, double *out, double *work, int *err, cudaStream_t s);
bool umma_clean_ov_supported(int n_occ, long long ng);
size_t umma_clean_ov_work_bytes(int n_cols, int n_occ, long long ng);
size_t umma_ov_phi_bytes(long long ng, int n_occ);
void umma_prepare_ov_phi(const float *phi, int n_occ, long long ng, uint8_t *out, cudaStream_t s);

// cleaning update on the tensor cores: d_c -= sum_s O[2c+h][s] phi_s (h = re / im parts), plus
// per-tile norm partials npart[tile][c][2] (tiles of umma_clean_update_tiles(ng) rows). phi_can holds
// the occupied orbitals as pre-split canonical operand tiles (umma_prepare_update_phi, once per
// propagation); o_can is scratch of umma_update_o_bytes for the overlaps' tiles.
void launch_umma_clean_update(const double *ov, int n_cols, const uint8_t *phi_can, int n_occ, long long ng,
                              float *d_interleaved, const float *a_interleaved, int L, double *npart,
                              uint8_t *o_can, int *err, cudaStream_t s);
long long umma_clean_update_tiles(long long ng);
size_t umma_update_phi_bytes(long long ng, int n_occ);
size_t umma_update_o_bytes(int n_cols, int n_occ);
void umma_prepare_update_phi(const float *phi, int n_occ, long long ng, uint8_t *phi_can, cudaStream_t s);

// ---- finite-box correction W(k -> 0) (finite_box.cu)
// n0 = 2 sum_s phi_s^2 over n_occ FP64 rows of ng points
void launch_ground_density(const double *phi, int n_occ, long long ng, double *n0, cudaStream_t s);
// sums[0] = sum of v over the grid, sums[1] = sum of v + u over the boundary points (ix, iy or
// iz = 0); work: 2 x 256 doubles
void launch_box_sums(const double *v, const double *u, int N, double *work, double *sums, cudaStream_t s);

// ---- localized occupied window (localized.cu)
// cos, sin(2 pi x_alpha / L) for alpha = x, y, z: six fields of N^3 points
void launch_phase_fields(int N, double *out, cudaStream_t s);
// out[k] = sum_i U_ik phi[base + i], k < n (n x n row-major U, n <= 96 for the shared copy of U)
void launch_rotate_rows(const double *phi, int base, int n, const double *U, long long ng, double *out,
                        cudaStream_t s);
// out[p] = scale sum_r (phi[pairs[p].x] phi[pairs[p].y])^2; work: pair_norms_work_doubles(n_pairs)
size_t pair_norms_work_doubles(int n_pairs);
void launch_pair_norms(const double *phi, const int2 *pairs, int n_pairs, long long ng, double scale,
                       double *work, double *out, cudaStream_t s);

// ---- mixed hole-grid representation of A (mixed.cu), FP64; f, out: n_o rows of ng points
void launch_exciton_density(const double *phi_o, const double *f, int n_o, long long ng, double *dn, cudaStream_t s);
// out_j = tf_j + (v + scissor - eps_j - shift) f_j + dv phi_j - sum_i f_i W_ij
void launch_abar(const double *tf, const double *f, const double *v, const double *eps_o, double scissor, double shift,
                 const double *dv, const double *phi_o, const double *W, int n_o, long long ng, double *out,
                 cudaStream_t s);
// keep = 0: out_j -= sum_s <basis_s|out_j> basis_s; keep = 1: out_j = sum_s <basis_s|out_j> basis_s
size_t project_work_doubles(int n_o, int n_b, long long ng);
void launch_project(double *out, int n_o, const double *basis, int n_b, long long ng, double dV, int keep,
                    double *work, cudaStream_t s);
void launch_coord_times(const double *phi_o, int n_o, int N, double h, double box, int axis, double *out,
                        cudaStream_t s);
void launch_axpby(double a, const double *x, double b, double *y, long long n, cudaStream_t s);
size_t dot_work_doubles();
// out[0] = scale x . y (fixed-order reduction)
void launch_dot(const double *x, const double *y, long long n, double scale, double *work, double *out,
                cudaStream_t s);
// sigma(omega) from residues R (K of them) with cw = {c, w}: D (K doubles) scratch (spectrum.cu)
void launch_sigma_from_residues(const double *R, int K, const double *cw, const double *omega, int n_omega,
                                double s, double *D, double *sigma, cudaStream_t st);

// ---- absorption spectrum by a Chebyshev expansion of A (spectrum.cu)
struct SpectrumBufs {
  double *f0, *cw, *v[3], *prod, *R, *D, *omega, *sigma;
};
size_t spectrum_work_bytes(int n, int n_terms, int n_omega);
SpectrumBufs spectrum_bufs(double *work, int n, int n_terms, int n_omega);
// the caller fills b.omega (n_omega frequencies) before; b.sigma and b.R (n_terms residues) after
void launch_absorption(const SpectrumBufs &b, const double *phi_o, const double *phi_c, int n_o, int n_c, int N,
                       double h, double box, double dV, const double *A, int axis, int n_terms, double s,
                       int n_omega, cudaStream_t st);

// ---- eigensolver (eig.cu)
int launch_eig_lowest(double *A, int n, int k, double *evals_dev, double *work, cudaStream_t s);
size_t eig_work_bytes(int n);
// the same eigenvalues with their eigenvectors (device, row-major n x k, largest component positive)
int launch_eig_vectors(const double *A, int n, int k, double *evals_dev, double *evecs_dev, double *work,
                       cudaStream_t s);
size_t eig_vectors_work_bytes(int n, int k);

}  // namespace sbse
