// C ABI of the sbse library (declared in include/sbse.h): context management, validation, the
// host-side splitmix64 coefficient stream and the orchestration of the device kernels.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <new>
#include <mutex>
#include <shared_mutex>
#include <string>
#include <unordered_map>
#include <vector>

#include "kernels.h"
#include "sbse.h"

namespace {
thread_local std::string g_create_error;
}

namespace sbse {
void init_fft_kernels();
void set_thread_error(const std::string &msg) { g_create_error = msg; }
static std::atomic<long long> g_launches{0};
void count_launch(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
// readers of the debug bounds records, one per translation unit (debug build only)
static std::vector<int (*)(unsigned long long *)> &bounds_readers() {
  static std::vector<int (*)(unsigned long long *)> r;
  return r;
}
void register_bounds_reader(int (*reader)(unsigned long long *)) { bounds_readers().push_back(reader); }
// The dynamic shared memory limit is an attribute of the kernel, shared by every context and host
// thread: lowering it for one launch could make another thread's larger launch of the same kernel
// fail in between. So it is only ever raised, under a lock.
void raise_smem_limit(const void *fn, size_t bytes) {
  static std::mutex mx;
  static std::unordered_map<const void *, size_t> cur;
  std::lock_guard<std::mutex> lk(mx);
  size_t &c = cur[fn];
  if (bytes > c && cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) == cudaSuccess)
    c = bytes;
}
}

using namespace sbse;

namespace {

struct DevBuf {
  void *p = nullptr;
  size_t cap = 0;
};

// scratch slots of a context
enum Ws {
  WS_A0 = 0, WS_A1, WS_D, WS_U, WS_DN, WS_PW, WS_WACC, WS_N0, WS_PART, WS_CLEAN, WS_COEF,
  WS_IDX, WS_GEMM, WS_K, WS_DAB, WS_EIG, WS_ACC32, WS_EM1, WS_QUEUE, WS_PHICAN, WS_SPEC, WS_FBOX,
  WS_LOC, WS_DBLK, WS_MIX, WS_PHIOV, WS_COUNT
};

struct PhaseClock {
  std::vector<cudaEvent_t> ev;  // start/stop pairs
  std::vector<int> phase;
  size_t used = 0;
};

}  // namespace

struct sbse_ctx {
  int device = 0;
  int precision = SBSE_FP64;
  cudaStream_t stream = nullptr;
  cudaStream_t aux = nullptr;  // eta0 propagation, concurrent with the pair batch
  cudaEvent_t ev_start = nullptr, ev_a = nullptr;
  std::string err;
  // grid
  int N = 0;
  double box = 0, h = 0, dV = 0;
  long long ng = 0;
  GridTables<float> g32;
  GridTables<double> g64;
  double *v64 = nullptr;
  double kin_dt = -1.0;
  // orbitals
  int n_occ = 0, n_o = 0, n_c = 0, n_states = 0;
  double scissor = 0;
  double *phi64 = nullptr;
  float *phi32 = nullptr;
  std::vector<double> eps;
  double *eps_dev = nullptr;  // eps_o (n_o) then eps_c (n_c)
  // a rotated (localized) occupied window: the occupied block of H0 in it (n_o x n_o, device)
  double *fock_o = nullptr;
  bool localized = false;
  // results
  double *W = nullptr;  // P_all x ng, canonical pair order
  std::vector<char> have;
  double *A = nullptr;
  bool have_A = false;
  bool dab_given = false;  // the direct term's D columns were set by sbse_set_direct (in WS_DAB)
  // scratch
  DevBuf ws[WS_COUNT];
  int *flag = nullptr;
  // mixed mode: grid-sum contractions on the tensor cores (SBSE_OPT_TENSOR_CORES)
  int tensor_cores = 1;
  // split-operator step as one persistent kernel (SBSE_OPT_PERSISTENT)
  int persistent = 0;
  // inverse plane pass of the pair batch streamed by bulk copies (SBSE_OPT_TMA_PLANES)
  int tma_planes = 1;
  // time loop of sbse_apply_W captured once and replayed as a CUDA graph (SBSE_OPT_GRAPH)
  int use_graph = 1;
  cudaGraphExec_t graph_exec = nullptr;
  std::vector<unsigned long long> graph_key;
  long long graph_launches = 0;  // kernel launches recorded in graph_exec (counted on every replay)
  // bytes of propagated orbitals per chunk of pairs (SBSE_OPT_CHUNK_MB); 0 = all pairs at once
  double l2_chunk_bytes = 1e30;
  // profiling
  bool prof = false;
  PhaseClock clk;
  // device memory held by the context (dalloc / release) and its limit (SBSE_OPT_MEM_LIMIT_MB; 0: none)
  std::unordered_map<void *, size_t> held;
  size_t held_bytes = 0, mem_limit = 0;
  // iteration limit of the persistent step kernel's waits on other tiles (SBSE_OPT_WAIT_LIMIT)
  unsigned wait_limit = 1u << 23;
  // a propagation stopped part way (sbse_apply_W_range): its parameters, pairs and next step; the
  // state itself is in the workspace (WS_D, WS_A0, WS_WACC, WS_ACC32, WS_EM1, WS_N0)
  struct {
    bool valid = false;
    int next = 0;
    sbse_tdh_params params{};
    std::vector<int> slots;
  } run;
};

namespace {

int fail(sbse_ctx *c, int code, const std::string &msg) {
  c->err = msg;
  return code;
}

int cuda_fail(sbse_ctx *c, cudaError_t e, const char *where) {
  c->err = std::string("CUDA error in ") + where + ": " + cudaGetErrorString(e);
  return SBSE_ERR_CUDA;
}

#define CK(call)                                              \
  do {                                                        \
    cudaError_t e_ = (call);                                  \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call);  \
  } while (0)

#define CHECK_LAUNCH(where)                                   \
  do {                                                        \
    cudaError_t e_ = cudaGetLastError();                      \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, where);  \
  } while (0)

// Graph captures of different contexts may run in parallel host threads; cudaMalloc / cudaFree
// from one thread while another thread's stream is being captured invalidates that capture. So
// captures hold this lock shared and allocations hold it exclusively.
std::shared_mutex g_capture_mx;

// Every device allocation of a context goes through dalloc / release, which keep the context's
// total (SBSE_OPT_MEM_LIMIT_MB refuses an allocation that would exceed the limit).
template <typename X> int dalloc(sbse_ctx *ctx, X **p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) return SBSE_OK;
  if (ctx->mem_limit && ctx->held_bytes + bytes > ctx->mem_limit)
    return fail(ctx, SBSE_ERR_OOM, "device allocation of " + std::to_string(bytes) +
                                       " bytes would exceed the context's memory limit of " +
                                       std::to_string(ctx->mem_limit) + " bytes");
  cudaError_t e;
  {
    std::unique_lock<std::shared_mutex> lk(g_capture_mx);
    e = cudaMalloc((void **)p, bytes);
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return fail(ctx, SBSE_ERR_OOM, "device allocation of " + std::to_string(bytes) + " bytes failed");
  }
  ctx->held[(void *)*p] = bytes;
  ctx->held_bytes += bytes;
  return SBSE_OK;
}

void release(sbse_ctx *ctx, void *p) {
  if (!p) return;
  auto it = ctx->held.find(p);
  if (it != ctx->held.end()) {
    ctx->held_bytes -= it->second;
    ctx->held.erase(it);
  }
  std::unique_lock<std::shared_mutex> lk(g_capture_mx);
  cudaFree(p);
}

template <typename X> void dfree(sbse_ctx *ctx, X *&p) {
  release(ctx, (void *)p);
  p = nullptr;
}

int ensure(sbse_ctx *ctx, int slot, size_t bytes, void **out) {
  DevBuf &b = ctx->ws[slot];
  if (b.cap < bytes) {
    // a stopped propagation keeps its state in these slots: growing one of them discards it
    if (slot == WS_A0 || slot == WS_D || slot == WS_WACC || slot == WS_ACC32 || slot == WS_EM1 || slot == WS_N0)
      ctx->run.valid = false;
    release(ctx, b.p);
    b.p = nullptr;
    b.cap = 0;
    int rc = dalloc(ctx, &b.p, bytes);
    if (rc) return rc;
    b.cap = bytes;
  }
  *out = b.p;
  return SBSE_OK;
}

void free_scratch(sbse_ctx *ctx) {
  ctx->run.valid = false;
  for (auto &b : ctx->ws) {
    release(ctx, b.p);
    b.p = nullptr;
    b.cap = 0;
  }
}

void free_results(sbse_ctx *ctx) {
  dfree(ctx, ctx->W);
  dfree(ctx, ctx->A);
  ctx->have.clear();
  ctx->have_A = false;
  ctx->dab_given = false;
}

void free_orbitals(sbse_ctx *ctx) {
  dfree(ctx, ctx->fock_o);
  ctx->localized = false;
  dfree(ctx, ctx->phi64);
  dfree(ctx, ctx->phi32);
  dfree(ctx, ctx->eps_dev);
  ctx->eps.clear();
  ctx->n_occ = ctx->n_o = ctx->n_c = ctx->n_states = 0;
  free_results(ctx);
}

template <typename T> void free_tables(sbse_ctx *ctx, GridTables<T> &g) {
  dfree(ctx, g.pv_dt);
  dfree(ctx, g.pv_half);
  dfree(ctx, g.tw);
  dfree(ctx, g.kin);
  dfree(ctx, g.k2);
  dfree(ctx, g.v_loc);
  g = GridTables<T>{};
}

void free_grid(sbse_ctx *ctx) {
  free_orbitals(ctx);
  free_tables(ctx, ctx->g32);
  free_tables(ctx, ctx->g64);
  dfree(ctx, ctx->v64);
  ctx->N = 0;
  ctx->ng = 0;
  ctx->kin_dt = -1.0;
}

bool make_plan(int n, FftPlan *pl) {
  pl->n = n;
  pl->nst = 0;
  int m = n;
  while (m % 4 == 0 && pl->nst < kMaxStages) { pl->radix[pl->nst++] = 4; m /= 4; }
  while (m % 2 == 0 && pl->nst < kMaxStages) { pl->radix[pl->nst++] = 2; m /= 2; }
  while (m % 3 == 0 && pl->nst < kMaxStages) { pl->radix[pl->nst++] = 3; m /= 3; }
  while (m % 5 == 0 && pl->nst < kMaxStages) { pl->radix[pl->nst++] = 5; m /= 5; }
  return m == 1;
}

// angular wave number of FFT index m on an n-point axis of edge L (symmetric at Nyquist in k^2)
double kval(int m, int n, double L) {
  const int mm = (m <= (n - 1) / 2) ? m : m - n;
  return 2.0 * M_PI / L * (double)mm;
}

template <typename T> int build_tables(sbse_ctx *ctx, GridTables<T> &g, const double *v_host) {
  const int N = ctx->N;
  g.N = N;
  g.ng = ctx->ng;
  make_plan(N, &g.plan);
  std::vector<C2<T>> tw(N);
  std::vector<T> k2(N);
  for (int k = 0; k < N; ++k) {
    const double a = -2.0 * M_PI * (double)k / (double)N;
    tw[k] = C2<T>{(T)cos(a), (T)sin(a)};
    const double kk = kval(k, N, ctx->box);
    k2[k] = (T)(kk * kk);
  }
  int rc;
  if ((rc = dalloc(ctx, &g.tw, N * sizeof(C2<T>)))) return rc;
  // per-axis kinetic factors (N), then for even N the lane-pair round-trip multipliers (3 N / 2)
  if ((rc = dalloc(ctx, &g.kin, (N + 3 * (N / 2)) * sizeof(C2<T>)))) return rc;
  if ((rc = dalloc(ctx, &g.k2, N * sizeof(T)))) return rc;
  if ((rc = dalloc(ctx, &g.v_loc, ctx->ng * sizeof(T)))) return rc;
  if ((rc = dalloc(ctx, &g.pv_dt, ctx->ng * sizeof(C2<T>)))) return rc;
  if ((rc = dalloc(ctx, &g.pv_half, ctx->ng * sizeof(C2<T>)))) return rc;
  CK(cudaMemcpyAsync(g.tw, tw.data(), N * sizeof(C2<T>), cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaMemcpyAsync(g.k2, k2.data(), N * sizeof(T), cudaMemcpyHostToDevice, ctx->stream));
  (void)v_host;
  launch_convert<T>(ctx->v64, g.v_loc, ctx->ng, ctx->stream);
  CHECK_LAUNCH("convert v_loc");
  CK(cudaStreamSynchronize(ctx->stream));
  return SBSE_OK;
}

// kinetic propagator per axis: exp(-i k_m^2 dt / 2); the 3D factor is the product over axes
template <typename T> int set_kinetic(sbse_ctx *ctx, GridTables<T> &g, double dt) {
  const int N = ctx->N, H = N / 2;
  std::vector<C2<T>> kin(N + 3 * H);
  std::vector<double> kr(N), ki(N);
  for (int m = 0; m < N; ++m) {
    const double kk = kval(m, N, ctx->box);
    const double ph = -0.5 * dt * kk * kk;
    kr[m] = cos(ph);
    ki[m] = sin(ph);
    kin[m] = C2<T>{(T)kr[m], (T)ki[m]};
  }
  // The one-dimensional kinetic operator F^-1 diag(K) F on the even and odd samples (one per lane
  // of a lane pair): with E, O the half-length transforms, the even outputs are the inverse
  // half-length transform of E Kp + O M1 and the odd ones of O Kp + E M2, where
  // Kp = (K_k + K_k+H) / N, M1 = W^k (K_k - K_k+H) / N, M2 = W^-k (K_k - K_k+H) / N, W = exp(-2 pi i / N).
  if (N % 2 == 0) {
    for (int k = 0; k < H; ++k) {
      const double pr = (kr[k] + kr[k + H]) / N, pi = (ki[k] + ki[k + H]) / N;
      const double mr = (kr[k] - kr[k + H]) / N, mi = (ki[k] - ki[k + H]) / N;
      const double wr = cos(-2.0 * M_PI * k / N), wi = sin(-2.0 * M_PI * k / N);
      kin[N + k] = C2<T>{(T)pr, (T)pi};
      kin[N + H + k] = C2<T>{(T)(wr * mr - wi * mi), (T)(wr * mi + wi * mr)};
      kin[N + 2 * H + k] = C2<T>{(T)(wr * mr + wi * mi), (T)(wr * mi - wi * mr)};
    }
  }
  CK(cudaMemcpyAsync(g.kin, kin.data(), kin.size() * sizeof(C2<T>), cudaMemcpyHostToDevice, ctx->stream));
  // potential factors exp(-i V dt) (two merged half steps) and exp(-i V dt / 2)
  launch_phase_table<T>(ctx->v64, ctx->ng, dt, g.pv_dt, ctx->stream);
  launch_phase_table<T>(ctx->v64, ctx->ng, 0.5 * dt, g.pv_half, ctx->stream);
  CHECK_LAUNCH("phase tables");
  CK(cudaStreamSynchronize(ctx->stream));
  return SBSE_OK;
}

uint64_t splitmix64_out(uint64_t seed, uint64_t k) {
  uint64_t z = seed + (k + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

int pair_index(int n_o, int i, int j) {
  const int lo = std::min(i, j), hi = std::max(i, j);
  return lo * n_o - lo * (lo - 1) / 2 + (hi - lo);
}

// ---- phase timing
void clk_begin(sbse_ctx *ctx, int phase, size_t *slot) {
  if (!ctx->prof) return;
  PhaseClock &c = ctx->clk;
  if (c.used + 2 > c.ev.size()) {
    const size_t add = std::max<size_t>(256, c.ev.size());
    for (size_t i = 0; i < add; ++i) {
      cudaEvent_t e;
      cudaEventCreate(&e);
      c.ev.push_back(e);
    }
    c.phase.resize(c.ev.size() / 2 + 1);
  }
  *slot = c.used;
  c.phase[c.used / 2] = phase;
  cudaEventRecord(c.ev[c.used], ctx->stream);
  c.used += 2;
}
void clk_end(sbse_ctx *ctx, size_t slot) {
  if (!ctx->prof) return;
  cudaEventRecord(ctx->clk.ev[slot + 1], ctx->stream);
}

// ---- templated pieces of the hot path

template <typename T> GridTables<T> &tables(sbse_ctx *ctx);
template <> GridTables<float> &tables<float>(sbse_ctx *ctx) { return ctx->g32; }
template <> GridTables<double> &tables<double>(sbse_ctx *ctx) { return ctx->g64; }
template <typename T> const T *phi_T(sbse_ctx *ctx);
template <> const float *phi_T<float>(sbse_ctx *ctx) { return ctx->phi32; }
template <> const double *phi_T<double>(sbse_ctx *ctx) { return ctx->phi64; }

// u_k = v dens_k (k < n) through packed complex FFTs; acc_k += coef u_k when acc != null
// forward 3D FFT with the fused pre-operation, the z multiplier, and the inverse 3D FFT of the
// orbitals of fa (n_items contiguous fields in `data`); the epilogue writes the induced density of
// every pair (dens != null, L orbitals per pair) or just stores the propagated orbitals
enum RoundTripParts { RT_FWD_Z = 1, RT_INV = 2, RT_ALL = 3 };

template <typename T>
void round_trip_orbitals(sbse_ctx *ctx, const GridTables<T> &g, const XfwdArgs<T> &fa, C2<T> *data,
                         int n_items, const C2<T> *a_next, int L, T *dens, cudaStream_t st = nullptr,
                         int parts = RT_ALL) {
  if (!st) st = ctx->stream;
  // the pair batch (dens != null) times each pass separately when profiling (phases 5, 6, 7)
  const bool sub = dens != nullptr && st == ctx->stream;
  size_t ck = 0;
  if constexpr (sizeof(T) == 4) {
    if (split_size(g.N)) {
      // two sweeps: potential phase + x, y kinetic operators; z kinetic operator (+ density)
      if (parts & RT_FWD_Z) {
        if (sub) clk_begin(ctx, 5, &ck);
        launch_plane_kin2(g, fa, st);
        count_launch(1);
        if (sub) clk_end(ctx, ck);
      }
      if (parts & RT_INV) {
        if (sub) clk_begin(ctx, 7, &ck);
        launch_zkin2(g, data, n_items, a_next, L, dens, st, ctx->tma_planes ? ctx->flag : nullptr);
        count_launch(1);
        if (sub) clk_end(ctx, ck);
      }
      return;
    }
  }
  if (fast_supported<T>(g.N)) {
    if (parts & RT_FWD_Z) {
      if (sub) clk_begin(ctx, 5, &ck);
      launch_plane_fwd<T>(g, fa, st);
      if (sub) clk_end(ctx, ck);
      if (sub) clk_begin(ctx, 6, &ck);
      launch_zcol<T>(g, data, n_items, Z_KINETIC, st, ctx->tma_planes ? ctx->flag : nullptr);
      if (sub) clk_end(ctx, ck);
    }
    if (parts & RT_INV) {
      if (sub) clk_begin(ctx, 7, &ck);
      launch_plane_inv_orb<T>(g, data, n_items, a_next, L, dens, st, ctx->tma_planes ? ctx->flag : nullptr);
      if (sub) clk_end(ctx, ck);
    }
  } else {
    if (parts & RT_FWD_Z) {
      launch_xfwd<T>(g, fa, st);
      launch_ypass<T>(g, data, n_items, -1, st);
      launch_zpass<T>(g, data, n_items, Z_KINETIC, st);
      launch_ypass<T>(g, data, n_items, +1, st);
    }
    if (parts & RT_INV) launch_xinv_orb<T>(g, data, n_items, a_next, L, dens, st);
  }
}

// Poisson round trip of packed slots (fa.mode is XF_PACK_DN or XF_PACK_PROD)
template <typename T>
void round_trip_poisson(sbse_ctx *ctx, const GridTables<T> &g, const XfwdArgs<T> &fa,
                        const PoissonOut &po, T *u_out, T *acc, C2<T> *em1_out, int zmult = Z_POISSON) {
  cudaStream_t st = ctx->stream;
  C2<T> *pw = fa.out;
  const int S = fa.n_items;
  if (fast_supported<T>(g.N)) {
    launch_plane_fwd<T>(g, fa, st);
    launch_zcol<T>(g, pw, S, zmult, st);  // few items: the plain column kernel has more blocks
    launch_plane_inv_poisson<T>(g, pw, S, po, u_out, acc, em1_out, st);
  } else {
    launch_xfwd<T>(g, fa, st);
    launch_ypass<T>(g, pw, S, -1, st);
    launch_zpass<T>(g, pw, S, zmult, st);
    launch_ypass<T>(g, pw, S, +1, st);
    launch_xinv_poisson<T>(g, pw, S, po, u_out, acc, em1_out, st);
  }
}

// u_k = v dens_k; acc_k += coef u_k (acc != null); em1_k = exp(-i u_k tau_next) - 1 (em1 != null)
template <typename T>
int poisson(sbse_ctx *ctx, const GridTables<T> &g, const T *dens, int n, C2<T> *pw, T *u_out,
            T *acc, double coef, C2<T> *em1, double tau_next) {
  const int S = (n + 1) / 2;
  XfwdArgs<T> xa{};
  xa.mode = XF_PACK_DN;
  xa.n_items = S;
  xa.out = pw;
  xa.dn = dens;
  xa.n_dn = n;
  round_trip_poisson<T>(ctx, g, xa, PoissonOut{n, coef, 1.0, tau_next}, u_out, acc, em1);
  CHECK_LAUNCH("poisson");
  return SBSE_OK;
}

// potentials of pair products prod[s] = (i1, j1, i2, j2) -> out (T) and/or acc (FP64, assigned)
template <typename T>
int poisson_products(sbse_ctx *ctx, const GridTables<T> &g, const T *orb, const int4 *prod_dev,
                     int n_out, C2<T> *pw, T *u_out, T *acc) {
  const int S = (n_out + 1) / 2;
  XfwdArgs<T> xa{};
  xa.mode = XF_PACK_PROD;
  xa.n_items = S;
  xa.out = pw;
  xa.orb = orb;
  xa.prod = prod_dev;
  round_trip_poisson<T>(ctx, g, xa, PoissonOut{n_out, 1.0, 0.0, 0.0}, u_out, acc, nullptr);
  CHECK_LAUNCH("poisson_products");
  return SBSE_OK;
}

// Runs the time steps [n_begin, n_end) of the propagation (0 and p->n_steps for a whole run).
// n_begin > 0 continues from the state held in the workspace (d, eta0 of the step in WS_A0, the
// time integral, E - 1, the norms), left by a range ending there or loaded by sbse_load_state;
// n_end < n_steps leaves that state in the workspace instead of storing W.
template <typename T>
int run_apply_W(sbse_ctx *ctx, const sbse_tdh_params *p, const std::vector<int> &slots,
                const std::vector<double> &coef_host, int n_begin, int n_end) {
  using C = C2<T>;
  GridTables<T> &g = tables<T>(ctx);
  const long long ng = ctx->ng;
  const int P = (int)slots.size();
  const int L = p->n_s;
  const int S = (P + 1) / 2;
  cudaStream_t st = ctx->stream;
  int rc;
  if (ctx->kin_dt != p->dt) {
    if ((rc = set_kinetic<float>(ctx, ctx->g32, p->dt))) return rc;
    if ((rc = set_kinetic<double>(ctx, ctx->g64, p->dt))) return rc;
    ctx->kin_dt = p->dt;
  }
  void *vp;
  C *a0, *a1, *d, *pw;
  T *dn;
  double *wacc, *n0, *part, *cwork, *coef;
  int4 *prod;
  if ((rc = ensure(ctx, WS_A0, (size_t)L * ng * sizeof(C), &vp))) return rc;
  a0 = (C *)vp;
  if ((rc = ensure(ctx, WS_A1, (size_t)L * ng * sizeof(C), &vp))) return rc;
  a1 = (C *)vp;
  if ((rc = ensure(ctx, WS_D, (size_t)P * L * ng * sizeof(C), &vp))) return rc;
  d = (C *)vp;
  if ((rc = ensure(ctx, WS_DN, (size_t)P * ng * sizeof(T), &vp))) return rc;
  dn = (T *)vp;
  const size_t pw_bytes = std::max((size_t)S * ng * sizeof(C), (size_t)S * ng * sizeof(C2<double>));
  if ((rc = ensure(ctx, WS_PW, pw_bytes, &vp))) return rc;
  pw = (C *)vp;
  if ((rc = ensure(ctx, WS_WACC, (size_t)P * ng * sizeof(double), &vp))) return rc;
  wacc = (double *)vp;
  // the damped time integral of Eq. (13) is summed in working precision and folded into the FP64
  // accumulator every kFlush steps (FP64 arithmetic is ~70x slower than FP32 on this GPU)
  constexpr int kFlush = 16;
  T *accT = (T *)wacc;
  if (sizeof(T) != sizeof(double)) {
    if ((rc = ensure(ctx, WS_ACC32, (size_t)P * ng * sizeof(T), &vp))) return rc;
    accT = (T *)vp;
    if (n_begin == 0) CK(cudaMemsetAsync(accT, 0, (size_t)P * ng * sizeof(T), st));
  }
  C *em1 = nullptr;
  if (p->feedback) {
    if ((rc = ensure(ctx, WS_EM1, (size_t)P * ng * sizeof(C), &vp))) return rc;
    em1 = (C *)vp;
    if (n_begin == 0) CK(cudaMemsetAsync(em1, 0, (size_t)P * ng * sizeof(C), st));
  }
  if ((rc = ensure(ctx, WS_N0, (size_t)L * sizeof(double), &vp))) return rc;
  n0 = (double *)vp;
  const long long nblk = (ng + 255) / 256;
  if ((rc = ensure(ctx, WS_PART, (size_t)nblk * L * sizeof(double), &vp))) return rc;
  part = (double *)vp;
  const size_t cw = clean_work_bytes<T>(ng, ctx->n_occ, P, L);
  if ((rc = ensure(ctx, WS_CLEAN, cw, &vp))) return rc;
  cwork = (double *)vp;
  // tensor-core cleaning update (FP32): the occupied orbitals as pre-split operand tiles
  const uint8_t *phi_can = nullptr, *phi_ov = nullptr;
  if (sizeof(T) == sizeof(float) && ctx->tensor_cores) {
    if ((rc = ensure(ctx, WS_PHICAN, umma_update_phi_bytes(ng, ctx->n_occ), &vp))) return rc;
    umma_prepare_update_phi(ctx->phi32, ctx->n_occ, ng, (uint8_t *)vp, st);
    phi_can = (const uint8_t *)vp;
    if (umma_clean_ov_supported(ctx->n_occ, ng) && p->clean_every > 0) {
      if ((rc = ensure(ctx, WS_PHIOV, umma_ov_phi_bytes(ng, ctx->n_occ), &vp))) return rc;
      umma_prepare_ov_phi(ctx->phi32, ctx->n_occ, ng, (uint8_t *)vp, st);
      phi_ov = (const uint8_t *)vp;
    }
  }
  if ((rc = ensure(ctx, WS_COEF, coef_host.size() * sizeof(double), &vp))) return rc;
  coef = (double *)vp;
  if ((rc = ensure(ctx, WS_IDX, (size_t)S * sizeof(int4), &vp))) return rc;
  prod = (int4 *)vp;

  CK(cudaMemsetAsync(ctx->flag, 0, sizeof(int), st));
  if (n_begin == 0) {
  // ---- init: eta0_l (Eq. 14), N0_l, q_ij (FP64), kick
  CK(cudaMemcpyAsync(coef, coef_host.data(), coef_host.size() * sizeof(double),
                     cudaMemcpyHostToDevice, st));
  int n_part = 0;
  launch_init_a<T>(g, ctx->phi64, ctx->n_occ, coef, L, a0, part, &n_part, st);
  launch_reduce_cols(part, n_part, L, ctx->dV, n0, st);
  CHECK_LAUNCH("init_a");
  std::vector<int4> pr(S);
  const int base = ctx->n_occ - ctx->n_o;
  std::vector<int> pi_of(P), pj_of(P);
  for (int k = 0; k < P; ++k) {
    // canonical slot -> (i, j)
    int s = slots[k], i = 0;
    while (s >= ctx->n_o - i) { s -= ctx->n_o - i; ++i; }
    pi_of[k] = i;
    pj_of[k] = i + s;
  }
  for (int s = 0; s < S; ++s) {
    const int k0 = 2 * s, k1 = 2 * s + 1;
    pr[s] = make_int4(base + pi_of[k0], base + pj_of[k0], k1 < P ? base + pi_of[k1] : -1,
                      k1 < P ? base + pj_of[k1] : -1);
  }
  CK(cudaMemcpyAsync(prod, pr.data(), S * sizeof(int4), cudaMemcpyHostToDevice, st));
  if ((rc = poisson_products<double>(ctx, ctx->g64, ctx->phi64, prod, P, (C2<double> *)pw, nullptr,
                                     wacc)))
    return rc;
  launch_kick<T>(g, wacc, P, a0, L, p->alpha, d, st);
  CHECK_LAUNCH("kick");
  }

  // ---- time loop (Eq. 10 split-operator, Eq. 15 cleaning, Eq. 13 damped trapezoid)
  const int Nt = p->n_steps, M = p->clean_every;
  std::vector<double> wts(Nt + 1);
  for (int n = 0; n <= Nt; ++n) {
    const double t = n * p->dt;
    const double w = (n == 0 || n == Nt) ? 0.5 : 1.0;
    wts[n] = w * exp(-0.5 * p->gamma * p->gamma * t * t) * p->dt / p->alpha;
  }
  C *acur = a0, *anext = a1;
  // persistent step kernel: dependency-ordered tile queue and completion counters
  // (the persistent step kernel exists for the thread-per-pencil sizes only, not for 80 and 96)
  const bool persistent = ctx->persistent && fast_supported<T>(ctx->N) && !split_size(ctx->N);
  StepQueue sq{};
  int step_grid = 0;
  long long epoch = 0;
  if (persistent) {
    const int G = step_tiles_per_orbital<T>(ctx->N);
    std::vector<int4> items;
    auto add_orb = [&](int kind, int o) {
      for (int t = 0; t < G; ++t) items.push_back(make_int4(kind, o, t, 0));
    };
    auto fwd_pair = [&](int j) { for (int l = 0; l < L; ++l) add_orb(SI_P_FWD, j * L + l); };
    auto z_pair = [&](int j) { for (int l = 0; l < L; ++l) add_orb(SI_P_Z, j * L + l); };
    auto inv_pair = [&](int j) { for (int t = 0; t < G; ++t) items.push_back(make_int4(SI_P_INV, j, t, 0)); };
    for (int l = 0; l < L; ++l) add_orb(SI_A_FWD, l);
    fwd_pair(0);
    for (int l = 0; l < L; ++l) add_orb(SI_A_Z, l);
    if (P > 1) fwd_pair(1);
    z_pair(0);
    for (int l = 0; l < L; ++l) add_orb(SI_A_INV, l);
    for (int j = 2; j < P + 2; ++j) {  // pair j forward, pair j-1 z, pair j-2 inverse + density
      if (j < P) fwd_pair(j);
      if (j - 1 < P) z_pair(j - 1);
      inv_pair(j - 2);
    }
    const size_t n_cnt = 2 + 2 * (size_t)L + 2 * (size_t)P * L;
    if ((rc = ensure(ctx, WS_QUEUE, items.size() * sizeof(int4) + n_cnt * sizeof(unsigned), &vp))) return rc;
    int4 *items_dev = (int4 *)vp;
    unsigned *cnt = (unsigned *)(items_dev + items.size());
    CK(cudaMemcpyAsync(items_dev, items.data(), items.size() * sizeof(int4), cudaMemcpyHostToDevice, st));
    CK(cudaMemsetAsync(cnt, 0, n_cnt * sizeof(unsigned), st));
    sq.items = items_dev;
    sq.n_items = (int)items.size();
    sq.claim = cnt;
    sq.a_fwd = cnt + 1;
    sq.a_z = sq.a_fwd + L;
    sq.a_inv = sq.a_z + L;
    sq.p_fwd = sq.a_inv + 1;
    sq.p_z = sq.p_fwd + (size_t)P * L;
    sq.err = ctx->flag;
    sq.wait_limit = ctx->wait_limit;
    step_grid = step_resident_blocks<T>(ctx->N);
    if (step_grid <= 0) return fail(ctx, SBSE_ERR_CUDA, "persistent step kernel cannot be resident");
  }
  const double pair_bytes = (double)L * ng * sizeof(C);
  const int chunk_pairs = std::max(1, std::min(P, (int)(ctx->l2_chunk_bytes / pair_bytes)));
  // the eta0 set's round trip of step n, on the auxiliary stream once the pair batch of the step
  // before has finished reading the buffer it overwrites
  auto eta0_step = [&](const C *a_in, C *a_out, const C2<T> *pv) -> int {
    XfwdArgs<T> xa{};
    xa.mode = XF_PHASE_A;
    xa.n_items = L;
    xa.in = a_in;
    xa.out = a_out;
    xa.pv = pv;
    CK(cudaEventRecord(ctx->ev_start, st));
    CK(cudaStreamWaitEvent(ctx->aux, ctx->ev_start, 0));
    round_trip_orbitals<T>(ctx, g, xa, a_out, L, nullptr, L, nullptr, ctx->aux, RT_ALL);
    CK(cudaEventRecord(ctx->ev_a, ctx->aux));
    return SBSE_OK;
  };
  bool eta0_issued = false;  // the eta0 round trip of this step was issued during the last Poisson
  auto time_loop = [&]() -> int {
  for (int n = n_begin; n < n_end; ++n) {
    bool pending = n > 0;
    const double *cm1_pending = nullptr;
    if (M > 0 && n % M == 0) {
      size_t ck = 0;
      clk_begin(ctx, 2, &ck);
      if (pending) launch_half_phase<T>(g, acur, d, em1, P, L, st);
      pending = false;
      // the renormalisation is applied by this step's forward pre-operation (one sweep of d less)
      cm1_pending = launch_clean<T>(g, phi_T<T>(ctx), ctx->n_occ, acur, d, P, L, n0, ctx->dV, cwork, cw,
                                    ctx->tensor_cores != 0, phi_can, ctx->flag, st, dn, phi_ov);
      CHECK_LAUNCH("clean");
      if ((rc = poisson<T>(ctx, g, dn, P, pw, nullptr, accT, wts[n], em1, 0.5 * p->dt))) return rc;
      clk_end(ctx, ck);
    }
    size_t c0 = 0;
    clk_begin(ctx, 0, &c0);
    XfwdArgs<T> xa{};
    xa.mode = XF_PHASE_A;
    xa.n_items = L;
    xa.in = acur;
    xa.out = anext;
    xa.pv = pending ? g.pv_dt : g.pv_half;
    if (persistent) {
      XfwdArgs<T> xb{};
      xb.mode = XF_PHASE_PAIR;
      xb.n_items = P * L;
      xb.in = d;
      xb.out = d;
      xb.a = acur;
      xb.em1 = em1;
      xb.cm1 = cm1_pending;
      xb.L = L;
      xb.pv = xa.pv;
      sq.claim_base = (unsigned)(epoch * (unsigned long long)(sq.n_items + step_grid));
      sq.epoch = (unsigned)epoch;
      launch_step_persistent<T>(g, xa, xb, anext, d, dn, L, sq, step_grid, st);
      ++epoch;
      CHECK_LAUNCH("persistent step");
      clk_end(ctx, c0);
      goto poisson_step;
    }
    // the eta0 set (small launches) runs on the auxiliary stream: issued during the previous
    // step's Poisson solve (latency-bound, SMs to spare) unless a cleaning came in between, else
    // here, concurrently with the first two passes of the pair batch; the pairs' inverse pass
    // (which needs the new eta0) waits for it
    if (!eta0_issued && (rc = eta0_step(acur, anext, xa.pv))) return rc;
    eta0_issued = false;
    // the three passes run over chunks of pairs (SBSE_OPT_CHUNK_MB, default: all pairs at once)
    for (int p0 = 0; p0 < P; p0 += chunk_pairs) {
      const int pc = std::min(chunk_pairs, P - p0);
      C *dc = d + (long long)p0 * L * ng;
      XfwdArgs<T> xb{};
      xb.mode = XF_PHASE_PAIR;
      xb.n_items = pc * L;
      xb.in = dc;
      xb.out = dc;
      xb.a = acur;
      xb.em1 = em1 ? em1 + (long long)p0 * ng : nullptr;
      xb.cm1 = cm1_pending ? cm1_pending + (long long)p0 * L : nullptr;
      xb.L = L;
      xb.pv = pending ? g.pv_dt : g.pv_half;
      round_trip_orbitals<T>(ctx, g, xb, dc, pc * L, anext, L, dn + (long long)p0 * ng, st, RT_FWD_Z);
      if (p0 == 0) CK(cudaStreamWaitEvent(st, ctx->ev_a, 0));
      round_trip_orbitals<T>(ctx, g, xb, dc, pc * L, anext, L, dn + (long long)p0 * ng, st, RT_INV);
    }
    CHECK_LAUNCH("step");
    clk_end(ctx, c0);
    if (n + 1 < n_end && !(M > 0 && (n + 1) % M == 0)) {
      // next step's eta0 round trip: reads this step's new eta0 (anext), overwrites acur, which
      // the pair batch above has finished reading; no cleaning in between, so its phase is full
      if ((rc = eta0_step(anext, acur, g.pv_dt))) return rc;
      eta0_issued = true;
    }
  poisson_step:
    size_t c1 = 0;
    clk_begin(ctx, 1, &c1);
    // before a cleaning the potential is recomputed from the cleaned orbitals (and accumulated
    // then); this one only supplies E - 1 at dt/2 for the pending half step
    const bool recomputed = (M > 0 && (n + 1) % M == 0 && n + 1 < Nt);
    if ((rc = poisson<T>(ctx, g, dn, P, pw, nullptr, recomputed ? nullptr : accT,
                         recomputed ? 0.0 : wts[n + 1], em1, recomputed ? 0.5 * p->dt : p->dt)))
      return rc;
    if (sizeof(T) != sizeof(double) && ((n + 1) % kFlush == 0 || n + 1 == Nt))
      launch_flush_acc<T>(wacc, accT, (long long)P * ng, st);
    clk_end(ctx, c1);
    std::swap(acur, anext);
  }
  return SBSE_OK;
  };
  // The time loop's launches depend only on the values in this key (device buffers and tables,
  // sizes, parameters, options); a call with an equal key replays the captured graph. Table and
  // buffer contents are not part of it: they are written before the loop on every call.
  auto ptr = [](const void *q) { return (unsigned long long)(uintptr_t)q; };
  std::vector<unsigned long long> key = {
      ptr(g.tw), ptr(g.kin), ptr(g.k2), ptr(g.v_loc), ptr(phi_T<T>(ctx)), (unsigned long long)ctx->N,
      (unsigned long long)ctx->n_occ, (unsigned long long)ctx->tensor_cores, (unsigned long long)ctx->tma_planes,
      (unsigned long long)(uintptr_t)d, (unsigned long long)(uintptr_t)a0,
      (unsigned long long)(uintptr_t)a1, (unsigned long long)(uintptr_t)dn, (unsigned long long)(uintptr_t)pw,
      (unsigned long long)(uintptr_t)wacc, (unsigned long long)(uintptr_t)accT, (unsigned long long)(uintptr_t)em1,
      (unsigned long long)(uintptr_t)n0, (unsigned long long)(uintptr_t)cwork, (unsigned long long)(uintptr_t)phi_can,
      (unsigned long long)(uintptr_t)g.pv_dt, (unsigned long long)(uintptr_t)g.pv_half, (unsigned long long)P,
      (unsigned long long)L, (unsigned long long)Nt, (unsigned long long)M, (unsigned long long)p->feedback,
      (unsigned long long)chunk_pairs, (unsigned long long)persistent, (unsigned long long)sizeof(T),
      (unsigned long long)(uintptr_t)sq.items, (unsigned long long)(uintptr_t)sq.claim,
      (unsigned long long)sq.wait_limit, (unsigned long long)n_begin, (unsigned long long)n_end};
  for (double v : {p->dt, p->gamma, p->alpha, ctx->dV}) {
    unsigned long long b;
    memcpy(&b, &v, sizeof b);
    key.push_back(b);
  }
  bool replayed = false;
  if (ctx->use_graph && !ctx->prof) {
    if (ctx->graph_exec && ctx->graph_key == key) {
      CK(cudaGraphLaunch(ctx->graph_exec, st));
      count_launch((int)ctx->graph_launches);
      replayed = true;
    } else {
      if (ctx->graph_exec) {
        cudaGraphExecDestroy(ctx->graph_exec);
        ctx->graph_exec = nullptr;
      }
      cudaGraph_t graph = nullptr;
      std::shared_lock<std::shared_mutex> capture_lock(g_capture_mx);
      if (cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed) == cudaSuccess) {
        // launches issued while capturing are counted once here; they run in the replay below
        const long long l0 = g_launches.load();
        const int rc_loop = time_loop();
        ctx->graph_launches = g_launches.load() - l0;
        const cudaError_t e_end = cudaStreamEndCapture(st, &graph);
        if (rc_loop) {
          if (graph) cudaGraphDestroy(graph);
          return rc_loop;
        }
        cudaGraphExec_t exec = nullptr;
        if (e_end == cudaSuccess && graph && cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess) {
          ctx->graph_exec = exec;
          ctx->graph_key = key;
          CK(cudaGraphLaunch(exec, st));
          replayed = true;
        } else {
          count_launch(-(int)ctx->graph_launches);  // recorded, never run
        }
        if (graph) cudaGraphDestroy(graph);
      }
      cudaGetLastError();  // a capture that could not be used leaves no error behind
    }
  }
  if (!replayed) {  // (a capture that could not be used only recorded work: start the loop afresh)
    eta0_issued = false;
    acur = a0;
    anext = a1;
    epoch = 0;
    if ((rc = time_loop())) return rc;
  }
  {
    int h = 0;
    CK(cudaMemcpyAsync(&h, ctx->flag, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (h) return fail(ctx, SBSE_ERR_DEVICE_TIMEOUT, "a bounded device-side wait timed out (persistent step or tensor-core cleaning)");
  }
  if (n_end < Nt) {
    // a range that stops early: the state stays in the workspace, with the current eta0 in WS_A0
    // (every step swaps the two eta0 buffers)
    if ((n_end - n_begin) % 2 == 1)
      CK(cudaMemcpyAsync(a0, a1, (size_t)L * ng * sizeof(C), cudaMemcpyDeviceToDevice, st));
    CK(cudaStreamSynchronize(st));
    ctx->run.valid = true;
    ctx->run.next = n_end;
    return SBSE_OK;
  }
  ctx->run.valid = false;
  // results into the canonical slots
  for (int k = 0; k < P; ++k)
    CK(cudaMemcpyAsync(ctx->W + (long long)slots[k] * ng, wacc + (long long)k * ng,
                       ng * sizeof(double), cudaMemcpyDeviceToDevice, st));
  CK(cudaStreamSynchronize(st));
  return SBSE_OK;
}

// out[m][n] = dV sum_r phi_xi[m].x phi_xi[m].y (r) Y_n(r): on the tensor cores (tcgen05, BF16 split,
// FP32 accumulation) in the mixed mode, in FP64 SIMT in the FP64 mode
template <typename T>
int contract(sbse_ctx *ctx, const int2 *xi_dev, int M, const T *Y, int Nn, double *out) {
  void *vp;
  int rc;
  cudaStream_t st = ctx->stream;
  if (sizeof(T) == sizeof(float) && ctx->tensor_cores) {
    const size_t gw = umma_prod_gemm_work_bytes(M, Nn, ctx->ng);
    if ((rc = ensure(ctx, WS_GEMM, gw, &vp))) return rc;
    CK(cudaMemsetAsync(ctx->flag, 0, sizeof(int), st));
    launch_umma_prod_gemm((const float *)phi_T<T>(ctx), xi_dev, M, (const float *)Y, Nn, ctx->ng,
                          ctx->dV, out, (double *)vp, ctx->flag, st);
    CHECK_LAUNCH("tensor-core contraction");
    int h = 0;
    CK(cudaMemcpyAsync(&h, ctx->flag, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (h) return fail(ctx, SBSE_ERR_DEVICE_TIMEOUT, "tensor-core contraction: wait on the MMA timed out");
    return SBSE_OK;
  }
  const size_t gw = prod_gemm_work_bytes<T>(M, Nn, ctx->ng);
  if ((rc = ensure(ctx, WS_GEMM, gw, &vp))) return rc;
  launch_prod_gemm<T>(phi_T<T>(ctx), xi_dev, M, Y, Nn, ctx->ng, ctx->dV, out, (double *)vp, gw, st);
  return SBSE_OK;
}

template <typename T> int run_build_A(sbse_ctx *ctx, unsigned terms) {
  GridTables<T> &g = tables<T>(ctx);
  const long long ng = ctx->ng;
  const int n_o = ctx->n_o, n_c = ctx->n_c, n = n_o * n_c;
  const int P = n_o * (n_o + 1) / 2;
  const int base = ctx->n_occ - n_o;
  cudaStream_t st = ctx->stream;
  int rc;
  void *vp;
  double *K = nullptr, *Dab = nullptr;
  size_t c3 = 0;
  clk_begin(ctx, 3, &c3);
  if (terms & SBSE_EXCHANGE) {
    // potentials v(phi_j phi_b) for jb = j * n_c + b, then K = dV sum_r (phi_i phi_a)(r) U_jb(r)
    const int S = (n + 1) / 2;
    std::vector<int4> pr(S);
    for (int s = 0; s < S; ++s) {
      const int m0 = 2 * s, m1 = 2 * s + 1;
      pr[s] = make_int4(base + m0 / n_c, ctx->n_occ + m0 % n_c, m1 < n ? base + m1 / n_c : -1,
                        m1 < n ? ctx->n_occ + m1 % n_c : -1);
    }
    int4 *prod;
    if ((rc = ensure(ctx, WS_IDX, std::max((size_t)S * sizeof(int4), (size_t)n * n_c * sizeof(int2) + 64),
                     &vp)))
      return rc;
    prod = (int4 *)vp;
    CK(cudaMemcpyAsync(prod, pr.data(), S * sizeof(int4), cudaMemcpyHostToDevice, st));
    C2<T> *pw;
    if ((rc = ensure(ctx, WS_PW, (size_t)S * ng * sizeof(C2<T>), &vp))) return rc;
    pw = (C2<T> *)vp;
    T *U;
    if ((rc = ensure(ctx, WS_D, (size_t)n * ng * sizeof(T) + (size_t)n_c * n_c * sizeof(int2) + 256,
                     &vp)))
      return rc;
    U = (T *)vp;
    if ((rc = poisson_products<T>(ctx, g, phi_T<T>(ctx), prod, n, pw, U, nullptr))) return rc;
    std::vector<int2> xi(n);
    for (int m = 0; m < n; ++m) xi[m] = make_int2(base + m / n_c, ctx->n_occ + m % n_c);
    int2 *xi_dev = (int2 *)prod;  // prod no longer needed after the Poisson passes above
    CK(cudaStreamSynchronize(st));
    CK(cudaMemcpyAsync(xi_dev, xi.data(), n * sizeof(int2), cudaMemcpyHostToDevice, st));
    if ((rc = ensure(ctx, WS_K, (size_t)n * n * sizeof(double), &vp))) return rc;
    K = (double *)vp;
    if ((rc = contract<T>(ctx, xi_dev, n, U, n, K))) return rc;
    CHECK_LAUNCH("exchange");
    CK(cudaStreamSynchronize(st));
  }
  if ((terms & SBSE_DIRECT) && ctx->dab_given) {
    // D columns of every pair set by sbse_set_direct (e.g. gathered from other ranks)
    if ((rc = ensure(ctx, WS_DAB, (size_t)n_c * n_c * P * sizeof(double), &vp))) return rc;
    Dab = (double *)vp;
  } else if (terms & (SBSE_DIRECT | SBSE_DIRECT_PARTIAL)) {
    for (int q = 0; q < P; ++q) {
      if (ctx->have[q]) continue;
      if (!(terms & SBSE_DIRECT_PARTIAL))
        return fail(ctx, SBSE_ERR_NOT_READY, "W missing for some pairs: call sbse_apply_W for all n_o(n_o+1)/2 pairs first");
      // a screened-out pair: its W is taken as zero
      CK(cudaMemsetAsync(ctx->W + (long long)q * ng, 0, ng * sizeof(double), st));
    }
    const int Mab = n_c * n_c;
    std::vector<int2> xi(Mab);
    for (int m = 0; m < Mab; ++m) xi[m] = make_int2(ctx->n_occ + m / n_c, ctx->n_occ + m % n_c);
    if ((rc = ensure(ctx, WS_IDX, std::max((size_t)Mab * sizeof(int2), (size_t)16), &vp))) return rc;
    int2 *xi_dev = (int2 *)vp;
    CK(cudaMemcpyAsync(xi_dev, xi.data(), Mab * sizeof(int2), cudaMemcpyHostToDevice, st));
    const T *Wt;
    if (sizeof(T) == sizeof(double)) {
      Wt = (const T *)ctx->W;
    } else {
      if ((rc = ensure(ctx, WS_U, (size_t)P * ng * sizeof(T), &vp))) return rc;
      launch_convert<T>(ctx->W, (T *)vp, (long long)P * ng, st);
      Wt = (const T *)vp;
    }
    if ((rc = ensure(ctx, WS_DAB, (size_t)Mab * P * sizeof(double), &vp))) return rc;
    Dab = (double *)vp;
    if ((rc = contract<T>(ctx, xi_dev, Mab, Wt, P, Dab))) return rc;
    CHECK_LAUNCH("direct");
  }
  clk_end(ctx, c3);
  size_t c4 = 0;
  clk_begin(ctx, 4, &c4);
  launch_assemble_A(ctx->eps_dev, ctx->eps_dev + n_o, n_o, n_c, ctx->scissor, K, Dab, P, ctx->A, st,
                    ctx->localized ? ctx->fock_o : nullptr);
  CHECK_LAUNCH("assemble_A");
  clk_end(ctx, c4);
  CK(cudaStreamSynchronize(st));
  return SBSE_OK;
}

}  // namespace

// ---- accessors for the surrogate entry points (fno.cu)
namespace sbse {
struct CtxView {
  int N, n_occ, n_o, device;
  long long ng;
  const float *phi32;
  const double *v64;
  double *W;
  cudaStream_t stream;
};
int ctx_view(sbse_ctx *ctx, CtxView *v) {
  if (!ctx || ctx->n_states == 0) return SBSE_ERR_NOT_READY;
  *v = CtxView{ctx->N, ctx->n_occ, ctx->n_o, ctx->device, ctx->ng, ctx->phi32, ctx->v64, ctx->W, ctx->stream};
  return SBSE_OK;
}
int ctx_pair_slot(sbse_ctx *ctx, int i, int j) { return pair_index(ctx->n_o, i, j); }
void ctx_mark_pair(sbse_ctx *ctx, int slot) {
  ctx->have[slot] = 1;
  ctx->have_A = false;
}
void ctx_set_error(sbse_ctx *ctx, const std::string &m) { ctx->err = m; }
bool ctx_have_pair(sbse_ctx *ctx, int slot) { return ctx->have[slot] != 0; }
int ctx_device(sbse_ctx *ctx, int *device) {
  if (!ctx) return SBSE_ERR_INVALID_ARG;
  *device = ctx->device;
  return SBSE_OK;
}
}  // namespace sbse


// =============================================================================================
// D columns (n_c^2 rows, a-major: ab = a n_c + b) of the given canonical slots into out (device,
// n_c^2 x n_slots row-major)
template <typename T> int run_direct_block(sbse_ctx *ctx, const std::vector<int> &slots, double *out) {
  const long long ng = ctx->ng;
  const int n_c = ctx->n_c, Mab = n_c * n_c, ns = (int)slots.size();
  cudaStream_t st = ctx->stream;
  void *vp;
  int rc;
  std::vector<int2> xi(Mab);
  for (int m = 0; m < Mab; ++m) xi[m] = make_int2(ctx->n_occ + m / n_c, ctx->n_occ + m % n_c);
  if ((rc = ensure(ctx, WS_IDX, (size_t)Mab * sizeof(int2), &vp))) return rc;
  int2 *xi_dev = (int2 *)vp;
  CK(cudaMemcpyAsync(xi_dev, xi.data(), Mab * sizeof(int2), cudaMemcpyHostToDevice, st));
  if ((rc = ensure(ctx, WS_U, (size_t)ns * ng * sizeof(T), &vp))) return rc;
  T *Wt = (T *)vp;
  for (int k = 0; k < ns; ++k) {
    if (sizeof(T) == sizeof(double))
      CK(cudaMemcpyAsync(Wt + (long long)k * ng, ctx->W + (long long)slots[k] * ng, ng * sizeof(double),
                         cudaMemcpyDeviceToDevice, st));
    else
      launch_convert<T>(ctx->W + (long long)slots[k] * ng, Wt + (long long)k * ng, ng, st);
  }
  CHECK_LAUNCH("direct block operands");
  return contract<T>(ctx, xi_dev, Mab, Wt, ns, out);
}

// ---- mixed hole-grid representation (Sec. II.C): A = Q A-bar on f_j(r), FP64 on the device
struct MixedBufs {
  double *tf, *dn, *dv, *pwork, *dwork;
  C2<double> *pw;
};

int mixed_bufs(sbse_ctx *ctx, int n_extra_fields, MixedBufs *mb, double **extra) {
  const long long ng = ctx->ng;
  const int n_o = ctx->n_o;
  const int nb = std::max(ctx->n_occ, ctx->n_c);
  const size_t pwd = project_work_doubles(n_o, nb, ng);
  const size_t doubles = (size_t)n_o * ng + 2 * (size_t)ng + pwd + dot_work_doubles() + (size_t)n_extra_fields * n_o * ng;
  void *vp;
  int rc;
  if ((rc = ensure(ctx, WS_MIX, doubles * sizeof(double), &vp))) return rc;
  double *p = (double *)vp;
  mb->tf = p;
  mb->dn = mb->tf + (long long)n_o * ng;
  mb->dv = mb->dn + ng;
  mb->pwork = mb->dv + ng;
  mb->dwork = mb->pwork + pwd;
  *extra = mb->dwork + dot_work_doubles();
  if ((rc = ensure(ctx, WS_PW, (size_t)((n_o + 1) / 2) * ng * sizeof(C2<double>), &vp))) return rc;
  mb->pw = (C2<double> *)vp;
  return SBSE_OK;
}

// out = Q (A-bar - shift) f for the n_o window rows f (device); projector 0: Q = 1 - P_occ, 1: onto
// the conduction states
int mixed_apply(sbse_ctx *ctx, int projector, const double *f, double *out, double shift, const MixedBufs &mb) {
  const long long ng = ctx->ng;
  const int n_o = ctx->n_o;
  const double *phi_o = ctx->phi64 + (long long)(ctx->n_occ - n_o) * ng;
  cudaStream_t st = ctx->stream;
  XfwdArgs<double> xa{};
  xa.mode = XF_PACK_DN;
  xa.n_items = (n_o + 1) / 2;
  xa.out = mb.pw;
  xa.dn = f;
  xa.n_dn = n_o;
  round_trip_poisson<double>(ctx, ctx->g64, xa, PoissonOut{n_o, 1.0, 0.0, 0.0}, mb.tf, nullptr, nullptr, Z_HALF_G2);
  launch_exciton_density(phi_o, f, n_o, ng, mb.dn, st);
  int rc;
  if ((rc = poisson<double>(ctx, ctx->g64, mb.dn, 1, mb.pw, mb.dv, nullptr, 0.0, nullptr, 0.0))) return rc;
  launch_abar(mb.tf, f, ctx->v64, ctx->eps_dev, ctx->scissor, shift, mb.dv, phi_o, ctx->W, n_o, ng, out, st);
  if (projector == 0)
    launch_project(out, n_o, ctx->phi64, ctx->n_occ, ng, ctx->dV, 0, mb.pwork, st);
  else
    launch_project(out, n_o, ctx->phi64 + (long long)ctx->n_occ * ng, ctx->n_c, ng, ctx->dV, 1, mb.pwork, st);
  CHECK_LAUNCH("mixed A");
  return SBSE_OK;
}

int mixed_ready(sbse_ctx *ctx, int projector) {
  if (ctx->n_states == 0) return fail(ctx, SBSE_ERR_NOT_READY, "call sbse_set_orbitals first");
  if (projector != 0 && projector != 1) return fail(ctx, SBSE_ERR_INVALID_ARG, "projector must be 0 or 1");
  if (ctx->localized) return fail(ctx, SBSE_ERR_UNSUPPORTED, "the mixed representation needs the canonical window");
  for (char h : ctx->have)
    if (!h) return fail(ctx, SBSE_ERR_NOT_READY, "W missing for some pairs: call sbse_apply_W for all pairs first");
  return SBSE_OK;
}

// f0_j = Q x phi_j (device)
void mixed_start(sbse_ctx *ctx, int projector, int axis, double *f0, const MixedBufs &mb) {
  const long long ng = ctx->ng;
  const int n_o = ctx->n_o;
  launch_coord_times(ctx->phi64 + (long long)(ctx->n_occ - n_o) * ng, n_o, ctx->N, ctx->h, ctx->box, axis, f0,
                     ctx->stream);
  if (projector == 0)
    launch_project(f0, n_o, ctx->phi64, ctx->n_occ, ng, ctx->dV, 0, mb.pwork, ctx->stream);
  else
    launch_project(f0, n_o, ctx->phi64 + (long long)ctx->n_occ * ng, ctx->n_c, ng, ctx->dV, 1, mb.pwork, ctx->stream);
}

// smallest and largest eigenvalue of the symmetric tridiagonal matrix (al, be) by Sturm bisection
void tridiag_extremes(const std::vector<double> &al, const std::vector<double> &be, double *lo, double *hi) {
  const int m = (int)al.size();
  double glo = INFINITY, ghi = -INFINITY;
  for (int i = 0; i < m; ++i) {
    const double r = (i > 0 ? fabs(be[i - 1]) : 0.0) + (i + 1 < m ? fabs(be[i]) : 0.0);
    glo = std::min(glo, al[i] - r);
    ghi = std::max(ghi, al[i] + r);
  }
  auto count_below = [&](double x) {  // eigenvalues < x
    int c = 0;
    double d = al[0] - x;
    if (d < 0) ++c;
    for (int i = 1; i < m; ++i) {
      if (d == 0.0) d = 1e-300;
      d = al[i] - x - be[i - 1] * be[i - 1] / d;
      if (d < 0) ++c;
    }
    return c;
  };
  auto kth = [&](int k) {  // k-th smallest eigenvalue (0-based)
    double a = glo, b = ghi;
    for (int it = 0; it < 200; ++it) {
      const double mid = 0.5 * (a + b);
      if (count_below(mid) > k) b = mid;
      else a = mid;
    }
    return 0.5 * (a + b);
  };
  *lo = kth(0);
  *hi = kth(m - 1);
}

namespace {
// layout of a saved propagation state: header, the pairs' canonical slots, then the device sections
struct StateHeader {
  char magic[8];  // "SBSESTA1"
  int precision, N, P, L, feedback, next, n_slots_pad;
  sbse_tdh_params params;
};
struct StateSection {
  int slot;
  size_t bytes;
};
std::vector<StateSection> state_sections(const sbse_ctx *ctx, int P, int L, int feedback) {
  const size_t ng = (size_t)ctx->ng, c = ctx->precision == SBSE_FP64 ? 16 : 8;
  std::vector<StateSection> s = {{WS_N0, (size_t)L * 8}, {WS_A0, L * ng * c}, {WS_D, (size_t)P * L * ng * c},
                                 {WS_WACC, (size_t)P * ng * 8}};
  if (ctx->precision != SBSE_FP64) s.push_back({WS_ACC32, (size_t)P * ng * 4});
  if (feedback) s.push_back({WS_EM1, (size_t)P * ng * c});
  return s;
}
size_t state_header_bytes(int P) { return (sizeof(StateHeader) + (size_t)P * sizeof(int) + 15) / 16 * 16; }
}  // namespace

extern "C" {

int sbse_create(sbse_ctx **out, int device, int precision) {
  if (!out) {
    g_create_error = "out is NULL";
    return SBSE_ERR_INVALID_ARG;
  }
  *out = nullptr;
  if (precision != SBSE_FP64 && precision != SBSE_MIXED) {
    g_create_error = "precision must be SBSE_FP64 or SBSE_MIXED";
    return SBSE_ERR_INVALID_ARG;
  }
  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess || device < 0 || device >= ndev) {
    g_create_error = std::string("no CUDA device ") + std::to_string(device) + ": " +
                     (e != cudaSuccess ? cudaGetErrorString(e) : "index out of range");
    cudaGetLastError();
    return e != cudaSuccess ? SBSE_ERR_CUDA : SBSE_ERR_INVALID_ARG;
  }
  sbse_ctx *c = new (std::nothrow) sbse_ctx();
  if (!c) {
    g_create_error = "host allocation failed";
    return SBSE_ERR_OOM;
  }
  c->device = device;
  c->precision = precision;
  if ((e = cudaSetDevice(device)) != cudaSuccess ||
      (e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking)) != cudaSuccess ||
      (e = cudaStreamCreateWithFlags(&c->aux, cudaStreamNonBlocking)) != cudaSuccess ||
      (e = cudaEventCreateWithFlags(&c->ev_start, cudaEventDisableTiming)) != cudaSuccess ||
      (e = cudaEventCreateWithFlags(&c->ev_a, cudaEventDisableTiming)) != cudaSuccess ||
      (e = cudaMalloc((void **)&c->flag, sizeof(int))) != cudaSuccess) {
    g_create_error = std::string("CUDA setup failed: ") + cudaGetErrorString(e);
    if (c->stream) cudaStreamDestroy(c->stream);
    delete c;
    return SBSE_ERR_CUDA;
  }
  sbse::init_fft_kernels();
  sbse::init_fast_kernels<float>();
  sbse::init_fast_kernels<double>();
  sbse::init_split_kernels();
  if (sbse::upload_reg_twiddles() != 0 || sbse::upload_split_twiddles() != 0) {
    g_create_error = "upload of the FFT twiddle tables failed";
    sbse_destroy(c);
    return SBSE_ERR_CUDA;
  }
  *out = c;
  return SBSE_OK;
}

void sbse_destroy(sbse_ctx *ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  if (ctx->graph_exec) cudaGraphExecDestroy(ctx->graph_exec);
  free_grid(ctx);
  free_scratch(ctx);
  dfree(ctx, ctx->flag);
  for (auto e : ctx->clk.ev) cudaEventDestroy(e);
  if (ctx->aux) cudaStreamSynchronize(ctx->aux);
  if (ctx->ev_start) cudaEventDestroy(ctx->ev_start);
  if (ctx->ev_a) cudaEventDestroy(ctx->ev_a);
  if (ctx->aux) cudaStreamDestroy(ctx->aux);
  if (ctx->stream) cudaStreamDestroy(ctx->stream);
  delete ctx;
}

const char *sbse_last_error(const sbse_ctx *ctx) {
  return ctx ? ctx->err.c_str() : g_create_error.c_str();
}

int sbse_get_stream(const sbse_ctx *ctx, void **stream) {
  if (!ctx || !stream) return SBSE_ERR_INVALID_ARG;
  *stream = (void *)ctx->stream;
  return SBSE_OK;
}

int sbse_set_grid(sbse_ctx *ctx, int n, double box, const double *v_loc) {
  if (!ctx) return SBSE_ERR_INVALID_ARG;
  ctx->err.clear();
  if (!v_loc) return fail(ctx, SBSE_ERR_INVALID_ARG, "v_loc is NULL");
  if (!(box > 0.0) || !isfinite(box)) return fail(ctx, SBSE_ERR_INVALID_ARG, "box must be > 0");
  FftPlan pl;
  if (n < 4 || n > kMaxN || !make_plan(n, &pl))
    return fail(ctx, SBSE_ERR_SHAPE, "grid edge must be 4..128 with prime factors 2, 3, 5");
  const long long ng = (long long)n * n * n;
  for (long long i = 0; i < ng; ++i)
    if (!isfinite(v_loc[i])) return fail(ctx, SBSE_ERR_NUMERIC, "v_loc has NaN or Inf");
  CK(cudaSetDevice(ctx->device));
  free_grid(ctx);
  ctx->N = n;
  ctx->ng = ng;
  ctx->box = box;
  ctx->h = box / n;
  ctx->dV = ctx->h * ctx->h * ctx->h;
  int rc;
  if ((rc = dalloc(ctx, &ctx->v64, ng * sizeof(double)))) return rc;
  CK(cudaMemcpyAsync(ctx->v64, v_loc, ng * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
  if ((rc = build_tables<float>(ctx, ctx->g32, v_loc))) return rc;
  if ((rc = build_tables<double>(ctx, ctx->g64, v_loc))) return rc;
  return SBSE_OK;
}

int sbse_set_orbitals(sbse_ctx *ctx, int n_occ, int n_o, int n_c, const double *phi,
                      const double *eps, double scissor) {
  if (!ctx) return SBSE_ERR_INVALID_ARG;
  ctx->err.clear();
  if (ctx->N == 0) return fail(ctx, SBSE_ERR_NOT_READY, "call sbse_set_grid first");
  if (!phi || !eps) return fail(ctx, SBSE_ERR_INVALID_ARG, "phi or eps is NULL");
  if (n_occ < 1 || n_o < 1 || n_c < 1 || n_o > n_occ)
    return fail(ctx, SBSE_ERR_INVALID_ARG, "need 1 <= n_o <= n_occ and n_c >= 1");
  if (!isfinite(scissor)) return fail(ctx, SBSE_ERR_NUMERIC, "scissor is not finite");
  const int ns = n_occ + n_c;
  const long long tot = (long long)ns * ctx->ng;
  for (int s = 0; s < ns; ++s)
    if (!isfinite(eps[s])) return fail(ctx, SBSE_ERR_NUMERIC, "eps has NaN or Inf");
  for (long long i = 0; i < tot; ++i)
    if (!isfinite(phi[i])) return fail(ctx, SBSE_ERR_NUMERIC, "phi has NaN or Inf");
  CK(cudaSetDevice(ctx->device));
  free_orbitals(ctx);
  int rc;
  if ((rc = dalloc(ctx, &ctx->phi64, tot * sizeof(double)))) return rc;
  CK(cudaMemcpyAsync(ctx->phi64, phi, tot * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
  if ((rc = dalloc(ctx, &ctx->phi32, tot * sizeof(float)))) return rc;
  launch_convert<float>(ctx->phi64, ctx->phi32, tot, ctx->stream);
  CHECK_LAUNCH("convert phi");
  std::vector<double> ew(n_o + n_c);
  for (int i = 0; i < n_o; ++i) ew[i] = eps[n_occ - n_o + i];
  for (int a = 0; a < n_c; ++a) ew[n_o + a] = eps[n_occ + a];
  if ((rc = dalloc(ctx, &ctx->eps_dev, ew.size() * sizeof(double)))) return rc;
  CK(cudaMemcpyAsync(ctx->eps_dev, ew.data(), ew.size() * sizeof(double), cudaMemcpyHostToDevice,
                     ctx->stream));
  ctx->n_occ = n_occ;
  ctx->n_o = n_o;
  ctx->n_c = n_c;
  ctx->n_states = ns;
  ctx->scissor = scissor;
  ctx->eps.assign(eps, eps + ns);
  const int P = n_o * (n_o + 1) / 2;
  if ((rc = dalloc(ctx, &ctx->W, (size_t)P * ctx->ng * sizeof(double)))) return rc;
  ctx->have.assign(P, 0);
  const int n = n_o * n_c;
  if ((rc = dalloc(ctx, &ctx->A, (size_t)n * n * sizeof(double)))) return rc;
  CK(cudaStreamSynchronize(ctx->stream));
  return SBSE_OK;
}

int sbse_coefficients(uint64_t seed, int n_s, int n_occ, int dist, double *out) {
  if (!out || n_s < 1 || n_occ < 1 || (dist != SBSE_COEFF_GAUSSIAN && dist != SBSE_COEFF_SIGN))
    return SBSE_ERR_INVALID_ARG;
  const double two53 = 1.0 / 9007199254740992.0;
  for (int l = 0; l < n_s; ++l)
    for (int s = 0; s < n_occ; ++s) {
      const uint64_t idx = (uint64_t)l * n_occ + s;
      double c;
      if (dist == SBSE_COEFF_SIGN) {
        c = (splitmix64_out(seed, idx) >> 63) ? -1.0 : 1.0;
      } else {
        const double u1 = (double)(splitmix64_out(seed, 2 * idx) >> 11) * two53;
        const double u2 = (double)(splitmix64_out(seed, 2 * idx + 1) >> 11) * two53;
        c = sqrt(-2.0 * log(1.0 - u1)) * cos(2.0 * M_PI * u2);
      }
      out[(size_t)l * n_occ + s] = c;
    }
  return SBSE_OK;
}

int sbse_apply_W(sbse_ctx *ctx, const sbse_tdh_params *p, int n_pairs, const int *pi, const int *pj,
                 const double *coeff, double *w_out) {
  return sbse_apply_W_range(ctx, p, n_pairs, pi, pj, coeff, w_out, 0, p ? p->n_steps : 0);
}

int sbse_apply_W_range(sbse_ctx *ctx, const sbse_tdh_params *p, int n_pairs, const int *pi, const int *pj,
                       const double *coeff, double *w_out, int n_begin, int n_end) {
  if (!ctx) return SBSE_ERR_INVALID_ARG;
  ctx->err.clear();
  if (ctx->n_states == 0) return fail(ctx, SBSE_ERR_NOT_READY, "call sbse_set_orbitals first");
  if (!p || !pi || !pj || n_pairs < 1) return fail(ctx, SBSE_ERR_INVALID_ARG, "params/pairs missing");
  if (p->n_s < 1 || p->n_s > 64) return fail(ctx, SBSE_ERR_INVALID_ARG, "n_s must be 1..64");
  if (p->n_steps < 1) return fail(ctx, SBSE_ERR_INVALID_ARG, "n_steps must be >= 1");
  if (p->clean_every < 0) return fail(ctx, SBSE_ERR_INVALID_ARG, "clean_every must be >= 0");
  if (!(p->dt > 0.0) || !(p->alpha > 0.0) || !(p->gamma >= 0.0) || !isfinite(p->dt) ||
      !isfinite(p->alpha) || !isfinite(p->gamma))
    return fail(ctx, SBSE_ERR_INVALID_ARG, "need dt > 0, alpha > 0, gamma >= 0");
  if (p->coeff_dist != SBSE_COEFF_GAUSSIAN && p->coeff_dist != SBSE_COEFF_SIGN)
    return fail(ctx, SBSE_ERR_INVALID_ARG, "coeff_dist must be GAUSSIAN or SIGN");
  const int P_all = ctx->n_o * (ctx->n_o + 1) / 2;
  if (n_pairs > P_all) return fail(ctx, SBSE_ERR_INVALID_ARG, "more pairs than n_o(n_o+1)/2");
  std::vector<int> slots(n_pairs);
  std::vector<char> seen(P_all, 0);
  for (int k = 0; k < n_pairs; ++k) {
    if (pi[k] < 0 || pj[k] < pi[k] || pj[k] >= ctx->n_o)
      return fail(ctx, SBSE_ERR_INVALID_ARG, "pair indices must satisfy 0 <= i <= j < n_o");
    slots[k] = pair_index(ctx->n_o, pi[k], pj[k]);
    if (seen[slots[k]]) return fail(ctx, SBSE_ERR_INVALID_ARG, "duplicate pair");
    seen[slots[k]] = 1;
  }
  std::vector<double> c((size_t)p->n_s * ctx->n_occ);
  if (coeff) {
    for (size_t i = 0; i < c.size(); ++i) {
      if (!isfinite(coeff[i])) return fail(ctx, SBSE_ERR_NUMERIC, "coeff has NaN or Inf");
      c[i] = coeff[i];
    }
  } else {
    sbse_coefficients(p->seed, p->n_s, ctx->n_occ, p->coeff_dist, c.data());
  }
  if (n_begin < 0 || n_end <= n_begin || n_end > p->n_steps)
    return fail(ctx, SBSE_ERR_INVALID_ARG, "need 0 <= n_begin < n_end <= n_steps");
  auto same = [](const sbse_tdh_params &x, const sbse_tdh_params &y) {
    return x.n_s == y.n_s && x.n_steps == y.n_steps && x.clean_every == y.clean_every && x.dt == y.dt &&
           x.gamma == y.gamma && x.alpha == y.alpha && x.seed == y.seed && x.coeff_dist == y.coeff_dist &&
           x.feedback == y.feedback;
  };
  if (n_begin > 0 && !(ctx->run.valid && ctx->run.next == n_begin && ctx->run.slots == slots &&
                       same(ctx->run.params, *p)))
    return fail(ctx, SBSE_ERR_NOT_READY,
                "no propagation state of these parameters and pairs stopped at n_begin (run the range before it "
                "or load its state)");
  CK(cudaSetDevice(ctx->device));
  ctx->have_A = false;
  if (n_begin == 0) ctx->run.valid = false;
  ctx->run.params = *p;
  ctx->run.slots = slots;
  const int rc = ctx->precision == SBSE_FP64 ? run_apply_W<double>(ctx, p, slots, c, n_begin, n_end)
                                             : run_apply_W<float>(ctx, p, slots, c, n_begin, n_end);
  if (rc) {
    ctx->run.valid = false;
    return rc;
  }
  if (n_end < p->n_steps) return SBSE_OK;  // W is stored when the last step has run
  for (int k = 0; k < n_pairs; ++k) {
    if (scan_nonfinite(ctx->W + (long long)slots[k] * ctx->ng, ctx->ng, ctx->flag, ctx->stream))
      return fail(ctx, SBSE_ERR_NUMERIC, "W has NaN or Inf (unstable propagation: reduce dt)");
    ctx->have[slots[k]] = 1;
    ctx->dab_given = false;
  }
  if (w_out)
    for (int k = 0; k < n_pairs; ++k)
      CK(cudaMemcpy(w_out + (long long)k * ctx->ng, ctx->W + (long long)slots[k] * ctx->ng,
                    ctx->ng * sizeof(double), cudaMemcpyDeviceToHost));
  return SBSE_OK;
}


int sbse_state_bytes(sbse_ctx *ctx, size_t *bytes) {
  if (!ctx || !bytes) return SBSE_ERR_INVALID_ARG;
  ctx->err.clear();
  if (!ctx->run.valid) return fail(ctx, SBSE_ERR_NOT_READY, "no propagation stopped part way in this context");
  const int P = (int)ctx->run.slots.size(), L = ctx->run.params.n_s;
  size_t b = state_header_bytes(P);
  for (const auto &s : state_sections(ctx, P, L, ctx->run.params.feedback)) b += s.bytes;
  *bytes = b;
  return SBSE_OK;
}

int sbse_save_state(sbse_ctx *ctx, void *host, size_t bytes) {
  size_t need = 0;
  int rc = sbse_state_bytes(ctx, &need);
  if (rc) return rc;
  if (!host || bytes < need) return fail(ctx, SBSE_ERR_INVALID_ARG, "state buffer missing or smaller than sbse_state_bytes");
  const int P = (int)ctx->run.slots.size(), L = ctx->run.params.n_s;
  StateHeader h{};
  memcpy(h.magic, "SBSESTA1", 8);
  h.precision = ctx->precision;
  h.N = ctx->N;
  h.P = P;
  h.L = L;
  h.feedback = ctx->run.params.feedback;
  h.next = ctx->run.next;
  h.params = ctx->run.params;
  uint8_t *o = static_cast<uint8_t *>(host);
  memcpy(o, &h, sizeof h);
  memcpy(o + sizeof h, ctx->run.slots.data(), (size_t)P * sizeof(int));
  size_t off = state_header_bytes(P);
  CK(cudaSetDevice(ctx->device));
  for (const auto &s : state_sections(ctx, P, L, h.feedback)) {
    CK(cudaMemcpyAsync(o + off, ctx->ws[s.slot].p, s.bytes, cudaMemcpyDeviceToHost, ctx->stream));
    off += s.bytes;
  }
  CK(cudaStreamSynchronize(ctx->stream));
  return SBSE_OK;
}

int sbse_load_state(sbse_ctx *ctx, const void *host, size_t bytes) {
  if (!ctx) return SBSE_ERR_INVALID_ARG;
  ctx->err.clear();
  if (ctx->n_states == 0) return fail(ctx, SBSE_ERR_NOT_READY, "call sbse_set_orbitals first");
  StateHeader h{};
  if (!host || bytes < sizeof h) return fail(ctx, SBSE_ERR_INVALID_ARG, "state buffer missing or too small");
  const uint8_t *in = static_cast<const uint8_t *>(host);
  memcpy(&h, in, sizeof h);
  if (memcmp(h.magic, "SBSESTA1", 8) != 0) return fail(ctx, SBSE_ERR_INVALID_ARG, "not a saved propagation state");
  if (h.precision != ctx->precision || h.N != ctx->N)
    return fail(ctx, SBSE_ERR_SHAPE, "state saved on another grid or in another precision mode");
  const int P_all = ctx->n_o * (ctx->n_o + 1) / 2;
  if (h.P < 1 || h.P > P_all || h.L < 1 || h.L > 64 || h.next < 1 || h.next >= h.params.n_steps)
    return fail(ctx, SBSE_ERR_INVALID_ARG, "state header out of range for this context");
  size_t need = state_header_bytes(h.P);
  const auto secs = state_sections(ctx, h.P, h.L, h.feedback);
  for (const auto &s : secs) need += s.bytes;
  if (bytes < need) return fail(ctx, SBSE_ERR_INVALID_ARG, "state buffer shorter than its header says");
  std::vector<int> slots(h.P);
  memcpy(slots.data(), in + sizeof h, (size_t)h.P * sizeof(int));
  for (int s : slots)
    if (s < 0 || s >= P_all) return fail(ctx, SBSE_ERR_INVALID_ARG, "state holds a pair outside the window");
  CK(cudaSetDevice(ctx->device));
  size_t off = state_header_bytes(h.P);
  for (const auto &s : secs) {
    void *vp;
    int rc;
    if ((rc = ensure(ctx, s.slot, s.bytes, &vp))) return rc;
    CK(cudaMemcpyAsync(vp, in + off, s.bytes, cudaMemcpyHostToDevice, ctx->stream));
    off += s.bytes;
  }
  CK(cudaStreamSynchronize(ctx->stream));
  ctx->run.valid = true;
  ctx->run.next = h.next;
  ctx->run.params = h.params;
  ctx->run.slots = slots;
  return SBSE_OK;
}

int sbse_bare_W(sbse_ctx *ctx, int n_pairs, const int *pi, const int *pj) {
  if (!ctx) return SBSE_ERR_INVALID_ARG;
  ctx->err.clear();
  if (ctx->n_states == 0) return fail(ctx, SBSE_ERR_NOT_READY, "call sbse_set_orbitals first");
  if (!pi || !pj || n_pairs < 1) return fail(ctx, SBSE_ERR_INVALID_ARG, "pairs missing");
  const int P_all = ctx->n_o * (ctx->n_o + 1) / 2;
  if (n_pairs > P_all) return fail(ctx, SBSE_ERR_INVALID_ARG, "more pairs than n_o(n_o+1)/2");
  std::vector<int> slots(n_pairs);
  std::vector<char> seen(P_all, 0);
  for (int k = 0; k < n_pairs; ++k) {
    if (pi[k] < 0 || pj[k] < pi[k] || pj[k] >= ctx->n_o)
      return fail(ctx, SBSE_ERR_INVALID_ARG, "pair indices must satisfy 0 <= i <= j < n_o");
    slots[k] = pair_index(ctx->n_o, pi[k], pj[k]);
    if (seen[slots[k]]) return fail(ctx, SBSE_ERR_INVALID_ARG, "duplicate pair");
    seen[slots[k]] = 1;
  }
  CK(cudaSetDevice(ctx->device));
  const long long ng = ctx->ng;
  const int S = (n_pairs + 1) / 2;
  const int base = ctx->n_occ - ctx->n_o;
  void *vp;
  int rc;
  if ((rc = ensure(ctx, WS_IDX, (size_t)S * sizeof(int4), &vp))) return rc;
  int4 *prod = (int4 *)vp;
  if ((rc = ensure(ctx, WS_PW, (size_t)S * ng * sizeof(C2<double>), &vp))) return rc;
  C2<double> *pw = (C2<double> *)vp;
  if ((rc = ensure(ctx, WS_WACC, (size_t)n_pairs * ng * sizeof(double), &vp))) return rc;
  double *q = (double *)vp;
  std::vector<int4> pr(S);
  for (int s = 0; s < S; ++s) {
    const int k0 = 2 * s, k1 = 2 * s + 1;
    pr[s] = make_int4(base + pi[k0], base + pj[k0], k1 < n_pairs ? base + pi[k1] : -1,
                      k1 < n_pairs ? base + pj[k1] : -1);
  }
  CK(cudaMemcpyAsync(prod, pr.data(), S * sizeof(int4), cudaMemcpyHostToDevice, ctx->stream));
  // q_ij = v (phi_i phi_j), FP64, the orbitals of the FP64 tables whatever the precision mode
  if ((rc = poisson_products<double>(ctx, ctx->g64, ctx->phi64, prod, n_pairs, pw, nullptr, q))) return rc;
  for (int k = 0; k < n_pairs; ++k) {
    CK(cudaMemcpyAsync(ctx->W + (long long)slots[k] * ng, q + (long long)k * ng, ng * sizeof(double),
                       cudaMemcpyDeviceToDevice, ctx->stream));
    ctx->have[slots[k]] = 1;
  }
  ctx->dab_given = false;
  ctx->have_A = false;
  CK(cudaStreamSynchronize(ctx->stream));
  return SBSE_OK;
}

int sbse_get_W(sbse_ctx *ctx, int n_pairs, const int *pi, const int *pj, double *w) {
  if (!ctx) return SBSE_ERR_INVALID_ARG;
  ctx->err.clear();
  if (ctx->n_states == 0) return fail(ctx, SBSE_ERR_NOT_READY, "call sbse_set_orbitals first");
  if (!pi || !pj || !w || n_pairs < 1) return fail(ctx, SBSE_ERR_INVALID_ARG, "pairs or w missing");
  CK(cudaSetDevice(ctx->device));
  for (int k = 0; k < n_pairs; ++k) {
    if (pi[k] < 0 || pj[k] < pi[k] || pj[k] >= ctx->n_o)
      return fail(ctx, SBSE_ERR_INVALID_ARG, "pair indices must satisfy 0 <= i <= j < n_o");
    const int slot = pair_index(ctx->n_o, pi[k], pj[k]);
    if (!ctx->have[slot]) return fail(ctx, SBSE_ERR_NOT_READY, "W of a requested pair is not available");
    CK(cudaMemcpy(w + (long long)k * ctx->ng, ctx->W + (long long)slot * ctx->ng, ctx->ng * sizeof(double),
                  cudaMemcpyDeviceToHost));
  }
  return SBSE_OK;
}

int sbse_set_W(sbse_ctx *ctx, int n_pairs, const int *pi, const int *pj, const double *w) {
  if (!ctx) return SBSE_ERR_INVALID_ARG;
  ctx->err.clear();
  if (ctx->n_states == 0) return fail(ctx, SBSE_ERR_NOT_READY, "call sbse_set_orbitals first");
  if (!pi || !pj || !w || n_pairs < 1) return fail(ctx, SBSE_ERR_INVALID_ARG, "pairs or w missing");
  std::vector<int> slots(n_pairs);
  for (int k = 0; k < n_pairs; ++k) {
    if (pi[k] < 0 || pj[k] < pi[k] || pj[k] >= ctx->n_o)
      return fail(ctx, SBSE_ERR_INVALID_ARG, "pair indices must satisfy 0 <= i <= j < n_o");
    slots[k] = pair_index(ctx->n_o, pi[k], pj[k]);
  }
  const long long tot = (long long)n_pairs * ctx->ng;
  for (long long i = 0; i < tot; ++i)
    if (!isfinite(w[i])) return fail(ctx, SBSE_ERR_NUMERIC, "w has NaN or Inf");
  CK(cudaSetDevice(ctx->device));
  for (int k = 0; k < n_pairs; ++k) {
    CK(cudaMemcpyAsync(ctx->W + (long long)slots[k] * ctx->ng, w + (long long)k * ctx->ng,
                       ctx->ng * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    ctx->have[slots[k]] = 1;
    ctx->dab_given = false;
  }
  ctx->have_A = false;
  CK(cudaStreamSynchronize(ctx->stream));
  return SBSE_OK;
}

int sbse_get_direct(sbse_ctx *ctx, int n_pairs, const int *pi, const int *pj, double *dab) {
  if (!ctx) return SBSE_ERR_INVALID_ARG;
  ctx->err.clear();
  if (ctx->n_states == 0) return fail(ctx, SBSE_ERR_NOT_READY, "call sbse_set_orbitals first");
  if (!pi || !pj || !dab || n_pairs < 1) return fail(ctx, SBSE_ERR_INVALID_ARG, "pairs or dab missing");
  std::vector<int> slots(n_pairs);
  for (int k = 0; k < n_pairs; ++k) {
    if (pi[k] < 0 || pj[k] < pi[k] || pj[k] >= ctx->n_o)
      return fail(ctx, SBSE_ERR_INVALID_ARG, "pair indices must satisfy 0 <= i <= j < n_o");
    slots[k] = pair_index(ctx->n_o, pi[k], pj[k]);
    if (!ctx->have[slots[k]]) return fail(ctx, SBSE_ERR_NOT_READY, "W of a requested pair is not available");
  }
  CK(cudaSetDevice(ctx->device));
  const size_t bytes = (size_t)ctx->n_c * ctx->n_c * n_pairs * sizeof(double);
  void *vp;
  int rc;
  if ((rc = ensure(ctx, WS_DBLK, bytes, &vp))) return rc;
  rc = ctx->precision == SBSE_FP64 ? run_direct_block<double>(ctx, slots, (double *)vp)
                                   : run_direct_block<float>(ctx, slots, (double *)vp);
  if (rc) return rc;
  CK(cudaMemcpyAsync(dab, vp, bytes, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return SBSE_OK;
}

int sbse_set_direct(sbse_ctx *ctx, const double *dab) {
  if (!ctx) return SBSE_ERR_INVALID_ARG;
  ctx->err.clear();
  if (ctx->n_states == 0) return fail(ctx, SBSE_ERR_NOT_READY, "call sbse_set_orbitals first");
  if (!dab) return fail(ctx, SBSE_ERR_INVALID_ARG, "dab missing");
  const int P = ctx->n_o * (ctx->n_o + 1) / 2;
  const size_t cnt = (size_t)ctx->n_c * ctx->n_c * P;
  for (size_t i = 0; i < cnt; ++i)
    if (!isfinite(dab[i])) return fail(ctx, SBSE_ERR_NUMERIC, "dab has NaN or Inf");
  CK(cudaSetDevice(ctx->device));
  void *vp;
  int rc;
  if ((rc = ensure(ctx, WS_DAB, cnt * sizeof(double), &vp))) return rc;
  CK(cudaMemcpyAsync(vp, dab, cnt * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  ctx->dab_given = true;
  ctx->have_A = false;
  return SBSE_OK;
}

int sbse_build_A(sbse_ctx *ctx, unsigned terms, double *a_out) {
  if (!ctx) return SBSE_ERR_INVALID_ARG;
  ctx->err.clear();
  if (ctx->n_states == 0) return fail(ctx, SBSE_ERR_NOT_READY, "call sbse_set_orbitals first");
  if (terms & ~(SBSE_EXCHANGE | SBSE_DIRECT | SBSE_DIRECT_PARTIAL))
    return fail(ctx, SBSE_ERR_INVALID_ARG, "unknown terms bits");
  CK(cudaSetDevice(ctx->device));
  const int rc = ctx->precision == SBSE_FP64 ? run_build_A<double>(ctx, terms)
                                             : run_build_A<float>(ctx, terms);
  if (rc) return rc;
  ctx->have_A = true;
  const int n = ctx->n_o * ctx->n_c;
  if (a_out) CK(cudaMemcpy(a_out, ctx->A, (size_t)n * n * sizeof(double), cudaMemcpyDeviceToHost));
  return SBSE_OK;
}

int sbse_spectrum(sbse_ctx *ctx, int k, double *evals, double *evecs) {
  if (!ctx) return SBSE_ERR_INVALID_ARG;
  ctx->err.clear();
  if (!ctx->have_A) return fail(ctx, SBSE_ERR_NOT_READY, "call sbse_build_A first");
  const int n = ctx->n_o * ctx->n_c;
  if (!evals || k < 1 || k > n) return fail(ctx, SBSE_ERR_INVALID_ARG, "need evals and 1 <= k <= n_o n_c");
  CK(cudaSetDevice(ctx->device));
  void *vp;
  int rc;
  if (evecs) {
    const size_t wb = (eig_vectors_work_bytes(n, k) + 255) / 256 * 256;
    if ((rc = ensure(ctx, WS_EIG, wb + (size_t)(k + (size_t)n * k) * sizeof(double), &vp))) return rc;
    double *ev = (double *)((char *)vp + wb), *vec = ev + k;
    size_t c4 = 0;
    clk_begin(ctx, 4, &c4);
    launch_eig_vectors(ctx->A, n, k, ev, vec, (double *)vp, ctx->stream);
    CHECK_LAUNCH("eig vectors");
    clk_end(ctx, c4);
    CK(cudaMemcpyAsync(evals, ev, k * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(evecs, vec, (size_t)n * k * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    for (long long i = 0; i < (long long)n * k; ++i)
      if (!isfinite(evecs[i])) return fail(ctx, SBSE_ERR_NUMERIC, "eigenvector is not finite");
    for (int i = 0; i < k; ++i)
      if (!isfinite(evals[i])) return fail(ctx, SBSE_ERR_NUMERIC, "eigenvalue is not finite");
    return SBSE_OK;
  }
  if ((rc = ensure(ctx, WS_EIG, eig_work_bytes(n) + (size_t)(k + 1) * sizeof(double), &vp))) return rc;
  double *ev = (double *)vp + (long long)n * n + 2 * n;
  size_t c4 = 0;
  clk_begin(ctx, 4, &c4);
  launch_eig_lowest(ctx->A, n, k, ev, (double *)vp, ctx->stream);
  CHECK_LAUNCH("eig");
  clk_end(ctx, c4);
  CK(cudaMemcpyAsync(evals, ev, k * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  for (int i = 0; i < k; ++i)
    if (!isfinite(evals[i])) return fail(ctx, SBSE_ERR_NUMERIC, "eigenvalue is not finite");
  return SBSE_OK;
}

int sbse_boundary_potential(sbse_ctx *ctx, double *v_bndry) {
  if (!ctx) return SBSE_ERR_INVALID_ARG;
  ctx->err.clear();
  if (!v_bndry) return fail(ctx, SBSE_ERR_INVALID_ARG, "v_bndry missing");
  if (ctx->n_states == 0) return fail(ctx, SBSE_ERR_NOT_READY, "call sbse_set_orbitals first");
  CK(cudaSetDevice(ctx->device));
  const long long ng = ctx->ng;
  cudaStream_t st = ctx->stream;
  void *vp;
  int rc;
  // n0 and u (ng each), the block partial sums and the two totals
  if ((rc = ensure(ctx, WS_FBOX, (2 * (size_t)ng + 2 * 256 + 2) * sizeof(double), &vp))) return rc;
  double *n0 = (double *)vp, *u = n0 + ng, *part = u + ng, *sums = part + 2 * 256;
  if ((rc = ensure(ctx, WS_PW, (size_t)ng * sizeof(C2<double>), &vp))) return rc;
  launch_ground_density(ctx->phi64, ctx->n_occ, ng, n0, st);
  if ((rc = poisson<double>(ctx, ctx->g64, n0, 1, (C2<double> *)vp, u, nullptr, 0.0, nullptr, 0.0))) return rc;
  launch_box_sums(ctx->v64, u, ctx->N, part, sums, st);
  CHECK_LAUNCH("boundary potential");
  double h[2];
  CK(cudaMemcpyAsync(h, sums, sizeof(h), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  const double nb = 3.0 * ctx->N * (double)ctx->N - 3.0 * ctx->N + 1.0;
  *v_bndry = h[1] / nb - h[0] / (double)ng;
  if (!isfinite(*v_bndry)) return fail(ctx, SBSE_ERR_NUMERIC, "boundary potential is not finite");
  return SBSE_OK;
}

int sbse_fit_inverse_dielectric(int n_box, int k, const double *E, const double *v, double *eps_inv) {
  if (n_box < 2 || k < 1 || !E || !v || !eps_inv) {
    sbse::set_thread_error("need n_box >= 2, k >= 1 and non-null E, v, eps_inv");
    return SBSE_ERR_INVALID_ARG;
  }
  double vbar = 0.0;
  for (int b = 0; b < n_box; ++b) vbar += v[b];
  vbar /= n_box;
  double num = 0.0, den = 0.0;
  for (int b = 0; b < n_box; ++b) den += (v[b] - vbar) * (v[b] - vbar);
  for (int j = 0; j < k; ++j) {
    double ebar = 0.0;
    for (int b = 0; b < n_box; ++b) ebar += E[(long long)b * k + j];
    ebar /= n_box;
    for (int b = 0; b < n_box; ++b) num += (E[(long long)b * k + j] - ebar) * (v[b] - vbar);
  }
  if (!(den > 0.0)) {
    sbse::set_thread_error("the boundary potentials of the boxes must differ");
    return SBSE_ERR_INVALID_ARG;
  }
  *eps_inv = num / (k * den);
  return SBSE_OK;
}

int sbse_localize_occupied(sbse_ctx *ctx, int max_sweeps, double tol, double *U_out) {
  if (!ctx) return SBSE_ERR_INVALID_ARG;
  ctx->err.clear();
  if (ctx->n_states == 0) return fail(ctx, SBSE_ERR_NOT_READY, "call sbse_set_orbitals first");
  if (max_sweeps < 1 || !(tol >= 0.0)) return fail(ctx, SBSE_ERR_INVALID_ARG, "need max_sweeps >= 1, tol >= 0");
  CK(cudaSetDevice(ctx->device));
  const int n = ctx->n_o, P = n * (n + 1) / 2, base = ctx->n_occ - n;
  const long long ng = ctx->ng;
  cudaStream_t st = ctx->stream;
  void *vp;
  int rc;
  // the spread matrices Z_alpha,ij = dV sum_r phi_i phi_j exp(i 2 pi x_alpha / L), i <= j: a grid sum
  // of the window's pair products against the six fields cos, sin(2 pi x_alpha / L)
  if ((rc = ensure(ctx, WS_LOC, (6 * (size_t)ng + (size_t)n * ng + 6 * (size_t)P + 2 * (size_t)n * n) * sizeof(double), &vp)))
    return rc;
  double *fields = (double *)vp, *rot = fields + 6 * ng, *zout = rot + (long long)n * ng, *Udev = zout + 6 * P;
  std::vector<int2> xi(P);
  for (int i = 0, p = 0; i < n; ++i)
    for (int j = i; j < n; ++j, ++p) xi[p] = make_int2(base + i, base + j);
  if ((rc = ensure(ctx, WS_IDX, (size_t)P * sizeof(int2), &vp))) return rc;
  int2 *xi_dev = (int2 *)vp;
  CK(cudaMemcpyAsync(xi_dev, xi.data(), P * sizeof(int2), cudaMemcpyHostToDevice, st));
  launch_phase_fields(ctx->N, fields, st);
  const size_t gw = prod_gemm_work_bytes<double>(P, 6, ng);
  if ((rc = ensure(ctx, WS_GEMM, gw, &vp))) return rc;
  launch_prod_gemm<double>(ctx->phi64, xi_dev, P, fields, 6, ng, ctx->dV, zout, (double *)vp, gw, st);
  CHECK_LAUNCH("spread matrices");
  std::vector<double> zh(6 * (size_t)P);
  CK(cudaMemcpyAsync(zh.data(), zout, zh.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  // Jacobi maximisation of sum_alpha sum_k |Z_alpha,kk|^2 over orthogonal rotations (host)
  std::vector<double> zr(3 * (size_t)n * n), zi(3 * (size_t)n * n), U((size_t)n * n, 0.0);
  for (int i = 0, p = 0; i < n; ++i)
    for (int j = i; j < n; ++j, ++p)
      for (int a = 0; a < 3; ++a) {
        zr[((size_t)a * n + i) * n + j] = zr[((size_t)a * n + j) * n + i] = zh[(size_t)p * 6 + 2 * a];
        zi[((size_t)a * n + i) * n + j] = zi[((size_t)a * n + j) * n + i] = zh[(size_t)p * 6 + 2 * a + 1];
      }
  for (int i = 0; i < n; ++i) U[(size_t)i * n + i] = 1.0;
  auto functional = [&]() {
    double f = 0.0;
    for (int a = 0; a < 3; ++a)
      for (int k = 0; k < n; ++k) {
        const size_t d = ((size_t)a * n + k) * n + k;
        f += zr[d] * zr[d] + zi[d] * zi[d];
      }
    return f;
  };
  double prev = functional();
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    for (int i = 0; i < n - 1; ++i)
      for (int j = i + 1; j < n; ++j) {
        double Pv = 0.0, Qv = 0.0, Rv = 0.0;
        for (int a = 0; a < 3; ++a) {
          const size_t ii = ((size_t)a * n + i) * n + i, jj = ((size_t)a * n + j) * n + j, ij = ((size_t)a * n + i) * n + j;
          const double ur = 0.5 * (zr[ii] - zr[jj]), ui = 0.5 * (zi[ii] - zi[jj]);
          Pv += ur * ur + ui * ui;
          Qv += zr[ij] * zr[ij] + zi[ij] * zi[ij];
          Rv += ur * zr[ij] + ui * zi[ij];
        }
        const double theta = 0.25 * atan2(Rv, 0.5 * (Pv - Qv));
        if (fabs(theta) < 1e-15) continue;
        const double c = cos(theta), sn = sin(theta);
        // new i = c i + s j, new j = -s i + c j: columns, then rows of each Z_alpha, then U
        for (int a = 0; a < 3; ++a)
          for (double *z : {zr.data(), zi.data()}) {
            double *Z = z + (size_t)a * n * n;
            for (int k = 0; k < n; ++k) {
              const double zki = Z[(size_t)k * n + i], zkj = Z[(size_t)k * n + j];
              Z[(size_t)k * n + i] = c * zki + sn * zkj;
              Z[(size_t)k * n + j] = -sn * zki + c * zkj;
            }
            for (int k = 0; k < n; ++k) {
              const double zik = Z[(size_t)i * n + k], zjk = Z[(size_t)j * n + k];
              Z[(size_t)i * n + k] = c * zik + sn * zjk;
              Z[(size_t)j * n + k] = -sn * zik + c * zjk;
            }
          }
        for (int k = 0; k < n; ++k) {
          const double uki = U[(size_t)k * n + i], ukj = U[(size_t)k * n + j];
          U[(size_t)k * n + i] = c * uki + sn * ukj;
          U[(size_t)k * n + j] = -sn * uki + c * ukj;
        }
      }
    const double f = functional();
    const bool done = f - prev <= tol * std::max(1.0, fabs(f));
    prev = f;
    if (done) break;
  }
  // rotate the window rows on the device, refresh the FP32 copy; F = U^T diag(eps_o) U
  std::vector<double> F((size_t)n * n);
  for (int k = 0; k < n; ++k)
    for (int l = 0; l < n; ++l) {
      double v = 0.0;
      for (int i = 0; i < n; ++i) v += U[(size_t)i * n + k] * ctx->eps[base + i] * U[(size_t)i * n + l];
      F[(size_t)k * n + l] = v;
    }
  if (!ctx->fock_o && (rc = dalloc(ctx, &ctx->fock_o, (size_t)n * n * sizeof(double)))) return rc;
  CK(cudaMemcpyAsync(Udev, U.data(), U.size() * sizeof(double), cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(ctx->fock_o, F.data(), F.size() * sizeof(double), cudaMemcpyHostToDevice, st));
  launch_rotate_rows(ctx->phi64, base, n, Udev, ng, rot, st);
  CK(cudaMemcpyAsync(ctx->phi64 + (long long)base * ng, rot, (size_t)n * ng * sizeof(double), cudaMemcpyDeviceToDevice, st));
  launch_convert<float>(ctx->phi64 + (long long)base * ng, ctx->phi32 + (long long)base * ng, (long long)n * ng, st);
  CHECK_LAUNCH("rotate window");
  std::fill(ctx->have.begin(), ctx->have.end(), 0);
  ctx->dab_given = false;
  ctx->have_A = false;
  ctx->localized = true;
  if (U_out) std::copy(U.begin(), U.end(), U_out);
  CK(cudaStreamSynchronize(st));
  return SBSE_OK;
}

int sbse_pair_weights(sbse_ctx *ctx, double *w_out) {
  if (!ctx) return SBSE_ERR_INVALID_ARG;
  ctx->err.clear();
  if (!w_out) return fail(ctx, SBSE_ERR_INVALID_ARG, "w_out missing");
  if (ctx->n_states == 0) return fail(ctx, SBSE_ERR_NOT_READY, "call sbse_set_orbitals first");
  CK(cudaSetDevice(ctx->device));
  const int n = ctx->n_o, P = n * (n + 1) / 2, base = ctx->n_occ - n;
  cudaStream_t st = ctx->stream;
  void *vp;
  int rc;
  std::vector<int2> xi(P);
  for (int i = 0, p = 0; i < n; ++i)
    for (int j = i; j < n; ++j, ++p) xi[p] = make_int2(base + i, base + j);
  if ((rc = ensure(ctx, WS_IDX, (size_t)P * sizeof(int2), &vp))) return rc;
  int2 *xi_dev = (int2 *)vp;
  CK(cudaMemcpyAsync(xi_dev, xi.data(), P * sizeof(int2), cudaMemcpyHostToDevice, st));
  if ((rc = ensure(ctx, WS_LOC, (pair_norms_work_doubles(P) + P) * sizeof(double), &vp))) return rc;
  double *work = (double *)vp, *out = work + pair_norms_work_doubles(P);
  launch_pair_norms(ctx->phi64, xi_dev, P, ctx->ng, ctx->dV, work, out, st);
  CHECK_LAUNCH("pair norms");
  CK(cudaMemcpyAsync(w_out, out, P * sizeof(double), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  for (int p = 0; p < P; ++p) w_out[p] = sqrt(w_out[p]);
  return SBSE_OK;
}

int sbse_apply_A_mixed(sbse_ctx *ctx, int projector, const double *f_in, double *f_out) {
  if (!ctx) return SBSE_ERR_INVALID_ARG;
  ctx->err.clear();
  if (!f_in || !f_out) return fail(ctx, SBSE_ERR_INVALID_ARG, "f_in or f_out missing");
  int rc;
  if ((rc = mixed_ready(ctx, projector))) return rc;
  CK(cudaSetDevice(ctx->device));
  const size_t bytes = (size_t)ctx->n_o * ctx->ng * sizeof(double);
  MixedBufs mb;
  double *ex;
  if ((rc = mixed_bufs(ctx, 2, &mb, &ex))) return rc;
  double *f = ex, *out = ex + (long long)ctx->n_o * ctx->ng;
  CK(cudaMemcpyAsync(f, f_in, bytes, cudaMemcpyHostToDevice, ctx->stream));
  if ((rc = mixed_apply(ctx, projector, f, out, 0.0, mb))) return rc;
  CK(cudaMemcpyAsync(f_out, out, bytes, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return SBSE_OK;
}

int sbse_mixed_bounds(sbse_ctx *ctx, int projector, int axis, int n_lanczos, double *lo, double *hi) {
  if (!ctx) return SBSE_ERR_INVALID_ARG;
  ctx->err.clear();
  if (!lo || !hi || axis < 0 || axis > 2 || n_lanczos < 2 || n_lanczos > 10000)
    return fail(ctx, SBSE_ERR_INVALID_ARG, "need lo, hi, axis in 0..2 and 2 <= n_lanczos <= 10000");
  int rc;
  if ((rc = mixed_ready(ctx, projector))) return rc;
  CK(cudaSetDevice(ctx->device));
  const long long n = (long long)ctx->n_o * ctx->ng;
  cudaStream_t st = ctx->stream;
  MixedBufs mb;
  double *ex;
  if ((rc = mixed_bufs(ctx, 3, &mb, &ex))) return rc;
  double *q = ex, *qp = ex + n, *z = ex + 2 * n;
  double *dev_s = mb.dwork + dot_work_doubles() - 1;  // (the dot scratch's last slot is free: 256 partials use it all)
  (void)dev_s;
  void *vp;
  if ((rc = ensure(ctx, WS_EIG, 8 * sizeof(double), &vp))) return rc;
  double *sc = (double *)vp;
  auto dot = [&](const double *x, const double *y) -> double {
    double h = 0.0;
    launch_dot(x, y, n, ctx->dV, mb.dwork, sc, st);
    cudaMemcpyAsync(&h, sc, sizeof(double), cudaMemcpyDeviceToHost, st);
    cudaStreamSynchronize(st);
    return h;
  };
  mixed_start(ctx, projector, axis, q, mb);
  const double n0 = sqrt(dot(q, q));
  if (!(n0 > 0.0)) return fail(ctx, SBSE_ERR_NUMERIC, "the start vector vanishes");
  launch_axpby(0.0, q, 1.0 / n0, q, n, st);
  CK(cudaMemsetAsync(qp, 0, n * sizeof(double), st));
  std::vector<double> al, be;
  double b = 0.0;
  for (int k = 0; k < n_lanczos; ++k) {
    if ((rc = mixed_apply(ctx, projector, q, z, 0.0, mb))) return rc;
    launch_axpby(-b, qp, 1.0, z, n, st);
    const double a = dot(q, z);
    launch_axpby(-a, q, 1.0, z, n, st);
    if (projector == 0)
      launch_project(z, ctx->n_o, ctx->phi64, ctx->n_occ, ctx->ng, ctx->dV, 0, mb.pwork, st);
    else
      launch_project(z, ctx->n_o, ctx->phi64 + (long long)ctx->n_occ * ctx->ng, ctx->n_c, ctx->ng, ctx->dV, 1,
                     mb.pwork, st);
    al.push_back(a);
    b = sqrt(dot(z, z));
    if (k == n_lanczos - 1 || b == 0.0) break;
    be.push_back(b);
    std::swap(q, qp);           // qp <- q
    launch_axpby(1.0 / b, z, 0.0, q, n, st);  // q <- z / b (q now points at the old qp buffer)
  }
  CHECK_LAUNCH("lanczos");
  double tlo, thi;
  tridiag_extremes(al, be, &tlo, &thi);
  const double spread = thi - tlo;
  *lo = tlo - 0.05 * spread;
  *hi = thi + 0.05 * spread;
  return SBSE_OK;
}

int sbse_absorption_mixed(sbse_ctx *ctx, int projector, int axis, int n_terms, double lo, double hi,
                          double broadening, int n_omega, const double *omega, double *sigma, double *residues) {
  if (!ctx) return SBSE_ERR_INVALID_ARG;
  ctx->err.clear();
  if (axis < 0 || axis > 2 || n_terms < 2 || n_terms > 65536 || !(broadening > 0.0) || n_omega < 1 ||
      n_omega > (1 << 24) || !omega || !sigma || !(hi > lo))
    return fail(ctx, SBSE_ERR_INVALID_ARG, "bad axis, n_terms, interval, broadening or frequency arrays");
  int rc;
  if ((rc = mixed_ready(ctx, projector))) return rc;
  CK(cudaSetDevice(ctx->device));
  const long long n = (long long)ctx->n_o * ctx->ng;
  cudaStream_t st = ctx->stream;
  MixedBufs mb;
  double *ex;
  if ((rc = mixed_bufs(ctx, 4, &mb, &ex))) return rc;
  double *f0 = ex, *va = ex + n, *vb = ex + 2 * n, *tmp = ex + 3 * n;
  void *vp;
  if ((rc = ensure(ctx, WS_SPEC, (2 * (size_t)n_terms + 2 * (size_t)n_omega + 2) * sizeof(double), &vp))) return rc;
  double *R = (double *)vp, *D = R + n_terms, *om = D + n_terms, *sg = om + n_omega, *cw = sg + n_omega;
  const double c = 0.5 * (lo + hi), w = 0.5 * (hi - lo);
  const double cwh[2] = {c, w};
  CK(cudaMemcpyAsync(cw, cwh, sizeof(cwh), cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(om, omega, (size_t)n_omega * sizeof(double), cudaMemcpyHostToDevice, st));
  mixed_start(ctx, projector, axis, f0, mb);
  // v_0 = f0 (in va), v_1 = A~ f0 (in vb), v_{t+1} = 2 A~ v_t - v_{t-1} overwriting v_{t-1}
  CK(cudaMemcpyAsync(va, f0, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
  launch_dot(f0, va, n, ctx->dV, mb.dwork, R, st);
  double *prev = va, *cur = vb;
  if ((rc = mixed_apply(ctx, projector, va, tmp, c, mb))) return rc;
  launch_axpby(1.0 / w, tmp, 0.0, cur, n, st);
  for (int t = 1; t < n_terms; ++t) {
    launch_dot(f0, cur, n, ctx->dV, mb.dwork, R + t, st);
    if (t + 1 == n_terms) break;
    if ((rc = mixed_apply(ctx, projector, cur, tmp, c, mb))) return rc;
    launch_axpby(2.0 / w, tmp, -1.0, prev, n, st);  // prev <- 2 A~ cur - prev = v_{t+1}
    std::swap(prev, cur);
  }
  launch_sigma_from_residues(R, n_terms, cw, om, n_omega, broadening, D, sg, st);
  CHECK_LAUNCH("mixed absorption");
  CK(cudaMemcpyAsync(sigma, sg, (size_t)n_omega * sizeof(double), cudaMemcpyDeviceToHost, st));
  if (residues) CK(cudaMemcpyAsync(residues, R, (size_t)n_terms * sizeof(double), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  for (int j = 0; j < n_omega; ++j)
    if (!isfinite(sigma[j])) return fail(ctx, SBSE_ERR_NUMERIC, "spectrum is not finite (interval too narrow?)");
  return SBSE_OK;
}

int sbse_set_scissor(sbse_ctx *ctx, double scissor) {
  if (!ctx) return SBSE_ERR_INVALID_ARG;
  ctx->err.clear();
  if (!isfinite(scissor)) return fail(ctx, SBSE_ERR_NUMERIC, "scissor is not finite");
  if (ctx->n_states == 0) return fail(ctx, SBSE_ERR_NOT_READY, "call sbse_set_orbitals first");
  ctx->scissor = scissor;
  ctx->have_A = false;
  return SBSE_OK;
}

int sbse_absorption(sbse_ctx *ctx, int axis, int n_terms, double broadening, int n_omega, const double *omega,
                    double *sigma, double *residues) {
  if (!ctx) return SBSE_ERR_INVALID_ARG;
  ctx->err.clear();
  if (!ctx->have_A) return fail(ctx, SBSE_ERR_NOT_READY, "call sbse_build_A first");
  if (axis < 0 || axis > 2) return fail(ctx, SBSE_ERR_INVALID_ARG, "axis must be 0 (x), 1 (y) or 2 (z)");
  if (n_terms < 2 || n_terms > (1 << 16))
    return fail(ctx, SBSE_ERR_INVALID_ARG, "n_terms must be in [2, 65536]");
  if (!(broadening > 0.0) || !isfinite(broadening))
    return fail(ctx, SBSE_ERR_INVALID_ARG, "broadening must be a positive finite energy (Ha)");
  if (n_omega < 1 || n_omega > (1 << 24) || !omega || !sigma)
    return fail(ctx, SBSE_ERR_INVALID_ARG, "need 1 <= n_omega <= 2^24 and the omega and sigma arrays");
  CK(cudaSetDevice(ctx->device));
  const int n = ctx->n_o * ctx->n_c;
  void *vp;
  int rc;
  if ((rc = ensure(ctx, WS_SPEC, spectrum_work_bytes(n, n_terms, n_omega), &vp))) return rc;
  const SpectrumBufs b = spectrum_bufs((double *)vp, n, n_terms, n_omega);
  cudaStream_t st = ctx->stream;
  CK(cudaMemcpyAsync(b.omega, omega, (size_t)n_omega * sizeof(double), cudaMemcpyHostToDevice, st));
  const double *phi_o = ctx->phi64 + (long long)(ctx->n_occ - ctx->n_o) * ctx->ng;
  const double *phi_c = ctx->phi64 + (long long)ctx->n_occ * ctx->ng;
  launch_absorption(b, phi_o, phi_c, ctx->n_o, ctx->n_c, ctx->N, ctx->h, ctx->box, ctx->dV, ctx->A, axis, n_terms,
                    broadening, n_omega, st);
  CHECK_LAUNCH("absorption");
  CK(cudaMemcpyAsync(sigma, b.sigma, (size_t)n_omega * sizeof(double), cudaMemcpyDeviceToHost, st));
  if (residues)
    CK(cudaMemcpyAsync(residues, b.R, (size_t)n_terms * sizeof(double), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  for (int j = 0; j < n_omega; ++j)
    if (!isfinite(sigma[j])) return fail(ctx, SBSE_ERR_NUMERIC, "spectrum is not finite");
  return SBSE_OK;
}

int sbse_set_option(sbse_ctx *ctx, int option, int value) {
  if (!ctx) return SBSE_ERR_INVALID_ARG;
  if (option == SBSE_OPT_TENSOR_CORES) {
    ctx->tensor_cores = value != 0;
      return SBSE_OK;
  }
  if (option == SBSE_OPT_PERSISTENT) {
    ctx->persistent = value != 0;
      return SBSE_OK;
  }
  if (option == SBSE_OPT_TMA_PLANES) {
    ctx->tma_planes = value != 0;
      return SBSE_OK;
  }
  if (option == SBSE_OPT_GRAPH) {
    ctx->use_graph = value != 0;
    return SBSE_OK;
  }
  if (option == SBSE_OPT_MEM_LIMIT_MB) {
    if (value < 0) return fail(ctx, SBSE_ERR_INVALID_ARG, "memory limit must be >= 0");
    ctx->mem_limit = (size_t)value << 20;
    return SBSE_OK;
  }
  if (option == SBSE_OPT_WAIT_LIMIT) {
    if (value < 0) return fail(ctx, SBSE_ERR_INVALID_ARG, "wait limit must be >= 0");
    ctx->wait_limit = value == 0 ? (1u << 23) : (unsigned)value;
    return SBSE_OK;
  }
  if (option == SBSE_OPT_CHUNK_MB) {
    if (value < 0) return fail(ctx, SBSE_ERR_INVALID_ARG, "chunk size must be >= 0");
    ctx->l2_chunk_bytes = value == 0 ? 1e30 : (double)value * (1 << 20);
      return SBSE_OK;
  }
  return fail(ctx, SBSE_ERR_INVALID_ARG, "unknown option");
}

int sbse_debug_bounds(int *enabled, unsigned long long *first_fault) {
  if (!enabled || !first_fault) return SBSE_ERR_INVALID_ARG;
#ifdef SBSE_DEBUG_BOUNDS
  *enabled = 1;
#else
  *enabled = 0;
#endif
  *first_fault = 0;
  int n = 0;
  for (auto rd : sbse::bounds_readers()) {
    unsigned long long v = 0;
    const int r = rd(&v);
    if (r < 0) return SBSE_ERR_CUDA;
    if (r > 0) {
      if (!*first_fault) *first_fault = v;
      ++n;
    }
  }
  return n > 0 ? SBSE_ERR_NUMERIC : SBSE_OK;
}

int sbse_kernel_launches(long long *count) {
  if (!count) return SBSE_ERR_INVALID_ARG;
  *count = sbse::g_launches.load();
  return SBSE_OK;
}

int sbse_profile(sbse_ctx *ctx, int enable) {
  if (!ctx) return SBSE_ERR_INVALID_ARG;
  ctx->prof = enable != 0;
  ctx->clk.used = 0;
  return SBSE_OK;
}

int sbse_phase_time(sbse_ctx *ctx, int phase, double *ms, long long *launches) {
  if (!ctx || !ms || !launches || phase < 0 || phase > 7) return SBSE_ERR_INVALID_ARG;
  CK(cudaStreamSynchronize(ctx->stream));
  double tot = 0.0;
  long long cnt = 0;
  for (size_t i = 0; i + 1 < ctx->clk.used; i += 2) {
    if (ctx->clk.phase[i / 2] != phase) continue;
    float f = 0.f;
    CK(cudaEventElapsedTime(&f, ctx->clk.ev[i], ctx->clk.ev[i + 1]));
    tot += f;
    ++cnt;
  }
  *ms = tot;
  *launches = cnt;
  return SBSE_OK;
}

}  // extern "C"
