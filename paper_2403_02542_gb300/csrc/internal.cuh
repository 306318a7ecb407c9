// Internal declarations of the GB300 walker-step library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstddef>
#include <cstdlib>

#include "../../include/afqmc.h"

namespace afq {

// ---------------------------------------------------------------- complex
// Storage type of a complex number for real type R (interleaved re, im).
template <typename R> struct C2;
template <> struct C2<double> { typedef double2 t; };
template <> struct C2<float> { typedef float2 t; };

// FP64 complex used for all sensitive arithmetic.
struct cd {
  double re, im;
};
__host__ __device__ __forceinline__ cd mk(double r, double i) { return cd{r, i}; }
__host__ __device__ __forceinline__ cd operator+(cd a, cd b) { return cd{a.re + b.re, a.im + b.im}; }
__host__ __device__ __forceinline__ cd operator-(cd a, cd b) { return cd{a.re - b.re, a.im - b.im}; }
__host__ __device__ __forceinline__ cd operator*(cd a, cd b) {
  return cd{a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
__host__ __device__ __forceinline__ cd operator*(double s, cd a) { return cd{s * a.re, s * a.im}; }
__host__ __device__ __forceinline__ cd conj(cd a) { return cd{a.re, -a.im}; }
__host__ __device__ __forceinline__ double abs2(cd a) { return a.re * a.re + a.im * a.im; }
__device__ __forceinline__ cd cdiv(cd a, cd b) {
  // Smith's algorithm keeps the intermediate magnitudes bounded.
  if (fabs(b.re) >= fabs(b.im)) {
    double r = b.im / b.re, den = b.re + b.im * r;
    return cd{(a.re + a.im * r) / den, (a.im - a.re * r) / den};
  } else {
    double r = b.re / b.im, den = b.re * r + b.im;
    return cd{(a.re * r + a.im) / den, (a.im * r - a.re) / den};
  }
}
__device__ __forceinline__ cd ld(const double2* p) { double2 v = *p; return cd{v.x, v.y}; }
__device__ __forceinline__ cd ld(const float2* p) { float2 v = *p; return cd{(double)v.x, (double)v.y}; }
__device__ __forceinline__ void st(double2* p, cd v) { *p = make_double2(v.re, v.im); }
__device__ __forceinline__ void st(float2* p, cd v) { *p = make_float2((float)v.re, (float)v.im); }

// ---------------------------------------------------------------- GEMM
// C[b][m][n] = alpha * sum_k A[b][m][k] * B[b][n][k]  (strides in elements),
// A real or complex, B complex; the epilogue mode decides what is stored.
enum GemmEpi { EPI_STORE = 0, EPI_STORE_ADD = 1, EPI_ACC = 2 };  // EPI_ACC: C += result
struct GemmArgs {
  int M, Nn, K, batch;
  const void* A;
  long long sa_m, sa_k, sa_b;
  const void* B;
  long long sb_n, sb_k, sb_b;
  void* C;
  long long sc_m, sc_n, sc_b;
  void* D;  // EPI_STORE_ADD: D += result (same strides as C)
  double alpha_re, alpha_im;
  // split-K (batch == 1, EPI_STORE or EPI_ACC): `splitk` K-ranges write partial tiles to
  // `part` [splitk][M][Nn] (complex, R), summed in fixed order afterwards
  int splitk;
  void* part;
  int variant;  // output tile: 0 = 64x64, 1 = 128x32, 2 = 32x128, 3 = 64x32, 4 = per-walker A*V
  int accum;    // set by gemm() for EPI_ACC: the epilogue adds to C instead of storing
  const int* skip;  // device flag or NULL: every block returns at once when *skip != 0
};
constexpr int GEMM_VARIANTS = 5;
// GEMM call sites of the step, each with its own tuned tile variant
enum GemmSite { SITE_FORCEBIAS = 0, SITE_FIELD = 1, SITE_HALFSTEP = 2, SITE_EXPM = 3, N_SITES = 4 };
template <typename R>
cudaError_t gemm(const GemmArgs& a, bool a_complex, int epi, cudaStream_t s);
// Half steps of complex64 walkers (mixed contexts, N <= 128):
// out[w][j][p] = sum_q B[p][q] in[w][j][q] with the FP32 copy of B resident
// in shared memory (k_gemm.cu); halfstep_prepare_kernel sets its shared-memory
// limit (before any graph capture).
bool halfstep_ok(const afqmc_ctx* c);
cudaError_t halfstep_prepare_kernel(const afqmc_ctx* c);
cudaError_t halfstep_launch(const afqmc_ctx* c, int Nw, const void* in, void* out, cudaStream_t s);

// ---------------------------------------------------------------- context
struct Workspace {
  int n_walkers = 0;  // capacity
  int kmax = 0;       // Krylov basis capacity
  void* theta = nullptr;     // [Nw][nc][N] C2<R>
  void* t = nullptr;         // [Nw][G] C2<R>   mixed <L_g> (force bias input)
  void* c = nullptr;         // [Nw][G] C2<R>   c_g = x_g - f_g
  void* A = nullptr;         // [Nw][N][N] C2<R>
  void* psi_b = nullptr;     // [Nw][nc][N]
  void* term0 = nullptr;     // [Nw][nc][N]
  void* term1 = nullptr;     // [Nw][nc][N]
  void* acc = nullptr;       // [Nw][nc][N]
  void* psi_new = nullptr;   // [Nw][nc][N]
  void* splitk = nullptr;    // [8][Nw][G] partial force-bias tiles
  void* basis = nullptr;     // [kmax][Nw][nc][N]
  double* hess = nullptr;    // [Nw*nc][kmax][kmax][2]
  double* beta = nullptr;    // [Nw*nc]
  double2* cbeta = nullptr;  // [Nw*nc] (psi^T psi)^{1/2} of the Lanczos action
  double* scal = nullptr;    // [Nw][16] per-walker scalars (see SC_*)
  double* logdet = nullptr;  // [Nw][2 spins][2]
  double* epart = nullptr;   // [Nw][G][2 spins][4]  (tr re, tr im, exch re, exch im)
  double* eloc = nullptr;    // [Nw][2]  scratch E_L when the caller passes none
  double* ecap = nullptr;    // [Nw]     capped Re E_L
  double* emix = nullptr;    // [4]
  uint8_t* alive = nullptr;  // [Nw]     W > 0 at the start of the step
  // block Krylov: per (walker, spin) A_k, R and F (k_block_krylov.cu), k_eff
  void* bk = nullptr;
  int* bk_keff = nullptr;    // [Nw][2]
  int bk_cap = 0, bk_k = 0;  // walker capacity and number of blocks of the layout
};

// per-walker scalar slots in Workspace::scal
enum {
  SC_LOGI_RE = 0, SC_LOGI_IM = 1,   // log I = sum_g x_g f_g - f_g^2/2
  SC_CL_RE = 2, SC_CL_IM = 3,       // sum_g c_g L_bar_g
  SC_NFCAP = 4,                     // removed force-bias components
  SC_NORMA = 5,                     // ||A||_F
  SC_E1_RE = 6, SC_E1_IM = 7,       // one-body energy sum_sigma tr(h_half Theta)
  SC_COUNT = 16
};

}  // namespace afq

namespace afq {
// Device allocation of every library buffer.  With the environment variable
// AFQMC_POISON_ALLOC=1 each new allocation is filled with 0xFF bytes (NaN in
// every floating-point type) before use, so that a read of memory no kernel
// wrote shows up as NaN instead of as whatever the allocation last held.
// AFQMC_POISON_ALLOC=<mask> restricts it to groups of allocations: bit 0
// context constants, bit 1 step workspace, bit 2 walk-adjoint workspace, bit
// 3 tensor-core operand planes, bit 4 everything else ("1" poisons all).
enum AllocGroup { AG_CONTEXT = 0, AG_WORKSPACE = 1, AG_ADJOINT = 2, AG_PLANES = 3, AG_OTHER = 4 };
inline int& alloc_group() {
  static thread_local int g = AG_OTHER;
  return g;
}
struct AllocScope {  // allocations inside the scope belong to group g
  int prev;
  explicit AllocScope(int g) : prev(alloc_group()) { alloc_group() = g; }
  ~AllocScope() { alloc_group() = prev; }
};
inline bool poison_allocations() {
  static const unsigned mask = [] {
    const char* v = getenv("AFQMC_POISON_ALLOC");
    if (!v || !v[0]) return 0u;
    if (v[0] == '1' && v[1] == 0) return 0xFFu;
    return (unsigned)strtoul(v, nullptr, 0);
  }();
  return (mask >> alloc_group()) & 1u;
}
inline cudaError_t dmalloc(void** p, size_t bytes) {
  cudaError_t e = cudaMalloc(p, bytes);
  if (e == cudaSuccess && poison_allocations()) {
    e = cudaMemset(*p, 0xFF, bytes);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
  }
  return e;
}
template <typename T>
inline cudaError_t dmalloc(T** p, size_t bytes) {
  return dmalloc(reinterpret_cast<void**>(p), bytes);
}
}  // namespace afq

namespace afq {
// Kernel-class event profiler (see afqmc_profile in the header).
struct Prof {
  bool on = false;
  uint32_t mask = 0;            // bit k: record launches of class k
  cudaEvent_t* pool = nullptr;  // 2 events per recorded launch
  int* cls = nullptr;           // class of each recorded launch
  int cap = 0, used = 0, open_cls = -1;
  double ms[AFQMC_K_COUNT] = {0};
  uint64_t n[AFQMC_K_COUNT] = {0};
};
}  // namespace afq

namespace afq {
// Plan and buffers of the tensor-core exchange contraction (mixed contexts).
struct TcPlan {
  bool ok = false;
  int n = 0, gpt = 0, T = 0, Kp = 0, KC = 0, Wc = 0, NB = 0, S = 0, b_cap = 0;
  int gpw = 0;      // n <= 32: g blocks per 32-row warp slot (0: blocks packed across the tile)
  int ewg = 2;      // epilogue warpgroups
  bool sb = false;  // B streamed with every K slab (else resident for the whole item)
  void* a_hi = nullptr;  // [2 spins][T][128][Kp] bf16, Lh split hi/lo
  void* a_lo = nullptr;
  void* b_hi = nullptr;  // [2 spins][cap][re,im][n][Kp] bf16, Theta split hi/lo
  void* b_lo = nullptr;
  void* err = nullptr;   // device int: nonzero after a bounded wait timed out
  alignas(64) unsigned char map_a_hi[128];
  alignas(64) unsigned char map_a_lo[128];
  alignas(64) unsigned char map_b_hi[128];
  alignas(64) unsigned char map_b_lo[128];
};
}  // namespace afq

namespace afq {
// Plan and operands of the tensor-core field assembly (mixed contexts).
struct TgPlan {
  bool ok = false;
  int Kp = 0, m_cap = 0;
  int Nq = 0;  // N rounded up to a multiple of 8: q stride of the field's column space
  int Kh = 0;  // Nq rounded up to a multiple of 64: offset of the Im half in the A' and X planes
  size_t Np = 0;
  void* l_hi = nullptr;  // [Np][Kp] bf16: L^T split hi/lo
  void* l_lo = nullptr;
  void* x_hi = nullptr;  // [m_cap][Kp] bf16: (-sqrt(tau) Im c, sqrt(tau) Re c) rows split hi/lo
  void* x_lo = nullptr;
  void* err = nullptr;   // device int: nonzero after a bounded wait timed out
  alignas(64) unsigned char map_l_hi[128];
  alignas(64) unsigned char map_l_lo[128];
  alignas(64) unsigned char map_x_hi[128];
  alignas(64) unsigned char map_x_lo[128];
  // products A_w V on the tensor cores: the field kernel then writes A_w as
  // bf16 hi/lo planes A'[w][p][KA] = [Re A_w[p][:] | Im A_w[p][:]] (Im from
  // column Kh, KA = 2 Kh)
  bool av_ok = false;
  int KA = 0, NBp = 0, S_av = 0, av_cap = 0;
  void* a_hi = nullptr;  // [cap * N][KA]
  void* a_lo = nullptr;
  void* v_hi = nullptr;  // [cap * NBp][KA]: rows j [Re v_j | Im v_j] (Im from column Kh), rows >= nc zero
  void* v_lo = nullptr;
  void* nrm = nullptr;   // [m_cap][Np / 256] float: sum of squares of each field tile row (||A_w||_F)
  alignas(64) unsigned char map_a_hi[128];
  alignas(64) unsigned char map_a_lo[128];
  alignas(64) unsigned char map_v_hi[128];
  alignas(64) unsigned char map_v_lo[128];
  // half steps B Psi on the tensor cores as Psi + D Psi, D = B - I (B is
  // close to the identity, so the split-bf16 error scales with ||D||):
  // rows p of D against rows 2 (w nc + j) + part = Re / Im psi_wj of the
  // walker planes, K = q
  bool hs_ok = false;
  int hs_Mp = 0, hs_Kp = 0, hs_rows = 0;  // D rows (128-padded), K (64-padded), plane rows allocated
  void* d_hi = nullptr;  // [hs_Mp][hs_Kp] bf16: D = e^{-tau h''/2} - I split hi/lo (set with tau)
  void* d_lo = nullptr;
  void* p_hi = nullptr;  // [hs_rows][hs_Kp] bf16: walker planes split hi/lo (every half step)
  void* p_lo = nullptr;
  alignas(64) unsigned char map_d_hi[128];
  alignas(64) unsigned char map_d_lo[128];
  alignas(64) unsigned char map_p_hi[128];
  alignas(64) unsigned char map_p_lo[128];
};
}  // namespace afq

struct afqmc_ctx {
  int N, na, nb, nc, G, prec;
  double e_const = 0.0, ec_prime = 0.0, tau = -1.0;
  cudaStream_t stream = nullptr;
  // FP64 device constants
  double* d_L = nullptr;      // [G][N][N]
  double* d_Lh = nullptr;     // [G][nc][N]  Lh[g][j][q] = sum_p trial[j][p] L[g][p][q]
  double* d_trial = nullptr;  // [nc][N]
  double* d_hhalf = nullptr;  // [nc][N]     sum_p trial[j][p] h1[p][q]
  double* d_Lbar = nullptr;   // [G]
  double* d_thT = nullptr;    // [nc][N]     Theta_T = trial_s (trial_s^T trial_s)^{-1} per spin
  // force bias from the last measurement: d_bias_key = {psi pointer, Nw} of the
  // walkers whose traces ws.epart holds (0 = none); d_bias_skip = 1 while the
  // current step takes <L_g> from those traces
  unsigned long long* d_bias_key = nullptr;
  int* d_bias_skip = nullptr;
  double* d_B = nullptr;      // [N][N]
  double* d_hpp = nullptr;    // [N][N]     h'' (the Taylor propagator's one-body part)
  // FP32 copies for mixed contexts
  float* f_L = nullptr;
  float* f_Lh = nullptr;
  float* f_B = nullptr;
  float* f_trial = nullptr;  // [nc][N]
  float2* f_hh2 = nullptr;   // [nc][N] h_half split into FP32 (hi, lo)
  // eigendecomposition of h'' (host, for B at any tau)
  double* h_evals = nullptr;  // [N]
  double* h_evecs = nullptr;  // [N][N], column k is eigenvector k
  afq::Workspace ws;
  afq::Prof prof;
  afq::TcPlan tc;
  afq::TgPlan tg;
  int tune[afq::N_SITES] = {0, 0, 0, 4};  // GEMM tile variant per call site
  bool capturing = false;                  // inside a graph capture (afqmc_batch_step)
  uint64_t launches = 0;
  int device = -1;                         // CUDA device current at afqmc_create (holds the context's memory)
};

namespace afq {

// True while the context's work is being captured into a graph (kernel
// attributes were set before the capture and are not touched then).
inline bool capturing(const afqmc_ctx* c);
// Set the dynamic shared-memory limits of every kernel a context uses (before
// any graph capture).  The limit is a per-kernel attribute shared by all
// contexts, so it is always raised to the device's opt-in maximum (it permits
// larger launches; it reserves nothing).
cudaError_t prepare_kernels(afqmc_ctx* c);
int max_dyn_smem();
// Raise a kernel's dynamic shared-memory limit to the opt-in maximum minus its
// static shared memory.
template <typename F>
cudaError_t raise_smem_limit(F* func) {
  cudaFuncAttributes a;
  cudaError_t e = cudaFuncGetAttributes(&a, reinterpret_cast<const void*>(func));
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(reinterpret_cast<const void*>(func), cudaFuncAttributeMaxDynamicSharedMemorySize,
                              max_dyn_smem() - (int)a.sharedSizeBytes);
}

// Record the start (begin=true) or end of a launch of class `cls` when the
// context's profiler is on.
void prof_mark(afqmc_ctx* c, int cls, bool begin, cudaStream_t s);

// kernels (launch wrappers); every wrapper returns the launch error
template <typename R>
cudaError_t launch_overlap(const afqmc_ctx* c, int Nw, const void* psi, void* theta,
                           double* logdet, uint32_t* status, cudaStream_t s, const int* skip = nullptr);
template <typename R>
cudaError_t launch_bias_finalize(const afqmc_ctx* c, int Nw, const double* x, double sqrt_tau,
                                 cudaStream_t s, uint8_t* keep = nullptr,  // keep[w][g]: 1 = f_g kept
                                 const int* from_traces = nullptr);      // device flag: <L_g> from ws.epart
// d_bias_skip = (opt_in && d_bias_key == {psi, Nw}); the key is cleared
cudaError_t launch_bias_gate(const afqmc_ctx* c, const void* psi, int Nw, int opt_in, cudaStream_t s);
// d_bias_key = {psi, Nw}: ws.epart now holds the traces of these walkers
cudaError_t launch_bias_mark(const afqmc_ctx* c, const void* psi, int Nw, cudaStream_t s);
template <typename R>
cudaError_t launch_normA(const afqmc_ctx* c, int Nw, cudaStream_t s);
// Y[w] <- (I - X[w]/2)^{-1} Y[w] for Nw walkers (Crank-Nicolson; X [Nw][N][N]
// is overwritten by the factors, Y [Nw][nc][N] in place; see cn_solve_kernel
// in k_linalg.cu)
template <typename R>
cudaError_t launch_cn_solve(const afqmc_ctx* c, int Nw, void* X, void* Y, cudaStream_t s);
// One step of the Chebyshev recurrence on Nw walkers' [nc][N] vectors (see
// cheb_step_kernel in k_energy.cu)
template <typename R>
cudaError_t launch_cheb_step(const afqmc_ctx* c, int Nw, const void* prod, void* t, void* acc, double a, double b,
                             int first, cudaStream_t s);
// ws.A[w] -= tau h'' (real part) for Nw walkers: the Taylor propagator's exponent
template <typename R>
cudaError_t launch_shift_field(const afqmc_ctx* c, int Nw, double tau, cudaStream_t s);
template <typename R>
cudaError_t launch_krylov_init(const afqmc_ctx* c, int Nw, cudaStream_t s);
// Arnoldi step `it` with the product A b_it in wv (NULL: ws.term0)
template <typename R>
cudaError_t launch_krylov_orth(const afqmc_ctx* c, int Nw, int it, int k, cudaStream_t s, const void* wv = nullptr);
// small exponential y = beta e^{H} e_1 (beta = cbeta for the Lanczos action)
// and the combination acc = sum_i y_i b_i
template <typename R>
cudaError_t launch_krylov_finish(const afqmc_ctx* c, int Nw, int k, cudaStream_t s, bool lanczos = false);
// complex-symmetric Lanczos: v_0 = psi_b / (psi_b^T psi_b)^{1/2}, then per
// step the three-term recurrence on the product A v_it (wv, NULL: ws.term0)
template <typename R>
cudaError_t launch_lanczos_init(const afqmc_ctx* c, int Nw, cudaStream_t s);
template <typename R>
cudaError_t launch_lanczos_step(const afqmc_ctx* c, int Nw, int it, int k, cudaStream_t s, const void* wv = nullptr);
template <typename R>
cudaError_t launch_weights(const afqmc_ctx* c, const afqmc_walkers* w, double tau, double e0,
                           cudaStream_t s);
template <typename R>
cudaError_t launch_commit(const afqmc_ctx* c, const afqmc_walkers* w, int reortho, cudaStream_t s);
template <typename R>
cudaError_t launch_mgs(const afqmc_ctx* c, int Nw, void* psi, const uint8_t* mask, double* logr, cudaStream_t s);
template <typename R>
cudaError_t launch_energy(afqmc_ctx* c, int Nw, const double* weight, double e0, double tau,
                          double* e_loc, double* e_mix, cudaStream_t s, int* n_launch);
template <typename R>
cudaError_t launch_init_walkers(const afqmc_ctx* c, const afqmc_walkers* w, cudaStream_t s);
cudaError_t launch_setup(afqmc_ctx* c, cudaStream_t s);
cudaError_t launch_logovl_from_logdet(const afqmc_ctx* c, const afqmc_walkers* w,
                                      const uint8_t* mask, cudaStream_t s);
// logovl[w] -= sum_s log det R_s from the MGS kernel's output in ws.logdet
cudaError_t launch_logovl_shift(const afqmc_ctx* c, const afqmc_walkers* w, const uint8_t* mask, cudaStream_t s);
cudaError_t launch_copy_alive(const afqmc_ctx* c, const afqmc_walkers* w, cudaStream_t s);

// block-Krylov action of the exponential (k_block_krylov.cu): bk_ensure sizes
// the per (walker, spin) area for k blocks; start = QR of psi_b into basis
// slot 0; orth(j) = block Arnoldi step on W = A B_j in ws.term0; finish =
// e^{A_k} E_n R and B_k F into ws.acc.
size_t bk_expm_smem(int k, int nmax, size_t csize);
size_t bk_orth_smem(int N, int nmax, size_t csize);
size_t bk_combine_smem(int N, int k, int nmax, size_t csize);
cudaError_t bk_ensure(afqmc_ctx* c, int Nw, int k);
template <typename R>
cudaError_t launch_bk_start(const afqmc_ctx* c, int Nw, int k, cudaStream_t s);
template <typename R>
cudaError_t launch_bk_orth(const afqmc_ctx* c, int Nw, int j, cudaStream_t s);
template <typename R>
cudaError_t launch_bk_finish(const afqmc_ctx* c, int Nw, cudaStream_t s);
template <typename R>
cudaError_t prepare_bk(const afqmc_ctx* c);

// comb population control (k_population.cu)
template <typename R>
cudaError_t launch_comb(afqmc_ctx* c, const afqmc_walkers* w, double u, int* index_out, cudaStream_t s);

// adjoint of the mixed estimator (k_adjoint.cu); R = the walkers' real type
template <typename R>
cudaError_t launch_energy_backward(afqmc_ctx* c, int Nw, const double* weight, const double* e_loc, double e0,
                                   double tau, double dJ, double* grad_h1, double* grad_L, double2* yscratch,
                                   cudaStream_t s);

// adjoint of the fixed-field walk (k_walk_adjoint.cu); walker states and
// their adjoints in C2<R>, overlap inverses, coefficients and sums in FP64
template <typename R>
cudaError_t adj_sanitize(const typename C2<R>::t* src, typename C2<R>::t* dst, const double* wfin,
                         const double* trial, size_t per, int Nw, cudaStream_t s);
template <typename R>
cudaError_t adj_sum_terms(const typename C2<R>::t* T, typename C2<R>::t* out, int K1, size_t per, int Nw,
                          cudaStream_t s);
template <typename R>
cudaError_t adj_scale_copy(const typename C2<R>::t* src, size_t sstride, typename C2<R>::t* dst, size_t dstride,
                           double sc, size_t per, int Nw, cudaStream_t s);
// dst[i] += src[i], i < n (FP64 accumulation of complex64 contributions)
cudaError_t adj_fold(const float2* src, double2* dst, size_t n, cudaStream_t s);
size_t adj_lu_smem(int nmax);
size_t adj_small_smem(int nmax);
template <typename R>
cudaError_t adj_lu(const afqmc_ctx* c, int Nw, const typename C2<R>::t* psi, double2* oinv, double* logdet,
                   cudaStream_t s);
cudaError_t adj_ratio_coef(int Nw, const double* wfin, const double* omega, const double* ld3, const double* logovl,
                           const double* scal, double2* aR, double sqrt_tau, cudaStream_t s);
template <typename R>
cudaError_t adj_ratio(const afqmc_ctx* c, int Nw, const typename C2<R>::t* pnext, const typename C2<R>::t* psinext,
                      const double2* oinv3, const double2* aR, const double* wfin, typename C2<R>::t* p3, int qr,
                      cudaStream_t s);
template <typename R>
cudaError_t adj_force(const afqmc_ctx* c, int Nw, const typename C2<R>::t* cbar, const typename C2<R>::t* cc,
                      const uint8_t* keep, const double2* aR, const double* omega, typename C2<R>::t* tbar,
                      double* mu_part, double* mubar, double sqrt_tau, double tau, cudaStream_t s);
template <typename R>
cudaError_t adj_theta(const afqmc_ctx* c, int Nw, const typename C2<R>::t* thbar, const typename C2<R>::t* theta,
                      const double2* oinv, const double2* aR, const double* wfin, typename C2<R>::t* pbar,
                      cudaStream_t s);
cudaError_t adj_seed_coef(int Nw, const double* wfin, const double* ecap, const double* e_loc, const double* emix,
                          double* omega, double* ecoef, double e0, double dE, double dJ, cudaStream_t s);
// Krylov-action reverse (basis, Hessenberg and beta of the forward in the
// workspace; Hs a copy of the Hessenberg block taken before the small
// exponential overwrote its first column; Gb the basis adjoints, planes
// gstride apart, stored as holomorphic-style adjoints g = conj(Gamma)).
// `lanczos` selects the complex start norm gamma (ws.cbeta) and writes the
// start-norm adjoint as a complex g_gamma; Arnoldi's is (Gamma_beta, 0).
template <typename R>
cudaError_t kadj_seed(const afqmc_ctx* c, int Nw, int k, const typename C2<R>::t* gout, typename C2<R>::t* Gb,
                      size_t gstride, double2* gy, cudaStream_t s);
template <typename R>
cudaError_t kadj_expm(const afqmc_ctx* c, int Nw, int k, const typename C2<R>::t* Hs, const double2* gy, double2* GH,
                      double2* gbeta, bool lanczos, cudaStream_t s);
template <typename R>
cudaError_t kadj_orth(const afqmc_ctx* c, int Nw, int j, int k, const typename C2<R>::t* wj,
                      const typename C2<R>::t* Hs, const double2* GH, typename C2<R>::t* Gb, size_t gstride,
                      typename C2<R>::t* U, cudaStream_t s);
template <typename R>
cudaError_t kadj_input(const afqmc_ctx* c, int Nw, const typename C2<R>::t* Gb0, const double2* gbeta,
                       typename C2<R>::t* gx, bool lanczos, cudaStream_t s);
// reverse of Lanczos step j; carry: one double2 per column, written by step j
// for step j - 1 (read only where j + 1 < k, so it needs no initial value)
template <typename R>
cudaError_t lzadj_step(const afqmc_ctx* c, int Nw, int j, int k, const typename C2<R>::t* wj,
                       const typename C2<R>::t* Hs, const double2* GH, typename C2<R>::t* Gb, size_t gstride,
                       typename C2<R>::t* U, double2* carry, cudaStream_t s);
template <typename R>
cudaError_t adj_eloc_seed(const afqmc_ctx* c, int Nw, const typename C2<R>::t* theta, const typename C2<R>::t* t,
                          const double* ecoef, typename C2<R>::t* thbar, cudaStream_t s);
cudaError_t adj_finish(const afqmc_ctx* c, const double2* Bbar, const double* V, const double* lam, double tau,
                       double* Bs, double* T1, double* M1, double* hbar, double* X, double* D, const double2* gLc,
                       const double2* Lhb, double* mubar, double* grad_h1, double* grad_L, int* n_launch,
                       cudaStream_t s);

// tensor-core exchange (k_exchange_tc.cu)
bool tc_exchange_plan(afqmc_ctx* c);
cudaError_t tc_exchange_setup(afqmc_ctx* c, cudaStream_t s);
cudaError_t tc_exchange_ws(afqmc_ctx* c);
size_t tc_exchange_plane_bytes(const TcPlan& P, int cap);
cudaError_t tc_exchange_bind(TcPlan& P, void* b_hi, void* b_lo, int cap);
void tc_exchange_free(afqmc_ctx* c);
// split Theta planes of Nw walkers, then the contraction (writes epart)
cudaError_t tc_exchange_planes(afqmc_ctx* c, int Nw, const void* theta, cudaStream_t s);
cudaError_t tc_exchange_contract(afqmc_ctx* c, int Nw, double* epart, cudaStream_t s);

// tensor-core field assembly (k_gemm_tc.cu)
cudaError_t tc_field_setup(afqmc_ctx* c, cudaStream_t s);
cudaError_t tc_field_ws(afqmc_ctx* c);
cudaError_t tc_field_prepare(const afqmc_ctx* c);
void tc_field_free(afqmc_ctx* c);
// to_memory: write A_w as interleaved complex [Nw][N][N] to ws.A instead of the
// split-bf16 A' planes (for the propagators that shift A_w in memory)
cudaError_t tc_field_launch(afqmc_ctx* c, int Nw, double sqrt_tau, cudaStream_t s, bool to_memory = false);
// C[w][j][p] = alpha sum_q A_w[p][q] V[w][j][q] (D[w] += C[w] when D is given),
// complex64, walker batch strides in complex elements; A_w from the planes.
// V == NULL: the V planes were already written (by the Arnoldi kernels).
cudaError_t tc_av_launch(afqmc_ctx* c, int Nw, const void* V, long long v_stride, void* C, void* D,
                         long long c_stride, double alpha, cudaStream_t s);
// ||A_w||_F from the planes into ws.scal[w][SC_NORMA]
cudaError_t tc_av_normA(afqmc_ctx* c, int Nw, cudaStream_t s);
// half step out = B in (complex64 [Nw][nc][N], in != out) on the tensor cores,
// as in + D in with D = B - I; D's planes from tc_halfstep_set_b (after B changes)
cudaError_t tc_halfstep_set_b(afqmc_ctx* c, cudaStream_t s);
cudaError_t tc_halfstep_launch(afqmc_ctx* c, int Nw, const void* in, void* out, cudaStream_t s);

}  // namespace afq

namespace afq {
inline bool capturing(const afqmc_ctx* c) { return c->capturing; }
}  // namespace afq
