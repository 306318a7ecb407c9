// C ABI of the walker-step library: context set-up and the step schedule.
//
// Set-up (once per Hamiltonian): half-rotated Cholesky vectors trial^T L_g,
// the mean-field shift L_bar_g (Eq. force_shift), h'' = h1 - 1/2 sum_g L_g L_g
// + sum_g L_bar_g L_g with E_c' = E_const - 1/2 sum_g L_bar_g^2, and the
// eigendecomposition of h'' (host Jacobi) from which B = e^{-tau h''/2} is
// built exactly for any tau (Sec. III.B).
//
// Step schedule (all on the context's stream):
//   overlap/Theta -> force-bias GEMM -> bias finalisation -> field GEMM (tensor
//   cores for complex64 walkers)
//   -> B Psi -> Taylor or Arnoldi/Krylov -> B Psi -> new overlap -> weights
//   -> commit -> [MGS -> overlap] -> [overlap -> local energy -> E_k]
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <type_traits>
#include <utility>
#include <vector>

#include "internal.cuh"

namespace afq {
template <typename R> cudaError_t prepare_overlap(const afqmc_ctx* c);
template <typename R> cudaError_t prepare_energy(const afqmc_ctx* c);
cudaError_t tc_exchange_prepare(const afqmc_ctx* c);
cudaError_t launch_lsq(const double* L, double* LL, int N, int G, cudaStream_t s);
cudaError_t launch_lbar(const double* Lh, const double* thT, double* Lbar, int G, size_t per, cudaStream_t s);
cudaError_t launch_to_float(const double* a, float* b, size_t n, cudaStream_t s);
}  // namespace afq

using namespace afq;

static thread_local char g_cuda_err[256] = "no error";

static afqmc_status cuda_fail(cudaError_t e, const char* where = nullptr) {
  if (where)
    snprintf(g_cuda_err, sizeof g_cuda_err, "%s: %s: %s", where, cudaGetErrorName(e), cudaGetErrorString(e));
  else
    snprintf(g_cuda_err, sizeof g_cuda_err, "%s: %s", cudaGetErrorName(e), cudaGetErrorString(e));
  if (e == cudaErrorMemoryAllocation) return AFQMC_ENOMEM;
  return AFQMC_ECUDA;
}
#define CKW(expr, where)                                 \
  do {                                                   \
    cudaError_t _e = (expr);                             \
    if (_e != cudaSuccess) return cuda_fail(_e, where);  \
  } while (0)

#define CK(expr)                                     \
  do {                                               \
    cudaError_t _e = (expr);                         \
    if (_e != cudaSuccess) return cuda_fail(_e);     \
  } while (0)

static bool all_finite(const double* a, size_t n) {
  for (size_t i = 0; i < n; ++i)
    if (!std::isfinite(a[i])) return false;
  return true;
}

// ---------------------------------------------------------------- host eigh
// Cyclic Jacobi for a real symmetric matrix (row-major, destroyed).  On
// return evals[k] and column k of evecs (row-major n x n) are an eigenpair.
static void jacobi_eigh(int n, double* a, double* evals, double* evecs) {
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) evecs[(size_t)i * n + j] = (i == j) ? 1.0 : 0.0;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0, diag = 0.0;
    for (int p = 0; p < n; ++p) {
      diag += a[(size_t)p * n + p] * a[(size_t)p * n + p];
      for (int q = p + 1; q < n; ++q) off += a[(size_t)p * n + q] * a[(size_t)p * n + q];
    }
    if (off <= 1e-34 * (diag + off) || off == 0.0) break;
    for (int p = 0; p < n - 1; ++p)
      for (int q = p + 1; q < n; ++q) {
        const double apq = a[(size_t)p * n + q];
        if (apq == 0.0) continue;
        const double app = a[(size_t)p * n + p], aqq = a[(size_t)q * n + q];
        const double theta = (aqq - app) / (2.0 * apq);
        double t;
        if (std::fabs(theta) > 1e150)
          t = 0.5 / theta;
        else
          t = (theta >= 0.0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        const double cth = 1.0 / std::sqrt(t * t + 1.0), sth = t * cth;
        for (int k = 0; k < n; ++k) {  // columns p, q
          const double akp = a[(size_t)k * n + p], akq = a[(size_t)k * n + q];
          a[(size_t)k * n + p] = cth * akp - sth * akq;
          a[(size_t)k * n + q] = sth * akp + cth * akq;
        }
        for (int k = 0; k < n; ++k) {  // rows p, q
          const double apk = a[(size_t)p * n + k], aqk = a[(size_t)q * n + k];
          a[(size_t)p * n + k] = cth * apk - sth * aqk;
          a[(size_t)q * n + k] = sth * apk + cth * aqk;
        }
        a[(size_t)p * n + q] = 0.0;
        a[(size_t)q * n + p] = 0.0;
        for (int k = 0; k < n; ++k) {
          const double vkp = evecs[(size_t)k * n + p], vkq = evecs[(size_t)k * n + q];
          evecs[(size_t)k * n + p] = cth * vkp - sth * vkq;
          evecs[(size_t)k * n + q] = sth * vkp + cth * vkq;
        }
      }
  }
  for (int i = 0; i < n; ++i) evals[i] = a[(size_t)i * n + i];
}

// Invert a small real SPD matrix by Gauss-Jordan with partial pivoting.
static bool small_inverse(int n, std::vector<double> m, std::vector<double>& inv) {
  inv.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) inv[(size_t)i * n + i] = 1.0;
  for (int k = 0; k < n; ++k) {
    int piv = k;
    for (int i = k + 1; i < n; ++i)
      if (std::fabs(m[(size_t)i * n + k]) > std::fabs(m[(size_t)piv * n + k])) piv = i;
    if (m[(size_t)piv * n + k] == 0.0) return false;
    if (piv != k)
      for (int j = 0; j < n; ++j) {
        std::swap(m[(size_t)k * n + j], m[(size_t)piv * n + j]);
        std::swap(inv[(size_t)k * n + j], inv[(size_t)piv * n + j]);
      }
    const double d = m[(size_t)k * n + k];
    for (int j = 0; j < n; ++j) { m[(size_t)k * n + j] /= d; inv[(size_t)k * n + j] /= d; }
    for (int i = 0; i < n; ++i) {
      if (i == k) continue;
      const double f = m[(size_t)i * n + k];
      if (f == 0.0) continue;
      for (int j = 0; j < n; ++j) {
        m[(size_t)i * n + j] -= f * m[(size_t)k * n + j];
        inv[(size_t)i * n + j] -= f * inv[(size_t)k * n + j];
      }
    }
  }
  return true;
}

// ---------------------------------------------------------------- workspace
static void ws_free(Workspace& ws) {
  void* ptrs[] = {ws.theta, ws.t, ws.c, ws.A, ws.psi_b, ws.term0, ws.term1, ws.acc, ws.psi_new, ws.splitk, ws.basis,
                  ws.hess, ws.beta, ws.cbeta, ws.scal, ws.logdet, ws.epart, ws.eloc, ws.ecap, ws.emix, ws.alive,
                  ws.bk, ws.bk_keff};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  ws = Workspace();
}

static afqmc_status ws_ensure(afqmc_ctx* c, int Nw, int kmax) {
  AllocScope alloc_scope(AG_WORKSPACE);
  if (Nw <= c->ws.n_walkers && kmax <= c->ws.kmax) return AFQMC_OK;
  const int nw = Nw > c->ws.n_walkers ? Nw : c->ws.n_walkers;
  const int km = kmax > c->ws.kmax ? kmax : c->ws.kmax;
  CK(cudaStreamSynchronize(c->stream));
  ws_free(c->ws);
  Workspace& ws = c->ws;
  const size_t cs = c->prec == AFQMC_FP64 ? 16 : 8;  // complex storage bytes
  const size_t per = (size_t)c->nc * c->N;
  CK(dmalloc(&ws.theta, nw * per * cs));
  CK(dmalloc(&ws.t, (size_t)nw * c->G * cs));
  CK(dmalloc(&ws.c, (size_t)nw * c->G * cs));
  CK(dmalloc(&ws.A, (size_t)nw * c->N * c->N * cs));
  CK(dmalloc(&ws.psi_b, nw * per * cs));
  CK(dmalloc(&ws.term0, nw * per * cs));
  CK(dmalloc(&ws.term1, nw * per * cs));
  CK(dmalloc(&ws.acc, nw * per * cs));
  CK(dmalloc(&ws.psi_new, nw * per * cs));
  CK(dmalloc(&ws.splitk, (size_t)8 * nw * c->G * cs));
  if (km > 0) {
    CK(dmalloc(&ws.basis, (size_t)km * nw * per * cs));
    CK(dmalloc(&ws.hess, (size_t)nw * c->nc * km * km * 2 * sizeof(double)));
    CK(dmalloc(&ws.beta, (size_t)nw * c->nc * sizeof(double)));
    CK(dmalloc(&ws.cbeta, (size_t)nw * c->nc * sizeof(double2)));
  }
  CK(dmalloc(&ws.scal, (size_t)nw * SC_COUNT * sizeof(double)));
  CK(dmalloc(&ws.logdet, (size_t)nw * 4 * sizeof(double)));
  CK(dmalloc(&ws.epart, (size_t)nw * c->G * 8 * sizeof(double)));
  CK(dmalloc(&ws.eloc, (size_t)nw * 2 * sizeof(double)));
  CK(dmalloc(&ws.ecap, (size_t)nw * sizeof(double)));
  CK(dmalloc(&ws.emix, 4 * sizeof(double)));
  CK(dmalloc(&ws.alive, (size_t)nw));
  ws.n_walkers = nw;
  ws.kmax = km;
  // the traces a later step could reuse for its force bias were in the freed buffers
  if (c->d_bias_key) CK(cudaMemsetAsync(c->d_bias_key, 0, 2 * sizeof(unsigned long long), c->stream));
  if (c->tc.ok) CK(tc_exchange_ws(c));
  if (c->tg.ok) CK(tc_field_ws(c));
  return AFQMC_OK;
}

namespace afq {
int max_dyn_smem() {
  static int cached = 0;
  if (!cached) {
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) == cudaSuccess && v > 0)
      cached = v;
    else
      cached = 48 * 1024;
  }
  return cached;
}

cudaError_t prepare_kernels(afqmc_ctx* c) {
  cudaError_t e = c->prec == AFQMC_FP64 ? prepare_overlap<double>(c) : prepare_overlap<float>(c);
  if (e == cudaSuccess) e = c->prec == AFQMC_FP64 ? prepare_energy<double>(c) : prepare_energy<float>(c);
  if (e == cudaSuccess) e = tc_exchange_prepare(c);
  if (e == cudaSuccess) e = tc_field_prepare(c);
  if (e == cudaSuccess) e = halfstep_prepare_kernel(c);
  if (e == cudaSuccess) e = c->prec == AFQMC_FP64 ? prepare_bk<double>(c) : prepare_bk<float>(c);
  return e;
}
}  // namespace afq

// ---------------------------------------------------------------- profiler
namespace afq {
void prof_mark(afqmc_ctx* c, int cls, bool begin, cudaStream_t s) {
  Prof& p = c->prof;
  if (!p.on || !((p.mask >> cls) & 1u)) return;
  if (begin) {
    if (p.used >= p.cap) { p.open_cls = -1; return; }
    cudaEventRecord(p.pool[2 * p.used], s);
    p.cls[p.used] = cls;
    p.open_cls = cls;
  } else {
    if (p.open_cls < 0) return;
    cudaEventRecord(p.pool[2 * p.used + 1], s);
    ++p.used;
    p.open_cls = -1;
  }
}
}  // namespace afq

static void prof_release(Prof& p) {
  if (p.pool)
    for (int i = 0; i < 2 * p.cap; ++i) cudaEventDestroy(p.pool[i]);
  free(p.pool);
  free(p.cls);
  p = Prof();
}

// ---------------------------------------------------------------- set-up
static void ctx_free(afqmc_ctx* c) {
  if (!c) return;
  prof_release(c->prof);
  tc_exchange_free(c);
  tc_field_free(c);
  ws_free(c->ws);
  void* ptrs[] = {c->d_L, c->d_Lh,  c->d_trial, c->d_hhalf,    c->d_Lbar,     c->d_thT,
                  c->d_B, c->f_L,   c->f_Lh,    c->f_B,        c->f_trial,    c->f_hh2,      c->d_bias_key,
                  c->d_bias_skip, c->d_hpp};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  free(c->h_evals);
  free(c->h_evecs);
  delete c;
}

static afqmc_status ctx_setup(afqmc_ctx* c, const double* h1, const double* L, const double* trial) {
  AllocScope alloc_scope(AG_CONTEXT);
  const int N = c->N, nc = c->nc, G = c->G;
  const size_t NN = (size_t)N * N;
  cudaStream_t s = c->stream;
  CK(dmalloc(&c->d_L, (size_t)G * NN * sizeof(double)));
  CK(dmalloc(&c->d_Lh, (size_t)G * nc * N * sizeof(double)));
  CK(dmalloc(&c->d_trial, (size_t)nc * N * sizeof(double)));
  CK(dmalloc(&c->d_hhalf, (size_t)nc * N * sizeof(double)));
  CK(dmalloc(&c->d_Lbar, (size_t)G * sizeof(double)));
  CK(dmalloc(&c->d_B, NN * sizeof(double)));
  CK(dmalloc(&c->d_hpp, NN * sizeof(double)));
  CK(dmalloc(&c->d_bias_key, 2 * sizeof(unsigned long long)));
  CK(dmalloc(&c->d_bias_skip, sizeof(int)));
  CK(cudaMemsetAsync(c->d_bias_key, 0, 2 * sizeof(unsigned long long), s));
  CK(cudaMemsetAsync(c->d_bias_skip, 0, sizeof(int), s));
  if (c->prec == AFQMC_MIXED) {
    CK(dmalloc(&c->f_L, (size_t)G * NN * sizeof(float)));
    CK(dmalloc(&c->f_Lh, (size_t)G * nc * N * sizeof(float)));
    CK(dmalloc(&c->f_B, NN * sizeof(float)));
    CK(dmalloc(&c->f_trial, (size_t)nc * N * sizeof(float)));
    CK(dmalloc(&c->f_hh2, (size_t)nc * N * sizeof(float2)));
  }
  CK(cudaMemcpyAsync(c->d_L, L, (size_t)G * NN * sizeof(double), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(c->d_trial, trial, (size_t)nc * N * sizeof(double), cudaMemcpyHostToDevice, s));

  // h_half[j][q] = sum_p trial[j][p] h1[p][q]
  std::vector<double> hh((size_t)nc * N, 0.0);
  for (int j = 0; j < nc; ++j)
    for (int p = 0; p < N; ++p) {
      const double t = trial[(size_t)j * N + p];
      if (t == 0.0) continue;
      for (int q = 0; q < N; ++q) hh[(size_t)j * N + q] += t * h1[(size_t)p * N + q];
    }
  CK(cudaMemcpyAsync(c->d_hhalf, hh.data(), hh.size() * sizeof(double), cudaMemcpyHostToDevice, s));
  if (c->prec == AFQMC_MIXED) {  // h_half = hi + lo in FP32 for the complex64 one-body trace
    std::vector<float2> hh2(hh.size());
    for (size_t e = 0; e < hh.size(); ++e) {
      const float hi = (float)hh[e];
      hh2[e] = make_float2(hi, (float)(hh[e] - (double)hi));
    }
    CK(cudaMemcpy(c->f_hh2, hh2.data(), hh2.size() * sizeof(float2), cudaMemcpyHostToDevice));
  }

  // Theta_T = trial (trial_s^T trial_s)^{-1} per spin (orthonormal trial: Theta_T = trial)
  std::vector<double> thT((size_t)nc * N, 0.0);
  for (int spin = 0; spin < 2; ++spin) {
    const int n = spin ? c->nb : c->na, off = spin ? c->na : 0;
    if (n == 0) continue;
    std::vector<double> S((size_t)n * n, 0.0), Si;
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        double v = 0.0;
        for (int p = 0; p < N; ++p) v += trial[(size_t)(off + i) * N + p] * trial[(size_t)(off + j) * N + p];
        S[(size_t)i * n + j] = v;
      }
    if (!small_inverse(n, S, Si)) return AFQMC_EINVAL;
    for (int j = 0; j < n; ++j)
      for (int p = 0; p < N; ++p) {
        double v = 0.0;
        for (int i = 0; i < n; ++i) v += trial[(size_t)(off + i) * N + p] * Si[(size_t)i * n + j];
        thT[(size_t)(off + j) * N + p] = v;
      }
  }
  double* d_LL = nullptr;
  CK(dmalloc(&c->d_thT, thT.size() * sizeof(double)));
  double* d_thT = c->d_thT;
  CK(dmalloc(&d_LL, NN * sizeof(double)));
  CK(cudaMemcpyAsync(d_thT, thT.data(), thT.size() * sizeof(double), cudaMemcpyHostToDevice, s));
  CK(launch_setup(c, s));
  if (c->prec == AFQMC_MIXED) {
    CK(launch_to_float(c->d_trial, c->f_trial, (size_t)nc * N, s));
    c->launches += 1;
  }
  CK(launch_lbar(c->d_Lh, d_thT, c->d_Lbar, G, (size_t)nc * N, s));
  CK(launch_lsq(c->d_L, d_LL, N, G, s));
  c->launches += (c->prec == AFQMC_MIXED ? 3 : 1) + 2;
  std::vector<double> LL(NN), Lbar(G);
  CK(cudaMemcpyAsync(LL.data(), d_LL, NN * sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(Lbar.data(), c->d_Lbar, G * sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  cudaFree(d_LL);

  // h'' and E_c' (mean-field shift as an operator constant)
  std::vector<double> hpp(NN);
  for (size_t e = 0; e < NN; ++e) hpp[e] = h1[e] - 0.5 * LL[e];
  double lb2 = 0.0;
  for (int g = 0; g < G; ++g) {
    const double lb = Lbar[g];
    lb2 += lb * lb;
    const double* Lg = L + (size_t)g * NN;
    for (size_t e = 0; e < NN; ++e) hpp[e] += lb * Lg[e];
  }
  for (int p = 0; p < N; ++p)  // symmetrise against rounding
    for (int q = p + 1; q < N; ++q) {
      const double v = 0.5 * (hpp[(size_t)p * N + q] + hpp[(size_t)q * N + p]);
      hpp[(size_t)p * N + q] = hpp[(size_t)q * N + p] = v;
    }
  c->ec_prime = c->e_const - 0.5 * lb2;
  CK(cudaMemcpyAsync(c->d_hpp, hpp.data(), NN * sizeof(double), cudaMemcpyHostToDevice, s));
  CK(cudaStreamSynchronize(s));  // hpp is a host temporary
  c->h_evals = (double*)malloc(N * sizeof(double));
  c->h_evecs = (double*)malloc(NN * sizeof(double));
  if (!c->h_evals || !c->h_evecs) return AFQMC_ENOMEM;
  jacobi_eigh(N, hpp.data(), c->h_evals, c->h_evecs);
  if (c->prec == AFQMC_MIXED && tc_exchange_plan(c)) {
    CK(tc_exchange_setup(c, s));
    c->launches += 1;
    CK(cudaStreamSynchronize(s));
  }
  if (c->prec == AFQMC_MIXED) {
    CK(tc_field_setup(c, s));
    c->launches += c->tg.ok ? 1 : 0;
    CK(cudaStreamSynchronize(s));
  }
  return AFQMC_OK;
}

// ---------------------------------------------------------------- step
#define PK(cls, expr)                    \
  do {                                   \
    prof_mark(c, (cls), true, s);        \
    CKW(expr, #expr);                    \
    prof_mark(c, (cls), false, s);       \
  } while (0)

template <typename R>
static const R* pick(const double* d, const float* f);
template <>
const double* pick<double>(const double* d, const float*) { return d; }
template <>
const float* pick<float>(const double*, const float* f) { return f; }

template <typename R>
static afqmc_status run_energy(afqmc_ctx* c, const afqmc_walkers* w, double e0, double tau, double* e_loc,
                               double* e_mix, bool theta_ready = false) {
  cudaStream_t s = c->stream;
  const int Nw = w->n_walkers;
  if (!theta_ready)
    PK(AFQMC_K_OVERLAP, launch_overlap<R>(c, Nw, w->psi, c->ws.theta, c->ws.logdet, w->status, s));
  int nl = 0;
  CK(launch_energy<R>(c, Nw, w->weight, e0, tau, e_loc ? e_loc : c->ws.eloc, e_mix ? e_mix : c->ws.emix, s, &nl));
  // ws.epart now holds sum_s tr(Lh_gs Theta_s) of these walkers (a later step may reuse it)
  CK(launch_bias_mark(c, w->psi, Nw, s));
  c->launches += (theta_ready ? 0 : 1) + nl + 1;
  return AFQMC_OK;
}

// Arguments of the GEMM at one call site of the step (in -> out), tile variant
// from the context's tuning table.
template <typename R>
static GemmArgs site_args(const afqmc_ctx* c, int site, int Nw, double sqrt_tau, const void* in, void* out) {
  const int N = c->N, nc = c->nc, G = c->G;
  const long long per = (long long)nc * N, NN = (long long)N * N;
  GemmArgs g{};
  g.variant = c->tune[site];
  g.alpha_re = 1.0;
  g.B = in;
  g.C = out;
  g.batch = 1;
  switch (site) {
    case SITE_FORCEBIAS: {  // <L_g>_mixed[w][g] = sum_{jq} Lh[g][j][q] Theta[w][j][q]
      g.M = G; g.Nn = Nw; g.K = (int)per;
      g.A = pick<R>(c->d_Lh, c->f_Lh); g.sa_m = per; g.sa_k = 1;
      g.sb_n = per; g.sb_k = 1;
      g.sc_m = 1; g.sc_n = G;
      // few output tiles and a long K: split K over up to 8 slices (deterministic sum)
      const long long tiles = (long long)((G + 63) / 64) * ((Nw + 63) / 64);
      int sk = 1;
      while (sk < 8 && tiles * sk < 4 * 152 && per / (2 * sk) >= 256) sk *= 2;
      g.splitk = sk;
      g.part = c->ws.splitk;
      break;
    }
    case SITE_FIELD:  // A_w[pq] = i sqrt(tau) sum_g c_wg L_g[pq]
      g.M = (int)NN; g.Nn = Nw; g.K = G;
      g.A = pick<R>(c->d_L, c->f_L); g.sa_m = 1; g.sa_k = NN;
      g.sb_n = G; g.sb_k = 1;
      g.sc_m = 1; g.sc_n = NN;
      g.alpha_re = 0.0; g.alpha_im = sqrt_tau;
      break;
    case SITE_HALFSTEP:  // out[w][j][p] = sum_q B[p][q] in[w][j][q]
      g.M = N; g.Nn = Nw * nc; g.K = N;
      g.A = pick<R>(c->d_B, c->f_B); g.sa_m = N; g.sa_k = 1;
      g.sb_n = N; g.sb_k = 1;
      g.sc_m = 1; g.sc_n = N;
      break;
    default:  // SITE_EXPM: out[w][j][p] = sum_q A_w[p][q] in[w][j][q], batched over walkers
      g.M = N; g.Nn = nc; g.K = N; g.batch = Nw;
      g.A = c->ws.A; g.sa_m = N; g.sa_k = 1; g.sa_b = NN;
      g.sb_n = N; g.sb_k = 1; g.sb_b = per;
      g.sc_m = 1; g.sc_n = N; g.sc_b = per;
      break;
  }
  return g;
}

// Chebyshev coefficient c_n of e^x (Sec. IV.B): c_0 = J_0(i) = I_0(1) and
// c_n = 2 i^n J_n(-i) = 2 I_n(1), with the modified Bessel function from its
// power series I_n(1) = sum_m (1/2)^{2m+n} / (m! (m+n)!)
static double cheb_coef(int n) {
  double term = 1.0;
  for (int j = 1; j <= n; ++j) term *= 0.5 / j;  // (1/2)^n / n!
  double sum = 0.0;
  for (int m = 0; m < 40 && term > 1e-18 * sum; ++m) {
    sum += term;
    term *= 0.25 / ((m + 1.0) * (m + 1.0 + n));
  }
  return n == 0 ? sum : 2.0 * sum;
}

// Blocks of the block-Krylov layout for order k: room for min(k, N / n)
// blocks of either spin (at most N rows of A_k).
static int bk_blocks(const afqmc_ctx* c, int k) {
  const int nmax = c->na > c->nb ? c->na : c->nb;
  const int cap = (c->N + nmax - 1) / nmax;
  return k < cap ? k : cap;
}
// Whether the block-Krylov kernels' shared memory fits for order k.
static bool bk_fits(const afqmc_ctx* c, int k) {
  const int nmax = c->na > c->nb ? c->na : c->nb;
  if (nmax < 1) return false;
  const size_t cs = c->prec == AFQMC_FP64 ? 16 : 8;
  const size_t lim = (size_t)max_dyn_smem();
  return bk_expm_smem(bk_blocks(c, k), nmax, cs) <= lim && bk_orth_smem(c->N, nmax, cs) <= lim &&
         bk_combine_smem(c->N, bk_blocks(c, k), nmax, cs) <= lim;
}

template <typename R>
static afqmc_status run_step(afqmc_ctx* c, const afqmc_walkers* w, const double* x, const afqmc_step_params* p,
                             double* e_loc, double* e_mix) {
  cudaStream_t s = c->stream;
  const int Nw = w->n_walkers, nc = c->nc, N = c->N;
  const long long per = (long long)nc * N;
  const double st = std::sqrt(p->tau);
  Workspace& ws = c->ws;
  const size_t cs = sizeof(typename C2<R>::t);
  // out = B in: complex64 walkers on the tensor cores (in + (B - I) in; two
  // launches: the walker planes, then the contraction), else the tiled GEMM
  auto half = [&](const void* in, void* out) -> cudaError_t {
    if (std::is_same<R, float>::value && c->tg.hs_ok) {
      c->launches += 1;
      return tc_halfstep_launch(c, Nw, in, out, s);
    }
    if (std::is_same<R, float>::value && halfstep_ok(c)) return halfstep_launch(c, Nw, in, out, s);
    return gemm<R>(site_args<R>(c, SITE_HALFSTEP, Nw, st, in, out), false, EPI_STORE, s);
  };

  // <L_g> from the last measurement of these walkers when allowed and valid
  // (then the overlap and force-bias kernels return at once), else Theta and
  // the force-bias contraction
  PK(AFQMC_K_OTHER, launch_bias_gate(c, w->psi, Nw, p->reuse_bias ? 1 : 0, s));
  const int* skip = c->d_bias_skip;
  PK(AFQMC_K_OVERLAP, launch_overlap<R>(c, Nw, w->psi, ws.theta, ws.logdet, w->status, s, skip));
  // force bias (Eq. force_shift) and c_g = x_g - f_g
  GemmArgs gfb = site_args<R>(c, SITE_FORCEBIAS, Nw, st, ws.theta, ws.t);
  gfb.skip = skip;
  PK(AFQMC_K_FORCEBIAS, gemm<R>(gfb, false, EPI_STORE, s));
  PK(AFQMC_K_OTHER, launch_bias_finalize<R>(c, Nw, x, st, s, nullptr, skip));
  // A_w = i sqrt(tau) sum_g c_wg L_g (Eq. heffTOT); complex64 walkers: on the
  // tensor cores, into the A' operand planes, or for the Taylor and
  // Crank-Nicolson propagators, which need X_w = A_w - tau h'' in memory, into
  // ws.A (then the shift)
  const bool split1 = p->propagator == AFQMC_SPLIT1, tprop = p->propagator == AFQMC_TAYLORPROP,
             cn = p->propagator == AFQMC_CN, xmat = tprop || cn;
  if (std::is_same<R, float>::value && c->tg.ok) {
    PK(AFQMC_K_FIELD, tc_field_launch(c, Nw, st, s, xmat));
    c->launches += 1;
  } else {
    PK(AFQMC_K_FIELD, gemm<R>(site_args<R>(c, SITE_FIELD, Nw, st, ws.c, ws.A), false, EPI_STORE, s));
  }
  if (xmat) {
    PK(AFQMC_K_FIELD, launch_shift_field<R>(c, Nw, p->tau, s));
    c->launches += 1;
  }
  // psi_b = B psi (Split-2); the other propagators start from psi itself
  if (split1 || xmat) {
    CKW(cudaMemcpyAsync(ws.psi_b, w->psi, (size_t)Nw * per * cs, cudaMemcpyDeviceToDevice, s), "psi copy");
  } else {
    PK(AFQMC_K_HALFSTEP, half(w->psi, ws.psi_b));
  }
  c->launches += (split1 || xmat) ? 5 : 6;

  // per-walker products with A_w (tensor cores for complex64 walkers)
  GemmArgs ga = site_args<R>(c, SITE_EXPM, Nw, st, nullptr, nullptr);
  const bool tc_av = std::is_same<R, float>::value && c->tg.av_ok && !xmat;
  auto av = [&](const void* in, void* out, void* add, double alpha) -> cudaError_t {
    if (tc_av) return tc_av_launch(c, Nw, in, per, out, add, per, alpha, s);
    ga.B = in; ga.C = out; ga.D = add;
    ga.alpha_re = alpha; ga.alpha_im = 0.0;
    return gemm<R>(ga, true, add ? EPI_STORE_ADD : EPI_STORE, s);
  };
  if (cn) {
    // Crank-Nicolson (Sec. III.D): psi_new = (I - X/2)^{-1} (psi + X psi / 2),
    // the right-hand side by one product, then one pivoted solve per walker
    CKW(cudaMemcpyAsync(ws.acc, ws.psi_b, (size_t)Nw * per * cs, cudaMemcpyDeviceToDevice, s), "acc copy");
    PK(AFQMC_K_EXPM, av(ws.psi_b, ws.term0, ws.acc, 0.5));
    CKW(cudaMemcpyAsync(ws.psi_new, ws.acc, (size_t)Nw * per * cs, cudaMemcpyDeviceToDevice, s), "rhs copy");
    PK(AFQMC_K_OTHER, launch_cn_solve<R>(c, Nw, ws.A, ws.psi_new, s));
    c->launches += 2;
  } else if (p->expm == AFQMC_EXPM_TAYLOR) {
    CKW(cudaMemcpyAsync(ws.acc, ws.psi_b, (size_t)Nw * per * cs, cudaMemcpyDeviceToDevice, s), "acc copy");
    const void* cur = ws.psi_b;
    for (int n = 1; n <= p->order; ++n) {
      void* nxt = (n & 1) ? ws.term0 : ws.term1;
      PK(AFQMC_K_EXPM, av(cur, nxt, ws.acc, 1.0 / n));
      cur = nxt;
    }
    c->launches += p->order * (tc_av ? 2 : 1);
  } else if (p->expm == AFQMC_EXPM_CHEBYSHEV) {
    // Chebyshev (Eq. chebpoly): T_0 Psi = psi_b, T_1 Psi = A psi_b, then
    // T_n Psi = 2 A T_{n-1} Psi - T_{n-2} Psi in place of T_{n-2} Psi (the
    // product goes to psi_new, free until the last half step), acc = sum c_n T_n Psi
    const int k = p->order;
    if (k == 0) {
      PK(AFQMC_K_OTHER, launch_cheb_step<R>(c, Nw, ws.psi_b, ws.psi_b, ws.acc, cheb_coef(0), 0.0, 1, s));
      c->launches += 1;
    } else {
      PK(AFQMC_K_EXPM, av(ws.psi_b, ws.term0, nullptr, 1.0));
      PK(AFQMC_K_OTHER, launch_cheb_step<R>(c, Nw, ws.term0, ws.psi_b, ws.acc, cheb_coef(0), cheb_coef(1), 1, s));
      void* prev = ws.psi_b;
      void* cur = ws.term0;
      for (int n = 2; n <= k; ++n) {
        PK(AFQMC_K_EXPM, av(cur, ws.psi_new, nullptr, 2.0));
        PK(AFQMC_K_OTHER, launch_cheb_step<R>(c, Nw, ws.psi_new, prev, ws.acc, 0.0, cheb_coef(n), 0, s));
        std::swap(prev, cur);
      }
      c->launches += k * ((tc_av ? 2 : 1) + 1);
    }
  } else if (p->expm == AFQMC_EXPM_BLOCK_KRYLOV) {
    // block Krylov (Eq. bkrylov): QR, then per block the products A B_j and
    // one block Arnoldi step, then e^{A_k} E_n R and B_k F into acc
    const int k = p->order;
    const size_t bstride = (size_t)ws.n_walkers * per;
    const int nmin = (c->na > 0 && c->nb > 0) ? (c->na < c->nb ? c->na : c->nb) : (c->na > 0 ? c->na : c->nb);
    const int jmax = k < N / nmin ? k : N / nmin;  // blocks of the spin with the most
    if (tc_av)
      PK(AFQMC_K_OTHER, tc_av_normA(c, Nw, s));
    else
      PK(AFQMC_K_OTHER, launch_normA<R>(c, Nw, s));
    PK(AFQMC_K_OTHER, launch_bk_start<R>(c, Nw, k, s));
    for (int j = 0; j < jmax; ++j) {
      PK(AFQMC_K_EXPM, av(static_cast<char*>(ws.basis) + j * bstride * cs, ws.term0, nullptr, 1.0));
      PK(AFQMC_K_OTHER, launch_bk_orth<R>(c, Nw, j, s));
    }
    PK(AFQMC_K_OTHER, launch_bk_finish<R>(c, Nw, s));
    c->launches += 2 + jmax * (tc_av ? 3 : 2) + 2;
  } else {
    // Krylov (Eq. krylov): Arnoldi with modified Gram-Schmidt, or the
    // complex-symmetric Lanczos recurrence on the same space
    const int k = p->order;
    const bool lz = p->expm == AFQMC_EXPM_LANCZOS;
    const size_t bstride = (size_t)ws.n_walkers * per;
    if (tc_av)
      PK(AFQMC_K_OTHER, tc_av_normA(c, Nw, s));
    else
      PK(AFQMC_K_OTHER, launch_normA<R>(c, Nw, s));
    PK(AFQMC_K_OTHER, lz ? launch_lanczos_init<R>(c, Nw, s) : launch_krylov_init<R>(c, Nw, s));
    for (int it = 0; it < k; ++it) {
      // tensor-core products read b_it from the planes the Arnoldi kernels wrote
      PK(AFQMC_K_EXPM, av(tc_av ? nullptr : static_cast<char*>(ws.basis) + it * bstride * cs, ws.term0, nullptr,
                          1.0));
      PK(AFQMC_K_OTHER, lz ? launch_lanczos_step<R>(c, Nw, it, k, s) : launch_krylov_orth<R>(c, Nw, it, k, s));
    }
    PK(AFQMC_K_OTHER, launch_krylov_finish<R>(c, Nw, k, s, lz));
    c->launches += 2 + 2 * k + 2;
  }
  // psi_new = B acc (Split-2); B B acc = e^{-tau h''} acc (Split-1); acc itself
  // (the Taylor propagator)
  if (cn) {
    c->launches -= 1;  // psi_new holds the solution
  } else if (tprop) {
    CKW(cudaMemcpyAsync(ws.psi_new, ws.acc, (size_t)Nw * per * cs, cudaMemcpyDeviceToDevice, s), "acc copy");
    c->launches -= 1;
  } else if (split1) {
    PK(AFQMC_K_HALFSTEP, half(ws.acc, ws.term1));
    PK(AFQMC_K_HALFSTEP, half(ws.term1, ws.psi_new));
    c->launches += 1;
  } else {
    PK(AFQMC_K_HALFSTEP, half(ws.acc, ws.psi_new));
  }
  // new overlap (and Theta for the local energy), weights, commit.  Theta =
  // Psi (trial^T Psi)^{-1} is unchanged by the re-orthonormalisation Psi ->
  // Psi R^{-1}, and the log-overlap moves by -sum log R_jj, so no second
  // overlap is needed after it.
  void* th_new = p->measure ? ws.theta : nullptr;
  PK(AFQMC_K_OVERLAP, launch_overlap<R>(c, Nw, ws.psi_new, th_new, ws.logdet, w->status, s));
  PK(AFQMC_K_OTHER, launch_weights<R>(c, w, p->tau, p->e0, s));
  PK(AFQMC_K_OTHER, launch_commit<R>(c, w, p->reortho, s));
  c->launches += 4;
  if (p->reortho) {
    PK(AFQMC_K_OTHER, launch_mgs<R>(c, Nw, w->psi, ws.alive, ws.logdet, s));
    PK(AFQMC_K_OTHER, launch_logovl_shift(c, w, ws.alive, s));
    c->launches += 2;
  }
  // Theta of every live walker is the one of its committed determinant (for
  // walkers that were already dead it is that of the discarded proposal; their
  // local energy is unspecified and they do not enter E_k)
  if (p->measure) return run_energy<R>(c, w, p->e0, p->tau, e_loc, e_mix, true);
  return AFQMC_OK;
}

// Time every tile variant of every GEMM call site on the workspace (contents
// irrelevant for timing) and keep the fastest in the context.
template <typename R>
static afqmc_status autotune_impl(afqmc_ctx* c, int Nw, int order) {
  cudaStream_t s = c->stream;
  Workspace& ws = c->ws;
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  const bool prof = c->prof.on;
  c->prof.on = false;
  afqmc_status rc = AFQMC_OK;
  for (int site = 0; site < N_SITES && rc == AFQMC_OK; ++site) {
    if (site == SITE_EXPM && order < 1) continue;
    float best = 1e30f;
    int best_v = 0;
    for (int v = 0; v < GEMM_VARIANTS; ++v) {
      c->tune[site] = v;
      GemmArgs g;
      bool ac = false;
      if (site == SITE_FORCEBIAS) g = site_args<R>(c, site, Nw, 0.2, ws.theta, ws.t);
      else if (site == SITE_FIELD) g = site_args<R>(c, site, Nw, 0.2, ws.c, ws.A);
      else if (site == SITE_HALFSTEP) g = site_args<R>(c, site, Nw, 0.2, ws.psi_b, ws.psi_new);
      else { g = site_args<R>(c, site, Nw, 0.2, ws.psi_b, ws.term0); ac = true; }
      float tmin = 1e30f;
      for (int rep = 0; rep < 4 && rc == AFQMC_OK; ++rep) {
        cudaError_t e = cudaEventRecord(e0, s);
        if (e == cudaSuccess) e = gemm<R>(g, ac, EPI_STORE, s);
        if (e == cudaSuccess) e = cudaEventRecord(e1, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess) { rc = cuda_fail(e); break; }
        if (rep > 0 && ms < tmin) tmin = ms;  // the first launch is a warm-up
        c->launches += g.splitk > 1 ? 2 : 1;
      }
      if (tmin < best) { best = tmin; best_v = v; }
    }
    c->tune[site] = best_v;
  }
  c->prof.on = prof;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return rc;
}

// ---------------------------------------------------------------- batches
namespace {
constexpr int kBatchGraphs = 4;
struct BatchGraph {
  bool used = false;
  uint64_t stamp = 0;
  std::vector<unsigned char> key;
  cudaGraphExec_t exec = nullptr;
  std::vector<uint64_t> launches;  // kernel launches per system in one replay
};
}  // namespace

struct afqmc_batch {
  std::vector<afqmc_ctx*> ctxs;
  std::vector<cudaStream_t> branch;
  std::vector<cudaEvent_t> join;
  cudaStream_t origin = nullptr;
  cudaEvent_t fork = nullptr, done = nullptr;
  BatchGraph graphs[kBatchGraphs];
  uint64_t clock = 0;
};

static void batch_free(afqmc_batch* b) {
  if (!b) return;
  for (auto& g : b->graphs)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  for (auto s : b->branch) cudaStreamDestroy(s);
  for (auto e : b->join) cudaEventDestroy(e);
  if (b->origin) cudaStreamDestroy(b->origin);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->done) cudaEventDestroy(b->done);
  delete b;
}

// ---------------------------------------------------------------- walk adjoint
namespace {
// Bump allocator over one device allocation (a dry run with base == nullptr
// only counts the bytes).
struct Arena {
  char* base = nullptr;
  size_t used = 0;
  template <typename T>
  T* take(size_t n) {
    const size_t a = (used + 255) & ~(size_t)255;
    used = a + n * sizeof(T);
    return base ? reinterpret_cast<T*>(base + a) : nullptr;
  }
};

template <typename R>
struct AdjBufs {
  typedef typename C2<R>::t P;
  // walker states, their adjoints and the walker-shaped intermediates
  P *ck_psi, *seg_psi, *run_psi, *P0, *Tb, *Ub, *psi2, *psi3, *pb, *p3, *p2, *p1, *thbar, *Abar, *cbar, *tbar, *part;
  // complex64 walkers: one step's contributions to Bbar, gLc and Lhb before
  // they are added to the FP64 sums (NULL for complex128 walkers)
  P *sB, *sL, *sLh;
  double2 *oinv3, *oinvk, *aR, *gLc, *Lhb, *Bbar, *ys;
  double *ck_W, *ck_lo, *seg_lo, *run_W, *run_lo, *Wfin, *mu_part, *ld3, *ldk, *omega, *ecoef, *mubar, *V, *lam, *Bs,
      *T1, *M1, *hbar, *X, *D, *eloc, *emix;
  uint32_t *ck_st, *run_st, *st_scr;
  uint8_t* keep;
  int skc, skb;  // split-K factors of the two long-K contractions
  // Krylov action (NULL for the Taylor one): the Hessenberg block before the
  // small exponential, its adjoint, g_y, the start-norm adjoint, the adjoint
  // U_j of A b_j and the Lanczos recurrence's per-column carry
  P *Hs, *kU;
  double2 *GH, *gy, *gbeta, *carry;
};

int pick_splitk(long long M, long long Nn, long long K, int cap) {
  const long long tiles = ((M + 63) / 64) * ((Nn + 63) / 64);
  int sk = 1;
  while (sk < cap && tiles * sk < 4 * 152 && K / (2 * sk) >= 256) sk *= 2;
  return sk;
}

GemmArgs gargs(int M, int Nn, int K, int batch, const void* A, long long sa_m, long long sa_k, long long sa_b,
               const void* B, long long sb_n, long long sb_k, long long sb_b, void* C, long long sc_m, long long sc_n,
               long long sc_b, double are = 1.0, double aim = 0.0) {
  GemmArgs g{};
  g.M = M; g.Nn = Nn; g.K = K; g.batch = batch;
  g.A = A; g.sa_m = sa_m; g.sa_k = sa_k; g.sa_b = sa_b;
  g.B = B; g.sb_n = sb_n; g.sb_k = sb_k; g.sb_b = sb_b;
  g.C = C; g.sc_m = sc_m; g.sc_n = sc_n; g.sc_b = sc_b;
  g.alpha_re = are; g.alpha_im = aim;
  return g;
}
}  // namespace

template <typename R>
static void adj_carve(Arena& a, AdjBufs<R>& b, const afqmc_ctx* c, int Nw, int K, int C, int nck, bool krylov) {
  const size_t nw = (size_t)Nw, per = (size_t)c->nc * c->N, NN = (size_t)c->N * c->N, G = (size_t)c->G;
  typedef typename C2<R>::t P;
  const size_t nmax = (size_t)(c->na > c->nb ? c->na : c->nb);
  b.ck_psi = a.take<P>((size_t)nck * nw * per);
  b.ck_W = a.take<double>((size_t)nck * nw);
  b.ck_lo = a.take<double>((size_t)nck * nw * 2);
  b.ck_st = a.take<uint32_t>((size_t)nck * nw);
  b.seg_psi = a.take<P>((size_t)(C + 1) * nw * per);
  b.seg_lo = a.take<double>((size_t)(C + 1) * nw * 2);
  b.run_psi = a.take<P>(nw * per);
  b.run_W = a.take<double>(nw);
  b.run_lo = a.take<double>(nw * 2);
  b.run_st = a.take<uint32_t>(nw);
  b.st_scr = a.take<uint32_t>(nw);
  b.Wfin = a.take<double>(nw);
  b.P0 = a.take<P>(nw * per);
  b.Tb = a.take<P>(nw * (K + 1) * per);
  b.Ub = a.take<P>(nw * K * per);
  b.psi2 = a.take<P>(nw * per);
  b.psi3 = a.take<P>(nw * per);
  b.pb = a.take<P>(nw * per);
  b.p3 = a.take<P>(nw * per);
  b.p2 = a.take<P>(nw * per);
  b.p1 = a.take<P>(nw * per);
  b.thbar = a.take<P>(nw * per);
  b.Abar = a.take<P>(nw * NN);
  b.cbar = a.take<P>(nw * G);
  b.tbar = a.take<P>(nw * G);
  b.keep = a.take<uint8_t>(nw * G);
  b.mu_part = a.take<double>(nw * G);
  b.oinv3 = a.take<double2>(nw * 2 * nmax * nmax);
  b.oinvk = a.take<double2>(nw * 2 * nmax * nmax);
  b.ld3 = a.take<double>(nw * 4);
  b.ldk = a.take<double>(nw * 4);
  b.aR = a.take<double2>(nw);
  b.omega = a.take<double>(nw);
  b.ecoef = a.take<double>(nw);
  b.gLc = a.take<double2>(G * NN);
  b.Lhb = a.take<double2>(G * per);
  b.Bbar = a.take<double2>(NN);
  b.mubar = a.take<double>(G);
  const size_t pc = (size_t)b.skc * G * nw, pbb = (size_t)b.skb * NN;
  b.part = a.take<P>(pc > pbb ? pc : pbb);
  b.ys = a.take<double2>(per + G * per);
  const bool split = std::is_same<R, float>::value;
  b.sB = split ? a.take<P>(NN) : nullptr;
  b.sL = split ? a.take<P>(G * NN) : nullptr;
  b.sLh = split ? a.take<P>(G * per) : nullptr;
  b.V = a.take<double>(NN);
  b.lam = a.take<double>((size_t)c->N);
  b.Bs = a.take<double>(NN);
  b.T1 = a.take<double>(NN);
  b.M1 = a.take<double>(NN);
  b.hbar = a.take<double>(NN);
  b.X = a.take<double>(G * NN);
  b.D = a.take<double>(NN);
  b.eloc = a.take<double>(nw * 2);
  b.emix = a.take<double>(4);
  const size_t hs = (size_t)c->ws.n_walkers * c->nc, km = (size_t)c->ws.kmax;
  b.Hs = krylov ? a.take<P>(km * km * hs) : nullptr;
  b.GH = krylov ? a.take<double2>(km * km * hs) : nullptr;
  b.gy = krylov ? a.take<double2>(km * hs) : nullptr;
  b.gbeta = krylov ? a.take<double2>(hs) : nullptr;
  b.carry = krylov ? a.take<double2>(hs) : nullptr;
  b.kU = krylov ? a.take<P>(nw * per) : nullptr;
}

// One reverse step k of the walk: recompute Theta_k, f, c, A, the action of
// e^A (Taylor terms, or the Krylov basis, Hessenberg (or Lanczos tridiagonal,
// lz) matrix and products A b_j when kry > 0 is the Krylov dimension) and
// Psi3 from the stored Psi_k,
// then pull the adjoint Psi_bar_{k+1} (in b.pb) back to Psi_bar_k (in b.pb)
// and accumulate the parameter adjoints.  With complex64 walkers the
// contractions run in FP32 and the parameter adjoints of the step are added
// to their FP64 sums once per step.
template <typename R>
static afqmc_status adj_step(afqmc_ctx* c, const AdjBufs<R>& b, int Nw, const double* x,
                             const typename C2<R>::t* psik, const double* lok, const typename C2<R>::t* psinext, int qr,
                             int K, int kry, bool lz, double tau) {
  typedef typename C2<R>::t P;
  constexpr bool split = std::is_same<R, float>::value;
  cudaStream_t s = c->stream;
  Workspace& ws = c->ws;
  const int N = c->N, nc = c->nc, G = c->G;
  const size_t per = (size_t)nc * N, NN = (size_t)N * N, cs = sizeof(P);
  const long long perl = (long long)per, NNl = (long long)NN;
  const double st = std::sqrt(tau);
  uint64_t nl = 0;
  auto gm = [&](const GemmArgs& g, bool ac, int epi) -> cudaError_t {
    nl += (g.splitk > 1 && g.part && g.batch == 1 && epi != EPI_STORE_ADD) ? 2 : 1;
    return gemm<R>(g, ac, epi, s);
  };
  // parameter adjoint: straight into the FP64 sum, or into the step's
  // complex64 buffer (stored by the first contribution, added by the rest)
  auto pacc = [&](double2* sum, P* step_buf, bool first) -> std::pair<void*, int> {
    if (!split) return {sum, EPI_ACC};
    return {step_buf, first ? EPI_STORE : EPI_ACC};
  };
  P* theta = static_cast<P*>(ws.theta);
  // forward quantities of step k (same kernels as the step, so the kept
  // force-bias components are the forward's)
  CKW(adj_sanitize<R>(psik, b.P0, b.Wfin, c->d_trial, per, Nw, s), "adjoint: sanitise");
  CKW(launch_overlap<R>(c, Nw, b.P0, ws.theta, ws.logdet, b.st_scr, s), "adjoint: overlap");
  CKW(gm(site_args<R>(c, SITE_FORCEBIAS, Nw, st, ws.theta, ws.t), false, EPI_STORE), "adjoint: force bias");
  CKW(launch_bias_finalize<R>(c, Nw, x, st, s, b.keep), "adjoint: bias finalise");
  CKW(gm(site_args<R>(c, SITE_FIELD, Nw, st, ws.c, ws.A), false, EPI_STORE), "adjoint: field");
  nl += 3;
  const long long tstride = (long long)(K + 1) * perl, ustride = (long long)K * perl;
  // Krylov planes: product A b_j in Tb plane j, g_b_j in Ub plane j (kp apart)
  const size_t kp = (size_t)Nw * per;
  if (kry > 0) {
    CKW(gm(site_args<R>(c, SITE_HALFSTEP, Nw, st, b.P0, ws.psi_b), false, EPI_STORE), "adjoint: half step");
    CKW(launch_normA<R>(c, Nw, s), "adjoint: norm of A");
    CKW(lz ? launch_lanczos_init<R>(c, Nw, s) : launch_krylov_init<R>(c, Nw, s), "adjoint: Krylov start");
    GemmArgs ga = site_args<R>(c, SITE_EXPM, Nw, st, nullptr, nullptr);
    const size_t bstride = (size_t)ws.n_walkers * per;
    for (int j = 0; j < kry; ++j) {
      ga.B = static_cast<const P*>(ws.basis) + j * bstride;
      ga.C = b.Tb + j * kp;
      CKW(gm(ga, true, EPI_STORE), "adjoint: Krylov product");
      CKW(lz ? launch_lanczos_step<R>(c, Nw, j, kry, s, b.Tb + j * kp)
             : launch_krylov_orth<R>(c, Nw, j, kry, s, b.Tb + j * kp),
          "adjoint: Krylov step");
    }
    const size_t hs = (size_t)ws.n_walkers * nc;
    CKW(cudaMemcpyAsync(b.Hs, ws.hess, (size_t)ws.kmax * ws.kmax * hs * cs, cudaMemcpyDeviceToDevice, s),
        "adjoint: Hessenberg copy");
    CKW(launch_krylov_finish<R>(c, Nw, kry, s, lz), "adjoint: Krylov finish");
    CKW(cudaMemcpyAsync(b.psi2, ws.acc, (size_t)Nw * per * cs, cudaMemcpyDeviceToDevice, s), "adjoint: copy");
    nl += kry + 3;  // norm, start, Arnoldi steps, small exponential and combination; no Taylor sum
  } else {
    CKW(gm(gargs(N, nc, N, Nw, pick<R>(c->d_B, c->f_B), N, 1, 0, b.P0, N, 1, perl, b.Tb, 1, N, tstride), false,
           EPI_STORE),
        "adjoint: half step");
    GemmArgs ga = site_args<R>(c, SITE_EXPM, Nw, st, nullptr, nullptr);
    ga.sb_b = tstride;
    ga.sc_b = tstride;
    for (int j = 1; j <= K; ++j) {
      ga.B = b.Tb + (size_t)(j - 1) * per;
      ga.C = b.Tb + (size_t)j * per;
      ga.alpha_re = 1.0 / j;
      ga.alpha_im = 0.0;
      CKW(gm(ga, true, EPI_STORE), "adjoint: Taylor term");
    }
    CKW(adj_sum_terms<R>(b.Tb, b.psi2, K + 1, per, Nw, s), "adjoint: Taylor sum");
  }
  CKW(gm(site_args<R>(c, SITE_HALFSTEP, Nw, st, b.psi2, b.psi3), false, EPI_STORE), "adjoint: half step");
  // overlap ratio and weight: Psi3_bar
  CKW(adj_lu<R>(c, Nw, b.psi3, b.oinv3, b.ld3, s), "adjoint: new overlap");
  CKW(adj_ratio_coef(Nw, b.Wfin, b.omega, b.ld3, lok, ws.scal, b.aR, st, s), "adjoint: ratio coefficient");
  CKW(adj_ratio<R>(c, Nw, b.pb, psinext, b.oinv3, b.aR, b.Wfin, b.p3, qr, s), "adjoint: ratio");
  nl += 4;
  // second half step: Psi2_bar = B Psi3_bar, Bbar += Psi3_bar Psi2^T
  CKW(gm(site_args<R>(c, SITE_HALFSTEP, Nw, st, b.p3, b.p2), false, EPI_STORE), "adjoint: half step");
  auto bb = pacc(b.Bbar, b.sB, true);
  GemmArgs gb = gargs(N, N, Nw * nc, 1, b.p3, 1, N, 0, b.psi2, 1, N, 0, bb.first, N, 1, 0);
  gb.splitk = b.skb;
  gb.part = b.part;
  CKW(gm(gb, true, bb.second), "adjoint: B adjoint");
  if (kry > 0) {
    // Krylov action: seed from out = sum_i y_i b_i, the adjoint of the small
    // exponential, then the Arnoldi (or Lanczos) steps in reverse; per step j
    // the adjoint U_j of A b_j gives g_b_j += A U_j and A_bar += U_j b_j^T
    CKW(kadj_seed<R>(c, Nw, kry, b.p2, b.Ub, kp, b.gy, s), "adjoint: Krylov seed");
    CKW(kadj_expm<R>(c, Nw, kry, b.Hs, b.gy, b.GH, b.gbeta, lz, s), "adjoint: small exponential");
    const size_t bstride = (size_t)ws.n_walkers * per;
    for (int j = kry - 1; j >= 0; --j) {
      CKW(lz ? lzadj_step<R>(c, Nw, j, kry, b.Tb + j * kp, b.Hs, b.GH, b.Ub, kp, b.kU, b.carry, s)
             : kadj_orth<R>(c, Nw, j, kry, b.Tb + j * kp, b.Hs, b.GH, b.Ub, kp, b.kU, s),
          "adjoint: Krylov step");
      CKW(gm(site_args<R>(c, SITE_EXPM, Nw, st, b.kU, b.Ub + j * kp), true, EPI_ACC), "adjoint: Krylov product");
      CKW(gm(gargs(N, N, nc, Nw, b.kU, 1, N, perl, static_cast<const P*>(ws.basis) + j * bstride, 1, N, perl, b.Abar,
                   N, 1, NNl),
             true, j == kry - 1 ? EPI_STORE : EPI_ACC),
          "adjoint: A adjoint");
    }
    CKW(kadj_input<R>(c, Nw, b.Ub, b.gbeta, b.p1, lz, s), "adjoint: Krylov start");
    nl += kry + 3;  // seed, small exponential, Arnoldi steps, start
  } else {
    // Taylor action: U_j = T_bar_j / j in Ub slot j-1, T_bar_{j-1} = Psi2_bar + A U_j
    CKW(adj_scale_copy<R>(b.p2, per, b.Ub + (size_t)(K - 1) * per, (size_t)K * per, 1.0 / K, per, Nw, s),
        "adjoint: Taylor seed");
    ++nl;
    GemmArgs gu = site_args<R>(c, SITE_EXPM, Nw, st, nullptr, nullptr);
    gu.sb_b = ustride;
    gu.sc_b = ustride;
    for (int j = K; j >= 2; --j) {
      CKW(adj_scale_copy<R>(b.p2, per, b.Ub + (size_t)(j - 2) * per, (size_t)K * per, 1.0 / (j - 1), per, Nw, s),
          "adjoint: Taylor copy");
      gu.B = b.Ub + (size_t)(j - 1) * per;
      gu.C = b.Ub + (size_t)(j - 2) * per;
      gu.alpha_re = 1.0 / (j - 1);
      gu.alpha_im = 0.0;
      CKW(gm(gu, true, EPI_ACC), "adjoint: Taylor adjoint");
      ++nl;
    }
    CKW(cudaMemcpyAsync(b.p1, b.p2, (size_t)Nw * per * cs, cudaMemcpyDeviceToDevice, s), "adjoint: copy");
    GemmArgs g1 = site_args<R>(c, SITE_EXPM, Nw, st, b.Ub, b.p1);
    g1.sb_b = ustride;
    CKW(gm(g1, true, EPI_ACC), "adjoint: Taylor adjoint");
    // A_bar[w] = sum_j U_j T_{j-1}^T
    CKW(gm(gargs(N, N, K * nc, Nw, b.Ub, 1, N, ustride, b.Tb, 1, N, tstride, b.Abar, N, 1, NNl), true, EPI_STORE),
        "adjoint: A adjoint");
  }
  // A = i sqrt(tau) sum_g c_g L_g: c_bar = i sqrt(tau) <L_g, A_bar>, L_bar_g += i sqrt(tau) sum_w c_wg A_bar_w
  GemmArgs gc = gargs(G, Nw, (int)NN, 1, pick<R>(c->d_L, c->f_L), NNl, 1, 0, b.Abar, NNl, 1, 0, b.cbar, 1, G, 0, 0.0,
                      st);
  gc.splitk = b.skc;
  gc.part = b.part;
  CKW(gm(gc, false, EPI_STORE), "adjoint: c adjoint");
  auto bl = pacc(b.gLc, b.sL, true);
  CKW(gm(gargs(G, (int)NN, Nw, 1, ws.c, 1, G, 0, b.Abar, 1, NNl, 0, bl.first, NNl, 1, 0, 0.0, st), true, bl.second),
      "adjoint: L adjoint (field)");
  // force bias and scalar factor
  CKW(adj_force<R>(c, Nw, b.cbar, static_cast<const P*>(ws.c), b.keep, b.aR, b.omega, b.tbar, b.mu_part, b.mubar,
                   st, tau, s),
      "adjoint: force bias");
  nl += 2;
  // t_g = sum tr(Lh_g Theta): Theta_bar = sum_g t_bar_g Lh_g^T, Lh_bar_g += sum_w t_bar_wg Theta_w
  CKW(gm(gargs((int)per, Nw, G, 1, pick<R>(c->d_Lh, c->f_Lh), 1, perl, 0, b.tbar, G, 1, 0, b.thbar, 1, perl, 0), false,
         EPI_STORE),
      "adjoint: Theta adjoint");
  auto bh = pacc(b.Lhb, b.sLh, true);
  CKW(gm(gargs(G, (int)per, Nw, 1, b.tbar, 1, G, 0, ws.theta, 1, perl, 0, bh.first, perl, 1, 0), true, bh.second),
      "adjoint: Lh adjoint");
  // first half step and Theta = Psi O^{-1}: Psi_bar_k
  CKW(gm(site_args<R>(c, SITE_HALFSTEP, Nw, st, b.p1, b.pb), false, EPI_STORE), "adjoint: half step");
  auto bb2 = pacc(b.Bbar, b.sB, false);
  GemmArgs gb2 = gargs(N, N, Nw * nc, 1, b.p1, 1, N, 0, b.P0, 1, N, 0, bb2.first, N, 1, 0);
  gb2.splitk = b.skb;
  gb2.part = b.part;
  CKW(gm(gb2, true, bb2.second), "adjoint: B adjoint");
  CKW(adj_lu<R>(c, Nw, b.P0, b.oinvk, b.ldk, s), "adjoint: overlap inverse");
  CKW(adj_theta<R>(c, Nw, b.thbar, theta, b.oinvk, b.aR, b.Wfin, b.pb, s), "adjoint: Theta pull-back");
  nl += 2;
  if (split) {
    CKW(adj_fold(reinterpret_cast<const float2*>(b.sB), b.Bbar, NN, s), "adjoint: B sum");
    CKW(adj_fold(reinterpret_cast<const float2*>(b.sL), b.gLc, (size_t)G * NN, s), "adjoint: L sum");
    CKW(adj_fold(reinterpret_cast<const float2*>(b.sLh), b.Lhb, (size_t)G * per, s), "adjoint: Lh sum");
    nl += 3;
  }
  c->launches += nl;
  return AFQMC_OK;
}

template <typename R>
static afqmc_status walk_backward_run(afqmc_ctx* c, const afqmc_walkers* w0, const double* fields,
                                      const afqmc_walk_adjoint_params* p, double* J_out, double* grad_h1,
                                      double* grad_L, void* grad_psi0, const AdjBufs<R>& b) {
  typedef typename C2<R>::t P;
  cudaStream_t s = c->stream;
  const int Nw = w0->n_walkers, N = c->N, nc = c->nc, G = c->G, K = p->order, C = p->ckpt_every, n = p->n_steps;
  const size_t per = (size_t)nc * N, NN = (size_t)N * N, cs = sizeof(P), nw = (size_t)Nw;
  const size_t fstride = nw * G;
  const int nck = (n + C - 1) / C;
  const cudaMemcpyKind dd = cudaMemcpyDeviceToDevice;
  afqmc_walkers run{};
  run.n_walkers = Nw;
  run.psi = b.run_psi;
  run.weight = b.run_W;
  run.logovl = b.run_lo;
  run.status = b.run_st;
  auto copy_state = [&](void* dp, double* dW, double* dl, uint32_t* ds, const void* sp, const double* sW,
                        const double* sl, const uint32_t* ss) -> cudaError_t {
    cudaError_t e = cudaMemcpyAsync(dp, sp, nw * per * cs, dd, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dW, sW, nw * sizeof(double), dd, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dl, sl, nw * 2 * sizeof(double), dd, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(ds, ss, nw * sizeof(uint32_t), dd, s);
    return e;
  };
  afqmc_step_params sp{};
  sp.tau = p->tau;
  sp.e0 = p->e0;
  sp.propagator = AFQMC_SPLIT2;
  // Taylor action of order K, or the Krylov (Arnoldi or Lanczos) one of
  // dimension kry = min(K, N)
  const bool lz = p->expm == AFQMC_EXPM_LANCZOS;
  const int kry = (p->expm == AFQMC_EXPM_KRYLOV || lz) ? (K < N ? K : N) : 0;
  sp.expm = kry > 0 ? p->expm : AFQMC_EXPM_TAYLOR;
  sp.order = kry > 0 ? kry : K;
  sp.measure = 0;
  auto qr_at = [&](int k) { return (p->reortho_every > 0 && (k + 1) % p->reortho_every == 0) ? 1 : 0; };

  // forward walk with checkpoints, then J
  CKW(copy_state(run.psi, run.weight, run.logovl, run.status, w0->psi, w0->weight, w0->logovl, w0->status),
      "adjoint: copy walkers");
  for (int k = 0; k < n; ++k) {
    if (k % C == 0) {
      const size_t sl = (size_t)(k / C);
      CKW(copy_state(b.ck_psi + sl * nw * per, b.ck_W + sl * nw, b.ck_lo + sl * nw * 2, b.ck_st + sl * nw, run.psi,
                     run.weight, run.logovl, run.status),
          "adjoint: checkpoint");
    }
    sp.reortho = qr_at(k);
    afqmc_status rc = run_step<R>(c, &run, fields + (size_t)k * fstride, &sp, nullptr, nullptr);
    if (rc != AFQMC_OK) return rc;
  }
  afqmc_status rc = run_energy<R>(c, &run, p->e0, p->tau, b.eloc, b.emix);
  if (rc != AFQMC_OK) return rc;
  CKW(cudaMemcpyAsync(b.Wfin, run.weight, nw * sizeof(double), dd, s), "adjoint: copy");
  if (J_out) CKW(cudaMemcpyAsync(J_out, b.emix, 4 * sizeof(double), dd, s), "adjoint: copy");

  // seeds: E_L part of the parameter gradients and Psi_bar_n
  const int ne = c->na + c->nb;
  const double dE = 0.5 * std::sqrt(ne / p->tau) + std::sqrt(ne * p->tau);
  const double st = std::sqrt(p->tau);
  CKW(adj_seed_coef(Nw, b.Wfin, c->ws.ecap, b.eloc, b.emix, b.omega, b.ecoef, p->e0, dE, p->dJ, s), "adjoint: seed");
  CKW(launch_energy_backward<R>(c, Nw, b.Wfin, b.eloc, p->e0, p->tau, p->dJ, grad_h1, grad_L, b.ys, s),
      "adjoint: energy");
  GemmArgs gfb = site_args<R>(c, SITE_FORCEBIAS, Nw, st, c->ws.theta, c->ws.t);
  CKW(gemm<R>(gfb, false, EPI_STORE, s), "adjoint: force bias");
  CKW(adj_eloc_seed<R>(c, Nw, static_cast<const P*>(c->ws.theta), static_cast<const P*>(c->ws.t), b.ecoef, b.thbar,
                       s),
      "adjoint: energy seed");
  CKW(adj_sanitize<R>(b.run_psi, b.P0, b.Wfin, c->d_trial, per, Nw, s), "adjoint: sanitise");
  CKW(adj_lu<R>(c, Nw, b.P0, b.oinvk, b.ldk, s), "adjoint: overlap inverse");
  CKW(cudaMemsetAsync(b.pb, 0, nw * per * cs, s), "adjoint: memset");
  CKW(adj_theta<R>(c, Nw, b.thbar, static_cast<const P*>(c->ws.theta), b.oinvk, nullptr, b.Wfin, b.pb, s),
      "adjoint: Theta pull-back");
  c->launches += 1 + 5 + (gfb.splitk > 1 ? 2 : 1) + 1 + 1 + 1 + 1;
  // the parameter-adjoint sums are FP64 complex (double2) for both walker types
  CKW(cudaMemsetAsync(b.gLc, 0, (size_t)G * NN * sizeof(double2), s), "adjoint: memset");
  CKW(cudaMemsetAsync(b.Lhb, 0, (size_t)G * per * sizeof(double2), s), "adjoint: memset");
  CKW(cudaMemsetAsync(b.Bbar, 0, NN * sizeof(double2), s), "adjoint: memset");
  CKW(cudaMemsetAsync(b.mubar, 0, (size_t)G * sizeof(double), s), "adjoint: memset");

  // segments in reverse: recompute the states of the segment, then step back
  for (int sg = nck - 1; sg >= 0; --sg) {
    const int k0 = sg * C, k1 = (k0 + C < n) ? k0 + C : n;
    const size_t sl = (size_t)sg;
    CKW(copy_state(run.psi, run.weight, run.logovl, run.status, b.ck_psi + sl * nw * per, b.ck_W + sl * nw,
                   b.ck_lo + sl * nw * 2, b.ck_st + sl * nw),
        "adjoint: restore");
    for (int k = k0; k < k1; ++k) {
      const size_t i = (size_t)(k - k0);
      CKW(cudaMemcpyAsync(b.seg_psi + i * nw * per, run.psi, nw * per * cs, dd, s), "adjoint: store");
      CKW(cudaMemcpyAsync(b.seg_lo + i * nw * 2, run.logovl, nw * 2 * sizeof(double), dd, s), "adjoint: store");
      sp.reortho = qr_at(k);
      rc = run_step<R>(c, &run, fields + (size_t)k * fstride, &sp, nullptr, nullptr);
      if (rc != AFQMC_OK) return rc;
    }
    CKW(cudaMemcpyAsync(b.seg_psi + (size_t)(k1 - k0) * nw * per, run.psi, nw * per * cs, dd, s), "adjoint: store");
    for (int k = k1 - 1; k >= k0; --k) {
      const size_t i = (size_t)(k - k0);
      rc = adj_step<R>(c, b, Nw, fields + (size_t)k * fstride, b.seg_psi + i * nw * per, b.seg_lo + i * nw * 2,
                    b.seg_psi + (i + 1) * nw * per, qr_at(k), K, kry, lz, p->tau);
      if (rc != AFQMC_OK) return rc;
    }
  }
  if (grad_psi0) CKW(cudaMemcpyAsync(grad_psi0, b.pb, nw * per * cs, dd, s), "adjoint: copy");

  // e^{-tau h''/2} through the eigendecomposition, then the final gradients
  CKW(cudaMemcpyAsync(b.V, c->h_evecs, NN * sizeof(double), cudaMemcpyHostToDevice, s), "adjoint: upload");
  CKW(cudaMemcpyAsync(b.lam, c->h_evals, (size_t)N * sizeof(double), cudaMemcpyHostToDevice, s), "adjoint: upload");
  int nfin = 0;
  CKW(adj_finish(c, b.Bbar, b.V, b.lam, p->tau, b.Bs, b.T1, b.M1, b.hbar, b.X, b.D, b.gLc, b.Lhb, b.mubar, grad_h1,
                 grad_L, &nfin, s),
      "adjoint: final");
  c->launches += nfin;
  return AFQMC_OK;
}

// Allocate the adjoint's workspace (one block, carved twice: once to size it),
// run the walk backward and free the block.
template <typename R>
static afqmc_status walk_backward_alloc(afqmc_ctx* c, const afqmc_walkers* w0, const double* fields,
                                        const afqmc_walk_adjoint_params* q, int nck, double* J_out, double* grad_h1,
                                        double* grad_L, void* grad_psi0) {
  AllocScope alloc_scope(AG_ADJOINT);
  const int Nw = w0->n_walkers;
  const size_t NN = (size_t)c->N * c->N;
  AdjBufs<R> b{};
  b.skc = pick_splitk(c->G, Nw, (long long)NN, 32);
  b.skb = pick_splitk(c->N, c->N, (long long)Nw * c->nc, 64);
  Arena a;
  adj_carve<R>(a, b, c, Nw, q->order, q->ckpt_every, nck, q->expm != AFQMC_EXPM_TAYLOR);
  CK(cudaStreamSynchronize(c->stream));
  char* base = nullptr;
  cudaError_t e = dmalloc(&base, a.used);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return cuda_fail(e, "adjoint workspace");
  }
  a = Arena{base, 0};
  adj_carve<R>(a, b, c, Nw, q->order, q->ckpt_every, nck, q->expm != AFQMC_EXPM_TAYLOR);
  afqmc_status st = walk_backward_run<R>(c, w0, fields, q, J_out, grad_h1, grad_L, grad_psi0, b);
  e = cudaStreamSynchronize(c->stream);
  cudaFree(base);
  if (st != AFQMC_OK) return st;
  if (e != cudaSuccess) return cuda_fail(e, "adjoint");
  return AFQMC_OK;
}

// ---------------------------------------------------------------- ABI
extern "C" {

const char* afqmc_strerror(afqmc_status s) {
  switch (s) {
    case AFQMC_OK: return "ok";
    case AFQMC_EINVAL: return "invalid argument";
    case AFQMC_EDOM: return "non-finite input";
    case AFQMC_ENOMEM: return "out of memory";
    case AFQMC_ECUDA: return "CUDA error";
    case AFQMC_ENOTSUP: return "not supported";
    case AFQMC_ESTATE: return "call out of order";
  }
  return "unknown status";
}

const char* afqmc_last_cuda_error(void) { return g_cuda_err; }

afqmc_status afqmc_create(afqmc_ctx** out, int N, int n_alpha, int n_beta, int n_chol, const double* h1,
                          const double* L, const double* trial, double e_const, int precision, void* stream) {
  if (!out || !h1 || !L || !trial) return AFQMC_EINVAL;
  *out = nullptr;
  if (N < 1 || N > 512 || n_alpha < 0 || n_beta < 0 || n_alpha > 80 || n_beta > 80 || n_alpha + n_beta < 1 ||
      n_alpha > N || n_beta > N || n_chol < 1)
    return AFQMC_EINVAL;
  if (precision != AFQMC_FP64 && precision != AFQMC_MIXED) return AFQMC_EINVAL;
  const size_t NN = (size_t)N * N, nc = (size_t)(n_alpha + n_beta);
  if (!std::isfinite(e_const) || !all_finite(h1, NN) || !all_finite(L, (size_t)n_chol * NN) ||
      !all_finite(trial, nc * N))
    return AFQMC_EDOM;
  afqmc_ctx* c = new (std::nothrow) afqmc_ctx();
  if (!c) return AFQMC_ENOMEM;
  c->N = N; c->na = n_alpha; c->nb = n_beta; c->nc = (int)nc; c->G = n_chol; c->prec = precision;
  c->e_const = e_const;
  c->stream = static_cast<cudaStream_t>(stream);
  if (cudaGetDevice(&c->device) != cudaSuccess) {
    delete c;
    return AFQMC_ECUDA;
  }
  afqmc_status st = ctx_setup(c, h1, L, trial);
  if (st != AFQMC_OK) {
    ctx_free(c);
    return st;
  }
  *out = c;
  return AFQMC_OK;
}

afqmc_status afqmc_set_tau(afqmc_ctx* c, double tau) {
  if (!c) return AFQMC_EINVAL;
  if (!std::isfinite(tau)) return AFQMC_EDOM;
  if (!(tau > 0.0)) return AFQMC_EINVAL;
  const int N = c->N;
  std::vector<double> Bh((size_t)N * N, 0.0), ex(N);
  for (int k = 0; k < N; ++k) ex[k] = std::exp(-0.5 * tau * c->h_evals[k]);
  for (int p = 0; p < N; ++p)
    for (int q = 0; q < N; ++q) {
      double v = 0.0;
      for (int k = 0; k < N; ++k) v += c->h_evecs[(size_t)p * N + k] * ex[k] * c->h_evecs[(size_t)q * N + k];
      Bh[(size_t)p * N + q] = v;
    }
  CK(cudaStreamSynchronize(c->stream));
  CK(cudaMemcpy(c->d_B, Bh.data(), Bh.size() * sizeof(double), cudaMemcpyHostToDevice));
  if (c->prec == AFQMC_MIXED) {
    CK(launch_to_float(c->d_B, c->f_B, Bh.size(), c->stream));
    c->launches += 1;
    if (c->tg.hs_ok) {  // D = B - I planes of the tensor-core half step
      CK(tc_halfstep_set_b(c, c->stream));
      c->launches += 1;
    }
    CK(cudaStreamSynchronize(c->stream));
  }
  c->tau = tau;
  return AFQMC_OK;
}

afqmc_status afqmc_set_stream(afqmc_ctx* c, void* stream) {
  if (!c) return AFQMC_EINVAL;
  c->stream = static_cast<cudaStream_t>(stream);
  return AFQMC_OK;
}

static afqmc_status check_walkers(const afqmc_ctx* c, const afqmc_walkers* w) {
  if (!c || !w || w->n_walkers < 0 || w->n_walkers > (1 << 24)) return AFQMC_EINVAL;
  if (w->n_walkers > 0 && (!w->psi || !w->weight || !w->logovl || !w->status)) return AFQMC_EINVAL;
  const size_t align = c->prec == AFQMC_FP64 ? 16 : 8;
  if (((uintptr_t)w->psi) % align || ((uintptr_t)w->weight) % 8 || ((uintptr_t)w->logovl) % 8 ||
      ((uintptr_t)w->status) % 4)
    return AFQMC_EINVAL;
  return AFQMC_OK;
}

afqmc_status afqmc_walkers_init(afqmc_ctx* c, const afqmc_walkers* w) {
  afqmc_status st = check_walkers(c, w);
  if (st != AFQMC_OK) return st;
  if (w->n_walkers == 0) return AFQMC_OK;
  st = ws_ensure(c, w->n_walkers, c->ws.kmax);
  if (st != AFQMC_OK) return st;
  CK(cudaMemsetAsync(c->d_bias_key, 0, 2 * sizeof(unsigned long long), c->stream));  // walkers replaced
  if (c->prec == AFQMC_FP64) {
    CK(launch_init_walkers<double>(c, w, c->stream));
    CK(launch_overlap<double>(c, w->n_walkers, w->psi, nullptr, c->ws.logdet, w->status, c->stream));
  } else {
    CK(launch_init_walkers<float>(c, w, c->stream));
    CK(launch_overlap<float>(c, w->n_walkers, w->psi, nullptr, c->ws.logdet, w->status, c->stream));
  }
  CK(launch_logovl_from_logdet(c, w, nullptr, c->stream));
  c->launches += 3;
  return AFQMC_OK;
}

afqmc_status afqmc_step(afqmc_ctx* c, const afqmc_walkers* w, const double* fields, const afqmc_step_params* p,
                        double* e_loc, double* e_mix) {
  afqmc_status st = check_walkers(c, w);
  if (st != AFQMC_OK) return st;
  if (!p || (!fields && w->n_walkers > 0)) return AFQMC_EINVAL;
  if (!std::isfinite(p->tau) || !std::isfinite(p->e0)) return AFQMC_EDOM;
  if (!(p->tau > 0.0)) return AFQMC_EINVAL;
  if (p->propagator != AFQMC_SPLIT2 && p->propagator != AFQMC_SPLIT1 && p->propagator != AFQMC_TAYLORPROP &&
      p->propagator != AFQMC_CN)
    return AFQMC_ENOTSUP;
  if (p->propagator == AFQMC_TAYLORPROP && p->expm != AFQMC_EXPM_TAYLOR) return AFQMC_ENOTSUP;
  if (p->expm == AFQMC_EXPM_TAYLOR || p->expm == AFQMC_EXPM_CHEBYSHEV) {
    if (p->order < 0 || p->order > 64) return AFQMC_ENOTSUP;
  } else if (p->expm == AFQMC_EXPM_KRYLOV || p->expm == AFQMC_EXPM_LANCZOS) {
    if (p->order < 1 || p->order > 32) return AFQMC_ENOTSUP;
  } else if (p->expm == AFQMC_EXPM_BLOCK_KRYLOV) {
    if (p->order < 1 || p->order > 16 || !bk_fits(c, p->order)) return AFQMC_ENOTSUP;
  } else {
    return AFQMC_ENOTSUP;
  }
  if (w->n_walkers == 0) return AFQMC_OK;
  if (p->tau != c->tau) {
    st = afqmc_set_tau(c, p->tau);
    if (st != AFQMC_OK) return st;
  }
  const bool kry = p->expm == AFQMC_EXPM_KRYLOV || p->expm == AFQMC_EXPM_LANCZOS ||
                   p->expm == AFQMC_EXPM_BLOCK_KRYLOV;
  const int k = kry ? (p->order < c->N ? p->order : c->N) : 0;
  st = ws_ensure(c, w->n_walkers, k);
  if (st != AFQMC_OK) return st;
  if (p->expm == AFQMC_EXPM_BLOCK_KRYLOV) CK(bk_ensure(c, w->n_walkers, bk_blocks(c, p->order)));
  afqmc_step_params q = *p;
  q.order = kry ? k : p->order;
  if (c->prec == AFQMC_FP64) return run_step<double>(c, w, fields, &q, e_loc, e_mix);
  return run_step<float>(c, w, fields, &q, e_loc, e_mix);
}

afqmc_status afqmc_local_energy(afqmc_ctx* c, const afqmc_walkers* w, double e0, double tau, double* e_loc,
                                double* e_mix) {
  afqmc_status st = check_walkers(c, w);
  if (st != AFQMC_OK) return st;
  if (!std::isfinite(tau) || !std::isfinite(e0)) return AFQMC_EDOM;
  if (!(tau > 0.0)) return AFQMC_EINVAL;
  if (w->n_walkers == 0) return AFQMC_OK;
  st = ws_ensure(c, w->n_walkers, c->ws.kmax);
  if (st != AFQMC_OK) return st;
  if (c->prec == AFQMC_FP64) return run_energy<double>(c, w, e0, tau, e_loc, e_mix);
  return run_energy<float>(c, w, e0, tau, e_loc, e_mix);
}

afqmc_status afqmc_population_control(afqmc_ctx* c, const afqmc_walkers* w, double u, int32_t* index_out) {
  afqmc_status st = check_walkers(c, w);
  if (st != AFQMC_OK) return st;
  if (!std::isfinite(u)) return AFQMC_EDOM;
  if (!(u >= 0.0 && u < 1.0)) return AFQMC_EINVAL;
  if (index_out && ((uintptr_t)index_out) % 4) return AFQMC_EINVAL;
  if (w->n_walkers == 0) return AFQMC_OK;
  st = ws_ensure(c, w->n_walkers, c->ws.kmax);
  if (st != AFQMC_OK) return st;
  CK(cudaMemsetAsync(c->d_bias_key, 0, 2 * sizeof(unsigned long long), c->stream));  // walkers replaced
  prof_mark(c, AFQMC_K_OTHER, true, c->stream);
  if (c->prec == AFQMC_FP64)
    CK(launch_comb<double>(c, w, u, index_out, c->stream));
  else
    CK(launch_comb<float>(c, w, u, index_out, c->stream));
  prof_mark(c, AFQMC_K_OTHER, false, c->stream);
  c->launches += 4;
  return AFQMC_OK;
}

afqmc_status afqmc_energy_backward(afqmc_ctx* c, const afqmc_walkers* w, double e0, double tau, double dJ,
                                   double* grad_h1, double* grad_L) {
  afqmc_status st = check_walkers(c, w);
  if (st != AFQMC_OK) return st;
  if (!grad_h1 || !grad_L || ((uintptr_t)grad_h1) % 8 || ((uintptr_t)grad_L) % 8) return AFQMC_EINVAL;
  if (!std::isfinite(tau) || !std::isfinite(e0) || !std::isfinite(dJ)) return AFQMC_EDOM;
  if (!(tau > 0.0)) return AFQMC_EINVAL;
  const int nmax = c->na > c->nb ? c->na : c->nb;
  if ((size_t)(nmax * nmax + nmax * c->N) * 16 > (size_t)max_dyn_smem() - 1024) return AFQMC_ENOTSUP;
  const size_t NN = (size_t)c->N * c->N;
  if (w->n_walkers == 0) {
    CK(cudaMemsetAsync(grad_h1, 0, NN * sizeof(double), c->stream));
    CK(cudaMemsetAsync(grad_L, 0, (size_t)c->G * NN * sizeof(double), c->stream));
    return AFQMC_OK;
  }
  st = ws_ensure(c, w->n_walkers, c->ws.kmax);
  if (st != AFQMC_OK) return st;
  // Theta and E_L at the walkers (window mask), then the adjoint contractions
  const bool fp64 = c->prec == AFQMC_FP64;
  st = fp64 ? run_energy<double>(c, w, e0, tau, c->ws.eloc, c->ws.emix)
            : run_energy<float>(c, w, e0, tau, c->ws.eloc, c->ws.emix);
  if (st != AFQMC_OK) return st;
  double2* ys = nullptr;
  CK(dmalloc(&ys, ((size_t)c->nc * c->N + (size_t)c->G * c->nc * c->N) * sizeof(double2)));
  cudaError_t e = fp64 ? launch_energy_backward<double>(c, w->n_walkers, w->weight, c->ws.eloc, e0, tau, dJ, grad_h1,
                                                        grad_L, ys, c->stream)
                       : launch_energy_backward<float>(c, w->n_walkers, w->weight, c->ws.eloc, e0, tau, dJ, grad_h1,
                                                       grad_L, ys, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  cudaFree(ys);
  if (e != cudaSuccess) return cuda_fail(e, "energy backward");
  c->launches += 5;
  return AFQMC_OK;
}

afqmc_status afqmc_walk_backward(afqmc_ctx* c, const afqmc_walkers* w0, const double* fields,
                                 const afqmc_walk_adjoint_params* p, double* J_out, double* grad_h1, double* grad_L,
                                 void* grad_psi0) {
  afqmc_status st = check_walkers(c, w0);
  if (st != AFQMC_OK) return st;
  if (!p || !grad_h1 || !grad_L || ((uintptr_t)grad_h1) % 8 || ((uintptr_t)grad_L) % 8) return AFQMC_EINVAL;
  if ((J_out && ((uintptr_t)J_out) % 8) || (grad_psi0 && ((uintptr_t)grad_psi0) % 16)) return AFQMC_EINVAL;
  if (!std::isfinite(p->tau) || !std::isfinite(p->e0) || !std::isfinite(p->dJ)) return AFQMC_EDOM;
  if (!(p->tau > 0.0) || p->n_steps < 1 || p->ckpt_every < 1 || p->reortho_every < 0) return AFQMC_EINVAL;
  if (p->order < 1 || p->order > 32) return AFQMC_ENOTSUP;
  if (p->expm != AFQMC_EXPM_TAYLOR && p->expm != AFQMC_EXPM_KRYLOV && p->expm != AFQMC_EXPM_LANCZOS)
    return AFQMC_ENOTSUP;
  const int nmax = c->na > c->nb ? c->na : c->nb;
  if (nmax > 64 || w0->n_walkers > 65535) return AFQMC_ENOTSUP;
  if ((size_t)(nmax * nmax + nmax * c->N) * 16 > (size_t)max_dyn_smem() - 1024) return AFQMC_ENOTSUP;
  const int Nw = w0->n_walkers;
  if (Nw > 0 && !fields) return AFQMC_EINVAL;
  const size_t NN = (size_t)c->N * c->N;
  if (Nw == 0) {
    CK(cudaMemsetAsync(grad_h1, 0, NN * sizeof(double), c->stream));
    CK(cudaMemsetAsync(grad_L, 0, (size_t)c->G * NN * sizeof(double), c->stream));
    if (J_out) CK(cudaMemsetAsync(J_out, 0, 4 * sizeof(double), c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return AFQMC_OK;
  }
  if (p->tau != c->tau) {
    st = afqmc_set_tau(c, p->tau);
    if (st != AFQMC_OK) return st;
  }
  const int kry =
      (p->expm == AFQMC_EXPM_KRYLOV || p->expm == AFQMC_EXPM_LANCZOS) ? (p->order < c->N ? p->order : c->N) : 0;
  st = ws_ensure(c, Nw, kry > c->ws.kmax ? kry : c->ws.kmax);
  if (st != AFQMC_OK) return st;
  const int C = p->ckpt_every < p->n_steps ? p->ckpt_every : p->n_steps;
  const int nck = (p->n_steps + C - 1) / C;
  afqmc_walk_adjoint_params q = *p;
  q.ckpt_every = C;
  return c->prec == AFQMC_FP64 ? walk_backward_alloc<double>(c, w0, fields, &q, nck, J_out, grad_h1, grad_L, grad_psi0)
                               : walk_backward_alloc<float>(c, w0, fields, &q, nck, J_out, grad_h1, grad_L, grad_psi0);
}

afqmc_status afqmc_sync(afqmc_ctx* c) {
  if (!c) return AFQMC_EINVAL;
  CK(cudaStreamSynchronize(c->stream));
  CK(cudaGetLastError());
  // a bounded wait of a tensor-core kernel gave up
  const struct { void* flag; const char* what; } tc_flags[] = {{c->tc.err, "tensor-core exchange"},
                                                                {c->tg.err, "tensor-core field assembly"}};
  for (const auto& f : tc_flags) {
    if (!f.flag) continue;
    int flag = 0;
    CK(cudaMemcpy(&flag, f.flag, sizeof(int), cudaMemcpyDeviceToHost));
    if (flag) {
      // reported once: the flag is cleared, so the context stays usable
      CK(cudaMemsetAsync(f.flag, 0, sizeof(int), c->stream));
      CK(cudaStreamSynchronize(c->stream));
      snprintf(g_cuda_err, sizeof g_cuda_err, "%s: pipeline wait timed out (code %d)", f.what, flag);
      return AFQMC_ECUDA;
    }
  }
  return AFQMC_OK;
}

uint64_t afqmc_launch_count(const afqmc_ctx* c) { return c ? c->launches : 0; }

afqmc_status afqmc_profile(afqmc_ctx* c, int enable) {
  return afqmc_profile_mask(c, enable ? (1u << AFQMC_K_COUNT) - 1u : 0u);
}

afqmc_status afqmc_profile_mask(afqmc_ctx* c, uint32_t mask) {
  if (!c) return AFQMC_EINVAL;
  if (mask >> AFQMC_K_COUNT) return AFQMC_EINVAL;
  Prof& p = c->prof;
  if (mask) {
    if (!p.pool) {
      const int cap = 32768;
      p.pool = (cudaEvent_t*)calloc((size_t)2 * cap, sizeof(cudaEvent_t));
      p.cls = (int*)calloc(cap, sizeof(int));
      if (!p.pool || !p.cls) { prof_release(p); return AFQMC_ENOMEM; }
      for (int i = 0; i < 2 * cap; ++i) {
        cudaError_t e = cudaEventCreate(&p.pool[i]);
        if (e != cudaSuccess) {
          p.cap = i / 2;
          prof_release(p);
          return cuda_fail(e);
        }
        p.cap = (i + 1) / 2;
      }
    }
    CK(cudaStreamSynchronize(c->stream));
    p.used = 0;
    p.open_cls = -1;
    for (int k = 0; k < AFQMC_K_COUNT; ++k) { p.ms[k] = 0.0; p.n[k] = 0; }
    p.mask = mask;
    p.on = true;
  } else {
    p.on = false;
  }
  return AFQMC_OK;
}

afqmc_status afqmc_profile_read(afqmc_ctx* c, double* ms, uint64_t* n) {
  if (!c || !ms || !n) return AFQMC_EINVAL;
  Prof& p = c->prof;
  CK(cudaStreamSynchronize(c->stream));
  for (int i = 0; i < p.used; ++i) {
    float t = 0.f;
    CK(cudaEventElapsedTime(&t, p.pool[2 * i], p.pool[2 * i + 1]));
    p.ms[p.cls[i]] += t;
    p.n[p.cls[i]] += 1;
  }
  p.used = 0;
  for (int k = 0; k < AFQMC_K_COUNT; ++k) { ms[k] = p.ms[k]; n[k] = p.n[k]; }
  return AFQMC_OK;
}

void afqmc_destroy(afqmc_ctx* c) {
  if (!c) return;
  cudaStreamSynchronize(c->stream);
  ctx_free(c);
}

afqmc_status afqmc_autotune(afqmc_ctx* c, int n_walkers, int32_t* table_out) {
  if (!c || n_walkers < 1 || n_walkers > (1 << 24)) return AFQMC_EINVAL;
  afqmc_status st = ws_ensure(c, n_walkers, c->ws.kmax);
  if (st != AFQMC_OK) return st;
  st = c->prec == AFQMC_FP64 ? autotune_impl<double>(c, n_walkers, 1) : autotune_impl<float>(c, n_walkers, 1);
  if (st != AFQMC_OK) return st;
  if (table_out)
    for (int i = 0; i < N_SITES; ++i) table_out[i] = c->tune[i];
  return AFQMC_OK;
}

afqmc_status afqmc_tune_set(afqmc_ctx* c, const int32_t* table) {
  if (!c || !table) return AFQMC_EINVAL;
  for (int i = 0; i < N_SITES; ++i)
    if (table[i] < 0 || table[i] >= GEMM_VARIANTS) return AFQMC_EINVAL;
  for (int i = 0; i < N_SITES; ++i) c->tune[i] = table[i];
  return AFQMC_OK;
}

afqmc_status afqmc_tune_get(const afqmc_ctx* c, int32_t* table) {
  if (!c || !table) return AFQMC_EINVAL;
  for (int i = 0; i < N_SITES; ++i) table[i] = c->tune[i];
  return AFQMC_OK;
}

afqmc_status afqmc_batch_create(afqmc_batch** out, afqmc_ctx* const* ctxs, int n_sys) {
  if (!out || !ctxs || n_sys < 1 || n_sys > 4096) return AFQMC_EINVAL;
  *out = nullptr;
  for (int i = 0; i < n_sys; ++i)
    if (!ctxs[i]) return AFQMC_EINVAL;
  afqmc_batch* b = new (std::nothrow) afqmc_batch();
  if (!b) return AFQMC_ENOMEM;
  b->ctxs.assign(ctxs, ctxs + n_sys);
  cudaError_t e = cudaStreamCreateWithFlags(&b->origin, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming);
  for (int i = 0; i < n_sys && e == cudaSuccess; ++i) {
    cudaStream_t st = nullptr;
    cudaEvent_t ev = nullptr;
    e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e == cudaSuccess) b->branch.push_back(st);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e == cudaSuccess) b->join.push_back(ev);
  }
  if (e != cudaSuccess) {
    batch_free(b);
    return cuda_fail(e);
  }
  *out = b;
  return AFQMC_OK;
}

void afqmc_batch_destroy(afqmc_batch* b) {
  if (!b) return;
  if (b->origin) cudaStreamSynchronize(b->origin);
  batch_free(b);
}

static afqmc_status step_checks(afqmc_ctx* c, const afqmc_walkers* w, const double* fields,
                                const afqmc_step_params* p) {
  afqmc_status st = check_walkers(c, w);
  if (st != AFQMC_OK) return st;
  if (!p || (!fields && w->n_walkers > 0)) return AFQMC_EINVAL;
  if (!std::isfinite(p->tau) || !std::isfinite(p->e0)) return AFQMC_EDOM;
  if (!(p->tau > 0.0)) return AFQMC_EINVAL;
  if (p->propagator != AFQMC_SPLIT2 && p->propagator != AFQMC_SPLIT1 && p->propagator != AFQMC_TAYLORPROP &&
      p->propagator != AFQMC_CN)
    return AFQMC_ENOTSUP;
  if (p->propagator == AFQMC_TAYLORPROP && p->expm != AFQMC_EXPM_TAYLOR) return AFQMC_ENOTSUP;
  if (p->expm == AFQMC_EXPM_TAYLOR || p->expm == AFQMC_EXPM_CHEBYSHEV) {
    if (p->order < 0 || p->order > 64) return AFQMC_ENOTSUP;
  } else if (p->expm == AFQMC_EXPM_KRYLOV || p->expm == AFQMC_EXPM_LANCZOS) {
    if (p->order < 1 || p->order > 32) return AFQMC_ENOTSUP;
  } else if (p->expm == AFQMC_EXPM_BLOCK_KRYLOV) {
    if (p->order < 1 || p->order > 16 || !bk_fits(c, p->order)) return AFQMC_ENOTSUP;
  } else {
    return AFQMC_ENOTSUP;
  }
  return AFQMC_OK;
}

afqmc_status afqmc_batch_step(afqmc_batch* b, const afqmc_walkers* ws, const double* const* fields,
                              const afqmc_step_params* p, double* const* e_loc, double* const* e_mix,
                              void* stream) {
  if (!b || !ws || !fields || !p) return AFQMC_EINVAL;
  const int n = (int)b->ctxs.size();
  std::vector<afqmc_step_params> q(p, p + n);
  std::vector<unsigned char> key;
  auto put = [&key](const void* src, size_t bytes) {
    const unsigned char* c8 = static_cast<const unsigned char*>(src);
    key.insert(key.end(), c8, c8 + bytes);
  };
  for (int i = 0; i < n; ++i) {
    afqmc_ctx* c = b->ctxs[i];
    afqmc_status st = step_checks(c, &ws[i], fields[i], &p[i]);
    if (st != AFQMC_OK) return st;
    if (p[i].expm == AFQMC_EXPM_KRYLOV || p[i].expm == AFQMC_EXPM_LANCZOS || p[i].expm == AFQMC_EXPM_BLOCK_KRYLOV)
      q[i].order = p[i].order < c->N ? p[i].order : c->N;
    double* el = e_loc ? e_loc[i] : nullptr;
    double* em = e_mix ? e_mix[i] : nullptr;
    put(&ws[i], sizeof(afqmc_walkers));
    put(&fields[i], sizeof(void*));
    put(&q[i], sizeof(afqmc_step_params));
    put(&el, sizeof(void*));
    put(&em, sizeof(void*));
  }
  cudaStream_t user = static_cast<cudaStream_t>(stream);
  BatchGraph* hit = nullptr;
  for (auto& g : b->graphs)
    if (g.used && g.key == key) hit = &g;
  if (!hit) {
    // prepare outside the capture: time step, workspace, kernel attributes
    for (int i = 0; i < n; ++i) {
      afqmc_ctx* c = b->ctxs[i];
      if (ws[i].n_walkers == 0) continue;
      if (p[i].tau != c->tau) {
        afqmc_status st = afqmc_set_tau(c, p[i].tau);
        if (st != AFQMC_OK) return st;
      }
      const bool kry = q[i].expm == AFQMC_EXPM_KRYLOV || q[i].expm == AFQMC_EXPM_LANCZOS ||
                       q[i].expm == AFQMC_EXPM_BLOCK_KRYLOV;
      afqmc_status st = ws_ensure(c, ws[i].n_walkers, kry ? q[i].order : 0);
      if (st != AFQMC_OK) return st;
      if (q[i].expm == AFQMC_EXPM_BLOCK_KRYLOV)
        CKW(bk_ensure(c, ws[i].n_walkers, bk_blocks(c, q[i].order)), "block-Krylov workspace");
      CKW(prepare_kernels(c), "prepare_kernels");
      CKW(cudaStreamSynchronize(c->stream), "prepare sync");
    }
    // capture: one branch per system between a fork and a join
    std::vector<cudaStream_t> saved(n);
    std::vector<bool> saved_prof(n);
    std::vector<uint64_t> launches(n, 0);
    CKW(cudaStreamBeginCapture(b->origin, cudaStreamCaptureModeThreadLocal), "cudaStreamBeginCapture");
    afqmc_status rc = AFQMC_OK;
    cudaError_t e = cudaEventRecord(b->fork, b->origin);
    for (int i = 0; i < n && e == cudaSuccess && rc == AFQMC_OK; ++i) {
      afqmc_ctx* c = b->ctxs[i];
      saved[i] = c->stream;
      saved_prof[i] = c->prof.on;
      e = cudaStreamWaitEvent(b->branch[i], b->fork, 0);
      if (e != cudaSuccess) break;
      c->stream = b->branch[i];
      c->prof.on = false;
      c->capturing = true;
      const uint64_t l0 = c->launches;
      if (ws[i].n_walkers > 0)
        rc = c->prec == AFQMC_FP64
                 ? run_step<double>(c, &ws[i], fields[i], &q[i], e_loc ? e_loc[i] : nullptr, e_mix ? e_mix[i] : nullptr)
                 : run_step<float>(c, &ws[i], fields[i], &q[i], e_loc ? e_loc[i] : nullptr, e_mix ? e_mix[i] : nullptr);
      launches[i] = c->launches - l0;
      c->launches = l0;
      c->stream = saved[i];
      c->prof.on = saved_prof[i];
      c->capturing = false;
      if (e == cudaSuccess) e = cudaEventRecord(b->join[i], b->branch[i]);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(b->origin, b->join[i], 0);
    }
    cudaGraph_t graph = nullptr;
    const cudaError_t ee = cudaStreamEndCapture(b->origin, &graph);
    if (rc != AFQMC_OK) {
      if (graph) cudaGraphDestroy(graph);
      return rc;
    }
    if (e != cudaSuccess || ee != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      return cuda_fail(e != cudaSuccess ? e : ee, e != cudaSuccess ? "capture fork/join" : "cudaStreamEndCapture");
    }
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
    BatchGraph* slot = &b->graphs[0];
    for (auto& g : b->graphs) {
      if (!g.used) { slot = &g; break; }
      if (g.stamp < slot->stamp) slot = &g;
    }
    if (slot->exec) cudaGraphExecDestroy(slot->exec);
    slot->used = true;
    slot->key = key;
    slot->exec = exec;
    slot->launches = launches;
    hit = slot;
  }
  hit->stamp = ++b->clock;
  CKW(cudaGraphLaunch(hit->exec, user), "cudaGraphLaunch");
  for (int i = 0; i < n; ++i) b->ctxs[i]->launches += hit->launches[i];
  return AFQMC_OK;
}

afqmc_status afqmc_host_eigh(int n, const double* a, double* evals, double* evecs) {
  if (n < 1 || !a || !evals || !evecs) return AFQMC_EINVAL;
  if (!all_finite(a, (size_t)n * n)) return AFQMC_EDOM;
  std::vector<double> m(a, a + (size_t)n * n);
  jacobi_eigh(n, m.data(), evals, evecs);
  return AFQMC_OK;
}

}  // extern "C"
