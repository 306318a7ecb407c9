// Force-bias finalisation, weights, local energy and set-up kernels.
//
//  * bias_finalize: f_g = -i sqrt(tau) (<L_g>_mixed - L_bar_g) (Eq. force_shift),
//    removed when |f_g| >= 1 (Sec. V.C); c_g = x_g - f_g; log I = sum_g x_g f_g
//    - f_g^2/2; sum_g c_g L_bar_g for the mean-field scalar factor.
//  * weights: log ratio, hybrid energy E_H = -(log ratio + log I)/tau (Eq.
//    hyben), dtheta = Im log ratio (Eq. theta), reweighting factor capped at
//    10 (Sec. V.B), W' = W fac max(0, cos dtheta) (Eq. phaseless).
//  * energy: E_L = E_const + sum_s tr(h_half Theta_s) + 1/2 sum_g [(sum_s tr T_gs)^2
//    - sum_s tr(T_gs T_gs)] with T_gs = Lh_gs Theta_s (Eq. eloc with
//    <pq|rs> = sum_g L_g,pr L_g,qs), the window of Eq. enwin and the mixed
//    estimator E_k (Sec. II.A).
// All sums are FP64 and deterministic (fixed partition and tree order).
#include <math_constants.h>

#include <type_traits>

#include "internal.cuh"

namespace afq {

namespace {

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Deterministic block sum of K doubles for a 256-thread block.
template <int K>
__device__ __forceinline__ void block_sum(double* v, double* sh) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < K; ++i) v[i] = warp_sum(v[i]);
  __syncthreads();
  if (lane == 0)
#pragma unroll
    for (int i = 0; i < K; ++i) sh[wid * K + i] = v[i];
  __syncthreads();
#pragma unroll
  for (int i = 0; i < K; ++i) {
    double r = 0.0;
    for (int j = 0; j < 8; ++j) r += sh[j * K + i];
    v[i] = r;
  }
}

// ---------------------------------------------------------------- force bias
template <typename R>
__global__ void __launch_bounds__(256) bias_finalize_kernel(const typename C2<R>::t* __restrict__ t,
                                                            const double* __restrict__ x,
                                                            const double* __restrict__ Lbar,
                                                            typename C2<R>::t* __restrict__ cout, double* scal,
                                                            uint8_t* __restrict__ keep, int G, double sqrt_tau,
                                                            const double* __restrict__ epart,
                                                            const int* __restrict__ from_traces) {
  __shared__ double sh[8 * 5];
  const int w = blockIdx.x;
  // <L_g> = sum_s tr(Lh_gs Theta_s): the traces of the last measurement of these
  // walkers (ws.epart [w][g][spin][tr re, tr im, ...]) or the force-bias GEMM
  const bool tr = from_traces && *from_traces;
  double v[5] = {0.0, 0.0, 0.0, 0.0, 0.0};  // logI re, im, cl re, im, nfcap
  for (int g = threadIdx.x; g < G; g += 256) {
    cd tg;
    if (tr) {
      const double* q = epart + ((size_t)w * G + g) * 8;
      tg = mk(q[0] + q[4], q[1] + q[5]);
    } else {
      tg = ld(t + (size_t)w * G + g);
    }
    const double lb = Lbar[g];
    // f = -i s (t - Lbar)
    cd f = mk(sqrt_tau * tg.im, -sqrt_tau * (tg.re - lb));
    const bool kept = sqrt(abs2(f)) < 1.0;
    if (!kept) {
      f = mk(0.0, 0.0);
      v[4] += 1.0;
    }
    if (keep) keep[(size_t)w * G + g] = kept ? 1 : 0;
    const double xg = x[(size_t)w * G + g];
    const cd c = mk(xg - f.re, -f.im);
    st(cout + (size_t)w * G + g, c);
    const cd ff = f * f;
    v[0] += xg * f.re - 0.5 * ff.re;
    v[1] += xg * f.im - 0.5 * ff.im;
    v[2] += c.re * lb;
    v[3] += c.im * lb;
  }
  block_sum<5>(v, sh);
  if (threadIdx.x == 0) {
    double* s = scal + (size_t)w * SC_COUNT;
    s[SC_LOGI_RE] = v[0];
    s[SC_LOGI_IM] = v[1];
    s[SC_CL_RE] = v[2];
    s[SC_CL_IM] = v[3];
    s[SC_NFCAP] = v[4];
  }
}

template <typename R>
__global__ void __launch_bounds__(256) normA_kernel(const typename C2<R>::t* __restrict__ A, double* scal,
                                                    size_t nn) {
  __shared__ double sh[8];
  const int w = blockIdx.x;
  R part = R(0);  // per-thread partial in the storage precision
  for (size_t e = threadIdx.x; e < nn; e += 256) {
    const typename C2<R>::t a = A[(size_t)w * nn + e];
    part += a.x * a.x + a.y * a.y;
  }
  double v[1] = {(double)part};
  block_sum<1>(v, sh);
  if (threadIdx.x == 0) scal[(size_t)w * SC_COUNT + SC_NORMA] = sqrt(v[0]);
}

// ---------------------------------------------------------------- weights
__global__ void weights_kernel(double* __restrict__ weight, double* __restrict__ logovl,
                               uint32_t* __restrict__ status, const double* __restrict__ logdet,
                               const double* __restrict__ scal, uint8_t* __restrict__ alive, int Nw,
                               double tau, double e0, double ecp) {
  const int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= Nw) return;
  const double W = weight[w];
  const bool live = W > 0.0;
  alive[w] = live ? 1 : 0;
  if (!live) return;
  const double* s = scal + (size_t)w * SC_COUNT;
  const double st_ = sqrt(tau);
  const cd ldn = mk(logdet[w * 4 + 0] + logdet[w * 4 + 2], logdet[w * 4 + 1] + logdet[w * 4 + 3]);
  // log s = -tau E_c' - i sqrt(tau) sum_g c_g L_bar_g
  const cd logs = mk(-tau * ecp + st_ * s[SC_CL_IM], -st_ * s[SC_CL_RE]);
  const cd lr = mk(ldn.re - logovl[2 * w] + logs.re, ldn.im - logovl[2 * w + 1] + logs.im);
  const cd eh = mk(-(lr.re + s[SC_LOGI_RE]) / tau, -(lr.im + s[SC_LOGI_IM]) / tau);
  double dth = lr.im - 2.0 * CUDART_PI * floor((lr.im + CUDART_PI) / (2.0 * CUDART_PI));
  if (dth == -CUDART_PI) dth = CUDART_PI;
  uint32_t flags = s[SC_NFCAP] > 0.0 ? AFQMC_W_FCAP : 0u;
  double fac = exp(-tau * (eh.re - e0));
  if (!(fac < 10.0)) {
    if (fac >= 10.0) flags |= AFQMC_W_REWEIGHT;
    fac = 0.0;
  }
  const double cs = cos(dth);
  if (!(cs > 0.0)) flags |= AFQMC_W_PHASE;
  double Wn = W * fac * fmax(0.0, cs);
  if (!isfinite(Wn) || !isfinite(eh.re)) {
    Wn = 0.0;
    flags |= AFQMC_W_NONFINITE;
  }
  // a singular overlap matrix at the start of this step (the bit is set by the
  // overlap kernel; a walker that had it before was killed then): its Theta
  // and force bias are meaningless, so the walker is dropped
  if (status[w] & AFQMC_W_SINGULAR) Wn = 0.0;
  weight[w] = Wn;
  logovl[2 * w] = ldn.re;
  logovl[2 * w + 1] = ldn.im;
  status[w] |= flags;
}

template <typename R>
__global__ void commit_kernel(typename C2<R>::t* __restrict__ psi, const typename C2<R>::t* __restrict__ psi_new,
                              const uint8_t* __restrict__ alive, size_t per, size_t total) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x)
    if (alive[e / per]) psi[e] = psi_new[e];
}

__global__ void logovl_kernel(double* __restrict__ logovl, const double* __restrict__ logdet,
                              const uint8_t* __restrict__ mask, int Nw) {
  const int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= Nw || (mask && !mask[w])) return;
  logovl[2 * w] = logdet[w * 4 + 0] + logdet[w * 4 + 2];
  logovl[2 * w + 1] = logdet[w * 4 + 1] + logdet[w * 4 + 3];
}

// ---------------------------------------------------------------- energy
// one-body part sum_{j,q} h_half[j][q] Theta[w][j][q]
template <typename R>
__global__ void __launch_bounds__(256) onebody_kernel(const typename C2<R>::t* __restrict__ theta,
                                                      const double* __restrict__ hhalf, double* scal,
                                                      size_t per) {
  __shared__ double sh[16];
  const int w = blockIdx.x;
  double v[2] = {0.0, 0.0};
  for (size_t e = threadIdx.x; e < per; e += 256) {
    const cd th = ld(theta + (size_t)w * per + e);
    v[0] += hhalf[e] * th.re;
    v[1] += hhalf[e] * th.im;
  }
  block_sum<2>(v, sh);
  if (threadIdx.x == 0) {
    scal[(size_t)w * SC_COUNT + SC_E1_RE] = v[0];
    scal[(size_t)w * SC_COUNT + SC_E1_IM] = v[1];
  }
}

// The same trace for complex64 walkers without an FP64 instruction per
// element (the FP64 pipe is narrow): h_half = hi + lo in FP32, each product
// hi * theta split error-free into its rounded value and the FMA residual,
// the rounded values summed per thread by TwoSum (Knuth) into a
// (sum, compensation) pair that also collects the residuals and the lo
// products; the per-thread pairs are then added in FP64.  The intrinsics keep
// the compiler from contracting the products into the sums.
__device__ __forceinline__ void acc_prod(float a, float b, float& s, float& c) {
  const float p = __fmul_rn(a, b);
  const float pe = __fmaf_rn(a, b, -p);
  const float t = __fadd_rn(s, p);
  const float z = __fsub_rn(t, s);
  const float te = __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(p, z));
  s = t;
  c = __fadd_rn(c, __fadd_rn(te, pe));
}
__global__ void __launch_bounds__(256) onebody_c64_kernel(const float2* __restrict__ theta,
                                                          const float2* __restrict__ hh2, double* scal,
                                                          size_t per) {
  __shared__ double sh[16];
  const int w = blockIdx.x;
  float sr = 0.f, cr = 0.f, si = 0.f, ci = 0.f;
  for (size_t e = threadIdx.x; e < per; e += 256) {
    const float2 th = theta[(size_t)w * per + e];
    const float2 h = hh2[e];
    acc_prod(h.x, th.x, sr, cr);
    acc_prod(h.x, th.y, si, ci);
    cr = __fmaf_rn(h.y, th.x, cr);
    ci = __fmaf_rn(h.y, th.y, ci);
  }
  double v[2] = {(double)sr + (double)cr, (double)si + (double)ci};
  block_sum<2>(v, sh);
  if (threadIdx.x == 0) {
    scal[(size_t)w * SC_COUNT + SC_E1_RE] = v[0];
    scal[(size_t)w * SC_COUNT + SC_E1_IM] = v[1];
  }
}

// Coulomb and exchange contractions per (walker, spin, g-chunk).
// T[i][j] = sum_q Lh[g][off+i][q] Theta[w][off+j][q]; each thread owns up to
// MAXE entries of T in registers; q is staged through shared memory in
// slabs of QT.  Outputs epart[w][g][spin] = (tr T, sum_ij T_ij T_ji).
constexpr int EX_NT = 256, EX_QT = 32, EX_GCHUNK = 16;
constexpr int EX_QS = EX_QT + 1;  // padded row stride: rows j of a slab fall in distinct banks
template <typename R, int MAXE>
__global__ void __launch_bounds__(EX_NT) exchange_kernel(const typename C2<R>::t* __restrict__ theta,
                                                         const R* __restrict__ Lh, double* __restrict__ epart,
                                                         int N, int na, int nb, int G) {
  extern __shared__ double smem_ex[];
  __shared__ double sh[8 * 4];
  const int w = blockIdx.x, spin = blockIdx.y;
  const int n = spin ? nb : na, off = spin ? na : 0, nc = na + nb;
  const int g0 = blockIdx.z * EX_GCHUNK;
  const int g1 = min(G, g0 + EX_GCHUNK);
  if (n == 0) {  // empty spin block: zero contributions
    for (int g = g0 + threadIdx.x; g < g1; g += EX_NT) {
      double* o = epart + (((size_t)w * G + g) * 2 + spin) * 4;
      o[0] = o[1] = o[2] = o[3] = 0.0;
    }
    return;
  }
  R* sL = reinterpret_cast<R*>(smem_ex);                 // [n][QT]
  R* sTr = sL + n * EX_QS;                               // [n][QS]
  R* sTi = sTr + n * EX_QS;                              // [n][QS]
  cd* sT = reinterpret_cast<cd*>(smem_ex + (3 * n * EX_QS * sizeof(R) + 7) / 8);  // [n][n]
  const int nn = n * n;
  const typename C2<R>::t* Th = theta + ((size_t)w * nc + off) * N;
  for (int g = g0; g < g1; ++g) {
    const R* L = Lh + ((size_t)g * nc + off) * N;
    R ar[MAXE], ai[MAXE];
#pragma unroll
    for (int e = 0; e < MAXE; ++e) { ar[e] = R(0); ai[e] = R(0); }
    for (int q0 = 0; q0 < N; q0 += EX_QT) {
      const int qt = min(EX_QT, N - q0);
      for (int l = threadIdx.x; l < n * EX_QT; l += EX_NT) {
        const int i = l / EX_QT, qq = l % EX_QT;
        R lv = R(0), tr = R(0), ti = R(0);
        if (qq < qt) {
          lv = L[(size_t)i * N + q0 + qq];
          const typename C2<R>::t v = Th[(size_t)i * N + q0 + qq];
          tr = v.x;
          ti = v.y;
        }
        sL[i * EX_QS + qq] = lv;
        sTr[i * EX_QS + qq] = tr;
        sTi[i * EX_QS + qq] = ti;
      }
      __syncthreads();
#pragma unroll
      for (int e = 0; e < MAXE; ++e) {
        const int idx = threadIdx.x + e * EX_NT;
        if (idx < nn) {
          const int i = idx / n, j = idx % n;
          const R* a = sL + i * EX_QS;
          const R* br = sTr + j * EX_QS;
          const R* bi = sTi + j * EX_QS;
          R sr = ar[e], si = ai[e];
#pragma unroll 8
          for (int qq = 0; qq < EX_QT; ++qq) {
            sr = fma(a[qq], br[qq], sr);
            si = fma(a[qq], bi[qq], si);
          }
          ar[e] = sr;
          ai[e] = si;
        }
      }
      __syncthreads();
    }
#pragma unroll
    for (int e = 0; e < MAXE; ++e) {
      const int idx = threadIdx.x + e * EX_NT;
      if (idx < nn) sT[idx] = mk((double)ar[e], (double)ai[e]);
    }
    __syncthreads();
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    for (int idx = threadIdx.x; idx < nn; idx += EX_NT) {
      const int i = idx / n, j = idx % n;
      const cd tij = sT[idx];
      const cd p = tij * sT[j * n + i];
      v[2] += p.re;
      v[3] += p.im;
      if (i == j) { v[0] += tij.re; v[1] += tij.im; }
    }
    block_sum<4>(v, sh);
    if (threadIdx.x == 0) {
      double* o = epart + (((size_t)w * G + g) * 2 + spin) * 4;
      o[0] = v[0]; o[1] = v[1]; o[2] = v[2]; o[3] = v[3];
    }
    __syncthreads();
  }
}

// E_L per walker from the partial sums, the energy window, then (block 0 of a
// second kernel) the mixed estimator.
__global__ void __launch_bounds__(256) energy_finalize_kernel(const double* __restrict__ epart,
                                                              const double* __restrict__ scal,
                                                              double* __restrict__ e_loc,
                                                              double* __restrict__ ecap, int G, double e_const,
                                                              double e0, double dE) {
  __shared__ double sh[8 * 2];
  const int w = blockIdx.x;
  double v[2] = {0.0, 0.0};
  for (int g = threadIdx.x; g < G; g += 256) {
    const double* o = epart + ((size_t)w * G + g) * 8;
    const cd tr = mk(o[0] + o[4], o[1] + o[5]);
    const cd ex = mk(o[2] + o[6], o[3] + o[7]);
    const cd t2 = tr * tr;
    v[0] += t2.re - ex.re;
    v[1] += t2.im - ex.im;
  }
  block_sum<2>(v, sh);
  if (threadIdx.x == 0) {
    const double* s = scal + (size_t)w * SC_COUNT;
    const double er = e_const + s[SC_E1_RE] + 0.5 * v[0];
    const double ei = s[SC_E1_IM] + 0.5 * v[1];
    e_loc[2 * w] = er;
    e_loc[2 * w + 1] = ei;
    ecap[w] = fmin(fmax(er, e0 - dE), e0 + dE);
  }
}

__global__ void __launch_bounds__(256) mix_kernel(const double* __restrict__ weight, const double* __restrict__ ecap,
                                                  double* __restrict__ e_mix, int Nw) {
  __shared__ double sh[8 * 3];
  double v[3] = {0.0, 0.0, 0.0};
  for (int w = threadIdx.x; w < Nw; w += 256) {
    const double W = weight[w];
    if (W > 0.0) {
      v[0] += W * ecap[w];
      v[1] += W;
      v[2] += 1.0;
    }
  }
  block_sum<3>(v, sh);
  if (threadIdx.x == 0) {
    e_mix[0] = v[0];
    e_mix[1] = v[1];
    e_mix[2] = v[1] > 0.0 ? v[0] / v[1] : CUDART_NAN;
    e_mix[3] = v[2];
  }
}

// ---------------------------------------------------------------- set-up
// Lh[g][j][q] = sum_p trial[j][p] L[g][p][q]
__global__ void half_rotate_kernel(const double* __restrict__ L, const double* __restrict__ trial,
                                   double* __restrict__ Lh, int N, int nc, int G) {
  const size_t total = (size_t)G * nc * N;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int q = e % N;
    const int j = (e / N) % nc;
    const size_t g = e / ((size_t)N * nc);
    const double* Lg = L + g * N * N;
    double s = 0.0;
    for (int p = 0; p < N; ++p) s = fma(trial[(size_t)j * N + p], Lg[(size_t)p * N + q], s);
    Lh[e] = s;
  }
}

// LL[p][q] = sum_g sum_r L[g][p][r] L[g][r][q]
__global__ void lsq_kernel(const double* __restrict__ L, double* __restrict__ LL, int N, int G) {
  const size_t total = (size_t)N * N;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int p = e / N, q = e % N;
    double s = 0.0;
    for (int g = 0; g < G; ++g) {
      const double* Lg = L + (size_t)g * N * N;
      for (int r = 0; r < N; ++r) s = fma(Lg[(size_t)p * N + r], Lg[(size_t)r * N + q], s);
    }
    LL[e] = s;
  }
}

// L_bar_g = sum_{j,q} Lh[g][j][q] ThetaT[j][q]
__global__ void __launch_bounds__(256) lbar_kernel(const double* __restrict__ Lh, const double* __restrict__ thT,
                                                   double* __restrict__ Lbar, size_t per) {
  __shared__ double sh[8];
  const int g = blockIdx.x;
  double v[1] = {0.0};
  for (size_t e = threadIdx.x; e < per; e += 256) v[0] += Lh[(size_t)g * per + e] * thT[e];
  block_sum<1>(v, sh);
  if (threadIdx.x == 0) Lbar[g] = v[0];
}

__global__ void to_float_kernel(const double* __restrict__ a, float* __restrict__ b, size_t n) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
    b[e] = (float)a[e];
}

// A_w <- A_w - tau h'' for every walker: the exponent -tau H_eff = A - tau h''
// of the Taylor propagator (Sec. III); h'' is real and shared by the walkers,
// so only the real parts change.  Threads over the N^2 entries (x) and walker
// groups (y): tau h''_pq is formed once per entry and subtracted in the
// walkers' precision from that entry of each walker of the group.
template <typename R>
__global__ void shift_field_kernel(typename C2<R>::t* __restrict__ A, const double* __restrict__ hpp, double tau,
                                   size_t NN, int Nw) {
  const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i >= NN) return;
  const R hv = (R)(tau * hpp[i]);
  for (int w = blockIdx.y; w < Nw; w += gridDim.y) A[(size_t)w * NN + i].x -= hv;
}

// One step of the Chebyshev recurrence (Eq. chebpoly) over `total` complex
// entries.  first: acc = a t + b prod (t = T_0 Psi, prod = T_1 Psi; prod may be
// t when b = 0).  Otherwise t <- prod - t (prod = 2 A T_{n-1} Psi and
// t = T_{n-2} Psi, so t becomes T_n Psi) and acc += b t.  The arithmetic is in
// the walkers' precision (FP32 for complex64 walkers: an FP64 operation per
// element would bind the kernel to the narrow FP64 pipe instead of HBM).
template <typename R>
__global__ void cheb_step_kernel(const typename C2<R>::t* prod, typename C2<R>::t* t,
                                 typename C2<R>::t* __restrict__ acc, double a, double b, int first, size_t total) {
  const R ra = (R)a, rb = (R)b;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const auto pv = prod[e];
    const auto tv = t[e];
    auto av = acc[e];
    if (first) {
      av.x = ra * tv.x + rb * pv.x;
      av.y = ra * tv.y + rb * pv.y;
    } else {
      auto nv = tv;
      nv.x = pv.x - tv.x;
      nv.y = pv.y - tv.y;
      t[e] = nv;
      av.x = av.x + rb * nv.x;
      av.y = av.y + rb * nv.y;
    }
    acc[e] = av;
  }
}

inline int grid_for(size_t n) {
  size_t b = (n + 255) / 256;
  return (int)(b > 152 * 64 ? 152 * 64 : (b == 0 ? 1 : b));
}

}  // namespace

// ---------------------------------------------------------------- wrappers
template <typename R>
cudaError_t launch_bias_finalize(const afqmc_ctx* c, int Nw, const double* x, double sqrt_tau, cudaStream_t s,
                                 uint8_t* keep, const int* from_traces) {
  bias_finalize_kernel<R><<<Nw, 256, 0, s>>>(static_cast<const typename C2<R>::t*>(c->ws.t), x, c->d_Lbar,
                                             static_cast<typename C2<R>::t*>(c->ws.c), c->ws.scal, keep, c->G,
                                             sqrt_tau, c->ws.epart, from_traces);
  return cudaGetLastError();
}

// Force-bias source of the step: skip = opt_in and the traces in ws.epart are
// those of these walkers; the key is cleared because the step changes them.
__global__ void bias_gate_kernel(unsigned long long* key, int* skip, unsigned long long psi, int Nw, int opt_in) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    *skip = (opt_in && key[0] == psi && key[1] == (unsigned long long)Nw && psi != 0ull) ? 1 : 0;
    key[0] = 0ull;
    key[1] = 0ull;
  }
}

__global__ void bias_mark_kernel(unsigned long long* key, unsigned long long psi, int Nw) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    key[0] = psi;
    key[1] = (unsigned long long)Nw;
  }
}

cudaError_t launch_bias_gate(const afqmc_ctx* c, const void* psi, int Nw, int opt_in, cudaStream_t s) {
  bias_gate_kernel<<<1, 32, 0, s>>>(c->d_bias_key, c->d_bias_skip, (unsigned long long)(uintptr_t)psi, Nw, opt_in);
  return cudaGetLastError();
}

cudaError_t launch_bias_mark(const afqmc_ctx* c, const void* psi, int Nw, cudaStream_t s) {
  bias_mark_kernel<<<1, 32, 0, s>>>(c->d_bias_key, (unsigned long long)(uintptr_t)psi, Nw);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_normA(const afqmc_ctx* c, int Nw, cudaStream_t s) {
  normA_kernel<R><<<Nw, 256, 0, s>>>(static_cast<const typename C2<R>::t*>(c->ws.A), c->ws.scal,
                                     (size_t)c->N * c->N);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_weights(const afqmc_ctx* c, const afqmc_walkers* w, double tau, double e0, cudaStream_t s) {
  weights_kernel<<<(w->n_walkers + 127) / 128, 128, 0, s>>>(w->weight, w->logovl, w->status, c->ws.logdet,
                                                             c->ws.scal, c->ws.alive, w->n_walkers, tau, e0,
                                                             c->ec_prime);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_commit(const afqmc_ctx* c, const afqmc_walkers* w, int, cudaStream_t s) {
  const size_t per = (size_t)c->nc * c->N, total = per * w->n_walkers;
  commit_kernel<R><<<grid_for(total), 256, 0, s>>>(static_cast<typename C2<R>::t*>(w->psi),
                                                   static_cast<const typename C2<R>::t*>(c->ws.psi_new), c->ws.alive,
                                                   per, total);
  return cudaGetLastError();
}

// after re-orthonormalisation Psi = Q R: log<Psi_T|Q> = log<Psi_T|Psi> - sum_s sum_j log R_jj
// (the sums per spin in logdet[w][2 spin], written by the MGS kernel)
__global__ void logovl_shift_kernel(double* __restrict__ logovl, const double* __restrict__ logr,
                                    const uint8_t* __restrict__ mask, int Nw) {
  const int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= Nw || (mask && !mask[w])) return;
  logovl[2 * w] -= logr[w * 4 + 0] + logr[w * 4 + 2];
}

cudaError_t launch_logovl_shift(const afqmc_ctx* c, const afqmc_walkers* w, const uint8_t* mask, cudaStream_t s) {
  logovl_shift_kernel<<<(w->n_walkers + 127) / 128, 128, 0, s>>>(w->logovl, c->ws.logdet, mask, w->n_walkers);
  return cudaGetLastError();
}

cudaError_t launch_logovl_from_logdet(const afqmc_ctx* c, const afqmc_walkers* w, const uint8_t* mask,
                                      cudaStream_t s) {
  logovl_kernel<<<(w->n_walkers + 127) / 128, 128, 0, s>>>(w->logovl, c->ws.logdet, mask, w->n_walkers);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_energy(afqmc_ctx* c, int Nw, const double* weight, double e0, double tau, double* e_loc,
                          double* e_mix, cudaStream_t s, int* n_launch) {
  const size_t per = (size_t)c->nc * c->N;
  prof_mark(c, AFQMC_K_OTHER, true, s);
  if constexpr (std::is_same<R, float>::value)
    onebody_c64_kernel<<<Nw, 256, 0, s>>>(static_cast<const float2*>(c->ws.theta), c->f_hh2, c->ws.scal, per);
  else
    onebody_kernel<R><<<Nw, 256, 0, s>>>(static_cast<const typename C2<R>::t*>(c->ws.theta), c->d_hhalf,
                                         c->ws.scal, per);
  cudaError_t e = cudaGetLastError();
  prof_mark(c, AFQMC_K_OTHER, false, s);
  if (e != cudaSuccess) return e;
  const int nmax = c->na > c->nb ? c->na : c->nb;
  const int nn = nmax * nmax;
  const size_t shm = ((3 * nmax * EX_QS * sizeof(R) + 7) / 8) * 8 + (size_t)nn * sizeof(cd);
  const dim3 grid(Nw, 2, (c->G + EX_GCHUNK - 1) / EX_GCHUNK);
  const R* Lh = std::is_same<R, double>::value ? reinterpret_cast<const R*>(c->d_Lh)
                                               : reinterpret_cast<const R*>(c->f_Lh);
  const typename C2<R>::t* th = static_cast<const typename C2<R>::t*>(c->ws.theta);
#define AFQ_EX(ME)                                                                                       \
  do {                                                                                                   \
    if (!capturing(c)) {                                                                                 \
      e = raise_smem_limit(exchange_kernel<R, ME>); \
      if (e != cudaSuccess) return e;                                                                    \
    }                                                                                                    \
    prof_mark(c, AFQMC_K_EXCHANGE, true, s);                                                             \
    exchange_kernel<R, ME><<<grid, EX_NT, shm, s>>>(th, Lh, c->ws.epart, c->N, c->na, c->nb, c->G);       \
    prof_mark(c, AFQMC_K_EXCHANGE, false, s);                                                            \
  } while (0)
  if (std::is_same<R, float>::value && c->tc.ok) {
    // complex64 walkers: the contraction runs on the tensor cores (BF16x3)
    // from the split planes of Theta (timed apart: the class times the contraction)
    prof_mark(c, AFQMC_K_OTHER, true, s);
    e = tc_exchange_planes(c, Nw, c->ws.theta, s);
    prof_mark(c, AFQMC_K_OTHER, false, s);
    if (e != cudaSuccess) return e;
    prof_mark(c, AFQMC_K_EXCHANGE, true, s);
    e = tc_exchange_contract(c, Nw, c->ws.epart, s);
    prof_mark(c, AFQMC_K_EXCHANGE, false, s);
    if (e != cudaSuccess) return e;
  } else if (nn <= 4 * EX_NT)
    AFQ_EX(4);
  else if (nn <= 16 * EX_NT)
    AFQ_EX(16);
  else
    AFQ_EX(26);
#undef AFQ_EX
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int ne = c->na + c->nb;
  const double dE = 0.5 * sqrt(ne / tau) + sqrt(ne * tau);
  prof_mark(c, AFQMC_K_OTHER, true, s);
  energy_finalize_kernel<<<Nw, 256, 0, s>>>(c->ws.epart, c->ws.scal, e_loc, c->ws.ecap, c->G, c->e_const, e0, dE);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  mix_kernel<<<1, 256, 0, s>>>(weight, c->ws.ecap, e_mix, Nw);
  prof_mark(c, AFQMC_K_OTHER, false, s);
  if (n_launch) *n_launch = (std::is_same<R, float>::value && c->tc.ok) ? 5 : 4;  // + the Theta planes
  return cudaGetLastError();
}

template <typename R>
cudaError_t prepare_energy(const afqmc_ctx*) {
  cudaError_t e = raise_smem_limit(exchange_kernel<R, 4>);
  if (e == cudaSuccess)
    e = raise_smem_limit(exchange_kernel<R, 16>);
  if (e == cudaSuccess)
    e = raise_smem_limit(exchange_kernel<R, 26>);
  return e;
}
template cudaError_t prepare_energy<double>(const afqmc_ctx*);
template cudaError_t prepare_energy<float>(const afqmc_ctx*);

cudaError_t launch_setup(afqmc_ctx* c, cudaStream_t s) {
  // device temporaries: Lh (FP64), LL, ThetaT
  half_rotate_kernel<<<grid_for((size_t)c->G * c->nc * c->N), 256, 0, s>>>(c->d_L, c->d_trial, c->d_Lh, c->N,
                                                                           c->nc, c->G);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (c->prec == AFQMC_MIXED) {
    const size_t nL = (size_t)c->G * c->N * c->N, nLh = (size_t)c->G * c->nc * c->N;
    to_float_kernel<<<grid_for(nL), 256, 0, s>>>(c->d_L, c->f_L, nL);
    to_float_kernel<<<grid_for(nLh), 256, 0, s>>>(c->d_Lh, c->f_Lh, nLh);
  }
  return cudaGetLastError();
}

// exported helpers used by the host set-up in api.cu
cudaError_t launch_lsq(const double* L, double* LL, int N, int G, cudaStream_t s) {
  lsq_kernel<<<grid_for((size_t)N * N), 256, 0, s>>>(L, LL, N, G);
  return cudaGetLastError();
}
cudaError_t launch_lbar(const double* Lh, const double* thT, double* Lbar, int G, size_t per, cudaStream_t s) {
  lbar_kernel<<<G, 256, 0, s>>>(Lh, thT, Lbar, per);
  return cudaGetLastError();
}
cudaError_t launch_to_float(const double* a, float* b, size_t n, cudaStream_t s) {
  to_float_kernel<<<grid_for(n), 256, 0, s>>>(a, b, n);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_shift_field(const afqmc_ctx* c, int Nw, double tau, cudaStream_t s) {
  const size_t NN = (size_t)c->N * c->N, total = (size_t)Nw * NN;
  if (total == 0) return cudaSuccess;
  const dim3 grid((unsigned)((NN + 255) / 256), (unsigned)(Nw < 64 ? Nw : 64));
  shift_field_kernel<R><<<grid, 256, 0, s>>>(static_cast<typename C2<R>::t*>(c->ws.A), c->d_hpp, tau, NN, Nw);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_cheb_step(const afqmc_ctx* c, int Nw, const void* prod, void* t, void* acc, double a, double b,
                             int first, cudaStream_t s) {
  typedef typename C2<R>::t C;
  const size_t total = (size_t)Nw * c->nc * c->N;
  if (total == 0) return cudaSuccess;
  cheb_step_kernel<R><<<grid_for(total), 256, 0, s>>>(static_cast<const C*>(prod), static_cast<C*>(t),
                                                      static_cast<C*>(acc), a, b, first, total);
  return cudaGetLastError();
}

#define AFQ_INST(R)                                                                                         \
  template cudaError_t launch_shift_field<R>(const afqmc_ctx*, int, double, cudaStream_t);                  \
  template cudaError_t launch_cheb_step<R>(const afqmc_ctx*, int, const void*, void*, void*, double, double, \
                                           int, cudaStream_t);                                              \
  template cudaError_t launch_bias_finalize<R>(const afqmc_ctx*, int, const double*, double, cudaStream_t, uint8_t*, \
                                               const int*);                                                      \
  template cudaError_t launch_normA<R>(const afqmc_ctx*, int, cudaStream_t);                                \
  template cudaError_t launch_weights<R>(const afqmc_ctx*, const afqmc_walkers*, double, double, cudaStream_t); \
  template cudaError_t launch_commit<R>(const afqmc_ctx*, const afqmc_walkers*, int, cudaStream_t);         \
  template cudaError_t launch_energy<R>(afqmc_ctx*, int, const double*, double, double, double*,      \
                                        double*, cudaStream_t, int*);
AFQ_INST(double)
AFQ_INST(float)

}  // namespace afq
