// Reverse-mode kernels of the fixed-field walk (adjoint of the Split-2 step
// with the Taylor exponential, Sec. III.B and Eq. taylor; the paper has no
// gradients).
//
// The objective J = E_n is real; every non-holomorphic piece of the forward
// walk is a real part, an imaginary part or a threshold:
//   log W_{k+1} = log W_k + Re(log R_k + log I_k) + tau e0 + log cos Im log R_k
//   J = sum_w W_n Ebar_L / sum W,  Ebar_L = clamp(Re E_L)
// With the thresholds held fixed, dJ = Re dF for the holomorphic function
//   F = sum_{w,k} a_R,wk log R_wk + a_I,w log I_wk + sum_w e_w E_L,w
// with a_R = omega (1 + i tan dtheta), a_I = omega, omega_w = W_w (Ebar_w - J)
// / sum W and e_w = W_w / sum W inside the window.  The adjoint of every
// complex intermediate z is therefore the plain holomorphic derivative
// dF/dz (a linear map z' = M z pulls back with M^T, no conjugation), and the
// gradient with respect to a real parameter is the real part of its adjoint.
//
// Per step (walker w, spin s; Theta = Psi O^{-1}, O = trial_s^T Psi_s):
//   d log det O / d Psi       = trial O^{-T}
//   adjoint of Theta -> Psi    : Psi_bar += [Theta_bar - trial (Theta^T Theta_bar)] O^{-T}
//   t_g = sum_s tr(Lh_gs Theta_s), f_g = -i sqrt(tau)(t_g - L_bar_g) (kept
//   components), c_g = x_g - f_g, A = i sqrt(tau) sum_g c_g L_g,
//   log s = -tau E_c' - i sqrt(tau) sum_g c_g L_bar_g, log I = sum_g x_g f_g - f_g^2/2.
// Precision: the walker states and their adjoints have the walkers' complex
// type (complex128 in FP64 contexts, complex64 in mixed ones, where the long
// contractions over N run in FP32); the per-walker overlap matrices, their
// inverses and log-determinants, the scalar coefficients and every parameter
// adjoint summed over walkers or steps are FP64.
#include <math_constants.h>

#include "internal.cuh"

namespace afq {

namespace {

constexpr int AT = 256;

inline int grid_for(size_t n) {
  size_t b = (n + AT - 1) / AT;
  return (int)(b > 152 * 32 ? 152 * 32 : (b == 0 ? 1 : b));
}

// complex number of the walkers' real type R
template <typename R>
struct cx {
  R re, im;
};
template <typename R>
__device__ __forceinline__ cx<R> operator+(cx<R> a, cx<R> b) { return cx<R>{a.re + b.re, a.im + b.im}; }
template <typename R>
__device__ __forceinline__ cx<R> operator-(cx<R> a, cx<R> b) { return cx<R>{a.re - b.re, a.im - b.im}; }
template <typename R>
__device__ __forceinline__ cx<R> operator*(cx<R> a, cx<R> b) {
  return cx<R>{a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <typename R>
__device__ __forceinline__ cx<R> operator*(R s, cx<R> a) { return cx<R>{s * a.re, s * a.im}; }
__device__ __forceinline__ cx<double> ldx(const double2& v) { return cx<double>{v.x, v.y}; }
__device__ __forceinline__ cx<float> ldx(const float2& v) { return cx<float>{v.x, v.y}; }
__device__ __forceinline__ double2 stx(cx<double> v) { return make_double2(v.re, v.im); }
__device__ __forceinline__ float2 stx(cx<float> v) { return make_float2(v.re, v.im); }
template <typename R>
__device__ __forceinline__ cx<R> narrow(const double2& v) { return cx<R>{(R)v.x, (R)v.y}; }
template <typename R>
__device__ __forceinline__ cx<R> narrow(cd v) { return cx<R>{(R)v.re, (R)v.im}; }
__device__ __forceinline__ cd widen(cx<double> v) { return mk(v.re, v.im); }
__device__ __forceinline__ cd widen(cx<float> v) { return mk((double)v.re, (double)v.im); }
__device__ __forceinline__ double fmx(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float fmx(float a, float b, float c) { return fmaf(a, b, c); }

// (-i s) z
__device__ __forceinline__ cd mul_mis(double s, cd z) { return mk(s * z.im, -s * z.re); }
__device__ __forceinline__ cd ldc(const double2& v) { return mk(v.x, v.y); }

// dst = src for walkers alive at the end of the walk, the trial otherwise
// (dead walkers carry no adjoint; their stand-in state only keeps every
// intermediate finite).
template <typename R>
__global__ void adj_sanitize_kernel(const typename C2<R>::t* __restrict__ src, typename C2<R>::t* __restrict__ dst,
                                    const double* __restrict__ wfin, const double* __restrict__ trial, size_t per,
                                    size_t total) {
  for (size_t e = blockIdx.x * (size_t)AT + threadIdx.x; e < total; e += (size_t)gridDim.x * AT) {
    const size_t w = e / per;
    dst[e] = wfin[w] > 0.0 ? src[e] : stx(cx<R>{(R)trial[e - w * per], R(0)});
  }
}

// out[w] = sum_{j=0}^{K} T[w][j] in the order j = 0, 1, ..., K
template <typename R>
__global__ void adj_sum_terms_kernel(const typename C2<R>::t* __restrict__ T, typename C2<R>::t* __restrict__ out,
                                     int K1, size_t per, size_t total) {
  for (size_t e = blockIdx.x * (size_t)AT + threadIdx.x; e < total; e += (size_t)gridDim.x * AT) {
    const size_t w = e / per, r = e - w * per;
    const typename C2<R>::t* t = T + w * K1 * per + r;
    R sr = t[0].x, si = t[0].y;
    for (int j = 1; j < K1; ++j) {
      sr += t[(size_t)j * per].x;
      si += t[(size_t)j * per].y;
    }
    out[e] = stx(cx<R>{sr, si});
  }
}

// dst[w][r] = s * src[w][r] with per-walker strides
template <typename R>
__global__ void adj_scale_copy_kernel(const typename C2<R>::t* __restrict__ src, size_t sstride,
                                      typename C2<R>::t* __restrict__ dst, size_t dstride, double s, size_t per,
                                      size_t total) {
  const R sc = (R)s;
  for (size_t e = blockIdx.x * (size_t)AT + threadIdx.x; e < total; e += (size_t)gridDim.x * AT) {
    const size_t w = e / per, r = e - w * per;
    dst[w * dstride + r] = stx(sc * ldx(src[w * sstride + r]));
  }
}

// dst += src (FP64 accumulator of a complex64 contribution)
__global__ void adj_fold_kernel(const float2* __restrict__ src, double2* __restrict__ dst, size_t total) {
  for (size_t e = blockIdx.x * (size_t)AT + threadIdx.x; e < total; e += (size_t)gridDim.x * AT) {
    const float2 v = src[e];
    double2 d = dst[e];
    d.x += (double)v.x;
    d.y += (double)v.y;
    dst[e] = d;
  }
}

// O = trial_s^T psi_s for one (walker, spin) (dot products over N in the
// walkers' precision); FP64 Gauss-Jordan elimination with partial pivoting
// gives O^{-1} ([i][j], row stride n, in a slot of nmax^2) and
// log det O = sum_k log pivot_k + i pi (odd number of row swaps).
// A zero pivot gives log det = NaN and O^{-1} = 0.
template <typename R>
__global__ void __launch_bounds__(AT) adj_lu_kernel(const typename C2<R>::t* __restrict__ psi,
                                                    const R* __restrict__ trial, double2* __restrict__ oinv,
                                                    double* __restrict__ logdet, int N, int na, int nb, int nmax) {
  extern __shared__ double2 sm_lu[];
  const int w = blockIdx.x, spin = blockIdx.y;
  const int n = spin ? nb : na, off = spin ? na : 0, nc = na + nb;
  double* ldo = logdet + ((size_t)w * 2 + spin) * 2;
  if (n == 0) {
    if (threadIdx.x == 0) ldo[0] = ldo[1] = 0.0;
    return;
  }
  const int n2 = 2 * n;
  double2* M = sm_lu;       // [n][2n]  (O | I)
  double2* fac = M + n * n2;  // [n]      column k before elimination
  __shared__ int s_piv, s_sing, s_swaps;
  __shared__ double s_lr, s_li;
  __shared__ double2 s_pinv;
  const typename C2<R>::t* P = psi + (size_t)w * nc * N;
  for (int e = threadIdx.x; e < n * n; e += AT) {
    const int i = e / n, j = e - (e / n) * n;
    const R* a = trial + (size_t)(off + i) * N;
    const typename C2<R>::t* b = P + (size_t)(off + j) * N;
    R sr = R(0), si = R(0);
    for (int q = 0; q < N; ++q) {
      sr = fmx(a[q], b[q].x, sr);
      si = fmx(a[q], b[q].y, si);
    }
    M[i * n2 + j] = make_double2((double)sr, (double)si);
    M[i * n2 + n + j] = make_double2(i == j ? 1.0 : 0.0, 0.0);
  }
  if (threadIdx.x == 0) {
    s_lr = s_li = 0.0;
    s_sing = s_swaps = 0;
  }
  __syncthreads();
  for (int k = 0; k < n; ++k) {
    if (threadIdx.x == 0) {
      int piv = k;
      double best = -1.0;
      for (int i = k; i < n; ++i) {
        const double2 v = M[i * n2 + k];
        const double a = v.x * v.x + v.y * v.y;
        if (a > best) {
          best = a;
          piv = i;
        }
      }
      s_piv = piv;
      if (!(best > 0.0) || !isfinite(best)) {
        s_sing = 1;
      } else {
        if (piv != k) s_swaps ^= 1;
        const double2 u = M[piv * n2 + k];
        s_lr += 0.5 * log(best);
        s_li += atan2(u.y, u.x);
      }
    }
    __syncthreads();
    if (s_sing) break;
    const int piv = s_piv;
    if (piv != k)
      for (int q = threadIdx.x; q < n2; q += AT) {
        const double2 t = M[k * n2 + q];
        M[k * n2 + q] = M[piv * n2 + q];
        M[piv * n2 + q] = t;
      }
    __syncthreads();
    if (threadIdx.x == 0) {
      const cd r = cdiv(mk(1.0, 0.0), ldc(M[k * n2 + k]));
      s_pinv = make_double2(r.re, r.im);
    }
    for (int i = threadIdx.x; i < n; i += AT) fac[i] = M[i * n2 + k];
    __syncthreads();
    const cd pinv = ldc(s_pinv);
    for (int q = threadIdx.x; q < n2; q += AT) {
      const cd v = ldc(M[k * n2 + q]) * pinv;
      M[k * n2 + q] = make_double2(v.re, v.im);
    }
    __syncthreads();
    for (int e = threadIdx.x; e < n * n2; e += AT) {
      const int i = e / n2, q = e - (e / n2) * n2;
      if (i == k) continue;
      const cd v = ldc(M[i * n2 + q]) - ldc(fac[i]) * ldc(M[k * n2 + q]);
      M[i * n2 + q] = make_double2(v.re, v.im);
    }
    __syncthreads();
  }
  double2* out = oinv + ((size_t)w * 2 + spin) * nmax * nmax;
  const bool sing = s_sing != 0;
  for (int e = threadIdx.x; e < n * n; e += AT) {
    const int i = e / n, j = e - (e / n) * n;
    out[i * n + j] = sing ? make_double2(0.0, 0.0) : M[i * n2 + n + j];
  }
  if (threadIdx.x == 0) {
    ldo[0] = sing ? CUDART_NAN : s_lr;
    ldo[1] = sing ? CUDART_NAN : s_li + (s_swaps ? CUDART_PI : 0.0);
  }
}

// a_R = omega (1 + i tan dtheta) with dtheta = Im log R (Eq. theta): the
// imaginary part of log det O' - logovl_k + log s; zero for dead walkers.
__global__ void adj_ratio_coef_kernel(const double* __restrict__ wfin, const double* __restrict__ omega,
                                      const double* __restrict__ ld3, const double* __restrict__ logovl,
                                      const double* __restrict__ scal, double2* __restrict__ aR, double sqrt_tau,
                                      int Nw) {
  const int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= Nw) return;
  if (!(wfin[w] > 0.0)) {
    aR[w] = make_double2(0.0, 0.0);
    return;
  }
  const double dth = ld3[w * 4 + 1] + ld3[w * 4 + 3] - logovl[2 * w + 1] - sqrt_tau * scal[(size_t)w * SC_COUNT + SC_CL_RE];
  const double om = omega[w];
  aR[w] = make_double2(om, om * tan(dth));
}

// Psi3_bar for one (walker, spin):
//   no re-orthonormalisation: Psi3_bar = Psi'_bar + a_R trial O3^{-T}
//   re-orthonormalised Psi' = Psi3 R^{-1} = Psi3 O3^{-1} O':
//                             Psi3_bar = (Psi'_bar O'^T + a_R trial) O3^{-T}
// with O' = trial^T Psi'.  Dead walkers get zero.
template <typename R>
__global__ void __launch_bounds__(AT) adj_ratio_kernel(const typename C2<R>::t* __restrict__ pnext,
                                                       const typename C2<R>::t* __restrict__ psinext,
                                                       const R* __restrict__ trial,
                                                       const double2* __restrict__ oinv3,
                                                       const double2* __restrict__ aR, const double* __restrict__ wfin,
                                                       typename C2<R>::t* __restrict__ p3, int N, int na, int nb,
                                                       int nmax, int qr) {
  typedef typename C2<R>::t P;
  extern __shared__ double2 sm_ra_raw[];
  P* sm_ra = reinterpret_cast<P*>(sm_ra_raw);
  const int w = blockIdx.x, spin = blockIdx.y;
  const int n = spin ? nb : na, off = spin ? na : 0, nc = na + nb;
  if (n == 0) return;
  P* out = p3 + ((size_t)w * nc + off) * N;
  if (!(wfin[w] > 0.0)) {
    for (int e = threadIdx.x; e < n * N; e += AT) out[e] = stx(cx<R>{R(0), R(0)});
    return;
  }
  P* Oi = sm_ra;        // [n][n]  O3^{-1}
  P* On = Oi + n * n;   // [n][n]  O'
  P* Mx = On + n * n;   // [n][n]  O3^{-1} O'
  const double2* src = oinv3 + ((size_t)w * 2 + spin) * nmax * nmax;
  for (int e = threadIdx.x; e < n * n; e += AT) Oi[e] = stx(narrow<R>(src[e]));
  const P* Pn = pnext + ((size_t)w * nc + off) * N;
  if (qr) {
    const P* Sn = psinext + ((size_t)w * nc + off) * N;
    for (int e = threadIdx.x; e < n * n; e += AT) {
      const int i = e / n, l = e - (e / n) * n;
      const R* a = trial + (size_t)(off + i) * N;
      const P* b = Sn + (size_t)l * N;
      R sr = R(0), si = R(0);
      for (int q = 0; q < N; ++q) {
        sr = fmx(a[q], b[q].x, sr);
        si = fmx(a[q], b[q].y, si);
      }
      On[e] = stx(cx<R>{sr, si});
    }
    __syncthreads();
    for (int e = threadIdx.x; e < n * n; e += AT) {
      const int j = e / n, l = e - (e / n) * n;
      cx<R> s{R(0), R(0)};
      for (int i = 0; i < n; ++i) s = s + ldx(Oi[j * n + i]) * ldx(On[i * n + l]);
      Mx[e] = stx(s);
    }
  }
  __syncthreads();
  const cx<R> a = narrow<R>(aR[w]);
  for (int e = threadIdx.x; e < n * N; e += AT) {
    const int j = e / N, p = e - (e / N) * N;
    cx<R> v{R(0), R(0)};
    if (qr) {
      for (int l = 0; l < n; ++l) v = v + ldx(Pn[(size_t)l * N + p]) * ldx(Mx[j * n + l]);
    } else {
      v = ldx(Pn[(size_t)j * N + p]);
    }
    cx<R> u{R(0), R(0)};
    for (int i = 0; i < n; ++i) u = u + trial[(size_t)(off + i) * N + p] * ldx(Oi[j * n + i]);
    v = v + a * u;
    out[e] = stx(v);
  }
}

// Adjoint of the force bias and of the scalar factor for every (walker, g):
//   c_bar  += a_R (-i sqrt(tau) L_bar_g)              (log s)
//   f_bar   = -c_bar + omega c_g                       (c = x - f; log I)
//   t_bar   = kept ? -i sqrt(tau) f_bar : 0            (Eq. force_shift)
//   Lbar_bar contribution: Re[-t_bar + a_R (-i sqrt(tau) c_g + tau L_bar_g)]
template <typename R>
__global__ void adj_force_kernel(const typename C2<R>::t* __restrict__ cbar, const typename C2<R>::t* __restrict__ c,
                                 const uint8_t* __restrict__ keep, const double2* __restrict__ aR,
                                 const double* __restrict__ omega, const double* __restrict__ Lbar,
                                 typename C2<R>::t* __restrict__ tbar, double* __restrict__ mu_part, int G,
                                 double sqrt_tau, double tau, size_t total) {
  for (size_t e = blockIdx.x * (size_t)AT + threadIdx.x; e < total; e += (size_t)gridDim.x * AT) {
    const size_t w = e / G;
    const int g = (int)(e - w * G);
    const cd a = ldc(aR[w]);
    const double om = omega[w], mu = Lbar[g];
    const cd cg = widen(ldx(c[e]));
    const cd ctot = widen(ldx(cbar[e])) + a * mul_mis(sqrt_tau, mk(mu, 0.0));
    const cd fb = mk(-ctot.re + om * cg.re, -ctot.im + om * cg.im);
    const cd tb = keep[e] ? mul_mis(sqrt_tau, fb) : mk(0.0, 0.0);
    tbar[e] = stx(narrow<R>(tb));
    const cd m = a * (mul_mis(sqrt_tau, cg) + mk(tau * mu, 0.0));
    mu_part[e] = -tb.re + m.re;
  }
}

// mubar[g] += sum_w part[w][g] (walkers in order)
__global__ void adj_mu_reduce_kernel(const double* __restrict__ part, double* __restrict__ mubar, int Nw, int G) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= G) return;
  double s = 0.0;
  for (int w = 0; w < Nw; ++w) s += part[(size_t)w * G + g];
  mubar[g] += s;
}

// Psi_bar += [Theta_bar - trial (Theta^T Theta_bar + a I)] O^{-T} for one
// (walker, spin): the pull-back through Theta = Psi O^{-1} minus a times the
// derivative trial O^{-T} of log det O (a = a_R: the old overlap enters log R
// with a minus sign; a = 0 when aR is NULL).  Dead walkers are skipped.
template <typename R>
__global__ void __launch_bounds__(AT) adj_theta_kernel(const typename C2<R>::t* __restrict__ thbar,
                                                       const typename C2<R>::t* __restrict__ theta,
                                                       const R* __restrict__ trial,
                                                       const double2* __restrict__ oinv,
                                                       const double2* __restrict__ aR, const double* __restrict__ wfin,
                                                       typename C2<R>::t* __restrict__ pbar, int N, int na, int nb,
                                                       int nmax) {
  typedef typename C2<R>::t P;
  extern __shared__ double2 sm_th_raw[];
  P* sm_th = reinterpret_cast<P*>(sm_th_raw);
  const int w = blockIdx.x, spin = blockIdx.y;
  const int n = spin ? nb : na, off = spin ? na : 0, nc = na + nb;
  if (n == 0 || !(wfin[w] > 0.0)) return;
  P* Oi = sm_th;       // [n][n] O^{-1}
  P* S = Oi + n * n;   // [n][n] S[l][i] = (Theta^T Theta_bar)_li + a delta_li
  P* Q = S + n * n;    // [n][n] Q[j][l] = sum_i O^{-1}[j][i] S[l][i]
  const double2* src = oinv + ((size_t)w * 2 + spin) * nmax * nmax;
  for (int e = threadIdx.x; e < n * n; e += AT) Oi[e] = stx(narrow<R>(src[e]));
  const P* Tb = thbar + ((size_t)w * nc + off) * N;
  const P* Th = theta + ((size_t)w * nc + off) * N;
  const cx<R> a = aR ? narrow<R>(aR[w]) : cx<R>{R(0), R(0)};
  for (int e = threadIdx.x; e < n * n; e += AT) {
    const int l = e / n, i = e - (e / n) * n;
    const P* x = Th + (size_t)l * N;
    const P* y = Tb + (size_t)i * N;
    R sr = R(0), si = R(0);
    for (int p = 0; p < N; ++p) {
      sr = fmx(x[p].x, y[p].x, sr);
      sr = fmx(-x[p].y, y[p].y, sr);
      si = fmx(x[p].x, y[p].y, si);
      si = fmx(x[p].y, y[p].x, si);
    }
    if (l == i) {
      sr += a.re;
      si += a.im;
    }
    S[e] = stx(cx<R>{sr, si});
  }
  __syncthreads();
  for (int e = threadIdx.x; e < n * n; e += AT) {
    const int j = e / n, l = e - (e / n) * n;
    cx<R> s{R(0), R(0)};
    for (int i = 0; i < n; ++i) s = s + ldx(Oi[j * n + i]) * ldx(S[l * n + i]);
    Q[e] = stx(s);
  }
  __syncthreads();
  P* out = pbar + ((size_t)w * nc + off) * N;
  for (int e = threadIdx.x; e < n * N; e += AT) {
    const int j = e / N, p = e - (e / N) * N;
    cx<R> v = ldx(out[e]);
    for (int i = 0; i < n; ++i) v = v + ldx(Tb[(size_t)i * N + p]) * ldx(Oi[j * n + i]);
    for (int l = 0; l < n; ++l) v = v - trial[(size_t)(off + l) * N + p] * ldx(Q[j * n + l]);
    out[e] = stx(v);
  }
}

// omega_w = dJ W_w (Ebar_w - J) / sum W and e_w = dJ W_w / sum W strictly
// inside the energy window (Eq. enwin); both zero for dead walkers.
__global__ void adj_seed_coef_kernel(const double* __restrict__ wfin, const double* __restrict__ ecap,
                                     const double* __restrict__ e_loc, const double* __restrict__ emix,
                                     double* __restrict__ omega, double* __restrict__ ecoef, int Nw, double e0,
                                     double dE, double dJ) {
  const double tot = emix[1], J = emix[2];
  for (int w = blockIdx.x * blockDim.x + threadIdx.x; w < Nw; w += gridDim.x * blockDim.x) {
    const double W = wfin[w];
    const bool live = W > 0.0 && tot > 0.0;
    const double e = e_loc[2 * w];
    const bool inside = e > e0 - dE && e < e0 + dE;
    omega[w] = live ? dJ * W * (ecap[w] - J) / tot : 0.0;
    ecoef[w] = (live && inside) ? dJ * W / tot : 0.0;
  }
}

// Theta_bar of the local energy for one (walker, spin, row chunk):
//   dE_L/dTheta_s[p][j] = h_half[j][p] + sum_g [ t_g Lh_g[j][p] - sum_i Lh_g[i][p] T_gs[j][i] ]
// with T_gs[j][i] = sum_q Lh_g[j][q] Theta_s[i][q] and t_g the trace over
// both spins; scaled by e_w.  The term of each g is formed in the walkers'
// precision and summed over g in FP64.
constexpr int SEED_R = 16;  // outputs per thread
template <typename R>
__global__ void __launch_bounds__(AT) adj_eloc_seed_kernel(const typename C2<R>::t* __restrict__ theta,
                                                           const typename C2<R>::t* __restrict__ t,
                                                           const R* __restrict__ Lh,
                                                           const double* __restrict__ hhalf,
                                                           const double* __restrict__ ecoef,
                                                           typename C2<R>::t* __restrict__ thbar, int N, int na,
                                                           int nb, int G, int prows) {
  typedef typename C2<R>::t P;
  extern __shared__ double2 sm_es_raw[];
  P* T = reinterpret_cast<P*>(sm_es_raw);  // [n][n]
  const int w = blockIdx.x, spin = blockIdx.y;
  const int n = spin ? nb : na, off = spin ? na : 0, nc = na + nb;
  const int p0 = blockIdx.z * prows;
  const int pr = min(prows, N - p0);
  if (n == 0 || pr <= 0) return;
  P* out = thbar + ((size_t)w * nc + off) * N;
  const double ew = ecoef[w];
  if (ew == 0.0) {
    for (int e = threadIdx.x; e < n * pr; e += AT) {
      const int j = e / pr, p = p0 + e - (e / pr) * pr;
      out[(size_t)j * N + p] = stx(cx<R>{R(0), R(0)});
    }
    return;
  }
  const P* Th = theta + ((size_t)w * nc + off) * N;
  cd acc[SEED_R];
  int jj[SEED_R], pp[SEED_R];
#pragma unroll
  for (int r = 0; r < SEED_R; ++r) {
    const int e = threadIdx.x + r * AT;
    jj[r] = -1;
    pp[r] = 0;
    acc[r] = mk(0.0, 0.0);
    if (e < n * pr) {
      jj[r] = e / pr;
      pp[r] = p0 + e - (e / pr) * pr;
      acc[r] = mk(hhalf[(size_t)(off + jj[r]) * N + pp[r]], 0.0);
    }
  }
  for (int g = 0; g < G; ++g) {
    const R* Lg = Lh + ((size_t)g * nc + off) * N;
    __syncthreads();
    for (int e = threadIdx.x; e < n * n; e += AT) {
      const int j = e / n, i = e - (e / n) * n;
      const R* a = Lg + (size_t)j * N;
      const P* b = Th + (size_t)i * N;
      R sr = R(0), si = R(0);
      for (int q = 0; q < N; ++q) {
        sr = fmx(a[q], b[q].x, sr);
        si = fmx(a[q], b[q].y, si);
      }
      T[e] = stx(cx<R>{sr, si});
    }
    __syncthreads();
    const cx<R> tg = ldx(t[(size_t)w * G + g]);
#pragma unroll
    for (int r = 0; r < SEED_R; ++r) {
      if (jj[r] < 0) continue;
      const int j = jj[r], p = pp[r];
      cx<R> v = Lg[(size_t)j * N + p] * tg;
      for (int i = 0; i < n; ++i) v = v - Lg[(size_t)i * N + p] * ldx(T[j * n + i]);
      acc[r] = acc[r] + widen(v);
    }
  }
#pragma unroll
  for (int r = 0; r < SEED_R; ++r)
    if (jj[r] >= 0) out[(size_t)jj[r] * N + pp[r]] = stx(narrow<R>(mk(ew * acc[r].re, ew * acc[r].im)));
}

// ------------------------------------------------------------ final assembly
// Bs = (Re Bbar + Re Bbar^T) / 2
__global__ void adj_bsym_kernel(const double2* __restrict__ Bbar, double* __restrict__ Bs, int N) {
  const size_t NN = (size_t)N * N;
  for (size_t e = blockIdx.x * (size_t)AT + threadIdx.x; e < NN; e += (size_t)gridDim.x * AT) {
    const size_t p = e / N, q = e - p * N;
    Bs[e] = 0.5 * (Bbar[e].x + Bbar[q * N + p].x);
  }
}

// C[b] = op(A[b]) op(B[b]) for n x n real matrices (op = transpose when the
// flag is set), batch b = blockIdx.z with element strides sA, sB, sC.
__global__ void __launch_bounds__(256) adj_mm_kernel(const double* __restrict__ A, long long sA, int tA,
                                                     const double* __restrict__ B, long long sB, int tB,
                                                     double* __restrict__ C, long long sC, int n) {
  __shared__ double sa[16][17], sb[16][17];
  const int b = blockIdx.z;
  const double* Ab = A + (size_t)b * sA;
  const double* Bb = B + (size_t)b * sB;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int row = blockIdx.y * 16 + ty, col = blockIdx.x * 16 + tx;
  double acc = 0.0;
  for (int k0 = 0; k0 < n; k0 += 16) {
    const int ka = k0 + tx, kb = k0 + ty;
    double va = 0.0, vb = 0.0;
    if (row < n && ka < n) va = tA ? Ab[(size_t)ka * n + row] : Ab[(size_t)row * n + ka];
    if (col < n && kb < n) vb = tB ? Bb[(size_t)col * n + kb] : Bb[(size_t)kb * n + col];
    sa[ty][tx] = va;
    sb[ty][tx] = vb;
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 16; ++k) acc = fma(sa[ty][k], sb[k][tx], acc);
    __syncthreads();
  }
  if (row < n && col < n) C[(size_t)b * sC + (size_t)row * n + col] = acc;
}

// M[i][j] *= (f_i - f_j) / (lam_i - lam_j) with f = exp(-tau lam / 2)
// (f'(lam_i) when equal), written as -(tau/2) f_j expm1(x)/x, x = -tau (lam_i - lam_j)/2
__global__ void adj_dk_kernel(double* __restrict__ M, const double* __restrict__ lam, double tau, int N) {
  const size_t NN = (size_t)N * N;
  for (size_t e = blockIdx.x * (size_t)AT + threadIdx.x; e < NN; e += (size_t)gridDim.x * AT) {
    const int i = (int)(e / N), j = (int)(e - (size_t)i * N);
    const double x = -0.5 * tau * (lam[i] - lam[j]);
    const double phi = x == 0.0 ? 1.0 : expm1(x) / x;
    M[e] *= -0.5 * tau * exp(-0.5 * tau * lam[j]) * phi;
  }
}

// mubar[g] += sum_pq hbar[p][q] L_g[p][q]  (one block per g, fixed tree)
__global__ void __launch_bounds__(256) adj_mu_h_kernel(const double* __restrict__ L, const double* __restrict__ hbar,
                                                       double* __restrict__ mubar, size_t NN) {
  __shared__ double sh[8];
  const int g = blockIdx.x;
  const double* Lg = L + (size_t)g * NN;
  double s = 0.0;
  for (size_t e = threadIdx.x; e < NN; e += 256) s = fma(hbar[e], Lg[e], s);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < 8; ++i) t += sh[i];
    mubar[g] += t;
  }
}

// D[p][q] = sum_j trial[j][p] thT[j][q] = dL_bar_g / dL_g[p][q]
__global__ void adj_density_kernel(const double* __restrict__ trial, const double* __restrict__ thT,
                                   double* __restrict__ D, int N, int nc) {
  const size_t NN = (size_t)N * N;
  for (size_t e = blockIdx.x * (size_t)AT + threadIdx.x; e < NN; e += (size_t)gridDim.x * AT) {
    const int p = (int)(e / N), q = (int)(e - (size_t)p * N);
    double s = 0.0;
    for (int j = 0; j < nc; ++j) s = fma(trial[(size_t)j * N + p], thT[(size_t)j * N + q], s);
    D[e] = s;
  }
}

// grad_L[g] = sym( E_L part (in grad_L) + Re gLc[g] + Re sum_j trial[j][p] Lhb[g][j][q]
//                  - (X_g + X_g^T)/2 + L_bar_g hbar + mubar_g D ),  X_g = L_g hbar.
// One thread per unordered pair (p <= q) writes both entries.
__global__ void adj_final_L_kernel(double* __restrict__ gL, const double2* __restrict__ gLc,
                                   const double2* __restrict__ Lhb, const double* __restrict__ X,
                                   const double* __restrict__ hbar, const double* __restrict__ D,
                                   const double* __restrict__ trial, const double* __restrict__ Lbar,
                                   const double* __restrict__ mubar, int N, int nc, int G) {
  const size_t NN = (size_t)N * N, total = (size_t)G * NN;
  for (size_t e = blockIdx.x * (size_t)AT + threadIdx.x; e < total; e += (size_t)gridDim.x * AT) {
    const size_t g = e / NN, r = e - g * NN;
    const int p = (int)(r / N), q = (int)(r - (size_t)p * N);
    if (p > q) continue;
    const size_t pq = g * NN + (size_t)p * N + q, qp = g * NN + (size_t)q * N + p;
    const double2* Lg = Lhb + g * nc * N;
    double ep = 0.0, eq = 0.0;  // sum_j trial[j][p] Lhb[j][q] and the transposed entry
    for (int j = 0; j < nc; ++j) {
      ep = fma(trial[(size_t)j * N + p], Lg[(size_t)j * N + q].x, ep);
      eq = fma(trial[(size_t)j * N + q], Lg[(size_t)j * N + p].x, eq);
    }
    const double x = -0.5 * (X[pq] + X[qp]);
    const double mu = Lbar[g], mb = mubar[g];
    const double vpq = gL[pq] + gLc[pq].x + ep + x + mu * hbar[(size_t)p * N + q] + mb * D[(size_t)p * N + q];
    const double vqp = gL[qp] + gLc[qp].x + eq + x + mu * hbar[(size_t)q * N + p] + mb * D[(size_t)q * N + p];
    const double v = 0.5 * (vpq + vqp);
    gL[pq] = v;
    gL[qp] = v;
  }
}

// grad_h1 = sym(E_L part + hbar)
__global__ void adj_final_h_kernel(double* __restrict__ gh, const double* __restrict__ hbar, int N) {
  const size_t NN = (size_t)N * N;
  for (size_t e = blockIdx.x * (size_t)AT + threadIdx.x; e < NN; e += (size_t)gridDim.x * AT) {
    const int p = (int)(e / N), q = (int)(e - (size_t)p * N);
    if (p > q) continue;
    const size_t qp = (size_t)q * N + p;
    const double v = 0.5 * (gh[e] + gh[qp] + hbar[e] + hbar[qp]);
    gh[e] = v;
    gh[qp] = v;
  }
}

template <typename F>
cudaError_t smem_ok(F* f, size_t bytes) {
  if (bytes <= 48 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(reinterpret_cast<const void*>(f), cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)bytes);
}

// ---------------------------------------------------------------- Krylov action
// Reverse of the Arnoldi approximation e^A x ~ beta B_k e^{H_k} e_1 of one
// orbital column (Eqs. krylovsub-krylov; the forward is krylov_init/orth/
// expm/combine).  The norms and the inner products b_i^H w are not
// holomorphic, so inside these kernels the adjoint of a complex z is
// Gamma_z with dJ = Re sum conj(Gamma_z) dz; at their boundary it is
// converted to the holomorphic-style adjoint g = conj(Gamma) that the rest
// of the reverse pass uses.  The basis adjoints are stored as g (Gb), so
// that the product with A (g_b_j += A U_j, A symmetric) is a plain GEMM.

template <typename R>
__device__ __forceinline__ R wsum(R v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Seed of the output out = sum_i y_i b_i with adjoint g_out (= p2):
// g_y_i = b_i^T g_out and Gb_i = y_i g_out, i < k.  One warp per column.
template <typename R>
__global__ void kadj_seed_kernel(const typename C2<R>::t* __restrict__ gout, const typename C2<R>::t* __restrict__ basis,
                                 size_t bstride, const typename C2<R>::t* __restrict__ hy, size_t hs, int kmax,
                                 typename C2<R>::t* __restrict__ Gb, size_t gstride, double2* __restrict__ gy, int N,
                                 int ncols, int k) {
  const int col = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (col >= ncols) return;
  const typename C2<R>::t* g = gout + (size_t)col * N;
  for (int i = 0; i < k; ++i) {
    const cx<R> y = ldx(hy[(size_t)(i * kmax) * hs + col]);
    const typename C2<R>::t* b = basis + i * bstride + (size_t)col * N;
    typename C2<R>::t* o = Gb + i * gstride + (size_t)col * N;
    R sr = R(0), si = R(0);
    for (int p = lane; p < N; p += 32) {
      const cx<R> gv = ldx(g[p]), bv = ldx(b[p]);
      sr += bv.re * gv.re - bv.im * gv.im;
      si += bv.re * gv.im + bv.im * gv.re;
      o[p] = stx(y * gv);
    }
    sr = wsum(sr);
    si = wsum(si);
    if (lane == 0) gy[(size_t)i * hs + col] = make_double2((double)sr, (double)si);
  }
}

// Adjoint of y = beta e^{H} e_1 (FP64, one thread per column; beta is the
// real norm of the Arnoldi start, or the complex gamma = (psi^T psi)^{1/2}
// of the Lanczos one when cbeta is given).  With Gamma_y = conj(g_y) and
// u = conj(beta g_y):
//   Gamma_H = L(H^H, u e_1^T), the Frechet derivative of exp at H^H in the
//   direction u e_1^T; its column m is the top half of exp(M) [0; e_m] for
//   M = [[H^H, u e_1^T], [0, H^H]] (block-triangular exponential), taken by
//   sub-steps of a Taylor series on the 2k-vector (u scaled to unit norm,
//   the result scaled back: L is linear in its direction);
//   the start-norm adjoint, written to gbeta: Arnoldi Gamma_beta =
//   Re sum_i g_y_i y_i / beta (real part only), Lanczos g_gamma =
//   sum_i g_y_i y_i / gamma (holomorphic).
// Only the upper-Hessenberg entries of Gamma_H are written (the others are
// constant zeros of H).
template <typename R, int KM>
__global__ void __launch_bounds__(64) kadj_expm_kernel(const typename C2<R>::t* __restrict__ Hs,
                                                       const typename C2<R>::t* __restrict__ hy, size_t hs, int kmax,
                                                       const double* __restrict__ beta,
                                                       const double2* __restrict__ cbeta,
                                                       const double2* __restrict__ gy, double2* __restrict__ GH,
                                                       double2* __restrict__ gbeta, int ncols, int k) {
  const int col = blockIdx.x * 64 + threadIdx.x;
  if (col >= ncols) return;
  auto H = [&](int i, int j) -> cd { return ld(Hs + (size_t)(i * kmax + j) * hs + col); };
  const cd bc = cbeta ? ld(cbeta + col) : mk(beta[col], 0.0);
  const double bm2 = abs2(bc);
  cd u[KM];
  cd gsum = mk(0.0, 0.0);
  double un = 0.0;
#pragma unroll
  for (int i = 0; i < KM; ++i) {
    u[i] = mk(0.0, 0.0);
    if (i < k) {
      const cd g = ldc(gy[(size_t)i * hs + col]);
      gsum = gsum + g * ld(hy + (size_t)(i * kmax) * hs + col);
      u[i] = conj(bc * g);
      un += abs2(u[i]);
    }
  }
  const cd gb = bm2 > 0.0 ? (1.0 / bm2) * (gsum * conj(bc)) : mk(0.0, 0.0);
  gbeta[col] = make_double2(gb.re, cbeta ? gb.im : 0.0);
  un = sqrt(un);
  if (!(un > 0.0) || !(bm2 > 0.0)) {
    for (int m = 0; m < k; ++m)
      for (int i = 0; i <= m + 1 && i < k; ++i) GH[(size_t)(i * kmax + m) * hs + col] = make_double2(0.0, 0.0);
    return;
  }
  double u1 = 0.0;
#pragma unroll
  for (int i = 0; i < KM; ++i) {
    u[i] = (1.0 / un) * u[i];
    u1 += sqrt(abs2(u[i]));
  }
  // 1- and infinity-norms of H (H^H has them swapped)
  double n1 = 0.0, ni = 0.0;
  for (int j = 0; j < k; ++j) {
    double cs = 0.0, rs = 0.0;
    for (int i = 0; i <= j + 1 && i < k; ++i) cs += sqrt(abs2(H(i, j)));
    for (int i = (j > 0 ? j - 1 : 0); i < k; ++i) rs += sqrt(abs2(H(j, i)));
    n1 = fmax(n1, cs);
    ni = fmax(ni, rs);
  }
  const double nm = fmax(n1, ni) + u1;
  int msub = 1;
  if (nm < 1e30) msub = (int)ceil(nm / 2.0);
  if (msub < 1) msub = 1;
  if (msub > 4096) msub = 4096;
  const double sc = 1.0 / msub;
  for (int m = 0; m < k; ++m) {
    cd top[KM], bot[KM], tt[KM], tb[KM], nt[KM], nb[KM];
#pragma unroll
    for (int i = 0; i < KM; ++i) {
      top[i] = mk(0.0, 0.0);
      bot[i] = mk(i == m ? 1.0 : 0.0, 0.0);
    }
    for (int s = 0; s < msub; ++s) {
#pragma unroll
      for (int i = 0; i < KM; ++i) {
        tt[i] = top[i];
        tb[i] = bot[i];
      }
      for (int d = 1; d <= 80; ++d) {
        const double f = sc / d;
        // (H^H)_{ij} = conj(H_{ji}), nonzero for j <= i + 1
#pragma unroll
        for (int i = 0; i < KM; ++i) {
          cd at = mk(0.0, 0.0), ab = mk(0.0, 0.0);
          if (i < k) {
#pragma unroll
            for (int j = 0; j < KM; ++j)
              if (j <= i + 1 && j < k) {
                const cd a = conj(H(j, i));
                at = at + a * tt[j];
                ab = ab + a * tb[j];
              }
            at = at + u[i] * tb[0];
          }
          nt[i] = f * at;
          nb[i] = f * ab;
        }
        double tn = 0.0, an = 0.0;
#pragma unroll
        for (int i = 0; i < KM; ++i) {
          top[i] = top[i] + nt[i];
          bot[i] = bot[i] + nb[i];
          tt[i] = nt[i];
          tb[i] = nb[i];
          tn += abs2(nt[i]) + abs2(nb[i]);
          an += abs2(top[i]) + abs2(bot[i]);
        }
        if (tn <= 1e-36 * an) break;
      }
    }
#pragma unroll
    for (int i = 0; i < KM; ++i)
      if (i <= m + 1 && i < k) GH[(size_t)(i * kmax + m) * hs + col] = make_double2(un * top[i].re, un * top[i].im);
  }
}

// Reverse of Arnoldi step j (one warp per column, w in registers):
//   forward  w^(0) = A b_j;  h_ij = b_i^H w^(i), w^(i+1) = w^(i) - h_ij b_i
//            (i = 0..j);  nu = ||w^(j+1)||, b_{j+1} = w^(j+1) / nu (j+1 < k)
//   reverse  Gamma_nu = Re Gamma_H[j+1][j] - Re(Gamma_b_{j+1}^H b_{j+1}) / nu
//            Gamma_w  = Gamma_b_{j+1} / nu + Gamma_nu b_{j+1}
//            for i = j..0:  Gamma_h = Gamma_H[i][j] - b_i^H Gamma_w,
//              w^(i) = w^(i+1) + h_ij b_i,
//              Gamma_b_i += -conj(h_ij) Gamma_w + conj(Gamma_h) w^(i),
//              Gamma_w += Gamma_h b_i
//   U_j = conj(Gamma_w) is the adjoint of A b_j (the caller adds A U_j to
//   g_b_j and U_j b_j^T to the adjoint of A).  w^(j+1) is rebuilt from the
//   stored product A b_j and the stored h_ij in the forward's order.  A
//   column that broke down (nu = 0, b_{j+1} = 0) has Gamma_w = 0.
template <typename R, int EPL>
__global__ void kadj_orth_kernel(const typename C2<R>::t* __restrict__ basis, size_t bstride,
                                 const typename C2<R>::t* __restrict__ wj, const typename C2<R>::t* __restrict__ Hs,
                                 size_t hs, int kmax, const double2* __restrict__ GH, typename C2<R>::t* __restrict__ Gb,
                                 size_t gstride, typename C2<R>::t* __restrict__ U, int N, int ncols, int j, int k) {
  typedef typename C2<R>::t P;
  const int col = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (col >= ncols) return;
  const size_t co = (size_t)col * N;
  cx<R> w[EPL], gw[EPL];
#pragma unroll
  for (int e = 0; e < EPL; ++e) {
    const int p = lane + 32 * e;
    w[e] = cx<R>{R(0), R(0)};
    gw[e] = cx<R>{R(0), R(0)};
    if (p < N) w[e] = ldx(wj[co + p]);
  }
  for (int i = 0; i <= j; ++i) {
    const cx<R> h = ldx(Hs[(size_t)(i * kmax + j) * hs + col]);
    const P* b = basis + i * bstride + co;
#pragma unroll
    for (int e = 0; e < EPL; ++e) {
      const int p = lane + 32 * e;
      if (p < N) {
        const cx<R> v = ldx(b[p]);
        w[e].re -= h.re * v.re - h.im * v.im;
        w[e].im -= h.re * v.im + h.im * v.re;
      }
    }
  }
  if (j + 1 < k) {
    const R nu = Hs[(size_t)((j + 1) * kmax + j) * hs + col].x;
    if (nu > R(0)) {
      const P* bn = basis + (j + 1) * bstride + co;
      const P* gn = Gb + (j + 1) * gstride + co;
      cx<R> bv[EPL], gv[EPL];
      R dot = R(0);  // Re(Gamma_b^H b) = Re sum g b
#pragma unroll
      for (int e = 0; e < EPL; ++e) {
        const int p = lane + 32 * e;
        bv[e] = cx<R>{R(0), R(0)};
        gv[e] = cx<R>{R(0), R(0)};
        if (p < N) {
          bv[e] = ldx(bn[p]);
          gv[e] = ldx(gn[p]);
        }
        dot += gv[e].re * bv[e].re - gv[e].im * bv[e].im;
      }
      dot = wsum(dot);
      const double gnu = GH[(size_t)((j + 1) * kmax + j) * hs + col].x - (double)dot / (double)nu;
      const R inv = R(1) / nu, gr = (R)gnu;
#pragma unroll
      for (int e = 0; e < EPL; ++e) {
        gw[e].re = gv[e].re * inv + gr * bv[e].re;
        gw[e].im = -gv[e].im * inv + gr * bv[e].im;
      }
    }
  }
  for (int i = j; i >= 0; --i) {
    const cx<R> h = ldx(Hs[(size_t)(i * kmax + j) * hs + col]);
    const P* b = basis + i * bstride + co;
    P* gi = Gb + i * gstride + co;
    cx<R> bv[EPL];
    R sr = R(0), si = R(0);  // b_i^H Gamma_w
#pragma unroll
    for (int e = 0; e < EPL; ++e) {
      const int p = lane + 32 * e;
      bv[e] = cx<R>{R(0), R(0)};
      if (p < N) bv[e] = ldx(b[p]);
      sr += bv[e].re * gw[e].re + bv[e].im * gw[e].im;
      si += bv[e].re * gw[e].im - bv[e].im * gw[e].re;
    }
    sr = wsum(sr);
    si = wsum(si);
    const double2 gH = GH[(size_t)(i * kmax + j) * hs + col];
    const cx<R> gh{(R)(gH.x - (double)sr), (R)(gH.y - (double)si)};
#pragma unroll
    for (int e = 0; e < EPL; ++e) {
      const int p = lane + 32 * e;
      const cx<R> wp = w[e] + h * bv[e];  // w^(i)
      if (p < N) {
        // stored conjugated: g_b_i += -h conj(Gamma_w) + Gamma_h conj(w^(i))
        cx<R> g = ldx(gi[p]);
        g.re += -(h.re * gw[e].re + h.im * gw[e].im) + (gh.re * wp.re + gh.im * wp.im);
        g.im += -(h.im * gw[e].re - h.re * gw[e].im) + (gh.im * wp.re - gh.re * wp.im);
        gi[p] = stx(g);
      }
      gw[e] = gw[e] + gh * bv[e];
      w[e] = wp;
    }
  }
#pragma unroll
  for (int e = 0; e < EPL; ++e) {
    const int p = lane + 32 * e;
    if (p < N) U[co + p] = stx(cx<R>{gw[e].re, -gw[e].im});
  }
}

// Adjoint of b_0 = x / beta, beta = ||x||, into g_x = conj(Gamma_x):
//   Gamma_beta_tot = Gamma_beta - Re(Gamma_b0^H b_0) / beta
//   Gamma_x = Gamma_b0 / beta + Gamma_beta_tot b_0
// (g_x = 0 for a zero column, whose forward output is identically zero).
template <typename R>
__global__ void kadj_input_kernel(const typename C2<R>::t* __restrict__ basis, const typename C2<R>::t* __restrict__ Gb0,
                                  const double* __restrict__ beta, const double2* __restrict__ gbeta,
                                  typename C2<R>::t* __restrict__ gx, int N, int ncols) {
  const int col = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (col >= ncols) return;
  const size_t co = (size_t)col * N;
  const double b = beta[col];
  if (!(b > 0.0)) {
    for (int p = lane; p < N; p += 32) gx[co + p] = stx(cx<R>{R(0), R(0)});
    return;
  }
  R dot = R(0);
  for (int p = lane; p < N; p += 32) {
    const cx<R> g = ldx(Gb0[co + p]), v = ldx(basis[co + p]);
    dot += g.re * v.re - g.im * v.im;
  }
  dot = wsum(dot);
  const R gbt = (R)(gbeta[col].x - (double)dot / b), inv = (R)(1.0 / b);
  for (int p = lane; p < N; p += 32) {
    const cx<R> g = ldx(Gb0[co + p]), v = ldx(basis[co + p]);
    gx[co + p] = stx(cx<R>{g.re * inv + gbt * v.re, g.im * inv - gbt * v.im});
  }
}

// Reverse of Lanczos step j (one warp per column).  The three-term
// recurrence uses bilinear forms and principal square roots, both
// holomorphic, so here every adjoint is the g of dJ = Re sum g dz and the
// small exponential's Gamma_T enters as g_T = conj(Gamma_T):
//   forward  w1 = A v_j - beta_{j-1} v_{j-1},  alpha_j = v_j^T w1,
//            w2 = w1 - alpha_j v_j,  beta_j = (w2^T w2)^{1/2},
//            v_{j+1} = w2 / beta_j  (j + 1 < k; zero after a breakdown)
//   reverse  g_beta_j = g_T[j+1][j] + g_T[j][j+1] + carry
//                       - (g_v_{j+1}^T v_{j+1}) / beta_j
//            g_w2 = g_v_{j+1} / beta_j + g_beta_j v_{j+1}   (0 if beta_j = 0)
//            g_alpha = g_T[j][j] - g_w2^T v_j
//            g_v_j += -alpha_j g_w2 + g_alpha w1
//            U_j = g_w1 = g_w2 + g_alpha v_j
//            g_v_{j-1} += -beta_{j-1} U_j,  carry <- -U_j^T v_{j-1}
// The per-column carry passes the part of g_beta_{j-1} that the term
// -beta_{j-1} v_{j-1} of w1 contributes from step j to step j - 1.  The
// caller adds A U_j to g_v_j and U_j v_j^T to the adjoint of A.  w1 is
// rebuilt from the stored product A v_j; the scalar arithmetic runs in the
// walkers' precision, as in the forward.
template <typename R, int EPL>
__global__ void lzadj_step_kernel(const typename C2<R>::t* __restrict__ basis, size_t bstride,
                                  const typename C2<R>::t* __restrict__ wj, const typename C2<R>::t* __restrict__ Hs,
                                  size_t hs, int kmax, const double2* __restrict__ GH,
                                  typename C2<R>::t* __restrict__ Gb, size_t gstride, typename C2<R>::t* __restrict__ U,
                                  double2* __restrict__ carry, int N, int ncols, int j, int k) {
  typedef typename C2<R>::t P;
  const int col = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (col >= ncols) return;
  const size_t co = (size_t)col * N;
  auto T = [&](int r, int q) { return ldx(Hs[(size_t)(r * kmax + q) * hs + col]); };
  auto gT = [&](int r, int q) {
    const double2 g = GH[(size_t)(r * kmax + q) * hs + col];
    return cx<R>{(R)g.x, (R)(-g.y)};
  };
  const cx<R> zero{R(0), R(0)};
  const cx<R> bp = j > 0 ? T(j, j - 1) : zero, al = T(j, j);
  const double2 cj = carry[col];
  const P* vj = basis + j * bstride + co;
  const P* vm = basis + (j > 0 ? j - 1 : 0) * bstride + co;
  cx<R> w1[EPL], v[EPL], gw[EPL];
#pragma unroll
  for (int e = 0; e < EPL; ++e) {
    const int p = lane + 32 * e;
    w1[e] = zero;
    v[e] = zero;
    gw[e] = zero;
    if (p < N) {
      w1[e] = ldx(wj[co + p]);
      v[e] = ldx(vj[p]);
      if (j > 0) w1[e] = w1[e] - bp * ldx(vm[p]);
    }
  }
  if (j + 1 < k) {
    const cx<R> be = T(j + 1, j);
    const R m2 = be.re * be.re + be.im * be.im;
    if (m2 > R(0)) {
      const P* vn = basis + (j + 1) * bstride + co;
      const P* gn = Gb + (j + 1) * gstride + co;
      cx<R> vv[EPL], gv[EPL];
      R dr = R(0), di = R(0);  // g_v_{j+1}^T v_{j+1}
#pragma unroll
      for (int e = 0; e < EPL; ++e) {
        const int p = lane + 32 * e;
        vv[e] = zero;
        gv[e] = zero;
        if (p < N) {
          vv[e] = ldx(vn[p]);
          gv[e] = ldx(gn[p]);
        }
        dr += gv[e].re * vv[e].re - gv[e].im * vv[e].im;
        di += gv[e].re * vv[e].im + gv[e].im * vv[e].re;
      }
      dr = wsum(dr);
      di = wsum(di);
      const cx<R> ib{be.re / m2, -be.im / m2};
      const cx<R> gb = gT(j + 1, j) + gT(j, j + 1) + cx<R>{(R)cj.x, (R)cj.y} - ib * cx<R>{dr, di};
#pragma unroll
      for (int e = 0; e < EPL; ++e) gw[e] = ib * gv[e] + gb * vv[e];
    }
  }
  R sr = R(0), si = R(0);  // g_w2^T v_j
#pragma unroll
  for (int e = 0; e < EPL; ++e) {
    sr += gw[e].re * v[e].re - gw[e].im * v[e].im;
    si += gw[e].re * v[e].im + gw[e].im * v[e].re;
  }
  sr = wsum(sr);
  si = wsum(si);
  const cx<R> ga = gT(j, j) - cx<R>{sr, si};
  P* gj = Gb + j * gstride + co;
  P* gm = Gb + (j > 0 ? j - 1 : 0) * gstride + co;
  R cr = R(0), ci = R(0);  // U_j^T v_{j-1}
#pragma unroll
  for (int e = 0; e < EPL; ++e) {
    const int p = lane + 32 * e;
    if (p < N) {
      const cx<R> u = gw[e] + ga * v[e];
      gj[p] = stx(ldx(gj[p]) - al * gw[e] + ga * w1[e]);
      U[co + p] = stx(u);
      if (j > 0) {
        const cx<R> vp = ldx(vm[p]);
        cr += u.re * vp.re - u.im * vp.im;
        ci += u.re * vp.im + u.im * vp.re;
        gm[p] = stx(ldx(gm[p]) - bp * u);
      }
    }
  }
  if (j > 0) {
    cr = wsum(cr);
    ci = wsum(ci);
    if (lane == 0) carry[col] = make_double2(-(double)cr, -(double)ci);
  }
}

// Adjoint of the Lanczos start v_0 = x / gamma, gamma = (x^T x)^{1/2}:
//   g_gamma_tot = g_gamma - (g_v0^T v_0) / gamma
//   g_x = g_v0 / gamma + g_gamma_tot v_0
// with g_gamma from the small exponential's adjoint (y = gamma e^{T} e_1);
// g_x = 0 for a column with gamma = 0, whose output is identically zero.
template <typename R>
__global__ void lzadj_input_kernel(const typename C2<R>::t* __restrict__ basis,
                                   const typename C2<R>::t* __restrict__ Gb0, const double2* __restrict__ cbeta,
                                   const double2* __restrict__ ggam, typename C2<R>::t* __restrict__ gx, int N,
                                   int ncols) {
  const int col = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (col >= ncols) return;
  const size_t co = (size_t)col * N;
  const double2 gm = cbeta[col];
  const R m2 = (R)gm.x * (R)gm.x + (R)gm.y * (R)gm.y;
  if (!(m2 > R(0))) {
    for (int p = lane; p < N; p += 32) gx[co + p] = stx(cx<R>{R(0), R(0)});
    return;
  }
  R dr = R(0), di = R(0);
  for (int p = lane; p < N; p += 32) {
    const cx<R> g = ldx(Gb0[co + p]), v = ldx(basis[co + p]);
    dr += g.re * v.re - g.im * v.im;
    di += g.re * v.im + g.im * v.re;
  }
  dr = wsum(dr);
  di = wsum(di);
  const cx<R> ig{(R)gm.x / m2, -(R)gm.y / m2};
  const double2 gg = ggam[col];
  const cx<R> gt = cx<R>{(R)gg.x, (R)gg.y} - ig * cx<R>{dr, di};
  for (int p = lane; p < N; p += 32) {
    const cx<R> g = ldx(Gb0[co + p]), v = ldx(basis[co + p]);
    gx[co + p] = stx(ig * g + gt * v);
  }
}

}  // namespace

// ------------------------------------------------------------ launch wrappers
// the trial and Lh in the walkers' precision (mixed contexts hold FP32 copies)
template <typename R>
const R* trial_of(const afqmc_ctx* c);
template <>
const double* trial_of<double>(const afqmc_ctx* c) { return c->d_trial; }
template <>
const float* trial_of<float>(const afqmc_ctx* c) { return c->f_trial; }
template <typename R>
const R* lh_of(const afqmc_ctx* c);
template <>
const double* lh_of<double>(const afqmc_ctx* c) { return c->d_Lh; }
template <>
const float* lh_of<float>(const afqmc_ctx* c) { return c->f_Lh; }

template <typename R>
cudaError_t adj_sanitize(const typename C2<R>::t* src, typename C2<R>::t* dst, const double* wfin,
                         const double* trial, size_t per, int Nw, cudaStream_t s) {
  const size_t total = per * Nw;
  adj_sanitize_kernel<R><<<grid_for(total), AT, 0, s>>>(src, dst, wfin, trial, per, total);
  return cudaGetLastError();
}

template <typename R>
cudaError_t adj_sum_terms(const typename C2<R>::t* T, typename C2<R>::t* out, int K1, size_t per, int Nw,
                          cudaStream_t s) {
  const size_t total = per * Nw;
  adj_sum_terms_kernel<R><<<grid_for(total), AT, 0, s>>>(T, out, K1, per, total);
  return cudaGetLastError();
}

template <typename R>
cudaError_t adj_scale_copy(const typename C2<R>::t* src, size_t sstride, typename C2<R>::t* dst, size_t dstride,
                           double sc, size_t per, int Nw, cudaStream_t s) {
  const size_t total = per * Nw;
  adj_scale_copy_kernel<R><<<grid_for(total), AT, 0, s>>>(src, sstride, dst, dstride, sc, per, total);
  return cudaGetLastError();
}

cudaError_t adj_fold(const float2* src, double2* dst, size_t n, cudaStream_t s) {
  adj_fold_kernel<<<grid_for(n), AT, 0, s>>>(src, dst, n);
  return cudaGetLastError();
}

size_t adj_lu_smem(int nmax) { return (size_t)(2 * nmax * nmax + nmax) * sizeof(double2); }
size_t adj_small_smem(int nmax) { return (size_t)3 * nmax * nmax * sizeof(double2); }

template <typename R>
cudaError_t adj_lu(const afqmc_ctx* c, int Nw, const typename C2<R>::t* psi, double2* oinv, double* logdet,
                   cudaStream_t s) {
  const int nmax = c->na > c->nb ? c->na : c->nb;
  const size_t shm = adj_lu_smem(nmax);
  cudaError_t e = smem_ok(adj_lu_kernel<R>, shm);
  if (e != cudaSuccess) return e;
  adj_lu_kernel<R><<<dim3(Nw, 2), AT, shm, s>>>(psi, trial_of<R>(c), oinv, logdet, c->N, c->na, c->nb, nmax);
  return cudaGetLastError();
}

cudaError_t adj_ratio_coef(int Nw, const double* wfin, const double* omega, const double* ld3, const double* logovl,
                           const double* scal, double2* aR, double sqrt_tau, cudaStream_t s) {
  adj_ratio_coef_kernel<<<(Nw + 127) / 128, 128, 0, s>>>(wfin, omega, ld3, logovl, scal, aR, sqrt_tau, Nw);
  return cudaGetLastError();
}

template <typename R>
cudaError_t adj_ratio(const afqmc_ctx* c, int Nw, const typename C2<R>::t* pnext, const typename C2<R>::t* psinext,
                      const double2* oinv3, const double2* aR, const double* wfin, typename C2<R>::t* p3, int qr,
                      cudaStream_t s) {
  const int nmax = c->na > c->nb ? c->na : c->nb;
  const size_t shm = adj_small_smem(nmax);
  cudaError_t e = smem_ok(adj_ratio_kernel<R>, shm);
  if (e != cudaSuccess) return e;
  adj_ratio_kernel<R><<<dim3(Nw, 2), AT, shm, s>>>(pnext, psinext, trial_of<R>(c), oinv3, aR, wfin, p3, c->N, c->na,
                                                   c->nb, nmax, qr);
  return cudaGetLastError();
}

template <typename R>
cudaError_t adj_force(const afqmc_ctx* c, int Nw, const typename C2<R>::t* cbar, const typename C2<R>::t* cc,
                      const uint8_t* keep, const double2* aR, const double* omega, typename C2<R>::t* tbar,
                      double* mu_part, double* mubar, double sqrt_tau, double tau, cudaStream_t s) {
  const size_t total = (size_t)Nw * c->G;
  adj_force_kernel<R><<<grid_for(total), AT, 0, s>>>(cbar, cc, keep, aR, omega, c->d_Lbar, tbar, mu_part, c->G,
                                                     sqrt_tau, tau, total);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  adj_mu_reduce_kernel<<<(c->G + 127) / 128, 128, 0, s>>>(mu_part, mubar, Nw, c->G);
  return cudaGetLastError();
}

template <typename R>
cudaError_t adj_theta(const afqmc_ctx* c, int Nw, const typename C2<R>::t* thbar, const typename C2<R>::t* theta,
                      const double2* oinv, const double2* aR, const double* wfin, typename C2<R>::t* pbar,
                      cudaStream_t s) {
  const int nmax = c->na > c->nb ? c->na : c->nb;
  const size_t shm = adj_small_smem(nmax);
  cudaError_t e = smem_ok(adj_theta_kernel<R>, shm);
  if (e != cudaSuccess) return e;
  adj_theta_kernel<R><<<dim3(Nw, 2), AT, shm, s>>>(thbar, theta, trial_of<R>(c), oinv, aR, wfin, pbar, c->N, c->na,
                                                   c->nb, nmax);
  return cudaGetLastError();
}

cudaError_t adj_seed_coef(int Nw, const double* wfin, const double* ecap, const double* e_loc, const double* emix,
                          double* omega, double* ecoef, double e0, double dE, double dJ, cudaStream_t s) {
  adj_seed_coef_kernel<<<(Nw + 255) / 256, 256, 0, s>>>(wfin, ecap, e_loc, emix, omega, ecoef, Nw, e0, dE, dJ);
  return cudaGetLastError();
}

template <typename R>
cudaError_t adj_eloc_seed(const afqmc_ctx* c, int Nw, const typename C2<R>::t* theta, const typename C2<R>::t* t,
                          const double* ecoef, typename C2<R>::t* thbar, cudaStream_t s) {
  const int nmax = c->na > c->nb ? c->na : c->nb;
  if (nmax == 0) return cudaSuccess;
  int prows = (SEED_R * AT) / nmax;
  if (prows > c->N) prows = c->N;
  const int chunks = (c->N + prows - 1) / prows;
  const size_t shm = (size_t)nmax * nmax * sizeof(typename C2<R>::t);
  cudaError_t e = smem_ok(adj_eloc_seed_kernel<R>, shm);
  if (e != cudaSuccess) return e;
  adj_eloc_seed_kernel<R><<<dim3(Nw, 2, chunks), AT, shm, s>>>(theta, t, lh_of<R>(c), c->d_hhalf, ecoef, thbar,
                                                              c->N, c->na, c->nb, c->G, prows);
  return cudaGetLastError();
}

// Krylov-action reverse (the forward's basis, Hessenberg and beta in the
// workspace; hs = column capacity of the Hessenberg arrays)
template <typename R>
cudaError_t kadj_seed(const afqmc_ctx* c, int Nw, int k, const typename C2<R>::t* gout, typename C2<R>::t* Gb,
                      size_t gstride, double2* gy, cudaStream_t s) {
  const int ncols = Nw * c->nc;
  const size_t hs = (size_t)c->ws.n_walkers * c->nc, bstride = hs * c->N;
  kadj_seed_kernel<R><<<(ncols + 7) / 8, 256, 0, s>>>(
      gout, static_cast<const typename C2<R>::t*>(c->ws.basis), bstride,
      reinterpret_cast<const typename C2<R>::t*>(c->ws.hess), hs, c->ws.kmax, Gb, gstride, gy, c->N, ncols, k);
  return cudaGetLastError();
}

template <typename R, int KM>
static cudaError_t kadj_expm_k(const afqmc_ctx* c, int ncols, int k, const typename C2<R>::t* Hs, const double2* gy,
                               double2* GH, double2* gbeta, bool lanczos, cudaStream_t s) {
  const size_t hs = (size_t)c->ws.n_walkers * c->nc;
  kadj_expm_kernel<R, KM><<<(ncols + 63) / 64, 64, 0, s>>>(
      Hs, reinterpret_cast<const typename C2<R>::t*>(c->ws.hess), hs, c->ws.kmax, c->ws.beta,
      lanczos ? c->ws.cbeta : nullptr, gy, GH, gbeta, ncols, k);
  return cudaGetLastError();
}

template <typename R>
cudaError_t kadj_expm(const afqmc_ctx* c, int Nw, int k, const typename C2<R>::t* Hs, const double2* gy, double2* GH,
                      double2* gbeta, bool lanczos, cudaStream_t s) {
  const int ncols = Nw * c->nc;
  return k <= 8 ? kadj_expm_k<R, 8>(c, ncols, k, Hs, gy, GH, gbeta, lanczos, s)
         : k <= 16 ? kadj_expm_k<R, 16>(c, ncols, k, Hs, gy, GH, gbeta, lanczos, s)
                   : kadj_expm_k<R, 32>(c, ncols, k, Hs, gy, GH, gbeta, lanczos, s);
}

template <typename R>
cudaError_t kadj_orth(const afqmc_ctx* c, int Nw, int j, int k, const typename C2<R>::t* wj,
                      const typename C2<R>::t* Hs, const double2* GH, typename C2<R>::t* Gb, size_t gstride,
                      typename C2<R>::t* U, cudaStream_t s) {
  const int ncols = Nw * c->nc;
  const size_t hs = (size_t)c->ws.n_walkers * c->nc, bstride = hs * c->N;
  const typename C2<R>::t* B = static_cast<const typename C2<R>::t*>(c->ws.basis);
  const dim3 grid((ncols + 7) / 8);
  if (c->N <= 128)
    kadj_orth_kernel<R, 4><<<grid, 256, 0, s>>>(B, bstride, wj, Hs, hs, c->ws.kmax, GH, Gb, gstride, U, c->N, ncols,
                                                j, k);
  else if (c->N <= 256)
    kadj_orth_kernel<R, 8><<<grid, 256, 0, s>>>(B, bstride, wj, Hs, hs, c->ws.kmax, GH, Gb, gstride, U, c->N, ncols,
                                                j, k);
  else
    kadj_orth_kernel<R, 16><<<grid, 256, 0, s>>>(B, bstride, wj, Hs, hs, c->ws.kmax, GH, Gb, gstride, U, c->N,
                                                 ncols, j, k);
  return cudaGetLastError();
}

template <typename R>
cudaError_t kadj_input(const afqmc_ctx* c, int Nw, const typename C2<R>::t* Gb0, const double2* gbeta,
                       typename C2<R>::t* gx, bool lanczos, cudaStream_t s) {
  const int ncols = Nw * c->nc;
  const typename C2<R>::t* B = static_cast<const typename C2<R>::t*>(c->ws.basis);
  if (lanczos)
    lzadj_input_kernel<R><<<(ncols + 7) / 8, 256, 0, s>>>(B, Gb0, c->ws.cbeta, gbeta, gx, c->N, ncols);
  else
    kadj_input_kernel<R><<<(ncols + 7) / 8, 256, 0, s>>>(B, Gb0, c->ws.beta, gbeta, gx, c->N, ncols);
  return cudaGetLastError();
}

template <typename R>
cudaError_t lzadj_step(const afqmc_ctx* c, int Nw, int j, int k, const typename C2<R>::t* wj,
                       const typename C2<R>::t* Hs, const double2* GH, typename C2<R>::t* Gb, size_t gstride,
                       typename C2<R>::t* U, double2* carry, cudaStream_t s) {
  const int ncols = Nw * c->nc;
  const size_t hs = (size_t)c->ws.n_walkers * c->nc, bstride = hs * c->N;
  const typename C2<R>::t* B = static_cast<const typename C2<R>::t*>(c->ws.basis);
  const dim3 grid((ncols + 7) / 8);
  if (c->N <= 128)
    lzadj_step_kernel<R, 4><<<grid, 256, 0, s>>>(B, bstride, wj, Hs, hs, c->ws.kmax, GH, Gb, gstride, U, carry, c->N,
                                                 ncols, j, k);
  else if (c->N <= 256)
    lzadj_step_kernel<R, 8><<<grid, 256, 0, s>>>(B, bstride, wj, Hs, hs, c->ws.kmax, GH, Gb, gstride, U, carry, c->N,
                                                 ncols, j, k);
  else
    lzadj_step_kernel<R, 16><<<grid, 256, 0, s>>>(B, bstride, wj, Hs, hs, c->ws.kmax, GH, Gb, gstride, U, carry,
                                                  c->N, ncols, j, k);
  return cudaGetLastError();
}

#define AFQ_ADJ_INST(R)                                                                                            \
  template cudaError_t kadj_seed<R>(const afqmc_ctx*, int, int, const C2<R>::t*, C2<R>::t*, size_t, double2*,      \
                                    cudaStream_t);                                                                 \
  template cudaError_t kadj_expm<R>(const afqmc_ctx*, int, int, const C2<R>::t*, const double2*, double2*,        \
                                    double2*, bool, cudaStream_t);                                                 \
  template cudaError_t kadj_orth<R>(const afqmc_ctx*, int, int, int, const C2<R>::t*, const C2<R>::t*,              \
                                    const double2*, C2<R>::t*, size_t, C2<R>::t*, cudaStream_t);                   \
  template cudaError_t kadj_input<R>(const afqmc_ctx*, int, const C2<R>::t*, const double2*, C2<R>::t*, bool,      \
                                     cudaStream_t);                                                                \
  template cudaError_t lzadj_step<R>(const afqmc_ctx*, int, int, int, const C2<R>::t*, const C2<R>::t*,             \
                                     const double2*, C2<R>::t*, size_t, C2<R>::t*, double2*, cudaStream_t);        \
  template cudaError_t adj_sanitize<R>(const C2<R>::t*, C2<R>::t*, const double*, const double*, size_t, int,     \
                                       cudaStream_t);                                                              \
  template cudaError_t adj_sum_terms<R>(const C2<R>::t*, C2<R>::t*, int, size_t, int, cudaStream_t);               \
  template cudaError_t adj_scale_copy<R>(const C2<R>::t*, size_t, C2<R>::t*, size_t, double, size_t, int,          \
                                         cudaStream_t);                                                            \
  template cudaError_t adj_lu<R>(const afqmc_ctx*, int, const C2<R>::t*, double2*, double*, cudaStream_t);         \
  template cudaError_t adj_ratio<R>(const afqmc_ctx*, int, const C2<R>::t*, const C2<R>::t*, const double2*,       \
                                    const double2*, const double*, C2<R>::t*, int, cudaStream_t);                  \
  template cudaError_t adj_force<R>(const afqmc_ctx*, int, const C2<R>::t*, const C2<R>::t*, const uint8_t*,       \
                                    const double2*, const double*, C2<R>::t*, double*, double*, double, double,    \
                                    cudaStream_t);                                                                 \
  template cudaError_t adj_theta<R>(const afqmc_ctx*, int, const C2<R>::t*, const C2<R>::t*, const double2*,       \
                                    const double2*, const double*, C2<R>::t*, cudaStream_t);                       \
  template cudaError_t adj_eloc_seed<R>(const afqmc_ctx*, int, const C2<R>::t*, const C2<R>::t*, const double*,    \
                                        C2<R>::t*, cudaStream_t);
AFQ_ADJ_INST(double)
AFQ_ADJ_INST(float)
#undef AFQ_ADJ_INST

// hbar'' from Bbar: hbar = V (F o (V^T sym(Re Bbar) V)) V^T; then
// mubar += <hbar, L_g>, X_g = L_g hbar, and the final symmetrised gradients.
cudaError_t adj_finish(const afqmc_ctx* c, const double2* Bbar, const double* V, const double* lam, double tau,
                       double* Bs, double* T1, double* M1, double* hbar, double* X, double* D, const double2* gLc,
                       const double2* Lhb, double* mubar, double* grad_h1, double* grad_L, int* n_launch,
                       cudaStream_t s) {
  const int N = c->N, G = c->G, nc = c->nc;
  const size_t NN = (size_t)N * N;
  const dim3 mg((N + 15) / 16, (N + 15) / 16, 1);
  cudaError_t e;
#define AFQ_L(expr)                      \
  do {                                   \
    expr;                                \
    e = cudaGetLastError();              \
    if (e != cudaSuccess) return e;      \
    ++*n_launch;                         \
  } while (0)
  AFQ_L((adj_bsym_kernel<<<grid_for(NN), AT, 0, s>>>(Bbar, Bs, N)));
  AFQ_L((adj_mm_kernel<<<mg, 256, 0, s>>>(V, 0, 1, Bs, 0, 0, T1, 0, N)));      // V^T Bs
  AFQ_L((adj_mm_kernel<<<mg, 256, 0, s>>>(T1, 0, 0, V, 0, 0, M1, 0, N)));      // (V^T Bs) V
  AFQ_L((adj_dk_kernel<<<grid_for(NN), AT, 0, s>>>(M1, lam, tau, N)));
  AFQ_L((adj_mm_kernel<<<mg, 256, 0, s>>>(V, 0, 0, M1, 0, 0, T1, 0, N)));      // V M
  AFQ_L((adj_mm_kernel<<<mg, 256, 0, s>>>(T1, 0, 0, V, 0, 1, hbar, 0, N)));    // (V M) V^T
  AFQ_L((adj_mu_h_kernel<<<G, 256, 0, s>>>(c->d_L, hbar, mubar, NN)));
  AFQ_L((adj_mm_kernel<<<dim3(mg.x, mg.y, G), 256, 0, s>>>(c->d_L, (long long)NN, 0, hbar, 0, 0, X,
                                                          (long long)NN, N)));  // X_g = L_g hbar
  AFQ_L((adj_density_kernel<<<grid_for(NN), AT, 0, s>>>(c->d_trial, c->d_thT, D, N, nc)));
  AFQ_L((adj_final_L_kernel<<<grid_for((size_t)G * NN), AT, 0, s>>>(grad_L, gLc, Lhb, X, hbar, D, c->d_trial,
                                                                    c->d_Lbar, mubar, N, nc, G)));
  AFQ_L((adj_final_h_kernel<<<grid_for(NN), AT, 0, s>>>(grad_h1, hbar, N)));
#undef AFQ_L
  return cudaSuccess;
}

}  // namespace afq
