// Adjoint of the mixed energy estimator at fixed walkers and weights.
//
// With M_ws = Theta_ws trial_s^T (N x N, the transposed mixed density of
// walker w, spin s), the local energy of Eq. eloc reads
//   E_L = E_const + sum_s tr(h1 M_ws)
//         + 1/2 sum_g [ (sum_s tr(L_g M_ws))^2 - sum_s tr(L_g M_ws L_g M_ws) ],
// so (derivatives with respect to the entries of h1 and of each L_g)
//   dE_L/dh1  = sum_s trial_s Theta_ws^T
//   dE_L/dL_g = sum_s trial_s [ t_wg I - T_wgs^T ] Theta_ws^T,
// where T_wgs = trial_s^T L_g Theta_ws (n x n) and t_wg = sum_s tr T_wgs.
// The mixed estimator E_k = sum_w W_w Ebar_L,w / sum_w W_w (Sec. II.A) with
// the window of Eq. enwin has dEbar/dRe E_L = 1 strictly inside the window
// and 0 outside, so
//   dE_k/dh1  = Re sum_s trial_s Z_s,        Z_s   = sum_w c_w Theta_ws^T
//   dE_k/dL_g = Re sum_s trial_s Y_gs,       Y_gs  = sum_w c_w [t_wg Theta_ws^T - T_wgs^T Theta_ws^T]
// with c_w = m_w W_w / sum W (m_w the window mask).  The per-walker terms are
// formed in the walkers' precision (FP32 for the complex64 walkers of mixed
// contexts) and summed over walkers in FP64.
#include <type_traits>

#include "internal.cuh"

namespace afq {

namespace {

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// c_w = m_w W_w / sum_{live} W (one block); m_w = 1 strictly inside the window.
__global__ void __launch_bounds__(256) adj_coef_kernel(const double* __restrict__ weight,
                                                       const double* __restrict__ e_loc, double* __restrict__ coef,
                                                       int Nw, double e0, double dE, double dJ) {
  __shared__ double sh[8];
  double s = 0.0;
  for (int w = threadIdx.x; w < Nw; w += 256)
    if (weight[w] > 0.0) s += weight[w];
  s = warp_sum_d(s);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  double tot = 0.0;
  for (int i = 0; i < 8; ++i) tot += sh[i];
  for (int w = threadIdx.x; w < Nw; w += 256) {
    const double W = weight[w], e = e_loc[2 * w];
    const bool inside = e > e0 - dE && e < e0 + dE;
    coef[w] = (W > 0.0 && inside && tot > 0.0) ? dJ * W / tot : 0.0;
  }
}

// Z_s[i][q] = sum_w c_w Theta[w][off+i][q]   (grid: nc rows; fixed walker order)
template <typename R>
__global__ void adj_z_kernel(const typename C2<R>::t* __restrict__ theta, const double* __restrict__ coef,
                             double2* __restrict__ Z, int N, int nc, int Nw) {
  const int j = blockIdx.x;
  for (int q = threadIdx.x; q < N; q += blockDim.x) {
    double zr = 0.0, zi = 0.0;
    for (int w = 0; w < Nw; ++w) {
      const double cw = coef[w];
      if (cw == 0.0) continue;
      const typename C2<R>::t t = theta[((size_t)w * nc + j) * N + q];
      zr += cw * (double)t.x;
      zi += cw * (double)t.y;
    }
    Z[(size_t)j * N + q] = make_double2(zr, zi);
  }
}

__device__ __forceinline__ double fmx(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float fmx(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_sum(double v) { return warp_sum_d(v); }

// Y_gs[i][q] = sum_w c_w [ t_wg Theta_ws[q][i] - sum_j T_wgs[j][i] Theta_ws[q][j] ]
// One block per (g, spin); walkers in order; T_wgs = Lh_gs Theta_ws (as in E_L).
// Shared: the FP64 accumulator Y [n][N], then T [n][n] and t in the walkers'
// precision.
template <typename R>
__global__ void __launch_bounds__(256) adj_y_kernel(const typename C2<R>::t* __restrict__ theta,
                                                    const R* __restrict__ Lh, const double* __restrict__ coef,
                                                    double2* __restrict__ Y, int N, int na, int nb, int G, int Nw) {
  typedef typename C2<R>::t P;
  extern __shared__ double2 smem_adj[];
  const int g = blockIdx.x, spin = blockIdx.y;
  const int n = spin ? nb : na, off = spin ? na : 0, nc = na + nb;
  double2* Yo = Y + ((size_t)g * nc + off) * N;
  if (n == 0) return;
  double2* sY = smem_adj;                             // [n][N]  accumulator
  P* sT = reinterpret_cast<P*>(sY + (size_t)n * N);   // [n][n]  T[i][j]
  __shared__ P s_t;                                   // t_wg summed over both spins
  for (int e = threadIdx.x; e < n * N; e += blockDim.x) sY[e] = make_double2(0.0, 0.0);
  const R* Lg = Lh + (size_t)g * nc * N;
  for (int w = 0; w < Nw; ++w) {
    const double cw = coef[w];
    if (cw == 0.0) continue;  // uniform across the block
    const P* Th = theta + (size_t)w * nc * N;
    // T[i][j] for this spin, and the trace over both spins
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
      const int i = e / n, j = e % n;
      const R* a = Lg + (size_t)(off + i) * N;
      const P* b = Th + (size_t)(off + j) * N;
      R sr = R(0), si = R(0);
      for (int q = 0; q < N; ++q) {
        sr = fmx(a[q], b[q].x, sr);
        si = fmx(a[q], b[q].y, si);
      }
      sT[e].x = sr;
      sT[e].y = si;
    }
    if (threadIdx.x < 32) {  // t_wg = sum over both spins of tr(Lh_g Theta)
      R tr = R(0), ti = R(0);
      for (int j = threadIdx.x; j < nc; j += 32) {
        const R* a = Lg + (size_t)j * N;
        const P* b = Th + (size_t)j * N;
        for (int q = 0; q < N; ++q) {
          tr = fmx(a[q], b[q].x, tr);
          ti = fmx(a[q], b[q].y, ti);
        }
      }
      tr = warp_sum(tr);
      ti = warp_sum(ti);
      if (threadIdx.x == 0) {
        s_t.x = tr;
        s_t.y = ti;
      }
    }
    __syncthreads();
    const P t = s_t;
    for (int e = threadIdx.x; e < n * N; e += blockDim.x) {
      const int i = e / N, q = e % N;
      const P th_i = Th[(size_t)(off + i) * N + q];
      // t * Theta[q][i]
      R ar = t.x * th_i.x - t.y * th_i.y, ai = t.x * th_i.y + t.y * th_i.x;
      for (int j = 0; j < n; ++j) {  // - sum_j T[j][i] Theta[q][j]
        const P tji = sT[j * n + i];
        const P thj = Th[(size_t)(off + j) * N + q];
        ar -= tji.x * thj.x - tji.y * thj.y;
        ai -= tji.x * thj.y + tji.y * thj.x;
      }
      sY[e].x += cw * (double)ar;
      sY[e].y += cw * (double)ai;
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < n * N; e += blockDim.x) Yo[e] = sY[e];
}

// out[b][p][q] = Re sum_j trial[j][p] X[b][j][q]   (b = g, or a single h1 block)
__global__ void adj_expand_kernel(const double* __restrict__ trial, const double2* __restrict__ X,
                                  double* __restrict__ out, int N, int nc, int nblocks) {
  const size_t total = (size_t)nblocks * N * N;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int q = e % N;
    const int p = (e / N) % N;
    const size_t b = e / ((size_t)N * N);
    const double2* Xb = X + b * nc * N;
    double s = 0.0;
    for (int j = 0; j < nc; ++j) s = fma(trial[(size_t)j * N + p], Xb[(size_t)j * N + q].x, s);
    out[e] = s;
  }
}

inline int grid_for(size_t n) {
  size_t b = (n + 255) / 256;
  return (int)(b > 152 * 32 ? 152 * 32 : (b == 0 ? 1 : b));
}

}  // namespace

// Theta (walkers' precision) must be in ws.theta and E_L in e_loc; writes
// grad_h1 [N][N] and grad_L [G][N][N].  Scratch: ws.scal (c_w) and yscratch
// (Z, Y: FP64).
template <typename R>
cudaError_t launch_energy_backward(afqmc_ctx* c, int Nw, const double* weight, const double* e_loc, double e0,
                                   double tau, double dJ, double* grad_h1, double* grad_L, double2* yscratch,
                                   cudaStream_t s) {
  typedef typename C2<R>::t P;
  const int N = c->N, nc = c->nc, G = c->G;
  const int ne = c->na + c->nb;
  const double dE = 0.5 * sqrt(ne / tau) + sqrt(ne * tau);
  double* coef = c->ws.scal;  // [Nw]
  adj_coef_kernel<<<1, 256, 0, s>>>(weight, e_loc, coef, Nw, e0, dE, dJ);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  double2* Z = yscratch;                          // [nc][N]
  double2* Y = yscratch + (size_t)nc * N;         // [G][nc][N]
  const P* th = static_cast<const P*>(c->ws.theta);
  adj_z_kernel<R><<<nc, 128, 0, s>>>(th, coef, Z, N, nc, Nw);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int nmax = c->na > c->nb ? c->na : c->nb;
  const size_t shm = (size_t)nmax * N * sizeof(double2) + (size_t)nmax * nmax * sizeof(P);
  if (!capturing(c)) {
    e = raise_smem_limit(adj_y_kernel<R>);
    if (e != cudaSuccess) return e;
  }
  const R* Lh = nullptr;
  if constexpr (std::is_same<R, double>::value) Lh = c->d_Lh;
  else Lh = c->f_Lh;
  adj_y_kernel<R><<<dim3(G, 2), 256, shm, s>>>(th, Lh, coef, Y, N, c->na, c->nb, G, Nw);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  adj_expand_kernel<<<grid_for((size_t)N * N), 256, 0, s>>>(c->d_trial, Z, grad_h1, N, nc, 1);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  adj_expand_kernel<<<grid_for((size_t)G * N * N), 256, 0, s>>>(c->d_trial, Y, grad_L, N, nc, G);
  return cudaGetLastError();
}
template cudaError_t launch_energy_backward<double>(afqmc_ctx*, int, const double*, const double*, double, double,
                                                    double, double*, double*, double2*, cudaStream_t);
template cudaError_t launch_energy_backward<float>(afqmc_ctx*, int, const double*, const double*, double, double,
                                                   double, double*, double*, double2*, cudaStream_t);

}  // namespace afq
