// Per-walker FP64 linear algebra of the walker step:
//  * overlap matrix O = trial^T Psi, LU with partial pivoting, log det O and
//    Theta = Psi O^{-1} (the factor of the mixed density used by the force
//    bias, Eq. force_shift, and the local energy, Eq. eloc);
//  * modified Gram-Schmidt re-orthonormalisation of each determinant;
//  * Arnoldi (one MGS pass) for the Krylov action of e^A (Eqs. krylovsub,
//    projham, krylov) and the small exponential e^{A_k} e_1 (Sec. IV.C).
// Overlaps, log-determinants and the small exponential are FP64 in both
// precisions; the Arnoldi steps and the Gram-Schmidt projections run in the
// walkers' precision.
#include <cuda_bf16.h>
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
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ---------------------------------------------------------------- overlap
// grid (Nw, 2 spins), block 256.  Shared: LU [n][n], O^{-1} [n][n] + [n],
// FP64 complex.  On this GPU an FP64 warp instruction occupies the FP64 pipe
// for its full duration whatever the number of active lanes, so the FP64
// parts are kept few and warp-wide: the LU (FP64), one reciprocal per pivot,
// the log-determinant summed across a warp.  Complex64 walkers get Theta from
// FP32 triangular solves on the rounded LU factors; FP64 walkers from the
// FP64 inverse.
__device__ __forceinline__ cd crecip(cd z) {  // 1/z = conj(z)/|z|^2
  const double r = 1.0 / abs2(z);
  return cd{z.re * r, -z.im * r};
}

template <typename R>
__global__ void __launch_bounds__(256) overlap_kernel(const typename C2<R>::t* __restrict__ psi,
                                                      const double* __restrict__ trial,
                                                      const float* __restrict__ trial_f, int N, int na,
                                                      int nb, typename C2<R>::t* __restrict__ theta,
                                                      double* __restrict__ logdet,
                                                      uint32_t* __restrict__ status,
                                                      const int* __restrict__ skip) {
  extern __shared__ double smem_ov[];
  if (skip && *skip) return;
  const int w = blockIdx.x, spin = blockIdx.y;
  const int n = spin ? nb : na, off = spin ? na : 0, nc = na + nb;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int wid = tid >> 5, lane = tid & 31, nwarp = nt >> 5;
  double* ldw = logdet + (size_t)w * 4 + spin * 2;
  if (n == 0) {
    if (tid == 0) { ldw[0] = 0.0; ldw[1] = 0.0; }
    return;
  }
  cd* LU = reinterpret_cast<cd*>(smem_ov);  // [n][n] row-major
  cd* Inv = LU + n * n;                     // [n][n] (+ [n] reciprocal diagonal)
  __shared__ int perm[128];
  __shared__ int s_piv, s_swaps, s_sing;
  __shared__ cd s_rpk;
  const typename C2<R>::t* P = psi + ((size_t)w * nc + off) * N;

  // O[i][j] = sum_p trial[off+i][p] psi[off+j][p]
  if constexpr (std::is_same<R, float>::value) {
    // complex64 walkers: one warp per entry, lanes stride over p (coalesced),
    // FP32 lane partials and tree; the FP32 entries are widened in one pass
    float2* Of = reinterpret_cast<float2*>(Inv);  // scratch until the solves
    for (int e = wid; e < n * n; e += nwarp) {
      const int i = e / n, j = e % n;
      const float2* X = P + (size_t)j * N;
      const float* T = trial_f + (size_t)(off + i) * N;
      float fr = 0.f, fi = 0.f;
      for (int p = lane; p < N; p += 32) {
        const float2 x = X[p];
        fr = fmaf(T[p], x.x, fr);
        fi = fmaf(T[p], x.y, fi);
      }
      fr = warp_sum(fr);
      fi = warp_sum(fi);
      if (lane == 0) Of[e] = make_float2(fr, fi);
    }
    __syncthreads();
    for (int e = tid; e < n * n; e += nt) LU[e] = mk((double)Of[e].x, (double)Of[e].y);
  } else {
    // FP64: one thread per entry, sequential over p (fewest FP64 operations)
    for (int e = tid; e < n * n; e += nt) {
      const int i = e / n, j = e % n;
      const double* T = trial + (size_t)(off + i) * N;
      const typename C2<R>::t* X = P + (size_t)j * N;
      double sr = 0.0, si = 0.0;
      for (int p = 0; p < N; ++p) {
        const cd x = ld(X + p);
        sr = fma(T[p], x.re, sr);
        si = fma(T[p], x.im, si);
      }
      LU[e] = mk(sr, si);
    }
  }
  if (tid < n) perm[tid] = tid;
  if (tid == 0) { s_swaps = 0; s_sing = 0; }
  __syncthreads();

  // LU with partial pivoting: (P O) = L U, row i of PO is row perm[i] of O
  for (int k = 0; k < n; ++k) {
    if (wid == 0) {  // pivot: largest |LU[i][k]|, i >= k; ties keep the smaller row
      int piv = k;
      double best = -1.0;
      for (int i = k + lane; i < n; i += 32) {
        const double v = abs2(LU[i * n + k]);
        if (v > best) { best = v; piv = i; }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const double ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int op = __shfl_xor_sync(0xffffffffu, piv, o);
        if (ob > best || (ob == best && op < piv)) { best = ob; piv = op; }
      }
      if (lane == 0) {
        s_piv = piv;
        if (!(best > 0.0)) s_sing = 1;
        s_rpk = crecip(LU[piv * n + k]);
        if (piv != k) {
          s_swaps ^= 1;
          int t = perm[k]; perm[k] = perm[piv]; perm[piv] = t;
        }
      }
    }
    __syncthreads();
    const int piv = s_piv;
    if (piv != k)
      for (int j = tid; j < n; j += nt) {
        cd t = LU[k * n + j]; LU[k * n + j] = LU[piv * n + j]; LU[piv * n + j] = t;
      }
    __syncthreads();
    const cd rpk = s_rpk;
    for (int i = k + 1 + tid; i < n; i += nt) LU[i * n + k] = LU[i * n + k] * rpk;
    __syncthreads();
    const int rem = n - k - 1;
    for (int e = tid; e < rem * rem; e += nt) {
      const int i = k + 1 + e / rem, j = k + 1 + e % rem;
      LU[i * n + j] = LU[i * n + j] - LU[i * n + k] * LU[k * n + j];
    }
    __syncthreads();
  }

  // log det = sum_i log U_ii + i pi [odd number of swaps], summed across warp 0
  if (wid == 0) {
    double lr = 0.0, li = 0.0;
    for (int k = lane; k < n; k += 32) {
      const cd u = LU[k * n + k];
      lr += 0.5 * log(abs2(u));
      li += atan2(u.im, u.re);
    }
    lr = warp_sum(lr);
    li = warp_sum(li);
    if (lane == 0) {
      li += s_swaps ? M_PI : 0.0;
      if (s_sing) { lr = CUDART_NAN; li = CUDART_NAN; }
      ldw[0] = lr;
      ldw[1] = li;
      if (s_sing && status) atomicOr(status + w, (uint32_t)AFQMC_W_SINGULAR);
    }
  }
  if (!theta) return;
  typename C2<R>::t* Th = theta + ((size_t)w * nc + off) * N;

  if constexpr (std::is_same<R, float>::value) {
    // Theta row p solves theta_p O = psi_p: with PO = LU, theta_p = u_p P where
    // v U = psi_p (forward over columns of U) and u L = v (backward, unit L).
    float2* Lf = reinterpret_cast<float2*>(Inv);  // rounded factors, [n][n]
    __shared__ float2 s_rdiag[128];
    for (int e = tid; e < n * n; e += nt) Lf[e] = make_float2((float)LU[e].re, (float)LU[e].im);
    for (int i = tid; i < n; i += nt) {
      const cd r = crecip(LU[i * n + i]);
      s_rdiag[i] = make_float2((float)r.re, (float)r.im);
    }
    __syncthreads();
    float vr[80], vi[80];  // n <= 80
    for (int p = tid; p < N; p += nt) {
      for (int j = 0; j < n; ++j) {  // v U = psi_p
        const float2 x = P[(size_t)j * N + p];
        float ar = x.x, ai = x.y;
        for (int i = 0; i < j; ++i) {
          const float2 u = Lf[i * n + j];
          ar -= vr[i] * u.x - vi[i] * u.y;
          ai -= vr[i] * u.y + vi[i] * u.x;
        }
        const float2 d = s_rdiag[j];
        vr[j] = ar * d.x - ai * d.y;
        vi[j] = ar * d.y + ai * d.x;
      }
      for (int i = n - 1; i >= 0; --i) {  // u L = v  (L unit lower: L[k][i], k > i)
        float ar = vr[i], ai = vi[i];
        for (int k = i + 1; k < n; ++k) {
          const float2 l = Lf[k * n + i];
          ar -= vr[k] * l.x - vi[k] * l.y;
          ai -= vr[k] * l.y + vi[k] * l.x;
        }
        vr[i] = ar;
        vi[i] = ai;
      }
      for (int i = 0; i < n; ++i) Th[(size_t)perm[i] * N + p] = make_float2(vr[i], vi[i]);
    }
  } else {
    // O^{-1} column j: L y = P e_j, U x = y.  (P e_j)_i = [perm[i] == j], so y
    // vanishes above row r = perm^{-1}(j); the diagonal of U is inverted once.
    cd* rdiag = Inv + n * n;
    for (int i = tid; i < n; i += nt) rdiag[i] = crecip(LU[i * n + i]);
    __syncthreads();
    for (int j = tid; j < n; j += nt) {
      int r = 0;
      while (r < n - 1 && perm[r] != j) ++r;
      for (int i = 0; i < r; ++i) Inv[i * n + j] = mk(0.0, 0.0);
      Inv[r * n + j] = mk(1.0, 0.0);
      for (int i = r + 1; i < n; ++i) {
        cd y = mk(0.0, 0.0);
        for (int k = r; k < i; ++k) y = y - LU[i * n + k] * Inv[k * n + j];
        Inv[i * n + j] = y;
      }
      for (int i = n - 1; i >= 0; --i) {
        cd x = Inv[i * n + j];
        for (int k = i + 1; k < n; ++k) x = x - LU[i * n + k] * Inv[k * n + j];
        Inv[i * n + j] = x * rdiag[i];
      }
    }
    __syncthreads();
    // Theta[j][p] = sum_i psi[i][p] Oinv[i][j]
    for (int e = tid; e < n * N; e += nt) {
      const int j = e / N, p = e % N;
      cd sacc = mk(0.0, 0.0);
      for (int i = 0; i < n; ++i) sacc = sacc + ld(P + (size_t)i * N + p) * Inv[i * n + j];
      st(Th + (size_t)j * N + p, sacc);
    }
  }
}

// ---------------------------------------------------------------- overlap, complex64 walkers
// grid (Nw, 2 spins), block 256.  The same quantities as overlap_kernel with
// the work laid out for FP32 walkers:
//   O = trial_s^T Psi_s in FP32, p in tiles of 32 staged through shared
//     memory (each thread owns 2 x 5 blocks of O in registers);
//   the LU of O with partial pivoting and log det O in FP64 (rows stay in
//     place; the trailing update of each step runs over the flat range of
//     remaining rows x columns);
//   O^{-1} in FP32 from the rounded factors, one thread per column
//     (P O = L U, so column j of O^{-1} is U^{-1} L^{-1} P e_j);
//   Theta = Psi O^{-1}: threads over (p, block of OV_JB columns j), the
//     rows of O^{-1} read from shared memory (broadcast within a warp), Psi
//     from L1, Theta stored coalesced over p.
// Shared: LU [n][n] FP64 complex, Lf and Inv [n][n] FP32 complex; the O
// staging tiles trial [32][n] and Psi [32][n] occupy the Lf area, which is
// written only after the LU.
// p tile; O register block of OV_TI x OV_TJ entries per thread; Theta column block
constexpr int OV_TP = 32, OV_TI = 2, OV_TJ = 5, OV_JB = 10;
size_t overlap_c64_smem(int nmax) {
  const size_t inv = (size_t)nmax * nmax * 8, stage = (size_t)OV_TP * nmax * 12;
  return (size_t)nmax * nmax * 16 + (inv > stage ? inv : stage);
}

__global__ void __launch_bounds__(256) overlap_c64_kernel(const float2* __restrict__ psi,
                                                          const float* __restrict__ trial_f, int N, int na, int nb,
                                                          float2* __restrict__ theta, double* __restrict__ logdet,
                                                          uint32_t* __restrict__ status, const int* __restrict__ skip) {
  extern __shared__ double smem_oc[];
  if (skip && *skip) return;
  const int w = blockIdx.x, spin = blockIdx.y;
  const int n = spin ? nb : na, off = spin ? na : 0, nc = na + nb;
  const int tid = threadIdx.x, wid = tid >> 5, lane = tid & 31;
  double* ldw = logdet + (size_t)w * 4 + spin * 2;
  if (n == 0) {
    if (tid == 0) { ldw[0] = 0.0; ldw[1] = 0.0; }
    return;
  }
  // shared memory: the FP64 LU [n][n], then one region that holds in turn the
  // O staging tiles, the rounded factors (before they move into the LU area)
  // and O^{-1}
  cd* LU = reinterpret_cast<cd*>(smem_oc);                 // [n][n]
  float2* Lf = reinterpret_cast<float2*>(LU);              // [n][n] rounded factors (after the LU)
  float2* Rg = reinterpret_cast<float2*>(LU + n * n);      // the second region
  float* Ts = reinterpret_cast<float*>(Rg);                // [OV_TP][n] (before the LU)
  float2* Ps = reinterpret_cast<float2*>(Ts + OV_TP * n);  // [OV_TP][n] (before the LU)
  float2* Inv = Rg;                                        // [n][n] O^{-1} (after the factors moved)
  __shared__ int perm[128], rank[128], rem[128];
  __shared__ double cand[128];
  __shared__ cd lik[128];
  __shared__ int s_swaps, s_sing, s_nrem;
  const float2* P = psi + ((size_t)w * nc + off) * N;
  const float* T = trial_f + (size_t)off * N;
  const int nn = n * n;

  // O[i][j] = sum_p T[i][p] P[j][p]: each thread accumulates one block of
  // OV_TI x OV_TJ entries in registers over the staged p tiles (rounds of 256
  // blocks; a single round for n <= 50)
  const int nbi = (n + OV_TI - 1) / OV_TI, nbj = (n + OV_TJ - 1) / OV_TJ, nblocks = nbi * nbj;
  for (int blk0 = 0; blk0 < nblocks; blk0 += 256) {
    const int blk = blk0 + tid;
    const bool has = blk < nblocks;
    const int bi = has ? blk / nbj : 0, bj = has ? blk - bi * nbj : 0;
    const int i0 = bi * OV_TI, j0 = bj * OV_TJ;
    float ar[OV_TI][OV_TJ], ai[OV_TI][OV_TJ];
#pragma unroll
    for (int a0 = 0; a0 < OV_TI; ++a0)
#pragma unroll
      for (int b0 = 0; b0 < OV_TJ; ++b0) { ar[a0][b0] = 0.f; ai[a0][b0] = 0.f; }
    for (int p0 = 0; p0 < N; p0 += OV_TP) {
      __syncthreads();
      for (int e = tid; e < OV_TP * n; e += 256) {  // e = i * OV_TP + pp: consecutive pp are consecutive p
        const int i = e / OV_TP, pp = e - i * OV_TP, p = p0 + pp;
        Ts[pp * n + i] = p < N ? T[(size_t)i * N + p] : 0.f;
        Ps[pp * n + i] = p < N ? P[(size_t)i * N + p] : make_float2(0.f, 0.f);
      }
      __syncthreads();
      if (has) {
#pragma unroll 4
        for (int pp = 0; pp < OV_TP; ++pp) {
          float t[OV_TI];
          float2 x[OV_TJ];
#pragma unroll
          for (int a0 = 0; a0 < OV_TI; ++a0) t[a0] = i0 + a0 < n ? Ts[pp * n + i0 + a0] : 0.f;
#pragma unroll
          for (int b0 = 0; b0 < OV_TJ; ++b0) x[b0] = j0 + b0 < n ? Ps[pp * n + j0 + b0] : make_float2(0.f, 0.f);
#pragma unroll
          for (int a0 = 0; a0 < OV_TI; ++a0)
#pragma unroll
            for (int b0 = 0; b0 < OV_TJ; ++b0) {
              ar[a0][b0] = fmaf(t[a0], x[b0].x, ar[a0][b0]);
              ai[a0][b0] = fmaf(t[a0], x[b0].y, ai[a0][b0]);
            }
        }
      }
    }
    if (has) {
#pragma unroll
      for (int a0 = 0; a0 < OV_TI; ++a0)
#pragma unroll
        for (int b0 = 0; b0 < OV_TJ; ++b0) {
          const int i = i0 + a0, j = j0 + b0;
          if (i < n && j < n) LU[i * n + j] = mk((double)ar[a0][b0], (double)ai[a0][b0]);
        }
    }
  }
  // rank[i]: the step at which row i became the pivot (n: not yet); rem[0..nrem)
  // the rows not chosen yet (in no particular order)
  for (int i = tid; i < n; i += 256) {
    rank[i] = n;
    rem[i] = i;
    cand[i] = abs2(LU[i * n]);
  }
  if (tid == 0) {
    s_sing = 0;
    s_nrem = n;
  }
  __syncthreads();

  // LU with partial pivoting in FP64, rows left in place (implicit pivoting):
  // at step k the pivot is the largest |LU[i][k]| among the rows not chosen
  // yet (ties keep the smaller row; NaN counts as zero, and a zero pivot marks
  // the walker singular); every other remaining row i gets
  // l_ik = LU[i][k] / LU[piv][k] (stored in place of LU[i][k]) and
  // LU[i][j] -= l_ik LU[piv][j] for j > k.  perm[k] = piv, so row k of P O is
  // row perm[k] of O.  Warp 0 picks the pivot from the candidates |LU[i][k]|^2
  // left by the previous update, drops it from the list of remaining rows and
  // forms the multipliers (one per row, lanes over rows); then all threads run
  // the trailing update over the flat range (remaining row, column j > k), so
  // that the FP64 warp instructions run with full warps (the FP64 pipe costs
  // the same for a partly active warp), and leave the candidates of step k + 1.
  for (int k = 0; k < n; ++k) {
    if (wid == 0) {
      const int nr = s_nrem;
      double v = -1.0;
      int row = n, slot = 0;
      for (int r = lane; r < nr; r += 32) {
        const double a2 = cand[r];
        const double vv = a2 >= 0.0 ? a2 : 0.0;  // NaN counts as a zero pivot
        const int i = rem[r];
        if (vv > v || (vv == v && i < row)) { v = vv; row = i; slot = r; }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const double ov = __shfl_xor_sync(0xffffffffu, v, o);
        const int orow = __shfl_xor_sync(0xffffffffu, row, o);
        const int oslot = __shfl_xor_sync(0xffffffffu, slot, o);
        if (ov > v || (ov == v && orow < row)) { v = ov; row = orow; slot = oslot; }
      }
      const int piv = row;
      if (lane == 0) {
        perm[k] = piv;
        rank[piv] = k;
        if (!(v > 0.0)) s_sing = 1;
        rem[slot] = rem[nr - 1];  // drop the pivot from the remaining rows
        s_nrem = nr - 1;
      }
      __syncwarp();
      const cd rpk = crecip(LU[piv * n + k]);
      for (int r = lane; r < nr - 1; r += 32) {
        const int i = rem[r];
        const cd l = LU[i * n + k] * rpk;
        LU[i * n + k] = l;
        lik[r] = l;
      }
    }
    __syncthreads();
    const int nr = s_nrem, cols = n - k - 1;
    if (cols > 0) {
      const cd* up = LU + perm[k] * n + k + 1;
      for (int e = tid; e < nr * cols; e += 256) {
        const int r = e / cols, jj = e - r * cols;
        cd* x = LU + rem[r] * n + k + 1 + jj;
        const cd l = lik[r], u = up[jj];
        cd v = *x;
        v.re = fma(-l.re, u.re, fma(l.im, u.im, v.re));
        v.im = fma(-l.re, u.im, fma(-l.im, u.re, v.im));
        *x = v;
        if (jj == 0) cand[r] = abs2(v);
      }
    }
    __syncthreads();
  }
  // sign of the permutation: parity of n minus its number of cycles
  if (tid == 0) {
    int cycles = 0;
    for (int i = 0; i < n; ++i) {
      if (rank[i] < 0) continue;
      ++cycles;
      for (int j = i; rank[j] >= 0;) {  // follow the cycle through i, marking it
        const int nx = perm[j];
        rank[j] = -1;
        j = nx;
      }
    }
    s_swaps = (n - cycles) & 1;
  }
  __syncthreads();

  // log det = sum_k log U_kk + i pi [odd permutation], summed across warp 0
  if (wid == 0) {
    double lr = 0.0, li = 0.0;
    for (int k = lane; k < n; k += 32) {
      const cd u = LU[perm[k] * n + k];
      lr += 0.5 * log(abs2(u));
      li += atan2(u.im, u.re);
    }
    lr = warp_sum(lr);
    li = warp_sum(li);
    if (lane == 0) {
      li += s_swaps ? M_PI : 0.0;
      if (s_sing) { lr = CUDART_NAN; li = CUDART_NAN; }
      ldw[0] = lr;
      ldw[1] = li;
      if (s_sing && status) atomicOr(status + w, (uint32_t)AFQMC_W_SINGULAR);
    }
  }
  if (!theta) return;

  // O^{-1} = U^{-1} L^{-1} P in FP32 from the rounded factors (the diagonal of U inverted in FP64)
  // factors in pivot order: row k of L and U is physical row perm[k]; the
  // diagonal of U inverted once in FP64
  __shared__ float2 s_rdiag[128];
  for (int e = tid; e < nn; e += 256) {
    const int kr = e / n, j = e - kr * n;
    const cd v = LU[perm[kr] * n + j];
    Rg[e] = make_float2((float)v.re, (float)v.im);
  }
  for (int i = tid; i < n; i += 256) {
    const cd rd = crecip(LU[perm[i] * n + i]);
    s_rdiag[i] = make_float2((float)rd.re, (float)rd.im);
  }
  __syncthreads();
  for (int e = tid; e < nn; e += 256) Lf[e] = Rg[e];  // the FP64 LU is no longer needed
  __syncthreads();
  if (tid < n) {
    const int j = tid;
    int r = 0;
    while (r < n - 1 && perm[r] != j) ++r;
    for (int i = 0; i < r; ++i) Inv[i * n + j] = make_float2(0.f, 0.f);
    Inv[r * n + j] = make_float2(1.f, 0.f);
    for (int i = r + 1; i < n; ++i) {  // L y = P e_j (unit lower L)
      float yr = 0.f, yi = 0.f;
      for (int k = r; k < i; ++k) {
        const float2 l = Lf[i * n + k], y = Inv[k * n + j];
        yr -= l.x * y.x - l.y * y.y;
        yi -= l.x * y.y + l.y * y.x;
      }
      Inv[i * n + j] = make_float2(yr, yi);
    }
    for (int i = n - 1; i >= 0; --i) {  // U x = y
      float2 x = Inv[i * n + j];
      for (int k = i + 1; k < n; ++k) {
        const float2 u = Lf[i * n + k], v = Inv[k * n + j];
        x.x -= u.x * v.x - u.y * v.y;
        x.y -= u.x * v.y + u.y * v.x;
      }
      const float dr = s_rdiag[i].x, di = s_rdiag[i].y;
      Inv[i * n + j] = make_float2(x.x * dr - x.y * di, x.x * di + x.y * dr);
    }
  }
  __syncthreads();

  // Theta[j][p] = sum_i Psi[i][p] O^{-1}[i][j]
  float2* Th = theta + ((size_t)w * nc + off) * N;
  const int nblk = (n + OV_JB - 1) / OV_JB;
  for (int it = tid; it < N * nblk; it += 256) {
    const int jb = it / N, p = it - jb * N, j0 = jb * OV_JB;
    float sr[OV_JB], si[OV_JB];
#pragma unroll
    for (int t = 0; t < OV_JB; ++t) { sr[t] = 0.f; si[t] = 0.f; }
    for (int i = 0; i < n; ++i) {
      const float2 x = P[(size_t)i * N + p];
#pragma unroll
      for (int t = 0; t < OV_JB; ++t) {
        if (j0 + t < n) {
          const float2 v = Inv[i * n + j0 + t];
          sr[t] = fmaf(x.x, v.x, fmaf(-x.y, v.y, sr[t]));
          si[t] = fmaf(x.x, v.y, fmaf(x.y, v.x, si[t]));
        }
      }
    }
#pragma unroll
    for (int t = 0; t < OV_JB; ++t)
      if (j0 + t < n) Th[(size_t)(j0 + t) * N + p] = make_float2(sr[t], si[t]);
  }
}

// ---------------------------------------------------------------- MGS QR
// One warp per determinant (walker w, spin): columns in order, the current
// column in registers (EPL elements per lane), projections and norms reduced
// with warp shuffles in the walkers' precision (the reciprocal norm in FP64).
// Psi = Q R with R_jj = ||q_j|| > 0, so log det(trial^T Q) = log det(trial^T
// Psi) - sum_j log R_jj: the kernel writes sum_j log R_jj (FP64) of
// determinant (w, spin) to logr[w * 4 + 2 * spin].
template <typename R, int EPL>
__global__ void mgs_kernel(typename C2<R>::t* __restrict__ psi, int N, int na, int nb, int Nw,
                           const uint8_t* __restrict__ mask, double* __restrict__ logr) {
  typedef typename C2<R>::t cplx;
  const int det = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (det >= 2 * Nw) return;
  const int w = det >> 1, spin = det & 1;
  if (mask && !mask[w]) return;
  const int n = spin ? nb : na, off = spin ? na : 0, nc = na + nb;
  cplx* P = psi + ((size_t)w * nc + off) * N;
  double lr = 0.0;
  for (int j = 0; j < n; ++j) {
    R qr[EPL], qi[EPL];
#pragma unroll
    for (int e = 0; e < EPL; ++e) {
      const int p = lane + 32 * e;
      qr[e] = R(0);
      qi[e] = R(0);
      if (p < N) {
        const cplx v = P[(size_t)j * N + p];
        qr[e] = v.x;
        qi[e] = v.y;
      }
    }
    for (int i = 0; i < j; ++i) {
      const cplx* Qi = P + (size_t)i * N;
      cplx a[EPL];
      R pr = R(0), pi = R(0);
#pragma unroll
      for (int e = 0; e < EPL; ++e) {
        const int p = lane + 32 * e;
        a[e].x = R(0);
        a[e].y = R(0);
        if (p < N) a[e] = Qi[p];
        pr += a[e].x * qr[e] + a[e].y * qi[e];  // conj(q_i) q_j
        pi += a[e].x * qi[e] - a[e].y * qr[e];
      }
      const R rr = warp_sum(pr), ri = warp_sum(pi);
#pragma unroll
      for (int e = 0; e < EPL; ++e) {
        qr[e] -= rr * a[e].x - ri * a[e].y;
        qi[e] -= rr * a[e].y + ri * a[e].x;
      }
    }
    R ps = R(0);
#pragma unroll
    for (int e = 0; e < EPL; ++e) ps += qr[e] * qr[e] + qi[e] * qi[e];
    const double nrm2 = (double)warp_sum(ps);
    lr += 0.5 * log(nrm2);
    const R inv = (R)(1.0 / sqrt(nrm2));
#pragma unroll
    for (int e = 0; e < EPL; ++e) {
      const int p = lane + 32 * e;
      if (p < N) {
        cplx o;
        o.x = inv * qr[e];
        o.y = inv * qi[e];
        P[(size_t)j * N + p] = o;
      }
    }
    __syncwarp();
  }
  if (logr && lane == 0) logr[(size_t)w * 4 + 2 * spin] = lr;
}

// ---------------------------------------------------------------- Krylov
// One warp per orbital column (walker w, column j); columns are numbered
// col = w * nc + j and all column vectors are contiguous [N].
// Basis vector element p of column col = (w, j) into the split right operand
// of the tensor-core products A V: row j of walker w = [Re v | Im v], the
// second half from column Kh (bf16 hi/lo planes, row length KA = 2 Kh).
struct VPlanes {
  __nv_bfloat16* hi = nullptr;
  __nv_bfloat16* lo = nullptr;
  int NBp = 0, KA = 0, Kh = 0;
};
__device__ __forceinline__ void put_vplanes(const VPlanes& P, int col, int nc, int p, float vr, float vi) {
  const int w = col / nc, j = col - (col / nc) * nc;
  const size_t ra = ((size_t)w * P.NBp + j) * P.KA;
  const __nv_bfloat16 hr = __float2bfloat16(vr), hi = __float2bfloat16(vi);
  const __nv_bfloat16 lr = __float2bfloat16(vr - __bfloat162float(hr)), li = __float2bfloat16(vi - __bfloat162float(hi));
  P.hi[ra + p] = hr;
  P.lo[ra + p] = lr;
  P.hi[ra + P.Kh + p] = hi;
  P.lo[ra + P.Kh + p] = li;
}

// Hessenberg storage: entry (column col, row i, column j) of H_k at
// hess[(i * kmax + j) * hs + col] in the walkers' complex storage type (hs =
// column capacity), so that per-column threads of the small exponential read
// one entry of many columns contiguously.  Complex64 walkers: the inner
// products come from FP32 data and are stored in FP32; the small exponential
// runs in FP64 and its result y is stored back in FP32.

template <typename R>
__global__ void krylov_init_kernel(const typename C2<R>::t* __restrict__ x, typename C2<R>::t* __restrict__ v0,
                                   double* __restrict__ beta, typename C2<R>::t* __restrict__ hess, size_t hs,
                                   int kmax, int N, int ncols, int nc, VPlanes vp) {
  typedef typename C2<R>::t cplx;
  const int col = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (col >= ncols) return;
  // the Hessenberg block starts at zero: entries below the subdiagonal are never written
  for (int e = lane; e < kmax * kmax; e += 32) {
    cplx z;
    z.x = R(0);
    z.y = R(0);
    hess[(size_t)e * hs + col] = z;
  }
  const cplx* X = x + (size_t)col * N;
  R sp = R(0);
  for (int p = lane; p < N; p += 32) {
    const cplx v = X[p];
    sp += v.x * v.x + v.y * v.y;
  }
  const R b = sqrt(warp_sum(sp));
  const R inv = b > R(0) ? R(1) / b : R(0);
  for (int p = lane; p < N; p += 32) {
    cplx v = X[p];
    v.x *= inv;
    v.y *= inv;
    v0[(size_t)col * N + p] = v;
    if (vp.hi) put_vplanes(vp, col, nc, p, (float)v.x, (float)v.y);
  }
  if (lane == 0) beta[col] = (double)b;
}

// Step `it` of Arnoldi: w = A b_it is in `wv`; MGS against b_0..b_it, then the
// next basis vector (or zero after an invariant subspace was found).  One warp
// per column; w lives in registers (EPL elements per lane, N <= 32 * EPL).
// All arithmetic in the walkers' precision.
template <typename R, int EPL>
__global__ void krylov_orth_kernel(const typename C2<R>::t* __restrict__ wv, typename C2<R>::t* __restrict__ basis,
                                   typename C2<R>::t* __restrict__ hess, size_t hs, const double* __restrict__ scal,
                                   int N, int nc, int ncols, int it, int k, int kmax, size_t bstride, VPlanes vp) {
  typedef typename C2<R>::t cplx;
  const int col = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (col >= ncols) return;
  const cplx* W = wv + (size_t)col * N;
  R wr[EPL], wi[EPL];
#pragma unroll
  for (int e = 0; e < EPL; ++e) {
    const int p = lane + 32 * e;
    wr[e] = R(0);
    wi[e] = R(0);
    if (p < N) {
      const cplx v = W[p];
      wr[e] = v.x;
      wi[e] = v.y;
    }
  }
  for (int i = 0; i <= it; ++i) {
    const cplx* V = basis + i * bstride + (size_t)col * N;
    cplx vv[EPL];
    R pr = R(0), pi = R(0);  // lane partial of b_i^H w
#pragma unroll
    for (int e = 0; e < EPL; ++e) {
      const int p = lane + 32 * e;
      vv[e].x = R(0);
      vv[e].y = R(0);
      if (p < N) vv[e] = V[p];
      pr += vv[e].x * wr[e] + vv[e].y * wi[e];
      pi += vv[e].x * wi[e] - vv[e].y * wr[e];
    }
    const R hr = warp_sum(pr), hi = warp_sum(pi);
#pragma unroll
    for (int e = 0; e < EPL; ++e) {
      wr[e] -= hr * vv[e].x - hi * vv[e].y;
      wi[e] -= hr * vv[e].y + hi * vv[e].x;
    }
    if (lane == 0) {
      cplx h;
      h.x = hr;
      h.y = hi;
      hess[(size_t)(i * kmax + it) * hs + col] = h;
    }
  }
  if (it + 1 < k) {
    R ps = R(0);
#pragma unroll
    for (int e = 0; e < EPL; ++e) ps += wr[e] * wr[e] + wi[e] * wi[e];
    R hn = sqrt(warp_sum(ps));
    const R thr = (R)(1e-12 * scal[(size_t)(col / nc) * SC_COUNT + SC_NORMA]);
    const bool brk = !(hn > thr);
    const R inv = brk ? R(0) : R(1) / hn;
    if (brk) hn = R(0);
    cplx* Vn = basis + (it + 1) * bstride + (size_t)col * N;
#pragma unroll
    for (int e = 0; e < EPL; ++e) {
      const int p = lane + 32 * e;
      if (p < N) {
        cplx o;
        o.x = inv * wr[e];
        o.y = inv * wi[e];
        Vn[p] = o;
        if (vp.hi) put_vplanes(vp, col, nc, p, (float)o.x, (float)o.y);
      }
    }
    if (lane == 0) {
      cplx h;
      h.x = hn;
      h.y = R(0);
      hess[(size_t)((it + 1) * kmax + it) * hs + col] = h;
    }
  }
}

// ---------------------------------------------------------------- Lanczos
// Complex-symmetric Lanczos (the field matrix A is complex symmetric): the
// three-term recurrence with the bilinear form u^T v.  The tridiagonal T_k
// is kept in the Hessenberg storage above (diagonal alpha_j, both
// off-diagonals beta_j; the rest stays zero), so the small exponential and
// the combination are those of the Arnoldi action.  One warp per column, the
// arithmetic in the walkers' precision; (psi^T psi)^{1/2} and every beta_j
// is the principal complex square root.

// principal square root of z = x + i y: with r = |z|, t = sqrt((r + |x|) / 2),
// the root is (t, y / 2t) for x >= 0 and (|y| / 2t, +-t) otherwise (the sign
// of y), from (a + i b)^2 = a^2 - b^2 + 2 i a b.  In the walkers' precision:
// FP32 for complex64 walkers (an FP64 instruction occupies the narrow FP64
// pipe for the whole warp, even on one lane), FP64 for complex128 ones.
__device__ __forceinline__ void csqrt_principal(float x, float y, float& a, float& b) {
  const float r = hypotf(x, y);
  if (r == 0.f) { a = 0.f; b = 0.f; return; }
  const float t = sqrtf(0.5f * (r + fabsf(x)));
  if (x >= 0.f) { a = t; b = y / (2.f * t); }
  else { a = fabsf(y) / (2.f * t); b = copysignf(t, y); }
}
__device__ __forceinline__ void csqrt_principal(double x, double y, double& a, double& b) {
  const double r = hypot(x, y);
  if (r == 0.0) { a = 0.0; b = 0.0; return; }
  const double t = sqrt(0.5 * (r + fabs(x)));
  if (x >= 0.0) { a = t; b = y / (2.0 * t); }
  else { a = fabs(y) / (2.0 * t); b = copysign(t, y); }
}

template <typename R>
__global__ void lanczos_init_kernel(const typename C2<R>::t* __restrict__ x, typename C2<R>::t* __restrict__ v0,
                                    double* __restrict__ beta, double2* __restrict__ cbeta,
                                    typename C2<R>::t* __restrict__ hess, size_t hs, int kmax, int N, int ncols,
                                    int nc, VPlanes vp) {
  typedef typename C2<R>::t cplx;
  const int col = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (col >= ncols) return;
  for (int e = lane; e < kmax * kmax; e += 32) {
    cplx z;
    z.x = R(0);
    z.y = R(0);
    hess[(size_t)e * hs + col] = z;
  }
  const cplx* X = x + (size_t)col * N;
  R sr = R(0), si = R(0);  // x^T x
  for (int p = lane; p < N; p += 32) {
    const cplx v = X[p];
    sr += v.x * v.x - v.y * v.y;
    si += R(2) * v.x * v.y;
  }
  R br, bi;
  csqrt_principal(warp_sum(sr), warp_sum(si), br, bi);
  const R m2 = br * br + bi * bi;
  const R ir = m2 > R(0) ? br / m2 : R(0), ii = m2 > R(0) ? -bi / m2 : R(0);
  if (lane == 0) {
    beta[col] = 1.0;
    cbeta[col] = make_double2((double)br, (double)bi);
  }
  for (int p = lane; p < N; p += 32) {
    const cplx v = X[p];
    cplx o;
    o.x = v.x * ir - v.y * ii;
    o.y = v.x * ii + v.y * ir;
    v0[(size_t)col * N + p] = o;
    if (vp.hi) put_vplanes(vp, col, nc, p, (float)o.x, (float)o.y);
  }
}

// Step `it`: w = A v_it is in `wv`; w -= beta_{it-1} v_{it-1};
// alpha_it = v_it^T w; w -= alpha_it v_it; then (it + 1 < k)
// beta_it = (w^T w)^{1/2} and v_{it+1} = w / beta_it, or zero when
// |beta_it| <= 1e-12 ||A||_F (the space is exhausted; the later steps then
// see zero vectors).
template <typename R, int EPL>
__global__ void lanczos_step_kernel(const typename C2<R>::t* __restrict__ wv, typename C2<R>::t* __restrict__ basis,
                                    typename C2<R>::t* __restrict__ hess, size_t hs, const double* __restrict__ scal,
                                    int N, int nc, int ncols, int it, int k, int kmax, size_t bstride, VPlanes vp) {
  typedef typename C2<R>::t cplx;
  const int col = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (col >= ncols) return;
  const cplx* W = wv + (size_t)col * N;
  R wr[EPL], wi[EPL];
#pragma unroll
  for (int e = 0; e < EPL; ++e) {
    const int p = lane + 32 * e;
    wr[e] = R(0);
    wi[e] = R(0);
    if (p < N) {
      const cplx v = W[p];
      wr[e] = v.x;
      wi[e] = v.y;
    }
  }
  if (it > 0) {
    const cplx bp = hess[(size_t)(it * kmax + it - 1) * hs + col];
    const cplx* Vp = basis + (it - 1) * bstride + (size_t)col * N;
#pragma unroll
    for (int e = 0; e < EPL; ++e) {
      const int p = lane + 32 * e;
      if (p < N) {
        const cplx v = Vp[p];
        wr[e] -= bp.x * v.x - bp.y * v.y;
        wi[e] -= bp.x * v.y + bp.y * v.x;
      }
    }
  }
  const cplx* V = basis + it * bstride + (size_t)col * N;
  cplx vv[EPL];
  R pr = R(0), pi = R(0);  // v_it^T w
#pragma unroll
  for (int e = 0; e < EPL; ++e) {
    const int p = lane + 32 * e;
    vv[e].x = R(0);
    vv[e].y = R(0);
    if (p < N) vv[e] = V[p];
    pr += vv[e].x * wr[e] - vv[e].y * wi[e];
    pi += vv[e].x * wi[e] + vv[e].y * wr[e];
  }
  const R ar = warp_sum(pr), ai = warp_sum(pi);
#pragma unroll
  for (int e = 0; e < EPL; ++e) {
    wr[e] -= ar * vv[e].x - ai * vv[e].y;
    wi[e] -= ar * vv[e].y + ai * vv[e].x;
  }
  if (lane == 0) {
    cplx a;
    a.x = ar;
    a.y = ai;
    hess[(size_t)(it * kmax + it) * hs + col] = a;
  }
  if (it + 1 < k) {
    R sr = R(0), si = R(0);  // w^T w
#pragma unroll
    for (int e = 0; e < EPL; ++e) {
      sr += wr[e] * wr[e] - wi[e] * wi[e];
      si += R(2) * wr[e] * wi[e];
    }
    R br, bi;
    csqrt_principal(warp_sum(sr), warp_sum(si), br, bi);
    const R thr = (R)(1e-12 * scal[(size_t)(col / nc) * SC_COUNT + SC_NORMA]);
    const R m2 = br * br + bi * bi;
    const bool brk = !(sqrt(m2) > thr);
    if (brk) {
      br = R(0);
      bi = R(0);
    }
    const R ir = brk ? R(0) : br / m2, ii = brk ? R(0) : -bi / m2;
    cplx* Vn = basis + (it + 1) * bstride + (size_t)col * N;
#pragma unroll
    for (int e = 0; e < EPL; ++e) {
      const int p = lane + 32 * e;
      if (p < N) {
        cplx o;
        o.x = wr[e] * ir - wi[e] * ii;
        o.y = wr[e] * ii + wi[e] * ir;
        Vn[p] = o;
        if (vp.hi) put_vplanes(vp, col, nc, p, (float)o.x, (float)o.y);
      }
    }
    if (lane == 0) {
      cplx h;
      h.x = br;
      h.y = bi;
      hess[(size_t)((it + 1) * kmax + it) * hs + col] = h;
      hess[(size_t)(it * kmax + it + 1) * hs + col] = h;
    }
  }
}

// y = beta e^{H_k} e_1 (beta the real norm of the Arnoldi start, or the
// complex (psi^T psi)^{1/2} of the Lanczos one) in FP64 by sub-stepping: (e^{H/m})^m e_1, each factor
// a Taylor series on the vector summed until its terms fall below a relative
// 1e-10 (complex64 walkers) or 1e-18 (FP64 walkers) of the sum; m chosen so
// that ||H/m||_1 <= 4 (complex64; the partial sums cancel at most e^4 of FP64
// precision) or <= 2 (FP64).  One thread per column: the nonzero (upper
// Hessenberg) entries of its H are staged once in shared memory as FP64, the
// vectors live in registers (k <= KM).  y overwrites column 0 of H.  SM =
// false (large k): H is read from global memory at every use instead.
template <typename R, int KM, bool SM>
__global__ void __launch_bounds__(64) krylov_expm_kernel(typename C2<R>::t* __restrict__ hess, size_t hs,
                                                         const double* __restrict__ beta,
                                                         const double2* __restrict__ cbeta, int ncols, int k,
                                                         int kmax) {
  extern __shared__ double2 hsm[];  // [npk][64]: packed rows i, columns j >= max(i - 1, 0)
  const int t = threadIdx.x;
  const int col = blockIdx.x * 64 + t;
  const bool active = col < ncols;
  // packed offset of row i: row 0 has k entries, row i >= 1 has k - i + 1
  double n1 = 0.0;
  if (active) {
    double cs[KM];
#pragma unroll
    for (int j = 0; j < KM; ++j) cs[j] = 0.0;
    int o = 0;
    for (int i = 0; i < k; ++i) {
      const int j0 = i > 0 ? i - 1 : 0;
      for (int j = j0; j < k; ++j, ++o) {
        const typename C2<R>::t h = hess[(size_t)(i * kmax + j) * hs + col];
        const double2 hd = make_double2((double)h.x, (double)h.y);
        if (SM) hsm[o * 64 + t] = hd;
#pragma unroll
        for (int jj = 0; jj < KM; ++jj)
          if (jj == j) cs[jj] += sqrt(hd.x * hd.x + hd.y * hd.y);
      }
    }
#pragma unroll
    for (int j = 0; j < KM; ++j) n1 = fmax(n1, cs[j]);
  }
  if (!active) return;  // no block-wide synchronisation below: each thread reads only its own entries
  const bool f32 = std::is_same<R, float>::value;
  const double X = f32 ? 4.0 : 2.0;
  int m = 1;
  if (n1 < 1e30) m = (int)ceil(n1 / X);
  if (m < 1) m = 1;
  if (m > 4096) m = 4096;
  const double sc = 1.0 / m;
  const double tol = f32 ? 1e-20 : 1e-36;  // on squared norms
  cd v[KM], tv[KM], u[KM];
#pragma unroll
  for (int i = 0; i < KM; ++i) v[i] = mk(i == 0 ? 1.0 : 0.0, 0.0);
  for (int s = 0; s < m; ++s) {
#pragma unroll
    for (int i = 0; i < KM; ++i) tv[i] = v[i];
    for (int d = 1; d <= 60; ++d) {
      const double f = sc / d;
      int o = 0;
#pragma unroll
      for (int i = 0; i < KM; ++i) {
        cd a = mk(0.0, 0.0);
        if (i < k) {
#pragma unroll
          for (int j = (i > 0 ? i - 1 : 0); j < KM; ++j) {
            if (j < k) {
              double2 h;
              if (SM) {
                h = hsm[(o + j - (i > 0 ? i - 1 : 0)) * 64 + t];
              } else {
                const typename C2<R>::t hh = hess[(size_t)(i * kmax + j) * hs + col];
                h = make_double2((double)hh.x, (double)hh.y);
              }
              a.re = fma(h.x, tv[j].re, fma(-h.y, tv[j].im, a.re));  // a += h tv[j], four FMAs
              a.im = fma(h.x, tv[j].im, fma(h.y, tv[j].re, a.im));
            }
          }
          o += k - (i > 0 ? i - 1 : 0);
        }
        u[i] = f * a;
      }
      double tn = 0.0, an = 0.0;
#pragma unroll
      for (int i = 0; i < KM; ++i) {
        if (i < k) {
          tv[i] = u[i];
          v[i] = v[i] + u[i];
          tn += abs2(u[i]);
          an += abs2(v[i]);
        }
      }
      if (tn <= tol * an) break;
    }
  }
  const cd b = cbeta ? ld(cbeta + col) : mk(beta[col], 0.0);
#pragma unroll
  for (int i = 0; i < KM; ++i)
    if (i < k) {
      const cd yv = b * v[i];
      typename C2<R>::t y;
      y.x = (R)yv.re;
      y.y = (R)yv.im;
      hess[(size_t)(i * kmax) * hs + col] = y;
    }
}

// The same y = beta e^{T_k} e_1 for the symmetric tridiagonal T_k of the
// Lanczos action (diagonal alpha_i at (i, i), off-diagonal beta_i at
// (i + 1, i) = (i, i + 1)): three entries per row instead of the Hessenberg
// row, held in registers; sub-steps, stopping rule and FP64 arithmetic as
// above (the 1-norm of T_k is its infinity-norm).
template <typename R, int KM>
__global__ void __launch_bounds__(64) lanczos_expm_kernel(typename C2<R>::t* __restrict__ hess, size_t hs,
                                                          const double2* __restrict__ cbeta, int ncols, int k,
                                                          int kmax) {
  const int col = blockIdx.x * 64 + threadIdx.x;
  if (col >= ncols) return;
  cd a[KM], b[KM];  // b[i] couples i and i + 1
  double n1 = 0.0;
#pragma unroll
  for (int i = 0; i < KM; ++i) {
    a[i] = mk(0.0, 0.0);
    b[i] = mk(0.0, 0.0);
    if (i < k) {
      a[i] = ld(hess + (size_t)(i * kmax + i) * hs + col);
      if (i + 1 < k) b[i] = ld(hess + (size_t)((i + 1) * kmax + i) * hs + col);
    }
  }
#pragma unroll
  for (int i = 0; i < KM; ++i) {
    double r = sqrt(abs2(a[i])) + sqrt(abs2(b[i]));
    if (i > 0) r += sqrt(abs2(b[i - 1]));
    n1 = fmax(n1, r);
  }
  const bool f32 = std::is_same<R, float>::value;
  const double X = f32 ? 4.0 : 2.0;
  int m = 1;
  if (n1 < 1e30) m = (int)ceil(n1 / X);
  if (m < 1) m = 1;
  if (m > 4096) m = 4096;
  const double sc = 1.0 / m;
  const double tol = f32 ? 1e-20 : 1e-36;  // on squared norms
  cd v[KM], tv[KM], u[KM];
#pragma unroll
  for (int i = 0; i < KM; ++i) v[i] = mk(i == 0 ? 1.0 : 0.0, 0.0);
  for (int s = 0; s < m; ++s) {
#pragma unroll
    for (int i = 0; i < KM; ++i) tv[i] = v[i];
    for (int d = 1; d <= 60; ++d) {
      const double f = sc / d;
#pragma unroll
      for (int i = 0; i < KM; ++i) {
        cd t = a[i] * tv[i];
        if (i + 1 < KM) t = t + b[i] * tv[i + 1];
        if (i > 0) t = t + b[i - 1] * tv[i - 1];
        u[i] = f * t;
      }
      double tn = 0.0, an = 0.0;
#pragma unroll
      for (int i = 0; i < KM; ++i) {
        tv[i] = u[i];
        v[i] = v[i] + u[i];
        tn += abs2(u[i]);
        an += abs2(v[i]);
      }
      if (tn <= tol * an) break;
    }
  }
  const cd bb = ld(cbeta + col);
#pragma unroll
  for (int i = 0; i < KM; ++i)
    if (i < k) {
      const cd yv = bb * v[i];
      typename C2<R>::t y;
      y.x = (R)yv.re;
      y.y = (R)yv.im;
      hess[(size_t)(i * kmax) * hs + col] = y;
    }
}

// psi_out = B_k y: out = sum_i y_i b_i in the walkers' precision (y from column 0 of H)
template <typename R>
__global__ void krylov_combine_kernel(const typename C2<R>::t* __restrict__ hess, size_t hs,
                                      const typename C2<R>::t* __restrict__ basis, typename C2<R>::t* __restrict__ out,
                                      int N, int ncols, int k, int kmax, size_t bstride) {
  typedef typename C2<R>::t cplx;
  const int col = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (col >= ncols) return;
  for (int p = lane; p < N; p += 32) {
    R sr = R(0), si = R(0);
    for (int i = 0; i < k; ++i) {
      const cplx y = hess[(size_t)(i * kmax) * hs + col];
      const cplx v = basis[i * bstride + (size_t)col * N + p];
      sr += y.x * v.x - y.y * v.y;
      si += y.x * v.y + y.y * v.x;
    }
    cplx o;
    o.x = sr;
    o.y = si;
    out[(size_t)col * N + p] = o;
  }
}

// Crank-Nicolson solve (Sec. III.D), one walker per block: M = I - X/2 is
// formed in place of X (row-major [N][N]), Gaussian elimination with partial
// pivoting (the first row of largest |M_ik| is the pivot) runs on M and on the
// nc right-hand sides Y [nc][N] together, then back substitution leaves
// Y = (I - X/2)^{-1} Y.  FP64 arithmetic; M and Y keep the walkers' precision
// in memory.  A zero pivot gives non-finite entries, which the weight update
// turns into a dead walker.
template <typename R>
__global__ void __launch_bounds__(256) cn_solve_kernel(typename C2<R>::t* Xall, typename C2<R>::t* Yall, int N, int nc,
                                                       size_t per) {
  typedef typename C2<R>::t cplx;
  __shared__ double s_val[256];
  __shared__ int s_idx[256];
  const int tid = threadIdx.x;
  const size_t NN = (size_t)N * N;
  cplx* M = Xall + blockIdx.x * NN;
  cplx* Y = Yall + blockIdx.x * per;
  for (size_t e = tid; e < NN; e += 256) {
    const cd x = ld(M + e);
    st(M + e, mk((e / N == e % N ? 1.0 : 0.0) - 0.5 * x.re, -0.5 * x.im));
  }
  __syncthreads();
  for (int k = 0; k < N; ++k) {
    double best = -1.0;
    int bi = k;
    for (int i = k + tid; i < N; i += 256) {
      const double a = abs2(ld(M + (size_t)i * N + k));
      if (a > best) {
        best = a;
        bi = i;
      }
    }
    s_val[tid] = best;
    s_idx[tid] = bi;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
      if (tid < o) {
        const double v2 = s_val[tid + o];
        const int i2 = s_idx[tid + o];
        if (v2 > s_val[tid] || (v2 == s_val[tid] && i2 < s_idx[tid])) {
          s_val[tid] = v2;
          s_idx[tid] = i2;
        }
      }
      __syncthreads();
    }
    const int piv = s_idx[0];  // rewritten only after the syncs of this k's later phases
    if (piv != k) {
      for (int q = k + tid; q < N; q += 256) {
        const cplx a = M[(size_t)k * N + q];
        M[(size_t)k * N + q] = M[(size_t)piv * N + q];
        M[(size_t)piv * N + q] = a;
      }
      for (int j = tid; j < nc; j += 256) {
        const cplx a = Y[(size_t)j * N + k];
        Y[(size_t)j * N + k] = Y[(size_t)j * N + piv];
        Y[(size_t)j * N + piv] = a;
      }
    }
    __syncthreads();
    const cd d = ld(M + (size_t)k * N + k);
    for (int i = k + 1 + tid; i < N; i += 256) st(M + (size_t)i * N + k, cdiv(ld(M + (size_t)i * N + k), d));
    __syncthreads();
    const int r = N - k - 1;
    const size_t nup = (size_t)r * r, nyu = (size_t)nc * r;
    for (size_t e = tid; e < nup; e += 256) {
      const size_t i = k + 1 + e / r, q = k + 1 + e % r;
      st(M + i * N + q, ld(M + i * N + q) - ld(M + i * N + k) * ld(M + (size_t)k * N + q));
    }
    for (size_t e = tid; e < nyu; e += 256) {
      const size_t j = e / r, i = k + 1 + e % r;
      st(Y + j * N + i, ld(Y + j * N + i) - ld(M + i * N + k) * ld(Y + j * N + k));
    }
    __syncthreads();
  }
  for (int k = N - 1; k >= 0; --k) {
    const cd d = ld(M + (size_t)k * N + k);
    for (int j = tid; j < nc; j += 256) st(Y + (size_t)j * N + k, cdiv(ld(Y + (size_t)j * N + k), d));
    __syncthreads();
    const size_t nb = (size_t)nc * k;
    for (size_t e = tid; e < nb; e += 256) {
      const size_t j = e / k, i = e % k;
      st(Y + j * N + i, ld(Y + j * N + i) - ld(M + i * N + k) * ld(Y + j * N + k));
    }
    __syncthreads();
  }
}

template <typename R>
__global__ void init_walkers_kernel(typename C2<R>::t* __restrict__ psi, const double* __restrict__ trial,
                                    double* __restrict__ weight, uint32_t* __restrict__ status, int N, int nc,
                                    int Nw) {
  const size_t per = (size_t)nc * N;
  const size_t total = per * Nw;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    st(psi + e, mk(trial[e % per], 0.0));
    if (e % per == 0) {
      const size_t w = e / per;
      weight[w] = 1.0;
      status[w] = 0u;
    }
  }
}

}  // namespace

template <typename R>
cudaError_t launch_overlap(const afqmc_ctx* c, int Nw, const void* psi, void* theta, double* logdet,
                           uint32_t* status, cudaStream_t s, const int* skip) {
  const int nmax = c->na > c->nb ? c->na : c->nb;
  if constexpr (std::is_same<R, float>::value) {
    const size_t shc = overlap_c64_smem(nmax);
    if (shc <= (size_t)max_dyn_smem()) {
      if (!capturing(c)) {
        cudaError_t e = raise_smem_limit(overlap_c64_kernel);
        if (e != cudaSuccess) return e;
      }
      overlap_c64_kernel<<<dim3(Nw, 2), 256, shc, s>>>(static_cast<const float2*>(psi), c->f_trial, c->N, c->na,
                                                       c->nb, static_cast<float2*>(theta), logdet, status, skip);
      return cudaGetLastError();
    }
  }
  const size_t shm = (size_t)(2 * nmax * nmax + nmax) * sizeof(cd);
  if (!capturing(c)) {
    cudaError_t e = raise_smem_limit(overlap_kernel<R>);
    if (e != cudaSuccess) return e;
  }
  overlap_kernel<R><<<dim3(Nw, 2), 256, shm, s>>>(static_cast<const typename C2<R>::t*>(psi), c->d_trial,
                                                  c->f_trial, c->N,
                                                  c->na, c->nb, static_cast<typename C2<R>::t*>(theta), logdet,
                                                  status, skip);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_mgs(const afqmc_ctx* c, int Nw, void* psi, const uint8_t* mask, double* logr, cudaStream_t s) {
  const int dets = 2 * Nw;
  typename C2<R>::t* P = static_cast<typename C2<R>::t*>(psi);
  const dim3 grid((dets + 7) / 8);
  if (c->N <= 128)
    mgs_kernel<R, 4><<<grid, 256, 0, s>>>(P, c->N, c->na, c->nb, Nw, mask, logr);
  else if (c->N <= 256)
    mgs_kernel<R, 8><<<grid, 256, 0, s>>>(P, c->N, c->na, c->nb, Nw, mask, logr);
  else if (c->N <= 320)
    mgs_kernel<R, 10><<<grid, 256, 0, s>>>(P, c->N, c->na, c->nb, Nw, mask, logr);
  else
    mgs_kernel<R, 16><<<grid, 256, 0, s>>>(P, c->N, c->na, c->nb, Nw, mask, logr);
  return cudaGetLastError();
}

// complex64 walkers with the tensor-core products A V: the Arnoldi kernels
// also write each new basis vector into the split right operand
template <typename R>
VPlanes vplanes(const afqmc_ctx* c) {
  VPlanes v;
  if (std::is_same<R, float>::value && c->tg.av_ok) {
    v.hi = static_cast<__nv_bfloat16*>(c->tg.v_hi);
    v.lo = static_cast<__nv_bfloat16*>(c->tg.v_lo);
    v.NBp = c->tg.NBp;
    v.KA = c->tg.KA;
    v.Kh = c->tg.Kh;
  }
  return v;
}

template <typename R>
cudaError_t launch_krylov_init(const afqmc_ctx* c, int Nw, cudaStream_t s) {
  const int ncols = Nw * c->nc;
  const size_t hs = (size_t)c->ws.n_walkers * c->nc;
  krylov_init_kernel<R><<<(ncols + 7) / 8, 256, 0, s>>>(
      static_cast<const typename C2<R>::t*>(c->ws.psi_b), static_cast<typename C2<R>::t*>(c->ws.basis),
      c->ws.beta, reinterpret_cast<typename C2<R>::t*>(c->ws.hess), hs, c->ws.kmax, c->N, ncols, c->nc,
      vplanes<R>(c));
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_krylov_orth(const afqmc_ctx* c, int Nw, int it, int k, cudaStream_t s, const void* wv) {
  const int ncols = Nw * c->nc;
  const size_t bstride = (size_t)c->ws.n_walkers * c->nc * c->N;
  const size_t hs = (size_t)c->ws.n_walkers * c->nc;
  const typename C2<R>::t* W = static_cast<const typename C2<R>::t*>(wv ? wv : c->ws.term0);
  typename C2<R>::t* Bs = static_cast<typename C2<R>::t*>(c->ws.basis);
  typename C2<R>::t* H = reinterpret_cast<typename C2<R>::t*>(c->ws.hess);
  const dim3 grid((ncols + 7) / 8);
  const VPlanes vp = vplanes<R>(c);
  if (c->N <= 128)
    krylov_orth_kernel<R, 4><<<grid, 256, 0, s>>>(W, Bs, H, hs, c->ws.scal, c->N, c->nc, ncols, it, k, c->ws.kmax,
                                                  bstride, vp);
  else if (c->N <= 256)
    krylov_orth_kernel<R, 8><<<grid, 256, 0, s>>>(W, Bs, H, hs, c->ws.scal, c->N, c->nc, ncols, it, k, c->ws.kmax,
                                                  bstride, vp);
  else if (c->N <= 320)  // 10 elements per lane: fewer registers, more warps in flight than 16
    krylov_orth_kernel<R, 10><<<grid, 256, 0, s>>>(W, Bs, H, hs, c->ws.scal, c->N, c->nc, ncols, it, k, c->ws.kmax,
                                                   bstride, vp);
  else
    krylov_orth_kernel<R, 16><<<grid, 256, 0, s>>>(W, Bs, H, hs, c->ws.scal, c->N, c->nc, ncols, it, k,
                                                   c->ws.kmax, bstride, vp);
  return cudaGetLastError();
}

// packed upper-Hessenberg entries of a k x k matrix
inline int hess_packed(int k) { return k + k * (k + 1) / 2 - 1; }

template <typename R>
cudaError_t launch_lanczos_init(const afqmc_ctx* c, int Nw, cudaStream_t s) {
  const int ncols = Nw * c->nc;
  const size_t hs = (size_t)c->ws.n_walkers * c->nc;
  lanczos_init_kernel<R><<<(ncols + 7) / 8, 256, 0, s>>>(
      static_cast<const typename C2<R>::t*>(c->ws.psi_b), static_cast<typename C2<R>::t*>(c->ws.basis),
      c->ws.beta, c->ws.cbeta, reinterpret_cast<typename C2<R>::t*>(c->ws.hess), hs, c->ws.kmax, c->N, ncols, c->nc,
      vplanes<R>(c));
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_lanczos_step(const afqmc_ctx* c, int Nw, int it, int k, cudaStream_t s, const void* wv) {
  const int ncols = Nw * c->nc;
  const size_t bstride = (size_t)c->ws.n_walkers * c->nc * c->N;
  const size_t hs = (size_t)c->ws.n_walkers * c->nc;
  const typename C2<R>::t* W = static_cast<const typename C2<R>::t*>(wv ? wv : c->ws.term0);
  typename C2<R>::t* Bs = static_cast<typename C2<R>::t*>(c->ws.basis);
  typename C2<R>::t* H = reinterpret_cast<typename C2<R>::t*>(c->ws.hess);
  const dim3 grid((ncols + 7) / 8);
  const VPlanes vp = vplanes<R>(c);
  if (c->N <= 128)
    lanczos_step_kernel<R, 4><<<grid, 256, 0, s>>>(W, Bs, H, hs, c->ws.scal, c->N, c->nc, ncols, it, k, c->ws.kmax,
                                                   bstride, vp);
  else if (c->N <= 256)
    lanczos_step_kernel<R, 8><<<grid, 256, 0, s>>>(W, Bs, H, hs, c->ws.scal, c->N, c->nc, ncols, it, k, c->ws.kmax,
                                                   bstride, vp);
  else if (c->N <= 320)
    lanczos_step_kernel<R, 10><<<grid, 256, 0, s>>>(W, Bs, H, hs, c->ws.scal, c->N, c->nc, ncols, it, k,
                                                    c->ws.kmax, bstride, vp);
  else
    lanczos_step_kernel<R, 16><<<grid, 256, 0, s>>>(W, Bs, H, hs, c->ws.scal, c->N, c->nc, ncols, it, k,
                                                    c->ws.kmax, bstride, vp);
  return cudaGetLastError();
}

template <typename R, int KM>
cudaError_t expm_launch(const afqmc_ctx* c, int ncols, int k, cudaStream_t s, const double2* cbeta) {
  typename C2<R>::t* H = reinterpret_cast<typename C2<R>::t*>(c->ws.hess);
  const size_t hs = (size_t)c->ws.n_walkers * c->nc;
  const size_t shm = (size_t)hess_packed(k) * 64 * sizeof(double2);
  const dim3 grid((ncols + 63) / 64);
  if (shm <= (size_t)max_dyn_smem()) {
    if (!capturing(c)) {
      cudaError_t e = raise_smem_limit(krylov_expm_kernel<R, KM, true>);
      if (e != cudaSuccess) return e;
    }
    krylov_expm_kernel<R, KM, true><<<grid, 64, shm, s>>>(H, hs, c->ws.beta, cbeta, ncols, k, c->ws.kmax);
  } else {
    krylov_expm_kernel<R, KM, false><<<grid, 64, 0, s>>>(H, hs, c->ws.beta, cbeta, ncols, k, c->ws.kmax);
  }
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_krylov_finish(const afqmc_ctx* c, int Nw, int k, cudaStream_t s, bool lanczos) {
  const int ncols = Nw * c->nc;
  const size_t bstride = (size_t)c->ws.n_walkers * c->nc * c->N;
  const size_t hs = (size_t)c->ws.n_walkers * c->nc;
  cudaError_t e = cudaSuccess;
  if (lanczos) {
    typename C2<R>::t* H = reinterpret_cast<typename C2<R>::t*>(c->ws.hess);
    const dim3 grid((ncols + 63) / 64);
    if (k <= 8)
      lanczos_expm_kernel<R, 8><<<grid, 64, 0, s>>>(H, hs, c->ws.cbeta, ncols, k, c->ws.kmax);
    else if (k <= 12)
      lanczos_expm_kernel<R, 12><<<grid, 64, 0, s>>>(H, hs, c->ws.cbeta, ncols, k, c->ws.kmax);
    else if (k <= 16)
      lanczos_expm_kernel<R, 16><<<grid, 64, 0, s>>>(H, hs, c->ws.cbeta, ncols, k, c->ws.kmax);
    else
      lanczos_expm_kernel<R, 32><<<grid, 64, 0, s>>>(H, hs, c->ws.cbeta, ncols, k, c->ws.kmax);
    e = cudaGetLastError();
  } else {
    e = k <= 8 ? expm_launch<R, 8>(c, ncols, k, s, nullptr)
        : k <= 12 ? expm_launch<R, 12>(c, ncols, k, s, nullptr)
        : k <= 16 ? expm_launch<R, 16>(c, ncols, k, s, nullptr)
                  : expm_launch<R, 32>(c, ncols, k, s, nullptr);
  }
  if (e != cudaSuccess) return e;
  krylov_combine_kernel<R><<<(ncols + 7) / 8, 256, 0, s>>>(
      reinterpret_cast<const typename C2<R>::t*>(c->ws.hess), hs,
      static_cast<const typename C2<R>::t*>(c->ws.basis), static_cast<typename C2<R>::t*>(c->ws.acc), c->N, ncols, k,
      c->ws.kmax, bstride);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_init_walkers(const afqmc_ctx* c, const afqmc_walkers* w, cudaStream_t s) {
  const size_t total = (size_t)w->n_walkers * c->nc * c->N;
  int blocks = (int)((total + 255) / 256);
  if (blocks > 152 * 32) blocks = 152 * 32;
  init_walkers_kernel<R><<<blocks, 256, 0, s>>>(static_cast<typename C2<R>::t*>(w->psi), c->d_trial, w->weight,
                                                w->status, c->N, c->nc, w->n_walkers);
  return cudaGetLastError();
}

template <typename R>
cudaError_t prepare_overlap(const afqmc_ctx*) {
  cudaError_t e = raise_smem_limit(overlap_kernel<R>);
  if (e == cudaSuccess && std::is_same<R, float>::value) e = raise_smem_limit(overlap_c64_kernel);
  if (e == cudaSuccess) e = raise_smem_limit(krylov_expm_kernel<R, 8, true>);
  if (e == cudaSuccess) e = raise_smem_limit(krylov_expm_kernel<R, 12, true>);
  if (e == cudaSuccess) e = raise_smem_limit(krylov_expm_kernel<R, 16, true>);
  if (e == cudaSuccess) e = raise_smem_limit(krylov_expm_kernel<R, 32, true>);
  return e;
}
template cudaError_t prepare_overlap<double>(const afqmc_ctx*);
template cudaError_t prepare_overlap<float>(const afqmc_ctx*);

template <typename R>
cudaError_t launch_cn_solve(const afqmc_ctx* c, int Nw, void* X, void* Y, cudaStream_t s) {
  if (Nw <= 0) return cudaSuccess;
  typedef typename C2<R>::t C;
  cn_solve_kernel<R><<<Nw, 256, 0, s>>>(static_cast<C*>(X), static_cast<C*>(Y), c->N, c->nc, (size_t)c->nc * c->N);
  return cudaGetLastError();
}

#define AFQ_INST(R)                                                                                       \
  template cudaError_t launch_cn_solve<R>(const afqmc_ctx*, int, void*, void*, cudaStream_t);               \
  template cudaError_t launch_overlap<R>(const afqmc_ctx*, int, const void*, void*, double*, uint32_t*,   \
                                         cudaStream_t, const int*);                                        \
  template cudaError_t launch_mgs<R>(const afqmc_ctx*, int, void*, const uint8_t*, double*, cudaStream_t);  \
  template cudaError_t launch_krylov_init<R>(const afqmc_ctx*, int, cudaStream_t);                         \
  template cudaError_t launch_krylov_orth<R>(const afqmc_ctx*, int, int, int, cudaStream_t, const void*);  \
  template cudaError_t launch_krylov_finish<R>(const afqmc_ctx*, int, int, cudaStream_t, bool);                \
  template cudaError_t launch_lanczos_init<R>(const afqmc_ctx*, int, cudaStream_t);                               \
  template cudaError_t launch_lanczos_step<R>(const afqmc_ctx*, int, int, int, cudaStream_t, const void*);      \
  template cudaError_t launch_init_walkers<R>(const afqmc_ctx*, const afqmc_walkers*, cudaStream_t);
AFQ_INST(double)
AFQ_INST(float)

}  // namespace afq
