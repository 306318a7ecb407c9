// Tiled SIMT GEMM with a real or complex A and a complex B, used for the
// walker-batched contractions of the step: the force-bias contraction
// sum_{jq} Lh_g,jq Theta_jq (Eq. force_shift), the field assembly
// sum_g c_g L_g (Eq. heffTOT), the half step B Psi (Sec. III.B) and the
// per-walker products A Psi of the Taylor and Krylov actions (Sec. IV).
//
// C[b][m][n] = alpha * sum_k A[b][m][k] B[b][n][k], strides in elements.
// Output tile BM x BN (four variants: 64x64, 128x32, 32x128, 64x32, chosen per
// call site by the autotuner; a fifth, per-walker kernel for the products A*V), K slab of 8 staged in shared memory, 256
// threads with a (BM/16) x (BN/16) register tile each.  The thread-to-output
// map follows the unit stride of C so that the stores coalesce.
#include "internal.cuh"

namespace afq {

namespace {

constexpr int BK = 8, NT = 256;

template <typename R, bool ACPLX, int BM, int BN>
__global__ void __launch_bounds__(NT) gemm_kernel(GemmArgs g) {
  constexpr int TM = BM / 16, TN = BN / 16;
  typedef typename C2<R>::t cplx;
  __shared__ R sAr[BK][BM];
  __shared__ R sAi[ACPLX ? BK : 1][ACPLX ? BM : 1];
  __shared__ R sBr[BK][BN];
  __shared__ R sBi[BK][BN];
  if (g.skip && *g.skip) return;

  const bool split = g.splitk > 1;
  const int b = split ? 0 : blockIdx.z;
  const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
  // K range of this block (the whole K unless split)
  const int kchunk = split ? (((g.K + g.splitk - 1) / g.splitk + BK - 1) / BK) * BK : g.K;
  const int kbeg = split ? blockIdx.z * kchunk : 0;
  const int kend = split ? min(g.K, kbeg + kchunk) : g.K;
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const bool swap = (g.sc_m == 1);  // C contiguous along m: threads run along m
  const int tm = swap ? tx : ty, tn = swap ? ty : tx;

  // batch offset in elements of A's own type (a complex element is two reals)
  const R* A = static_cast<const R*>(g.A) + (long long)b * g.sa_b * (ACPLX ? 2 : 1);
  const cplx* Bp = static_cast<const cplx*>(g.B) + (long long)b * g.sb_b;
  const bool a_kc = (g.sa_k == 1);
  const bool b_kc = (g.sb_k == 1);

  R accr[TM][TN], acci[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) accr[i][j] = acci[i][j] = R(0);

  for (int k0 = kbeg; k0 < kend; k0 += BK) {
    for (int l = tid; l < BM * BK; l += NT) {
      int mm, kk;
      if (a_kc) { kk = l % BK; mm = l / BK; } else { mm = l % BM; kk = l / BM; }
      const int m = m0 + mm, k = k0 + kk;
      R vr = R(0), vi = R(0);
      if (m < g.M && k < kend) {
        const long long off = (long long)m * g.sa_m + (long long)k * g.sa_k;
        if (ACPLX) {
          cplx v = reinterpret_cast<const cplx*>(A)[off];
          vr = v.x; vi = v.y;
        } else {
          vr = A[off];
        }
      }
      sAr[kk][mm] = vr;
      if (ACPLX) sAi[kk][mm] = vi;
    }
    for (int l = tid; l < BN * BK; l += NT) {
      int nn, kk;
      if (b_kc) { kk = l % BK; nn = l / BK; } else { nn = l % BN; kk = l / BN; }
      const int n = n0 + nn, k = k0 + kk;
      cplx v;
      v.x = R(0); v.y = R(0);
      if (n < g.Nn && k < kend) v = Bp[(long long)n * g.sb_n + (long long)k * g.sb_k];
      sBr[kk][nn] = v.x;
      sBi[kk][nn] = v.y;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      R ar[TM], ai[TM], br[TN], bi[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) {
        ar[i] = sAr[kk][tm + 16 * i];
        ai[i] = ACPLX ? sAi[kk][tm + 16 * i] : R(0);
      }
#pragma unroll
      for (int j = 0; j < TN; ++j) {
        br[j] = sBr[kk][tn + 16 * j];
        bi[j] = sBi[kk][tn + 16 * j];
      }
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) {
          accr[i][j] = fma(ar[i], br[j], accr[i][j]);
          acci[i][j] = fma(ar[i], bi[j], acci[i][j]);
          if (ACPLX) {
            accr[i][j] = fma(-ai[i], bi[j], accr[i][j]);
            acci[i][j] = fma(ai[i], br[j], acci[i][j]);
          }
        }
    }
    __syncthreads();
  }

  if (split) {  // partial tile, no scaling
    cplx* Pp = static_cast<cplx*>(g.part) + (size_t)blockIdx.z * g.M * g.Nn;
#pragma unroll
    for (int i = 0; i < TM; ++i) {
      const int m = m0 + tm + 16 * i;
      if (m >= g.M) continue;
#pragma unroll
      for (int j = 0; j < TN; ++j) {
        const int n = n0 + tn + 16 * j;
        if (n >= g.Nn) continue;
        cplx v;
        v.x = accr[i][j];
        v.y = acci[i][j];
        Pp[(size_t)m * g.Nn + n] = v;
      }
    }
    return;
  }
  cplx* C = static_cast<cplx*>(g.C) + (long long)b * g.sc_b;
  cplx* D = g.D ? static_cast<cplx*>(g.D) + (long long)b * g.sc_b : nullptr;
  const R alr = (R)g.alpha_re, ali = (R)g.alpha_im;
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    const int m = m0 + tm + 16 * i;
    if (m >= g.M) continue;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int n = n0 + tn + 16 * j;
      if (n >= g.Nn) continue;
      cplx v;
      v.x = alr * accr[i][j] - ali * acci[i][j];
      v.y = alr * acci[i][j] + ali * accr[i][j];
      const long long off = (long long)m * g.sc_m + (long long)n * g.sc_n;
      if (g.accum) {
        cplx o = C[off];
        o.x += v.x;
        o.y += v.y;
        C[off] = o;
      } else {
        C[off] = v;
      }
      if (D) {
        cplx d = D[off];
        d.x += v.x;
        d.y += v.y;
        D[off] = d;
      }
    }
  }
}

// Per-walker product C[w][j][p] = alpha sum_q A[w][p][q] X[w][j][q] (complex A,
// X, C; D += C when given): one block per (64-row tile of p, walker), all nc
// columns of the walker in registers (JT per thread), K staged in slabs of 32.
// The per-element FMA sequence equals gemm_kernel's, so results agree bit for bit.
constexpr int WM_BM = 64;
template <typename R, int JT>
__global__ void __launch_bounds__(256) walker_gemm_kernel(GemmArgs g) {
  typedef typename C2<R>::t cplx;
  constexpr int WM_BK = sizeof(R) == 8 ? 16 : 32;  // static shared memory stays below 48 KB
  __shared__ cplx sA[WM_BK][WM_BM];        // A[p][k] slab, p contiguous
  __shared__ cplx sX[WM_BK][8 * JT];       // X[j][k] slab, j contiguous
  if (g.skip && *g.skip) return;
  const int w = blockIdx.y, m0 = blockIdx.x * WM_BM;
  const int N = g.M, nc = g.Nn, K = g.K;
  const int tid = threadIdx.x;
  const int pg = tid & 31, jg = tid >> 5;  // rows m0 + 2 pg + {0,1}, columns jg + 8 t
  const cplx* A = static_cast<const cplx*>(g.A) + (size_t)w * g.sa_b;
  const cplx* X = static_cast<const cplx*>(g.B) + (size_t)w * g.sb_b;
  R accr[2][JT], acci[2][JT];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int t = 0; t < JT; ++t) accr[i][t] = acci[i][t] = R(0);
  for (int k0 = 0; k0 < K; k0 += WM_BK) {
    for (int l = tid; l < WM_BM * WM_BK; l += 256) {  // coalesced along k (A[p][q], unit stride in q)
      const int kk = l % WM_BK, mm = l / WM_BK;
      const int m = m0 + mm, k = k0 + kk;
      cplx v;
      v.x = R(0); v.y = R(0);
      if (m < N && k < K) v = A[(size_t)m * g.sa_m + k];
      sA[kk][mm] = v;
    }
    for (int l = tid; l < 8 * JT * WM_BK; l += 256) {
      const int kk = l % WM_BK, jj = l / WM_BK;
      const int k = k0 + kk;
      cplx v;
      v.x = R(0); v.y = R(0);
      if (jj < nc && k < K) v = X[(size_t)jj * g.sb_n + k];
      sX[kk][jj] = v;
    }
    __syncthreads();
    const int kn = min(WM_BK, K - k0);
    for (int kk = 0; kk < kn; ++kk) {
      const cplx a0 = sA[kk][2 * pg], a1 = sA[kk][2 * pg + 1];
#pragma unroll
      for (int t = 0; t < JT; ++t) {
        const cplx b = sX[kk][jg + 8 * t];
        accr[0][t] = fma(a0.x, b.x, accr[0][t]);
        acci[0][t] = fma(a0.x, b.y, acci[0][t]);
        accr[0][t] = fma(-a0.y, b.y, accr[0][t]);
        acci[0][t] = fma(a0.y, b.x, acci[0][t]);
        accr[1][t] = fma(a1.x, b.x, accr[1][t]);
        acci[1][t] = fma(a1.x, b.y, acci[1][t]);
        accr[1][t] = fma(-a1.y, b.y, accr[1][t]);
        acci[1][t] = fma(a1.y, b.x, acci[1][t]);
      }
    }
    __syncthreads();
  }
  cplx* C = static_cast<cplx*>(g.C) + (size_t)w * g.sc_b;
  cplx* D = g.D ? static_cast<cplx*>(g.D) + (size_t)w * g.sc_b : nullptr;
  const R alr = (R)g.alpha_re, ali = (R)g.alpha_im;
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const int m = m0 + 2 * pg + i;
    if (m >= N) continue;
#pragma unroll
    for (int t = 0; t < JT; ++t) {
      const int j = jg + 8 * t;
      if (j >= nc) continue;
      cplx v;
      v.x = alr * accr[i][t] - ali * acci[i][t];
      v.y = alr * acci[i][t] + ali * accr[i][t];
      const size_t off = (size_t)m + (size_t)j * g.sc_n;
      if (g.accum) {
        cplx o = C[off];
        o.x += v.x;
        o.y += v.y;
        C[off] = o;
      } else {
        C[off] = v;
      }
      if (D) {
        cplx d = D[off];
        d.x += v.x;
        d.y += v.y;
        D[off] = d;
      }
    }
  }
}

template <typename R, int JT>
cudaError_t walker_gemm_launch(const GemmArgs& g, cudaStream_t s) {
  dim3 grid((g.M + WM_BM - 1) / WM_BM, g.batch);
  walker_gemm_kernel<R, JT><<<grid, 256, 0, s>>>(g);
  return cudaGetLastError();
}

// The walker kernel applies to complex A, per-walker batches with unit stride
// along K for A and X and along p for C.
bool walker_gemm_ok(const GemmArgs& g, bool a_complex) {
  return a_complex && g.batch >= 1 && g.sa_k == 1 && g.sb_k == 1 && g.sc_m == 1 && g.Nn <= 96 && g.batch <= 65535;
}

// Sum the split-K partials in fixed order, scale by alpha, store to (or add to) C.
template <typename R>
__global__ void splitk_reduce_kernel(GemmArgs g) {
  typedef typename C2<R>::t cplx;
  if (g.skip && *g.skip) return;
  const size_t MN = (size_t)g.M * g.Nn;
  const cplx* Pp = static_cast<const cplx*>(g.part);
  cplx* C = static_cast<cplx*>(g.C);
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < MN; e += (size_t)gridDim.x * blockDim.x) {
    R sr = R(0), si = R(0);
    for (int z = 0; z < g.splitk; ++z) {
      const cplx v = Pp[(size_t)z * MN + e];
      sr += v.x;
      si += v.y;
    }
    const int m = (int)(e / g.Nn), n = (int)(e % g.Nn);
    cplx o;
    o.x = (R)g.alpha_re * sr - (R)g.alpha_im * si;
    o.y = (R)g.alpha_re * si + (R)g.alpha_im * sr;
    cplx* dst = C + (long long)m * g.sc_m + (long long)n * g.sc_n;
    if (g.accum) {
      const cplx prev = *dst;
      o.x += prev.x;
      o.y += prev.y;
    }
    *dst = o;
  }
}

}  // namespace

template <typename R, bool AC, int BM, int BN>
cudaError_t gemm_launch(const GemmArgs& g, int zdim, cudaStream_t s) {
  dim3 grid((g.M + BM - 1) / BM, (g.Nn + BN - 1) / BN, zdim);
  gemm_kernel<R, AC, BM, BN><<<grid, NT, 0, s>>>(g);
  return cudaGetLastError();
}

template <typename R, bool AC>
cudaError_t gemm_variant(const GemmArgs& g, int zdim, cudaStream_t s) {
  switch (g.variant) {
    case 1: return gemm_launch<R, AC, 128, 32>(g, zdim, s);
    case 2: return gemm_launch<R, AC, 32, 128>(g, zdim, s);
    case 3: return gemm_launch<R, AC, 64, 32>(g, zdim, s);
    default: return gemm_launch<R, AC, 64, 64>(g, zdim, s);
  }
}

template <typename R>
cudaError_t gemm(const GemmArgs& a, bool a_complex, int epi, cudaStream_t s) {
  if (a.M <= 0 || a.Nn <= 0 || a.batch <= 0) return cudaSuccess;
  GemmArgs g = a;
  if (g.variant < 0 || g.variant >= GEMM_VARIANTS) g.variant = 0;
  if (g.variant == 4 && (a.splitk > 1 || !walker_gemm_ok(g, a_complex))) g.variant = 0;
  if (epi != EPI_STORE_ADD) g.D = nullptr;
  g.accum = epi == EPI_ACC ? 1 : 0;
  if (g.splitk > 1 && g.part && g.batch == 1 && epi != EPI_STORE_ADD) {
    cudaError_t e = a_complex ? gemm_variant<R, true>(g, g.splitk, s) : gemm_variant<R, false>(g, g.splitk, s);
    if (e != cudaSuccess) return e;
    const size_t MN = (size_t)a.M * a.Nn;
    size_t blocks = (MN + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    splitk_reduce_kernel<R><<<(int)blocks, 256, 0, s>>>(g);
    return cudaGetLastError();
  }
  g.splitk = 1;
  if (g.variant == 4 && walker_gemm_ok(g, a_complex)) {
    if (g.Nn <= 16) return walker_gemm_launch<R, 2>(g, s);
    if (g.Nn <= 40) return walker_gemm_launch<R, 5>(g, s);
    if (g.Nn <= 64) return walker_gemm_launch<R, 8>(g, s);
    return walker_gemm_launch<R, 12>(g, s);
  }
  if (g.variant >= 4) g.variant = 0;
  return a_complex ? gemm_variant<R, true>(g, a.batch, s) : gemm_variant<R, false>(g, a.batch, s);
}

template cudaError_t gemm<double>(const GemmArgs&, bool, int, cudaStream_t);
template cudaError_t gemm<float>(const GemmArgs&, bool, int, cudaStream_t);

}  // namespace afq
