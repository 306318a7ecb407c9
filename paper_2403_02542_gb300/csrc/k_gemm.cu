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

// Half step out[c][p] = sum_q B[p][q] in[c][q] of complex64 columns (the
// (walker, orbital) columns of Psi, N values each), N <= 128: B^T stays in
// shared memory for the whole (persistent) block, columns stream through in
// tiles of HS_COLS with all of K at once, and each thread accumulates an
// 8-row x 2-column complex tile (summation over q in order, as the tiled
// GEMM does).  Warp w covers rows 32 (w & 3) .. + 31 and columns
// 16 (w >> 2) .. + 15; its lanes form 4 row groups x 8 column pairs, so one
// q step reads 128 contiguous bytes of B^T and 8 distinct columns of the tile
// (four shared-memory wavefronts for 32 FMAs per lane).
constexpr int HS_COLS = 32, HS_T = 256, HS_NMAX = 128;
constexpr int HS_BS = HS_NMAX + 4;  // B^T row stride (16-byte rows; transposed writes 4-way at most)
size_t halfstep_smem() { return (size_t)HS_NMAX * HS_BS * 4 + (size_t)HS_COLS * (HS_NMAX + 1) * 8; }

__global__ void __launch_bounds__(HS_T, 2) halfstep_kernel(const float* __restrict__ B, const float2* __restrict__ in,
                                                           float2* __restrict__ out, int N, int ncols) {
  extern __shared__ __align__(16) float hs_smem[];
  float* Bt = hs_smem;                                                      // [128][HS_BS] Bt[q][p], zero beyond N
  float2* X = reinterpret_cast<float2*>(hs_smem + HS_NMAX * HS_BS);        // [HS_COLS][N + 1]
  const int XS = N + 1;
  for (int e = threadIdx.x; e < HS_NMAX * HS_BS; e += HS_T) Bt[e] = 0.f;
  __syncthreads();
  // B read along its rows (coalesced), eight loads in flight per thread
  const int NN = N * N;
  for (int e0 = 0; e0 < NN; e0 += 8 * HS_T) {
    float v[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int e = e0 + k * HS_T + threadIdx.x;
      v[k] = e < NN ? B[e] : 0.f;
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int e = e0 + k * HS_T + threadIdx.x;
      if (e < NN) Bt[(e % N) * HS_BS + e / N] = v[k];
    }
  }
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int p0 = (wid & 3) * 32 + (lane & 3) * 8;   // this thread's 8 rows
  const int cl = (wid >> 2) * 16 + (lane >> 2) * 2;  // and its 2 columns in the tile
  const int ntiles = (ncols + HS_COLS - 1) / HS_COLS;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int cbase = tile * HS_COLS;
    // the tile's columns: warp wid loads columns wid + 8a, lanes run along q,
    // all sixteen loads of a thread in flight before the first store
    float2 v[HS_COLS / 8][HS_NMAX / 32];
#pragma unroll
    for (int a = 0; a < HS_COLS / 8; ++a) {
      const int c = cbase + wid + 8 * a;
#pragma unroll
      for (int b = 0; b < HS_NMAX / 32; ++b) {
        const int q = lane + 32 * b;
        v[a][b] = (c < ncols && q < N) ? in[(size_t)c * N + q] : make_float2(0.f, 0.f);
      }
    }
    __syncthreads();  // B^T written; the previous tile's reads of X are done
#pragma unroll
    for (int a = 0; a < HS_COLS / 8; ++a)
#pragma unroll
      for (int b = 0; b < HS_NMAX / 32; ++b) {
        const int q = lane + 32 * b;
        if (q < N) X[(wid + 8 * a) * XS + q] = v[a][b];
      }
    __syncthreads();
    float ar[8][2], ai[8][2];
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      ar[r][0] = ar[r][1] = 0.f;
      ai[r][0] = ai[r][1] = 0.f;
    }
    const float2* x0p = X + cl * XS;
    const float2* x1p = x0p + XS;
    for (int q = 0; q < N; ++q) {
      const float4 b0 = *reinterpret_cast<const float4*>(Bt + q * HS_BS + p0);
      const float4 b1 = *reinterpret_cast<const float4*>(Bt + q * HS_BS + p0 + 4);
      const float bb[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
      const float2 x0 = x0p[q], x1 = x1p[q];
#pragma unroll
      for (int r = 0; r < 8; ++r) {
        ar[r][0] = fmaf(bb[r], x0.x, ar[r][0]);
        ai[r][0] = fmaf(bb[r], x0.y, ai[r][0]);
        ar[r][1] = fmaf(bb[r], x1.x, ar[r][1]);
        ai[r][1] = fmaf(bb[r], x1.y, ai[r][1]);
      }
    }
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const int c = cbase + cl + i;
      if (c >= ncols) continue;
      float2* o = out + (size_t)c * N;
#pragma unroll
      for (int r = 0; r < 8; ++r)
        if (p0 + r < N) o[p0 + r] = make_float2(ar[r][i], ai[r][i]);
    }
  }
}

cudaError_t halfstep_prepare() {
  return cudaFuncSetAttribute(reinterpret_cast<const void*>(halfstep_kernel),
                              cudaFuncAttributeMaxDynamicSharedMemorySize, (int)halfstep_smem());
}

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

bool halfstep_ok(const afqmc_ctx* c) { return c->prec == AFQMC_MIXED && c->N <= HS_NMAX && c->f_B != nullptr; }

cudaError_t halfstep_prepare_kernel(const afqmc_ctx* c) { return halfstep_ok(c) ? halfstep_prepare() : cudaSuccess; }

cudaError_t halfstep_launch(const afqmc_ctx* c, int Nw, const void* in, void* out, cudaStream_t s) {
  const int ncols = Nw * c->nc;
  if (ncols <= 0) return cudaSuccess;
  const int ntiles = (ncols + HS_COLS - 1) / HS_COLS;
  int sms = 152, dev = 0;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int grid = ntiles < 2 * sms ? ntiles : 2 * sms;
  if (!capturing(c)) {  // dynamic shared memory above the default limit
    cudaError_t e = halfstep_prepare();
    if (e != cudaSuccess) return e;
  }
  halfstep_kernel<<<grid, HS_T, halfstep_smem(), s>>>(c->f_B, static_cast<const float2*>(in), static_cast<float2*>(out),
                                                     c->N, ncols);
  return cudaGetLastError();
}

}  // namespace afq
