// Tiled SIMT GEMM with a real or complex A and a complex B, used for the
// walker-batched contractions of the step: the force-bias contraction
// sum_{jq} Lh_g,jq Theta_jq (Eq. force_shift), the field assembly
// sum_g c_g L_g (Eq. heffTOT), the half step B Psi (Sec. III.B) and the
// per-walker products A Psi of the Taylor and Krylov actions (Sec. IV).
//
// C[b][m][n] = alpha * sum_k A[b][m][k] B[b][n][k], strides in elements.
// 64 x 64 output tile, K slab of 8 staged in shared memory, 256 threads with
// a 4 x 4 register tile each.  The thread-to-output map follows the unit
// stride of C so that the stores coalesce.
#include "internal.cuh"

namespace afq {

namespace {

constexpr int BM = 64, BN = 64, BK = 8, NT = 256;

template <typename R, bool ACPLX>
__global__ void __launch_bounds__(NT) gemm_kernel(GemmArgs g) {
  typedef typename C2<R>::t cplx;
  __shared__ R sAr[BK][BM];
  __shared__ R sAi[ACPLX ? BK : 1][ACPLX ? BM : 1];
  __shared__ R sBr[BK][BN];
  __shared__ R sBi[BK][BN];

  const int b = blockIdx.z;
  const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const bool swap = (g.sc_m == 1);  // C contiguous along m: threads run along m
  const int tm = swap ? tx : ty, tn = swap ? ty : tx;

  // batch offset in elements of A's own type (a complex element is two reals)
  const R* A = static_cast<const R*>(g.A) + (long long)b * g.sa_b * (ACPLX ? 2 : 1);
  const cplx* Bp = static_cast<const cplx*>(g.B) + (long long)b * g.sb_b;
  const bool a_kc = (g.sa_k == 1);
  const bool b_kc = (g.sb_k == 1);

  R accr[4][4], acci[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) accr[i][j] = acci[i][j] = R(0);

  for (int k0 = 0; k0 < g.K; k0 += BK) {
    for (int l = tid; l < BM * BK; l += NT) {
      int mm, kk;
      if (a_kc) { kk = l % BK; mm = l / BK; } else { mm = l % BM; kk = l / BM; }
      const int m = m0 + mm, k = k0 + kk;
      R vr = R(0), vi = R(0);
      if (m < g.M && k < g.K) {
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
      if (n < g.Nn && k < g.K) v = Bp[(long long)n * g.sb_n + (long long)k * g.sb_k];
      sBr[kk][nn] = v.x;
      sBi[kk][nn] = v.y;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      R ar[4], ai[4], br[4], bi[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        ar[i] = sAr[kk][tm + 16 * i];
        ai[i] = ACPLX ? sAi[kk][tm + 16 * i] : R(0);
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        br[j] = sBr[kk][tn + 16 * j];
        bi[j] = sBi[kk][tn + 16 * j];
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
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

  cplx* C = static_cast<cplx*>(g.C) + (long long)b * g.sc_b;
  cplx* D = g.D ? static_cast<cplx*>(g.D) + (long long)b * g.sc_b : nullptr;
  const R alr = (R)g.alpha_re, ali = (R)g.alpha_im;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int m = m0 + tm + 16 * i;
    if (m >= g.M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int n = n0 + tn + 16 * j;
      if (n >= g.Nn) continue;
      cplx v;
      v.x = alr * accr[i][j] - ali * acci[i][j];
      v.y = alr * acci[i][j] + ali * accr[i][j];
      const long long off = (long long)m * g.sc_m + (long long)n * g.sc_n;
      C[off] = v;
      if (D) {
        cplx d = D[off];
        d.x += v.x;
        d.y += v.y;
        D[off] = d;
      }
    }
  }
}

}  // namespace

template <typename R>
cudaError_t gemm(const GemmArgs& a, bool a_complex, int epi, cudaStream_t s) {
  if (a.M <= 0 || a.Nn <= 0 || a.batch <= 0) return cudaSuccess;
  GemmArgs g = a;
  if (epi != EPI_STORE_ADD) g.D = nullptr;
  dim3 grid((a.M + BM - 1) / BM, (a.Nn + BN - 1) / BN, a.batch);
  if (a_complex)
    gemm_kernel<R, true><<<grid, NT, 0, s>>>(g);
  else
    gemm_kernel<R, false><<<grid, NT, 0, s>>>(g);
  return cudaGetLastError();
}

template cudaError_t gemm<double>(const GemmArgs&, bool, int, cudaStream_t);
template cudaError_t gemm<float>(const GemmArgs&, bool, int, cudaStream_t);

}  // namespace afq
