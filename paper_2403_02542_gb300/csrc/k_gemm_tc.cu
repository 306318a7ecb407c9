// Field assembly of the mixed step on the 5th-generation tensor cores.
//
// A_w = i sqrt(tau) sum_g c_wg L_g (Eq. heffTOT) for every walker is one dense
// contraction over g with a real right operand:
//   rows    m = 2w + part : X[2w] = -sqrt(tau) Im c_w,  X[2w+1] = sqrt(tau) Re c_w
//   columns e = (p, q)    : L^T, the Cholesky vectors with g contiguous
//   K       g
// so D[2w][e] = Re A_w[e] and D[2w+1][e] = Im A_w[e].  Both operands are split
// x = hi + lo into bfloat16 pairs and D = X_hi L_hi + X_hi L_lo + X_lo L_hi is
// accumulated in FP32 (three kind::f16 MMAs per K step).
//
// Tiles: 128 rows x 256 columns, K in slabs of 64 (one 128-byte swizzle row),
// two-stage TMA ring for both operands, accumulator double-buffered in TMEM
// (2 x 256 columns).  Persistent grid of one CTA per SM; work items run
// column-tile-major so the CTAs working at the same time share the L^T tiles
// in L2.  Warp roles: warp 0 TMA producer, warp 1 TMEM allocator and MMA
// issuer, warps 2..5 the epilogue (each thread owns one accumulator row; a
// lane pair (2w, 2w+1) exchanges halves so that each thread stores four
// complex values of A_w contiguously).  Every mbarrier wait is bounded; on a
// timeout the kernel raises an error flag, stops issuing work and frees TMEM.
#include <cuda.h>
#include <cuda_bf16.h>

#include <cstring>

#include "internal.cuh"
#include "tc_common.cuh"

namespace afq {

namespace {

constexpr int TG_THREADS = 192;
constexpr int TG_BM = 128, TG_BN = 256, TG_S = 2;
constexpr int TG_TMEM_COLS = 512;
constexpr uint32_t TG_A_BYTES = 128 * 128;        // one operand half: 128 rows x 64 bf16
constexpr uint32_t TG_B_BYTES = TG_BN * 128;      // 256 rows x 64 bf16
constexpr uint32_t TG_STAGE_BYTES = 2 * TG_A_BYTES + 2 * TG_B_BYTES;

struct TgArgs {
  int mt, nt, KC, n_items;
  int M, Nn;           // valid rows (2 Nw) and columns (N^2)
  float* out;          // A as interleaved complex [Nw][Nn]
  int* err;
};

__global__ void __launch_bounds__(TG_THREADS, 1)
    field_tc_kernel(const __grid_constant__ CUtensorMap tmX_hi, const __grid_constant__ CUtensorMap tmX_lo,
                    const __grid_constant__ CUtensorMap tmL_hi, const __grid_constant__ CUtensorMap tmL_lo,
                    const TgArgs p) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* base =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* bars = reinterpret_cast<uint64_t*>(base + (size_t)TG_S * TG_STAGE_BYTES);
  uint64_t* full = bars;            // [S]
  uint64_t* empty = bars + TG_S;    // [S]
  uint64_t* tfull = bars + 2 * TG_S;  // [2]
  uint64_t* tempty = tfull + 2;     // [2]
  uint64_t* drain = tempty + 2;     // [1]
  volatile uint32_t* tmem_slot = reinterpret_cast<volatile uint32_t*>(drain + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  volatile int* epi_ok = abort_flag + 1;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < TG_S; ++s) {
      mbar_init(full + s, 1);
      mbar_init(empty + s, 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(tfull + b, 1);
      mbar_init(tempty + b, 128);
    }
    mbar_init(drain, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(sa((const void*)tmem_slot)),
                 "r"(TG_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    // ------------------------------------------------------------ producer
    if (lane == 0) {
      int stage = 0;
      uint32_t ph = 0;
      uint32_t last_ph[TG_S];
      bool issued[TG_S];
      for (int s = 0; s < TG_S; ++s) issued[s] = false;
      for (int item = blockIdx.x; item < p.n_items && !*abort_flag; item += gridDim.x) {
        const int mt = item % p.mt, nt = item / p.mt;
        for (int kc = 0; kc < p.KC; ++kc) {
          if (!mbar_wait(empty + stage, ph ^ 1)) { atomicOr(p.err, 1); *abort_flag = 1; break; }
          mbar_expect_tx(full + stage, TG_STAGE_BYTES);
          unsigned char* dst = base + (size_t)stage * TG_STAGE_BYTES;
          tma_load_2d(dst, &tmX_hi, kc * 64, mt * TG_BM, full + stage);
          tma_load_2d(dst + TG_A_BYTES, &tmX_lo, kc * 64, mt * TG_BM, full + stage);
          tma_load_2d(dst + 2 * TG_A_BYTES, &tmL_hi, kc * 64, nt * TG_BN, full + stage);
          tma_load_2d(dst + 2 * TG_A_BYTES + TG_B_BYTES, &tmL_lo, kc * 64, nt * TG_BN, full + stage);
          issued[stage] = true;
          last_ph[stage] = ph;
          if (++stage == TG_S) { stage = 0; ph ^= 1; }
        }
      }
      for (int s = 0; s < TG_S; ++s)
        if (issued[s]) mbar_wait(full + s, last_ph[s]);
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      int stage = 0, buf = 0;
      uint32_t ph = 0, tph[2] = {0, 0};
      const uint32_t idesc = idesc_bf16(TG_BM, TG_BN);
      for (int item = blockIdx.x; item < p.n_items && !*abort_flag; item += gridDim.x) {
        if (!mbar_wait(tempty + buf, tph[buf] ^ 1)) { atomicOr(p.err, 2); *abort_flag = 1; break; }
        tc_fence_after();
        const uint32_t d = tmem + (uint32_t)(buf * TG_BN);
        for (int kc = 0; kc < p.KC; ++kc) {
          if (!mbar_wait(full + stage, ph)) { atomicOr(p.err, 4); *abort_flag = 1; break; }
          tc_fence_after();
          const uint32_t a_hi = sa(base + (size_t)stage * TG_STAGE_BYTES);
          const uint32_t a_lo = a_hi + TG_A_BYTES;
          const uint32_t b_hi = a_hi + 2 * TG_A_BYTES;
          const uint32_t b_lo = b_hi + TG_B_BYTES;
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const uint32_t off = k * 32;
            umma(d, sw128_desc(a_hi + off), sw128_desc(b_hi + off), idesc, (kc > 0 || k > 0) ? 1u : 0u);
            umma(d, sw128_desc(a_hi + off), sw128_desc(b_lo + off), idesc, 1u);
            umma(d, sw128_desc(a_lo + off), sw128_desc(b_hi + off), idesc, 1u);
          }
          umma_commit(empty + stage);
          if (++stage == TG_S) { stage = 0; ph ^= 1; }
        }
        umma_commit(tfull + buf);
        tph[buf] ^= 1;
        buf ^= 1;
      }
      umma_commit(drain);
      if (!mbar_wait(drain, 0)) atomicOr(p.err, 8);
    }
  } else {
    // ------------------------------------------------------------ epilogue
    const int quad = warp & 3;
    const int r = quad * 32 + lane;  // accumulator row of this thread
    const bool odd = lane & 1;
    int buf = 0;
    uint32_t tph[2] = {0, 0};
    for (int item = blockIdx.x; item < p.n_items; item += gridDim.x) {
      const int mt = item % p.mt, nt = item / p.mt;
      if (r == 0) {
        const bool ok = mbar_wait(tfull + buf, tph[buf]);
        if (!ok) { atomicOr(p.err, 16); *abort_flag = 1; }
        *epi_ok = ok ? 1 : 0;
      }
      named_bar(1, 128);
      const int ok = *epi_ok;
      named_bar(1, 128);
      if (!ok) break;
      tc_fence_after();
      const int m = mt * TG_BM + r;
      const int w = m >> 1;
      const bool row_ok = m < p.M;
      float* orow = p.out + (size_t)w * p.Nn * 2;
      const int e_base = nt * TG_BN;
      for (int c0 = 0; c0 < TG_BN; c0 += 8) {
        uint32_t v[8];
        tmem_ld8(tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(buf * TG_BN + c0), v);
        tmem_wait_ld();
        // even lane (row 2w = Re A) keeps columns c0..c0+3, odd lane (Im A) c0+4..c0+7
        float mine[4], other[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          const float send = __uint_as_float(odd ? v[t] : v[4 + t]);
          const float recv = __shfl_xor_sync(0xffffffffu, send, 1);
          mine[t] = __uint_as_float(odd ? v[4 + t] : v[t]);
          other[t] = recv;
        }
        if (row_ok) {
          const int e0 = e_base + c0 + (odd ? 4 : 0);
#pragma unroll
          for (int t = 0; t < 4; ++t) {
            if (e0 + t < p.Nn) {
              const float re = odd ? other[t] : mine[t], im = odd ? mine[t] : other[t];
              *reinterpret_cast<float2*>(orow + (size_t)(e0 + t) * 2) = make_float2(re, im);
            }
          }
        }
      }
      tc_fence_before();
      mbar_arrive(tempty + buf);
      tph[buf] ^= 1;
      buf ^= 1;
    }
  }
  // ------------------------------------------------------------ teardown
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    __syncwarp();
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TG_TMEM_COLS) : "memory");
  }
}

// Right operand, once per context: LT[e][g] = L[g][e] split into hi/lo,
// rows e < Np (zero beyond N^2), g < Kp (zero beyond G).
__global__ void build_lt_kernel(const double* __restrict__ L, __nv_bfloat16* __restrict__ hi,
                                __nv_bfloat16* __restrict__ lo, size_t NN, int G, size_t Np, int Kp) {
  const size_t total = Np * Kp;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int g = (int)(e % Kp);
    const size_t row = e / Kp;
    double x = 0.0;
    if (g < G && row < NN) x = L[(size_t)g * NN + row];
    split_bf16(x, hi[e], lo[e]);
  }
}

// Left operand, every step: X[2w][g] = -sqrt(tau) Im c_wg, X[2w+1][g] =
// sqrt(tau) Re c_wg, split into hi/lo; rows up to the 128-row padding are zero.
__global__ void build_x_kernel(const float2* __restrict__ c, __nv_bfloat16* __restrict__ hi,
                               __nv_bfloat16* __restrict__ lo, int Nw, int G, int Mp, int Kp, float sqrt_tau) {
  const size_t total = (size_t)Mp * Kp;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int g = (int)(e % Kp);
    const int m = (int)(e / Kp);
    const int w = m >> 1;
    float x = 0.f;
    if (w < Nw && g < G) {
      const float2 v = c[(size_t)w * G + g];
      x = (m & 1) ? sqrt_tau * v.x : -sqrt_tau * v.y;
    }
    const __nv_bfloat16 h = __float2bfloat16(x);
    hi[e] = h;
    lo[e] = __float2bfloat16(x - __bfloat162float(h));
  }
}

inline int grid_for(size_t n) {
  size_t b = (n + 255) / 256;
  return (int)(b > 152 * 64 ? 152 * 64 : (b == 0 ? 1 : b));
}

size_t tg_smem_bytes() { return 1024 + (size_t)TG_S * TG_STAGE_BYTES + (2 * TG_S + 5) * 8 + 16; }

}  // namespace

// Plan and right operand of the tensor-core field assembly (mixed contexts).
cudaError_t tc_field_setup(afqmc_ctx* c, cudaStream_t s) {
  TgPlan& P = c->tg;
  P = TgPlan();
  if (c->prec != AFQMC_MIXED) return cudaSuccess;
  if (tg_smem_bytes() > (size_t)max_dyn_smem()) return cudaSuccess;
  const size_t NN = (size_t)c->N * c->N;
  P.Kp = ((c->G + 63) / 64) * 64;
  P.Np = ((NN + TG_BN - 1) / TG_BN) * TG_BN;
  if (P.Np / TG_BN > (size_t)(1 << 20)) return cudaSuccess;
  cudaError_t e = cudaMalloc(&P.l_hi, P.Np * P.Kp * 2);
  if (e != cudaSuccess) return e;
  e = cudaMalloc(&P.l_lo, P.Np * P.Kp * 2);
  if (e != cudaSuccess) return e;
  e = cudaMalloc(&P.err, sizeof(int));
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(P.err, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  build_lt_kernel<<<grid_for(P.Np * P.Kp), 256, 0, s>>>(c->d_L, static_cast<__nv_bfloat16*>(P.l_hi),
                                                        static_cast<__nv_bfloat16*>(P.l_lo), NN, c->G, P.Np, P.Kp);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (!make_map(reinterpret_cast<CUtensorMap*>(P.map_l_hi), P.l_hi, P.Np, P.Kp, TG_BN) ||
      !make_map(reinterpret_cast<CUtensorMap*>(P.map_l_lo), P.l_lo, P.Np, P.Kp, TG_BN))
    return cudaErrorInvalidValue;
  P.ok = true;
  return cudaSuccess;
}

// Left-operand planes for the workspace's walker capacity.
cudaError_t tc_field_ws(afqmc_ctx* c) {
  TgPlan& P = c->tg;
  if (!P.ok) return cudaSuccess;
  if (P.x_hi) cudaFree(P.x_hi);
  if (P.x_lo) cudaFree(P.x_lo);
  P.x_hi = P.x_lo = nullptr;
  P.m_cap = 0;
  const int mp = ((2 * c->ws.n_walkers + TG_BM - 1) / TG_BM) * TG_BM;
  cudaError_t e = cudaMalloc(&P.x_hi, (size_t)mp * P.Kp * 2);
  if (e != cudaSuccess) return e;
  e = cudaMalloc(&P.x_lo, (size_t)mp * P.Kp * 2);
  if (e != cudaSuccess) return e;
  if (!make_map(reinterpret_cast<CUtensorMap*>(P.map_x_hi), P.x_hi, (size_t)mp, P.Kp, TG_BM) ||
      !make_map(reinterpret_cast<CUtensorMap*>(P.map_x_lo), P.x_lo, (size_t)mp, P.Kp, TG_BM))
    return cudaErrorInvalidValue;
  P.m_cap = mp;
  return cudaSuccess;
}

cudaError_t tc_field_prepare(const afqmc_ctx* c) {
  if (!c->tg.ok) return cudaSuccess;
  return raise_smem_limit(field_tc_kernel);
}

void tc_field_free(afqmc_ctx* c) {
  TgPlan& P = c->tg;
  void* ptrs[] = {P.l_hi, P.l_lo, P.x_hi, P.x_lo, P.err};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  P = TgPlan();
}

// A_w = i sqrt(tau) sum_g c_wg L_g for Nw walkers from ws.c into ws.A (complex64).
cudaError_t tc_field_launch(afqmc_ctx* c, int Nw, double sqrt_tau, cudaStream_t s) {
  TgPlan& P = c->tg;
  const int mp = ((2 * Nw + TG_BM - 1) / TG_BM) * TG_BM;
  if (mp > P.m_cap) return cudaErrorInvalidValue;
  build_x_kernel<<<grid_for((size_t)mp * P.Kp), 256, 0, s>>>(static_cast<const float2*>(c->ws.c),
                                                            static_cast<__nv_bfloat16*>(P.x_hi),
                                                            static_cast<__nv_bfloat16*>(P.x_lo), Nw, c->G, mp, P.Kp,
                                                            (float)sqrt_tau);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  TgArgs a;
  a.mt = mp / TG_BM;
  a.nt = (int)(P.Np / TG_BN);
  a.KC = P.Kp / 64;
  a.n_items = a.mt * a.nt;
  a.M = 2 * Nw;
  a.Nn = c->N * c->N;
  a.out = static_cast<float*>(c->ws.A);
  a.err = static_cast<int*>(P.err);
  if (!capturing(c)) {
    e = raise_smem_limit(field_tc_kernel);
    if (e != cudaSuccess) return e;
  }
  int sms = 152, dev = 0;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int grid = a.n_items < sms ? a.n_items : sms;
  CUtensorMap mxh, mxl, mlh, mll;
  memcpy(&mxh, P.map_x_hi, sizeof(CUtensorMap));
  memcpy(&mxl, P.map_x_lo, sizeof(CUtensorMap));
  memcpy(&mlh, P.map_l_hi, sizeof(CUtensorMap));
  memcpy(&mll, P.map_l_lo, sizeof(CUtensorMap));
  field_tc_kernel<<<grid, TG_THREADS, tg_smem_bytes(), s>>>(mxh, mxl, mlh, mll, a);
  return cudaGetLastError();
}

}  // namespace afq
