// Field assembly of the mixed step on the 5th-generation tensor cores.
//
// A_w = i sqrt(tau) sum_g c_wg L_g (Eq. heffTOT) for every walker is one dense
// contraction over g with a real right operand:
//   rows    m = 2w + part : X[2w] = -sqrt(tau) Im c_w,  X[2w+1] = sqrt(tau) Re c_w
//   columns e = p Nq + q  : L^T, the Cholesky vectors with g contiguous; q
//                           runs to Nq = N rounded up to a multiple of 8 (the
//                           rows q >= N are zero), so that every run of eight
//                           columns lies in one row p of A_w
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
//
// The same tiled kernel (MODE 2) runs the half steps B Psi of the Split-2
// propagator (Sec. III.B): rows p of D = B - I (B = e^{-tau h''/2} is within
// O(tau ||h''||) of the identity), columns 2 (w nc + j) + part of the walker
// planes (Re / Im of orbital j of walker w, split hi/lo), K = q; the epilogue
// adds the exact identity part, out[w][j][p] = in[w][j][p] + (D in)[w][j][p],
// so the split error is relative to ||D Psi||, not to ||Psi||.  Each thread
// owns row p, so for every column pair the 32 lanes of a warp store 32
// consecutive complex entries of one orbital.
//
// When the products A_w V of the exponential also run on the tensor cores,
// the field epilogue writes A_w instead as bfloat16 hi/lo planes
// A'[w][p][k] = [Re A_w[p][q] | Im A_w[p][q]] (k = q, Kh + q with Kh = Nq
// rounded up to 64; the columns N..Nq of each half are the zero accumulators
// of the zero rows of L^T, stored with the rest in 16-byte runs, and N..Kh
// stay zero), and the basis vectors sit once in planes X[w][j][k] =
// [Re v_j | Im v_j] (same halves).  With X* = X with its halves swapped,
//   (A V)_re = A' [Re V; -Im V] = A' X with B negated on the Im half,
//   (A V)_im = A' [Im V;  Re V] = A' X*,
// so av_tc_kernel (rows p in tiles of 128, K = 2 Kh in slabs of 64, same
// three-MMA split, pipeline and bounded waits) pairs every A' slab with its
// own X slab and the X slab of the other half, into two accumulators.
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
  int M, Nn;           // valid rows (2 Nw; mode 2: N) and columns (N Nq; mode 2: 2 Nw nc)
  float* out;          // mode 0: A as interleaved complex [Nw][N][N]
  __nv_bfloat16* a_hi;  // mode 1: A' planes [Nw * N][KA]
  __nv_bfloat16* a_lo;
  int N, KA, Nq, Kh;
  const float2* hs_in;  // mode 2: walkers in [Nw nc][N] complex64
  float2* hs_out;       // mode 2: walkers out, same layout
  float* nrm;           // mode 1: [rows][nt] sum of squares of each tile row (NULL: none)
  int* err;
};

// MODE 0 writes A as complex64 [w][p][q]; MODE 1 the split planes A'; MODE 2
// the half step out = in + D in.
template <int MODE>
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
      float* orow = MODE == 2 ? nullptr : p.out + (size_t)w * p.N * p.N * 2;
      const int e_base = nt * TG_BN;
      if constexpr (MODE == 2) {
        // row m = p; columns (Re, Im) of 128 orbitals, in chunks of 32
        // orbitals: the 32 input loads of a chunk are issued together (each a
        // 256-byte warp access over 32 consecutive p), then the chunk's 64
        // accumulator columns are read and the sums stored
        for (int c0 = 0; c0 < TG_BN; c0 += 64) {
          const int wj0 = (e_base + c0) >> 1;
          float2 x[32];
#pragma unroll
          for (int t = 0; t < 32; ++t) {
            x[t] = make_float2(0.f, 0.f);
            if (row_ok && 2 * (wj0 + t) < p.Nn) x[t] = p.hs_in[(size_t)(wj0 + t) * p.N + m];
          }
          uint32_t v[64];
          const uint32_t ta = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(buf * TG_BN + c0);
          tmem_ld32(ta, v);
          tmem_ld32(ta + 32, v + 32);
          tmem_wait_ld();
#pragma unroll
          for (int t = 0; t < 32; ++t) {
            if (row_ok && 2 * (wj0 + t) < p.Nn) {
              x[t].x += __uint_as_float(v[2 * t]);
              x[t].y += __uint_as_float(v[2 * t + 1]);
              p.hs_out[(size_t)(wj0 + t) * p.N + m] = x[t];
            }
          }
        }
      }
      float ss = 0.f;  // mode 1: sum of squares of this row of the tile
      for (int c0 = 0; MODE != 2 && c0 < TG_BN; c0 += 8) {
        uint32_t v[8];
        tmem_ld8(tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(buf * TG_BN + c0), v);
        tmem_wait_ld();
        if constexpr (MODE == 1) {
          // row 2w + part -> plane columns part * Kh + q .. q + 7 of row p of
          // walker w (e0, Nq and Kh are multiples of 8: one aligned 16-byte run)
          const int e0 = e_base + c0;
          if (!row_ok || e0 >= p.Nn) continue;
          const int part = m & 1;
          const int pr = e0 / p.Nq, q = e0 - pr * p.Nq;
          const size_t o = ((size_t)w * p.N + pr) * p.KA + (size_t)part * p.Kh + q;
          __align__(16) __nv_bfloat16 h[8], l[8];
#pragma unroll
          for (int t = 0; t < 8; ++t) {
            const float x = __uint_as_float(v[t]);
            h[t] = __float2bfloat16(x);
            l[t] = __float2bfloat16(x - __bfloat162float(h[t]));
            ss = fmaf(x, x, ss);
          }
          *reinterpret_cast<uint4*>(p.a_hi + o) = *reinterpret_cast<const uint4*>(h);
          *reinterpret_cast<uint4*>(p.a_lo + o) = *reinterpret_cast<const uint4*>(l);
        } else {
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
            // four columns in one row p (e0 and Nq are multiples of 4)
            const int e0 = e_base + c0 + (odd ? 4 : 0);
            const int pr = e0 / p.Nq, q0 = e0 - pr * p.Nq;
#pragma unroll
            for (int t = 0; t < 4; ++t) {
              if (pr < p.N && q0 + t < p.N) {
                const float re = odd ? other[t] : mine[t], im = odd ? mine[t] : other[t];
                *reinterpret_cast<float2*>(orow + ((size_t)pr * p.N + q0 + t) * 2) = make_float2(re, im);
              }
            }
          }
        }
      }
      if (MODE == 1 && p.nrm && row_ok) p.nrm[(size_t)m * p.nt + nt] = ss;
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

// Products A_w V for every walker: items (walker, 128-row tile of p), K = KA
// in slabs of 64; each stage carries the A' slab, the walker's X slab (NBp
// rows) and the X slab of the other half (slab kc +- KC/2).
struct AvArgs {
  int N, nc, NBp, KC, MT, n_items, S;
  uint32_t stage_bytes, b_bytes;
  float2* out;        // C[w][j][p] (walker stride c_stride)
  float2* add;        // D += C when non-null (same layout)
  long long c_stride;
  float alpha;
  int* err;
};

__global__ void __launch_bounds__(TG_THREADS, 1)
    av_tc_kernel(const __grid_constant__ CUtensorMap tmA_hi, const __grid_constant__ CUtensorMap tmA_lo,
                 const __grid_constant__ CUtensorMap tmV_hi, const __grid_constant__ CUtensorMap tmV_lo,
                 const AvArgs p) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* base =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* bars = reinterpret_cast<uint64_t*>(base + (size_t)p.S * p.stage_bytes);
  uint64_t* full = bars;             // [S]
  uint64_t* empty = bars + p.S;      // [S]
  uint64_t* tfull = bars + 2 * p.S;  // [2]
  uint64_t* tempty = tfull + 2;      // [2]
  uint64_t* drain = tempty + 2;      // [1]
  volatile uint32_t* tmem_slot = reinterpret_cast<volatile uint32_t*>(drain + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  volatile int* epi_ok = abort_flag + 1;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < p.S; ++s) {
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
      uint32_t last_ph[8];
      bool issued[8] = {false, false, false, false, false, false, false, false};
      for (int item = blockIdx.x; item < p.n_items && !*abort_flag; item += gridDim.x) {
        const int w = item / p.MT, mt = item - (item / p.MT) * p.MT;
        const int arow = w * p.N + mt * TG_BM, vrow = w * p.NBp;
        const int half = p.KC >> 1;
        for (int kc = 0; kc < p.KC; ++kc) {
          if (!mbar_wait(empty + stage, ph ^ 1)) { atomicOr(p.err, 1); *abort_flag = 1; break; }
          mbar_expect_tx(full + stage, p.stage_bytes);
          unsigned char* dst = base + (size_t)stage * p.stage_bytes;
          const int pk = kc < half ? kc + half : kc - half;  // the slab of the other half
          tma_load_2d(dst, &tmA_hi, kc * 64, arow, full + stage);
          tma_load_2d(dst + TG_A_BYTES, &tmA_lo, kc * 64, arow, full + stage);
          tma_load_2d(dst + 2 * TG_A_BYTES, &tmV_hi, kc * 64, vrow, full + stage);
          tma_load_2d(dst + 2 * TG_A_BYTES + p.b_bytes, &tmV_lo, kc * 64, vrow, full + stage);
          tma_load_2d(dst + 2 * TG_A_BYTES + 2 * p.b_bytes, &tmV_hi, pk * 64, vrow, full + stage);
          tma_load_2d(dst + 2 * TG_A_BYTES + 3 * p.b_bytes, &tmV_lo, pk * 64, vrow, full + stage);
          issued[stage] = true;
          last_ph[stage] = ph;
          if (++stage == p.S) { stage = 0; ph ^= 1; }
        }
      }
      for (int s = 0; s < p.S; ++s)
        if (issued[s]) mbar_wait(full + s, last_ph[s]);
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      int stage = 0, buf = 0;
      uint32_t ph = 0, tph[2] = {0, 0};
      const uint32_t idesc = idesc_bf16(TG_BM, p.NBp);
      const uint32_t idesc_neg = idesc | (1u << 14);  // B negated: the -Im A Im V term of the real part
      const int half = p.KC >> 1;
      for (int item = blockIdx.x; item < p.n_items && !*abort_flag; item += gridDim.x) {
        if (!mbar_wait(tempty + buf, tph[buf] ^ 1)) { atomicOr(p.err, 2); *abort_flag = 1; break; }
        tc_fence_after();
        const uint32_t d_re = tmem + (uint32_t)(buf * 2 * p.NBp), d_im = d_re + (uint32_t)p.NBp;
        for (int kc = 0; kc < p.KC; ++kc) {
          if (!mbar_wait(full + stage, ph)) { atomicOr(p.err, 4); *abort_flag = 1; break; }
          tc_fence_after();
          const uint32_t a_hi = sa(base + (size_t)stage * p.stage_bytes);
          const uint32_t a_lo = a_hi + TG_A_BYTES;
          const uint32_t x_hi = a_hi + 2 * TG_A_BYTES;  // X slab kc
          const uint32_t x_lo = x_hi + p.b_bytes;
          const uint32_t y_hi = x_lo + p.b_bytes;       // X slab of the other half
          const uint32_t y_lo = y_hi + p.b_bytes;
          const uint32_t id_re = kc < half ? idesc : idesc_neg;
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const uint32_t off = k * 32;
            const uint32_t first = (kc > 0 || k > 0) ? 1u : 0u;
            umma(d_re, sw128_desc(a_hi + off), sw128_desc(x_hi + off), id_re, first);
            umma(d_re, sw128_desc(a_hi + off), sw128_desc(x_lo + off), id_re, 1u);
            umma(d_re, sw128_desc(a_lo + off), sw128_desc(x_hi + off), id_re, 1u);
            umma(d_im, sw128_desc(a_hi + off), sw128_desc(y_hi + off), idesc, first);
            umma(d_im, sw128_desc(a_hi + off), sw128_desc(y_lo + off), idesc, 1u);
            umma(d_im, sw128_desc(a_lo + off), sw128_desc(y_hi + off), idesc, 1u);
          }
          umma_commit(empty + stage);
          if (++stage == p.S) { stage = 0; ph ^= 1; }
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
    const int r = quad * 32 + lane;
    int buf = 0;
    uint32_t tph[2] = {0, 0};
    for (int item = blockIdx.x; item < p.n_items; item += gridDim.x) {
      const int w = item / p.MT, mt = item - (item / p.MT) * p.MT;
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
      const int pr = mt * TG_BM + r;
      const bool row_ok = pr < p.N;
      float2* o = p.out + (size_t)w * p.c_stride + pr;
      float2* dd = p.add ? p.add + (size_t)w * p.c_stride + pr : nullptr;
      const uint32_t tbase = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(buf * 2 * p.NBp);
      for (int j0 = 0; j0 < p.nc; j0 += 8) {
        uint32_t vr[8], vi[8];
        tmem_ld8(tbase + (uint32_t)j0, vr);                 // real accumulator, column j
        tmem_ld8(tbase + (uint32_t)(p.NBp + j0), vi);       // imaginary accumulator, column j
        tmem_wait_ld();
        if (!row_ok) continue;
#pragma unroll
        for (int t = 0; t < 8; ++t) {
          const int j = j0 + t;
          if (j < p.nc) {
            const float2 v = make_float2(p.alpha * __uint_as_float(vr[t]), p.alpha * __uint_as_float(vi[t]));
            o[(size_t)j * p.N] = v;
            if (dd) {
              float2 x = dd[(size_t)j * p.N];
              x.x += v.x;
              x.y += v.y;
              dd[(size_t)j * p.N] = x;
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
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    __syncwarp();
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TG_TMEM_COLS) : "memory");
  }
}

// X_w from V (complex64 [w][j][q], walker stride vs): row j < nc holds
// [Re v_j | Im v_j] (the second half from column Kh = KA / 2); rows >= nc and
// columns q >= N of each half are zero.  Split into hi/lo.
__global__ void build_v_kernel(const float2* __restrict__ V, long long vs, __nv_bfloat16* __restrict__ hi,
                               __nv_bfloat16* __restrict__ lo, int Nw, int N, int nc, int NBp, int KA) {
  const size_t total = (size_t)Nw * NBp * KA;
  const int Kh = KA >> 1;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int k = (int)(e % KA);
    const size_t rw = e / KA;
    const int row = (int)(rw % NBp);
    const size_t w = rw / NBp;
    float x = 0.f;
    const bool first = k < Kh;
    const int q = first ? k : k - Kh;
    if (row < nc && q < N) {
      const float2 v = V[w * vs + (size_t)row * N + q];
      x = first ? v.x : v.y;
    }
    const __nv_bfloat16 h = __float2bfloat16(x);
    hi[e] = h;
    lo[e] = __float2bfloat16(x - __bfloat162float(h));
  }
}

// ||A_w||_F from the field epilogue's per-tile row sums of squares (rows 2w
// and 2w + 1 of every column tile), one warp per walker, summed in a fixed
// order (lane-strided FP64 partials, then a fixed shuffle tree).
__global__ void normA_rows_kernel(const float* __restrict__ nrm, double* __restrict__ scal, int Nw, int nt) {
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (w >= Nw) return;
  const float* r = nrm + (size_t)(2 * w) * nt;
  double v = 0.0;
  for (int e = lane; e < 2 * nt; e += 32) v += (double)r[e];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if (lane == 0) scal[(size_t)w * SC_COUNT + SC_NORMA] = sqrt(v);
}

// Right operand, once per context: LT[p Nq + q][g] = L[g][p][q] split into
// hi/lo, rows up to Np (zero for q >= N and beyond N Nq), g < Kp (zero
// beyond G).
__global__ void build_lt_kernel(const double* __restrict__ L, __nv_bfloat16* __restrict__ hi,
                                __nv_bfloat16* __restrict__ lo, int N, int Nq, int G, size_t Np, int Kp) {
  const size_t total = Np * Kp, NN = (size_t)N * N;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int g = (int)(e % Kp);
    const size_t row = e / Kp;
    const size_t pr = row / Nq;
    const int q = (int)(row - pr * Nq);
    double x = 0.0;
    if (g < G && pr < (size_t)N && q < N) x = L[(size_t)g * NN + pr * N + q];
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

// D = B - I from the FP64 half-step matrix, split into hi/lo; rows p < Mp and
// columns q < Kp, zero outside N x N.
__global__ void build_d_kernel(const double* __restrict__ B, __nv_bfloat16* __restrict__ hi,
                               __nv_bfloat16* __restrict__ lo, int N, int Mp, int Kp) {
  const size_t total = (size_t)Mp * Kp;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int q = (int)(e % Kp), pr = (int)(e / Kp);
    double x = 0.0;
    if (pr < N && q < N) x = B[(size_t)pr * N + q] - (pr == q ? 1.0 : 0.0);
    split_bf16(x, hi[e], lo[e]);
  }
}

// Walker planes of a half step: row 2 wj + part holds Re (part 0) or Im
// (part 1) of psi_wj[q] for q < N, split hi/lo; each thread converts eight
// consecutive q of one orbital (16-byte plane stores).  Columns N .. Kp stay
// zero from the allocation.
__global__ void build_psi_planes_kernel(const float2* __restrict__ in, __nv_bfloat16* __restrict__ hi,
                                        __nv_bfloat16* __restrict__ lo, int n_orb, int N, int Kp) {
  const int q8 = (N + 7) / 8;
  const size_t total = (size_t)n_orb * q8;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const size_t wj = e / q8;
    const int q0 = (int)(e - wj * q8) * 8;
    __align__(16) __nv_bfloat16 rh[8], rl[8], ih[8], il[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      float2 v = make_float2(0.f, 0.f);
      if (q0 + t < N) v = in[wj * N + q0 + t];
      rh[t] = __float2bfloat16(v.x);
      rl[t] = __float2bfloat16(v.x - __bfloat162float(rh[t]));
      ih[t] = __float2bfloat16(v.y);
      il[t] = __float2bfloat16(v.y - __bfloat162float(ih[t]));
    }
    const size_t o_re = (2 * wj) * (size_t)Kp + q0, o_im = o_re + Kp;
    *reinterpret_cast<uint4*>(hi + o_re) = *reinterpret_cast<const uint4*>(rh);
    *reinterpret_cast<uint4*>(lo + o_re) = *reinterpret_cast<const uint4*>(rl);
    *reinterpret_cast<uint4*>(hi + o_im) = *reinterpret_cast<const uint4*>(ih);
    *reinterpret_cast<uint4*>(lo + o_im) = *reinterpret_cast<const uint4*>(il);
  }
}

inline int grid_for(size_t n) {
  size_t b = (n + 255) / 256;
  return (int)(b > 152 * 64 ? 152 * 64 : (b == 0 ? 1 : b));
}

size_t tg_smem_bytes() { return 1024 + (size_t)TG_S * TG_STAGE_BYTES + (2 * TG_S + 5) * 8 + 16; }
// A' slab (hi, lo) and two X slabs (hi, lo each)
size_t av_stage_bytes(int NBp) { return 2 * (size_t)TG_A_BYTES + 4 * (size_t)NBp * 128; }
size_t av_smem_bytes(int NBp, int S) { return 1024 + (size_t)S * av_stage_bytes(NBp) + (2 * S + 5) * 8 + 16; }

int sm_count() {
  int sms = 152, dev = 0;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms;
}

}  // namespace

// Plan and right operand of the tensor-core field assembly (mixed contexts);
// the products A V go to the tensor cores as well when nc <= 128.
cudaError_t tc_field_setup(afqmc_ctx* c, cudaStream_t s) {
  TgPlan& P = c->tg;
  P = TgPlan();
  if (c->prec != AFQMC_MIXED) return cudaSuccess;
  if (tg_smem_bytes() > (size_t)max_dyn_smem()) return cudaSuccess;
  P.Nq = ((c->N + 7) / 8) * 8;
  const size_t NNq = (size_t)c->N * P.Nq;
  P.Kp = ((c->G + 63) / 64) * 64;
  P.Np = ((NNq + TG_BN - 1) / TG_BN) * TG_BN;
  if (P.Np / TG_BN > (size_t)(1 << 20)) return cudaSuccess;
  cudaError_t e = dmalloc(&P.l_hi, P.Np * P.Kp * 2);
  if (e != cudaSuccess) return e;
  e = dmalloc(&P.l_lo, P.Np * P.Kp * 2);
  if (e != cudaSuccess) return e;
  e = dmalloc(&P.err, sizeof(int));
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(P.err, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  build_lt_kernel<<<grid_for(P.Np * P.Kp), 256, 0, s>>>(c->d_L, static_cast<__nv_bfloat16*>(P.l_hi),
                                                        static_cast<__nv_bfloat16*>(P.l_lo), c->N, P.Nq, c->G, P.Np,
                                                        P.Kp);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (!make_map(reinterpret_cast<CUtensorMap*>(P.map_l_hi), P.l_hi, P.Np, P.Kp, TG_BN) ||
      !make_map(reinterpret_cast<CUtensorMap*>(P.map_l_lo), P.l_lo, P.Np, P.Kp, TG_BN))
    return cudaErrorInvalidValue;
  P.ok = true;
  // half steps: D planes [hs_Mp][hs_Kp] (filled by tc_halfstep_set_b)
  P.hs_Mp = ((c->N + TG_BM - 1) / TG_BM) * TG_BM;
  P.hs_Kp = ((c->N + 63) / 64) * 64;
  e = dmalloc(&P.d_hi, (size_t)P.hs_Mp * P.hs_Kp * 2);
  if (e != cudaSuccess) return e;
  e = dmalloc(&P.d_lo, (size_t)P.hs_Mp * P.hs_Kp * 2);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(P.d_hi, 0, (size_t)P.hs_Mp * P.hs_Kp * 2, s);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(P.d_lo, 0, (size_t)P.hs_Mp * P.hs_Kp * 2, s);
  if (e != cudaSuccess) return e;
  if (!make_map(reinterpret_cast<CUtensorMap*>(P.map_d_hi), P.d_hi, P.hs_Mp, P.hs_Kp, TG_BM) ||
      !make_map(reinterpret_cast<CUtensorMap*>(P.map_d_lo), P.d_lo, P.hs_Mp, P.hs_Kp, TG_BM))
    return cudaErrorInvalidValue;
  P.hs_ok = true;
  // X rows: the nc columns of a walker, padded to the MMA's N granularity;
  // two accumulators of nbp columns, double-buffered, in the 512 TMEM columns
  const int nbp = ((c->nc + 15) / 16) * 16;
  if (nbp <= 128) {
    int S = 4;
    while (S > 2 && av_smem_bytes(nbp, S) > (size_t)max_dyn_smem()) --S;
    if (av_smem_bytes(nbp, S) <= (size_t)max_dyn_smem()) {
      P.av_ok = true;
      P.NBp = nbp;
      P.S_av = S;
      P.Kh = ((P.Nq + 63) / 64) * 64;
      P.KA = 2 * P.Kh;
    }
  }
  return cudaSuccess;
}

// Operand planes sized for the workspace's walker capacity (zeroed on the
// context's stream, which is then synchronised).
cudaError_t tc_field_ws(afqmc_ctx* c) {
  AllocScope alloc_scope(AG_PLANES);
  TgPlan& P = c->tg;
  if (!P.ok) return cudaSuccess;
  void* old[] = {P.x_hi, P.x_lo, P.a_hi, P.a_lo, P.v_hi, P.v_lo, P.p_hi, P.p_lo, P.nrm};
  for (void* q : old)
    if (q) cudaFree(q);
  P.x_hi = P.x_lo = P.a_hi = P.a_lo = P.v_hi = P.v_lo = P.p_hi = P.p_lo = P.nrm = nullptr;
  P.m_cap = 0;
  P.av_cap = 0;
  P.hs_rows = 0;
  const int cap = c->ws.n_walkers;
  if (P.hs_ok) {
    // walker planes: rows 2 (w nc + j) + part, padded to the 256-row column tile;
    // the K padding N .. hs_Kp and the padding rows stay zero
    const size_t rows = (((size_t)2 * cap * c->nc + TG_BN - 1) / TG_BN) * TG_BN;
    cudaError_t e = dmalloc(&P.p_hi, rows * P.hs_Kp * 2);
    if (e != cudaSuccess) return e;
    e = dmalloc(&P.p_lo, rows * P.hs_Kp * 2);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(P.p_hi, 0, rows * P.hs_Kp * 2, c->stream);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(P.p_lo, 0, rows * P.hs_Kp * 2, c->stream);
    if (e != cudaSuccess) return e;
    if (!make_map(reinterpret_cast<CUtensorMap*>(P.map_p_hi), P.p_hi, rows, P.hs_Kp, TG_BN) ||
        !make_map(reinterpret_cast<CUtensorMap*>(P.map_p_lo), P.p_lo, rows, P.hs_Kp, TG_BN))
      return cudaErrorInvalidValue;
    P.hs_rows = (int)rows;
  }
  const int mp = ((2 * cap + TG_BM - 1) / TG_BM) * TG_BM;
  cudaError_t e = dmalloc(&P.x_hi, (size_t)mp * P.Kp * 2);
  if (e != cudaSuccess) return e;
  e = dmalloc(&P.x_lo, (size_t)mp * P.Kp * 2);
  if (e != cudaSuccess) return e;
  if (!make_map(reinterpret_cast<CUtensorMap*>(P.map_x_hi), P.x_hi, (size_t)mp, P.Kp, TG_BM) ||
      !make_map(reinterpret_cast<CUtensorMap*>(P.map_x_lo), P.x_lo, (size_t)mp, P.Kp, TG_BM))
    return cudaErrorInvalidValue;
  P.m_cap = mp;
  if (P.av_ok) {
    // row sums of squares of the field tiles: every row 2w, 2w + 1 (w < Nw) of every
    // column tile is written by each launch before it is read
    e = dmalloc(&P.nrm, (size_t)mp * (P.Np / TG_BN) * sizeof(float));
    if (e != cudaSuccess) return e;
    const size_t arows = (size_t)cap * c->N, vrows = (size_t)cap * P.NBp;
    e = dmalloc(&P.a_hi, arows * P.KA * 2);
    if (e != cudaSuccess) return e;
    e = dmalloc(&P.a_lo, arows * P.KA * 2);
    if (e != cudaSuccess) return e;
    // the columns Nq..Kh of each half stay zero (the field epilogue writes q < Nq only)
    e = cudaMemsetAsync(P.a_hi, 0, arows * P.KA * 2, c->stream);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(P.a_lo, 0, arows * P.KA * 2, c->stream);
    if (e != cudaSuccess) return e;
    e = dmalloc(&P.v_hi, vrows * P.KA * 2);
    if (e != cudaSuccess) return e;
    e = dmalloc(&P.v_lo, vrows * P.KA * 2);
    if (e != cudaSuccess) return e;
    // rows nc..NBp and the columns q >= N of each half stay zero when the
    // Krylov kernels fill the planes
    e = cudaMemsetAsync(P.v_hi, 0, vrows * P.KA * 2, c->stream);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(P.v_lo, 0, vrows * P.KA * 2, c->stream);
    if (e != cudaSuccess) return e;
    if (!make_map(reinterpret_cast<CUtensorMap*>(P.map_a_hi), P.a_hi, arows, P.KA, TG_BM) ||
        !make_map(reinterpret_cast<CUtensorMap*>(P.map_a_lo), P.a_lo, arows, P.KA, TG_BM) ||
        !make_map(reinterpret_cast<CUtensorMap*>(P.map_v_hi), P.v_hi, vrows, P.KA, P.NBp) ||
        !make_map(reinterpret_cast<CUtensorMap*>(P.map_v_lo), P.v_lo, vrows, P.KA, P.NBp))
      return cudaErrorInvalidValue;
    P.av_cap = cap;
  }
  // the zero padding is in place before any stream (the context's, or the
  // non-blocking streams of a batch graph) reads the planes
  return cudaStreamSynchronize(c->stream);
}

cudaError_t tc_field_prepare(const afqmc_ctx* c) {
  if (!c->tg.ok) return cudaSuccess;
  cudaError_t e = raise_smem_limit(field_tc_kernel<0>);
  if (e == cudaSuccess) e = raise_smem_limit(field_tc_kernel<1>);
  if (e == cudaSuccess && c->tg.hs_ok) e = raise_smem_limit(field_tc_kernel<2>);
  if (e == cudaSuccess && c->tg.av_ok) e = raise_smem_limit(av_tc_kernel);
  return e;
}

void tc_field_free(afqmc_ctx* c) {
  TgPlan& P = c->tg;
  void* ptrs[] = {P.l_hi, P.l_lo, P.x_hi, P.x_lo, P.a_hi, P.a_lo, P.v_hi, P.v_lo,
                  P.d_hi, P.d_lo, P.p_hi, P.p_lo, P.nrm, P.err};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  P = TgPlan();
}

// A_w = i sqrt(tau) sum_g c_wg L_g for Nw walkers from ws.c: into ws.A
// (complex64), or into the A' planes when the products A V use them.
cudaError_t tc_field_launch(afqmc_ctx* c, int Nw, double sqrt_tau, cudaStream_t s, bool to_memory) {
  TgPlan& P = c->tg;
  const bool planes = P.av_ok && !to_memory;
  const int mp = ((2 * Nw + TG_BM - 1) / TG_BM) * TG_BM;
  if (mp > P.m_cap || (P.av_ok && Nw > P.av_cap)) return cudaErrorInvalidValue;
  build_x_kernel<<<grid_for((size_t)mp * P.Kp), 256, 0, s>>>(static_cast<const float2*>(c->ws.c),
                                                            static_cast<__nv_bfloat16*>(P.x_hi),
                                                            static_cast<__nv_bfloat16*>(P.x_lo), Nw, c->G, mp, P.Kp,
                                                            (float)sqrt_tau);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  TgArgs a{};
  a.mt = mp / TG_BM;
  a.nt = (int)(P.Np / TG_BN);
  a.KC = P.Kp / 64;
  a.n_items = a.mt * a.nt;
  a.M = 2 * Nw;
  a.Nn = c->N * P.Nq;
  a.Nq = P.Nq;
  a.Kh = P.Kh;
  a.out = static_cast<float*>(c->ws.A);
  a.a_hi = static_cast<__nv_bfloat16*>(P.a_hi);
  a.a_lo = static_cast<__nv_bfloat16*>(P.a_lo);
  a.N = c->N;
  a.KA = P.KA;
  a.nrm = planes ? static_cast<float*>(P.nrm) : nullptr;
  a.err = static_cast<int*>(P.err);
  if (!capturing(c)) {
    e = planes ? raise_smem_limit(field_tc_kernel<1>) : raise_smem_limit(field_tc_kernel<0>);
    if (e != cudaSuccess) return e;
  }
  const int sms = sm_count();
  const int grid = a.n_items < sms ? a.n_items : sms;
  CUtensorMap mxh, mxl, mlh, mll;
  memcpy(&mxh, P.map_x_hi, sizeof(CUtensorMap));
  memcpy(&mxl, P.map_x_lo, sizeof(CUtensorMap));
  memcpy(&mlh, P.map_l_hi, sizeof(CUtensorMap));
  memcpy(&mll, P.map_l_lo, sizeof(CUtensorMap));
  if (planes)
    field_tc_kernel<1><<<grid, TG_THREADS, tg_smem_bytes(), s>>>(mxh, mxl, mlh, mll, a);
  else
    field_tc_kernel<0><<<grid, TG_THREADS, tg_smem_bytes(), s>>>(mxh, mxl, mlh, mll, a);
  return cudaGetLastError();
}

cudaError_t tc_av_launch(afqmc_ctx* c, int Nw, const void* V, long long v_stride, void* C, void* D,
                         long long c_stride, double alpha, cudaStream_t s) {
  TgPlan& P = c->tg;
  if (!P.av_ok || Nw > P.av_cap) return cudaErrorInvalidValue;
  cudaError_t e = cudaSuccess;
  if (V) {  // otherwise the planes already hold V (written by the Arnoldi kernels)
    const size_t elems = (size_t)Nw * P.NBp * P.KA;
    build_v_kernel<<<grid_for(elems), 256, 0, s>>>(static_cast<const float2*>(V), v_stride,
                                                   static_cast<__nv_bfloat16*>(P.v_hi),
                                                   static_cast<__nv_bfloat16*>(P.v_lo), Nw, c->N, c->nc, P.NBp, P.KA);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  AvArgs a;
  a.N = c->N;
  a.nc = c->nc;
  a.NBp = P.NBp;
  a.KC = P.KA / 64;
  a.MT = (c->N + TG_BM - 1) / TG_BM;
  a.n_items = Nw * a.MT;
  a.S = P.S_av;
  a.b_bytes = (uint32_t)P.NBp * 128;
  a.stage_bytes = (uint32_t)av_stage_bytes(P.NBp);
  a.out = static_cast<float2*>(C);
  a.add = static_cast<float2*>(D);
  a.c_stride = c_stride;
  a.alpha = (float)alpha;
  a.err = static_cast<int*>(P.err);
  if (!capturing(c)) {
    e = raise_smem_limit(av_tc_kernel);
    if (e != cudaSuccess) return e;
  }
  const int sms = sm_count();
  const int grid = a.n_items < sms ? a.n_items : sms;
  CUtensorMap mah, mal, mvh, mvl;
  memcpy(&mah, P.map_a_hi, sizeof(CUtensorMap));
  memcpy(&mal, P.map_a_lo, sizeof(CUtensorMap));
  memcpy(&mvh, P.map_v_hi, sizeof(CUtensorMap));
  memcpy(&mvl, P.map_v_lo, sizeof(CUtensorMap));
  av_tc_kernel<<<grid, TG_THREADS, av_smem_bytes(P.NBp, P.S_av), s>>>(mah, mal, mvh, mvl, a);
  return cudaGetLastError();
}

cudaError_t tc_halfstep_set_b(afqmc_ctx* c, cudaStream_t s) {
  TgPlan& P = c->tg;
  if (!P.hs_ok) return cudaSuccess;
  build_d_kernel<<<grid_for((size_t)P.hs_Mp * P.hs_Kp), 256, 0, s>>>(
      c->d_B, static_cast<__nv_bfloat16*>(P.d_hi), static_cast<__nv_bfloat16*>(P.d_lo), c->N, P.hs_Mp, P.hs_Kp);
  return cudaGetLastError();
}

cudaError_t tc_halfstep_launch(afqmc_ctx* c, int Nw, const void* in, void* out, cudaStream_t s) {
  TgPlan& P = c->tg;
  const int n_orb = Nw * c->nc;
  const int rows = ((2 * n_orb + TG_BN - 1) / TG_BN) * TG_BN;
  if (!P.hs_ok || rows > P.hs_rows || in == out) return cudaErrorInvalidValue;
  build_psi_planes_kernel<<<grid_for((size_t)n_orb * ((c->N + 7) / 8)), 256, 0, s>>>(
      static_cast<const float2*>(in), static_cast<__nv_bfloat16*>(P.p_hi), static_cast<__nv_bfloat16*>(P.p_lo),
      n_orb, c->N, P.hs_Kp);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  TgArgs a{};
  a.mt = P.hs_Mp / TG_BM;
  a.nt = rows / TG_BN;
  a.KC = P.hs_Kp / 64;
  a.n_items = a.mt * a.nt;
  a.M = c->N;
  a.Nn = 2 * n_orb;
  a.N = c->N;
  a.hs_in = static_cast<const float2*>(in);
  a.hs_out = static_cast<float2*>(out);
  a.err = static_cast<int*>(P.err);
  if (!capturing(c)) {
    e = raise_smem_limit(field_tc_kernel<2>);
    if (e != cudaSuccess) return e;
  }
  const int sms = sm_count();
  const int grid = a.n_items < sms ? a.n_items : sms;
  CUtensorMap mdh, mdl, mph, mpl;
  memcpy(&mdh, P.map_d_hi, sizeof(CUtensorMap));
  memcpy(&mdl, P.map_d_lo, sizeof(CUtensorMap));
  memcpy(&mph, P.map_p_hi, sizeof(CUtensorMap));
  memcpy(&mpl, P.map_p_lo, sizeof(CUtensorMap));
  field_tc_kernel<2><<<grid, TG_THREADS, tg_smem_bytes(), s>>>(mdh, mdl, mph, mpl, a);
  return cudaGetLastError();
}

// ||A_w||_F of the last field assembly (its epilogue left the row sums)
cudaError_t tc_av_normA(afqmc_ctx* c, int Nw, cudaStream_t s) {
  const TgPlan& P = c->tg;
  normA_rows_kernel<<<(Nw + 7) / 8, 256, 0, s>>>(static_cast<const float*>(P.nrm), c->ws.scal, Nw,
                                                 (int)(P.Np / TG_BN));
  return cudaGetLastError();
}

}  // namespace afq
