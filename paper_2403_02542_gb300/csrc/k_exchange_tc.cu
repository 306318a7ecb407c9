// Coulomb and exchange contractions of the local energy on the 5th-generation
// tensor cores (mixed-precision contexts).
//
// For every walker w, spin s and Cholesky vector g the local energy (Eq. eloc
// with <pq|rs> = sum_g L_g,pr L_g,qs) needs T = Lh_gs Theta_ws^T (n x n,
// K = N), its trace and sum_ij T_ij T_ji.  Across walkers and g this is one
// dense contraction with a block-diagonal epilogue:
//   rows    (g, i)        : the half-rotated Cholesky vectors Lh (operand A),
//   columns (w, re/im, j) : Theta split into real and imaginary planes (B),
//   K       q             : the orbital index.
// Precision: both operands are split x = hi + lo into bfloat16 pairs and
// T = A_hi B_hi + A_hi B_lo + A_lo B_hi is accumulated in FP32 (three
// kind::f16 MMAs per K step); the dropped lo*lo term is below 2^-16 relative.
//
// Work decomposition: one work item = (spin, group of Wc walkers); its B tile
// (Wc * 2n rows x K) stays in shared memory while the A tiles (128 rows =
// gpt g's x n rows, all K) stream through a TMA ring.  A persistent grid of
// one CTA per SM walks the items.  Warp roles:
//   warp 0      TMA producer (one elected lane)
//   warp 1      TMEM allocator and MMA issuer (one elected lane)
//   warps 2..9  two epilogue warpgroups; each reads its walkers' columns of the
//               TMEM accumulator, transposes the n x n blocks through shared
//               memory and writes (tr T, sum T_ij T_ji) per (w, g, s).
// Row layout of the A tiles: for n <= 32 every 32-row warp slot holds whole
// g blocks (gpw = 32 / n of them, the rest zero rows), so each epilogue warp
// owns its blocks: the transposition goes through the warp's own staging rows
// and the sums over a block's rows are segmented warp shuffles, with no
// barrier between warps.  For n > 32 the blocks are packed across the tile
// (128 / n per tile) and the four warps of a warpgroup share a staging area.
// The accumulator is double-buffered in TMEM so the epilogue of one A tile
// overlaps the MMAs of the next.  Every mbarrier wait is bounded; on a
// timeout the kernel raises an error flag, stops issuing work and frees its
// TMEM.
#include <cuda.h>
#include <cuda_bf16.h>

#include <cstring>

#include "internal.cuh"
#include "tc_common.cuh"

namespace afq {

namespace {

constexpr int TC_TMEM_COLS = 512;

struct TcArgs {
  int n, gpt, gpw, T, KC, NB, Wc, WG, Nw, cap, G, S, n_items;
  uint32_t sB_bytes, sA_stage_bytes, staging_floats;
  int sp;  // staging row stride in floats (a multiple of 4 with sp / 4 odd)
  double* epart;
  int* err;
};

// NM > 0: n <= NM <= 32 and each epilogue thread keeps its own accumulator
// row in registers; NM == 0: the row is read back from shared memory.  WL:
// warp-slot row layout (needs NM > 0), else packed rows.  EWG epilogue
// warpgroups.  SB = false: the item's B tile (all K) stays in shared memory
// for all its A tiles; SB = true (large N): each stage of the ring carries
// the B slab with the A slab (B re-read from L2 for every A tile).
template <int NM, int EWG, bool SB, bool WL>
__global__ void __launch_bounds__(64 + 128 * EWG, 1)
    exchange_tc_kernel(const __grid_constant__ CUtensorMap tmA_hi, const __grid_constant__ CUtensorMap tmA_lo,
                       const __grid_constant__ CUtensorMap tmB_hi, const __grid_constant__ CUtensorMap tmB_lo,
                       const TcArgs p) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // 1024-byte aligned base for the swizzled tiles
  unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  unsigned char* sB = base;                                   // [hi,lo][KC][NB][64] bf16
  unsigned char* sA = sB + p.sB_bytes;                        // [S][hi,lo][128][64] bf16
  float* stg = reinterpret_cast<float*>(sA + (size_t)p.S * p.sA_stage_bytes);  // [WG][128][sp]
  float* pbuf = stg + (size_t)EWG * p.staging_floats;  // [WG][128][4]
  uint64_t* bars = reinterpret_cast<uint64_t*>(pbuf + EWG * 128 * 4);
  uint64_t* full = bars;                 // [S]
  uint64_t* empty = bars + p.S;          // [S]
  uint64_t* bfull = bars + 2 * p.S;      // [1]
  uint64_t* bempty = bfull + 1;          // [1]
  uint64_t* tfull = bempty + 1;          // [2]
  uint64_t* tempty = tfull + 2;          // [2]
  uint64_t* drain = tempty + 2;          // [1] completion of every MMA this CTA issued
  volatile uint32_t* tmem_slot = reinterpret_cast<volatile uint32_t*>(drain + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  volatile int* epi_ok = abort_flag + 1;  // [EWG][2] wait result broadcast inside a warpgroup

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n = p.n, two_n = 2 * n;

  if (threadIdx.x == 0) {
    for (int s = 0; s < p.S; ++s) {
      mbar_init(full + s, 1);
      mbar_init(empty + s, 1);
    }
    mbar_init(bfull, 1);
    mbar_init(bempty, 1);
    for (int b = 0; b < 2; ++b) {
      mbar_init(tfull + b, 1);
      mbar_init(tempty + b, 128 * EWG);  // every epilogue thread arrives
    }
    mbar_init(drain, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(sa((const void*)tmem_slot)),
                 "r"(TC_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const uint32_t tiles_per_item = (uint32_t)p.T;

  if (warp == 0) {
    // ------------------------------------------------------------ producer
    if (lane == 0) {
      int stage = 0;
      uint32_t ph = 0, bph = 0;
      uint32_t last_ph[8];  // parity of the last load issued into each stage (S <= 8)
      bool issued[8] = {false, false, false, false, false, false, false, false};
      bool b_issued = false;
      const uint32_t a_bytes = 2u * 128u * 128u;  // hi + lo, 128 rows x 64 bf16
      const uint32_t b_bytes = 2u * (uint32_t)p.KC * (uint32_t)p.NB * 128u;
      const uint32_t b_slab = 2u * (uint32_t)p.NB * 128u;  // one K slab of B, hi + lo
      for (int item = blockIdx.x; item < p.n_items && !*abort_flag; item += gridDim.x) {
        const int spin = item / p.WG, wg = item % p.WG;
        const int brow = (spin * p.cap + wg * p.Wc) * two_n;
        if constexpr (!SB) {
          if (!mbar_wait(bempty, bph ^ 1)) { atomicOr(p.err, 1); *abort_flag = 1; break; }
          bph ^= 1;
          mbar_expect_tx(bfull, b_bytes);
          b_issued = true;
          for (int kc = 0; kc < p.KC; ++kc) {
            tma_load_2d(sB + (size_t)(0 * p.KC + kc) * p.NB * 128, &tmB_hi, kc * 64, brow, bfull);
            tma_load_2d(sB + (size_t)(1 * p.KC + kc) * p.NB * 128, &tmB_lo, kc * 64, brow, bfull);
          }
        }
        for (uint32_t t = 0; t < tiles_per_item && !*abort_flag; ++t) {
          const int arow = (spin * p.T + (int)t) * 128;
          for (int kc = 0; kc < p.KC; ++kc) {
            if (!mbar_wait(empty + stage, ph ^ 1)) { atomicOr(p.err, 2); *abort_flag = 1; break; }
            mbar_expect_tx(full + stage, SB ? a_bytes + b_slab : a_bytes);
            unsigned char* dst = sA + (size_t)stage * p.sA_stage_bytes;
            tma_load_2d(dst, &tmA_hi, kc * 64, arow, full + stage);
            tma_load_2d(dst + 128 * 128, &tmA_lo, kc * 64, arow, full + stage);
            if constexpr (SB) {
              tma_load_2d(dst + 2 * 128 * 128, &tmB_hi, kc * 64, brow, full + stage);
              tma_load_2d(dst + 2 * 128 * 128 + (size_t)p.NB * 128, &tmB_lo, kc * 64, brow, full + stage);
            }
            issued[stage] = true;
            last_ph[stage] = ph;
            if (++stage == p.S) { stage = 0; ph ^= 1; }
          }
        }
      }
      // let every copy this thread issued land before the CTA can exit (bounded)
      for (int s2 = 0; s2 < p.S; ++s2)
        if (issued[s2]) mbar_wait(full + s2, last_ph[s2]);
      if (b_issued) mbar_wait(bfull, bph ^ 1);
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      int stage = 0, buf = 0;
      uint32_t ph = 0, bph = 0, tph[2] = {0, 0};
      const uint32_t idesc = idesc_bf16(128, p.NB);
      for (int item = blockIdx.x; item < p.n_items && !*abort_flag; item += gridDim.x) {
        if constexpr (!SB) {
          if (!mbar_wait(bfull, bph)) { atomicOr(p.err, 4); *abort_flag = 1; break; }
          bph ^= 1;
          tc_fence_after();
        }
        for (uint32_t t = 0; t < tiles_per_item && !*abort_flag; ++t) {
          if (!mbar_wait(tempty + buf, tph[buf] ^ 1)) { atomicOr(p.err, 8); *abort_flag = 1; break; }
          tc_fence_after();
          const uint32_t d = tmem + (uint32_t)(buf * p.NB);
          for (int kc = 0; kc < p.KC; ++kc) {
            if (!mbar_wait(full + stage, ph)) { atomicOr(p.err, 16); *abort_flag = 1; break; }
            tc_fence_after();
            const uint32_t a_hi = sa(sA + (size_t)stage * p.sA_stage_bytes);
            const uint32_t a_lo = a_hi + 128 * 128;
            const uint32_t b_hi = SB ? a_hi + 2 * 128 * 128 : sa(sB + (size_t)(0 * p.KC + kc) * p.NB * 128);
            const uint32_t b_lo = SB ? b_hi + (uint32_t)p.NB * 128 : sa(sB + (size_t)(1 * p.KC + kc) * p.NB * 128);
#pragma unroll
            for (int k = 0; k < 4; ++k) {  // 4 x K=16 inside the 128-byte swizzle row
              const uint32_t off = k * 32;
              umma(d, sw128_desc(a_hi + off), sw128_desc(b_hi + off), idesc, (kc > 0 || k > 0) ? 1u : 0u);
              umma(d, sw128_desc(a_hi + off), sw128_desc(b_lo + off), idesc, 1u);
              umma(d, sw128_desc(a_lo + off), sw128_desc(b_hi + off), idesc, 1u);
            }
            umma_commit(empty + stage);  // the A stage is free once these MMAs complete
            if (++stage == p.S) { stage = 0; ph ^= 1; }
          }
          umma_commit(tfull + buf);  // accumulator ready for the epilogue
          tph[buf] ^= 1;
          buf ^= 1;
        }
        if constexpr (!SB) umma_commit(bempty);  // B may be overwritten once every MMA of the item is done
      }
      // every MMA issued by this thread has completed before TMEM is released (bounded)
      umma_commit(drain);
      if (!mbar_wait(drain, 0)) atomicOr(p.err, 64);
    }
  } else {
    // ------------------------------------------------------------ epilogue
    const int ewg = (warp - 2) >> 2;                 // epilogue warpgroup 0 / 1
    const int quad = warp & 3;                       // TMEM lane quadrant this warp may read
    const int r = quad * 32 + lane;                  // accumulator row
    const int SP = p.sp;
    const int hs = SP >> 1;                          // staging row stride in float2
    float* st = stg + (size_t)ewg * p.staging_floats;
    int buf = 0;
    uint32_t tph[2] = {0, 0};
    bool go = true;
    // sum_j T_ij T_ji for the thread's row i: T_ij from `own` (registers when
    // NM > 0, else the staged row), T_ji = tcol[j * hs]; eight independent
    // FMA chains (real/imaginary cross terms, even/odd j)
    auto exch = [&](const float* own, const float2* arow, const float2* tcol, float& er, float& ei) {
      float rr0 = 0.f, rr1 = 0.f, ii0 = 0.f, ii1 = 0.f, ri0 = 0.f, ri1 = 0.f, ir0 = 0.f, ir1 = 0.f;
      if constexpr (NM > 0) {
#pragma unroll
        for (int j = 0; j < NM; j += 2) {
          if (j < n) {
            const float2 b0 = tcol[j * hs];
            rr0 = fmaf(own[2 * j], b0.x, rr0);
            ii0 = fmaf(own[2 * j + 1], b0.y, ii0);
            ri0 = fmaf(own[2 * j], b0.y, ri0);
            ir0 = fmaf(own[2 * j + 1], b0.x, ir0);
          }
          if (j + 1 < n) {
            const float2 b1 = tcol[(j + 1) * hs];
            rr1 = fmaf(own[2 * j + 2], b1.x, rr1);
            ii1 = fmaf(own[2 * j + 3], b1.y, ii1);
            ri1 = fmaf(own[2 * j + 2], b1.y, ri1);
            ir1 = fmaf(own[2 * j + 3], b1.x, ir1);
          }
        }
      } else {
        int j = 0;
        for (; j + 1 < n; j += 2) {
          const float2 a0 = arow[j], a1 = arow[j + 1];
          const float2 b0 = tcol[j * hs], b1 = tcol[(j + 1) * hs];
          rr0 = fmaf(a0.x, b0.x, rr0);
          ii0 = fmaf(a0.y, b0.y, ii0);
          ri0 = fmaf(a0.x, b0.y, ri0);
          ir0 = fmaf(a0.y, b0.x, ir0);
          rr1 = fmaf(a1.x, b1.x, rr1);
          ii1 = fmaf(a1.y, b1.y, ii1);
          ri1 = fmaf(a1.x, b1.y, ri1);
          ir1 = fmaf(a1.y, b1.x, ir1);
        }
        if (j < n) {
          const float2 a0 = arow[j];
          const float2 b0 = tcol[j * hs];
          rr0 = fmaf(a0.x, b0.x, rr0);
          ii0 = fmaf(a0.y, b0.y, ii0);
          ri0 = fmaf(a0.x, b0.y, ri0);
          ir0 = fmaf(a0.y, b0.x, ir0);
        }
      }
      er = (rr0 + rr1) - (ii0 + ii1);
      ei = (ri0 + ri1) + (ir0 + ir1);
    };
    if constexpr (WL) {
      // warp slot: rows quad*32 + b*n + i hold block b (g = t*gpt + quad*gpw + b), row i
      const int b = lane / n, i = lane - (lane / n) * n;
      const bool lane_ok = b < p.gpw;
      const int seg_end = (b + 1) * n;                // one past the block's last lane
      float* wst = st + (size_t)quad * 32 * SP;       // this warp's staging rows
      float4* srow = reinterpret_cast<float4*>(wst + lane * SP);
      const float2* tcol = reinterpret_cast<const float2*>(wst + (size_t)(b * n) * SP + 2 * i);  // T[j][i]
      for (int item = blockIdx.x; item < p.n_items && go; item += gridDim.x) {
        const int spin = item / p.WG, wg = item % p.WG;
        for (uint32_t t = 0; t < tiles_per_item; ++t) {
          // lane 0 waits for the accumulator; the warp follows its verdict
          int ok = 1;
          if (lane == 0) {
            ok = mbar_wait(tfull + buf, tph[buf]) ? 1 : 0;
            if (!ok) { atomicOr(p.err, 32); *abort_flag = 1; }
          }
          ok = __shfl_sync(0xffffffffu, ok, 0);
          if (!ok) { go = false; break; }
          tc_fence_after();
          const int g = (int)t * p.gpt + quad * p.gpw + b;
          const bool valid = lane_ok && g < p.G;
          for (int wl = ewg; wl < p.Wc; wl += EWG) {
            const int w = wg * p.Wc + wl;
            if (w >= p.Nw) break;
            // this walker's 2n accumulator columns: (Re T[i][j], Im T[i][j]) for j = 0..n-1
            const uint32_t col0 = (uint32_t)(buf * p.NB + wl * two_n);
            const uint32_t tl = tmem + ((uint32_t)(quad * 32) << 16) + col0;
            float rr[2 * (NM > 0 ? NM : 1)];
#pragma unroll
            for (int c0 = 0; c0 < 2 * NM; c0 += 8)
              if (c0 < two_n) tmem_ld8(tl + (uint32_t)c0, reinterpret_cast<uint32_t*>(rr + c0));
            tmem_wait_ld();
            __syncwarp();  // every lane is past its reads of the previous walker's rows
#pragma unroll
            for (int c0 = 0; c0 < 2 * NM; c0 += 4)
              if (c0 < two_n) srow[c0 >> 2] = make_float4(rr[c0], rr[c0 + 1], rr[c0 + 2], rr[c0 + 3]);
            __syncwarp();
            float tr = 0.f, ti = 0.f, er = 0.f, ei = 0.f;
            if (valid) {
              exch(rr, nullptr, tcol, er, ei);
              const float2 tt = *reinterpret_cast<const float2*>(wst + lane * SP + 2 * i);
              tr = tt.x;
              ti = tt.y;
            }
            // sums over the block's n lanes, collected at its first lane in a fixed tree
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
              const float a0 = __shfl_down_sync(0xffffffffu, tr, off);
              const float a1 = __shfl_down_sync(0xffffffffu, ti, off);
              const float a2 = __shfl_down_sync(0xffffffffu, er, off);
              const float a3 = __shfl_down_sync(0xffffffffu, ei, off);
              if (lane + off < seg_end) {
                tr += a0;
                ti += a1;
                er += a2;
                ei += a3;
              }
            }
            if (valid && i == 0) {
              double* o = p.epart + (((size_t)w * p.G + g) * 2 + spin) * 4;
              o[0] = tr;
              o[1] = ti;
              o[2] = er;
              o[3] = ei;
            }
          }
          tc_fence_before();
          mbar_arrive(tempty + buf);
          tph[buf] ^= 1;
          buf ^= 1;
        }
      }
    } else {
      const int gl = r / n, i = r % n;
      const bool row_ok = gl < p.gpt;
      float* pb = pbuf + ewg * 128 * 4;
      const int bar_id = 1 + ewg;
      uint32_t tcount = 0;  // tiles handled so far (selects the verdict slot)
      // staging row r: 16-byte stores (a row holds 2n values and up to 3
      // padding floats; rows 16-byte aligned, sp / 4 odd: no bank conflicts)
      float4* srow = reinterpret_cast<float4*>(st + r * SP);
      const float2* arow = reinterpret_cast<const float2*>(st + r * SP);
      const float2* tcol = reinterpret_cast<const float2*>(st + (size_t)(gl * n) * SP + 2 * i);  // T[j][i]
      for (int item = blockIdx.x; item < p.n_items && go; item += gridDim.x) {
        const int spin = item / p.WG, wg = item % p.WG;
        for (uint32_t t = 0; t < tiles_per_item; ++t) {
          // one thread waits for the accumulator; the warpgroup follows its
          // verdict (two slots alternating with every tile the warpgroup
          // handles: a slot is rewritten two tiles later, after every thread
          // has passed the barrier of the tile in between)
          if (r == 0) {
            const bool ok = mbar_wait(tfull + buf, tph[buf]);
            if (!ok) { atomicOr(p.err, 32); *abort_flag = 1; }
            epi_ok[2 * ewg + (tcount & 1)] = ok ? 1 : 0;
          }
          named_bar(bar_id, 128);
          const int ok = epi_ok[2 * ewg + (tcount & 1)];
          ++tcount;
          if (!ok) { go = false; break; }
          tc_fence_after();
          const int g = (int)t * p.gpt + gl;
          const bool valid = row_ok && g < p.G;
          for (int wl = ewg; wl < p.Wc; wl += EWG) {
            const int w = wg * p.Wc + wl;
            if (w >= p.Nw) break;
            const uint32_t col0 = (uint32_t)(buf * p.NB + wl * two_n);
            const uint32_t tl = tmem + ((uint32_t)(quad * 32) << 16) + col0;
            float rr[2 * (NM > 0 ? NM : 1)];
            if constexpr (NM > 0) {
#pragma unroll
              for (int c0 = 0; c0 < 2 * NM; c0 += 8)
                if (c0 < two_n) tmem_ld8(tl + (uint32_t)c0, reinterpret_cast<uint32_t*>(rr + c0));
              tmem_wait_ld();
#pragma unroll
              for (int c0 = 0; c0 < 2 * NM; c0 += 4)
                if (c0 < two_n) srow[c0 >> 2] = make_float4(rr[c0], rr[c0 + 1], rr[c0 + 2], rr[c0 + 3]);
            } else {
              for (int c0 = 0; c0 < two_n; c0 += 8) {
                uint32_t v[8];
                tmem_ld8(tl + (uint32_t)c0, v);
                tmem_wait_ld();
                srow[c0 >> 2] = make_float4(__uint_as_float(v[0]), __uint_as_float(v[1]), __uint_as_float(v[2]),
                                            __uint_as_float(v[3]));
                if (c0 + 4 < two_n)
                  srow[(c0 >> 2) + 1] = make_float4(__uint_as_float(v[4]), __uint_as_float(v[5]),
                                                    __uint_as_float(v[6]), __uint_as_float(v[7]));
              }
            }
            named_bar(bar_id, 128);
            float tr = 0.f, ti = 0.f, er = 0.f, ei = 0.f;
            if (valid) {
              exch(rr, arow, tcol, er, ei);
              const float2 tt = arow[i];
              tr = tt.x;
              ti = tt.y;
            }
            reinterpret_cast<float4*>(pb)[r] = make_float4(tr, ti, er, ei);
            named_bar(bar_id, 128);
            // (g block, quantity) sums over the block's n rows: four lanes per
            // pair each add every fourth row, then two shuffles combine them in a
            // fixed order.  Whole warps run the loop (its bound is warp-uniform).
            const int nthr = 16 * p.gpt;
            for (int x0 = quad * 32; x0 < nthr; x0 += 128) {
              const int x = x0 + lane;
              const int pair = x >> 2, part = x & 3;
              const int gb = pair >> 2, qn = pair & 3;
              float sum = 0.f;
              if (x < nthr)
                for (int ii = part; ii < n; ii += 4) sum += pb[(gb * n + ii) * 4 + qn];
              sum += __shfl_xor_sync(0xffffffffu, sum, 1);
              sum += __shfl_xor_sync(0xffffffffu, sum, 2);
              const int gg = (int)t * p.gpt + gb;
              if (x < nthr && part == 0 && gg < p.G) p.epart[(((size_t)w * p.G + gg) * 2 + spin) * 4 + qn] = sum;
            }
            // no barrier here: the next walker's staging writes come after the barrier
            // above (every thread is past its staging reads) and its row partials after
            // the next walker's first barrier (every thread is past this tail)
          }
          tc_fence_before();
          mbar_arrive(tempty + buf);
          tph[buf] ^= 1;
          buf ^= 1;
        }
      }
    }
  }
  // ------------------------------------------------------------ teardown
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    __syncwarp();
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_TMEM_COLS) : "memory");
  }
}

// A operand: [2 spins][T][128 rows][Kp] from Lh[G][nc][N].  Rows of tile t:
// gpw > 0: row slot*32 + b*n + i = row i of g = t*gpt + slot*gpw + b (b < gpw,
// other rows zero); gpw == 0: row gg*n + i = row i of g = t*gpt + gg.
__global__ void build_lh_tiles_kernel(const double* __restrict__ Lh, __nv_bfloat16* __restrict__ hi,
                                      __nv_bfloat16* __restrict__ lo, int N, int n, int nc, int G, int gpt, int gpw,
                                      int T, int Kp) {
  const size_t total = (size_t)2 * T * 128 * Kp;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int q = e % Kp;
    const int r = (e / Kp) % 128;
    const int t = (e / ((size_t)Kp * 128)) % T;
    const int spin = (int)(e / ((size_t)Kp * 128 * T));
    int gg, i;
    bool in_block;
    if (gpw > 0) {
      const int slot = r >> 5, b = (r & 31) / n;
      i = (r & 31) - b * n;
      gg = slot * gpw + b;
      in_block = b < gpw;
    } else {
      gg = r / n;
      i = r % n;
      in_block = gg < gpt;
    }
    const int g = t * gpt + gg;
    double x = 0.0;
    if (in_block && g < G && q < N) x = Lh[((size_t)g * nc + spin * n + i) * N + q];
    split_bf16(x, hi[e], lo[e]);
  }
}

// B operand: [2 spins][cap][n][re,im][Kp] from Theta[Nw][nc][N] (complex64).
// One thread per 8 consecutive q of one (spin, walker, orbital): eight
// complex loads, four 16-byte stores (Re hi, Re lo, Im hi, Im lo).
__global__ void build_theta_planes_kernel(const float2* __restrict__ theta, __nv_bfloat16* __restrict__ hi,
                                          __nv_bfloat16* __restrict__ lo, int N, int n, int Nw, int cap, int Kp) {
  const int kq = Kp / 8;
  const size_t units = (size_t)2 * Nw * n * kq;
  for (size_t u = blockIdx.x * (size_t)blockDim.x + threadIdx.x; u < units; u += (size_t)gridDim.x * blockDim.x) {
    const int qc = (int)(u % kq);
    const size_t rest = u / kq;
    const int j = (int)(rest % n);
    const size_t rw = rest / n;
    const size_t w = rw % Nw;
    const int spin = (int)(rw / Nw);
    const float2* src = theta + (w * 2 * n + (size_t)spin * n + j) * N;
    __align__(16) __nv_bfloat16 rh[8], rl[8], ih[8], il[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      const int q = qc * 8 + t;
      const float2 v = q < N ? src[q] : make_float2(0.f, 0.f);
      rh[t] = __float2bfloat16(v.x);
      rl[t] = __float2bfloat16(v.x - __bfloat162float(rh[t]));
      ih[t] = __float2bfloat16(v.y);
      il[t] = __float2bfloat16(v.y - __bfloat162float(ih[t]));
    }
    const size_t row = ((size_t)spin * cap + w) * 2 * n + 2 * (size_t)j;  // rows (j, re) and (j, im)
    const size_t o_re = row * Kp + (size_t)qc * 8, o_im = o_re + Kp;
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

// Staging row stride in floats: at least 2n + 1, a multiple of 4 (16-byte
// rows) with an odd number of 16-byte chunks, so that the eight rows of one
// 16-byte store wavefront fall on distinct bank groups.
int tc_stage_stride(int n) {
  int m = (2 * n + 1 + 3) / 4;
  if ((m & 1) == 0) ++m;
  return 4 * m;
}

size_t tc_smem_bytes(int KC, int NB, int S, int n, int ewg, bool sb) {
  const size_t stg = (size_t)ewg * 128 * tc_stage_stride(n) * 4;
  const size_t resident_b = sb ? 0 : (size_t)2 * KC * NB * 128;
  const size_t stage = (size_t)2 * 128 * 128 + (sb ? (size_t)2 * NB * 128 : 0);
  return 1024 + resident_b + (size_t)S * stage + stg + (size_t)ewg * 128 * 4 * 4 + (size_t)(2 * S + 7) * 8 + 16 +
         8 * ewg;
}

template <int NM, int EWG, bool SB, bool WL>
void* exchange_fn() {
  return reinterpret_cast<void*>(exchange_tc_kernel<NM, EWG, SB, WL>);
}

// kernel instance for (n, epilogue warpgroups, streamed B, warp-slot rows)
void* exchange_instance(int n, int ewg, bool sb, bool wl) {
  const int nm = n <= 16 ? 16 : n <= 24 ? 24 : n <= 32 ? 32 : 0;
#define AFQ_X2(NM, WL)                                                                            \
  if (ewg == 2) return sb ? exchange_fn<NM, 2, true, WL>() : exchange_fn<NM, 2, false, WL>(); \
  return sb ? exchange_fn<NM, 1, true, WL>() : exchange_fn<NM, 1, false, WL>();
#define AFQ_X(NM)            \
  if (nm == NM) {            \
    if (wl) {                \
      AFQ_X2(NM, true)       \
    } else {                 \
      AFQ_X2(NM, false)      \
    }                        \
  }
  AFQ_X(16)
  AFQ_X(24)
  AFQ_X(32)
#undef AFQ_X
  if (nm == 0) {
    if (wl) return nullptr;
    AFQ_X2(0, false)
  }
#undef AFQ_X2
  return nullptr;
}

}  // namespace

// Plan the tensor-core exchange for a context; false when the shape is outside
// what the kernel handles (then the SIMT kernel runs).
bool tc_exchange_plan(afqmc_ctx* c) {
  TcPlan& P = c->tc;
  P = TcPlan();
  if (c->prec != AFQMC_MIXED || c->na != c->nb || c->na < 1) return false;
  const int n = c->na;
  const int Kp = ((c->N + 63) / 64) * 64;
  const int KC = Kp / 64;
  if (n > 64) return false;
  // whole g blocks per 32-row warp slot (n <= 32) where that puts as many g
  // in a tile as packing them across the tile does; else packed
  const int gpw = (n <= 32 && 4 * (32 / n) >= 128 / n) ? 32 / n : 0;
  const int gpt = gpw > 0 ? 4 * gpw : 128 / n;
  const size_t budget = 232448 - 1024;
  // preference: B resident with two epilogue warpgroups, then B streamed with
  // two, then with one (large N or n)
  const struct { int ewg; bool sb; } modes[] = {{2, false}, {2, true}, {1, true}};
  int best_wc = 0, best_nb = 0, best_s = 0, best_ewg = 0;
  bool best_sb = false;
  for (const auto& md : modes) {
    for (int S = 3; S >= 2 && !best_wc; --S)
      for (int wc = 256 / (2 * n); wc >= 1; --wc) {
        const int nb = ((wc * 2 * n + 15) / 16) * 16;
        if (nb > 240) continue;  // two accumulators plus the 8-column read granularity stay inside 512 columns
        if (tc_smem_bytes(KC, nb, S, n, md.ewg, md.sb) <= budget) {
          best_wc = wc;
          best_nb = nb;
          best_s = S;
          best_ewg = md.ewg;
          best_sb = md.sb;
          break;
        }
      }
    if (best_wc) break;
  }
  if (!best_wc) return false;
  P.ok = true;
  P.n = n;
  P.gpt = gpt;
  P.gpw = gpw;
  P.T = (c->G + gpt - 1) / gpt;
  P.Kp = Kp;
  P.KC = KC;
  P.Wc = best_wc;
  P.NB = best_nb;
  P.S = best_s;
  P.ewg = best_ewg;
  P.sb = best_sb;
  return true;
}

// Build the split A tiles (once per context) and their tensor maps.
cudaError_t tc_exchange_setup(afqmc_ctx* c, cudaStream_t s) {
  TcPlan& P = c->tc;
  const size_t elems = (size_t)2 * P.T * 128 * P.Kp;
  cudaError_t e = dmalloc(&P.a_hi, elems * 2);
  if (e != cudaSuccess) return e;
  e = dmalloc(&P.a_lo, elems * 2);
  if (e != cudaSuccess) return e;
  e = dmalloc(&P.err, sizeof(int));
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(P.err, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  build_lh_tiles_kernel<<<grid_for(elems), 256, 0, s>>>(c->d_Lh, static_cast<__nv_bfloat16*>(P.a_hi),
                                                        static_cast<__nv_bfloat16*>(P.a_lo), c->N, P.n, c->nc, c->G,
                                                        P.gpt, P.gpw, P.T, P.Kp);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (!make_map(reinterpret_cast<CUtensorMap*>(P.map_a_hi), P.a_hi, (size_t)2 * P.T * 128, P.Kp, 128) ||
      !make_map(reinterpret_cast<CUtensorMap*>(P.map_a_lo), P.a_lo, (size_t)2 * P.T * 128, P.Kp, 128))
    return cudaErrorInvalidValue;
  return cudaSuccess;
}

// Bytes of one split Theta plane (hi or lo) for `cap` walkers.
size_t tc_exchange_plane_bytes(const TcPlan& P, int cap) { return (size_t)2 * cap * 2 * P.n * P.Kp * 2; }

// Point the plan at caller-provided Theta planes for `cap` walkers and encode
// their tensor maps (no allocation).
cudaError_t tc_exchange_bind(TcPlan& P, void* b_hi, void* b_lo, int cap) {
  P.b_hi = b_hi;
  P.b_lo = b_lo;
  P.b_cap = 0;
  if (!make_map(reinterpret_cast<CUtensorMap*>(P.map_b_hi), b_hi, (size_t)2 * cap * 2 * P.n, P.Kp, P.NB) ||
      !make_map(reinterpret_cast<CUtensorMap*>(P.map_b_lo), b_lo, (size_t)2 * cap * 2 * P.n, P.Kp, P.NB))
    return cudaErrorInvalidValue;
  P.b_cap = cap;
  return cudaSuccess;
}

// (Re)allocate the split Theta planes for the workspace's walker capacity.
cudaError_t tc_exchange_ws(afqmc_ctx* c) {
  AllocScope alloc_scope(AG_PLANES);
  TcPlan& P = c->tc;
  if (P.b_hi) cudaFree(P.b_hi);
  if (P.b_lo) cudaFree(P.b_lo);
  P.b_hi = P.b_lo = nullptr;
  P.b_cap = 0;
  const int cap = c->ws.n_walkers;
  void *hi = nullptr, *lo = nullptr;
  cudaError_t e = dmalloc(&hi, tc_exchange_plane_bytes(P, cap));
  if (e != cudaSuccess) return e;
  P.b_hi = hi;
  e = dmalloc(&lo, tc_exchange_plane_bytes(P, cap));
  if (e != cudaSuccess) return e;
  P.b_lo = lo;
  return tc_exchange_bind(P, hi, lo, cap);
}

cudaError_t tc_exchange_prepare(const afqmc_ctx* c) {
  const TcPlan& P = c->tc;
  if (!P.ok) return cudaSuccess;
  void* f = exchange_instance(P.n, P.ewg, P.sb, P.gpw > 0);
  cudaFuncAttributes a;
  cudaError_t e = cudaFuncGetAttributes(&a, f);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, max_dyn_smem() - (int)a.sharedSizeBytes);
}

void tc_exchange_free(afqmc_ctx* c) {
  TcPlan& P = c->tc;
  void* ptrs[] = {P.a_hi, P.a_lo, P.b_hi, P.b_lo, P.err};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  P = TcPlan();
}

// Theta planes (split bf16) for Nw walkers.
cudaError_t tc_exchange_planes(afqmc_ctx* c, int Nw, const void* theta, cudaStream_t s) {
  TcPlan& P = c->tc;
  // the B tensor map spans the allocated capacity; planes beyond Nw are ignored
  if (Nw > P.b_cap) return cudaErrorInvalidValue;
  const size_t units = (size_t)2 * Nw * P.n * (P.Kp / 8);
  build_theta_planes_kernel<<<grid_for(units), 256, 0, s>>>(static_cast<const float2*>(theta),
                                                            static_cast<__nv_bfloat16*>(P.b_hi),
                                                            static_cast<__nv_bfloat16*>(P.b_lo), c->N, P.n, Nw,
                                                            P.b_cap, P.Kp);
  return cudaGetLastError();
}

// The tensor-core contraction for Nw walkers from the planes; writes epart.
cudaError_t tc_exchange_contract(afqmc_ctx* c, int Nw, double* epart, cudaStream_t s) {
  TcPlan& P = c->tc;
  if (Nw > P.b_cap) return cudaErrorInvalidValue;
  cudaError_t e;
  TcArgs a;
  a.n = P.n;
  a.gpt = P.gpt;
  a.gpw = P.gpw;
  a.T = P.T;
  a.KC = P.KC;
  a.NB = P.NB;
  a.Wc = P.Wc;
  a.WG = (Nw + P.Wc - 1) / P.Wc;
  a.Nw = Nw;
  a.cap = P.b_cap;
  a.G = c->G;
  a.S = P.S;
  a.n_items = 2 * a.WG;
  a.sB_bytes = P.sb ? 0u : (uint32_t)(2 * P.KC * P.NB * 128);
  a.sA_stage_bytes = 2 * 128 * 128 + (P.sb ? 2 * P.NB * 128 : 0);
  a.sp = tc_stage_stride(P.n);
  a.staging_floats = (uint32_t)(128 * a.sp);
  a.epart = epart;
  a.err = static_cast<int*>(P.err);
  const size_t shm = tc_smem_bytes(P.KC, P.NB, P.S, P.n, P.ewg, P.sb);
  if (!capturing(c)) {
    e = tc_exchange_prepare(c);
    if (e != cudaSuccess) return e;
  }
  int sms = 152;
  int dev = 0;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int grid = a.n_items < sms ? a.n_items : sms;
  CUtensorMap mah, mal, mbh, mbl;
  memcpy(&mah, P.map_a_hi, sizeof(CUtensorMap));
  memcpy(&mal, P.map_a_lo, sizeof(CUtensorMap));
  memcpy(&mbh, P.map_b_hi, sizeof(CUtensorMap));
  memcpy(&mbl, P.map_b_lo, sizeof(CUtensorMap));
  void* f = exchange_instance(P.n, P.ewg, P.sb, P.gpw > 0);
  void* args[] = {&mah, &mal, &mbh, &mbl, &a};
  e = cudaLaunchKernel(f, dim3(grid), dim3(64 + 128 * P.ewg), args, shm, s);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

}  // namespace afq
