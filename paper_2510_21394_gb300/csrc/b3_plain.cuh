// Plain split-BF16 mu-mode product Y = split(M X) (Sec. 3.2, one mode product),
// the inner step of every Tucker operator that carries no pointwise stage.
//
// Same GEMM orientation, tile shape and arithmetic as mp_b3_kernel
// (b3_kernel.cuh): 128 output indices i x (64 r of the real plane + the same
// 64 r of the imaginary plane) per unit, M_hi X_hi + M_hi X_lo + M_lo X_hi into
// an FP32 TMEM accumulator.  It differs in how the operands are streamed:
// the 128 x 64 chunks of M (L2-resident) and the 128-row chunks of X (from
// HBM) travel in two separate shared-memory rings with their own producers,
// so the X ring can be deeper than the M ring.  The epilogue splits the FP32
// accumulator into hi and lo bf16 and stores 32 x 32 boxes through TMA.
//
// Warp roles (one CTA per SM, persistent over (r-tile, i-block)):
//   warp 0      X producer (TMA, SWIZZLE_128B)
//   warp 1      TMEM allocator and single-thread MMA issuer
//   warp 2      M producer (TMA, SWIZZLE_128B)
//   warps 3-10  epilogue; warp w reads TMEM lane quarter w % 4 and the two
//               adjacent 16-column groups 2 h, 2 h + 1 with h = (w - 3) / 4,
//               and stores them as 32 x 32 boxes (64-byte rows).
// Every mbarrier wait is bounded (mbar_wait); on expiry the CTA records an
// error code, drains its own TMA and MMA work, frees its TMEM and returns.
//
// Requirement (checked by the host): R % 8 == 0, the 16-byte row-pitch rule
// of the output tensor maps.
//
// Grouped form (G = true): one persistent launch serves the plain mode
// products of several independent problems (the instances of a batch); the
// tensor maps and sizes of problem k come from the descriptor gd[k], which
// owns the global units [gd[k].ubegin, gd[k + 1].ubegin).  The arithmetic per
// unit is the same as in the single form.
//
// Operand formats (OP):
//   kOpBF16   split-BF16 in and out: x = hi + lo, two bf16 each; products
//             hi.hi + hi.lo + lo.hi with tcgen05.mma kind::f16 (K = 16).
//   kOpTF32   split-TF32 in and out: x = hi + lo, two FP32 words each holding
//             a TF32 value (hi = x rounded to TF32, lo = x - hi rounded to
//             TF32, about 21 significant bits together); the same three
//             products with kind::tf32 (K = 8).  A 128-byte shared-memory row
//             holds 32 TF32 values instead of 64 bf16, so a k-chunk is 32 wide
//             and every stage, box and descriptor keeps its byte layout.
//   kOpTF32F  split-TF32 in, plain FP32 out (the last product of a Tucker
//             operator whose result is an FP32 tensor).
// The TF32 forms serve the precise transforms at the two ends of a time
// integration, where the split-BF16 error (about 2^-17 per product) must not
// enter the state.
//
// Resident-M form (MR = true, single form only): when the grid is a multiple
// of m_blocks every CTA works on one fixed i-block (u = blockIdx.x + j gridDim.x
// keeps u % m_blocks), so with k_chunks <= 4 (p <= 256 for bf16) the CTA loads
// its 128 x p block of M once, into a 128 KB resident region, instead of
// streaming it from L2 for every unit; the X ring is then 2 deep.  This halves
// the operand bytes each SM pulls through L2 per unit at p = 256.
#pragma once

#include "b3_kernel.cuh"

namespace fcgle {
namespace b3 {

constexpr int kOpBF16 = 0, kOpTF32 = 1, kOpTF32F = 2;

// elements of one 128-byte operand row (the k extent of a chunk)
template <int OP>
constexpr int chunk_k() { return OP == kOpBF16 ? 64 : 32; }

constexpr int PL_NX = 4;                   // X ring depth
constexpr int PL_NM = 2;                   // M ring depth
constexpr int PL_NEPI = 8;                 // epilogue warps
constexpr int PL_THREADS = 32 * (3 + PL_NEPI);
constexpr uint32_t kXStage = 32768;        // X_hi (r0 | r1) 16K | X_lo (r0 | r1) 16K
constexpr uint32_t kMStage = 32768;        // M_hi 16K | M_lo 16K
constexpr uint32_t kPlOffM = PL_NX * kXStage;
constexpr uint32_t kPlOffEpi = kPlOffM + PL_NM * kMStage;
constexpr uint32_t kPlEpiWarp = 4096;      // two 32 x 32 bf16 boxes (hi, lo of one component)
constexpr uint32_t kPlOffBar = kPlOffEpi + PL_NEPI * kPlEpiWarp;
constexpr uint32_t kPlSmemBytes = kPlOffBar + 256 + 1024;   // + barriers + alignment slack
static_assert(kPlSmemBytes <= 232448, "shared memory budget");

// one problem of a grouped plain launch (aligned as its tensor maps)
struct PlainDesc {
  CUtensorMap xhi, xlo, mhi, mlo, yhi, ylo;
  KParams kp;
  long long ubegin;
};

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accum) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum)
      : "memory");
}
// x rounded to TF32 (10 explicit mantissa bits, ties away from zero), as an FP32 word
__device__ __forceinline__ float tf32_round(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

constexpr int kMRMaxChunks = 4;   // resident M: up to 4 chunks of 32 KB
constexpr int kMaxRing = 4;       // barrier slots per ring

// Ring configurations (X ring depth NXR; the M ring takes the rest of the
// 192 KB operand area, or the resident region when MR, single form only):
//   NXR = 4: X 4 x 32 KB + M 2 x 32 KB (the default, and the grouped form)
//   NXR = 3: X 3 + M 3;  NXR = 2: X 2 + M 4 (long k extents: more M in flight)
//   MR:      X 2 + resident M (p <= 256)
//   MH:      X 3 + resident M_hi (4 x 16 KB) + M_lo ring 2 x 16 KB (p <= 256):
//            a third less operand traffic per unit than streaming M, one X
//            stage more than MR
//   CX:      the complex (Kronecker-product exponential) form: M = Er + i Ei,
//            an M stage carries Er_hi, Er_lo, Ei_hi, Ei_lo (64 KB); X 2 + M 2
//            (the products are those of the complex fused form, b3_kernel.cuh)
//   W = 2:   wide tiles (single form, split-BF16): 128 r of each plane per
//            unit, MMA N = 256, X stages of 64 KB (X 2 + M 2), two 256-column
//            accumulators.  Every 32 KB chunk of M then feeds twice the MMA
//            work, so a unit pulls 3/4 of the operand bytes per flop that a
//            64-r unit does; the TMA ingest of an SM is what bounds the
//            product at p = 256.
template <bool G, int OP = kOpBF16, int NXR = PL_NX, bool MR = false, bool CX = false, bool MH = false, int W = 1>
__global__ void __launch_bounds__(PL_THREADS, 1)
    mp_b3_plain_kernel(const __grid_constant__ CUtensorMap tm_xhi, const __grid_constant__ CUtensorMap tm_xlo,
                       const __grid_constant__ CUtensorMap tm_mhi, const __grid_constant__ CUtensorMap tm_mlo,
                       const __grid_constant__ CUtensorMap tm_yhi, const __grid_constant__ CUtensorMap tm_ylo,
                       const KParams kp, const PlainDesc* __restrict__ gd, int ngd, long long gunits) {
  static_assert(!(G && (MR || CX || MH)), "the grouped form streams M through a ring");
  static_assert(!(CX && (MR || MH || OP != kOpBF16)), "the complex form is split-BF16 with M rings");
  static_assert(!(MH && (MR || OP != kOpBF16)), "resident M_hi is a split-BF16 form of its own");
  static_assert(W == 1 || (W == 2 && !G && !MR && !CX && !MH && OP == kOpBF16 && NXR == 2),
                "wide tiles: single split-BF16 form, X 2 + M 2");
  constexpr int WR = W * BR;                              // r of each plane per unit
  constexpr uint32_t kXSt = W * kXStage;                  // bytes per X ring stage
  // X ring depth and the offset of the M region (ring or resident); the
  // epilogue staging area starts at the same offset in every configuration
  constexpr uint32_t kHalf = kMStage / 2;                 // one 128 x 64 bf16 box (hi or lo)
  constexpr uint32_t kMSt = CX ? 2 * kMStage : (MH ? kHalf : kMStage);   // bytes per M ring stage
  constexpr int NX = (MR || CX) ? 2 : (MH ? 3 : NXR);
  constexpr int NM = MR ? kMRMaxChunks : (MH ? 2 : (int)((kPlOffEpi - NX * kXSt) / kMSt));
  constexpr uint32_t kOffM = NX * kXSt;
  constexpr uint32_t kOffMlo = kOffM + kMRMaxChunks * kHalf;   // MH: the M_lo ring after the resident M_hi
  static_assert(NX >= 2 && NX <= kMaxRing && NM >= 2 && NM <= kMaxRing - (MH ? 1 : 0), "ring depths");
  static_assert((MH ? kOffMlo : kOffM) + NM * kMSt == kPlOffEpi, "shared memory layout");
  extern __shared__ uint8_t smem_raw[];
  pdl_trigger();
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const uint32_t sbase = smem_u32(smem);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + kPlOffBar);
  auto full_x = [&](int s) { return smem_u32(&bars[s]); };
  auto empty_x = [&](int s) { return smem_u32(&bars[kMaxRing + s]); };
  auto full_m = [&](int s) { return smem_u32(&bars[2 * kMaxRing + s]); };
  auto empty_m = [&](int s) { return smem_u32(&bars[3 * kMaxRing + s]); };
  auto acc_full = [&](int a) { return smem_u32(&bars[4 * kMaxRing + a]); };
  auto acc_empty = [&](int a) { return smem_u32(&bars[4 * kMaxRing + 2 + a]); };
  const uint32_t fin_bar = smem_u32(&bars[4 * kMaxRing + 4]);
  static_assert((4 * kMaxRing + 5) * 8 <= 192, "barrier area");
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + kPlOffBar + 192);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + kPlOffBar + 200);

  if (threadIdx.x == 0) {
    for (int s = 0; s < kMaxRing; ++s) {
      mbar_init(full_x(s), 1);
      mbar_init(empty_x(s), 1);
      mbar_init(full_m(s), 1);
      mbar_init(empty_m(s), 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(acc_full(a), 1);
      mbar_init(acc_empty(a), PL_NEPI);
    }
    mbar_init(fin_bar, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(2 * W * BN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;
  pdl_wait();

  long long units;
  int* err;
  if constexpr (G) {
    units = gunits;
    err = gd[0].kp.err;
  } else {
    units = kp.tiles * kp.m_blocks;
    err = kp.err;
  }

  if (warp == 0) {
    // ------------------------------------------------------------ X producer
    if (lane == 0) {
      uint32_t g = 0;
      bool ok = true;
      int pid = 0;
      for (long long u = blockIdx.x; u < units && ok; u += gridDim.x) {
        long long lu = u, R = kp.R;
        int mbk = kp.m_blocks, KC = kp.k_chunks;
        const CUtensorMap *mxh = &tm_xhi, *mxl = &tm_xlo;
        if constexpr (G) {
          lu = locate(gd, ngd, u, pid);
          R = gd[pid].kp.R;
          mbk = gd[pid].kp.m_blocks;
          KC = gd[pid].kp.k_chunks;
          mxh = &gd[pid].xhi;
          mxl = &gd[pid].xlo;
        }
        const long long tile = lu / mbk;
        const int r0 = (int)(tile * WR);
        const int r1 = (int)(R + tile * WR);   // same r in the imaginary plane
        for (int kc = 0; kc < KC; ++kc, ++g) {
          const int s = (int)(g % NX);
          if (!mbar_wait(empty_x(s), ((g / NX) & 1) ^ 1, abort_flag, err, 11)) { ok = false; break; }
          const uint32_t st = sbase + s * kXSt;
          mbar_arrive_tx(full_x(s), kXSt);
          constexpr int CK = chunk_k<OP>();
          // boxes of WR rows: X_hi re | X_hi im | X_lo re | X_lo im
          tma_load_2d(st, mxh, kc * CK, r0, full_x(s));
          tma_load_2d(st + W * 8192, mxh, kc * CK, r1, full_x(s));
          tma_load_2d(st + W * 16384, mxl, kc * CK, r0, full_x(s));
          tma_load_2d(st + W * 24576, mxl, kc * CK, r1, full_x(s));
        }
      }
      const uint32_t issued = g;
      for (uint32_t q = issued >= (uint32_t)NX ? issued - NX : 0; q < issued; ++q)
        mbar_wait(full_x(q % NX), (q / NX) & 1, abort_flag, err, 17, true);
    }
  } else if (warp == 2) {
    // ------------------------------------------------------------ M producer
    if (MR && lane == 0) {
      // the CTA's fixed i-block of M, all k-chunks, loaded once
      if ((long long)blockIdx.x < units) {
        const int mb = (int)(blockIdx.x % kp.m_blocks);
        constexpr int CK = chunk_k<OP>();
        mbar_arrive_tx(full_m(0), (uint32_t)kp.k_chunks * kMStage);
        for (int kc = 0; kc < kp.k_chunks; ++kc) {
          const uint32_t st = sbase + kOffM + kc * kMStage;
          tma_load_2d(st, &tm_mhi, kc * CK, mb * BM, full_m(0));
          tma_load_2d(st + 16384, &tm_mlo, kc * CK, mb * BM, full_m(0));
        }
        mbar_wait(full_m(0), 0, abort_flag, err, 18, true);
      }
    } else if (lane == 0) {
      uint32_t g = 0;
      bool ok = true;
      int pid = 0;
      if (MH && (long long)blockIdx.x < units) {
        // the CTA's fixed i-block of M_hi, all k-chunks, loaded once (barrier slot 3)
        const int mb = (int)(blockIdx.x % kp.m_blocks);
        constexpr int CK = chunk_k<OP>();
        mbar_arrive_tx(full_m(kMaxRing - 1), (uint32_t)kp.k_chunks * kHalf);
        for (int kc = 0; kc < kp.k_chunks; ++kc)
          tma_load_2d(sbase + kOffM + kc * kHalf, &tm_mhi, kc * CK, mb * BM, full_m(kMaxRing - 1));
      }
      for (long long u = blockIdx.x; u < units && ok; u += gridDim.x) {
        long long lu = u;
        int mbk = kp.m_blocks, KC = kp.k_chunks;
        const CUtensorMap *mmh = &tm_mhi, *mml = &tm_mlo;
        if constexpr (G) {
          lu = locate(gd, ngd, u, pid);
          mbk = gd[pid].kp.m_blocks;
          KC = gd[pid].kp.k_chunks;
          mmh = &gd[pid].mhi;
          mml = &gd[pid].mlo;
        }
        const int mb = (int)(lu % mbk);
        for (int kc = 0; kc < KC; ++kc, ++g) {
          const int s = (int)(g % NM);
          if (!mbar_wait(empty_m(s), ((g / NM) & 1) ^ 1, abort_flag, err, 12)) { ok = false; break; }
          constexpr int CK = chunk_k<OP>();
          if constexpr (MH) {   // the M_lo ring only
            const uint32_t st = sbase + kOffMlo + s * kMSt;
            mbar_arrive_tx(full_m(s), kMSt);
            tma_load_2d(st, mml, kc * CK, mb * BM, full_m(s));
            continue;
          }
          const uint32_t st = sbase + kOffM + s * kMSt;
          mbar_arrive_tx(full_m(s), kMSt);
          tma_load_2d(st, mmh, kc * CK, mb * BM, full_m(s));
          tma_load_2d(st + 16384, mml, kc * CK, mb * BM, full_m(s));
          if constexpr (CX) {
            tma_load_2d(st + 32768, mmh, kc * CK, kp.ei_row + mb * BM, full_m(s));
            tma_load_2d(st + 49152, mml, kc * CK, kp.ei_row + mb * BM, full_m(s));
          }
        }
      }
      const uint32_t issued = g;
      for (uint32_t q = issued >= (uint32_t)NM ? issued - NM : 0; q < issued; ++q)
        mbar_wait(full_m(q % NM), (q / NM) & 1, abort_flag, err, 18, true);
      if (MH && (long long)blockIdx.x < units) mbar_wait(full_m(kMaxRing - 1), 0, abort_flag, err, 18, true);
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      // instruction descriptor: FP32 accumulator; A, B bf16 (1) or tf32 (2); K-major; N, M
      constexpr uint32_t kAB = OP == kOpBF16 ? 1u : 2u;
      constexpr uint32_t idesc = (1u << 4) | (kAB << 7) | (kAB << 10) | ((uint32_t)(W * BN >> 3) << 17) |
                                 ((uint32_t)(BM >> 4) << 24);
      constexpr uint32_t idesc64 = (1u << 4) | (kAB << 7) | (kAB << 10) | ((uint32_t)(BR >> 3) << 17) |
                                   ((uint32_t)(BM >> 4) << 24);
      uint32_t g = 0, t = 0;
      bool ok = true;
      int pid = 0;
      if (MR && (long long)blockIdx.x < units) ok = mbar_wait(full_m(0), 0, abort_flag, err, 14);
      if (MH && (long long)blockIdx.x < units) ok = mbar_wait(full_m(kMaxRing - 1), 0, abort_flag, err, 14);
      for (long long u = blockIdx.x; u < units && ok; u += gridDim.x, ++t) {
        int KC = kp.k_chunks;
        if constexpr (G) {
          locate(gd, ngd, u, pid);
          KC = gd[pid].kp.k_chunks;
        }
        const int a = t & 1;
        if (!mbar_wait(acc_empty(a), ((t >> 1) & 1) ^ 1, abort_flag, err, 13)) break;
        tc_fence_after();
        const uint32_t d_tmem = tmem_base + a * W * BN;
        for (int kc = 0; kc < KC; ++kc, ++g) {
          const int sx = (int)(g % NX), sm = MR ? kc : (int)(g % NM);
          if (!MR && !mbar_wait(full_m(sm), (g / NM) & 1, abort_flag, err, 14)) { ok = false; break; }
          if (!mbar_wait(full_x(sx), (g / NX) & 1, abort_flag, err, 15)) { ok = false; break; }
          tc_fence_after();
          const uint32_t ahi = MH ? sbase + kOffM + kc * kHalf : sbase + kOffM + sm * kMSt;
          const uint32_t alo = MH ? sbase + kOffMlo + sm * kMSt : ahi + 16384;
          const uint32_t bhi = sbase + sx * kXSt, blo = bhi + W * 16384;
          // four k-steps of 32 bytes per 128-byte row (K = 16 bf16 or 8 tf32 each)
#pragma unroll
          for (int ks = 0; ks < 4; ++ks) {
            const uint32_t off = ks * 32;
            const uint32_t acc0 = (kc > 0 || ks > 0) ? 1u : 0u;
            if constexpr (OP == kOpBF16) {
              mma_bf16(d_tmem, sw128_desc(ahi + off), sw128_desc(bhi + off), idesc, acc0);
              mma_bf16(d_tmem, sw128_desc(ahi + off), sw128_desc(blo + off), idesc, 1u);
              mma_bf16(d_tmem, sw128_desc(alo + off), sw128_desc(bhi + off), idesc, 1u);
              if constexpr (CX) {
                const uint32_t eh = ahi + 32768, el = ahi + 49152;
                mma_bf16(d_tmem, sw128_desc(eh + off), sw128_desc(bhi + 8192 + off), idesc64 | kNegA, 1u);
                mma_bf16(d_tmem, sw128_desc(eh + off), sw128_desc(blo + 8192 + off), idesc64 | kNegA, 1u);
                mma_bf16(d_tmem, sw128_desc(el + off), sw128_desc(bhi + 8192 + off), idesc64 | kNegA, 1u);
                mma_bf16(d_tmem + BR, sw128_desc(eh + off), sw128_desc(bhi + off), idesc64, 1u);
                mma_bf16(d_tmem + BR, sw128_desc(eh + off), sw128_desc(blo + off), idesc64, 1u);
                mma_bf16(d_tmem + BR, sw128_desc(el + off), sw128_desc(bhi + off), idesc64, 1u);
              }
            } else {
              mma_tf32(d_tmem, sw128_desc(ahi + off), sw128_desc(bhi + off), idesc, acc0);
              mma_tf32(d_tmem, sw128_desc(ahi + off), sw128_desc(blo + off), idesc, 1u);
              mma_tf32(d_tmem, sw128_desc(alo + off), sw128_desc(bhi + off), idesc, 1u);
            }
          }
          mma_commit(empty_x(sx));
          if (!MR) mma_commit(empty_m(sm));
        }
        if (!ok) break;
        mma_commit(acc_full(a));
      }
      mma_commit(fin_bar);
      mbar_wait(fin_bar, 0, abort_flag, err, 16, true);
    }
  } else {
    // ------------------------------------------------------------ epilogue
    const int q = warp & 3;            // TMEM lane quarter this warp may access
    const int half = (warp - 3) >> 2;  // 16-column groups 2 half and 2 half + 1
    uint32_t* box = reinterpret_cast<uint32_t*>(smem + kPlOffEpi + (warp - 3) * kPlEpiWarp);
    uint32_t t = 0;
    int pid = 0;
    for (long long u = blockIdx.x; u < units; u += gridDim.x, ++t) {
      const int a = t & 1;
      if (!mbar_wait(acc_full(a), (t >> 1) & 1, abort_flag, err, 19)) break;
      tc_fence_after();
      long long lu = u;
      int mbk = kp.m_blocks;
      const CUtensorMap *myh = &tm_yhi, *myl = &tm_ylo;
      if constexpr (G) {
        lu = locate(gd, ngd, u, pid);
        mbk = gd[pid].kp.m_blocks;
        myh = &gd[pid].yhi;
        myl = &gd[pid].ylo;
      }
      const long long tile = lu / mbk;
      const int mb = (int)(lu % mbk);
      const int i_base = mb * BM + q * 32;
#pragma unroll
      for (int sb = 0; sb < W; ++sb) {   // 64-r sub-blocks of a wide tile
      uint32_t vr[2][16], vi[2][16];
#pragma unroll
      for (int g2 = 0; g2 < 2; ++g2) {
        const int cc = 4 * sb + 2 * half + g2;
        const uint32_t tl = tmem_base + ((uint32_t)(q * 32) << 16) + a * W * BN + cc * 16;
        tmem_ld16(tl, vr[g2]);
        tmem_ld16(tl + W * BR, vi[g2]);
      }
      tmem_wait_ld();
      if (sb == W - 1) {   // the accumulator goes back to the MMA warp after the last read
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(acc_empty(a));
      }
      if constexpr (OP != kOpBF16) {
        // FP32 boxes of 32 x 32 (128-byte rows), one at a time through the 4 KB
        // staging area: per component the hi words (kOpTF32F: the FP32 value),
        // then (kOpTF32) the lo words
        float* fbox = reinterpret_cast<float*>(box);
        constexpr int NPART = OP == kOpTF32 ? 2 : 1;
#pragma unroll
        for (int comp = 0; comp < 2; ++comp) {
#pragma unroll
          for (int part = 0; part < NPART; ++part) {
            if (lane == 0) bulk_wait_read0();
            __syncwarp();
#pragma unroll
            for (int g2 = 0; g2 < 2; ++g2) {
              const uint32_t* v = comp == 0 ? vr[g2] : vi[g2];
#pragma unroll
              for (int j = 0; j < 16; j += 4) {
                float o[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                  const float x = __uint_as_float(v[j + e]);
                  if constexpr (OP == kOpTF32F) {
                    o[e] = x;
                  } else {
                    const float h = tf32_round(x);
                    o[e] = part == 0 ? h : tf32_round(x - h);
                  }
                }
                *reinterpret_cast<float4*>(fbox + lane * 32 + g2 * 16 + j) = make_float4(o[0], o[1], o[2], o[3]);
              }
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncwarp();
            if (lane == 0) {
              const int x = (int)(tile * BR + 32 * half);
              tma_store_3d(part == 0 ? myh : myl, smem_u32(fbox), x, i_base, comp);
              bulk_commit();
            }
            __syncwarp();
          }
        }
        continue;   // the TF32 forms have W == 1: on to the next unit
      }
      // this warp's two groups are adjacent (cc = 2 half, 2 half + 1): one 32 x 32 box
      // (64-byte rows) per component, real part first, then imaginary part
#pragma unroll
      for (int comp = 0; comp < 2; ++comp) {
        if (lane == 0) bulk_wait_read0();
        __syncwarp();
#pragma unroll
        for (int g2 = 0; g2 < 2; ++g2) {
#pragma unroll
          for (int j = 0; j < 16; j += 8) {
            uint4 h, l;
            const uint32_t* v = comp == 0 ? vr[g2] : vi[g2];
            h.x = split_pair(__uint_as_float(v[j + 0]), __uint_as_float(v[j + 1]), l.x);
            h.y = split_pair(__uint_as_float(v[j + 2]), __uint_as_float(v[j + 3]), l.y);
            h.z = split_pair(__uint_as_float(v[j + 4]), __uint_as_float(v[j + 5]), l.z);
            h.w = split_pair(__uint_as_float(v[j + 6]), __uint_as_float(v[j + 7]), l.w);
            const int w = lane * 16 + g2 * 8 + j / 2;   // 32-bit word of this row's 32 bf16
            *reinterpret_cast<uint4*>(box + w) = h;
            *reinterpret_cast<uint4*>(box + 512 + w) = l;
          }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        if (lane == 0) {
          const int x = (int)(tile * WR + 64 * sb + 32 * half);
          const uint32_t bs = smem_u32(box);
          tma_store_3d(myh, bs, x, i_base, comp);
          tma_store_3d(myl, bs + 2048, x, i_base, comp);
          bulk_commit();
        }
        __syncwarp();
      }
      }   // sub-blocks
    }
    if (lane == 0) bulk_wait0();
  }

  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(2 * W * BN));
}

}  // namespace b3
}  // namespace fcgle
