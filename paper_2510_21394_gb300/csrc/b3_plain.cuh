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
#pragma once

#include "b3_kernel.cuh"

namespace fcgle {
namespace b3 {

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

template <bool G>
__global__ void __launch_bounds__(PL_THREADS, 1)
    mp_b3_plain_kernel(const __grid_constant__ CUtensorMap tm_xhi, const __grid_constant__ CUtensorMap tm_xlo,
                       const __grid_constant__ CUtensorMap tm_mhi, const __grid_constant__ CUtensorMap tm_mlo,
                       const __grid_constant__ CUtensorMap tm_yhi, const __grid_constant__ CUtensorMap tm_ylo,
                       const KParams kp, const PlainDesc* __restrict__ gd, int ngd, long long gunits) {
  extern __shared__ uint8_t smem_raw[];
  pdl_trigger();
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const uint32_t sbase = smem_u32(smem);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + kPlOffBar);
  auto full_x = [&](int s) { return smem_u32(&bars[s]); };
  auto empty_x = [&](int s) { return smem_u32(&bars[PL_NX + s]); };
  auto full_m = [&](int s) { return smem_u32(&bars[2 * PL_NX + s]); };
  auto empty_m = [&](int s) { return smem_u32(&bars[2 * PL_NX + PL_NM + s]); };
  auto acc_full = [&](int a) { return smem_u32(&bars[2 * PL_NX + 2 * PL_NM + a]); };
  auto acc_empty = [&](int a) { return smem_u32(&bars[2 * PL_NX + 2 * PL_NM + 2 + a]); };
  const uint32_t fin_bar = smem_u32(&bars[2 * PL_NX + 2 * PL_NM + 4]);
  static_assert((2 * PL_NX + 2 * PL_NM + 5) * 8 <= 192, "barrier area");
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + kPlOffBar + 192);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + kPlOffBar + 200);

  if (threadIdx.x == 0) {
    for (int s = 0; s < PL_NX; ++s) {
      mbar_init(full_x(s), 1);
      mbar_init(empty_x(s), 1);
    }
    for (int s = 0; s < PL_NM; ++s) {
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
                 "r"(2 * BN));
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
        const int r0 = (int)(tile * BR);
        const int r1 = (int)(R + tile * BR);   // same r in the imaginary plane
        for (int kc = 0; kc < KC; ++kc, ++g) {
          const int s = (int)(g % PL_NX);
          if (!mbar_wait(empty_x(s), ((g / PL_NX) & 1) ^ 1, abort_flag, err, 11)) { ok = false; break; }
          const uint32_t st = sbase + s * kXStage;
          mbar_arrive_tx(full_x(s), kXStage);
          tma_load_2d(st, mxh, kc * BK, r0, full_x(s));
          tma_load_2d(st + 8192, mxh, kc * BK, r1, full_x(s));
          tma_load_2d(st + 16384, mxl, kc * BK, r0, full_x(s));
          tma_load_2d(st + 24576, mxl, kc * BK, r1, full_x(s));
        }
      }
      const uint32_t issued = g;
      for (uint32_t q = issued >= PL_NX ? issued - PL_NX : 0; q < issued; ++q)
        mbar_wait(full_x(q % PL_NX), (q / PL_NX) & 1, abort_flag, err, 17, true);
    }
  } else if (warp == 2) {
    // ------------------------------------------------------------ M producer
    if (lane == 0) {
      uint32_t g = 0;
      bool ok = true;
      int pid = 0;
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
          const int s = (int)(g % PL_NM);
          if (!mbar_wait(empty_m(s), ((g / PL_NM) & 1) ^ 1, abort_flag, err, 12)) { ok = false; break; }
          const uint32_t st = sbase + kPlOffM + s * kMStage;
          mbar_arrive_tx(full_m(s), kMStage);
          tma_load_2d(st, mmh, kc * BK, mb * BM, full_m(s));
          tma_load_2d(st + 16384, mml, kc * BK, mb * BM, full_m(s));
        }
      }
      const uint32_t issued = g;
      for (uint32_t q = issued >= PL_NM ? issued - PL_NM : 0; q < issued; ++q)
        mbar_wait(full_m(q % PL_NM), (q / PL_NM) & 1, abort_flag, err, 18, true);
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      constexpr uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
                                 ((uint32_t)(BM >> 4) << 24);
      uint32_t g = 0, t = 0;
      bool ok = true;
      int pid = 0;
      for (long long u = blockIdx.x; u < units && ok; u += gridDim.x, ++t) {
        int KC = kp.k_chunks;
        if constexpr (G) {
          locate(gd, ngd, u, pid);
          KC = gd[pid].kp.k_chunks;
        }
        const int a = t & 1;
        if (!mbar_wait(acc_empty(a), ((t >> 1) & 1) ^ 1, abort_flag, err, 13)) break;
        tc_fence_after();
        const uint32_t d_tmem = tmem_base + a * BN;
        for (int kc = 0; kc < KC; ++kc, ++g) {
          const int sx = (int)(g % PL_NX), sm = (int)(g % PL_NM);
          if (!mbar_wait(full_m(sm), (g / PL_NM) & 1, abort_flag, err, 14)) { ok = false; break; }
          if (!mbar_wait(full_x(sx), (g / PL_NX) & 1, abort_flag, err, 15)) { ok = false; break; }
          tc_fence_after();
          const uint32_t ahi = sbase + kPlOffM + sm * kMStage, alo = ahi + 16384;
          const uint32_t bhi = sbase + sx * kXStage, blo = bhi + 16384;
#pragma unroll
          for (int ks = 0; ks < BK / 16; ++ks) {
            const uint32_t off = ks * 32;
            const uint32_t acc0 = (kc > 0 || ks > 0) ? 1u : 0u;
            mma_bf16(d_tmem, sw128_desc(ahi + off), sw128_desc(bhi + off), idesc, acc0);
            mma_bf16(d_tmem, sw128_desc(ahi + off), sw128_desc(blo + off), idesc, 1u);
            mma_bf16(d_tmem, sw128_desc(alo + off), sw128_desc(bhi + off), idesc, 1u);
          }
          mma_commit(empty_x(sx));
          mma_commit(empty_m(sm));
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
      uint32_t vr[2][16], vi[2][16];
#pragma unroll
      for (int g2 = 0; g2 < 2; ++g2) {
        const int cc = 2 * half + g2;
        const uint32_t tl = tmem_base + ((uint32_t)(q * 32) << 16) + a * BN + cc * 16;
        tmem_ld16(tl, vr[g2]);
        tmem_ld16(tl + BR, vi[g2]);
      }
      tmem_wait_ld();
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(acc_empty(a));
      const int i_base = mb * BM + q * 32;
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
          const int x = (int)(tile * BR + 32 * half);
          const uint32_t sb = smem_u32(box);
          tma_store_3d(myh, sb, x, i_base, comp);
          tma_store_3d(myl, sb + 2048, x, i_base, comp);
          bulk_commit();
        }
        __syncwarp();
      }
    }
    if (lane == 0) bulk_wait0();
  }

  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(2 * BN));
}

}  // namespace b3
}  // namespace fcgle
