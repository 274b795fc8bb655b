// Slab-fused mode-1 and mode-2 products of a 3D tensor (Sec. 3.2: the first
// two factors of a Tucker operator, Eq. fKu_diag), split-BF16 on the sm_103a
// tensor cores, one j_3 slab at a time:
//
//   Y[c][j3][i2][i1] = sum_{j2} M2[i2][j2] sum_{j1} M1[i1][j1] X[c][j3][j2][j1]
//
// in the natural (vec) order in and out: the slab index j_3 stays the slowest
// index, so the mode-3 product that completes the Tucker operator reads its
// input with the contracted index slowest (the MN-major form of
// mp_b3_kernel).  The intermediate U = X_slab M1^T never leaves the SM: two
// mode products for the HBM bytes of one.
//
// Unit of work: (slab j3, block of 128 i1).  For each plane c (real, then
// imaginary; M1 and M2 are real, so the planes do not mix):
//   stage 1  D[i1][j2]  = sum_j1 M1[i1][j1] X[c][j3][j2][j1]
//            (A = 128 rows of M1, B = the slab's N2 rows j2, both K-major
//            from shared memory; N2 = p2 rounded up to 16, <= 256)
//   convert  U = split(D) into bf16 hi and lo, written back over D in tensor
//            memory (lane = i1; per 16 columns of D: 8 columns of hi, then 8
//            of lo, two bf16 per 32-bit column)
//   stage 2  E[i1][i2] = sum_j2 U[i1][j2] M2[i2][j2]
//            (A = U from tensor memory, B = N2 rows of M2 from shared memory)
//   store    E split into hi and lo and stored through 32 x 32 boxes
//            (rows i2, 64-byte rows of 32 consecutive i1)
// Each product is hi.hi + hi.lo + lo.hi with an FP32 accumulator, as in
// mp_b3_kernel.  Tensor memory: columns [0, 256) hold D and then U, columns
// [256, 512) hold E, so stage 1 of the next plane overlaps the store of E
// and stage 2 starts on each 64-column k-chunk of U as soon as it is written.
//
// Warp roles (one CTA per SM, persistent over the units):
//   warp 0      TMA producer: stage-1 chunks (M1 hi, lo 128 x 32; X hi, lo
//               N2 x 32) and stage-2 chunks (M2 hi, lo N2 x 32) through a
//               4-deep ring of 48 KB stages (32-wide k-chunks: 64-byte rows,
//               64-byte swizzle, so that more operand bytes are in flight
//               per byte the MMA holds)
//   warp 1      TMEM allocator (512 columns) and single-thread MMA issuer
//   warps 2-9   convert and store; warp w owns TMEM lane quarter w % 4 and
//               the 16-column groups (convert) or 32-column boxes (store) of
//               parity (w - 2) / 4
// Every mbarrier wait is bounded (mbar_wait); on expiry the CTA records an
// error code, drains its own TMA and MMA work, frees its TMEM and returns.
//
// Requirements (checked by the host): p2 <= 256; p1 and p2 multiples of 8
// (16-byte rows of every tensor map).
#pragma once

#include "b3_kernel.cuh"

namespace fcgle {
namespace b3 {

constexpr int SL_NEPI = 8;
constexpr int SL_THREADS = 32 * (2 + SL_NEPI);
constexpr int SL_NS = 4;                       // ring stages
constexpr int SL_K = 32;                       // k per chunk (one 64-byte bf16 row)
constexpr uint32_t kSlStage = 49152;           // M1 hi 8K | M1 lo 8K | X hi 16K | X lo 16K  (stage 2: M2 hi 16K | M2 lo 16K)
constexpr uint32_t kSlOffEpi = SL_NS * kSlStage;
constexpr uint32_t kSlEpiWarp = 4096;          // one 32 x 32 bf16 box, hi and lo
constexpr uint32_t kSlOffBar = kSlOffEpi + SL_NEPI * kSlEpiWarp;
constexpr uint32_t kSlSmemBytes = kSlOffBar + 256 + 1024;   // + barriers + alignment slack
static_assert(kSlSmemBytes <= 232448, "shared memory budget");
constexpr uint32_t kSlColE = 256;              // TMEM column of the stage-2 accumulator E

struct SlabParams {
  int p1, p2, p3;   // padded extents
  int n2;           // N of both products: p2 rounded up to a multiple of 16 (<= 256)
  int mb1;          // 128-row blocks of i1
  int kc1;          // 32-wide k-chunks of j1
  int kc2;          // 32-wide k-chunks of j2 (ceil(n2 / 32))
  int* err;
};

// tcgen05.mma with the A operand in tensor memory
__device__ __forceinline__ void mma_bf16_ts(uint32_t d_tmem, uint32_t a_tmem, uint64_t bdesc, uint32_t idesc,
                                            uint32_t accum) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}" ::"r"(d_tmem),
      "r"(a_tmem), "l"(bdesc), "r"(idesc), "r"(accum)
      : "memory");
}
__device__ __forceinline__ void tmem_st8(uint32_t taddr, const uint32_t (&v)[8]) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(taddr), "r"(v[0]),
               "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7])
               : "memory");
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }
// K-major, SWIZZLE_64B: rows of 64 bytes, 8-row groups 512 bytes apart.
__device__ __forceinline__ uint64_t sw64_desc(uint32_t addr) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(512 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)4 << 61);
}

__global__ void __launch_bounds__(SL_THREADS, 1)
    mp_b3_slab12_kernel(const __grid_constant__ CUtensorMap tm_xhi, const __grid_constant__ CUtensorMap tm_xlo,
                        const __grid_constant__ CUtensorMap tm_m1hi, const __grid_constant__ CUtensorMap tm_m1lo,
                        const __grid_constant__ CUtensorMap tm_m2hi, const __grid_constant__ CUtensorMap tm_m2lo,
                        const __grid_constant__ CUtensorMap tm_yhi, const __grid_constant__ CUtensorMap tm_ylo,
                        const SlabParams sp) {
  extern __shared__ uint8_t smem_raw[];
  pdl_trigger();
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const uint32_t sbase = smem_u32(smem);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + kSlOffBar);
  auto full_bar = [&](int s) { return smem_u32(&bars[s]); };
  auto empty_bar = [&](int s) { return smem_u32(&bars[SL_NS + s]); };
  const uint32_t d1_full = smem_u32(&bars[2 * SL_NS]);
  const uint32_t d2_full = smem_u32(&bars[2 * SL_NS + 1]);
  const uint32_t d_empty = smem_u32(&bars[2 * SL_NS + 2]);
  const uint32_t fin_bar = smem_u32(&bars[2 * SL_NS + 3]);
  // U ready, per 64 columns (at most 4)
  auto u_full = [&](int c) { return smem_u32(&bars[2 * SL_NS + 4 + c]); };
  static_assert((2 * SL_NS + 8) * 8 <= 192, "barrier area");
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + kSlOffBar + 192);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + kSlOffBar + 200);

  if (threadIdx.x == 0) {
    for (int s = 0; s < SL_NS; ++s) {
      mbar_init(full_bar(s), 1);
      mbar_init(empty_bar(s), 1);
    }
    mbar_init(d1_full, 1);
    for (int c = 0; c < 4; ++c) mbar_init(u_full(c), SL_NEPI);
    mbar_init(d2_full, 1);
    mbar_init(d_empty, SL_NEPI);
    mbar_init(fin_bar, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;
  pdl_wait();

  const long long units = (long long)sp.p3 * sp.mb1;
  int* err = sp.err;

  if (warp == 0) {
    // ------------------------------------------------------------ producer
    if (lane == 0) {
      uint32_t g = 0;
      bool ok = true;
      const uint32_t xbytes = (uint32_t)sp.n2 * 64;   // one N2 x 32 bf16 box
      const int m2boxes = sp.n2 > 128 ? 2 : 1;
      for (long long u = blockIdx.x; u < units && ok; u += gridDim.x) {
        const int j3 = (int)(u / sp.mb1), b1 = (int)(u % sp.mb1);
        for (int c = 0; c < 2 && ok; ++c) {
          const int z = c * sp.p3 + j3;
          for (int kc = 0; kc < sp.kc1; ++kc, ++g) {
            const int s = (int)(g % SL_NS);
            if (!mbar_wait(empty_bar(s), ((g / SL_NS) & 1) ^ 1, abort_flag, err, 31)) { ok = false; break; }
            const uint32_t st = sbase + s * kSlStage;
            mbar_arrive_tx(full_bar(s), 16384 + 2 * xbytes);
            tma_load_2d(st, &tm_m1hi, kc * SL_K, b1 * BM, full_bar(s));
            tma_load_2d(st + 8192, &tm_m1lo, kc * SL_K, b1 * BM, full_bar(s));
            tma_load_3d(st + 16384, &tm_xhi, kc * SL_K, 0, z, full_bar(s));
            tma_load_3d(st + 32768, &tm_xlo, kc * SL_K, 0, z, full_bar(s));
          }
          for (int kc = 0; kc < sp.kc2 && ok; ++kc, ++g) {
            const int s = (int)(g % SL_NS);
            if (!mbar_wait(empty_bar(s), ((g / SL_NS) & 1) ^ 1, abort_flag, err, 32)) { ok = false; break; }
            const uint32_t st = sbase + s * kSlStage;
            mbar_arrive_tx(full_bar(s), (uint32_t)m2boxes * 16384);
            for (int b = 0; b < m2boxes; ++b) {
              tma_load_2d(st + b * 8192, &tm_m2hi, kc * SL_K, b * BM, full_bar(s));
              tma_load_2d(st + 16384 + b * 8192, &tm_m2lo, kc * SL_K, b * BM, full_bar(s));
            }
          }
        }
      }
      // drain: every issued stage must have landed before the CTA may exit
      const uint32_t issued = g;
      for (uint32_t q = issued >= SL_NS ? issued - SL_NS : 0; q < issued; ++q)
        mbar_wait(full_bar(q % SL_NS), (q / SL_NS) & 1, abort_flag, err, 37, true);
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      // FP32 accumulator, A and B bf16, both K-major, M = 128, N = n2
      const uint32_t idesc =
          (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(sp.n2 >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
      const int ksteps2 = sp.n2 / 16;
      uint32_t g = 0, t = 0;
      bool ok = true;
      for (long long u = blockIdx.x; u < units && ok; u += gridDim.x) {
        for (int c = 0; c < 2 && ok; ++c, ++t) {
          // D may be overwritten once the previous plane's stage 2 has read U
          if (t > 0 && !mbar_wait(d2_full, (t - 1) & 1, abort_flag, err, 33)) { ok = false; break; }
          tc_fence_after();
          // stage 1: D[i1][j2] = sum_j1 M1[i1][j1] X[j2][j1]
          for (int kc = 0; kc < sp.kc1; ++kc, ++g) {
            const int s = (int)(g % SL_NS);
            if (!mbar_wait(full_bar(s), (g / SL_NS) & 1, abort_flag, err, 34)) { ok = false; break; }
            tc_fence_after();
            const uint32_t ahi = sbase + s * kSlStage, alo = ahi + 8192;
            const uint32_t bhi = ahi + 16384, blo = ahi + 32768;
#pragma unroll
            for (int ks = 0; ks < 2; ++ks) {
              const uint32_t off = ks * 32;
              const uint32_t acc0 = (kc > 0 || ks > 0) ? 1u : 0u;
              mma_bf16(tmem_base, sw64_desc(ahi + off), sw64_desc(bhi + off), idesc, acc0);
              mma_bf16(tmem_base, sw64_desc(ahi + off), sw64_desc(blo + off), idesc, 1u);
              mma_bf16(tmem_base, sw64_desc(alo + off), sw64_desc(bhi + off), idesc, 1u);
            }
            mma_commit(empty_bar(s));
          }
          if (!ok) break;
          mma_commit(d1_full);
          // stage 2: E[i1][i2] = sum_j2 U[i1][j2] M2[i2][j2], U from tensor
          // memory; E is free once the previous plane's E has been read out,
          // and k-chunk kc starts as soon as its 64 columns of U are written
          if (!mbar_wait(d_empty, (t & 1) ^ 1, abort_flag, err, 41)) { ok = false; break; }
          for (int kc = 0; kc < sp.kc2; ++kc, ++g) {
            const int s = (int)(g % SL_NS);
            if (!mbar_wait(u_full(kc >> 1), t & 1, abort_flag, err, 35)) { ok = false; break; }
            if (!mbar_wait(full_bar(s), (g / SL_NS) & 1, abort_flag, err, 36)) { ok = false; break; }
            tc_fence_after();
            const uint32_t bhi = sbase + s * kSlStage, blo = bhi + 16384;
#pragma unroll
            for (int ks = 0; ks < 2; ++ks) {
              const int kk = 2 * kc + ks;   // 16-wide k-step of j2
              if (kk < ksteps2) {
                const uint32_t uhi = tmem_base + 16 * kk, ulo = uhi + 8;
                const uint32_t off = ks * 32, e_tmem = tmem_base + kSlColE;
                mma_bf16_ts(e_tmem, uhi, sw64_desc(bhi + off), idesc, kk > 0 ? 1u : 0u);
                mma_bf16_ts(e_tmem, uhi, sw64_desc(blo + off), idesc, 1u);
                mma_bf16_ts(e_tmem, ulo, sw64_desc(bhi + off), idesc, 1u);
              }
            }
            mma_commit(empty_bar(s));
          }
          if (!ok) break;
          mma_commit(d2_full);
        }
      }
      // drain: all issued MMAs complete before TMEM is released
      mma_commit(fin_bar);
      mbar_wait(fin_bar, 0, abort_flag, err, 38, true);
    }
  } else {
    // ------------------------------------------------------------ convert and store
    const int q = warp & 3;             // TMEM lane quarter
    const int par = (warp - 2) >> 2;    // column-group parity of this warp
    const uint32_t lane_off = (uint32_t)(q * 32) << 16;
    uint8_t* box = smem + kSlOffEpi + (warp - 2) * kSlEpiWarp;
    const uint32_t box_u32 = smem_u32(box);
    const int ngrp = sp.n2 / 16;        // 16-column groups of D
    const int nbox = (sp.n2 + 31) / 32; // 32-column output boxes
    uint32_t t = 0;
    bool ok = true;
    for (long long u = blockIdx.x; u < units && ok; u += gridDim.x) {
      const int j3 = (int)(u / sp.mb1), b1 = (int)(u % sp.mb1);
      for (int c = 0; c < 2; ++c, ++t) {
        // ---- convert: D (FP32) -> U_hi, U_lo (bf16 pairs) in tensor memory, one
        // 64-column k-chunk (4 groups of 16, 2 per warp of a lane quarter) at a time
        if (!mbar_wait(d1_full, t & 1, abort_flag, err, 39)) { ok = false; break; }
        tc_fence_after();
        for (int kc = 0; kc < (sp.n2 + 63) / 64; ++kc) {
          uint32_t v[2][16];
#pragma unroll
          for (int e = 0; e < 2; ++e) {
            const int grp = 4 * kc + par + 2 * e;
            if (grp < ngrp) tmem_ld16(tmem_base + lane_off + 16 * grp, v[e]);
          }
          tmem_wait_ld();
#pragma unroll
          for (int e = 0; e < 2; ++e) {
            const int grp = 4 * kc + par + 2 * e;
            if (grp < ngrp) {
              uint32_t h[8], l[8];
#pragma unroll
              for (int j = 0; j < 8; ++j)
                h[j] = split_pair(__uint_as_float(v[e][2 * j]), __uint_as_float(v[e][2 * j + 1]), l[j]);
              tmem_st8(tmem_base + lane_off + 16 * grp, h);
              tmem_st8(tmem_base + lane_off + 16 * grp + 8, l);
            }
          }
          tmem_wait_st();
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(u_full(kc));
        }
        // ---- store: E (FP32) -> Y[c][j3][i2][i1], split, one 32-column box at a time
        if (!mbar_wait(d2_full, t & 1, abort_flag, err, 40)) { ok = false; break; }
        tc_fence_after();
        if (par >= nbox && lane == 0) mbar_arrive(d_empty);   // no box of E for this warp
        const int x = b1 * BM + q * 32;   // first i1 of this warp's rows
        const int z = c * sp.p3 + j3;
        for (int bx = par; bx < nbox; bx += 2) {
          uint32_t v[32];
          tmem_ld16(tmem_base + lane_off + kSlColE + 32 * bx, *reinterpret_cast<uint32_t(*)[16]>(&v[0]));
          tmem_ld16(tmem_base + lane_off + kSlColE + 32 * bx + 16, *reinterpret_cast<uint32_t(*)[16]>(&v[16]));
          tmem_wait_ld();
          if (bx + 2 >= nbox) {   // this warp's last read of E
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(d_empty);
          }
          if (lane == 0) bulk_wait_read0();
          __syncwarp();
          // box row j = i2 - 32 bx (64 bytes: 32 i1), this lane's i1 at byte 2 lane
#pragma unroll
          for (int j = 0; j < 32; j += 2) {
            uint32_t lo;
            const uint32_t hi = split_pair(__uint_as_float(v[j]), __uint_as_float(v[j + 1]), lo);
            const uint32_t a0 = box_u32 + j * 64 + lane * 2;
            asm volatile("st.shared.b16 [%0], %1;" ::"r"(a0), "h"((unsigned short)(hi & 0xFFFFu)) : "memory");
            asm volatile("st.shared.b16 [%0], %1;" ::"r"(a0 + 64), "h"((unsigned short)(hi >> 16)) : "memory");
            asm volatile("st.shared.b16 [%0], %1;" ::"r"(a0 + 2048), "h"((unsigned short)(lo & 0xFFFFu)) : "memory");
            asm volatile("st.shared.b16 [%0], %1;" ::"r"(a0 + 2048 + 64), "h"((unsigned short)(lo >> 16))
                         : "memory");
          }
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          __syncwarp();
          if (lane == 0 && x < sp.p1 && 32 * bx < sp.p2) {
            tma_store_3d(&tm_yhi, box_u32, x, 32 * bx, z);
            tma_store_3d(&tm_ylo, box_u32 + 2048, x, 32 * bx, z);
            bulk_commit();
          }
          __syncwarp();
        }
      }
    }
    if (lane == 0) bulk_wait0();
  }

  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(512));
}

}  // namespace b3
}  // namespace fcgle
