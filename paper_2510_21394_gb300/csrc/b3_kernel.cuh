// Split-BF16 mu-mode product on the sm_103a tensor cores (tcgen05 + TMEM + TMA)
// with a fused pointwise epilogue (the last mode product of a Tucker operator
// that carries a scheme's pointwise stage).
//
// One launch computes, in the rotating layout of common.h,
//     acc[c][i][r] = sum_k M[i][k] X[c][r][k]              (Sec. 3.2, one mode product)
// where every operand arrives pre-split into two bf16 numbers, x = x_hi + x_lo,
// and the product is M_hi X_hi + M_hi X_lo + M_lo X_hi with FP32 accumulation
// in tensor memory (the dropped M_lo X_lo term is below 2^-16 relative).
// The FP32 result is handed, element by element as a complex number
// (acc[0][i][r], acc[1][i][r]), to an epilogue functor `Epi` that may read
// other standard-order tensors, evaluate the nonlinearity or the stage
// combinations of a scheme and write any outputs, split or FP32.
//
// GEMM orientation: D[i][col] = sum_k A[i][k] B[col][k] with A = M (MMA M =
// 128 output indices i per block) and B = 128 data rows: the same 64 indices
// r0..r0+63 of the real plane (columns 0..63) and of the imaginary plane
// (columns 64..127), so each epilogue thread sees complete complex values.
//
// Warp roles (one CTA per SM, persistent over (r-tile, i-block)):
//   warp 0      TMA producer: M_hi, M_lo (128 x 64) and X_hi, X_lo (2 x 64 x 64)
//               bf16 chunks, SWIZZLE_128B, straight into the MMA layout.
//   warp 1      TMEM allocator and single-thread MMA issuer (3 MMAs per k-step).
//   warps 2-17  epilogue (see Cfg): TMEM -> registers, an smem transpose and
//               the functor on coalesced (i, r) runs.  Warp w reads TMEM lane
//               quarter w % 4.
// Pipelines: 2 smem stages (64 KB each), 2 TMEM accumulators (2 x 128 columns).
// Every mbarrier wait is bounded by a wall-clock limit; on expiry the CTA
// records an error code in *err, drains its own TMA and MMA work, frees its
// TMEM and returns.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>

#include "common.h"

namespace fcgle {
namespace b3 {

constexpr int BM = 128;     // output indices i per MMA
constexpr int BR = 64;      // r indices per tile (x 2 planes = MMA N)
constexpr int BN = 2 * BR;  // MMA N
constexpr int BK = 64;      // k per chunk (one 128-byte bf16 row)

constexpr uint32_t kStage = 65536;   // M_hi 16K | M_lo 16K | X_hi 16K | X_lo 16K
constexpr uint32_t kEpiWarp = 32 * 33 * 4;

// Launch shape of the fused-epilogue kernel.  The epilogues read and write
// several tensors per element besides the product, so their time goes into the
// epilogue's global loads: 16 epilogue warps (each owning one 16-column group
// of a TMEM lane quarter; an accumulator tile is 4 lane quarters x 4 groups of
// 16 r columns) and 2 smem stages, which is all the shared memory then leaves.
// (The plain product, b3_plain.cuh, streams its operands differently.)
//
// Complex form (CX = true, the Kronecker-product exponential of Eq. Neudeckerd):
// M = E = Er + i Ei is complex, so a stage also carries the Ei_hi, Ei_lo
// chunks (96 KB per stage) and the epilogue drops to 8 warps (two 16-column
// groups each) to fit the shared memory.
template <class Epi, bool CX = false>
struct Cfg {
  static constexpr int kEpi = CX ? 8 : 16;
  static constexpr int kStages = 2;
  static constexpr int kThreads = 32 * (2 + kEpi);
  static constexpr int kGroups = 16 / kEpi;   // 16-column groups per epilogue warp
  static constexpr uint32_t kStageBytes = CX ? 3 * kStage / 2 : kStage;
  static constexpr uint32_t kOffEpi = kStages * kStageBytes;
  static constexpr uint32_t kOffBar = kOffEpi + kEpi * kEpiWarp;
  static constexpr uint32_t kSmemBytes = kOffBar + 256 + 1024;   // + barriers + alignment slack
  static_assert(kSmemBytes <= 232448, "shared memory budget");
  static_assert(kEpi % 4 == 0 && 16 % kEpi == 0, "epilogue warps cover 4 quarters x 4 groups");
};

constexpr unsigned long long kTimeoutNs = 2000000000ull;   // 2 s per wait

struct KParams {
  long long R;      // rows per plane of X; row length of the output planes
  int p;            // extent of the contracted / produced index (rows of M)
  int m_blocks;     // ceil(p / 128)
  int k_chunks;     // ceil(p / 64)
  long long tiles;  // ceil(R / 64)
  int* err;
  int ei_row = 0;   // complex forms: row of Ei in the stacked [Er; Ei] matrix maps
};

// Complex mode product (Eq. Neudecker): with M = Er + i Ei and the tile's
// columns 0..63 = re rows, 64..127 = im rows of X,
//   D[:, 0:64]   = Er Xre - Ei Xim   (re part)
//   D[:, 64:128] = Er Xim + Ei Xre   (im part)
// as one N = 128 product with Er over both planes plus two N = 64 products
// with Ei: negated on the im rows into columns 0..63, plain on the re rows
// into columns 64..127 (instruction-descriptor bit 13 negates A).  Each of the
// three is split hi.hi + hi.lo + lo.hi.
constexpr uint32_t kNegA = 1u << 13;

// -------------------------------------------------------------- PTX helpers
// Programmatic dependent launch.  Every mode-product kernel lets the next
// kernel of its stream be scheduled as soon as all of its own CTAs are running
// (pdl_trigger at entry) and, after its prologue (mbarrier init, TMEM
// allocation), waits until the previous kernel of the stream has completed and
// its writes are visible (pdl_wait) before it touches global memory.  The
// wait ends when that kernel ends; without the launch attribute both are
// no-ops.
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ unsigned long long now_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void mbar_arrive_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait; returns false (and raises the CTA abort flag) on timeout or,
// unless `drain` is set, as soon as another role has aborted.  Drain waits
// (for this CTA's own TMA / MMA work before exit) only stop at the time limit.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag, int* err,
                                          int code, bool drain = false) {
  if (mbar_try(bar, parity)) return true;
  const unsigned long long t0 = now_ns();
  for (uint32_t it = 1;; ++it) {
    if (mbar_try(bar, parity)) return true;
    if ((it & 63) == 0) {
      if (!drain && *abort_flag) return false;
      if (now_ns() - t0 > kTimeoutNs) {
        *abort_flag = 1;
        atomicExch(err, code);
        return false;
      }
    }
  }
}
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, int x, int y, int z, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(
          dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(bar)
      : "memory");
}
__device__ __forceinline__ uint64_t sw128_desc(uint32_t addr) {
  // K-major, SWIZZLE_128B: rows of 128 bytes, 8-row groups 1024 bytes apart.
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}
// MN-major, SWIZZLE_128B: every k is a 128-byte row of 64 consecutive n, 8-row
// (k) groups 1024 bytes apart (stride byte offset); the next 64 n start
// `mn_stride` bytes further (leading byte offset).  Used with the instruction
// descriptor's transpose-B bit.
__device__ __forceinline__ uint64_t sw128_mn_desc(uint32_t addr, uint32_t mn_stride) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)((mn_stride >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)(1024 >> 4) << 32) | ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}
constexpr uint32_t kTransB = 1u << 16;   // instruction descriptor: B is MN-major
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accum) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
               : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
        "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// ------------------------------------------------------------------ kernel
__device__ __forceinline__ void tma_store_3d(const CUtensorMap* map, uint32_t src, int x, int y, int z) {
  asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.bulk_group [%0, {%2, %3, %4}], [%1];" ::"l"(
                   reinterpret_cast<uint64_t>(map)),
               "r"(src), "r"(x), "r"(y), "r"(z)
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read0() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait0() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

__device__ __forceinline__ uint32_t split_pair(float a, float b, uint32_t& lo) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  const float2 hf = __bfloat1622float2(h);
  const __nv_bfloat162 l = __floats2bfloat162_rn(a - hf.x, b - hf.y);
  lo = *reinterpret_cast<const uint32_t*>(&l);
  return *reinterpret_cast<const uint32_t*>(&h);
}

// Grouped launches: problem k of a descriptor array owns the global units
// [gd[k].ubegin, gd[k + 1].ubegin); every warp role walks its units in
// increasing order, so a forward-only cursor finds the problem of a unit.
template <class D>
__device__ __forceinline__ long long locate(const D* gd, int n, long long u, int& pid) {
  while (pid + 1 < n && u >= gd[pid + 1].ubegin) ++pid;
  return u - gd[pid].ubegin;
}

// Epilogue functor interface (b3_epilogues.cuh): a batched two-phase functor,
// load(q, i, r, in) for kBatch elements, then store(q, i, r, re, im, in) for
// each, so that the operand loads of a batch are in flight together.
// one problem of a grouped fused launch (aligned as its tensor maps)
template <class Epi>
struct FusedDesc {
  CUtensorMap xhi, xlo, mhi, mlo;
  KParams kp;
  long long ubegin;
  Epi epi;
};

// Grouped form (G = true): one persistent launch serves the last mode
// product of several independent problems; maps, sizes and the epilogue
// functor of problem k come from gd[k].  Same arithmetic per unit.
//
// Natural-order input (MN = true): X holds the contracted index as its
// SLOWEST index, X[c][k][r], the layout the slab-fused mode-1+2 product
// (b3_slab.cuh) leaves behind, so no rotation precedes this product.  The X
// tensor maps are 3D (r, k, plane) with 64 x 64 boxes (64 r of one k per
// 128-byte row), and the B operand is read MN-major; the accumulator, the
// epilogue and the output layout Y[c][i][r] are those of the K-major form.
template <class Epi, bool G = false, bool CX = false, bool MN = false>
__global__ void __launch_bounds__(Cfg<Epi, CX>::kThreads, 1)
    mp_b3_kernel(const __grid_constant__ CUtensorMap tm_xhi, const __grid_constant__ CUtensorMap tm_xlo,
                 const __grid_constant__ CUtensorMap tm_mhi, const __grid_constant__ CUtensorMap tm_mlo,
                 const KParams kp, const Epi epi, const FusedDesc<Epi>* __restrict__ gd, int ngd,
                 long long gunits) {
  static_assert(!(G && CX), "the complex form has no grouped variant");
  static_assert(!(MN && (G || CX)), "the natural-order form is single-problem and real");
  constexpr int NSTAGE = Cfg<Epi, CX>::kStages;
  constexpr int NEPI = Cfg<Epi, CX>::kEpi;
  constexpr uint32_t kStg = Cfg<Epi, CX>::kStageBytes;
  constexpr uint32_t kOffX = CX ? 65536 : 32768;   // X chunks after M (and Ei)
  constexpr uint32_t kOffEpi = Cfg<Epi, CX>::kOffEpi;
  constexpr uint32_t kOffBar = Cfg<Epi, CX>::kOffBar;
  extern __shared__ uint8_t smem_raw[];
  pdl_trigger();
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const uint32_t sbase = smem_u32(smem);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + kOffBar);
  auto full_bar = [&](int s) { return smem_u32(&bars[s]); };
  auto empty_bar = [&](int s) { return smem_u32(&bars[NSTAGE + s]); };
  auto acc_full = [&](int a) { return smem_u32(&bars[2 * NSTAGE + a]); };
  auto acc_empty = [&](int a) { return smem_u32(&bars[2 * NSTAGE + 2 + a]); };
  const uint32_t fin_bar = smem_u32(&bars[2 * NSTAGE + 4]);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + kOffBar + 128);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + kOffBar + 136);

  if (threadIdx.x == 0) {
    for (int s = 0; s < NSTAGE; ++s) {
      mbar_init(full_bar(s), 1);
      mbar_init(empty_bar(s), 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(acc_full(a), 1);
      mbar_init(acc_empty(a), NEPI);
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
    // ------------------------------------------------------------ producer
    if (lane == 0) {
      uint32_t g = 0;
      bool ok = true;
      int pid = 0;
      for (long long u = blockIdx.x; u < units && ok; u += gridDim.x) {
        long long lu = u, R = kp.R;
        int mbk = kp.m_blocks, KC = kp.k_chunks;
        const CUtensorMap *mxh = &tm_xhi, *mxl = &tm_xlo, *mmh = &tm_mhi, *mml = &tm_mlo;
        if constexpr (G) {
          lu = locate(gd, ngd, u, pid);
          R = gd[pid].kp.R;
          mbk = gd[pid].kp.m_blocks;
          KC = gd[pid].kp.k_chunks;
          mxh = &gd[pid].xhi;
          mxl = &gd[pid].xlo;
          mmh = &gd[pid].mhi;
          mml = &gd[pid].mlo;
        }
        const long long tile = lu / mbk;
        const int mb = (int)(lu % mbk);
        const int r0 = (int)(tile * BR);
        const int r1 = (int)(R + tile * BR);   // same r in the imaginary plane
        for (int kc = 0; kc < KC; ++kc, ++g) {
          const int s = (int)(g % NSTAGE);
          const uint32_t ph = (g / NSTAGE) & 1;
          if (!mbar_wait(empty_bar(s), ph ^ 1, abort_flag, err, 1)) { ok = false; break; }
          const uint32_t st = sbase + s * kStg;
          mbar_arrive_tx(full_bar(s), kStg);
          tma_load_2d(st, mmh, kc * BK, mb * BM, full_bar(s));
          tma_load_2d(st + 16384, mml, kc * BK, mb * BM, full_bar(s));
          if constexpr (CX) {
            tma_load_2d(st + 32768, mmh, kc * BK, kp.ei_row + mb * BM, full_bar(s));
            tma_load_2d(st + 49152, mml, kc * BK, kp.ei_row + mb * BM, full_bar(s));
          }
          if constexpr (MN) {
            // 64 k-rows of 64 r, real plane then imaginary plane
            tma_load_3d(st + kOffX, mxh, r0, kc * BK, 0, full_bar(s));
            tma_load_3d(st + kOffX + 8192, mxh, r0, kc * BK, 1, full_bar(s));
            tma_load_3d(st + kOffX + 16384, mxl, r0, kc * BK, 0, full_bar(s));
            tma_load_3d(st + kOffX + 16384 + 8192, mxl, r0, kc * BK, 1, full_bar(s));
          } else {
            tma_load_2d(st + kOffX, mxh, kc * BK, r0, full_bar(s));
            tma_load_2d(st + kOffX + 8192, mxh, kc * BK, r1, full_bar(s));
            tma_load_2d(st + kOffX + 16384, mxl, kc * BK, r0, full_bar(s));
            tma_load_2d(st + kOffX + 16384 + 8192, mxl, kc * BK, r1, full_bar(s));
          }
        }
      }
      // drain: every issued stage must have landed before the CTA may exit
      const uint32_t issued = g;
      for (uint32_t q = issued >= NSTAGE ? issued - NSTAGE : 0; q < issued; ++q)
        mbar_wait(full_bar(q % NSTAGE), (q / NSTAGE) & 1, abort_flag, err, 7, true);
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      constexpr uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
                                 ((uint32_t)(BM >> 4) << 24) | (MN ? kTransB : 0u);
      constexpr uint32_t idesc64 = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BR >> 3) << 17) |
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
        if (!mbar_wait(acc_empty(a), ((t >> 1) & 1) ^ 1, abort_flag, err, 2)) break;
        tc_fence_after();
        const uint32_t d_tmem = tmem_base + a * BN;
        for (int kc = 0; kc < KC; ++kc, ++g) {
          const int s = (int)(g % NSTAGE);
          const uint32_t ph = (g / NSTAGE) & 1;
          if (!mbar_wait(full_bar(s), ph, abort_flag, err, 3)) { ok = false; break; }
          tc_fence_after();
          const uint32_t ahi = sbase + s * kStg, alo = ahi + 16384;
          const uint32_t bhi = ahi + kOffX, blo = bhi + 16384;
#pragma unroll
          for (int ks = 0; ks < BK / 16; ++ks) {
            const uint32_t off = ks * 32;
            const uint32_t acc0 = (kc > 0 || ks > 0) ? 1u : 0u;
            if constexpr (MN) {
              // k-step ks = k-rows 16 ks .. 16 ks + 15 (2048 bytes in); the
              // imaginary plane's 64 r follow 8 KB after the real plane's
              const uint64_t bh = sw128_mn_desc(bhi + ks * 2048, 8192), bl = sw128_mn_desc(blo + ks * 2048, 8192);
              mma_bf16(d_tmem, sw128_desc(ahi + off), bh, idesc, acc0);
              mma_bf16(d_tmem, sw128_desc(ahi + off), bl, idesc, 1u);
              mma_bf16(d_tmem, sw128_desc(alo + off), bh, idesc, 1u);
              continue;
            }
            mma_bf16(d_tmem, sw128_desc(ahi + off), sw128_desc(bhi + off), idesc, acc0);
            mma_bf16(d_tmem, sw128_desc(ahi + off), sw128_desc(blo + off), idesc, 1u);
            mma_bf16(d_tmem, sw128_desc(alo + off), sw128_desc(bhi + off), idesc, 1u);
            if constexpr (CX) {
              // Ei chunks at +32 KB (hi) and +48 KB (lo); X re rows at bhi, im rows at bhi + 8 KB
              const uint32_t eh = ahi + 32768, el = ahi + 49152;
              mma_bf16(d_tmem, sw128_desc(eh + off), sw128_desc(bhi + 8192 + off), idesc64 | kNegA, 1u);
              mma_bf16(d_tmem, sw128_desc(eh + off), sw128_desc(blo + 8192 + off), idesc64 | kNegA, 1u);
              mma_bf16(d_tmem, sw128_desc(el + off), sw128_desc(bhi + 8192 + off), idesc64 | kNegA, 1u);
              mma_bf16(d_tmem + BR, sw128_desc(eh + off), sw128_desc(bhi + off), idesc64, 1u);
              mma_bf16(d_tmem + BR, sw128_desc(eh + off), sw128_desc(blo + off), idesc64, 1u);
              mma_bf16(d_tmem + BR, sw128_desc(el + off), sw128_desc(bhi + off), idesc64, 1u);
            }
          }
          mma_commit(empty_bar(s));
        }
        if (!ok) break;
        mma_commit(acc_full(a));
      }
      // drain: all issued MMAs complete before TMEM is released
      mma_commit(fin_bar);
      mbar_wait(fin_bar, 0, abort_flag, err, 8, true);
    }
  } else {
    // ------------------------------------------------------------ epilogue
    const int q = warp & 3;            // TMEM lane quarter this warp may access
    const int half = (warp - 2) >> 2;  // first of this warp's 16-column groups
    float* stg = reinterpret_cast<float*>(smem + kOffEpi + (warp - 2) * kEpiWarp);
    const int rr = lane & 15, hrow = (lane >> 4) * 16;
    uint32_t t = 0;
    int pid = 0;
    for (long long u = blockIdx.x; u < units; u += gridDim.x, ++t) {
      const int a = t & 1;
      if (!mbar_wait(acc_full(a), (t >> 1) & 1, abort_flag, err, 9)) break;
      tc_fence_after();
      long long lu = u, Rl = kp.R;
      int mbk = kp.m_blocks, pl = kp.p;
      const Epi* Ep = &epi;
      if constexpr (G) {
        lu = locate(gd, ngd, u, pid);
        Rl = gd[pid].kp.R;
        mbk = gd[pid].kp.m_blocks;
        pl = gd[pid].kp.p;
        Ep = &gd[pid].epi;
      }
      const Epi& E = *Ep;
      const long long tile = lu / mbk;
      const int mb = (int)(lu % mbk);
      const int i_base = mb * BM + q * 32;
      // all of this warp's accumulator columns into registers, then hand the
      // accumulator back to the MMA warp before any store or functor work
      constexpr int NG = Cfg<Epi, CX>::kGroups;
      uint32_t vr[NG][16], vi[NG][16];
#pragma unroll
      for (int g2 = 0; g2 < NG; ++g2) {
        const int cc = half + (NEPI / 4) * g2;
        const uint32_t tl = tmem_base + ((uint32_t)(q * 32) << 16) + a * BN + cc * 16;
        tmem_ld16(tl, vr[g2]);
        tmem_ld16(tl + BR, vi[g2]);
      }
      tmem_wait_ld();
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(acc_empty(a));
#pragma unroll
      for (int g2 = 0; g2 < NG; ++g2) {
        const int cc = half + (NEPI / 4) * g2;   // 16-column group: r = r0 + 16 cc + 0..15
        {
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            stg[lane * 33 + j] = __uint_as_float(vr[g2][j]);
            stg[lane * 33 + 16 + j] = __uint_as_float(vi[g2][j]);
          }
          __syncwarp();
          constexpr int B = Epi::kBatch;
          constexpr int NI = Epi::kIn > 0 ? Epi::kIn : 1;
          const uint32_t R32 = (uint32_t)Rl;
          if ((R32 & 3u) == 0) {
            // 4 consecutive r per lane: lane = 4 a + k covers rows a, a + 8, .. and r = 16 cc + 4 k + 0..3
            const int k4 = lane & 3, a8 = lane >> 2;
            const uint32_t r = (uint32_t)(tile * BR + cc * 16 + 4 * k4);
#pragma unroll 1
            for (int it0 = 0; it0 < 4; it0 += B) {
              float in[B][NI][4];
#pragma unroll
              for (int b = 0; b < B; ++b) {
                const int i = i_base + a8 + 8 * (it0 + b);
                if (i < pl && r < R32) E.template load<4>((uint32_t)i * R32 + r, i, r, in[b]);
              }
#pragma unroll
              for (int b = 0; b < B; ++b) {
                const int ii = a8 + 8 * (it0 + b);
                const int i = i_base + ii;
                if (i < pl && r < R32) {
                  float re[4], im[4];
#pragma unroll
                  for (int v = 0; v < 4; ++v) {
                    re[v] = stg[ii * 33 + 4 * k4 + v];
                    im[v] = stg[ii * 33 + 16 + 4 * k4 + v];
                  }
                  E.template store<4>((uint32_t)i * R32 + r, i, r, re, im, in[b]);
                }
              }
            }
          } else {
            const uint32_t r = (uint32_t)(tile * BR + cc * 16 + rr);
#pragma unroll 1
            for (int it0 = 0; it0 < 16; it0 += B) {
              float in[B][NI][1];
#pragma unroll
              for (int b = 0; b < B; ++b) {
                const int i = i_base + it0 + b + hrow;
                if (i < pl && r < R32) E.template load<1>((uint32_t)i * R32 + r, i, r, in[b]);
              }
#pragma unroll
              for (int b = 0; b < B; ++b) {
                const int ii = it0 + b + hrow;
                const int i = i_base + ii;
                if (i < pl && r < R32) {
                  const float re[1] = {stg[ii * 33 + rr]}, im[1] = {stg[ii * 33 + 16 + rr]};
                  E.template store<1>((uint32_t)i * R32 + r, i, r, re, im, in[b]);
                }
              }
            }
          }
          __syncwarp();
        }
      }
    }
  }

  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(2 * BN));
}

}  // namespace b3
}  // namespace fcgle
