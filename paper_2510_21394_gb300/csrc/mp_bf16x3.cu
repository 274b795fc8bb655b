// Split-BF16 mu-mode product on the sm_103a tensor cores (tcgen05 + TMEM + TMA).
//
// Computes, in the rotating layout of common.h,
//     Y[c][i][r] = sum_k M[i][k] X[c][r][k]      (one mode product, Sec. 3.2)
// for FP32 X (2R rows of K = p floats) and a real p x p matrix M (Q_mu or
// Q_mu^T), with every operand split into two bf16 numbers, x = x_hi + x_lo,
// and the product formed as M_hi X_hi + M_hi X_lo + M_lo X_hi, accumulated in
// FP32 in tensor memory (the dropped M_lo X_lo term is below 2^-16 relative).
//
// GEMM orientation: D[i][col] = sum_k A[i][k] B[col][k] with A = M (MMA M =
// 128 output indices i per block), B = 128 data rows (c, r0..r0+127) of X
// (MMA N = 128), K in chunks of 64.
//
// Warp roles (10 warps, one CTA per SM, persistent over (data tile, i-block)
// units):
//   warp 0      TMA producer: M_hi, M_lo chunks (bf16, SWIZZLE_128B, straight
//               into the MMA layout) and the FP32 X chunk (unswizzled).
//   warp 1      TMEM allocator and single-thread MMA issuer.
//   warps 2-5   converters: FP32 X chunk -> (hi, lo) bf16 chunks written in
//               the K-major SWIZZLE_128B layout the MMA reads.
//   warps 6-9   epilogue: TMEM -> registers -> smem transpose -> coalesced
//               128-byte stores of Y rows.
// Pipelines: 2 TMA stages, 2 converted stages, 2 TMEM accumulators (2 x 128
// columns).  Every mbarrier wait is bounded by a wall-clock limit; on expiry
// the CTA records an error code in *err, drains its own TMA and MMA work,
// frees its TMEM and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <cstring>
#include <stdexcept>
#include <vector>

#include "common.h"
#include "engine.h"

namespace fcgle {

namespace {

constexpr int BM = 128;   // output indices i per MMA
constexpr int BN = 128;   // data rows per tile (MMA N)
constexpr int BK = 64;    // k per chunk (one 128-byte bf16 row)
constexpr int NTHREADS = 320;

constexpr uint32_t kAbStage = 65536;        // A_hi 16K | A_lo 16K | X32 32K
constexpr uint32_t kCStage = 32768;         // B_hi 16K | B_lo 16K
constexpr uint32_t kOffC = 2 * kAbStage;
constexpr uint32_t kOffEpi = kOffC + 2 * kCStage;
constexpr uint32_t kEpiWarp = 32 * 33 * 4;
constexpr uint32_t kOffBar = kOffEpi + 4 * kEpiWarp;
constexpr uint32_t kSmemBytes = kOffBar + 256 + 1024;   // + barriers + alignment slack

constexpr unsigned long long kTimeoutNs = 2000000000ull;   // 2 s per wait

// -------------------------------------------------------------- PTX helpers
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
__device__ __forceinline__ uint64_t sw128_desc(uint32_t addr) {
  // K-major, SWIZZLE_128B: rows of 128 bytes, 8-row groups 1024 bytes apart.
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}
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

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
        "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
        "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
        "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ uint32_t pack_bf16x2(float a, float b) {
  __nv_bfloat162 h = __floats2bfloat162_rn(a, b);   // .x = a in the low half
  return *reinterpret_cast<uint32_t*>(&h);
}

struct Params {
  float* Y;
  long long R;        // rows per plane of X (= other indices), Y row length
  int p;              // output extent (rows of Y per plane) and K
  int m_blocks;       // ceil(p / 128)
  int k_chunks;       // ceil(p / 64)
  long long tiles;    // data tiles: 2 planes x ceil(R / 128)
  int* err;
};

__global__ void __launch_bounds__(NTHREADS, 1)
    mp_bf16x3_kernel(const __grid_constant__ CUtensorMap tm_x, const __grid_constant__ CUtensorMap tm_ahi,
                     const __grid_constant__ CUtensorMap tm_alo, const Params prm) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const uint32_t sbase = smem_u32(smem);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + kOffBar);
  // barrier indices
  auto ab_full = [&](int s) { return smem_u32(&bars[0 + s]); };
  auto ab_empty = [&](int s) { return smem_u32(&bars[2 + s]); };
  auto c_full = [&](int s) { return smem_u32(&bars[4 + s]); };
  auto c_empty = [&](int s) { return smem_u32(&bars[6 + s]); };
  auto acc_full = [&](int a) { return smem_u32(&bars[8 + a]); };
  auto acc_empty = [&](int a) { return smem_u32(&bars[10 + a]); };
  const uint32_t fin_bar = smem_u32(&bars[12]);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + kOffBar + 128);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + kOffBar + 136);

  if (threadIdx.x == 0) {
    for (int s = 0; s < 2; ++s) {
      mbar_init(ab_full(s), 1);
      mbar_init(ab_empty(s), 1 + 4);   // MMA commit + 4 converter warps
      mbar_init(c_full(s), 4);         // 4 converter warps
      mbar_init(c_empty(s), 1);        // MMA commit
      mbar_init(acc_full(s), 1);       // MMA commit
      mbar_init(acc_empty(s), 4);      // 4 epilogue warps
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

  const long long units = prm.tiles * prm.m_blocks;
  const long long tiles_per_plane = (prm.R + BN - 1) / BN;
  const int KC = prm.k_chunks;

  if (warp == 0) {
    // ------------------------------------------------------------ producer
    if (lane == 0) {
      uint32_t g = 0;   // global chunk counter
      bool ok = true;
      for (long long u = blockIdx.x; u < units && ok; u += gridDim.x) {
        const long long tile = u / prm.m_blocks;
        const int mb = (int)(u % prm.m_blocks);
        const int c = (int)(tile / tiles_per_plane);
        const long long r0 = (tile % tiles_per_plane) * BN;
        const int xrow = (int)(c * prm.R + r0);
        for (int kc = 0; kc < KC; ++kc, ++g) {
          const int s = g & 1;
          const uint32_t ph = (g >> 1) & 1;
          if (!mbar_wait(ab_empty(s), ph ^ 1, abort_flag, prm.err, 1)) { ok = false; break; }
          const uint32_t st = sbase + s * kAbStage;
          mbar_arrive_tx(ab_full(s), kAbStage);
          tma_load_2d(st, &tm_ahi, kc * BK, mb * BM, ab_full(s));
          tma_load_2d(st + 16384, &tm_alo, kc * BK, mb * BM, ab_full(s));
          tma_load_2d(st + 32768, &tm_x, kc * BK, xrow, ab_full(s));
        }
      }
      // drain: every issued stage must have landed before the CTA may exit
      const uint32_t issued = g;
      for (uint32_t q = issued >= 2 ? issued - 2 : 0; q < issued; ++q)
        mbar_wait(ab_full(q & 1), (q >> 1) & 1, abort_flag, prm.err, 7, true);
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      constexpr uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
                                 ((uint32_t)(BM >> 4) << 24);
      uint32_t g = 0, t = 0;
      bool ok = true;
      for (long long u = blockIdx.x; u < units && ok; u += gridDim.x, ++t) {
        const int a = t & 1;
        if (!mbar_wait(acc_empty(a), ((t >> 1) & 1) ^ 1, abort_flag, prm.err, 2)) break;
        tc_fence_after();
        const uint32_t d_tmem = tmem_base + a * BN;
        for (int kc = 0; kc < KC; ++kc, ++g) {
          const int s = g & 1;
          const uint32_t ph = (g >> 1) & 1;
          if (!mbar_wait(ab_full(s), ph, abort_flag, prm.err, 3)) { ok = false; break; }
          if (!mbar_wait(c_full(s), ph, abort_flag, prm.err, 4)) { ok = false; break; }
          tc_fence_after();
          const uint32_t ahi = sbase + s * kAbStage, alo = ahi + 16384;
          const uint32_t bhi = sbase + kOffC + s * kCStage, blo = bhi + 16384;
#pragma unroll
          for (int ks = 0; ks < BK / 16; ++ks) {
            const uint32_t off = ks * 32;
            const uint32_t acc0 = (kc > 0 || ks > 0) ? 1u : 0u;
            mma_bf16(d_tmem, sw128_desc(ahi + off), sw128_desc(bhi + off), idesc, acc0);
            mma_bf16(d_tmem, sw128_desc(ahi + off), sw128_desc(blo + off), idesc, 1u);
            mma_bf16(d_tmem, sw128_desc(alo + off), sw128_desc(bhi + off), idesc, 1u);
          }
          mma_commit(ab_empty(s));
          mma_commit(c_empty(s));
        }
        if (!ok) break;
        mma_commit(acc_full(a));
      }
      // drain: all issued MMAs complete before TMEM is released
      mma_commit(fin_bar);
      mbar_wait(fin_bar, 0, abort_flag, prm.err, 8, true);
    }
  } else if (warp < 6) {
    // ------------------------------------------------------------ converters
    const int ct = threadIdx.x - 64;   // 0..127
    uint32_t g = 0;
    bool ok = true;
    for (long long u = blockIdx.x; u < units && ok; u += gridDim.x) {
      for (int kc = 0; kc < KC; ++kc, ++g) {
        const int s = g & 1;
        const uint32_t ph = (g >> 1) & 1;
        if (!mbar_wait(ab_full(s), ph, abort_flag, prm.err, 5)) { ok = false; break; }
        if (!mbar_wait(c_empty(s), ph ^ 1, abort_flag, prm.err, 6)) { ok = false; break; }
        const float* x32 = reinterpret_cast<const float*>(smem + s * kAbStage + 32768);
        uint8_t* bhi = smem + kOffC + s * kCStage;
        uint8_t* blo = bhi + 16384;
#pragma unroll 4
        for (int j = 0; j < 16; ++j) {
          const int idx = j * 128 + ct;        // float4 index in the 128 x 64 chunk
          const int row = idx >> 4, f = idx & 15;
          const float4 v = *reinterpret_cast<const float4*>(x32 + row * 64 + f * 4);
          const __nv_bfloat16 h0 = __float2bfloat16_rn(v.x), h1 = __float2bfloat16_rn(v.y);
          const __nv_bfloat16 h2 = __float2bfloat16_rn(v.z), h3 = __float2bfloat16_rn(v.w);
          const float l0 = v.x - __bfloat162float(h0), l1 = v.y - __bfloat162float(h1);
          const float l2 = v.z - __bfloat162float(h2), l3 = v.w - __bfloat162float(h3);
          uint2 hv, lv;
          hv.x = pack_bf16x2(__bfloat162float(h0), __bfloat162float(h1));
          hv.y = pack_bf16x2(__bfloat162float(h2), __bfloat162float(h3));
          lv.x = pack_bf16x2(l0, l1);
          lv.y = pack_bf16x2(l2, l3);
          const uint32_t off = row * 128 + ((((f >> 1) ^ (row & 7))) << 4) + (f & 1) * 8;
          *reinterpret_cast<uint2*>(bhi + off) = hv;
          *reinterpret_cast<uint2*>(blo + off) = lv;
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        if (lane == 0) {
          mbar_arrive(c_full(s));
          mbar_arrive(ab_empty(s));
        }
      }
    }
  } else {
    // ------------------------------------------------------------ epilogue
    const int q = warp & 3;   // TMEM lane quarter this warp may access
    float* stg = reinterpret_cast<float*>(smem + kOffEpi + (warp - 6) * kEpiWarp);
    uint32_t t = 0;
    for (long long u = blockIdx.x; u < units; u += gridDim.x, ++t) {
      const int a = t & 1;
      if (!mbar_wait(acc_full(a), (t >> 1) & 1, abort_flag, prm.err, 9)) break;
      tc_fence_after();
      const long long tile = u / prm.m_blocks;
      const int mb = (int)(u % prm.m_blocks);
      const int c = (int)(tile / tiles_per_plane);
      const long long r0 = (tile % tiles_per_plane) * BN;
      const int i_base = mb * BM + q * 32;
      float* Yp = prm.Y + (long long)c * prm.p * prm.R;
#pragma unroll 1
      for (int cc = 0; cc < BN / 32; ++cc) {
        uint32_t v[32];
        tmem_ld32(tmem_base + ((uint32_t)(q * 32) << 16) + a * BN + cc * 32, v);
#pragma unroll
        for (int j = 0; j < 32; ++j) stg[lane * 33 + j] = __uint_as_float(v[j]);
        __syncwarp();
        const long long r = r0 + cc * 32 + lane;
#pragma unroll 4
        for (int ii = 0; ii < 32; ++ii) {
          const int i = i_base + ii;
          if (i < prm.p && r < prm.R) Yp[(long long)i * prm.R + r] = stg[ii * 33 + lane];
        }
        __syncwarp();
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(acc_empty(a));
    }
  }

  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(2 * BN));
}

// ------------------------------------------------------------------ host
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    cudaDriverEntryPointQueryResult q;
    void* p = nullptr;
    FCGLE_CUDA(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q));
    if (q != cudaDriverEntryPointSuccess || !p) throw std::runtime_error("cuTensorMapEncodeTiled unavailable");
    fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

void encode_2d(void* map, CUtensorMapDataType dt, const void* base, uint64_t inner, uint64_t outer,
               uint64_t row_bytes, uint32_t box_inner, uint32_t box_outer, CUtensorMapSwizzle sw) {
  cuuint64_t dims[2] = {inner, outer};
  cuuint64_t strides[1] = {row_bytes};
  cuuint32_t box[2] = {box_inner, box_outer};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = encode_fn()(reinterpret_cast<CUtensorMap*>(map), dt, 2, const_cast<void*>(base), dims, strides, box,
                           estr, CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) throw std::runtime_error("cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
}

int g_sms = 0;

}  // namespace

int bf16x3_num_sms() {
  if (!g_sms) {
    int dev = 0;
    FCGLE_CUDA(cudaGetDevice(&dev));
    FCGLE_CUDA(cudaDeviceGetAttribute(&g_sms, cudaDevAttrMultiProcessorCount, dev));
  }
  return g_sms;
}

void bf16x3_prepare(const double* M, int p, Bf16x3Op& op) {
  op.p = p;
  op.m_pad = (p + BM - 1) / BM * BM;
  op.k_pad = (p + BK - 1) / BK * BK;
  std::vector<__nv_bfloat16> hi((size_t)op.m_pad * op.k_pad, __float2bfloat16(0.0f));
  std::vector<__nv_bfloat16> lo(hi);
  for (int i = 0; i < p; ++i)
    for (int k = 0; k < p; ++k) {
      const double x = M[(size_t)i * p + k];
      const __nv_bfloat16 h = __float2bfloat16_rn((float)x);
      hi[(size_t)i * op.k_pad + k] = h;
      lo[(size_t)i * op.k_pad + k] = __float2bfloat16_rn((float)(x - (double)__bfloat162float(h)));
    }
  const size_t bytes = hi.size() * sizeof(__nv_bfloat16);
  FCGLE_CUDA(cudaMalloc(&op.hi, bytes));
  FCGLE_CUDA(cudaMalloc(&op.lo, bytes));
  FCGLE_CUDA(cudaMemcpy(op.hi, hi.data(), bytes, cudaMemcpyHostToDevice));
  FCGLE_CUDA(cudaMemcpy(op.lo, lo.data(), bytes, cudaMemcpyHostToDevice));
  encode_2d(op.tmap_hi, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, op.hi, op.k_pad, op.m_pad, (uint64_t)op.k_pad * 2, BK, BM,
            CU_TENSOR_MAP_SWIZZLE_128B);
  encode_2d(op.tmap_lo, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, op.lo, op.k_pad, op.m_pad, (uint64_t)op.k_pad * 2, BK, BM,
            CU_TENSOR_MAP_SWIZZLE_128B);
}

void bf16x3_release(Bf16x3Op& op) {
  if (op.hi) cudaFree(op.hi);
  if (op.lo) cudaFree(op.lo);
  op.hi = op.lo = nullptr;
}

void mp_bf16x3(const float* X, float* Y, const Bf16x3Op& op, size_t R, int* err, cudaStream_t st, long long& nl) {
  static bool attr = false;
  if (!attr) {
    FCGLE_CUDA(cudaFuncSetAttribute(mp_bf16x3_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes));
    attr = true;
  }
  alignas(64) CUtensorMap tm_x;
  encode_2d(&tm_x, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, X, (uint64_t)op.p, 2 * (uint64_t)R, (uint64_t)op.p * 4, BK, BN,
            CU_TENSOR_MAP_SWIZZLE_NONE);
  CUtensorMap tm_hi, tm_lo;
  std::memcpy(&tm_hi, op.tmap_hi, sizeof(CUtensorMap));
  std::memcpy(&tm_lo, op.tmap_lo, sizeof(CUtensorMap));
  Params prm;
  prm.Y = Y;
  prm.R = (long long)R;
  prm.p = op.p;
  prm.m_blocks = op.m_pad / BM;
  prm.k_chunks = op.k_pad / BK;
  prm.tiles = 2 * (((long long)R + BN - 1) / BN);
  prm.err = err;
  const long long units = prm.tiles * prm.m_blocks;
  const int grid = (int)std::min<long long>(units, bf16x3_num_sms());
  mp_bf16x3_kernel<<<grid, NTHREADS, kSmemBytes, st>>>(tm_x, tm_hi, tm_lo, prm);
  FCGLE_LAUNCHED(nl);
}

}  // namespace fcgle
