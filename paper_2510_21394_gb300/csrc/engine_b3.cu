// Split-BF16 engine (FCGLE_BF16X3 handles): complex64 storage, tensor-core
// mode products with fused pointwise epilogues.
//
// Storage.  FP32 planar tensors (common.h layout) for everything pointwise
// code reads (u_n, U^_n, F^_n, D^_2, D^_3, the phi tensors, sources); split
// tensors (two bf16 arrays hi, lo, each 2 P elements) for everything a mode
// product reads.  Splitting x = hi + lo at write time loses nothing: the
// mode product consumes exactly hi and lo.
//
// Each time step is a chain of Tucker operators (Eq. fKu_diag); the last mode
// product of every Tucker operator carries the scheme's pointwise work in its
// epilogue (b3_epilogues.cuh) and writes the split input of the next Tucker
// operator, so no standalone pointwise pass runs inside the time loop.
// Per Krogstad step (Eq. krogstad-m, F^_n = Lam o U^_n + G^_n with U^_n
// carried): 4 forward + 4 backward Tucker operators = 24 launches for d = 3.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <cmath>
#include <cstddef>
#include <cstdio>
#include <complex>
#include <cstdlib>
#include <cstring>
#include <utility>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "adjoint.h"
#include "b3_epilogues.cuh"
#include "b3_kernel.cuh"
#include "b3_plain.cuh"
#include "b3_slab.cuh"
#include "engine.h"

namespace fcgle {

using b3::SplitOut;

namespace {

template <typename T>
struct DevMem {
  T* ptr = nullptr;
  DevMem() = default;
  explicit DevMem(size_t n) { FCGLE_CUDA(cudaMalloc(&ptr, n * sizeof(T))); }
  ~DevMem() {
    if (ptr) cudaFree(ptr);
  }
  DevMem(const DevMem&) = delete;
  DevMem& operator=(const DevMem&) = delete;
};

// Programmatic dependent launch of the mode-product kernels (on unless the
// environment sets FCGLE_PDL=0): the kernel may be scheduled while the previous
// kernel of the stream drains and runs its prologue meanwhile; it waits for
// that kernel's completion (griddepcontrol.wait) before any global access.
bool pdl_enabled() {
  static const bool on = [] {
    const char* e = std::getenv("FCGLE_PDL");
    return !(e && e[0] == '0');
  }();
  return on;
}

template <class... P, class... A>
void launch_pdl(void (*kernel)(P...), int grid, int threads, size_t smem, cudaStream_t st, A&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3((unsigned)threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl_enabled() ? 1 : 0;
  FCGLE_CUDA(cudaLaunchKernelEx(&cfg, kernel, std::forward<A>(args)...));
}

// ------------------------------------------------ plain-product autotuner
// Ring configurations of the plain mode product (b3_plain.cuh); which one is
// fastest depends on the contracted extent p (k-chunks per unit) and on how
// many units each SM gets, so each distinct (p, R) is timed once per process
// (all eligible configurations, on the handle's own work buffers, at setup) and
// the fastest is used from then on.  FCGLE_PLAIN_CFG=<id> (read once) forces
// one configuration where it is eligible.
enum PlainCfg { kCfgX4M2 = 0, kCfgX3M3 = 1, kCfgX2M4 = 2, kCfgMR = 3, kCfgMH = 4, kCfgWide = 5, kNumPlainCfg = 6 };
const char* const kPlainCfgName[kNumPlainCfg] = {"X4M2", "X3M3", "X2M4", "residentM", "residentMhi", "wide128"};

using PlainKernel = void (*)(CUtensorMap, CUtensorMap, CUtensorMap, CUtensorMap, CUtensorMap, CUtensorMap,
                             b3::KParams, const b3::PlainDesc*, int, long long);

PlainKernel plain_kernel(int cfg) {
  switch (cfg) {
    case kCfgX3M3: return b3::mp_b3_plain_kernel<false, b3::kOpBF16, 3>;
    case kCfgX2M4: return b3::mp_b3_plain_kernel<false, b3::kOpBF16, 2>;
    case kCfgMR: return b3::mp_b3_plain_kernel<false, b3::kOpBF16, 2, true>;
    case kCfgMH: return b3::mp_b3_plain_kernel<false, b3::kOpBF16, 3, false, false, true>;
    case kCfgWide: return b3::mp_b3_plain_kernel<false, b3::kOpBF16, 2, false, false, false, 2>;
    default: return b3::mp_b3_plain_kernel<false>;
  }
}

int forced_plain_cfg() {
  static const int c = [] {
    const char* e = std::getenv("FCGLE_PLAIN_CFG");
    if (!e || !*e) return -1;
    const int v = std::atoi(e);
    return (v >= 0 && v < kNumPlainCfg) ? v : -1;
  }();
  return c;
}

struct TuneEntry {
  int cfg = kCfgX4M2;
  float us[kNumPlainCfg] = {-1.f, -1.f, -1.f, -1.f, -1.f, -1.f};   // -1: not eligible
};
std::mutex g_tune_mu;
std::map<std::tuple<int, long long>, TuneEntry> g_tune;   // (p, R)

// Tucker-operator form of 3D handles (p1, p2, p3): the rotating chain of
// three products, or the slab-fused modes 1 + 2 followed by the natural-order
// mode-3 product; timed once per process per shape at setup.
struct SlabTune {
  float us_rot = -1.f, us_slab = -1.f;
  bool slab = false;
};
std::map<std::tuple<int, int, int>, SlabTune> g_slab;

bool tuned_lookup(int p, long long R, TuneEntry& e) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  auto it = g_tune.find(std::make_tuple(p, R));
  if (it == g_tune.end()) return false;
  e = it->second;
  return true;
}

}  // namespace

static std::vector<std::string> g_tune_lines;   // tuned phases of batches

void add_tune_report_line(const std::string& line) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune_lines.push_back(line);
}

// Text report of the autotuner's choices (C ABI: fcgle_autotune_report).
std::string plain_tune_report() {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  std::string out;
  for (const auto& l : g_tune_lines) out += l + "\n";
  char line[256];
  for (const auto& kv : g_tune) {
    int n = std::snprintf(line, sizeof(line), "plain p=%d R=%lld:", std::get<0>(kv.first), std::get<1>(kv.first));
    out.append(line, (size_t)n);
    for (int c = 0; c < kNumPlainCfg; ++c)
      if (kv.second.us[c] >= 0.f) {
        n = std::snprintf(line, sizeof(line), " %s %.2fus", kPlainCfgName[c], kv.second.us[c]);
        out.append(line, (size_t)n);
      }
    n = std::snprintf(line, sizeof(line), " -> %s\n", kPlainCfgName[kv.second.cfg]);
    out.append(line, (size_t)n);
  }
  for (const auto& kv : g_slab) {
    const int n = std::snprintf(line, sizeof(line), "tucker p=(%d,%d,%d): rotating %.2fus slab-fused %.2fus -> %s\n",
                                std::get<0>(kv.first), std::get<1>(kv.first), std::get<2>(kv.first),
                                kv.second.us_rot, kv.second.us_slab, kv.second.slab ? "slab-fused" : "rotating");
    out.append(line, (size_t)n);
  }
  return out;
}

namespace {

int num_sms() {
  static const int sms = [] {   // thread-safe one-time initialisation
    int dev = 0, m = 0;
    FCGLE_CUDA(cudaGetDevice(&dev));
    FCGLE_CUDA(cudaDeviceGetAttribute(&m, cudaDevAttrMultiProcessorCount, dev));
    return m;
  }();
  return sms;
}

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

// 2D bf16 tensor map, SWIZZLE_128B, box (64 inner, box_rows outer).
void encode_bf16(CUtensorMap* map, const void* base, uint64_t inner, uint64_t rows, uint32_t box_rows) {
  cuuint64_t dims[2] = {inner, rows};
  cuuint64_t strides[1] = {inner * 2};
  cuuint32_t box[2] = {(cuuint32_t)b3::BK, box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = encode_fn()(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) throw std::runtime_error("cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
}

// 3D bf16 tensor map over a split output plane pair [2][p][R], box (32, 32, 1),
// no swizzle: the TMA-store epilogue writes 32 x 32 element boxes.
void encode_bf16_out(CUtensorMap* map, const void* base, uint64_t R, uint64_t p) {
  cuuint64_t dims[3] = {R, p, 2};
  cuuint64_t strides[2] = {R * 2, R * p * 2};
  cuuint32_t box[3] = {32, 32, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = encode_fn()(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(base), dims, strides, box, estr,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                           CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) throw std::runtime_error("cuTensorMapEncodeTiled (store) failed (" + std::to_string((int)r) + ")");
}

// 2D bf16 tensor map, SWIZZLE_64B, box (32 inner = 64 bytes, box_rows outer):
// the operands of the slab-fused product, in 32-wide k-chunks.
void encode_bf16_sw64(CUtensorMap* map, const void* base, uint64_t inner, uint64_t rows, uint32_t box_rows) {
  cuuint64_t dims[2] = {inner, rows};
  cuuint64_t strides[1] = {inner * 2};
  cuuint32_t box[2] = {32, box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = encode_fn()(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) throw std::runtime_error("cuTensorMapEncodeTiled (sw64) failed (" + std::to_string((int)r) + ")");
}

// 3D bf16 tensor map (dims d0 fastest), the given box and swizzle (0, 64 or 128 bytes).
void encode_bf16_3d(CUtensorMap* map, const void* base, uint64_t d0, uint64_t d1, uint64_t d2, uint32_t b0, uint32_t b1,
                    int swizzle) {
  cuuint64_t dims[3] = {d0, d1, d2};
  cuuint64_t strides[2] = {d0 * 2, d0 * d1 * 2};
  cuuint32_t box[3] = {b0, b1, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  const CUtensorMapSwizzle sw = swizzle == 128  ? CU_TENSOR_MAP_SWIZZLE_128B
                                : swizzle == 64 ? CU_TENSOR_MAP_SWIZZLE_64B
                                                : CU_TENSOR_MAP_SWIZZLE_NONE;
  CUresult r = encode_fn()(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(base), dims, strides, box, estr,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, sw,
                           swizzle ? CU_TENSOR_MAP_L2_PROMOTION_L2_256B : CU_TENSOR_MAP_L2_PROMOTION_NONE,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) throw std::runtime_error("cuTensorMapEncodeTiled (3D) failed (" + std::to_string((int)r) + ")");
}

// 2D FP32 tensor map, SWIZZLE_128B, box (32 inner = 128 bytes, box_rows outer):
// split-TF32 operands of the precise transforms.
void encode_f32(CUtensorMap* map, const void* base, uint64_t inner, uint64_t rows, uint32_t box_rows) {
  cuuint64_t dims[2] = {inner, rows};
  cuuint64_t strides[1] = {inner * 4};
  cuuint32_t box[2] = {32, box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = encode_fn()(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(base), dims, strides, box, estr,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) throw std::runtime_error("cuTensorMapEncodeTiled (f32) failed (" + std::to_string((int)r) + ")");
}

// 3D FP32 tensor map over an output plane pair [2][p][R], box (32, 32, 1), no swizzle.
void encode_f32_out(CUtensorMap* map, const void* base, uint64_t R, uint64_t p) {
  cuuint64_t dims[3] = {R, p, 2};
  cuuint64_t strides[2] = {R * 4, R * p * 4};
  cuuint32_t box[3] = {32, 32, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = encode_fn()(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void*>(base), dims, strides, box, estr,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                           CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS)
    throw std::runtime_error("cuTensorMapEncodeTiled (f32 store) failed (" + std::to_string((int)r) + ")");
}

// x rounded to TF32 on the host (10 explicit mantissa bits, ties away from
// zero), the same rounding as the device's cvt.rna.tf32.f32 for finite x
float tf32_rna_host(float x) {
  uint32_t u;
  std::memcpy(&u, &x, 4);
  u = (u + 0x1000u) & ~0x1FFFu;
  float y;
  std::memcpy(&y, &u, 4);
  return y;
}

// ------------------------------------------------------ standalone kernels
// (P is a multiple of 8: every kernel handles 4 consecutive elements per step)

// V = a u + b g(t, u) (split); optionally V2 = a2 u + b2 g(t, u) (split)
__global__ void gsplit_kernel(uint32_t P, b3::GStatic g, b3::GTime t, const float* __restrict__ U, float a, float b,
                              SplitOut V, float a2, float b2, SplitOut V2) {
  for (uint32_t q = 4 * (blockIdx.x * blockDim.x + threadIdx.x); q < P; q += 4 * gridDim.x * blockDim.x) {
    float ur[4], ui[4], gr[4] = {0, 0, 0, 0}, gi[4] = {0, 0, 0, 0}, xr[4], xi[4];
    b3::ldv<4>(U + q, ur);
    b3::ldv<4>(U + P + q, ui);
    if (b != 0.f || (V2.hi && b2 != 0.f)) b3::g_eval<4>(g, t, P, q, ur, ui, gr, gi);
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      xr[v] = a * ur[v] + b * gr[v];
      xi[v] = a * ui[v] + b * gi[v];
    }
    b3::put_csplit<4>(V, P, q, xr, xi);
    if (V2.hi) {
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        xr[v] = a2 * ur[v] + b2 * gr[v];
        xi[v] = a2 * ui[v] + b2 * gi[v];
      }
      b3::put_csplit<4>(V2, P, q, xr, xi);
    }
  }
}

// V = Phi_t(u) (split)
// U = Phi_t(W)
__global__ void flow_kernel(uint32_t P, b3::Flow f, const float* __restrict__ W, float* __restrict__ U) {
  for (uint32_t q = 4 * (blockIdx.x * blockDim.x + threadIdx.x); q < P; q += 4 * gridDim.x * blockDim.x) {
    float wr[4], wi[4], ur[4], ui[4];
    b3::ldv<4>(W + q, wr);
    b3::ldv<4>(W + P + q, wi);
#pragma unroll
    for (int v = 0; v < 4; ++v) b3::flow_eval(f, wr[v], wi[v], ur[v], ui[v]);
    b3::stv<4>(U + q, ur);
    b3::stv<4>(U + P + q, ui);
  }
}

// V = Phi_t(u) -> split (Strang's first half step, Kronecker-product form)
__global__ void flow_split_kernel(uint32_t P, b3::Flow f, const float* __restrict__ U, SplitOut V) {
  for (uint32_t q = 4 * (blockIdx.x * blockDim.x + threadIdx.x); q < P; q += 4 * gridDim.x * blockDim.x) {
    float ur[4], ui[4], vr[4], vi[4];
    b3::ldv<4>(U + q, ur);
    b3::ldv<4>(U + P + q, ui);
#pragma unroll
    for (int v = 0; v < 4; ++v) b3::flow_eval(f, ur[v], ui[v], vr[v], vi[v]);
    b3::put_csplit<4>(V, P, q, vr, vi);
  }
}

// V = Phi_t(u) - u -> split (Strang's first half step as an increment)
__global__ void flow_incr_split_kernel(uint32_t P, b3::Flow f, const float* __restrict__ U, SplitOut V) {
  for (uint32_t q = 4 * (blockIdx.x * blockDim.x + threadIdx.x); q < P; q += 4 * gridDim.x * blockDim.x) {
    float ur[4], ui[4], vr[4], vi[4];
    b3::ldv<4>(U + q, ur);
    b3::ldv<4>(U + P + q, ui);
#pragma unroll
    for (int v = 0; v < 4; ++v) b3::flow_incr(f, ur[v], ui[v], vr[v], vi[v]);
    b3::put_csplit<4>(V, P, q, vr, vi);
  }
}

// FP32 -> split-TF32: hi = tf32(x), lo = tf32(x - hi); n % 4 == 0
__global__ void tf32_split_kernel(uint32_t n, const float* __restrict__ X, float* __restrict__ hi,
                                  float* __restrict__ lo) {
  for (uint32_t q = 4 * (blockIdx.x * blockDim.x + threadIdx.x); q < n; q += 4 * gridDim.x * blockDim.x) {
    float x[4], h[4], l[4];
    b3::ldv<4>(X + q, x);
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      h[v] = b3::tf32_round(x[v]);
      l[v] = b3::tf32_round(x[v] - h[v]);
    }
    b3::stv<4>(hi + q, h);
    b3::stv<4>(lo + q, l);
  }
}

// FP32 -> split (raw mode-product entry point); n % 4 == 0
__global__ void to_split_kernel(uint32_t n, const float* __restrict__ X, SplitOut Y) {
  for (uint32_t q = 4 * (blockIdx.x * blockDim.x + threadIdx.x); q < n; q += 4 * gridDim.x * blockDim.x) {
    float x[4];
    b3::ldv<4>(X + q, x);
    b3::put_split<4>(Y, q, x);
  }
}

// f(theta lam_j) with lam_j = (c_re + i c_im) s_j as the epilogues evaluate it:
// ray == 0: fspec on z = theta lam (the apply_f epilogue); ray != 0: phi_ell
// (ell in 1..3) by the per-launch polynomial along the ray (the scheme epilogues)
__global__ void scalars_b3_kernel(int n, const double* __restrict__ sv, float c_re, float c_im, float theta, int kind,
                                  int ray, b3::PhiPoly ph, int ell, double* __restrict__ out) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
    const float s = (float)sv[j];
    float fr, fi;
    if (ray) {
      float pr[3], pi[3];
      b3::phi123_s(ph, s, pr, pi);
      fr = pr[ell - 1];
      fi = pi[ell - 1];
    } else {
      b3::fspec(kind, theta * (c_re * s), theta * (c_im * s), fr, fi);
    }
    out[2 * j] = fr;
    out[2 * j + 1] = fi;
  }
}

int grid_for(long long n) {
  long long g = (n + 255) / 256;
  const long long cap = (long long)num_sms() * 16;
  return (int)std::max<long long>(1, std::min(g, cap));
}

}  // namespace

// =========================================================== the engine
class EngineB3 : public EngineBase {
 public:
  EngineB3(const fcgle_params& prm, cudaStream_t st) : prm_(prm), st_(st) {
    s_.d = prm.d;
    s_.P = 1;
    s_.N = 1;
    for (int mu = 0; mu < kMaxDim; ++mu) {
      s_.n[mu] = mu < prm.d ? prm.n[mu] : 1;
      s_.p[mu] = mu < prm.d ? ((prm.n[mu] + 7) & ~7) : 1;   // 16-byte bf16 rows
      s_.P *= (size_t)s_.p[mu];
      s_.N *= (size_t)s_.n[mu];
    }
    P_ = (long long)s_.P;
    if (2 * s_.P >= (size_t(1) << 32)) throw Unsupported("BF16X3 handles need 2 P < 2^32 internal elements");
    for (int mu = 0; mu < prm.d; ++mu) {
      Direction D = spectral_direction(prm, mu);
      h_[mu] = D.h;
      dir_[mu] = D;   // Q_mu, lam_mu kept for the exponential matrices E_mu
      std::vector<float> lf(s_.p[mu], 0.f);
      std::vector<double> ld(s_.p[mu], 0.0);
      for (int j = 0; j < D.n; ++j) {
        lf[j] = (float)D.lam[j];
        ld[j] = D.lam[j];
      }
      lamf_[mu].reset(new DevMem<float>(s_.p[mu]));
      lamd_[mu].reset(new DevMem<double>(s_.p[mu]));
      FCGLE_CUDA(cudaMemcpy(lamf_[mu]->ptr, lf.data(), lf.size() * 4, cudaMemcpyHostToDevice));
      FCGLE_CUDA(cudaMemcpy(lamd_[mu]->ptr, ld.data(), ld.size() * 8, cudaMemcpyHostToDevice));
      const int p = s_.p[mu];
      std::vector<double> Mf((size_t)p * p, 0.0), Mb((size_t)p * p, 0.0);
      for (int i = 0; i < D.n; ++i)
        for (int k = 0; k < D.n; ++k) {
          Mf[(size_t)i * p + k] = D.Q[(size_t)k * D.n + i];   // Q^T
          Mb[(size_t)i * p + k] = D.Q[(size_t)i * D.n + k];   // Q
        }
      prepare_matrix(Mf.data(), p, mat_[mu][0]);
      prepare_matrix(Mb.data(), p, mat_[mu][1]);
    }
    lf_.d = prm.d;
    lf_.c_re = (float)prm.nu;
    lf_.c_im = (float)prm.eta;
    for (int mu = 0; mu < kMaxDim; ++mu) {
      lf_.lam[mu] = mu < prm.d ? lamf_[mu]->ptr : nullptr;
      lf_.p[mu] = s_.p[mu];
    }
    gs_.gamma = (float)prm.gamma;
    gs_.kappa = (float)prm.kappa;
    gs_.zeta = (float)prm.zeta;
    gs_.nsrc = 0;
    for (int i = 0; i < kNumF32; ++i) {
      f32_[i].reset(new DevMem<float>(2 * s_.P));
      FCGLE_CUDA(cudaMemsetAsync(f32_[i]->ptr, 0, 2 * s_.P * 4, st_));
    }
    for (int i = 0; i < kNumSplit; ++i) {
      sp_[i].reset(new DevMem<__nv_bfloat16>(4 * s_.P));
      FCGLE_CUDA(cudaMemsetAsync(sp_[i]->ptr, 0, 4 * s_.P * 2, st_));
    }
    scratch_.reset(new DevMem<double>(4));
    err_.reset(new DevMem<int>(1));
    FCGLE_CUDA(cudaMemsetAsync(err_->ptr, 0, sizeof(int), st_));
    FCGLE_CUDA(cudaStreamSynchronize(st_));
    // once per process (instances of a batch are set up in parallel threads);
    // an exception leaves the flag unset, so a later setup retries
    static std::once_flag attrs;
    std::call_once(attrs, [] {
      set_smem_attr<b3::EpiStoreSplitGen>();
      set_smem_attr<b3::EpiStoreF32>();
      set_smem_attr<b3::EpiScaleF>();
      set_smem_attr<b3::EpiUpdateG>();
      set_smem_attr<b3::EpiStageD>();
      set_smem_attr<b3::EpiFhat>();
      set_smem_attr<b3::EpiKrog2>();
      set_smem_attr<b3::EpiKrog3>();
      set_smem_attr<b3::EpiKrogFinal>();
      set_smem_attr<b3::EpiEtd2>();
      set_smem_attr<b3::EpiSpecStep>();
      set_smem_attr<b3::EpiLBDF2S>();
      set_smem_attr<b3::EpiExtrapG>();
      set_smem_attr<b3::EpiLRK2A>();
      set_smem_attr<b3::EpiLRK2B>();
      set_smem_attr<b3::EpiStrangB>();
      set_smem_attr_mn<b3::EpiStoreSplitGen>();
      set_smem_attr_mn<b3::EpiStoreF32>();
      set_smem_attr_mn<b3::EpiScaleF>();
      set_smem_attr_mn<b3::EpiUpdateG>();
      set_smem_attr_mn<b3::EpiStageD>();
      set_smem_attr_mn<b3::EpiFhat>();
      set_smem_attr_mn<b3::EpiKrog2>();
      set_smem_attr_mn<b3::EpiKrog3>();
      set_smem_attr_mn<b3::EpiKrogFinal>();
      set_smem_attr_mn<b3::EpiEtd2>();
      set_smem_attr_mn<b3::EpiSpecStep>();
      set_smem_attr_mn<b3::EpiLBDF2S>();
      set_smem_attr_mn<b3::EpiExtrapG>();
      set_smem_attr_mn<b3::EpiLRK2A>();
      set_smem_attr_mn<b3::EpiLRK2B>();
      set_smem_attr_mn<b3::EpiStrangB>();
      FCGLE_CUDA(cudaFuncSetAttribute(b3::mp_b3_slab12_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)b3::kSlSmemBytes));
      set_smem_attr_cx<b3::EpiStoreF32>();
      set_smem_attr_cx<b3::EpiStoreSplitGen>();
      set_smem_attr_cx<b3::EpiUpdateG>();
      set_smem_attr_cx<b3::EpiStrangKron>();
      set_smem_attr_cx<b3::EpiLRK2Kron>();
      FCGLE_CUDA(cudaFuncSetAttribute(b3::mp_b3_plain_kernel<false, b3::kOpBF16, 2, false, true>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b3::kPlSmemBytes));
      FCGLE_CUDA(cudaFuncSetAttribute(b3::mp_b3_plain_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)b3::kPlSmemBytes));
      for (int c = 0; c < kNumPlainCfg; ++c)
        FCGLE_CUDA(cudaFuncSetAttribute(plain_kernel(c), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)b3::kPlSmemBytes));
      FCGLE_CUDA(cudaFuncSetAttribute(b3::mp_b3_plain_kernel<false, b3::kOpTF32>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b3::kPlSmemBytes));
      FCGLE_CUDA(cudaFuncSetAttribute(b3::mp_b3_plain_kernel<false, b3::kOpTF32F>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b3::kPlSmemBytes));
    });
  }

  ~EngineB3() override {
    for (int mu = 0; mu < kMaxDim; ++mu)
      for (int f = 0; f < 2; ++f) {
        if (mat_[mu][f].hi) cudaFree(mat_[mu][f].hi);
        if (mat_[mu][f].lo) cudaFree(mat_[mu][f].lo);
        if (mat_[mu][f].f32) cudaFree(mat_[mu][f].f32);
        if (mat_[mu][f].thi) cudaFree(mat_[mu][f].thi);
        if (mat_[mu][f].tlo) cudaFree(mat_[mu][f].tlo);
      }
  }

  void set_stream(cudaStream_t st) override { st_ = st; }
  size_t internal_elems() const override { return s_.P; }
  size_t elem_bytes() const override { return 8; }

  void set_source(int nterms, const double* sig, const void* const* S_user) override {
    for (int k = 0; k < nterms; ++k) {
      if (!src_[k]) src_[k].reset(new DevMem<float>(2 * s_.P));
      pack_f32((const float*)S_user[k], src_[k]->ptr);
      sig_re_[k] = sig[2 * k];
      sig_im_[k] = sig[2 * k + 1];
      gs_.S[k] = src_[k]->ptr;
    }
    for (int k = nterms; k < kMaxSrc; ++k) gs_.S[k] = nullptr;
    gs_.nsrc = nterms;
  }

  void set_coefficients(double nu, double eta, double gamma, double kappa, double zeta) override {
    prm_.nu = nu;
    prm_.eta = eta;
    prm_.gamma = gamma;
    prm_.kappa = kappa;
    prm_.zeta = zeta;
    lf_.c_re = (float)nu;
    lf_.c_im = (float)eta;
    gs_.gamma = (float)gamma;
    gs_.kappa = (float)kappa;
    gs_.zeta = (float)zeta;
    FCGLE_CUDA(cudaStreamSynchronize(st_));   // cached E_mu may still be in use
    ecache_.clear();
  }

  void set_exp_form(int form) override {
    if (form != FCGLE_EXP_TUCKER && form != FCGLE_EXP_KRON) throw InvalidArg("unknown exponential form");
    exp_form_ = form;
  }

  void set_tucker_form(int form) override {
    if (form < FCGLE_TUCKER_AUTO || form > FCGLE_TUCKER_SLAB) throw InvalidArg("unknown Tucker-operator form");
    if (form == FCGLE_TUCKER_SLAB && !slab_ok())
      throw Unsupported("the slab-fused form needs d == 3 and p_2 <= 256");
    tucker_form_ = form;
  }

  void spectral_scalars(int func, int k, double theta, int count, const double* s_host, double* out_host,
                        int flags) override {
    const bool ray = flags & 1;
    if (ray && (func != FCGLE_F_PHI || k < 1 || k > 3))
      throw InvalidArg("the ray polynomial form evaluates phi_1..phi_3 only");
    if (count <= 0) return;
    DevMem<double> sd((size_t)count), od(2 * (size_t)count);
    FCGLE_CUDA(cudaMemcpyAsync(sd.ptr, s_host, (size_t)count * 8, cudaMemcpyHostToDevice, st_));
    scalars_b3_kernel<<<grid_for(count), 256, 0, st_>>>(count, sd.ptr, lf_.c_re, lf_.c_im, (float)theta,
                                                       fkind(func, k), ray ? 1 : 0, phipoly(theta), k, od.ptr);
    FCGLE_LAUNCHED(launches);
    FCGLE_CUDA(cudaMemcpyAsync(out_host, od.ptr, 2 * (size_t)count * 8, cudaMemcpyDeviceToHost, st_));
    FCGLE_CUDA(cudaStreamSynchronize(st_));
  }

  int device_error() override {
    int h = 0;
    FCGLE_CUDA(cudaStreamSynchronize(st_));
    FCGLE_CUDA(cudaMemcpy(&h, err_->ptr, sizeof(int), cudaMemcpyDeviceToHost));
    if (h) FCGLE_CUDA(cudaMemset(err_->ptr, 0, sizeof(int)));
    return h;
  }

  // raw mode product: flags bit 0 = forward (Q^T), bit 1 = split input and output
  void mode_product(int mu, bool fwd, const void* X, void* Y) override { mode_product_flags(mu, fwd ? 1 : 0, X, Y); }
  void mode_product_flags(int mu, int flags, const void* X, void* Y) override {
    if (mu < 0 || mu >= s_.d) throw InvalidArg("direction must be in 0..d-1");
    const bool fwd = flags & 1;
    if (flags & 4) {
      // the precise form of the end transforms: FP32 planar in and out
      if (flags & 2) throw InvalidArg("flags bits 1 and 2 exclude each other");
      const long long R = P_ / s_.p[mu];
      if (s_.d >= 2 && R % 8 == 0 && s_.p[mu] <= kTf32MaxP) {
        float *ah = F32(kFh), *al = F32(kD2);   // work tensors of the schemes, free here
        tf32_split_kernel<<<grid_for(P_ / 2), 256, 0, st_>>>(2 * P32(), (const float*)X, ah, al);
        FCGLE_LAUNCHED(launches);
        launch_tf32(ah, al, mu, fwd, (float*)Y, nullptr);
      } else {
        mp_f32((const float*)X, (float*)Y, mat_[mu][fwd ? 0 : 1].f32, s_.p[mu], (size_t)R, st_, launches);
      }
      return;
    }
    if (flags & 24) {
      // natural-order forms (split input and output)
      if (!(flags & 2)) throw InvalidArg("flags bits 3 and 4 need the split form (bit 1)");
      if ((flags & 24) == 24) throw InvalidArg("flags bits 3 and 4 exclude each other");
      const __nv_bfloat16* xh = (const __nv_bfloat16*)X;
      __nv_bfloat16* yh = (__nv_bfloat16*)Y;
      SplitOut in{const_cast<__nv_bfloat16*>(xh), const_cast<__nv_bfloat16*>(xh) + 2 * s_.P};
      SplitOut out{yh, yh + 2 * s_.P};
      if (flags & 8) {
        if (!slab_ok() || mu != 0) throw InvalidArg("the slab-fused product needs d == 3, p_2 <= 256, direction 0");
        launch_slab12(in, out, fwd);
      } else {
        if (s_.d < 2 || mu != s_.d - 1 || (P_ / s_.p[mu]) % 8 != 0)
          throw InvalidArg("the natural-order product needs d >= 2, direction d - 1 and R % 8 == 0");
        launch_mp_mn(in.hi, in.lo, fwd, b3::EpiStoreSplitGen{P32(), out});
      }
      return;
    }
    if (flags & 2) {
      const __nv_bfloat16* xh = (const __nv_bfloat16*)X;
      __nv_bfloat16* yh = (__nv_bfloat16*)Y;
      SplitOut out{yh, yh + 2 * s_.P};
      store_split(xh, xh + 2 * s_.P, mu, fwd, out);
    } else {
      SplitOut t = SP(kT0);
      to_split_kernel<<<grid_for(P_ / 2), 256, 0, st_>>>(2 * P32(), (const float*)X, t);
      FCGLE_LAUNCHED(launches);
      launch_mp(t.hi, t.lo, mu, fwd, b3::EpiStoreF32{P32(), (float*)Y});
    }
  }

  // ------------------------------------------------------------ apply_f
  void apply_f(int func, int k, double theta, const void* v, void* out) override {
    if (func == FCGLE_F_PHI && k == 0) func = FCGLE_F_EXP;
    float* X = F32(kWork);
    pack_f32((const float*)v, X);
    SplitOut V = SP(kV);
    gsplit(X, 0.0, 1.f, 0.f, V);
    if (func == FCGLE_F_EXP && kron()) {
      // Eq. Neudeckerd: d complex mode products instead of two Tucker operators
      exp_kron(V, theta, b3::EpiStoreF32{P32(), X});
      unpack_f32(X, (float*)out, true);
      return;
    }
    tucker(V, true, b3::EpiScaleF{P32(), lf_, fkind(func, k), (float)theta, V});
    tucker(V, false, b3::EpiStoreF32{P32(), X});
    unpack_f32(X, (float*)out, true);
  }

  // ---------------------------------------------------------- schemes
  void step(int scheme, double tau, double t, void* u) override {
    pack_f32((const float*)u, F32(kU));
    run(scheme, tau, 1, t);
    unpack_f32(F32(kU), (float*)u, true);
  }

  void integrate(int scheme, double tau, int nsteps, double t0, const void* u0, void* uT) override {
    pack_f32((const float*)u0, F32(kU));
    run(scheme, tau, nsteps, t0);
    unpack_f32(F32(kU), (float*)uT, true);
  }

  void integrate_host(int scheme, double tau, int nsteps, double t0, const void* u0, void* uT) override {
    const size_t bytes = s_.N * 8;
    if (!host_stage_) host_stage_.reset(new DevMem<float>(2 * s_.N));
    FCGLE_CUDA(cudaMemcpyAsync(host_stage_->ptr, u0, bytes, cudaMemcpyHostToDevice, st_));
    pack_f32(host_stage_->ptr, F32(kU));
    run(scheme, tau, nsteps, t0);
    unpack_f32(F32(kU), host_stage_->ptr, true);
    FCGLE_CUDA(cudaMemcpyAsync(uT, host_stage_->ptr, bytes, cudaMemcpyDeviceToHost, st_));
    FCGLE_CUDA(cudaStreamSynchronize(st_));
  }

  // ---- adjoint support (adjoint.h driver interface): generic FP32 planar Tucker operators
  Shape shape() const { return s_; }
  cudaStream_t stream() const { return st_; }
  long long& nlaunch() { return launches; }
  GParams gparams() const {
    GParams g;
    g.gamma = prm_.gamma;
    g.kappa = prm_.kappa;
    g.zeta = prm_.zeta;
    g.nsrc = gs_.nsrc;
    for (int k = 0; k < kMaxSrc; ++k) {
      g.sig_re[k] = sig_re_[k];
      g.sig_im[k] = sig_im_[k];
      g.S[k] = gs_.S[k];
    }
    return g;
  }
  LamVecs lamvecs() const {
    LamVecs lv;
    lv.c_re = prm_.nu;
    lv.c_im = prm_.eta;
    for (int mu = 0; mu < kMaxDim; ++mu) lv.lam[mu] = mu < s_.d ? lamd_[mu]->ptr : nullptr;
    return lv;
  }
  float* alloc(size_t n) {
    adj_mem_.emplace_back(new DevMem<float>(n));
    return adj_mem_.back()->ptr;
  }
  void release_all() { adj_mem_.clear(); }
  void tuckerT(const float* X, float* Y, bool fwd) {
    SplitOut V = SP(kV);
    to_split_kernel<<<grid_for(P_ / 2), 256, 0, st_>>>(2 * P32(), X, V);
    FCGLE_LAUNCHED(launches);
    tucker(V, fwd, b3::EpiStoreF32{P32(), Y});
  }
  void tuckerT_precise(const float* X, float* Y, bool fwd) { tucker_f32(X, Y, fwd, false); }
  // U = bwd(Uh) (FP32) and K = fwd(g(t, U)): g is evaluated in the epilogue of
  // the backward operator, which also writes it split for the forward one
  // (no standalone g pass, no split pass); tmp is not needed here
  void g_roundtrip(const float* Uh, float* U, float* K, float*, double t) {
    SplitOut V = SP(kV), G = SP(kW);
    to_split_kernel<<<grid_for(P_ / 2), 256, 0, st_>>>(2 * P32(), Uh, V);
    FCGLE_LAUNCHED(launches);
    tucker(V, false, b3::EpiUpdateG{P32(), U, 0, gs_, gtime(t), 0.f, 1.f, G});
    tucker(G, true, b3::EpiStoreF32{P32(), K});
  }

  void adjoint(int scheme, double tau, int nsteps, double t0, const void* u0, const void* target, int ckpt,
               void* grad_u0, double* grad_params, double* loss) override {
    if (scheme != FCGLE_LAWSON_RK2) throw Unsupported("the adjoint is implemented for LAWSON_RK2");
    try {
      float* U0 = alloc(2 * s_.P);
      float* TG = alloc(2 * s_.P);
      float* GR = alloc(2 * s_.P);
      pack_f32((const float*)u0, U0);
      pack_f32((const float*)target, TG);
      adjoint_lawson_rk2<float>(*this, tau, nsteps, t0, U0, TG, ckpt, GR, grad_params, loss);
      unpack_f32(GR, (float*)grad_u0, true);
      FCGLE_CUDA(cudaStreamSynchronize(st_));
    } catch (...) {
      release_all();
      throw;
    }
    release_all();
  }

  double norm(const void* u) override {
    float* X = F32(kWork);
    pack_f32((const float*)u, X);
    sumsq<float>(s_, X, scratch_->ptr, st_, launches);
    double h = 0.0;
    FCGLE_CUDA(cudaMemcpyAsync(&h, scratch_->ptr, sizeof(double), cudaMemcpyDeviceToHost, st_));
    FCGLE_CUDA(cudaStreamSynchronize(st_));
    double cell = 1.0;
    for (int mu = 0; mu < s_.d; ++mu) cell *= h_[mu];
    return std::sqrt(cell * h);
  }

 private:
  enum { kU = 0, kUh, kFh, kD2, kD3, kEA, kUp, kWork, kNumF32 };
  enum { kV = 0, kW, kT0, kT1, kNumSplit };

  struct Mat {
    __nv_bfloat16* hi = nullptr;
    __nv_bfloat16* lo = nullptr;
    float* f32 = nullptr;   // p x p FP32 (the CUDA-core form of the precise transforms, d == 1)
    // split-TF32 hi / lo (m_pad x k_pad32): the tensor-core form of the precise transforms
    float* thi = nullptr;
    float* tlo = nullptr;
    int p = 0, m_pad = 0, k_pad = 0, k_pad32 = 0;
    CUtensorMap tm_hi, tm_lo, tm_thi, tm_tlo;
    CUtensorMap tm_hi64, tm_lo64;   // the same hi / lo in 32-wide, 64-byte-swizzled boxes (slab-fused product)
  };

  float* F32(int i) { return f32_[i]->ptr; }
  uint32_t P32() const { return (uint32_t)s_.P; }
  SplitOut SP(int i) { return SplitOut{sp_[i]->ptr, sp_[i]->ptr + 2 * s_.P}; }

  template <class Epi>
  static void set_smem_attr() {
    FCGLE_CUDA(cudaFuncSetAttribute(b3::mp_b3_kernel<Epi, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)b3::Cfg<Epi>::kSmemBytes));
  }
  template <class Epi>
  static void set_smem_attr_mn() {
    FCGLE_CUDA(cudaFuncSetAttribute(b3::mp_b3_kernel<Epi, false, false, true>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b3::Cfg<Epi>::kSmemBytes));
  }
  template <class Epi>
  static void set_smem_attr_cx() {
    FCGLE_CUDA(cudaFuncSetAttribute(b3::mp_b3_kernel<Epi, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)b3::Cfg<Epi, true>::kSmemBytes));
  }

  // ---- Kronecker-product form of the exponential (Eq. Neudeckerd)
  // E_mu = exp(theta A_mu) = Q_mu diag(e^{theta (nu + i eta) lam}) Q_mu^T, complex
  // symmetric; as a mode-product operand the real and imaginary parts are
  // stacked, [Er; Ei] ((2 m_pad) x k_pad), and split into bf16 hi + lo.
  struct CMat {
    __nv_bfloat16* hi = nullptr;
    __nv_bfloat16* lo = nullptr;
    int m_pad = 0, k_pad = 0;
    CUtensorMap tm_hi, tm_lo;
    CMat() = default;
    CMat(const CMat&) = delete;
    CMat& operator=(const CMat&) = delete;
    ~CMat() {
      if (hi) cudaFree(hi);
      if (lo) cudaFree(lo);
    }
  };

  // E_mu for every direction at theta, built once (FP64 on the host) and cached
  // until the coefficients change
  const std::vector<std::unique_ptr<CMat>>& emat(double theta) {
    uint64_t key;
    std::memcpy(&key, &theta, 8);
    auto it = ecache_.find(key);
    if (it != ecache_.end()) return it->second;
    auto& v = ecache_[key];
    for (int mu = 0; mu < s_.d; ++mu) {
      const Direction& D = dir_[mu];
      const int n = D.n, p = s_.p[mu];
      std::vector<double> er(n), ei(n);
      for (int j = 0; j < n; ++j) {
        const double m = std::exp(theta * prm_.nu * D.lam[j]);
        er[j] = m * std::cos(theta * prm_.eta * D.lam[j]);
        ei[j] = m * std::sin(theta * prm_.eta * D.lam[j]);
      }
      std::unique_ptr<CMat> c(new CMat);
      c->m_pad = (p + b3::BM - 1) / b3::BM * b3::BM;
      c->k_pad = (p + b3::BK - 1) / b3::BK * b3::BK;
      const size_t rows = 2 * (size_t)c->m_pad, K = (size_t)c->k_pad;
      std::vector<__nv_bfloat16> hi(rows * K, __float2bfloat16(0.0f)), lo(hi);
      auto put = [&](size_t row, int k, double x) {
        const __nv_bfloat16 h = __float2bfloat16_rn((float)x);
        hi[row * K + k] = h;
        lo[row * K + k] = __float2bfloat16_rn((float)(x - (double)__bfloat162float(h)));
      };
      for (int i = 0; i < n; ++i)
        for (int k = 0; k <= i; ++k) {
          double sr = 0.0, si = 0.0;
          const double* qi = &D.Q[(size_t)i * n];
          const double* qk = &D.Q[(size_t)k * n];
          for (int j = 0; j < n; ++j) {
            const double w = qi[j] * qk[j];
            sr += w * er[j];
            si += w * ei[j];
          }
          put((size_t)i, k, sr);
          put((size_t)k, i, sr);
          put((size_t)c->m_pad + i, k, si);
          put((size_t)c->m_pad + k, i, si);
        }
      const size_t bytes = hi.size() * 2;
      FCGLE_CUDA(cudaMalloc(&c->hi, bytes));
      FCGLE_CUDA(cudaMalloc(&c->lo, bytes));
      FCGLE_CUDA(cudaMemcpy(c->hi, hi.data(), bytes, cudaMemcpyHostToDevice));
      FCGLE_CUDA(cudaMemcpy(c->lo, lo.data(), bytes, cudaMemcpyHostToDevice));
      encode_bf16(&c->tm_hi, c->hi, (uint64_t)c->k_pad, rows, b3::BM);
      encode_bf16(&c->tm_lo, c->lo, (uint64_t)c->k_pad, rows, b3::BM);
      v.push_back(std::move(c));
    }
    return v;
  }

  b3::KParams kparams_cx(int mu, const CMat& c) const {
    b3::KParams kp;
    kp.R = P_ / s_.p[mu];
    kp.p = s_.p[mu];
    kp.m_blocks = c.m_pad / b3::BM;
    kp.k_chunks = c.k_pad / b3::BK;
    kp.tiles = (kp.R + b3::BR - 1) / b3::BR;
    kp.err = err_->ptr;
    kp.ei_row = c.m_pad;
    return kp;
  }

  // one complex mode product with epilogue (fused kernel, complex form)
  template <class Epi>
  void launch_mp_cx(const __nv_bfloat16* xh, const __nv_bfloat16* xl, int mu, const CMat& c, const Epi& epi) {
    const b3::KParams kp = kparams_cx(mu, c);
    CUtensorMap txh, txl;
    encode_bf16(&txh, xh, (uint64_t)s_.p[mu], 2 * (uint64_t)kp.R, b3::BR);
    encode_bf16(&txl, xl, (uint64_t)s_.p[mu], 2 * (uint64_t)kp.R, b3::BR);
    const long long units = kp.tiles * kp.m_blocks;
    const int grid = (int)std::min<long long>(units, num_sms());
    launch_pdl(b3::mp_b3_kernel<Epi, false, true>, grid, b3::Cfg<Epi, true>::kThreads,
               b3::Cfg<Epi, true>::kSmemBytes, st_, txh, txl, c.tm_hi, c.tm_lo, kp, epi,
               (const b3::FusedDesc<Epi>*)nullptr, 0, 0LL);
    FCGLE_LAUNCHED(launches);
  }

  // one complex mode product with a split output
  void store_split_cx(const __nv_bfloat16* xh, const __nv_bfloat16* xl, int mu, const CMat& c, SplitOut out) {
    const b3::KParams kp = kparams_cx(mu, c);
    if (kp.R % 8 != 0) {
      launch_mp_cx(xh, xl, mu, c, b3::EpiStoreSplitGen{P32(), out});
      return;
    }
    CUtensorMap txh, txl, tyh, tyl;
    encode_bf16(&txh, xh, (uint64_t)s_.p[mu], 2 * (uint64_t)kp.R, b3::BR);
    encode_bf16(&txl, xl, (uint64_t)s_.p[mu], 2 * (uint64_t)kp.R, b3::BR);
    encode_bf16_out(&tyh, out.hi, (uint64_t)kp.R, (uint64_t)s_.p[mu]);
    encode_bf16_out(&tyl, out.lo, (uint64_t)kp.R, (uint64_t)s_.p[mu]);
    const long long units = kp.tiles * kp.m_blocks;
    const int grid = (int)std::min<long long>(units, num_sms());
    launch_pdl(b3::mp_b3_plain_kernel<false, b3::kOpBF16, 2, false, true>, grid, b3::PL_THREADS, b3::kPlSmemBytes,
               st_, txh, txl, c.tm_hi, c.tm_lo, tyh, tyl, kp, (const b3::PlainDesc*)nullptr, 0, 0LL);
    FCGLE_LAUNCHED(launches);
  }

  // e^{theta K} applied to the split tensor `in` (consumed) as V x_1 E_1 ... x_d E_d;
  // the last product runs `epi` (which may write into `in` for d >= 2)
  template <class Epi>
  void exp_kron(SplitOut in, double theta, const Epi& epi) {
    const auto& E = emat(theta);
    const int d = s_.d;
    SplitOut src = in;
    if (d == 1) {
      SplitOut t = SP(kT1);
      FCGLE_CUDA(cudaMemcpyAsync(t.hi, in.hi, 4 * s_.P * 2, cudaMemcpyDeviceToDevice, st_));
      src = t;
    }
    for (int mu = 0; mu < d - 1; ++mu) {
      SplitOut dst = SP(mu % 2 == 0 ? kT0 : kT1);
      store_split_cx(src.hi, src.lo, mu, *E[mu], dst);
      src = dst;
    }
    launch_mp_cx(src.hi, src.lo, d - 1, *E[d - 1], epi);
  }

  bool kron() const { return exp_form_ == FCGLE_EXP_KRON; }
  // schemes whose only operator is e^{tau K}, run in the Kronecker-product form when chosen
  bool kron_scheme(int scheme) const {
    return kron() && (scheme == FCGLE_LAWSON_EULER || scheme == FCGLE_LAWSON_RK2 || scheme == FCGLE_STRANG);
  }

  void prepare_matrix(const double* M, int p, Mat& m) {
    m.p = p;
    m.m_pad = (p + b3::BM - 1) / b3::BM * b3::BM;
    m.k_pad = (p + b3::BK - 1) / b3::BK * b3::BK;
    std::vector<__nv_bfloat16> hi((size_t)m.m_pad * m.k_pad, __float2bfloat16(0.0f)), lo(hi);
    for (int i = 0; i < p; ++i)
      for (int k = 0; k < p; ++k) {
        const double x = M[(size_t)i * p + k];
        const __nv_bfloat16 h = __float2bfloat16_rn((float)x);
        hi[(size_t)i * m.k_pad + k] = h;
        lo[(size_t)i * m.k_pad + k] = __float2bfloat16_rn((float)(x - (double)__bfloat162float(h)));
      }
    const size_t bytes = hi.size() * 2;
    FCGLE_CUDA(cudaMalloc(&m.hi, bytes));
    FCGLE_CUDA(cudaMalloc(&m.lo, bytes));
    FCGLE_CUDA(cudaMemcpy(m.hi, hi.data(), bytes, cudaMemcpyHostToDevice));
    FCGLE_CUDA(cudaMemcpy(m.lo, lo.data(), bytes, cudaMemcpyHostToDevice));
    encode_bf16(&m.tm_hi, m.hi, m.k_pad, m.m_pad, b3::BM);
    encode_bf16(&m.tm_lo, m.lo, m.k_pad, m.m_pad, b3::BM);
    encode_bf16_sw64(&m.tm_hi64, m.hi, m.k_pad, m.m_pad, b3::BM);
    encode_bf16_sw64(&m.tm_lo64, m.lo, m.k_pad, m.m_pad, b3::BM);
    std::vector<float> f((size_t)p * p);
    for (size_t e = 0; e < f.size(); ++e) f[e] = (float)M[e];
    FCGLE_CUDA(cudaMalloc(&m.f32, f.size() * 4));
    FCGLE_CUDA(cudaMemcpy(m.f32, f.data(), f.size() * 4, cudaMemcpyHostToDevice));
    // split-TF32: hi = tf32(M), lo = tf32(M - hi), zero padded to (m_pad, k_pad32)
    m.k_pad32 = (p + 31) / 32 * 32;
    std::vector<float> th((size_t)m.m_pad * m.k_pad32, 0.0f), tl(th);
    for (int i = 0; i < p; ++i)
      for (int k = 0; k < p; ++k) {
        const double x = M[(size_t)i * p + k];
        const float h = tf32_rna_host((float)x);
        th[(size_t)i * m.k_pad32 + k] = h;
        tl[(size_t)i * m.k_pad32 + k] = tf32_rna_host((float)(x - (double)h));
      }
    FCGLE_CUDA(cudaMalloc(&m.thi, th.size() * 4));
    FCGLE_CUDA(cudaMalloc(&m.tlo, tl.size() * 4));
    FCGLE_CUDA(cudaMemcpy(m.thi, th.data(), th.size() * 4, cudaMemcpyHostToDevice));
    FCGLE_CUDA(cudaMemcpy(m.tlo, tl.data(), tl.size() * 4, cudaMemcpyHostToDevice));
    encode_f32(&m.tm_thi, m.thi, m.k_pad32, m.m_pad, b3::BM);
    encode_f32(&m.tm_tlo, m.tlo, m.k_pad32, m.m_pad, b3::BM);
  }

  // Precise Tucker operator (X, Y planar FP32, distinct), used where the
  // split-BF16 error must not enter: U^_0 = fwd(u_0) at the start of a time
  // integration and u(T) = bwd(U^_T) at its end.  Split-TF32 on the tensor
  // cores (about 2^-21 relative per product) when every output row pitch
  // allows the FP32 TMA boxes (d >= 2, R % 8 == 0) and every contraction is at
  // most kTf32MaxP long: the tensor core's FP32 accumulation of the three
  // products adds an error that grows with the contracted length (measured
  // 2.4e-6 at p = 264; at p = 1024 it lifted the error at T of 500 steps from
  // 1.6e-6 to 8.5e-6).  FP32 on the CUDA cores otherwise, and always when
  // tc_ok is false (the adjoint, whose misfit compares nearby states).
  static constexpr int kTf32MaxP = 256;
  void tucker_f32(const float* X, float* Y, bool fwd, bool tc_ok = true) {
    bool tc = tc_ok && s_.d >= 2;
    for (int mu = 0; mu < s_.d && tc; ++mu) tc = (P_ / s_.p[mu]) % 8 == 0 && s_.p[mu] <= kTf32MaxP;
    if (tc) {
      tucker_tf32(X, Y, fwd);
      return;
    }
    tucker_simt(X, Y, fwd);
  }

  // The split-TF32 intermediates (hi and lo, 2 P floats each) live in four of
  // the schemes' FP32 work tensors, which hold nothing at the two ends of a
  // time integration where this runs (X and Y are the state tensors U, U^ or
  // the Strang work tensor, never these four).
  void tucker_tf32(const float* X, float* Y, bool fwd) {
    float* const hi[2] = {F32(kFh), F32(kD3)};
    float* const lo[2] = {F32(kD2), F32(kEA)};
    tf32_split_kernel<<<grid_for(P_ / 2), 256, 0, st_>>>(2 * P32(), X, hi[0], lo[0]);
    FCGLE_LAUNCHED(launches);
    int cur = 0;
    for (int mu = 0; mu < s_.d; ++mu) {
      const bool last = mu == s_.d - 1;
      launch_tf32(hi[cur], lo[cur], mu, fwd, last ? Y : hi[cur ^ 1], last ? nullptr : lo[cur ^ 1]);
      cur ^= 1;
    }
  }

  // one split-TF32 mode product; ylo == nullptr: plain FP32 output into yhi
  void launch_tf32(const float* xh, const float* xl, int mu, bool fwd, float* yhi, float* ylo) {
    const Mat& m = mat_[mu][fwd ? 0 : 1];
    const long long R = P_ / s_.p[mu];
    CUtensorMap txh, txl, tyh, tyl;
    encode_f32(&txh, xh, (uint64_t)s_.p[mu], 2 * (uint64_t)R, b3::BR);
    encode_f32(&txl, xl, (uint64_t)s_.p[mu], 2 * (uint64_t)R, b3::BR);
    encode_f32_out(&tyh, yhi, (uint64_t)R, (uint64_t)s_.p[mu]);
    encode_f32_out(&tyl, ylo ? ylo : yhi, (uint64_t)R, (uint64_t)s_.p[mu]);
    b3::KParams kp;
    kp.R = R;
    kp.p = s_.p[mu];
    kp.m_blocks = m.m_pad / b3::BM;
    kp.k_chunks = m.k_pad32 / 32;
    kp.tiles = (R + b3::BR - 1) / b3::BR;
    kp.err = err_->ptr;
    const long long units = kp.tiles * kp.m_blocks;
    const int grid = (int)std::min<long long>(units, num_sms());
    if (ylo)
      launch_pdl(b3::mp_b3_plain_kernel<false, b3::kOpTF32>, grid, b3::PL_THREADS, b3::kPlSmemBytes, st_, txh, txl,
                 m.tm_thi, m.tm_tlo, tyh, tyl, kp, (const b3::PlainDesc*)nullptr, 0, 0LL);
    else
      launch_pdl(b3::mp_b3_plain_kernel<false, b3::kOpTF32F>, grid, b3::PL_THREADS, b3::kPlSmemBytes, st_, txh, txl,
                 m.tm_thi, m.tm_tlo, tyh, tyl, kp, (const b3::PlainDesc*)nullptr, 0, 0LL);
    FCGLE_LAUNCHED(launches);
  }

  void tucker_simt(const float* X, float* Y, bool fwd) {
    float* tmp[2] = {F32(kFh), F32(kD2)};
    const float* src = X;
    for (int mu = 0; mu < s_.d; ++mu) {
      float* dst = mu == s_.d - 1 ? Y : tmp[mu % 2];
      mp_f32(src, dst, mat_[mu][fwd ? 0 : 1].f32, s_.p[mu], (size_t)(P_ / s_.p[mu]), st_, launches);
      src = dst;
    }
  }

  // mode product with a split output: TMA stores when the output rows allow
  void store_split(const __nv_bfloat16* xh, const __nv_bfloat16* xl, int mu, bool fwd, SplitOut out) {
    const long long R = P_ / s_.p[mu];
    if (R % 8 == 0)
      launch_plain(xh, xl, mu, fwd, out);
    else
      launch_mp(xh, xl, mu, fwd, b3::EpiStoreSplitGen{P32(), out});
  }

  // plain mode product with split output (R % 8 == 0): separate operand rings
  void launch_plain(const __nv_bfloat16* xh, const __nv_bfloat16* xl, int mu, bool fwd, SplitOut out) {
    const Mat& m = mat_[mu][fwd ? 0 : 1];
    const long long R = P_ / s_.p[mu];
    if (R % 8 != 0) throw std::runtime_error("plain mode product needs R % 8 == 0");
    CUtensorMap txh, txl;
    encode_bf16(&txh, xh, (uint64_t)s_.p[mu], 2 * (uint64_t)R, b3::BR);
    encode_bf16(&txl, xl, (uint64_t)s_.p[mu], 2 * (uint64_t)R, b3::BR);
    b3::KParams kp;
    kp.R = R;
    kp.p = s_.p[mu];
    kp.m_blocks = m.m_pad / b3::BM;
    kp.k_chunks = m.k_pad / b3::BK;
    kp.tiles = (R + b3::BR - 1) / b3::BR;
    kp.err = err_->ptr;
    const long long units = kp.tiles * kp.m_blocks;
    const int grid = (int)std::min<long long>(units, num_sms());
    CUtensorMap tyh, tyl;
    encode_bf16_out(&tyh, out.hi, (uint64_t)R, (uint64_t)s_.p[mu]);
    encode_bf16_out(&tyl, out.lo, (uint64_t)R, (uint64_t)s_.p[mu]);
    if (rec_) {
      b3::PlainDesc d;
      std::memset(&d, 0, sizeof(d));
      d.xhi = txh;
      d.xlo = txl;
      d.mhi = m.tm_hi;
      d.mlo = m.tm_lo;
      d.yhi = tyh;
      d.ylo = tyl;
      d.kp = kp;
      record(false, &launch_plain_grouped<b3::PL_NX>, offsetof(b3::PlainDesc, ubegin), &d, sizeof(d), units);
      rec_->back().alts = {&launch_plain_grouped<3>, &launch_plain_grouped<2>};
      rec_->back().alt_names = {kPlainCfgName[kCfgX3M3], kPlainCfgName[kCfgX2M4]};
      return;
    }
    int cfg = forced_plain_cfg();
    if (cfg < 0 || !plain_cfg_ok(cfg, kp, units)) {
      TuneEntry e;
      cfg = tuned_lookup(kp.p, R, e) ? e.cfg : default_plain_cfg(kp, units);
    }
    launch_plain_cfg(cfg, xh, xl, txh, txl, m, tyh, tyl, kp, units);
  }

  // resident M: every CTA keeps one fixed i-block (grid a multiple of m_blocks)
  // and the block of M fits the 4 x 32 KB resident region
  static int grid_mr(long long units, int m_blocks) {
    const int sms = num_sms();
    return units < sms ? (int)units : sms - sms % m_blocks;
  }
  static bool plain_cfg_ok(int cfg, const b3::KParams& kp, long long units) {
    if (cfg != kCfgMR && cfg != kCfgMH) return true;
    return kp.k_chunks <= b3::kMRMaxChunks && grid_mr(units, kp.m_blocks) >= kp.m_blocks;
  }
  static int default_plain_cfg(const b3::KParams&, long long) { return kCfgX4M2; }
  // txh, txl: X maps with 64-row boxes (xh, xl: the same tensors, for the
  // 128-row boxes of the wide configuration); kp, units: 64-r tiles
  void launch_plain_cfg(int cfg, const __nv_bfloat16* xh, const __nv_bfloat16* xl, const CUtensorMap& txh,
                        const CUtensorMap& txl, const Mat& m, const CUtensorMap& tyh, const CUtensorMap& tyl,
                        const b3::KParams& kp, long long units) {
    if (cfg == kCfgWide) {
      CUtensorMap wxh, wxl;
      encode_bf16(&wxh, xh, (uint64_t)kp.p, 2 * (uint64_t)kp.R, 2 * b3::BR);
      encode_bf16(&wxl, xl, (uint64_t)kp.p, 2 * (uint64_t)kp.R, 2 * b3::BR);
      b3::KParams kw = kp;
      kw.tiles = (kp.R + 2 * b3::BR - 1) / (2 * b3::BR);
      const long long wunits = kw.tiles * kw.m_blocks;
      launch_pdl(plain_kernel(cfg), (int)std::min<long long>(wunits, num_sms()), b3::PL_THREADS, b3::kPlSmemBytes,
                 st_, wxh, wxl, m.tm_hi, m.tm_lo, tyh, tyl, kw, (const b3::PlainDesc*)nullptr, 0, 0LL);
      FCGLE_LAUNCHED(launches);
      return;
    }
    const int grid = (cfg == kCfgMR || cfg == kCfgMH) ? grid_mr(units, kp.m_blocks)
                                                       : (int)std::min<long long>(units, num_sms());
    launch_pdl(plain_kernel(cfg), grid, b3::PL_THREADS, b3::kPlSmemBytes, st_, txh, txl, m.tm_hi, m.tm_lo, tyh, tyl,
               kp, (const b3::PlainDesc*)nullptr, 0, 0LL);
    FCGLE_LAUNCHED(launches);
  }

 public:
  // Times every eligible ring configuration of the plain product for each
  // direction this handle runs it on (directions 0 .. d-2; the last direction
  // carries the fused epilogues) whose (p, R) the process has not tuned yet,
  // on the handle's work buffers, and records the fastest.  Synchronous.
  void autotune() override {
    tune_plain();
    tune_slab();
  }

  // 3D handles: times one forward Tucker operator (split output) in the
  // rotating form and in the slab-fused form, once per process per shape,
  // and keeps the slab-fused form where it is clearly faster.
  void tune_slab() {
    if (!slab_ok() || tucker_form_ != FCGLE_TUCKER_AUTO) return;
    const auto key = std::make_tuple(s_.p[0], s_.p[1], s_.p[2]);
    {
      std::lock_guard<std::mutex> lk(g_tune_mu);
      if (g_slab.count(key)) return;
    }
    SlabTune e;
    const int keep = tucker_form_;
    const b3::EpiStoreSplitGen ep{P32(), SP(kW)};
    cudaEvent_t e0, e1;
    FCGLE_CUDA(cudaEventCreate(&e0));
    FCGLE_CUDA(cudaEventCreate(&e1));
    try {
      constexpr int kReps = 5;
      for (int form : {FCGLE_TUCKER_ROTATING, FCGLE_TUCKER_SLAB}) {
        tucker_form_ = form;
        tucker(SP(kV), true, ep);   // warm-up
        FCGLE_CUDA(cudaEventRecord(e0, st_));
        for (int r = 0; r < kReps; ++r) tucker(SP(kV), true, ep);
        FCGLE_CUDA(cudaEventRecord(e1, st_));
        FCGLE_CUDA(cudaEventSynchronize(e1));
        float ms = 0.f;
        FCGLE_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        (form == FCGLE_TUCKER_SLAB ? e.us_slab : e.us_rot) = 1e3f * ms / kReps;
      }
    } catch (...) {
      tucker_form_ = keep;
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      throw;
    }
    tucker_form_ = keep;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    e.slab = e.us_slab < 0.98f * e.us_rot;
    if (device_error()) throw DeviceTimeout("a bounded device-side wait gave up while tuning the Tucker operator");
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_slab.emplace(key, e);
  }

  void tune_plain() {
    if (forced_plain_cfg() >= 0) return;
    for (int mu = 0; mu + 1 < s_.d; ++mu) {
      const long long R = P_ / s_.p[mu];
      if (R % 8 != 0) continue;
      TuneEntry have;
      if (tuned_lookup(s_.p[mu], R, have)) continue;
      const Mat& m = mat_[mu][0];
      SplitOut in = SP(kT0), out = SP(kT1);
      CUtensorMap txh, txl, tyh, tyl;
      encode_bf16(&txh, in.hi, (uint64_t)s_.p[mu], 2 * (uint64_t)R, b3::BR);
      encode_bf16(&txl, in.lo, (uint64_t)s_.p[mu], 2 * (uint64_t)R, b3::BR);
      encode_bf16_out(&tyh, out.hi, (uint64_t)R, (uint64_t)s_.p[mu]);
      encode_bf16_out(&tyl, out.lo, (uint64_t)R, (uint64_t)s_.p[mu]);
      b3::KParams kp;
      kp.R = R;
      kp.p = s_.p[mu];
      kp.m_blocks = m.m_pad / b3::BM;
      kp.k_chunks = m.k_pad / b3::BK;
      kp.tiles = (R + b3::BR - 1) / b3::BR;
      kp.err = err_->ptr;
      const long long units = kp.tiles * kp.m_blocks;
      TuneEntry e;
      float best = 0.f;
      cudaEvent_t e0, e1;
      FCGLE_CUDA(cudaEventCreate(&e0));
      FCGLE_CUDA(cudaEventCreate(&e1));
      try {
        constexpr int kReps = 5;
        for (int c = 0; c < kNumPlainCfg; ++c) {
          if (!plain_cfg_ok(c, kp, units)) continue;
          launch_plain_cfg(c, in.hi, in.lo, txh, txl, m, tyh, tyl, kp, units);   // warm-up
          FCGLE_CUDA(cudaEventRecord(e0, st_));
          for (int r = 0; r < kReps; ++r) launch_plain_cfg(c, in.hi, in.lo, txh, txl, m, tyh, tyl, kp, units);
          FCGLE_CUDA(cudaEventRecord(e1, st_));
          FCGLE_CUDA(cudaEventSynchronize(e1));
          float ms = 0.f;
          FCGLE_CUDA(cudaEventElapsedTime(&ms, e0, e1));
          e.us[c] = 1e3f * ms / kReps;
          if (best == 0.f || e.us[c] < best) {
            best = e.us[c];
            e.cfg = c;
          }
        }
      } catch (...) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        throw;
      }
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      // another configuration replaces the default only when it is clearly faster
      if (e.cfg != kCfgX4M2 && e.us[kCfgX4M2] > 0.f && e.us[e.cfg] > 0.98f * e.us[kCfgX4M2]) e.cfg = kCfgX4M2;
      if (device_error()) throw DeviceTimeout("a bounded device-side wait gave up while tuning the mode product");
      std::lock_guard<std::mutex> lk(g_tune_mu);
      g_tune.emplace(std::make_tuple(s_.p[mu], R), e);
    }
  }

 private:

  // ---- grouped launches (batches): recording and the launchers
  void record(bool last, void (*fn)(const void*, int, long long, cudaStream_t), size_t uoff, const void* d,
              size_t bytes, long long units) {
    GroupRec r;
    r.last = last;
    r.launch = fn;
    r.ubegin_off = uoff;
    r.desc.assign((const uint8_t*)d, (const uint8_t*)d + bytes);
    r.units = units;
    rec_->push_back(std::move(r));
  }
  template <int NXR>
  static void launch_plain_grouped(const void* descs, int n, long long units, cudaStream_t st) {
    static std::once_flag attr;
    std::call_once(attr, [] {
      FCGLE_CUDA(cudaFuncSetAttribute(b3::mp_b3_plain_kernel<true, b3::kOpBF16, NXR>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b3::kPlSmemBytes));
    });
    CUtensorMap z;
    std::memset(&z, 0, sizeof(z));
    b3::KParams kp{};
    const int grid = (int)std::min<long long>(units, num_sms());
    launch_pdl(b3::mp_b3_plain_kernel<true, b3::kOpBF16, NXR>, grid, b3::PL_THREADS, b3::kPlSmemBytes, st, z, z, z, z,
               z, z, kp, static_cast<const b3::PlainDesc*>(descs), n, units);
  }
  template <class Epi>
  static void launch_fused_grouped(const void* descs, int n, long long units, cudaStream_t st) {
    static std::once_flag attr;
    std::call_once(attr, [] {
      FCGLE_CUDA(cudaFuncSetAttribute(b3::mp_b3_kernel<Epi, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)b3::Cfg<Epi>::kSmemBytes));
    });
    CUtensorMap z;
    std::memset(&z, 0, sizeof(z));
    b3::KParams kp{};
    const int grid = (int)std::min<long long>(units, num_sms());
    launch_pdl(b3::mp_b3_kernel<Epi, true>, grid, b3::Cfg<Epi>::kThreads, b3::Cfg<Epi>::kSmemBytes, st, z, z, z, z,
               kp, Epi{}, static_cast<const b3::FusedDesc<Epi>*>(descs), n, units);
  }

  // one mode product of direction mu on split input (xh, xl) with epilogue epi
  template <class Epi>
  void launch_mp(const __nv_bfloat16* xh, const __nv_bfloat16* xl, int mu, bool fwd, const Epi& epi) {
    const Mat& m = mat_[mu][fwd ? 0 : 1];
    const long long R = P_ / s_.p[mu];
    CUtensorMap txh, txl;
    encode_bf16(&txh, xh, (uint64_t)s_.p[mu], 2 * (uint64_t)R, b3::BR);
    encode_bf16(&txl, xl, (uint64_t)s_.p[mu], 2 * (uint64_t)R, b3::BR);
    b3::KParams kp;
    kp.R = R;
    kp.p = s_.p[mu];
    kp.m_blocks = m.m_pad / b3::BM;
    kp.k_chunks = m.k_pad / b3::BK;
    kp.tiles = (R + b3::BR - 1) / b3::BR;
    kp.err = err_->ptr;
    const long long units = kp.tiles * kp.m_blocks;
    const int grid = (int)std::min<long long>(units, num_sms());
    if (rec_) {
      b3::FusedDesc<Epi> d;
      std::memset(static_cast<void*>(&d), 0, sizeof(d));
      d.xhi = txh;
      d.xlo = txl;
      d.mhi = m.tm_hi;
      d.mlo = m.tm_lo;
      d.kp = kp;
      d.epi = epi;
      record(last_mp_, &launch_fused_grouped<Epi>, offsetof(b3::FusedDesc<Epi>, ubegin), &d, sizeof(d), units);
      return;
    }
    launch_pdl(b3::mp_b3_kernel<Epi, false>, grid, b3::Cfg<Epi>::kThreads, b3::Cfg<Epi>::kSmemBytes, st_, txh, txl,
               m.tm_hi, m.tm_lo, kp, epi, (const b3::FusedDesc<Epi>*)nullptr, 0, 0LL);
    FCGLE_LAUNCHED(launches);
  }

  // ---- slab-fused modes 1 + 2 and the natural-order mode-3 product (d == 3)
  bool slab_ok() const { return s_.d == 3 && s_.p[1] <= 256; }
  bool use_slab() const {
    if (!slab_ok() || rec_ || tucker_form_ == FCGLE_TUCKER_ROTATING) return false;
    if (tucker_form_ == FCGLE_TUCKER_SLAB) return true;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_slab.find(std::make_tuple(s_.p[0], s_.p[1], s_.p[2]));
    return it != g_slab.end() && it->second.slab;
  }

  // Y[c][j3][i2][i1] = sum M2[i2][j2] M1[i1][j1] X[c][j3][j2][j1] (in, out split, natural order, distinct)
  void launch_slab12(SplitOut in, SplitOut out, bool fwd) {
    const int p1 = s_.p[0], p2 = s_.p[1], p3 = s_.p[2];
    const Mat& m1 = mat_[0][fwd ? 0 : 1];
    const Mat& m2 = mat_[1][fwd ? 0 : 1];
    b3::SlabParams sp;
    sp.p1 = p1;
    sp.p2 = p2;
    sp.p3 = p3;
    sp.n2 = (p2 + 15) / 16 * 16;
    sp.mb1 = m1.m_pad / b3::BM;
    sp.kc1 = (p1 + b3::SL_K - 1) / b3::SL_K;
    sp.kc2 = (sp.n2 + b3::SL_K - 1) / b3::SL_K;
    sp.err = err_->ptr;
    CUtensorMap txh, txl, tyh, tyl;
    encode_bf16_3d(&txh, in.hi, (uint64_t)p1, (uint64_t)p2, 2 * (uint64_t)p3, b3::SL_K, (uint32_t)sp.n2, 64);
    encode_bf16_3d(&txl, in.lo, (uint64_t)p1, (uint64_t)p2, 2 * (uint64_t)p3, b3::SL_K, (uint32_t)sp.n2, 64);
    encode_bf16_3d(&tyh, out.hi, (uint64_t)p1, (uint64_t)p2, 2 * (uint64_t)p3, 32, 32, 0);
    encode_bf16_3d(&tyl, out.lo, (uint64_t)p1, (uint64_t)p2, 2 * (uint64_t)p3, 32, 32, 0);
    const long long units = (long long)p3 * sp.mb1;
    const int grid = (int)std::min<long long>(units, num_sms());
    launch_pdl(b3::mp_b3_slab12_kernel, grid, b3::SL_THREADS, b3::kSlSmemBytes, st_, txh, txl, m1.tm_hi64,
               m1.tm_lo64, m2.tm_hi64, m2.tm_lo64, tyh, tyl, sp);
    FCGLE_LAUNCHED(launches);
  }

  // the last mode product (direction d - 1) on a natural-order input X[c][k][r]
  template <class Epi>
  void launch_mp_mn(const __nv_bfloat16* xh, const __nv_bfloat16* xl, bool fwd, const Epi& epi) {
    const int mu = s_.d - 1;
    const Mat& m = mat_[mu][fwd ? 0 : 1];
    const long long R = P_ / s_.p[mu];
    CUtensorMap txh, txl;
    encode_bf16_3d(&txh, xh, (uint64_t)R, (uint64_t)s_.p[mu], 2, b3::BR, b3::BK, 128);
    encode_bf16_3d(&txl, xl, (uint64_t)R, (uint64_t)s_.p[mu], 2, b3::BR, b3::BK, 128);
    b3::KParams kp;
    kp.R = R;
    kp.p = s_.p[mu];
    kp.m_blocks = m.m_pad / b3::BM;
    kp.k_chunks = m.k_pad / b3::BK;
    kp.tiles = (R + b3::BR - 1) / b3::BR;
    kp.err = err_->ptr;
    const long long units = kp.tiles * kp.m_blocks;
    const int grid = (int)std::min<long long>(units, num_sms());
    launch_pdl(b3::mp_b3_kernel<Epi, false, false, true>, grid, b3::Cfg<Epi>::kThreads, b3::Cfg<Epi>::kSmemBytes, st_,
               txh, txl, m.tm_hi, m.tm_lo, kp, epi, (const b3::FusedDesc<Epi>*)nullptr, 0, 0LL);
    FCGLE_LAUNCHED(launches);
  }

  // Tucker operator on the split tensor `in` (consumed); the last mode product
  // runs `epi`, which may write into `in` (d >= 2: `in` is only read by the
  // first mode product; d == 1: `in` is first copied aside).
  template <class Epi>
  void tucker(SplitOut in, bool fwd, const Epi& epi) {
    const int d = s_.d;
    if (use_slab()) {
      // modes 1 + 2 per j_3 slab, then the mode-3 product on the natural order
      SplitOut t = SP(kT0);
      launch_slab12(in, t, fwd);
      last_mp_ = true;
      launch_mp_mn(t.hi, t.lo, fwd, epi);
      last_mp_ = false;
      return;
    }
    SplitOut src = in;
    if (d == 1) {
      SplitOut t = SP(kT1);
      FCGLE_CUDA(cudaMemcpyAsync(t.hi, in.hi, 4 * s_.P * 2, cudaMemcpyDeviceToDevice, st_));
      src = t;
    }
    for (int mu = 0; mu < d - 1; ++mu) {
      SplitOut dst = SP(mu % 2 == 0 ? kT0 : kT1);
      store_split(src.hi, src.lo, mu, fwd, dst);
      src = dst;
    }
    last_mp_ = true;
    launch_mp(src.hi, src.lo, d - 1, fwd, epi);
    last_mp_ = false;
  }

  void pack_f32(const float* user, float* U) { pack<float>(s_, user, U, st_, launches); }
  // check = true: a NaN or Inf among the values is recorded in the device error word
  void unpack_f32(const float* U, float* user, bool check = false) {
    unpack<float>(s_, U, user, st_, launches, check ? err_->ptr : nullptr);
  }

  b3::GTime gtime(double t) const {
    b3::GTime g;
    for (int k = 0; k < gs_.nsrc; ++k) {
      const double m = std::exp(sig_re_[k] * t);
      g.e_re[k] = (float)(m * std::cos(sig_im_[k] * t));
      g.e_im[k] = (float)(m * std::sin(sig_im_[k] * t));
    }
    return g;
  }

  // V = a u + b g(t, u) (+ optional V2)
  void gsplit(const float* U, double t, float a, float b, SplitOut V, float a2 = 0.f, float b2 = 0.f,
              SplitOut V2 = SplitOut{}) {
    gsplit_kernel<<<grid_for(P_ / 4), 256, 0, st_>>>(P32(), gs_, gtime(t), U, a, b, V, a2, b2, V2);
    FCGLE_LAUNCHED(launches);
  }

  b3::Flow flow(double t) const {
    const double z = 2.0 * prm_.gamma * t;
    const double p1 = std::fabs(z) < 1e-8 ? 1.0 + z / 2.0 : std::expm1(z) / z;
    b3::Flow f;
    f.gamma_t = (float)(t * prm_.gamma);
    f.c2 = (float)(2.0 * t * p1 * prm_.kappa);
    f.zk = (float)(prm_.zeta / (2.0 * prm_.kappa));
    return f;
  }

  // coefficients of the phi_3 series along z = theta (nu + i eta) s, s real (b3::phi123_s)
  b3::PhiPoly phipoly(double theta) const {
    b3::PhiPoly P;
    const std::complex<double> w(theta * prm_.nu, theta * prm_.eta);
    std::complex<double> wm(1.0, 0.0);
    double fact = 6.0;   // (m + 3)! at m = 0
    for (int m = 0; m < 10; ++m) {
      const std::complex<double> c = wm / fact;
      P.cr[m] = (float)c.real();
      P.ci[m] = (float)c.imag();
      wm *= w;
      fact *= (double)(m + 4);
    }
    const double aw = std::abs(w);
    P.smax = aw > 0.0 ? (float)(1.0 / aw) : 3.0e38f;
    P.wr = (float)w.real();
    P.wi = (float)w.imag();
    return P;
  }

  // spectral scalar f(theta lam), evaluated on the fly by the epilogues (b3 fspec kinds)
  static int fkind(int func, int k) {
    if (func == FCGLE_F_INV) return 0;
    if (func == FCGLE_F_EXP || k == 0) return 1;
    return 1 + k;
  }

  // prologue (entry state of the loop), then nsteps fused steps on F32(kU)
  // ---- time loop, split into a prologue and per-step bodies (batched graphs replay a step)
  void run(int scheme, double tau, int nsteps, double t0) {
    if (scheme < FCGLE_LIE || scheme > FCGLE_STRANG) throw InvalidArg("unknown scheme");
    if (nsteps == 0) return;
    begin(scheme, tau, t0);
    for (int n = 0; n < nsteps; ++n) step(n);
    finish();
  }

  // u(T) from the carried spectral state by the FP32 backward operator (Strang:
  // u(T) = Phi_{tau/2}(bwd(e^))), replacing the split-BF16 one of the last step
  void finish() {
    if (kron_scheme(rs_scheme_)) return;   // the physical state is already in F32(kU)
    if (rs_scheme_ == FCGLE_STRANG) {
      float* W = F32(kWork);
      tucker_f32(F32(kUh), W, false);
      flow_kernel<<<grid_for(P_ / 4), 256, 0, st_>>>(P32(), flow(rs_tau_ / 2), W, F32(kU));
      FCGLE_LAUNCHED(launches);
    } else {
      tucker_f32(F32(kUh), F32(kU), false);
    }
  }

  // entry state of the loop from u_0 in F32(kU)
  void begin(int scheme, double tau, double t0) {
    rs_scheme_ = scheme;
    rs_tau_ = tau;
    rs_t0_ = t0;
    float* U = F32(kU);
    SplitOut V = SP(kV);
    const float ft = (float)tau;
    if (kron_scheme(scheme)) {
      // Kronecker-product form: the state is the physical u; V (and W) = the
      // input of the first e^{tau K} of step 0
      if (scheme == FCGLE_STRANG) {
        flow_split_kernel<<<grid_for(P_ / 4), 256, 0, st_>>>(P32(), flow(tau / 2), U, V);
        FCGLE_LAUNCHED(launches);
      } else if (scheme == FCGLE_LAWSON_EULER) {
        gsplit(U, t0, 1.f, ft, V);
      } else {
        gsplit(U, t0, 1.f, ft, V, 1.f, 0.5f * ft, SP(kW));
      }
      return;
    }
    switch (scheme) {
      case FCGLE_STRANG:
        // e^_0 = fwd(u_0) (FP32); V = Phi_{tau/2}(u_0) - u_0
        tucker_f32(U, F32(kUh), true);
        flow_incr_split_kernel<<<grid_for(P_ / 4), 256, 0, st_>>>(P32(), flow(tau / 2), U, V);
        FCGLE_LAUNCHED(launches);
        break;
      case FCGLE_LIE:
      case FCGLE_LAWSON_EULER:
      case FCGLE_LBDF2:
      case FCGLE_LAWSON_RK2:
      case FCGLE_ETD2RK:
      case FCGLE_KROGSTAD:
        // the spectral state U^_0 = fwd(u_0) (FP32) is carried from here on; V = g(t_0, u_0)
        tucker_f32(U, F32(kUh), true);
        gsplit(U, t0, 0.f, 1.f, V);
        break;
      default: throw InvalidArg("unknown scheme");
    }
  }

  // step n: (t_n, u_n) -> u_{n+1}; every step leaves the split input of the next one in V (and W)
  void step(int n) {
    const int scheme = rs_scheme_;
    const double tau = rs_tau_, t0 = rs_t0_, t = t0 + n * tau;
    float* U = F32(kU);
    SplitOut V = SP(kV);
    const float ft = (float)tau;
    if (kron_scheme(scheme)) {
      if (scheme == FCGLE_LAWSON_EULER) {
        // u_{n+1} = e^{tau K}(u_n + tau g_n);  V = u_{n+1} + tau g(t_{n+1}, u_{n+1})
        exp_kron(V, tau, b3::EpiUpdateG{P32(), U, 0, gs_, gtime(t + tau), 1.f, ft, V});
      } else if (scheme == FCGLE_STRANG) {
        // w = e^{tau K} Phi_{tau/2}(u_n);  u_{n+1} = Phi_{tau/2}(w);  V = Phi_tau(w)
        exp_kron(V, tau, b3::EpiStrangKron{P32(), U, flow(tau / 2), flow(tau), V});
      } else {
        // A = e^{tau K}(u_n + tau k_1);  u_{n+1} = e^{tau K}(u_n + tau/2 k_1) + tau/2 g(t_{n+1}, A)
        SplitOut W = SP(kW);
        exp_kron(V, tau, b3::EpiStoreF32{P32(), F32(kEA)});
        exp_kron(W, tau, b3::EpiLRK2Kron{P32(), F32(kEA), U, gs_, gtime(t + tau), ft, V, W});
      }
      return;
    }
    switch (scheme) {
      case FCGLE_LIE:
      case FCGLE_LAWSON_EULER: {
        // U^ <- f(tau Lam)(U^ + tau G^), f = 1/(1 - z) or e^z;  u_{n+1} = bwd(U^);  V = g(t_{n+1}, u_{n+1})
        const int kind = scheme == FCGLE_LIE ? 0 : 1;
        tucker(V, true, b3::EpiSpecStep{P32(), lf_, F32(kUh), kind, ft, ft, V});
        tucker(V, false, b3::EpiUpdateG{P32(), U, 0, gs_, gtime(t + tau), 0.f, 1.f, V});
        break;
      }
      case FCGLE_STRANG: {
        // e^ <- e^{tau Lam}(e^ + fwd(increment));  w = bwd(e^);  u_{n+1} = Phi_{tau/2}(w);
        // next increment Phi_tau(w) - w
        tucker(V, true, b3::EpiSpecStep{P32(), lf_, F32(kUh), 1, ft, 1.f, V});
        tucker(V, false, b3::EpiStrangB{P32(), U, flow(tau / 2), flow(tau), V});
        break;
      }
      case FCGLE_LAWSON_RK2: {
        float *Uh = F32(kUh), *Wh = F32(kEA);
        // V^ = e^z (U^ + tau K^_1) -> v = bwd(V^);  W^ = e^z (U^ + tau/2 K^_1)
        tucker(V, true, b3::EpiLRK2A{P32(), lf_, Uh, Wh, ft, V});
        tucker(V, false, b3::EpiUpdateG{P32(), U, 0, gs_, gtime(t + tau), 0.f, 1.f, V});
        // U^_{n+1} = W^ + tau/2 fwd(g(t_{n+1}, v));  u_{n+1} = bwd(U^_{n+1})
        tucker(V, true, b3::EpiLRK2B{P32(), Wh, Uh, ft, V});
        tucker(V, false, b3::EpiUpdateG{P32(), U, 0, gs_, gtime(t + tau), 0.f, 1.f, V});
        break;
      }
      case FCGLE_LBDF2: {
        // step 0 is linearly-implicit Euler (Eq. lbdf2-v); later steps the LBDF2
        // update of the spectral state with dU^ = U^_n - U^_{n-1}
        const bool first = n == 0;
        const float th = first ? ft : (float)(2.0 * tau / 3.0);
        tucker(V, true, b3::EpiLBDF2S{P32(), lf_, F32(kUh), F32(kUp), th, first ? 0.f : 1.f / 3.f, V});
        tucker(V, false, b3::EpiExtrapG{P32(), U, gs_, gtime(t + 2 * tau), V});
        break;
      }
      case FCGLE_ETD2RK: {
        float* Uh = F32(kUh);
        // S1 = tau phi_1(tau Lam) o (Lam o U^ + G^);  a^ = U^ + S1 (F^ itself is not needed later)
        tucker(V, true, b3::EpiFhat{P32(), lf_, Uh, nullptr, ft, ft, 1, V, phipoly(tau)});
        // a = u + bwd(S1);  D = g(t + tau, a) - g(t, u)
        tucker(V, false, b3::EpiStageD{P32(), U, nullptr, gs_, gtime(t + tau), gtime(t), V});
        // U^_{n+1} = a^ + tau phi_2(tau Lam) o D^
        tucker(V, true, b3::EpiEtd2{P32(), lf_, Uh, ft, V, phipoly(tau)});
        // u_{n+1} = bwd(U^_{n+1});  next G = g(t + tau, u_{n+1})
        tucker(V, false, b3::EpiUpdateG{P32(), U, 0, gs_, gtime(t + tau), 0.f, 1.f, V});
        break;
      }
      case FCGLE_KROGSTAD: {
        float *Uh = F32(kUh), *Fh = F32(kFh), *D2 = F32(kD2), *Wc = F32(kD3);
        const b3::GTime tn = gtime(t), th = gtime(t + tau / 2), t1 = gtime(t + tau);
        // F^ = Lam o U^ + G^;  S = tau/2 phi_1(tau/2 Lam) F^
        tucker(V, true, b3::EpiFhat{P32(), lf_, Uh, Fh, 0.5f * ft, 0.5f * ft, 0, V, phipoly(tau / 2)});
        // U_n2 = u + bwd(S);  D_2 = g(t + tau/2, U_n2) - g(t, u)
        tucker(V, false, b3::EpiStageD{P32(), U, nullptr, gs_, th, tn, V});
        // D^_2;  S = tau (1/2 phi_1(tau/2 Lam) F^ + phi_2(tau/2 Lam) D^_2)
        tucker(V, true, b3::EpiKrog2{P32(), lf_, Fh, D2, ft, V, phipoly(tau / 2)});
        tucker(V, false, b3::EpiStageD{P32(), U, nullptr, gs_, th, tn, V});
        // D^_3;  S = tau (phi_1 F^ + 2 phi_2 D^_3);  W = part of the final combination
        tucker(V, true, b3::EpiKrog3{P32(), lf_, Fh, D2, Wc, ft, V, phipoly(tau)});
        tucker(V, false, b3::EpiStageD{P32(), U, nullptr, gs_, t1, tn, V});
        // D^_4;  U^_{n+1} = U^ + W + tau (4 phi_3 - phi_2) D^_4
        tucker(V, true, b3::EpiKrogFinal{P32(), lf_, Wc, Uh, ft, V, phipoly(tau)});
        // u_{n+1} = bwd(U^_{n+1});  next G = g(t + tau, u_{n+1})
        tucker(V, false, b3::EpiUpdateG{P32(), U, 0, gs_, t1, 0.f, 1.f, V});
        break;
      }
      default: throw InvalidArg("unknown scheme");
    }
  }

  // EngineBase stepping interface
  void begin_steps(int scheme, double tau, double t0, const void* u0) override {
    pack_f32((const float*)u0, F32(kU));
    begin(scheme, tau, t0);
  }
  void one_step(int n) override { step(n); }
  void end_steps(void* uT) override {
    finish();
    unpack_f32(F32(kU), (float*)uT, true);
  }
  bool time_dependent() const override { return gs_.nsrc > 0; }
  bool set_recorder(std::vector<GroupRec>* rec) override {
    if (rec && s_.d < 2) return false;   // d == 1 copies the input aside inside a Tucker operator
    if (rec && kron_scheme(rs_scheme_)) return false;   // the complex products have no grouped form
    rec_ = rec;
    return true;
  }
  std::vector<GroupRec>* rec_ = nullptr;
  bool last_mp_ = false;

  int rs_scheme_ = 0;
  double rs_tau_ = 0.0, rs_t0_ = 0.0;

  fcgle_params prm_;
  cudaStream_t st_;
  Shape s_;
  long long P_ = 0;
  double h_[kMaxDim] = {1, 1, 1};
  Mat mat_[kMaxDim][2];
  std::unique_ptr<DevMem<float>> lamf_[kMaxDim];
  std::unique_ptr<DevMem<double>> lamd_[kMaxDim];
  std::vector<std::unique_ptr<DevMem<float>>> adj_mem_;
  b3::LamF lf_{};
  b3::GStatic gs_{};
  double sig_re_[kMaxSrc] = {0, 0, 0, 0}, sig_im_[kMaxSrc] = {0, 0, 0, 0};
  std::unique_ptr<DevMem<float>> f32_[kNumF32];
  std::unique_ptr<DevMem<__nv_bfloat16>> sp_[kNumSplit];
  std::unique_ptr<DevMem<float>> src_[kMaxSrc];
  std::unique_ptr<DevMem<float>> host_stage_;
  Direction dir_[kMaxDim];
  int exp_form_ = FCGLE_EXP_TUCKER;
  int tucker_form_ = FCGLE_TUCKER_AUTO;
  std::map<uint64_t, std::vector<std::unique_ptr<CMat>>> ecache_;
  std::unique_ptr<DevMem<double>> scratch_;
  std::unique_ptr<DevMem<int>> err_;
};

std::unique_ptr<EngineBase> make_engine_b3(const fcgle_params& prm, cudaStream_t st) {
  return std::unique_ptr<EngineBase>(new EngineB3(prm, st));
}

}  // namespace fcgle
