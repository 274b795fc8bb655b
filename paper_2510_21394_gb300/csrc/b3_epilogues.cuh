// Epilogue functors of the split-BF16 mode product (b3_kernel.cuh).
//
// A functor receives V consecutive complex elements of the FP32 product,
// (re[v], im[v]) at plane indices q + v with q = i * R + r (for the last mode
// product of a Tucker operator this is the standard-order linear index), and
// implements the pointwise part of a scheme that follows the mode product:
//   * the nonlinearity g(t, u) = gamma u - (kappa + i zeta)|u|^2 u + sum_k e^{sigma_k t} S_k (Sec. 2),
//   * Hadamard products with the spectral tensors F = f(theta lam) (Eq. fKu_diag),
//   * the stage combinations of Eq. krogstad-m and the other schemes,
// writing FP32 planar tensors and/or split (hi, lo) bf16 tensors that feed
// the next mode product.  Each functor is a plain struct passed by value with
//   kTmaStore  true: no functor call, the kernel stores the product split
//              through TMA bulk tensor stores (needs R % 8 == 0);
//   kIn, kBatch, load<V>(q, i, r, in), store<V>(q, i, r, re, im, in): the
//              kernel loads the operands of kBatch groups first, then stores.
// V = 4 when R % 4 == 0 (16-byte FP32 and 8-byte split accesses, q % 4 == 0),
// V = 1 otherwise.  Plane indices are 32-bit (the host requires 2 P < 2^32).
#pragma once

#include <cuda_bf16.h>

#include "common.h"

namespace fcgle {
namespace b3 {

struct SplitOut {
  __nv_bfloat16* hi = nullptr;   // 2 P elements: re plane, im plane
  __nv_bfloat16* lo = nullptr;
};

// ------------------------------------------------------------ vector access
template <int V>
__device__ __forceinline__ void ldv(const float* p, float (&o)[V]) {
  if constexpr (V == 4) {
    const float4 x = *reinterpret_cast<const float4*>(p);
    o[0] = x.x; o[1] = x.y; o[2] = x.z; o[3] = x.w;
  } else {
#pragma unroll
    for (int v = 0; v < V; ++v) o[v] = p[v];
  }
}
template <int V>
__device__ __forceinline__ void ldv_ro(const float* p, float (&o)[V]) {   // read-only operands
  if constexpr (V == 4) {
    const float4 x = __ldg(reinterpret_cast<const float4*>(p));
    o[0] = x.x; o[1] = x.y; o[2] = x.z; o[3] = x.w;
  } else {
#pragma unroll
    for (int v = 0; v < V; ++v) o[v] = __ldg(p + v);
  }
}
template <int V>
__device__ __forceinline__ void stv(float* p, const float (&x)[V]) {
  if constexpr (V == 4) {
    *reinterpret_cast<float4*>(p) = make_float4(x[0], x[1], x[2], x[3]);
  } else {
#pragma unroll
    for (int v = 0; v < V; ++v) p[v] = x[v];
  }
}
__device__ __forceinline__ uint32_t bf2(float a, float b, uint32_t& lo) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  const float2 hf = __bfloat1622float2(h);
  const __nv_bfloat162 l = __floats2bfloat162_rn(a - hf.x, b - hf.y);
  lo = *reinterpret_cast<const uint32_t*>(&l);
  return *reinterpret_cast<const uint32_t*>(&h);
}
// x -> (hi, lo) at o.hi[idx..], o.lo[idx..]
template <int V>
__device__ __forceinline__ void put_split(const SplitOut& o, uint32_t idx, const float (&x)[V]) {
  if constexpr (V == 4) {
    uint2 h, l;
    h.x = bf2(x[0], x[1], l.x);
    h.y = bf2(x[2], x[3], l.y);
    *reinterpret_cast<uint2*>(o.hi + idx) = h;
    *reinterpret_cast<uint2*>(o.lo + idx) = l;
  } else {
#pragma unroll
    for (int v = 0; v < V; ++v) {
      const __nv_bfloat16 h = __float2bfloat16_rn(x[v]);
      o.hi[idx + v] = h;
      o.lo[idx + v] = __float2bfloat16_rn(x[v] - __bfloat162float(h));
    }
  }
}
template <int V>
__device__ __forceinline__ void put_csplit(const SplitOut& o, uint32_t P, uint32_t q, const float (&re)[V],
                                           const float (&im)[V]) {
  put_split<V>(o, q, re);
  put_split<V>(o, P + q, im);
}

// g(t, u) ingredients: static part and the factors e^{sigma_k t} of one time t.
struct GStatic {
  float gamma = 0, kappa = 0, zeta = 0;
  int nsrc = 0;
  const float* S[kMaxSrc] = {nullptr, nullptr, nullptr, nullptr};
};
struct GTime {
  float e_re[kMaxSrc] = {0, 0, 0, 0}, e_im[kMaxSrc] = {0, 0, 0, 0};
};

template <int V>
__device__ __forceinline__ void g_eval(const GStatic& g, const GTime& t, uint32_t P, uint32_t q, const float (&ur)[V],
                                       const float (&ui)[V], float (&gr)[V], float (&gi)[V]) {
#pragma unroll
  for (int v = 0; v < V; ++v) {
    const float m2 = ur[v] * ur[v] + ui[v] * ui[v];
    gr[v] = g.gamma * ur[v] - m2 * (g.kappa * ur[v] - g.zeta * ui[v]);
    gi[v] = g.gamma * ui[v] - m2 * (g.kappa * ui[v] + g.zeta * ur[v]);
  }
  for (int k = 0; k < g.nsrc; ++k) {
    float sr[V], si[V];
    ldv_ro<V>(g.S[k] + q, sr);
    ldv_ro<V>(g.S[k] + P + q, si);
#pragma unroll
    for (int v = 0; v < V; ++v) {
      gr[v] += t.e_re[k] * sr[v] - t.e_im[k] * si[v];
      gi[v] += t.e_re[k] * si[v] + t.e_im[k] * sr[v];
    }
  }
}

// Eigenvalues of K at standard-order indices q + v = i_d * R + r + v (Sec. 3.2):
// lam = (nu + i eta) (lam_d[i_d] + sum_{mu < d} lam_mu[digits of r + v]).
// For V = 4, r % 4 == 0 and p_1 % 8 == 0, so only the fastest digit changes.
struct LamF {
  const float* lam[kMaxDim] = {nullptr, nullptr, nullptr};
  int p[kMaxDim] = {1, 1, 1};
  int d = 1;
  float c_re = 0, c_im = 0;
};
template <int V>
__device__ __forceinline__ void lam_eval(const LamF& L, int i, uint32_t r, float (&lr)[V], float (&li)[V]) {
  float base = L.lam[L.d - 1][i];
  uint32_t j1 = r;
  if (L.d >= 2) {
    j1 = r % (uint32_t)L.p[0];
    if (L.d == 3) base += L.lam[1][r / (uint32_t)L.p[0]];
  }
#pragma unroll
  for (int v = 0; v < V; ++v) {
    const float s = L.d >= 2 ? base + L.lam[0][j1 + v] : base;
    lr[v] = L.c_re * s;
    li[v] = L.c_im * s;
  }
}

template <int V>
__device__ __forceinline__ void cmulv(const float (&ar)[V], const float (&ai)[V], const float (&br)[V],
                                      const float (&bi)[V], float (&cr)[V], float (&ci)[V]) {
#pragma unroll
  for (int v = 0; v < V; ++v) {
    cr[v] = ar[v] * br[v] - ai[v] * bi[v];
    ci[v] = ar[v] * bi[v] + ai[v] * br[v];
  }
}

// ---------------------------------------------------------------- functors
#define FCGLE_EPI(IN, BATCH)              \
  static constexpr bool kTmaStore = false; \
  static constexpr int kIn = IN;           \
  static constexpr int kBatch = BATCH;

// product -> split, through TMA stores
struct EpiStoreSplit {
  static constexpr bool kTmaStore = true;
  static constexpr int kIn = 0;
  static constexpr int kBatch = 1;
  template <int V>
  __device__ void load(uint32_t, int, uint32_t, float (&)[1][V]) const {}
  template <int V>
  __device__ void store(uint32_t, int, uint32_t, const float (&)[V], const float (&)[V], const float (&)[1][V]) const {}
};

// product -> split, element stores (any R)
struct EpiStoreSplitGen {
  FCGLE_EPI(0, 4)
  uint32_t P;
  SplitOut Y;
  template <int V>
  __device__ void load(uint32_t, int, uint32_t, float (&)[1][V]) const {}
  template <int V>
  __device__ void store(uint32_t q, int, uint32_t, const float (&re)[V], const float (&im)[V],
                        const float (&)[1][V]) const {
    put_csplit<V>(Y, P, q, re, im);
  }
};

// product -> FP32
struct EpiStoreF32 {
  FCGLE_EPI(0, 4)
  uint32_t P;
  float* Y;
  template <int V>
  __device__ void load(uint32_t, int, uint32_t, float (&)[1][V]) const {}
  template <int V>
  __device__ void store(uint32_t q, int, uint32_t, const float (&re)[V], const float (&im)[V],
                        const float (&)[1][V]) const {
    stv<V>(Y + q, re);
    stv<V>(Y + P + q, im);
  }
};

// Y = F o product  (split)
struct EpiScaleSplit {
  FCGLE_EPI(2, 2)
  uint32_t P;
  const float* F;
  SplitOut Y;
  template <int V>
  __device__ void load(uint32_t q, int, uint32_t, float (&in)[2][V]) const {
    ldv_ro<V>(F + q, in[0]);
    ldv_ro<V>(F + P + q, in[1]);
  }
  template <int V>
  __device__ void store(uint32_t q, int, uint32_t, const float (&re)[V], const float (&im)[V],
                        const float (&in)[2][V]) const {
    float yr[V], yi[V];
    cmulv<V>(in[0], in[1], re, im, yr, yi);
    put_csplit<V>(Y, P, q, yr, yi);
  }
};

// u = (add ? U : 0) + product -> U (FP32);  V = a u + b g(t', u) -> split
struct EpiUpdateG {
  FCGLE_EPI(2, 2)
  uint32_t P;
  float* U;
  int add;
  GStatic g;
  GTime t;
  float a, b;
  SplitOut Vout;
  template <int V>
  __device__ void load(uint32_t q, int, uint32_t, float (&in)[2][V]) const {
    if (add) {
      ldv<V>(U + q, in[0]);
      ldv<V>(U + P + q, in[1]);
    }
  }
  template <int V>
  __device__ void store(uint32_t q, int, uint32_t, const float (&re)[V], const float (&im)[V],
                        const float (&in)[2][V]) const {
    float ur[V], ui[V], gr[V], gi[V], vr[V], vi[V];
#pragma unroll
    for (int v = 0; v < V; ++v) {
      ur[v] = add ? re[v] + in[0][v] : re[v];
      ui[v] = add ? im[v] + in[1][v] : im[v];
      gr[v] = gi[v] = 0.f;
    }
    stv<V>(U + q, ur);
    stv<V>(U + P + q, ui);
    if (b != 0.f) g_eval<V>(g, t, P, q, ur, ui, gr, gi);
#pragma unroll
    for (int v = 0; v < V; ++v) {
      vr[v] = a * ur[v] + b * gr[v];
      vi[v] = a * ui[v] + b * gi[v];
    }
    put_csplit<V>(Vout, P, q, vr, vi);
  }
};

// u_s = U + product;  D = g(t_s, u_s) - g(t_n, U) -> split;  optionally U_out = u_s
struct EpiStageD {
  FCGLE_EPI(2, 2)
  uint32_t P;
  const float* U;
  float* Uout;
  GStatic g;
  GTime ts, tn;
  SplitOut D;
  template <int V>
  __device__ void load(uint32_t q, int, uint32_t, float (&in)[2][V]) const {
    ldv<V>(U + q, in[0]);
    ldv<V>(U + P + q, in[1]);
  }
  template <int V>
  __device__ void store(uint32_t q, int, uint32_t, const float (&re)[V], const float (&im)[V],
                        const float (&in)[2][V]) const {
    float sr[V], si[V], g1r[V], g1i[V], g0r[V], g0i[V];
#pragma unroll
    for (int v = 0; v < V; ++v) {
      sr[v] = in[0][v] + re[v];
      si[v] = in[1][v] + im[v];
    }
    g_eval<V>(g, ts, P, q, sr, si, g1r, g1i);
    g_eval<V>(g, tn, P, q, in[0], in[1], g0r, g0i);
#pragma unroll
    for (int v = 0; v < V; ++v) {
      g1r[v] -= g0r[v];
      g1i[v] -= g0i[v];
    }
    put_csplit<V>(D, P, q, g1r, g1i);
    if (Uout) {
      stv<V>(Uout + q, sr);
      stv<V>(Uout + P + q, si);
    }
  }
};

// G^ = product;  F^ = Lam o U^ + G^ -> Fh;  S = c P1 o F^ -> split;  optionally U^ += S
struct EpiFhat {
  FCGLE_EPI(4, 2)
  uint32_t P;
  LamF L;
  float* Uh;
  float* Fh;
  const float* P1;
  float c;
  int update_uh;
  SplitOut S;
  template <int V>
  __device__ void load(uint32_t q, int, uint32_t, float (&in)[4][V]) const {
    ldv<V>(Uh + q, in[0]);
    ldv<V>(Uh + P + q, in[1]);
    ldv_ro<V>(P1 + q, in[2]);
    ldv_ro<V>(P1 + P + q, in[3]);
  }
  template <int V>
  __device__ void store(uint32_t q, int i, uint32_t r, const float (&re)[V], const float (&im)[V],
                        const float (&in)[4][V]) const {
    float lr[V], li[V], fr[V], fi[V], sr[V], si[V];
    lam_eval<V>(L, i, r, lr, li);
    cmulv<V>(lr, li, in[0], in[1], fr, fi);
#pragma unroll
    for (int v = 0; v < V; ++v) {
      fr[v] += re[v];
      fi[v] += im[v];
    }
    stv<V>(Fh + q, fr);
    stv<V>(Fh + P + q, fi);
    cmulv<V>(in[2], in[3], fr, fi, sr, si);
#pragma unroll
    for (int v = 0; v < V; ++v) {
      sr[v] *= c;
      si[v] *= c;
    }
    put_csplit<V>(S, P, q, sr, si);
    if (update_uh) {
#pragma unroll
      for (int v = 0; v < V; ++v) {
        fr[v] = in[0][v] + sr[v];
        fi[v] = in[1][v] + si[v];
      }
      stv<V>(Uh + q, fr);
      stv<V>(Uh + P + q, fi);
    }
  }
};

// D^ = product -> Dsave (optional);  S = a Pa o F^ + b Pb o D^ -> split;  optionally U^ += S
struct EpiStage2 {
  FCGLE_EPI(8, 1)
  uint32_t P;
  const float* Fh;   // may be null when a == 0
  const float* Pa;
  float a;
  const float* Pb;
  float b;
  float* Dsave;
  float* Uh;         // null: no update
  SplitOut S;
  template <int V>
  __device__ void load(uint32_t q, int, uint32_t, float (&in)[8][V]) const {
    ldv_ro<V>(Pb + q, in[0]);
    ldv_ro<V>(Pb + P + q, in[1]);
    if (a != 0.f) {
      ldv_ro<V>(Pa + q, in[2]);
      ldv_ro<V>(Pa + P + q, in[3]);
      ldv_ro<V>(Fh + q, in[4]);
      ldv_ro<V>(Fh + P + q, in[5]);
    }
    if (Uh) {
      ldv<V>(Uh + q, in[6]);
      ldv<V>(Uh + P + q, in[7]);
    }
  }
  template <int V>
  __device__ void store(uint32_t q, int, uint32_t, const float (&re)[V], const float (&im)[V],
                        const float (&in)[8][V]) const {
    if (Dsave) {
      stv<V>(Dsave + q, re);
      stv<V>(Dsave + P + q, im);
    }
    float sr[V], si[V], tr[V], ti[V];
    cmulv<V>(in[0], in[1], re, im, sr, si);
    if (a != 0.f) cmulv<V>(in[2], in[3], in[4], in[5], tr, ti);
#pragma unroll
    for (int v = 0; v < V; ++v) {
      sr[v] *= b;
      si[v] *= b;
      if (a != 0.f) {
        sr[v] += a * tr[v];
        si[v] += a * ti[v];
      }
    }
    put_csplit<V>(S, P, q, sr, si);
    if (Uh) {
#pragma unroll
      for (int v = 0; v < V; ++v) {
        tr[v] = in[6][v] + sr[v];
        ti[v] = in[7][v] + si[v];
      }
      stv<V>(Uh + q, tr);
      stv<V>(Uh + P + q, ti);
    }
  }
};

// Krogstad's last combination (Eq. krogstad-m):
// S = tau (P1 F^ + P2 (2 D2 + 2 D3 - D4) + P3 (-4 D2 - 4 D3 + 4 D4)) -> split; U^ += S
struct EpiKrogFinal {
  FCGLE_EPI(14, 1)
  uint32_t P;
  const float *Fh, *D2, *D3, *P1, *P2, *P3;
  float* Uh;
  float tau;
  SplitOut S;
  template <int V>
  __device__ void load(uint32_t q, int, uint32_t, float (&in)[14][V]) const {
    ldv_ro<V>(Fh + q, in[0]);
    ldv_ro<V>(Fh + P + q, in[1]);
    ldv_ro<V>(D2 + q, in[2]);
    ldv_ro<V>(D2 + P + q, in[3]);
    ldv_ro<V>(D3 + q, in[4]);
    ldv_ro<V>(D3 + P + q, in[5]);
    ldv_ro<V>(P1 + q, in[6]);
    ldv_ro<V>(P1 + P + q, in[7]);
    ldv_ro<V>(P2 + q, in[8]);
    ldv_ro<V>(P2 + P + q, in[9]);
    ldv_ro<V>(P3 + q, in[10]);
    ldv_ro<V>(P3 + P + q, in[11]);
    ldv<V>(Uh + q, in[12]);
    ldv<V>(Uh + P + q, in[13]);
  }
  template <int V>
  __device__ void store(uint32_t q, int, uint32_t, const float (&re)[V], const float (&im)[V],
                        const float (&in)[14][V]) const {
    float sr[V], si[V], ur[V], ui[V];
#pragma unroll
    for (int v = 0; v < V; ++v) {
      const float br = 2.f * in[2][v] + 2.f * in[4][v] - re[v], bi = 2.f * in[3][v] + 2.f * in[5][v] - im[v];
      const float cr = 4.f * (re[v] - in[2][v] - in[4][v]), ci = 4.f * (im[v] - in[3][v] - in[5][v]);
      float xr = in[6][v] * in[0][v] - in[7][v] * in[1][v];
      float xi = in[6][v] * in[1][v] + in[7][v] * in[0][v];
      xr += in[8][v] * br - in[9][v] * bi;
      xi += in[8][v] * bi + in[9][v] * br;
      xr += in[10][v] * cr - in[11][v] * ci;
      xi += in[10][v] * ci + in[11][v] * cr;
      sr[v] = tau * xr;
      si[v] = tau * xi;
      ur[v] = in[12][v] + sr[v];
      ui[v] = in[13][v] + si[v];
    }
    put_csplit<V>(S, P, q, sr, si);
    stv<V>(Uh + q, ur);
    stv<V>(Uh + P + q, ui);
  }
};

// LBDF2 (Eq. lbdf2-v): u_{n+1} = product -> U, u_n -> Uprev;
// next right-hand side 4/3 u_{n+1} - 1/3 u_n + 2 tau/3 g(t_{n+2}, 2 u_{n+1} - u_n) -> split
struct EpiLBDF2 {
  FCGLE_EPI(2, 2)
  uint32_t P;
  float* U;
  float* Uprev;
  GStatic g;
  GTime t;
  float tau;
  SplitOut Vout;
  template <int V>
  __device__ void load(uint32_t q, int, uint32_t, float (&in)[2][V]) const {
    ldv<V>(U + q, in[0]);
    ldv<V>(U + P + q, in[1]);
  }
  template <int V>
  __device__ void store(uint32_t q, int, uint32_t, const float (&re)[V], const float (&im)[V],
                        const float (&in)[2][V]) const {
    stv<V>(Uprev + q, in[0]);
    stv<V>(Uprev + P + q, in[1]);
    stv<V>(U + q, re);
    stv<V>(U + P + q, im);
    float er[V], ei[V], gr[V], gi[V];
#pragma unroll
    for (int v = 0; v < V; ++v) {
      er[v] = 2.f * re[v] - in[0][v];
      ei[v] = 2.f * im[v] - in[1][v];
    }
    g_eval<V>(g, t, P, q, er, ei, gr, gi);
    const float c = 2.f * tau / 3.f;
#pragma unroll
    for (int v = 0; v < V; ++v) {
      er[v] = (4.f * re[v] - in[0][v]) / 3.f + c * gr[v];
      ei[v] = (4.f * im[v] - in[1][v]) / 3.f + c * gi[v];
    }
    put_csplit<V>(Vout, P, q, er, ei);
  }
};

// Lawson-RK2 (Heun): u_{n+1} = product + tau/2 g(t_{n+1}, EA) -> U;
// next k1 = g(t_{n+1}, u_{n+1}); A = u + tau k1, B = u + tau/2 k1 -> split
struct EpiLawsonRK2 {
  FCGLE_EPI(2, 2)
  uint32_t P;
  float* U;
  const float* EA;
  GStatic g;
  GTime t;   // t_{n+1}
  float tau;
  SplitOut A, Bv;
  template <int V>
  __device__ void load(uint32_t q, int, uint32_t, float (&in)[2][V]) const {
    ldv_ro<V>(EA + q, in[0]);
    ldv_ro<V>(EA + P + q, in[1]);
  }
  template <int V>
  __device__ void store(uint32_t q, int, uint32_t, const float (&re)[V], const float (&im)[V],
                        const float (&in)[2][V]) const {
    float gr[V], gi[V], ur[V], ui[V];
    g_eval<V>(g, t, P, q, in[0], in[1], gr, gi);
#pragma unroll
    for (int v = 0; v < V; ++v) {
      ur[v] = re[v] + 0.5f * tau * gr[v];
      ui[v] = im[v] + 0.5f * tau * gi[v];
    }
    stv<V>(U + q, ur);
    stv<V>(U + P + q, ui);
    g_eval<V>(g, t, P, q, ur, ui, gr, gi);
    float ar[V], ai[V];
#pragma unroll
    for (int v = 0; v < V; ++v) {
      ar[v] = ur[v] + tau * gr[v];
      ai[v] = ui[v] + tau * gi[v];
      ur[v] += 0.5f * tau * gr[v];
      ui[v] += 0.5f * tau * gi[v];
    }
    put_csplit<V>(A, P, q, ar, ai);
    put_csplit<V>(Bv, P, q, ur, ui);
  }
};

// Exact flow of w' = gamma w - (kappa + i zeta)|w|^2 w over time t (Sec. 4):
// w(t) = exp(t gamma - (kappa + i zeta)/(2 kappa) log(1 + 2 t phi_1(2 gamma t) kappa |w0|^2)) w0
struct Flow {
  float gamma_t;   // t gamma
  float c2;        // 2 t phi_1(2 gamma t) kappa
  float zk;        // zeta / (2 kappa)
};
__device__ __forceinline__ void flow_eval(const Flow& f, float wr, float wi, float& yr, float& yi) {
  const float L = log1pf(f.c2 * (wr * wr + wi * wi));
  const float m = expf(f.gamma_t - 0.5f * L);
  float s, c;
  sincosf(-f.zk * L, &s, &c);
  yr = m * (c * wr - s * wi);
  yi = m * (c * wi + s * wr);
}

// Strang (Eq. Strang): u_{n+1} = Phi(product) -> U;  next V = Phi(u_{n+1}) -> split
struct EpiStrang {
  FCGLE_EPI(0, 4)
  uint32_t P;
  float* U;
  Flow f;
  SplitOut Vout;
  template <int V>
  __device__ void load(uint32_t, int, uint32_t, float (&)[1][V]) const {}
  template <int V>
  __device__ void store(uint32_t q, int, uint32_t, const float (&re)[V], const float (&im)[V],
                        const float (&)[1][V]) const {
    float ur[V], ui[V], vr[V], vi[V];
#pragma unroll
    for (int v = 0; v < V; ++v) {
      flow_eval(f, re[v], im[v], ur[v], ui[v]);
      flow_eval(f, ur[v], ui[v], vr[v], vi[v]);
    }
    stv<V>(U + q, ur);
    stv<V>(U + P + q, ui);
    put_csplit<V>(Vout, P, q, vr, vi);
  }
};

#undef FCGLE_EPI

}  // namespace b3
}  // namespace fcgle
