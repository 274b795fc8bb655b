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
//   kIn, kBatch, load<V>(q, i, r, in), store<V>(q, i, r, re, im, in): the
//              kernel loads the operands of kBatch groups first, then stores.
// (The plain split product without a pointwise stage is b3_plain.cuh.)
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

// ---------------------------------------------------- spectral scalars, FP32
// phi_1, phi_2, phi_3 of z (Eq. phi).  |z| < 1: phi_3 by its power series
// sum_m z^m/(m+3)! (10 terms, remainder < 2e-9 relative), then the exact
// downward relations phi_2 = z phi_3 + 1/2, phi_1 = z phi_2 + 1, which involve
// no cancellation.  |z| >= 1: e^z and the recurrence of Eq. phi (each division
// by z amplifies rounding by at most ~4 there).
__device__ __forceinline__ void phi123(float zr, float zi, float (&pr)[3], float (&pi)[3]) {
  if (zr * zr + zi * zi < 1.f) {
    // 1/(m+3)!, m = 0..9
    constexpr float c[10] = {1.6666667e-01f, 4.1666668e-02f, 8.3333338e-03f, 1.3888889e-03f, 1.9841270e-04f,
                             2.4801587e-05f, 2.7557319e-06f, 2.7557319e-07f, 2.5052108e-08f, 2.0876756e-09f};
    float ar = c[9], ai = 0.f;
#pragma unroll
    for (int m = 8; m >= 0; --m) {
      const float tr = ar * zr - ai * zi + c[m];
      ai = ar * zi + ai * zr;
      ar = tr;
    }
    pr[2] = ar;
    pi[2] = ai;
    pr[1] = zr * ar - zi * ai + 0.5f;
    pi[1] = zr * ai + zi * ar;
    pr[0] = zr * pr[1] - zi * pi[1] + 1.f;
    pi[0] = zr * pi[1] + zi * pr[1];
  } else {
    float s, co;
    sincosf(zi, &s, &co);
    const float ex = expf(zr);
    const float inv = 1.f / (zr * zr + zi * zi);
    const float wr = zr * inv, wi = -zi * inv;   // 1/z
    float er = ex * co - 1.f, ei = ex * s;       // e^z - 1
    pr[0] = er * wr - ei * wi;
    pi[0] = er * wi + ei * wr;
    er = pr[0] - 1.f;
    ei = pi[0];
    pr[1] = er * wr - ei * wi;
    pi[1] = er * wi + ei * wr;
    er = pr[1] - 0.5f;
    ei = pi[1];
    pr[2] = er * wr - ei * wi;
    pi[2] = er * wi + ei * wr;
  }
}

// phi_1..phi_3 along the ray of one launch: z = w s with w = theta (nu + i eta)
// fixed and s the real eigenvalue sum of the element, so the series of phi_3
// becomes a polynomial in the real s with complex coefficients
// c_m = w^m / (m+3)! (computed on the host in FP64) and each Horner step costs
// two FMAs instead of a complex multiply-add.  |z| >= 1 (|s| >= smax) takes
// the recurrence branch of phi123.
struct PhiPoly {
  float cr[10] = {0}, ci[10] = {0};
  float smax = 0.f;
  float wr = 0.f, wi = 0.f;
};
__device__ __forceinline__ void phi123_s(const PhiPoly& P, float s, float (&pr)[3], float (&pi)[3]) {
  const float zr = P.wr * s, zi = P.wi * s;
  if (fabsf(s) < P.smax) {
    float ar = P.cr[9], ai = P.ci[9];
#pragma unroll
    for (int m = 8; m >= 0; --m) {
      ar = fmaf(ar, s, P.cr[m]);
      ai = fmaf(ai, s, P.ci[m]);
    }
    pr[2] = ar;
    pi[2] = ai;
    pr[1] = zr * ar - zi * ai + 0.5f;
    pi[1] = zr * ai + zi * ar;
    pr[0] = zr * pr[1] - zi * pi[1] + 1.f;
    pi[0] = zr * pi[1] + zi * pr[1];
  } else {
    phi123(zr, zi, pr, pi);
  }
}

// real eigenvalue sums s (lam = (nu + i eta) s) at the elements of lam_eval
template <int V>
__device__ __forceinline__ void lam_sum(const LamF& L, int i, uint32_t r, float (&sv)[V]) {
  float base = L.lam[L.d - 1][i];
  uint32_t j1 = r;
  if (L.d >= 2) {
    j1 = r % (uint32_t)L.p[0];
    if (L.d == 3) base += L.lam[1][r / (uint32_t)L.p[0]];
  }
#pragma unroll
  for (int v = 0; v < V; ++v) sv[v] = L.d >= 2 ? base + L.lam[0][j1 + v] : base;
}

// phi_k(z), any k >= 1: Horner form of the series
// (1/k!)(1 + z/(k+1)(1 + z/(k+2)(...))) for |z| < 1.5, recurrence otherwise.
__device__ __forceinline__ void phik(int k, float zr, float zi, float& fr, float& fi) {
  if (zr * zr + zi * zi < 2.25f) {
    float ar = 1.f, ai = 0.f;
    for (int m = 16; m >= 1; --m) {
      const float w = 1.f / (float)(m + k);
      const float tr = 1.f + w * (ar * zr - ai * zi);
      ai = w * (ar * zi + ai * zr);
      ar = tr;
    }
    float f = 1.f;
    for (int j = 2; j <= k; ++j) f *= (float)j;
    fr = ar / f;
    fi = ai / f;
  } else {
    float s, co;
    sincosf(zi, &s, &co);
    const float ex = expf(zr);
    const float inv = 1.f / (zr * zr + zi * zi);
    const float wr = zr * inv, wi = -zi * inv;
    float pr = ex * co, pi = ex * s, fact = 1.f;
    for (int l = 1; l <= k; ++l) {
      if (l >= 2) fact /= (float)(l - 1);
      const float er = pr - fact, ei = pi;
      pr = er * wr - ei * wi;
      pi = er * wi + ei * wr;
    }
    fr = pr;
    fi = pi;
  }
}

// f(z) for kind 0: 1/(1 - z), 1: e^z, 1 + l: phi_l (l >= 1)
__device__ __forceinline__ void fspec(int kind, float zr, float zi, float& fr, float& fi) {
  if (kind == 0) {
    const float ar = 1.f - zr, ai = -zi, inv = 1.f / (ar * ar + ai * ai);
    fr = ar * inv;
    fi = -ai * inv;
  } else if (kind == 1) {
    float s, co;
    sincosf(zi, &s, &co);
    const float ex = expf(zr);
    fr = ex * co;
    fi = ex * s;
  } else if (kind <= 4) {
    float pr[3], pi[3];
    phi123(zr, zi, pr, pi);
    fr = pr[kind - 2];
    fi = pi[kind - 2];
  } else {
    phik(kind - 1, zr, zi, fr, fi);
  }
}

// ---------------------------------------------------------------- functors
#define FCGLE_EPI(IN, BATCH)              \
  static constexpr int kIn = IN;           \
  static constexpr int kBatch = BATCH;

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

// Y = f(theta lam) o product  (split), f evaluated on the fly (fspec kinds)
struct EpiScaleF {
  FCGLE_EPI(0, 4)
  uint32_t P;
  LamF L;
  int kind;
  float theta;
  SplitOut Y;
  template <int V>
  __device__ void load(uint32_t, int, uint32_t, float (&)[1][V]) const {}
  template <int V>
  __device__ void store(uint32_t q, int i, uint32_t r, const float (&re)[V], const float (&im)[V],
                        const float (&)[1][V]) const {
    float lr[V], li[V], yr[V], yi[V];
    lam_eval<V>(L, i, r, lr, li);
#pragma unroll
    for (int v = 0; v < V; ++v) {
      float fr, fi;
      fspec(kind, theta * lr[v], theta * li[v], fr, fi);
      yr[v] = fr * re[v] - fi * im[v];
      yi[v] = fr * im[v] + fi * re[v];
    }
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

// G^ = product;  F^ = Lam o U^ + G^ -> Fh (not stored when Fh is null: ETD2RK
// needs F^ only here);  S = c phi_1(theta Lam) o F^ -> split;  optionally U^ += S
struct EpiFhat {
  FCGLE_EPI(2, 2)
  uint32_t P;
  LamF L;
  float* Uh;
  float* Fh;
  float theta;
  float c;
  int update_uh;
  SplitOut S;
  PhiPoly ph;   // phi series coefficients of this launch (theta = theta)
  template <int V>
  __device__ void load(uint32_t q, int, uint32_t, float (&in)[2][V]) const {
    ldv<V>(Uh + q, in[0]);
    ldv<V>(Uh + P + q, in[1]);
  }
  template <int V>
  __device__ void store(uint32_t q, int i, uint32_t r, const float (&re)[V], const float (&im)[V],
                        const float (&in)[2][V]) const {
    float lr[V], li[V], fr[V], fi[V], sr[V], si[V];
    float sv[V];
    lam_sum<V>(L, i, r, sv);
#pragma unroll
    for (int v = 0; v < V; ++v) {
      lr[v] = L.c_re * sv[v];
      li[v] = L.c_im * sv[v];
    }
    cmulv<V>(lr, li, in[0], in[1], fr, fi);
#pragma unroll
    for (int v = 0; v < V; ++v) {
      fr[v] += re[v];
      fi[v] += im[v];
      float pr[3], pi[3];
      phi123_s(ph, sv[v], pr, pi);
      sr[v] = c * (pr[0] * fr[v] - pi[0] * fi[v]);
      si[v] = c * (pr[0] * fi[v] + pi[0] * fr[v]);
    }
    if (Fh) {
      stv<V>(Fh + q, fr);
      stv<V>(Fh + P + q, fi);
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

// Krogstad stage 2 (Eq. krogstad-m), zh = tau/2 Lam:
// D^_2 = product -> D2;  S = tau (1/2 phi_1(zh) F^ + phi_2(zh) D^_2) -> split
struct EpiKrog2 {
  FCGLE_EPI(2, 2)
  uint32_t P;
  LamF L;
  const float* Fh;
  float* D2;
  float tau;
  SplitOut S;
  PhiPoly ph;   // phi series coefficients of this launch (theta = tau / 2)
  template <int V>
  __device__ void load(uint32_t q, int, uint32_t, float (&in)[2][V]) const {
    ldv_ro<V>(Fh + q, in[0]);
    ldv_ro<V>(Fh + P + q, in[1]);
  }
  template <int V>
  __device__ void store(uint32_t q, int i, uint32_t r, const float (&re)[V], const float (&im)[V],
                        const float (&in)[2][V]) const {
    stv<V>(D2 + q, re);
    stv<V>(D2 + P + q, im);
    float sr[V], si[V];
    float sv[V];
    lam_sum<V>(L, i, r, sv);
#pragma unroll
    for (int v = 0; v < V; ++v) {
      float pr[3], pi[3];
      phi123_s(ph, sv[v], pr, pi);
      const float ar = 0.5f * (pr[0] * in[0][v] - pi[0] * in[1][v]) + (pr[1] * re[v] - pi[1] * im[v]);
      const float ai = 0.5f * (pr[0] * in[1][v] + pi[0] * in[0][v]) + (pr[1] * im[v] + pi[1] * re[v]);
      sr[v] = tau * ar;
      si[v] = tau * ai;
    }
    put_csplit<V>(S, P, q, sr, si);
  }
};

// Krogstad stage 3 (Eq. krogstad-m), z = tau Lam, D^_3 = product:
// S = tau (phi_1 F^ + 2 phi_2 D^_3) -> split, and the part of the final
// combination that is known now,
// W = tau phi_1 F^ + (2 tau phi_2 - 4 tau phi_3) (D^_2 + D^_3) -> W (FP32),
// since P2 (2 D2 + 2 D3 - D4) + P3 (-4 D2 - 4 D3 + 4 D4) = (2 P2 - 4 P3)(D2 + D3) + (4 P3 - P2) D4.
struct EpiKrog3 {
  FCGLE_EPI(4, 2)
  uint32_t P;
  LamF L;
  const float* Fh;
  const float* D2;
  float* W;
  float tau;
  SplitOut S;
  PhiPoly ph;   // phi series coefficients of this launch (theta = tau)
  template <int V>
  __device__ void load(uint32_t q, int, uint32_t, float (&in)[4][V]) const {
    ldv_ro<V>(Fh + q, in[0]);
    ldv_ro<V>(Fh + P + q, in[1]);
    ldv_ro<V>(D2 + q, in[2]);
    ldv_ro<V>(D2 + P + q, in[3]);
  }
  template <int V>
  __device__ void store(uint32_t q, int i, uint32_t r, const float (&re)[V], const float (&im)[V],
                        const float (&in)[4][V]) const {
    float sr[V], si[V], wr[V], wi[V];
    float sv[V];
    lam_sum<V>(L, i, r, sv);
#pragma unroll
    for (int v = 0; v < V; ++v) {
      float pr[3], pi[3];
      phi123_s(ph, sv[v], pr, pi);
      const float fr = pr[0] * in[0][v] - pi[0] * in[1][v], fi = pr[0] * in[1][v] + pi[0] * in[0][v];
      sr[v] = tau * (fr + 2.f * (pr[1] * re[v] - pi[1] * im[v]));
      si[v] = tau * (fi + 2.f * (pr[1] * im[v] + pi[1] * re[v]));
      const float er = in[2][v] + re[v], ei = in[3][v] + im[v];
      const float cr = 2.f * pr[1] - 4.f * pr[2], ci = 2.f * pi[1] - 4.f * pi[2];
      wr[v] = tau * (fr + cr * er - ci * ei);
      wi[v] = tau * (fi + cr * ei + ci * er);
    }
    put_csplit<V>(S, P, q, sr, si);
    stv<V>(W + q, wr);
    stv<V>(W + P + q, wi);
  }
};

// Krogstad final combination, D^_4 = product, z = tau Lam:
// S = W + tau (4 phi_3 - phi_2) D^_4;  U^ += S, and U^_{n+1} -> split (the
// backward Tucker operator then gives u_{n+1} itself)
struct EpiKrogFinal {
  FCGLE_EPI(4, 2)
  uint32_t P;
  LamF L;
  const float* W;
  float* Uh;
  float tau;
  SplitOut S;
  PhiPoly ph;   // phi series coefficients of this launch (theta = tau)
  template <int V>
  __device__ void load(uint32_t q, int, uint32_t, float (&in)[4][V]) const {
    ldv_ro<V>(W + q, in[0]);
    ldv_ro<V>(W + P + q, in[1]);
    ldv<V>(Uh + q, in[2]);
    ldv<V>(Uh + P + q, in[3]);
  }
  template <int V>
  __device__ void store(uint32_t q, int i, uint32_t r, const float (&re)[V], const float (&im)[V],
                        const float (&in)[4][V]) const {
    float sr[V], si[V], ur[V], ui[V];
    float sv[V];
    lam_sum<V>(L, i, r, sv);
#pragma unroll
    for (int v = 0; v < V; ++v) {
      float pr[3], pi[3];
      phi123_s(ph, sv[v], pr, pi);
      const float cr = tau * (4.f * pr[2] - pr[1]), ci = tau * (4.f * pi[2] - pi[1]);
      sr[v] = in[0][v] + cr * re[v] - ci * im[v];
      si[v] = in[1][v] + cr * im[v] + ci * re[v];
      ur[v] = in[2][v] + sr[v];
      ui[v] = in[3][v] + si[v];
    }
    put_csplit<V>(S, P, q, ur, ui);
    stv<V>(Uh + q, ur);
    stv<V>(Uh + P + q, ui);
  }
};

// ETD2RK second stage, D^ = product, z = tau Lam: U^ += tau phi_2(z) D^, and the
// new spectral state U^_{n+1} -> split (the backward Tucker operator then gives
// u_{n+1} itself, so the physical state carries the error of one transform)
struct EpiEtd2 {
  FCGLE_EPI(2, 4)
  uint32_t P;
  LamF L;
  float* Uh;
  float tau;
  SplitOut S;
  PhiPoly ph;   // phi series coefficients of this launch (theta = tau)
  template <int V>
  __device__ void load(uint32_t q, int, uint32_t, float (&in)[2][V]) const {
    ldv<V>(Uh + q, in[0]);
    ldv<V>(Uh + P + q, in[1]);
  }
  template <int V>
  __device__ void store(uint32_t q, int i, uint32_t r, const float (&re)[V], const float (&im)[V],
                        const float (&in)[2][V]) const {
    float sr[V], si[V], ur[V], ui[V];
    float sv[V];
    lam_sum<V>(L, i, r, sv);
#pragma unroll
    for (int v = 0; v < V; ++v) {
      float pr[3], pi[3];
      phi123_s(ph, sv[v], pr, pi);
      sr[v] = tau * (pr[1] * re[v] - pi[1] * im[v]);
      si[v] = tau * (pr[1] * im[v] + pi[1] * re[v]);
      ur[v] = in[0][v] + sr[v];
      ui[v] = in[1][v] + si[v];
    }
    put_csplit<V>(S, P, q, ur, ui);
    stv<V>(Uh + q, ur);
    stv<V>(Uh + P + q, ui);
  }
};

// phi_1(z) = (e^z - 1)/z: Horner form of sum_m z^m/(m+1)! for |z| < 1.5 (16 terms),
// the quotient otherwise.  e^z - 1 = z phi_1(z) then carries no cancellation.
__device__ __forceinline__ void phi1f(float zr, float zi, float& fr, float& fi) {
  if (zr * zr + zi * zi < 2.25f) {
    float ar = 1.f, ai = 0.f;
    for (int m = 16; m >= 1; --m) {
      const float w = 1.f / (float)(m + 1);
      const float tr = 1.f + w * (ar * zr - ai * zi);
      ai = w * (ar * zi + ai * zr);
      ar = tr;
    }
    fr = ar;
    fi = ai;
  } else {
    float sn, co;
    sincosf(zi, &sn, &co);
    const float ex = expf(zr);
    const float er = ex * co - 1.f, ei = ex * sn;
    const float inv = 1.f / (zr * zr + zi * zi);
    fr = (er * zr + ei * zi) * inv;
    fi = (ei * zr - er * zi) * inv;
  }
}

// The schemes below keep the spectral state U^ = Q^T u (FP32) as the primary
// state: each step updates U^ in spectral space, and the backward Tucker
// operator of U^_{n+1} gives u_{n+1}.  The physical state then carries the
// error of one split-BF16 transform instead of one per step.

// Linearly-implicit Euler (kind 0, Eq. lbdf2-v first step), Lawson-Euler
// (kind 1, c = tau) and the linear part of Strang (kind 1, c = 1):
// product = X^ (fwd(g(t_n, u_n)), resp. the flow increment), z = theta Lam,
// f = 1/(1 - z) or e^z:  U^ <- U^ + (f - 1) U^ + c f X^, with f - 1 = z f
// resp. z phi_1(z) (no cancellation); U^_{n+1} -> Uh and -> split.
struct EpiSpecStep {
  FCGLE_EPI(2, 4)
  uint32_t P;
  LamF L;
  float* Uh;
  int kind;
  float theta;
  float c;
  SplitOut S;
  template <int V>
  __device__ void load(uint32_t q, int, uint32_t, float (&in)[2][V]) const {
    ldv<V>(Uh + q, in[0]);
    ldv<V>(Uh + P + q, in[1]);
  }
  template <int V>
  __device__ void store(uint32_t q, int i, uint32_t r, const float (&re)[V], const float (&im)[V],
                        const float (&in)[2][V]) const {
    float lr[V], li[V], ur[V], ui[V];
    lam_eval<V>(L, i, r, lr, li);
#pragma unroll
    for (int v = 0; v < V; ++v) {
      const float zr = theta * lr[v], zi = theta * li[v];
      float fr, fi, mr, mi;   // f and f - 1
      if (kind == 0) {
        const float ar = 1.f - zr, ai = -zi, inv = 1.f / (ar * ar + ai * ai);
        fr = ar * inv;
        fi = -ai * inv;
        mr = zr * fr - zi * fi;
        mi = zr * fi + zi * fr;
      } else {
        float pr, pi;
        phi1f(zr, zi, pr, pi);
        mr = zr * pr - zi * pi;
        mi = zr * pi + zi * pr;
        fr = 1.f + mr;
        fi = mi;
      }
      const float xr = in[0][v], xi = in[1][v];
      ur[v] = xr + (mr * xr - mi * xi) + c * (fr * re[v] - fi * im[v]);
      ui[v] = xi + (mr * xi + mi * xr) + c * (fr * im[v] + fi * re[v]);
    }
    stv<V>(Uh + q, ur);
    stv<V>(Uh + P + q, ui);
    put_csplit<V>(S, P, q, ur, ui);
  }
};

// LBDF2 (Eq. lbdf2-v) in the spectral state: product = G^_e = fwd(g(t_{n+1},
// 2 u_n - u_{n-1})), z = theta Lam, theta = 2 tau / 3; with dU^_n = U^_n - U^_{n-1}
// the step (1 - z) U^_{n+1} = 4/3 U^_n - 1/3 U^_{n-1} + theta G^_e reads
// dU^_{n+1} = (1 - z)^{-1} (dU^_n / 3 + z U^_n + theta G^_e).
// third = 0 and theta = tau give the linearly-implicit Euler first step.
// dU^_{n+1} -> dU, U^_{n+1} -> Uh and -> split.
struct EpiLBDF2S {
  FCGLE_EPI(4, 2)
  uint32_t P;
  LamF L;
  float* Uh;
  float* dU;
  float theta;
  float third;
  SplitOut S;
  template <int V>
  __device__ void load(uint32_t q, int, uint32_t, float (&in)[4][V]) const {
    ldv<V>(Uh + q, in[0]);
    ldv<V>(Uh + P + q, in[1]);
    if (third != 0.f) {
      ldv<V>(dU + q, in[2]);
      ldv<V>(dU + P + q, in[3]);
    } else {
#pragma unroll
      for (int v = 0; v < V; ++v) in[2][v] = in[3][v] = 0.f;
    }
  }
  template <int V>
  __device__ void store(uint32_t q, int i, uint32_t r, const float (&re)[V], const float (&im)[V],
                        const float (&in)[4][V]) const {
    float lr[V], li[V], dr[V], di[V], ur[V], ui[V];
    lam_eval<V>(L, i, r, lr, li);
#pragma unroll
    for (int v = 0; v < V; ++v) {
      const float zr = theta * lr[v], zi = theta * li[v];
      const float ar = 1.f - zr, ai = -zi, inv = 1.f / (ar * ar + ai * ai);
      const float fr = ar * inv, fi = -ai * inv;   // (1 - z)^{-1}
      const float xr = in[0][v], xi = in[1][v];
      const float br = third * in[2][v] + (zr * xr - zi * xi) + theta * re[v];
      const float bi = third * in[3][v] + (zr * xi + zi * xr) + theta * im[v];
      dr[v] = fr * br - fi * bi;
      di[v] = fr * bi + fi * br;
      ur[v] = xr + dr[v];
      ui[v] = xi + di[v];
    }
    stv<V>(dU + q, dr);
    stv<V>(dU + P + q, di);
    stv<V>(Uh + q, ur);
    stv<V>(Uh + P + q, ui);
    put_csplit<V>(S, P, q, ur, ui);
  }
};

// LBDF2 backward epilogue: u_{n+1} = product -> U (u_n read from U first);
// g(t, 2 u_{n+1} - u_n) -> split, the input of the next step's forward operator
struct EpiExtrapG {
  FCGLE_EPI(2, 4)
  uint32_t P;
  float* U;
  GStatic g;
  GTime t;
  SplitOut S;
  template <int V>
  __device__ void load(uint32_t q, int, uint32_t, float (&in)[2][V]) const {
    ldv<V>(U + q, in[0]);
    ldv<V>(U + P + q, in[1]);
  }
  template <int V>
  __device__ void store(uint32_t q, int, uint32_t, const float (&re)[V], const float (&im)[V],
                        const float (&in)[2][V]) const {
    float er[V], ei[V], gr[V], gi[V];
#pragma unroll
    for (int v = 0; v < V; ++v) {
      er[v] = 2.f * re[v] - in[0][v];
      ei[v] = 2.f * im[v] - in[1][v];
    }
    stv<V>(U + q, re);
    stv<V>(U + P + q, im);
    g_eval<V>(g, t, P, q, er, ei, gr, gi);
    put_csplit<V>(S, P, q, gr, gi);
  }
};

// Lawson-RK2 (Heun) in the spectral state, first forward epilogue:
// product = K^_1 = fwd(g(t_n, u_n)), z = tau Lam, e^z = 1 + z phi_1(z):
// V^ = e^z (U^ + tau K^_1) -> split (v = bwd(V^) is the Heun predictor),
// W^ = e^z (U^ + tau/2 K^_1) -> W (FP32)
struct EpiLRK2A {
  FCGLE_EPI(2, 4)
  uint32_t P;
  LamF L;
  const float* Uh;
  float* W;
  float tau;
  SplitOut S;
  template <int V>
  __device__ void load(uint32_t q, int, uint32_t, float (&in)[2][V]) const {
    ldv_ro<V>(Uh + q, in[0]);
    ldv_ro<V>(Uh + P + q, in[1]);
  }
  template <int V>
  __device__ void store(uint32_t q, int i, uint32_t r, const float (&re)[V], const float (&im)[V],
                        const float (&in)[2][V]) const {
    float lr[V], li[V], vr[V], vi[V], wr[V], wi[V];
    lam_eval<V>(L, i, r, lr, li);
#pragma unroll
    for (int v = 0; v < V; ++v) {
      const float zr = tau * lr[v], zi = tau * li[v];
      float pr, pi;
      phi1f(zr, zi, pr, pi);
      const float mr = zr * pr - zi * pi, mi = zr * pi + zi * pr;   // e^z - 1
      const float fr = 1.f + mr, fi = mi;                           // e^z
      const float xr = in[0][v], xi = in[1][v];
      const float br = xr + (mr * xr - mi * xi), bi = xi + (mr * xi + mi * xr);   // e^z U^
      const float kr = fr * re[v] - fi * im[v], ki = fr * im[v] + fi * re[v];     // e^z K^_1
      vr[v] = br + tau * kr;
      vi[v] = bi + tau * ki;
      wr[v] = br + 0.5f * tau * kr;
      wi[v] = bi + 0.5f * tau * ki;
    }
    put_csplit<V>(S, P, q, vr, vi);
    stv<V>(W + q, wr);
    stv<V>(W + P + q, wi);
  }
};

// Lawson-RK2 second forward epilogue: product = fwd(g(t_{n+1}, v)):
// U^_{n+1} = W^ + tau/2 product -> Uh and -> split
struct EpiLRK2B {
  FCGLE_EPI(2, 4)
  uint32_t P;
  const float* W;
  float* Uh;
  float tau;
  SplitOut S;
  template <int V>
  __device__ void load(uint32_t q, int, uint32_t, float (&in)[2][V]) const {
    ldv_ro<V>(W + q, in[0]);
    ldv_ro<V>(W + P + q, in[1]);
  }
  template <int V>
  __device__ void store(uint32_t q, int, uint32_t, const float (&re)[V], const float (&im)[V],
                        const float (&in)[2][V]) const {
    float ur[V], ui[V];
#pragma unroll
    for (int v = 0; v < V; ++v) {
      ur[v] = in[0][v] + 0.5f * tau * re[v];
      ui[v] = in[1][v] + 0.5f * tau * im[v];
    }
    stv<V>(Uh + q, ur);
    stv<V>(Uh + P + q, ui);
    put_csplit<V>(S, P, q, ur, ui);
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

// Phi_t(w) - w = (e^E - 1) w with E = t gamma - (1 + i zeta/kappa) L / 2,
// L = log(1 + c2 |w|^2): e^E - 1 = expm1(Re E) cos(Im E) - 2 sin^2(Im E / 2)
// + i e^{Re E} sin(Im E), without cancellation for small t.
__device__ __forceinline__ void flow_incr(const Flow& f, float wr, float wi, float& dr, float& di) {
  const float L = log1pf(f.c2 * (wr * wr + wi * wi));
  const float a = f.gamma_t - 0.5f * L, b = -f.zk * L;
  float s, c, sh, ch;
  sincosf(b, &s, &c);
  sincosf(0.5f * b, &sh, &ch);
  const float em = expm1f(a);
  const float er = em * c - 2.f * sh * sh, ei = (1.f + em) * s;
  dr = er * wr - ei * wi;
  di = er * wi + ei * wr;
}

// Strang (Eq. Strang) with the spectral state e^ = Q^T w, w the state after
// the linear flow: u_{n+1} = Phi_{tau/2}(w) with w = product -> U, and the
// increment Phi_tau(w) - w -> split, which the next step's forward operator
// turns into e^ <- e^{tau Lam}(e^ + fwd(Phi_tau(w) - w)) (EpiSpecStep, c = 1).
struct EpiStrangB {
  FCGLE_EPI(0, 4)
  uint32_t P;
  float* U;
  Flow half, full;
  SplitOut S;
  template <int V>
  __device__ void load(uint32_t, int, uint32_t, float (&)[1][V]) const {}
  template <int V>
  __device__ void store(uint32_t q, int, uint32_t, const float (&re)[V], const float (&im)[V],
                        const float (&)[1][V]) const {
    float ur[V], ui[V], dr[V], di[V];
#pragma unroll
    for (int v = 0; v < V; ++v) {
      flow_eval(half, re[v], im[v], ur[v], ui[v]);
      flow_incr(full, re[v], im[v], dr[v], di[v]);
    }
    stv<V>(U + q, ur);
    stv<V>(U + P + q, ui);
    put_csplit<V>(S, P, q, dr, di);
  }
};

// ---- Kronecker-product form of the exponential (Eq. Neudeckerd): the state is
// the physical u (FP32) and each e^{tau K} is d complex mode products.

// Strang: w = e^{tau K} Phi_{tau/2}(u_n) is the product; u_{n+1} = Phi_{tau/2}(w),
// and the next step's input Phi_{tau/2}(u_{n+1}) = Phi_tau(w) (the flows of the
// autonomous nonlinear part compose) -> split
struct EpiStrangKron {
  FCGLE_EPI(0, 4)
  uint32_t P;
  float* U;
  Flow half, full;
  SplitOut S;
  template <int V>
  __device__ void load(uint32_t, int, uint32_t, float (&)[1][V]) const {}
  template <int V>
  __device__ void store(uint32_t q, int, uint32_t, const float (&re)[V], const float (&im)[V],
                        const float (&)[1][V]) const {
    float ur[V], ui[V], sr[V], si[V];
#pragma unroll
    for (int v = 0; v < V; ++v) {
      flow_eval(half, re[v], im[v], ur[v], ui[v]);
      flow_eval(full, re[v], im[v], sr[v], si[v]);
    }
    stv<V>(U + q, ur);
    stv<V>(U + P + q, ui);
    put_csplit<V>(S, P, q, sr, si);
  }
};

// Lawson-RK2 (Heun on w = e^{-tK} u): with k_1 = g(t_n, u_n), A = e^{tau K}(u_n + tau k_1)
// already in FP32, the product is e^{tau K}(u_n + tau/2 k_1) and
//   u_{n+1} = product + tau/2 g(t_{n+1}, A);
// the next step's inputs u_{n+1} + tau g(t_{n+1}, u_{n+1}) and u_{n+1} + tau/2 g(...) -> split
struct EpiLRK2Kron {
  FCGLE_EPI(2, 2)
  uint32_t P;
  const float* A;
  float* U;
  GStatic g;
  GTime t;   // t_{n+1}
  float tau;
  SplitOut V1, V2;
  template <int V>
  __device__ void load(uint32_t q, int, uint32_t, float (&in)[2][V]) const {
    ldv<V>(A + q, in[0]);
    ldv<V>(A + P + q, in[1]);
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
    }
    put_csplit<V>(V1, P, q, ar, ai);
#pragma unroll
    for (int v = 0; v < V; ++v) {
      ar[v] = ur[v] + 0.5f * tau * gr[v];
      ai[v] = ui[v] + 0.5f * tau * gi[v];
    }
    put_csplit<V>(V2, P, q, ar, ai);
  }
};

#undef FCGLE_EPI

}  // namespace b3
}  // namespace fcgle
