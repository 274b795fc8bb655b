// Epilogue functors of the split-BF16 mode product (b3_kernel.cuh).
//
// A functor receives one complex element of the FP32 product, (re, im) at
// plane index q = i * R + r (for the last mode product of a Tucker operator
// this is the standard-order linear index of the element), and implements
// the pointwise part of a scheme that follows the mode product:
//   * the nonlinearity g(t, u) = gamma u - (kappa + i zeta)|u|^2 u + sum_k e^{sigma_k t} S_k (Sec. 2),
//   * Hadamard products with the spectral tensors F = f(theta lam) (Eq. fKu_diag),
//   * the stage combinations of Eq. krogstad-m and the other schemes,
// writing FP32 planar tensors and/or split (hi, lo) bf16 tensors that feed
// the next mode product.  Each functor is a plain struct passed by value with
//   kTmaStore  true: no functor call, the kernel stores the product split
//              through TMA bulk tensor stores (needs R % 8 == 0);
//   kIn, kBatch, load(q, i, r, in), store(q, i, r, re, im, in): the kernel
//              loads the operands of kBatch elements first, then stores.
#pragma once

#include <cuda_bf16.h>

#include "common.h"

namespace fcgle {
namespace b3 {

struct SplitOut {
  __nv_bfloat16* hi = nullptr;   // 2 P elements: re plane, im plane
  __nv_bfloat16* lo = nullptr;
};

__device__ __forceinline__ void put_split(const SplitOut& o, long long idx, float x) {
  const __nv_bfloat16 h = __float2bfloat16_rn(x);
  o.hi[idx] = h;
  o.lo[idx] = __float2bfloat16_rn(x - __bfloat162float(h));
}
__device__ __forceinline__ void put_csplit(const SplitOut& o, long long P, long long q, float re, float im) {
  put_split(o, q, re);
  put_split(o, P + q, im);
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

__device__ __forceinline__ void g_eval(const GStatic& g, const GTime& t, long long P, long long q, float ur, float ui,
                                       float& gr, float& gi) {
  const float m2 = ur * ur + ui * ui;
  gr = g.gamma * ur - m2 * (g.kappa * ur - g.zeta * ui);
  gi = g.gamma * ui - m2 * (g.kappa * ui + g.zeta * ur);
  for (int k = 0; k < g.nsrc; ++k) {
    const float sr = __ldg(g.S[k] + q), si = __ldg(g.S[k] + P + q);
    gr += t.e_re[k] * sr - t.e_im[k] * si;
    gi += t.e_re[k] * si + t.e_im[k] * sr;
  }
}

// Eigenvalues of K at the standard-order index q = i_d * R + r (Sec. 3.2):
// lam = (nu + i eta) (lam_d[i_d] + sum_{mu < d} lam_mu[digits of r]).
struct LamF {
  const float* lam[kMaxDim] = {nullptr, nullptr, nullptr};
  int p[kMaxDim] = {1, 1, 1};
  int d = 1;
  float c_re = 0, c_im = 0;
};
__device__ __forceinline__ void lam_eval(const LamF& L, int i, long long r, float& lr, float& li) {
  float s = L.lam[L.d - 1][i];
  long long rem = r;
  for (int mu = 0; mu + 1 < L.d; ++mu) {
    const int j = (int)(rem % L.p[mu]);
    rem /= L.p[mu];
    s += L.lam[mu][j];
  }
  lr = L.c_re * s;
  li = L.c_im * s;
}

__device__ __forceinline__ void cmul(float ar, float ai, float br, float bi, float& cr, float& ci) {
  cr = ar * br - ai * bi;
  ci = ar * bi + ai * br;
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
  __device__ void load(long long, int, long long, float*) const {}
  __device__ void store(long long, int, long long, float, float, const float*) const {}
};

// product -> split, element stores (any R)
struct EpiStoreSplitGen {
  FCGLE_EPI(0, 8)
  long long P;
  SplitOut Y;
  __device__ void load(long long, int, long long, float*) const {}
  __device__ void store(long long q, int, long long, float re, float im, const float*) const {
    put_csplit(Y, P, q, re, im);
  }
};

// product -> FP32
struct EpiStoreF32 {
  FCGLE_EPI(0, 8)
  long long P;
  float* Y;
  __device__ void load(long long, int, long long, float*) const {}
  __device__ void store(long long q, int, long long, float re, float im, const float*) const {
    Y[q] = re;
    Y[P + q] = im;
  }
};

// Y = F o product  (split)
struct EpiScaleSplit {
  FCGLE_EPI(2, 8)
  long long P;
  const float* F;
  SplitOut Y;
  __device__ void load(long long q, int, long long, float* in) const {
    in[0] = __ldg(F + q);
    in[1] = __ldg(F + P + q);
  }
  __device__ void store(long long q, int, long long, float re, float im, const float* in) const {
    float yr, yi;
    cmul(in[0], in[1], re, im, yr, yi);
    put_csplit(Y, P, q, yr, yi);
  }
};

// u = (add ? U : 0) + product -> U (FP32);  V = a u + b g(t', u) -> split
struct EpiUpdateG {
  FCGLE_EPI(2, 8)
  long long P;
  float* U;
  int add;
  GStatic g;
  GTime t;
  float a, b;
  SplitOut V;
  __device__ void load(long long q, int, long long, float* in) const {
    if (add) {
      in[0] = U[q];
      in[1] = U[P + q];
    }
  }
  __device__ void store(long long q, int, long long, float re, float im, const float* in) const {
    float ur = re, ui = im;
    if (add) {
      ur += in[0];
      ui += in[1];
    }
    U[q] = ur;
    U[P + q] = ui;
    float gr = 0.f, gi = 0.f;
    if (b != 0.f) g_eval(g, t, P, q, ur, ui, gr, gi);
    put_csplit(V, P, q, a * ur + b * gr, a * ui + b * gi);
  }
};

// u_s = U + product;  D = g(t_s, u_s) - g(t_n, U) -> split;  optionally U_out = u_s
struct EpiStageD {
  FCGLE_EPI(2, 8)
  long long P;
  const float* U;
  float* Uout;
  GStatic g;
  GTime ts, tn;
  SplitOut D;
  __device__ void load(long long q, int, long long, float* in) const {
    in[0] = U[q];
    in[1] = U[P + q];
  }
  __device__ void store(long long q, int, long long, float re, float im, const float* in) const {
    const float ur = in[0], ui = in[1];
    const float sr = ur + re, si = ui + im;
    float g1r, g1i, g0r, g0i;
    g_eval(g, ts, P, q, sr, si, g1r, g1i);
    g_eval(g, tn, P, q, ur, ui, g0r, g0i);
    put_csplit(D, P, q, g1r - g0r, g1i - g0i);
    if (Uout) {
      Uout[q] = sr;
      Uout[P + q] = si;
    }
  }
};

// G^ = product;  F^ = Lam o U^ + G^ -> Fh;  S = c P1 o F^ -> split;  optionally U^ += S
struct EpiFhat {
  FCGLE_EPI(4, 8)
  long long P;
  LamF L;
  float* Uh;
  float* Fh;
  const float* P1;
  float c;
  int update_uh;
  SplitOut S;
  __device__ void load(long long q, int, long long, float* in) const {
    in[0] = Uh[q];
    in[1] = Uh[P + q];
    in[2] = __ldg(P1 + q);
    in[3] = __ldg(P1 + P + q);
  }
  __device__ void store(long long q, int i, long long r, float re, float im, const float* in) const {
    float lr, li;
    lam_eval(L, i, r, lr, li);
    float fr, fi;
    cmul(lr, li, in[0], in[1], fr, fi);
    fr += re;
    fi += im;
    Fh[q] = fr;
    Fh[P + q] = fi;
    float sr, si;
    cmul(in[2], in[3], fr, fi, sr, si);
    sr *= c;
    si *= c;
    put_csplit(S, P, q, sr, si);
    if (update_uh) {
      Uh[q] = in[0] + sr;
      Uh[P + q] = in[1] + si;
    }
  }
};

// D^ = product -> Dsave (optional);  S = a Pa o F^ + b Pb o D^ -> split;  optionally U^ += S
struct EpiStage2 {
  FCGLE_EPI(8, 4)
  long long P;
  const float* Fh;   // may be null when a == 0
  const float* Pa;
  float a;
  const float* Pb;
  float b;
  float* Dsave;
  float* Uh;         // null: no update
  SplitOut S;
  __device__ void load(long long q, int, long long, float* in) const {
    in[0] = __ldg(Pb + q);
    in[1] = __ldg(Pb + P + q);
    if (a != 0.f) {
      in[2] = __ldg(Pa + q);
      in[3] = __ldg(Pa + P + q);
      in[4] = __ldg(Fh + q);
      in[5] = __ldg(Fh + P + q);
    }
    if (Uh) {
      in[6] = Uh[q];
      in[7] = Uh[P + q];
    }
  }
  __device__ void store(long long q, int, long long, float re, float im, const float* in) const {
    if (Dsave) {
      Dsave[q] = re;
      Dsave[P + q] = im;
    }
    float sr, si;
    cmul(in[0], in[1], re, im, sr, si);
    sr *= b;
    si *= b;
    if (a != 0.f) {
      float tr, ti;
      cmul(in[2], in[3], in[4], in[5], tr, ti);
      sr += a * tr;
      si += a * ti;
    }
    put_csplit(S, P, q, sr, si);
    if (Uh) {
      Uh[q] = in[6] + sr;
      Uh[P + q] = in[7] + si;
    }
  }
};

// Krogstad's last combination (Eq. krogstad-m):
// S = tau (P1 F^ + P2 (2 D2 + 2 D3 - D4) + P3 (-4 D2 - 4 D3 + 4 D4)) -> split; U^ += S
struct EpiKrogFinal {
  FCGLE_EPI(14, 4)
  long long P;
  const float *Fh, *D2, *D3, *P1, *P2, *P3;
  float* Uh;
  float tau;
  SplitOut S;
  __device__ void load(long long q, int, long long, float* in) const {
    in[0] = __ldg(Fh + q);
    in[1] = __ldg(Fh + P + q);
    in[2] = __ldg(D2 + q);
    in[3] = __ldg(D2 + P + q);
    in[4] = __ldg(D3 + q);
    in[5] = __ldg(D3 + P + q);
    in[6] = __ldg(P1 + q);
    in[7] = __ldg(P1 + P + q);
    in[8] = __ldg(P2 + q);
    in[9] = __ldg(P2 + P + q);
    in[10] = __ldg(P3 + q);
    in[11] = __ldg(P3 + P + q);
    in[12] = Uh[q];
    in[13] = Uh[P + q];
  }
  __device__ void store(long long q, int, long long, float re, float im, const float* in) const {
    const float br = 2.f * in[2] + 2.f * in[4] - re, bi = 2.f * in[3] + 2.f * in[5] - im;
    const float cr = 4.f * (re - in[2] - in[4]), ci = 4.f * (im - in[3] - in[5]);
    float sr, si, tr, ti;
    cmul(in[6], in[7], in[0], in[1], sr, si);
    cmul(in[8], in[9], br, bi, tr, ti);
    sr += tr;
    si += ti;
    cmul(in[10], in[11], cr, ci, tr, ti);
    sr = tau * (sr + tr);
    si = tau * (si + ti);
    put_csplit(S, P, q, sr, si);
    Uh[q] = in[12] + sr;
    Uh[P + q] = in[13] + si;
  }
};

// LBDF2 (Eq. lbdf2-v): u_{n+1} = product -> U, u_n -> Uprev;
// next right-hand side 4/3 u_{n+1} - 1/3 u_n + 2 tau/3 g(t_{n+2}, 2 u_{n+1} - u_n) -> split
struct EpiLBDF2 {
  FCGLE_EPI(2, 8)
  long long P;
  float* U;
  float* Uprev;
  GStatic g;
  GTime t;
  float tau;
  SplitOut V;
  __device__ void load(long long q, int, long long, float* in) const {
    in[0] = U[q];
    in[1] = U[P + q];
  }
  __device__ void store(long long q, int, long long, float re, float im, const float* in) const {
    const float or_ = in[0], oi = in[1];
    Uprev[q] = or_;
    Uprev[P + q] = oi;
    U[q] = re;
    U[P + q] = im;
    float gr, gi;
    g_eval(g, t, P, q, 2.f * re - or_, 2.f * im - oi, gr, gi);
    const float c = 2.f * tau / 3.f;
    put_csplit(V, P, q, (4.f * re - or_) / 3.f + c * gr, (4.f * im - oi) / 3.f + c * gi);
  }
};

// Lawson-RK2 (Heun): u_{n+1} = product + tau/2 g(t_{n+1}, EA) -> U;
// next k1 = g(t_{n+1}, u_{n+1}); A = u + tau k1, B = u + tau/2 k1 -> split
struct EpiLawsonRK2 {
  FCGLE_EPI(2, 8)
  long long P;
  float* U;
  const float* EA;
  GStatic g;
  GTime t;   // t_{n+1}
  float tau;
  SplitOut A, Bv;
  __device__ void load(long long q, int, long long, float* in) const {
    in[0] = __ldg(EA + q);
    in[1] = __ldg(EA + P + q);
  }
  __device__ void store(long long q, int, long long, float re, float im, const float* in) const {
    float gr, gi;
    g_eval(g, t, P, q, in[0], in[1], gr, gi);
    const float ur = re + 0.5f * tau * gr, ui = im + 0.5f * tau * gi;
    U[q] = ur;
    U[P + q] = ui;
    g_eval(g, t, P, q, ur, ui, gr, gi);
    put_csplit(A, P, q, ur + tau * gr, ui + tau * gi);
    put_csplit(Bv, P, q, ur + 0.5f * tau * gr, ui + 0.5f * tau * gi);
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
  FCGLE_EPI(0, 8)
  long long P;
  float* U;
  Flow f;
  SplitOut V;
  __device__ void load(long long, int, long long, float*) const {}
  __device__ void store(long long q, int, long long, float re, float im, const float*) const {
    float ur, ui, vr, vi;
    flow_eval(f, re, im, ur, ui);
    U[q] = ur;
    U[P + q] = ui;
    flow_eval(f, ur, ui, vr, vi);
    put_csplit(V, P, q, vr, vi);
  }
};

#undef FCGLE_EPI

}  // namespace b3
}  // namespace fcgle
