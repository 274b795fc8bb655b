// Discrete adjoint of the Heun-based Lawson-RK2 scheme on the device.
//
// The scheme is run in spectral form with the spectral state U^ = Q^T u as
// the primary variable (Q = Q_d (x) ... (x) Q_1, fwd = Q^T ., bwd = Q .;
// E = e^{tau K} acts on U^ as the diagonal e^{tau Lam}):
//     u = bwd(U^);  k1 = g(t, u);  K^ = fwd(k1);
//     V^ = E(U^ + tau K^);  W^ = E(U^ + tau/2 K^);  v = bwd(V^);
//     U^' = W^ + tau/2 fwd(g(t + tau, v)),
// which is the physical step (k1 = g(t, u); v = E(u + tau k1);
// u' = E(u + tau/2 k1) + tau/2 g(t + tau, v)) written in the eigenbasis.
// The first forward (U^_0 = fwd(u_0)) and the last backward (u_N = bwd(U^_N))
// operators use the engine's precise transform; the per-step ones may be
// reduced precision, whose error then enters only through tau-small terms.
// Misfit J = 1/2 sum |u_N - u_target|^2; gradients in the real sense
// (dJ/dRe + i dJ/dIm).  Spectral adjoint m^ = dJ/dU^; backward step:
//     m_v  = (D_v g)^* (tau/2 bwd(m^'))              (physical)
//     m^_V = fwd(m_v);  a = E^H m^_V;  b = E^H m^'   (E^H = conj(e^{tau Lam}))
//     m^   = a + b + fwd((D_u g)^* bwd(tau a + tau/2 b)),
// with (D_z g)^* w = conj(alpha) w + beta conj(w), alpha = gamma - 2(kappa+i zeta)|z|^2,
// beta = -(kappa + i zeta) z^2.  Parameter gradients:
//     dJ/dgamma, dkappa, dzeta: Re<bwd(tau a + tau/2 b), dg/dp(u)> + Re<tau/2 bwd(m^'), dg/dp(v)>,
//         dg/dgamma = z, dg/dkappa = -|z|^2 z, dg/dzeta = -i |z|^2 z;
//     dJ/dnu = tau Re Z, dJ/deta = -tau Im Z,  Z = sum_steps sum conj(m^') Lam_D W^ + conj(m^_V) Lam_D V^,
//         Lam_D the eigenvalues of K_D = (+)_mu D_mu,
//     because dE/dnu = tau K_D E and dE/deta = i tau K_D E.
// dJ/du_0 = bwd(m^_0).  Memory: U^ is checkpointed every C steps in the
// forward sweep; each segment is recomputed forward (storing u_n, v_n, V^_n,
// W^_n) and then swept backward, so the cost is about three forward
// integrations.
#pragma once

#include <cmath>
#include <memory>
#include <vector>

#include "common.h"

namespace fcgle {

// accumulator slots (device doubles)
enum { ADJ_Z_RE = 0, ADJ_Z_IM, ADJ_GAMMA, ADJ_KAPPA, ADJ_ZETA, ADJ_LOSS, ADJ_NACC = 8 };

// lambda = u - target; acc[LOSS] += 1/2 sum |lambda|^2
template <typename T>
void adj_misfit(const Shape& s, const T* u, const T* target, T* lam, double* acc, cudaStream_t st, long long& nl);

// mu = c (D_z g)^* w;  acc[GAMMA..ZETA] += Re<c w, (z, -|z|^2 z, -i|z|^2 z)>
template <typename T>
void adj_gv(const Shape& s, const GParams& gp, const T* z, const T* w, double c, T* mu, double* acc,
            cudaStream_t st, long long& nl);

// lk1 = ca la + cb lb;  out = la + lb + (D_u g)^* lk1;  acc[GAMMA..ZETA] += Re<lk1, (u, ...)>
template <typename T>
void adj_gu(const Shape& s, const GParams& gp, const T* u, const T* la, const T* lb, double ca, double cb, T* out,
            double* acc, cudaStream_t st, long long& nl);

// acc[Z_RE, Z_IM] += sum conj(x) Lam_D y  (Lam_D from the lam_mu vectors, weight 1)
template <typename T>
void adj_spec_dot(const Shape& s, const LamVecs& lv, const T* x, const T* y, double* acc, cudaStream_t st,
                  long long& nl);

// y = a x1 + b x2 (real coefficients; x2 may be null)
template <typename T>
void adj_axpby(const Shape& s, double a, const T* x1, double b, const T* x2, T* y, cudaStream_t st, long long& nl);

// y1 = E (x + c1 k), y2 = E (x + c2 k) with E = e^{theta (nu + i eta) Lam} (FP64
// exp / sincos, or the FP32 expm1 form), one pass
template <typename T>
void adj_exp_pair(const Shape& s, const LamVecs& lv, double theta, const T* x, const T* k, double c1, double c2,
                  T* y1, T* y2, cudaStream_t st, long long& nl);

// with a = E^H x, b = E^H m: y = ca a + cb b (y may alias x) and sum = a + b, one pass
template <typename T>
void adj_exp_h_combo(const Shape& s, const LamVecs& lv, double theta, const T* x, const T* m, double ca, double cb,
                     T* y, T* sum, cudaStream_t st, long long& nl);

// Driver.  Eng provides: Shape shape(); cudaStream_t stream(); long long& nlaunch();
// GParams gparams(); LamVecs lamvecs(); T* alloc(size_t n) (freed by the caller afterwards);
// void tuckerT(const T* X, T* Y, bool fwd) and tuckerT_precise(...) on planar
// tensors (X, Y distinct); void g_roundtrip(Uh, U, K, tmp, t): U = bwd(Uh),
// K = fwd(g(t, U)) (tmp: a work tensor the engine may use; all distinct).
template <typename T, class Eng>
void adjoint_lawson_rk2(Eng& e, double tau, int nsteps, double t0, const T* u0, const T* target, int C, T* grad_u0,
                        double* grad_params, double* loss) {
  const Shape s = e.shape();
  cudaStream_t st = e.stream();
  long long& nl = e.nlaunch();
  const GParams gp0 = e.gparams();
  const LamVecs lv = e.lamvecs();
  const size_t T2 = 2 * s.P;
  if (C <= 0) C = nsteps > 0 ? nsteps : 1;
  const int nseg = nsteps > 0 ? (nsteps + C - 1) / C : 0;

  // storage
  auto buf = [&](size_t n) { return e.alloc(n); };
  std::vector<T*> ck(nseg), su(C), sv(C), svh(C), swh(C);
  for (int k = 0; k < nseg; ++k) ck[k] = buf(T2);
  for (int k = 0; k < C; ++k) {
    su[k] = buf(T2);
    sv[k] = buf(T2);
    svh[k] = buf(T2);
    swh[k] = buf(T2);
  }
  T* uh = buf(T2);   // U^ (forward sweep)
  T* u = buf(T2);
  T* x1 = buf(T2);
  T* x2 = buf(T2);
  T* a = buf(T2);
  T* b = buf(T2);
  T* mh = buf(T2);   // m^
  T* mv = buf(T2);
  T* y = buf(T2);
  double* acc = reinterpret_cast<double*>(buf((ADJ_NACC * sizeof(double) + sizeof(T) - 1) / sizeof(T)));
  FCGLE_CUDA(cudaMemsetAsync(acc, 0, ADJ_NACC * sizeof(double), st));
  auto copy = [&](T* dst, const T* src) {
    FCGLE_CUDA(cudaMemcpyAsync(dst, src, T2 * sizeof(T), cudaMemcpyDeviceToDevice, st));
  };

  // one forward step on the spectral state uh, optionally keeping u_n, v_n, V^_n, W^_n
  auto fstep = [&](double t, T* keep_u, T* keep_v, T* keep_vh, T* keep_wh) {
    T* uu = keep_u ? keep_u : u;
    e.g_roundtrip(uh, uu, x2, x1, t);                                            // u = bwd(U^), K^ = fwd(g(t, u))
    T* vh = keep_vh ? keep_vh : a;
    T* wh = keep_wh ? keep_wh : b;
    // V^ = E(U^ + tau K^), W^ = E(U^ + tau/2 K^)
    adj_exp_pair<T>(s, lv, tau, uh, x2, tau, 0.5 * tau, vh, wh, st, nl);
    T* v = keep_v ? keep_v : x1;
    e.g_roundtrip(vh, v, x2, y, t + tau);                                       // v = bwd(V^), fwd(g(t + tau, v))
    adj_axpby<T>(s, 1.0, wh, 0.5 * tau, x2, uh, st, nl);                         // U^' = W^ + tau/2 fwd(g)
  };

  // ---- forward sweep with checkpoints of U^
  e.tuckerT_precise(u0, uh, true);
  for (int n = 0; n < nsteps; ++n) {
    if (n % C == 0) copy(ck[n / C], uh);
    fstep(t0 + n * tau, nullptr, nullptr, nullptr, nullptr);
  }
  e.tuckerT_precise(uh, u, false);                 // u_N
  adj_misfit<T>(s, u, target, x1, acc, st, nl);    // x1 = u_N - target, loss
  e.tuckerT_precise(x1, mh, true);                 // m^_N

  // ---- backward sweep, segment by segment
  for (int k = nseg - 1; k >= 0; --k) {
    const int n0 = k * C, n1 = std::min(nsteps, n0 + C);
    copy(uh, ck[k]);
    for (int n = n0; n < n1; ++n) fstep(t0 + n * tau, su[n - n0], sv[n - n0], svh[n - n0], swh[n - n0]);
    for (int n = n1 - 1; n >= n0; --n) {
      const int j = n - n0;
      adj_spec_dot<T>(s, lv, mh, swh[j], acc, st, nl);        // Z += conj(m^') Lam_D W^
      e.tuckerT(mh, y, false);                                 // bwd(m^')
      adj_gv<T>(s, gp0, sv[j], y, 0.5 * tau, mv, acc, st, nl);  // m_v = (D_v g)^* (tau/2 bwd(m^'))
      e.tuckerT(mv, x1, true);                                 // m^_V
      adj_spec_dot<T>(s, lv, x1, svh[j], acc, st, nl);        // Z += conj(m^_V) Lam_D V^
      // with a = E^H m^_V and b = E^H m^': x1 = tau a + tau/2 b, a <- a + b
      adj_exp_h_combo<T>(s, lv, tau, x1, mh, tau, 0.5 * tau, x1, a, st, nl);
      e.tuckerT(x1, y, false);
      adj_gv<T>(s, gp0, su[j], y, 1.0, mv, acc, st, nl);      // (D_u g)^* bwd(tau a + tau/2 b)
      e.tuckerT(mv, x2, true);
      adj_axpby<T>(s, 1.0, a, 1.0, x2, mh, st, nl);           // m^ = a + b + fwd(...)
    }
  }
  e.tuckerT_precise(mh, grad_u0, false);            // dJ/du_0 = bwd(m^_0)
  double h[ADJ_NACC];
  FCGLE_CUDA(cudaMemcpyAsync(h, acc, sizeof(h), cudaMemcpyDeviceToHost, st));
  FCGLE_CUDA(cudaStreamSynchronize(st));
  grad_params[0] = tau * h[ADJ_Z_RE];
  grad_params[1] = -tau * h[ADJ_Z_IM];
  grad_params[2] = h[ADJ_GAMMA];
  grad_params[3] = h[ADJ_KAPPA];
  grad_params[4] = h[ADJ_ZETA];
  *loss = h[ADJ_LOSS];
}

}  // namespace fcgle
