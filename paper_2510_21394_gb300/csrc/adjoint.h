// Discrete adjoint of the Heun-based Lawson-RK2 scheme on the device.
//
// Forward step (E = exp(tau K), applied in the Tucker form Q (e^{tau lam} o Q^T x)):
//     k1 = g(t, u);  a = u + tau k1;  v = E a;  b = u + tau/2 k1;  w = E b;
//     u' = w + tau/2 g(t + tau, v).
// Misfit J = 1/2 sum |u(T) - u_target|^2; gradients in the real sense
// (dJ/dRe + i dJ/dIm).  Backward step, lambda = dJ/du':
//     mu_v  = tau/2 (D_v g)^* lambda
//     lambda_b = E^H lambda,  lambda_a = E^H mu_v          (E^H = Q (conj(e^{tau lam}) o Q^T .))
//     lambda_k1 = tau lambda_a + tau/2 lambda_b
//     lambda <- lambda_a + lambda_b + (D_u g)^* lambda_k1,
// with (D_z g)^* w = conj(alpha) w + beta conj(w), alpha = gamma - 2(kappa+i zeta)|z|^2,
// beta = -(kappa + i zeta) z^2.  Parameter gradients:
//     dJ/dgamma, dkappa, dzeta: Re<lambda_k1, dg/dp(u)> + Re<tau/2 lambda, dg/dp(v)>,
//         dg/dgamma = z, dg/dkappa = -|z|^2 z, dg/dzeta = -i |z|^2 z;
//     dJ/dnu = tau Re Z, dJ/deta = -tau Im Z,  Z = sum_steps sum conj(Q^T lambda) Lam_D (Q^T w)
//         + conj(Q^T mu_v) Lam_D (Q^T v),  Lam_D the eigenvalues of K_D = (+)_mu D_mu,
//     because dE/dnu = tau K_D E and dE/deta = i tau K_D E.
// Memory: states are checkpointed every C steps in the forward sweep; each
// segment is recomputed forward (storing u_n, v_n, Q^T v_n, Q^T w_n) and then
// swept backward, so the cost is about three forward integrations.
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

// y = e^{theta (nu +/- i eta) lam} o x (conj selects the minus sign), evaluated in FP64
template <typename T>
void adj_scale_exp(const Shape& s, const LamVecs& lv, double theta, bool conj, const T* x, T* y, cudaStream_t st,
                   long long& nl);

// acc[Z_RE, Z_IM] += sum conj(x) Lam_D y  (Lam_D from the lam_mu vectors, weight 1)
template <typename T>
void adj_spec_dot(const Shape& s, const LamVecs& lv, const T* x, const T* y, double* acc, cudaStream_t st,
                  long long& nl);

// y = a x1 + b x2 (real coefficients; x2 may be null)
template <typename T>
void adj_axpby(const Shape& s, double a, const T* x1, double b, const T* x2, T* y, cudaStream_t st, long long& nl);

// Driver.  Eng provides: Shape shape(); cudaStream_t stream(); long long& nlaunch();
// GParams gparams(); LamVecs lamvecs(); T* alloc(size_t n) (freed by the caller afterwards);
// void tuckerT(const T* X, T* Y, bool fwd) on planar tensors (X, Y distinct).
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
  T* u = buf(T2);
  T* a = buf(T2);
  T* b = buf(T2);
  T* x1 = buf(T2);
  T* x2 = buf(T2);
  T* lam = buf(T2);
  T* mu = buf(T2);
  T* la = buf(T2);
  T* lb = buf(T2);
  double* acc = reinterpret_cast<double*>(buf((ADJ_NACC * sizeof(double) + sizeof(T) - 1) / sizeof(T)));
  FCGLE_CUDA(cudaMemsetAsync(acc, 0, ADJ_NACC * sizeof(double), st));

  // one forward step u -> u (Tucker-form exp), optionally storing u_n, v, Q^T v, Q^T w
  auto fstep = [&](double t, T* uu, T* keep_u, T* keep_v, T* keep_vh, T* keep_wh) {
    if (keep_u) FCGLE_CUDA(cudaMemcpyAsync(keep_u, uu, T2 * sizeof(T), cudaMemcpyDeviceToDevice, st));
    // a = u + tau g(t, u), b = u + tau/2 g(t, u)
    gcombo<T>(s, gp0, t, uu, nullptr, nullptr, 1, 0, 1, 0, tau, 0, a, st, nl);
    gcombo<T>(s, gp0, t, uu, nullptr, nullptr, 1, 0, 1, 0, 0.5 * tau, 0, b, st, nl);
    // v = E a
    e.tuckerT(a, x1, true);
    adj_scale_exp<T>(s, lv, tau, false, x1, x2, st, nl);
    if (keep_vh) FCGLE_CUDA(cudaMemcpyAsync(keep_vh, x2, T2 * sizeof(T), cudaMemcpyDeviceToDevice, st));
    T* v = keep_v ? keep_v : a;
    e.tuckerT(x2, v, false);
    // w = E b
    e.tuckerT(b, x1, true);
    adj_scale_exp<T>(s, lv, tau, false, x1, x2, st, nl);
    if (keep_wh) FCGLE_CUDA(cudaMemcpyAsync(keep_wh, x2, T2 * sizeof(T), cudaMemcpyDeviceToDevice, st));
    e.tuckerT(x2, b, false);
    // u' = w + tau/2 g(t + tau, v)
    gcombo<T>(s, gp0, t + tau, v, b, nullptr, 1, 0, 0, 1, 0.5 * tau, 0, uu, st, nl);
  };

  // ---- forward sweep with checkpoints
  FCGLE_CUDA(cudaMemcpyAsync(u, u0, T2 * sizeof(T), cudaMemcpyDeviceToDevice, st));
  for (int n = 0; n < nsteps; ++n) {
    if (n % C == 0) FCGLE_CUDA(cudaMemcpyAsync(ck[n / C], u, T2 * sizeof(T), cudaMemcpyDeviceToDevice, st));
    fstep(t0 + n * tau, u, nullptr, nullptr, nullptr, nullptr);
  }
  adj_misfit<T>(s, u, target, lam, acc, st, nl);

  // ---- backward sweep, segment by segment
  for (int k = nseg - 1; k >= 0; --k) {
    const int n0 = k * C, n1 = std::min(nsteps, n0 + C);
    FCGLE_CUDA(cudaMemcpyAsync(u, ck[k], T2 * sizeof(T), cudaMemcpyDeviceToDevice, st));
    for (int n = n0; n < n1; ++n) fstep(t0 + n * tau, u, su[n - n0], sv[n - n0], svh[n - n0], swh[n - n0]);
    for (int n = n1 - 1; n >= n0; --n) {
      const int j = n - n0;
      // mu_v = tau/2 (D_v g)^* lambda
      adj_gv<T>(s, gp0, sv[j], lam, 0.5 * tau, mu, acc, st, nl);
      // lambda_b = E^H lambda;  Z += conj(Q^T lambda) Lam_D (Q^T w)
      e.tuckerT(lam, x1, true);
      adj_spec_dot<T>(s, lv, x1, swh[j], acc, st, nl);
      adj_scale_exp<T>(s, lv, tau, true, x1, x2, st, nl);
      e.tuckerT(x2, lb, false);
      // lambda_a = E^H mu_v;  Z += conj(Q^T mu_v) Lam_D (Q^T v)
      e.tuckerT(mu, x1, true);
      adj_spec_dot<T>(s, lv, x1, svh[j], acc, st, nl);
      adj_scale_exp<T>(s, lv, tau, true, x1, x2, st, nl);
      e.tuckerT(x2, la, false);
      // lambda <- lambda_a + lambda_b + (D_u g)^* (tau lambda_a + tau/2 lambda_b)
      adj_gu<T>(s, gp0, su[j], la, lb, tau, 0.5 * tau, lam, acc, st, nl);
    }
  }
  FCGLE_CUDA(cudaMemcpyAsync(grad_u0, lam, T2 * sizeof(T), cudaMemcpyDeviceToDevice, st));
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
