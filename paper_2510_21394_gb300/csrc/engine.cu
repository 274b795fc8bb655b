// Engine of one FCGLE handle (see engine.h).
//
// Spectral setup (paper Sec. 2-3): D_mu = -h^{-alpha} toeplitz(g) with the
// FD2 recurrence (Sec. 2) or its FD4 extrapolation (Eq. FD4); D_mu = Q Lam Q^T
// (Eq. diag) on the host in FP64; Q_mu, lam_mu shipped to the device once.
//
// Schemes are written in spectral form (the matrix/tensor-oriented forms of
// Sec. 4: Eqs. lbdf2-m/-t, strang-t, krogstad-m), with the Tucker operator
// V x_1 M_1 ... x_d M_d of Eq. fKu_diag as the building block:
//   fwd(V)  = V x_1 Q_1^T ... x_d Q_d^T     bwd(W) = W x_1 Q_1 ... x_d Q_d
// For ETD2RK and Krogstad, F_n = Q^T (K u_n + g_n) is formed as
// Lam o U^_n + G^_n with U^_n = Q^T u_n carried from step to step
// (U^_{n+1} = U^_n + S when u_{n+1} = u_n + bwd(S)), which replaces the
// paper's explicit K u_n (Eq. krogstad-m) and saves a Tucker operator.
#include <cmath>
#include <cstring>
#include <cstdint>

#include "adjoint.h"
#include "engine.h"

namespace fcgle {

namespace {

double fd_g0(double alpha) { return std::tgamma(alpha + 1.0) / std::pow(std::tgamma(alpha / 2.0 + 1.0), 2); }

// D_n^alpha (Eq. Dnalpha / Eq. FD4), row-major n x n.
std::vector<double> build_D(int n, double alpha, double h, int order) {
  std::vector<double> g(n);
  g[0] = fd_g0(alpha);
  for (int k = 1; k < n; ++k) g[k] = (1.0 - (alpha + 1.0) / (alpha / 2.0 + k)) * g[k - 1];
  if (order == 4) {
    std::vector<double> gc(n);
    for (int k = 0; k < n; ++k) {
      gc[k] = 4.0 / 3.0 * g[k];
      if (k % 2 == 0) gc[k] -= (1.0 / 3.0) * g[k / 2] / std::pow(2.0, alpha);
    }
    g.swap(gc);
  }
  const double sc = -std::pow(h, -alpha);
  std::vector<double> D((size_t)n * n);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) D[(size_t)i * n + j] = sc * g[std::abs(i - j)];
  return D;
}

void check_eig(const std::vector<double>& A, const Direction& D) {
  const int n = D.n;
  double r = 0, a = 0, o = 0;
  // residual ||A Q - Q Lam||_F / ||A||_F and ||Q^T Q - I||_F, sampled on up to 64 columns
  const int stride = n > 64 ? n / 64 : 1;
  for (int j = 0; j < n; j += stride) {
    for (int i = 0; i < n; ++i) {
      double s = 0;
      for (int k = 0; k < n; ++k) s += A[(size_t)i * n + k] * D.Q[(size_t)k * n + j];
      s -= D.Q[(size_t)i * n + j] * D.lam[j];
      r += s * s;
    }
    for (int i = 0; i < n; ++i) {
      double s = 0;
      for (int k = 0; k < n; ++k) s += D.Q[(size_t)k * n + i] * D.Q[(size_t)k * n + j];
      if (i == j) s -= 1.0;
      o += s * s;
    }
  }
  for (size_t i = 0; i < A.size(); ++i) a += A[i] * A[i];
  const double frac = (double)((n + stride - 1) / stride) / n;
  if (!(std::sqrt(r / (a * frac)) <= 1e-11) || !(std::sqrt(o / frac) <= 1e-11 * std::sqrt((double)n)))
    throw NumericError("eigendecomposition residual above 1e-11");
}

uint64_t dbits(double x) {
  uint64_t u;
  std::memcpy(&u, &x, 8);
  return u;
}

template <typename T>
struct DevBuf {
  T* ptr = nullptr;
  DevBuf() = default;
  explicit DevBuf(size_t n) { FCGLE_CUDA(cudaMalloc(&ptr, n * sizeof(T))); }
  ~DevBuf() {
    if (ptr) cudaFree(ptr);
  }
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
};

}  // namespace

template <typename T>
class Engine : public EngineBase {
 public:
  static constexpr bool kF64 = sizeof(T) == 8;

  Engine(const fcgle_params& prm, cudaStream_t st) : prm_(prm), st_(st) {
    s_.d = prm.d;
    s_.P = 1;
    s_.N = 1;
    for (int mu = 0; mu < kMaxDim; ++mu) {
      s_.n[mu] = mu < prm.d ? prm.n[mu] : 1;
      s_.p[mu] = mu < prm.d ? pad4(prm.n[mu]) : 1;
      s_.P *= (size_t)s_.p[mu];
      s_.N *= (size_t)s_.n[mu];
    }
    // ---- per-direction spectral data (shared between identical directions)
    for (int mu = 0; mu < prm.d; ++mu) {
      int same = -1;
      const double h = (prm.b[mu] - prm.a[mu]) / (prm.n[mu] + 1);
      for (int o = 0; o < mu; ++o)
        if (prm.n[o] == prm.n[mu] && prm.alpha[o] == prm.alpha[mu] && dir_[o].h == h) same = o;
      if (same >= 0) {
        dir_[mu] = dir_[same];
        dir_[mu].p = s_.p[mu];
      } else {
        dir_[mu] = spectral_direction(prm, mu);
        dir_[mu].p = s_.p[mu];
      }
    }
    // ---- device copies: lam_mu (padded), mode-product matrices
    for (int mu = 0; mu < prm.d; ++mu) {
      const Direction& D = dir_[mu];
      std::vector<double> lp(D.p, 0.0);
      for (int j = 0; j < D.n; ++j) lp[j] = D.lam[j];
      lam_[mu].reset(new DevBuf<double>(D.p));
      FCGLE_CUDA(cudaMemcpy(lam_[mu]->ptr, lp.data(), D.p * sizeof(double), cudaMemcpyHostToDevice));
      // forward matrix M[i][k] = Q[k][i] (Q^T), backward M[i][k] = Q[i][k]; zero padded to p x p
      std::vector<double> Mf((size_t)D.p * D.p, 0.0), Mb((size_t)D.p * D.p, 0.0);
      for (int i = 0; i < D.n; ++i)
        for (int k = 0; k < D.n; ++k) {
          Mf[(size_t)i * D.p + k] = D.Q[(size_t)k * D.n + i];
          Mb[(size_t)i * D.p + k] = D.Q[(size_t)i * D.n + k];
        }
      mf64_[mu][0].reset(new DevBuf<double>(Mf.size()));
      mf64_[mu][1].reset(new DevBuf<double>(Mb.size()));
      FCGLE_CUDA(cudaMemcpy(mf64_[mu][0]->ptr, Mf.data(), Mf.size() * 8, cudaMemcpyHostToDevice));
      FCGLE_CUDA(cudaMemcpy(mf64_[mu][1]->ptr, Mb.data(), Mb.size() * 8, cudaMemcpyHostToDevice));
    }
    lv_.c_re = prm.nu;
    lv_.c_im = prm.eta;
    for (int mu = 0; mu < kMaxDim; ++mu) lv_.lam[mu] = mu < prm.d ? lam_[mu]->ptr : nullptr;
    gp_.gamma = prm.gamma;
    gp_.kappa = prm.kappa;
    gp_.zeta = prm.zeta;
    gp_.nsrc = 0;
    for (int k = 0; k < kMaxSrc; ++k) gp_.S[k] = nullptr;
    // ---- work buffers
    for (int i = 0; i < kNumBuf; ++i) buf_[i].reset(new DevBuf<T>(2 * s_.P));
    for (int i = 0; i < kNumBuf; ++i) FCGLE_CUDA(cudaMemsetAsync(buf_[i]->ptr, 0, 2 * s_.P * sizeof(T), st_));
    scratch_.reset(new DevBuf<double>(4));
    err_.reset(new DevBuf<int>(1));
    FCGLE_CUDA(cudaMemsetAsync(err_->ptr, 0, sizeof(int), st_));
    FCGLE_CUDA(cudaStreamSynchronize(st_));
  }


  void set_stream(cudaStream_t st) override { st_ = st; }
  size_t internal_elems() const override { return s_.P; }
  void mode_product(int mu, bool fwd, const void* X, void* Y) override {
    if (mu < 0 || mu >= s_.d) throw InvalidArg("direction must be in 0..d-1");
    mp((const T*)X, (T*)Y, mu, fwd);
  }
  size_t elem_bytes() const override { return 2 * sizeof(T); }

  void set_source(int nterms, const double* sig, const void* const* S_user) override {
    for (int k = 0; k < nterms; ++k) {
      if (!src_[k]) src_[k].reset(new DevBuf<T>(2 * s_.P));
      pack<T>(s_, (const T*)S_user[k], src_[k]->ptr, st_, launches);
      gp_.sig_re[k] = sig[2 * k];
      gp_.sig_im[k] = sig[2 * k + 1];
      gp_.S[k] = src_[k]->ptr;
    }
    for (int k = nterms; k < kMaxSrc; ++k) gp_.S[k] = nullptr;
    gp_.nsrc = nterms;
  }

  void set_coefficients(double nu, double eta, double gamma, double kappa, double zeta) override {
    FCGLE_CUDA(cudaStreamSynchronize(st_));   // cached tensors may still be in use
    prm_.nu = nu;
    prm_.eta = eta;
    prm_.gamma = gamma;
    prm_.kappa = kappa;
    prm_.zeta = zeta;
    lv_.c_re = nu;
    lv_.c_im = eta;
    gp_.gamma = gamma;
    gp_.kappa = kappa;
    gp_.zeta = zeta;
    fcache_.clear();
    ecache_.clear();
  }

  void spectral_scalars(int func, int k, double theta, int count, const double* s_host, double* out_host,
                        int) override {
    if (count <= 0) return;
    DevBuf<double> sd((size_t)count), od(2 * (size_t)count);
    FCGLE_CUDA(cudaMemcpyAsync(sd.ptr, s_host, (size_t)count * 8, cudaMemcpyHostToDevice, st_));
    const int f = (func == FCGLE_F_PHI && k == 0) ? FCGLE_F_EXP : func;
    spectral_scalars_f64(count, sd.ptr, prm_.nu, prm_.eta, f == FCGLE_F_INV ? 0 : (f == FCGLE_F_EXP ? 1 : 2), k,
                         theta, od.ptr, st_, launches);
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

  // ------------------------------------------------------------ apply_f
  void apply_f(int func, int k, double theta, const void* v, void* out) override {
    T* X = B(0);
    T* Xh = B(1);
    pack<T>(s_, (const T*)v, X, st_, launches);
    if (func == FCGLE_F_EXP || (func == FCGLE_F_PHI && k == 0)) {
      expK(theta, X, X);
    } else {
      tucker(X, Xh, true);
      scale(F(func, k, theta), Xh, Xh);
      tucker(Xh, X, false);
    }
    unpack<T>(s_, X, (T*)out, st_, launches, err_->ptr);
  }

  // ---------------------------------------------------------- schemes
  void step(int scheme, double tau, double t, void* u) override {
    T* U = B(kU);
    pack<T>(s_, (const T*)u, U, st_, launches);
    prepare(scheme, tau);
    if (needs_uhat(scheme)) tucker(U, B(kUh), true);
    one_step(scheme, tau, t);
    unpack<T>(s_, U, (T*)u, st_, launches, err_->ptr);
  }

  void integrate(int scheme, double tau, int nsteps, double t0, const void* u0, void* uT) override {
    T* U = B(kU);
    pack<T>(s_, (const T*)u0, U, st_, launches);
    run(scheme, tau, nsteps, t0);
    unpack<T>(s_, B(kU), (T*)uT, st_, launches, err_->ptr);
  }

  void begin_steps(int scheme, double tau, double t0, const void* u0) override {
    pack<T>(s_, (const T*)u0, B(kU), st_, launches);
    prepare(scheme, tau);
    rs_scheme_ = scheme;
    rs_tau_ = tau;
    rs_t0_ = t0;
    if (scheme == FCGLE_LBDF2)
      FCGLE_CUDA(cudaMemcpyAsync(B(kG), B(kU), 2 * s_.P * sizeof(T), cudaMemcpyDeviceToDevice, st_));
    if (needs_uhat(scheme)) tucker(B(kU), B(kUh), true);
  }
  void one_step(int n) override {
    const double t = rs_t0_ + n * rs_tau_;
    if (rs_scheme_ == FCGLE_LBDF2) {
      if (n == 0)
        one_step(FCGLE_LIE, rs_tau_, t);
      else
        lbdf2_step(rs_tau_, t);
    } else {
      one_step(rs_scheme_, rs_tau_, t);
    }
  }
  void end_steps(void* uT) override { unpack<T>(s_, B(kU), (T*)uT, st_, launches, err_->ptr); }
  bool time_dependent() const override { return gp_.nsrc > 0; }

  void integrate_host(int scheme, double tau, int nsteps, double t0, const void* u0, void* uT) override {
    const size_t bytes = s_.N * 2 * sizeof(T);
    if (!host_stage_) host_stage_.reset(new DevBuf<T>(2 * s_.N));
    FCGLE_CUDA(cudaMemcpyAsync(host_stage_->ptr, u0, bytes, cudaMemcpyHostToDevice, st_));
    pack<T>(s_, host_stage_->ptr, B(kU), st_, launches);
    run(scheme, tau, nsteps, t0);
    unpack<T>(s_, B(kU), host_stage_->ptr, st_, launches, err_->ptr);
    FCGLE_CUDA(cudaMemcpyAsync(uT, host_stage_->ptr, bytes, cudaMemcpyDeviceToHost, st_));
    FCGLE_CUDA(cudaStreamSynchronize(st_));
  }

  // ---- adjoint support (adjoint.h driver interface)
  Shape shape() const { return s_; }
  cudaStream_t stream() const { return st_; }
  long long& nlaunch() { return launches; }
  GParams gparams() const { return gp_; }
  LamVecs lamvecs() const { return lv_; }
  T* alloc(size_t n) {
    adj_mem_.emplace_back(new DevBuf<T>(n));
    return adj_mem_.back()->ptr;
  }
  void release_all() { adj_mem_.clear(); }
  void tuckerT(const T* X, T* Y, bool fwd) { tucker(X, Y, fwd); }
  void tuckerT_precise(const T* X, T* Y, bool fwd) { tucker(X, Y, fwd); }
  // U = bwd(Uh), K = fwd(g(t, U)); tmp: a work tensor of 2 P
  void g_roundtrip(const T* Uh, T* U, T* K, T* tmp, double t) {
    tucker(Uh, U, false);
    gcombo<T>(s_, gp_, t, U, nullptr, nullptr, 1, 0, 0, 0, 1, 0, tmp, st_, launches);
    tucker(tmp, K, true);
  }

  void adjoint(int scheme, double tau, int nsteps, double t0, const void* u0, const void* target, int ckpt,
               void* grad_u0, double* grad_params, double* loss) override {
    if (scheme != FCGLE_LAWSON_RK2) throw Unsupported("the adjoint is implemented for LAWSON_RK2");
    try {
      T* U0 = alloc(2 * s_.P);
      T* TG = alloc(2 * s_.P);
      T* GR = alloc(2 * s_.P);
      pack<T>(s_, (const T*)u0, U0, st_, launches);
      pack<T>(s_, (const T*)target, TG, st_, launches);
      adjoint_lawson_rk2<T>(*this, tau, nsteps, t0, U0, TG, ckpt, GR, grad_params, loss);
      unpack<T>(s_, GR, (T*)grad_u0, st_, launches, err_->ptr);
      FCGLE_CUDA(cudaStreamSynchronize(st_));
    } catch (...) {
      release_all();
      throw;
    }
    release_all();
  }

  double norm(const void* u) override {
    T* X = B(0);
    pack<T>(s_, (const T*)u, X, st_, launches);
    sumsq<T>(s_, X, scratch_->ptr, st_, launches);
    double h = 0.0;
    FCGLE_CUDA(cudaMemcpyAsync(&h, scratch_->ptr, sizeof(double), cudaMemcpyDeviceToHost, st_));
    FCGLE_CUDA(cudaStreamSynchronize(st_));
    double cell = 1.0;
    for (int mu = 0; mu < s_.d; ++mu) cell *= dir_[mu].h;
    return std::sqrt(cell * h);
  }

 private:
  // buffer roles
  enum { kU = 2, kUh = 3, kG = 4, kGh = 5, kFh = 6, kD2 = 7, kD3 = 8, kD4 = 9, kS = 10, kW = 11, kT0 = 12, kT1 = 13,
         kNumBuf = 14 };
  T* B(int i) { return buf_[i]->ptr; }

  static bool needs_uhat(int scheme) { return scheme == FCGLE_ETD2RK || scheme == FCGLE_KROGSTAD; }

  // ---- building blocks
  void mp(const T* X, T* Y, int mu, bool fwd) {
    const size_t R = s_.P / s_.p[mu];
    mp_f64(X, Y, mf64_[mu][fwd ? 0 : 1]->ptr, s_.p[mu], R, false, st_, launches);
  }

  // Tucker operator over directions 1..d in the rotating order; Y may equal X.
  void tucker(const T* X, T* Y, bool fwd) {
    const int d = s_.d;
    if (d == 1) {
      if (X == Y) {
        mp(X, B(kT0), 0, fwd);
        FCGLE_CUDA(cudaMemcpyAsync(Y, B(kT0), 2 * s_.P * sizeof(T), cudaMemcpyDeviceToDevice, st_));
      } else {
        mp(X, Y, 0, fwd);
      }
      return;
    }
    const T* in = X;
    for (int mu = 0; mu < d; ++mu) {
      T* out = (mu == d - 1) ? Y : B(mu % 2 == 0 ? kT0 : kT1);
      mp(in, out, mu, fwd);
      in = out;
    }
  }

  // Y = exp(theta K) X
  void expK(double theta, const T* X, T* Y) {
    if constexpr (kF64) {
      // Kronecker-product form (Eq. Neudeckerd): complex mode products with E_mu
      auto& E = Emat(theta);
      const T* in = X;
      for (int mu = 0; mu < s_.d; ++mu) {
        T* out = (mu == s_.d - 1) ? Y : B(mu % 2 == 0 ? kT0 : kT1);
        if (out == in) out = B(kW);
        mp_f64(in, out, E[mu]->ptr, s_.p[mu], s_.P / s_.p[mu], true, st_, launches);
        in = out;
      }
      if (in != Y) FCGLE_CUDA(cudaMemcpyAsync(Y, in, 2 * s_.P * sizeof(T), cudaMemcpyDeviceToDevice, st_));
    } else {
      // Tucker form (Eq. fKu_diag) with F = exp(theta lam)
      T* Xh = B(kW);
      tucker(X, Xh, true);
      scale(F(FCGLE_F_EXP, 0, theta), Xh, Xh);
      tucker(Xh, Y, false);
    }
  }

  // Y = F o X
  void scale(const T* Fp, const T* X, T* Y) {
    SpecArgs<T> a;
    a.nx = 1;
    a.nf = 1;
    a.X[0] = X;
    a.F[0] = Fp;
    a.fkind[0] = F_TENSOR;
    a.W[0][0] = 1.0;
    a.out = Y;
    spec_combo<T>(s_, lv_, a, st_, launches);
  }

  // out = X0 + X1 (physical-space stage update u_n + bwd(S))
  void add(const T* X0, const T* X1, T* out) {
    SpecArgs<T> a;
    a.nx = 2;
    a.nf = 1;
    a.X[0] = X0;
    a.X[1] = X1;
    a.fkind[0] = F_ONE;
    a.W[0][0] = a.W[0][1] = 1.0;
    a.out = out;
    spec_combo<T>(s_, lv_, a, st_, launches);
  }

  // spectral scalar tensor f(theta Lam), cached
  T* F(int func, int ell, double theta) {
    if (func == FCGLE_F_PHI && ell == 0) func = FCGLE_F_EXP;
    if (func != FCGLE_F_PHI) ell = 0;
    auto key = std::make_tuple(func, ell, dbits(theta));
    auto it = fcache_.find(key);
    if (it != fcache_.end()) return it->second->ptr;
    auto* b = new DevBuf<T>(2 * s_.P);
    fcache_[key].reset(b);
    fill_F<T>(s_, lv_, func, ell, theta, b->ptr, st_, launches);
    return b->ptr;
  }

  // E_mu = Q diag(exp(theta (nu + i eta) lam)) Q^T in real block form, cached
  std::vector<std::unique_ptr<DevBuf<double>>>& Emat(double theta) {
    auto key = dbits(theta);
    auto it = ecache_.find(key);
    if (it != ecache_.end()) return it->second;
    auto& v = ecache_[key];
    for (int mu = 0; mu < s_.d; ++mu) {
      const Direction& D = dir_[mu];
      const int n = D.n, p = D.p;
      std::vector<double> er(n), ei(n);
      for (int j = 0; j < n; ++j) {
        const double m = std::exp(theta * prm_.nu * D.lam[j]);
        er[j] = m * std::cos(theta * prm_.eta * D.lam[j]);
        ei[j] = m * std::sin(theta * prm_.eta * D.lam[j]);
      }
      std::vector<double> Bm((size_t)4 * p * p, 0.0);
      const size_t K = 2 * (size_t)p;
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
          for (int sym = 0; sym < 2; ++sym) {
            const int a = sym ? k : i, b = sym ? i : k;
            Bm[(size_t)a * K + b] = sr;           // (re out, re in)
            Bm[(size_t)a * K + p + b] = -si;      // (re out, im in)
            Bm[(size_t)(p + a) * K + b] = si;     // (im out, re in)
            Bm[(size_t)(p + a) * K + p + b] = sr; // (im out, im in)
          }
        }
      v.emplace_back(new DevBuf<double>(Bm.size()));
      FCGLE_CUDA(cudaMemcpyAsync(v.back()->ptr, Bm.data(), Bm.size() * 8, cudaMemcpyHostToDevice, st_));
      FCGLE_CUDA(cudaStreamSynchronize(st_));
    }
    return v;
  }

  // fill every cached tensor a scheme needs before its time loop
  void prepare(int scheme, double tau) {
    switch (scheme) {
      case FCGLE_LIE: F(FCGLE_F_INV, 0, tau); break;
      case FCGLE_LBDF2: F(FCGLE_F_INV, 0, tau); F(FCGLE_F_INV, 0, 2.0 * tau / 3.0); break;
      case FCGLE_LAWSON_EULER:
      case FCGLE_LAWSON_RK2:
      case FCGLE_STRANG:
        if constexpr (kF64) Emat(tau); else F(FCGLE_F_EXP, 0, tau);
        break;
      case FCGLE_ETD2RK: F(FCGLE_F_PHI, 1, tau); F(FCGLE_F_PHI, 2, tau); break;
      case FCGLE_KROGSTAD:
        F(FCGLE_F_PHI, 1, tau / 2); F(FCGLE_F_PHI, 2, tau / 2);
        F(FCGLE_F_PHI, 1, tau); F(FCGLE_F_PHI, 2, tau); F(FCGLE_F_PHI, 3, tau);
        break;
      default: throw InvalidArg("unknown scheme");
    }
  }

  void run(int scheme, double tau, int nsteps, double t0) {
    prepare(scheme, tau);
    if (nsteps == 0) return;
    double t = t0;
    if (scheme == FCGLE_LBDF2) {
      // u_prev = u_0, first step by LIE (Eq. lbdf2-v)
      FCGLE_CUDA(cudaMemcpyAsync(B(kG), B(kU), 2 * s_.P * sizeof(T), cudaMemcpyDeviceToDevice, st_));
      one_step(FCGLE_LIE, tau, t);
      t += tau;
      for (int n = 1; n < nsteps; ++n) {
        lbdf2_step(tau, t);
        t = t0 + (n + 1) * tau;
      }
      return;
    }
    if (needs_uhat(scheme)) tucker(B(kU), B(kUh), true);
    for (int n = 0; n < nsteps; ++n) {
      one_step(scheme, tau, t0 + n * tau);
    }
  }

  // one step on B(kU) (and the carried B(kUh) for ETD2RK / Krogstad)
  void one_step(int scheme, double tau, double t) {
    T* U = B(kU);
    switch (scheme) {
      case FCGLE_LIE: {
        // u_{n+1} = (I - tau K)^{-1} (u_n + tau g(t_n, u_n))
        T* V = B(kW);
        gcombo<T>(s_, gp_, t, U, nullptr, nullptr, 1, 0, 1, 0, tau, 0, V, st_, launches);
        tucker(V, V, true);
        scale(F(FCGLE_F_INV, 0, tau), V, V);
        tucker(V, U, false);
        break;
      }
      case FCGLE_LAWSON_EULER: {
        T* V = B(kS);
        gcombo<T>(s_, gp_, t, U, nullptr, nullptr, 1, 0, 1, 0, tau, 0, V, st_, launches);
        expK(tau, V, U);
        break;
      }
      case FCGLE_LAWSON_RK2: {
        T* A = B(kG);
        T* Bv = B(kS);
        gcombo<T>(s_, gp_, t, U, nullptr, nullptr, 1, 0, 1, 0, tau, 0, A, st_, launches);
        gcombo<T>(s_, gp_, t, U, nullptr, nullptr, 1, 0, 1, 0, tau / 2, 0, Bv, st_, launches);
        expK(tau, A, A);
        expK(tau, Bv, Bv);
        // u_{n+1} = E(u + tau/2 k1) + tau/2 g(t + tau, E(u + tau k1))
        gcombo<T>(s_, gp_, t + tau, A, Bv, nullptr, 1, 0, 0, 1, tau / 2, 0, U, st_, launches);
        break;
      }
      case FCGLE_STRANG: {
        exact_flow<T>(s_, prm_.gamma, prm_.kappa, prm_.zeta, tau / 2, U, U, st_, launches);
        expK(tau, U, U);
        exact_flow<T>(s_, prm_.gamma, prm_.kappa, prm_.zeta, tau / 2, U, U, st_, launches);
        break;
      }
      case FCGLE_ETD2RK: etd2rk_step(tau, t); break;
      case FCGLE_KROGSTAD: krogstad_step(tau, t); break;
      default: throw InvalidArg("scheme not valid for a single step");
    }
  }

  // F^ = Lam o U^ + G^
  void form_Fhat(const T* Uh, const T* Gh, T* Fh) {
    SpecArgs<T> a;
    a.nx = 2;
    a.nf = 2;
    a.X[0] = Uh;
    a.X[1] = Gh;
    a.fkind[0] = F_LAM;
    a.W[0][0] = 1.0;
    a.fkind[1] = F_ONE;
    a.W[1][1] = 1.0;
    a.out = Fh;
    spec_combo<T>(s_, lv_, a, st_, launches);
  }

  void etd2rk_step(double tau, double t) {
    T *U = B(kU), *Uh = B(kUh), *G = B(kG), *Gh = B(kGh), *Fh = B(kFh), *S = B(kS), *W = B(kW), *D = B(kD2);
    gcombo<T>(s_, gp_, t, U, nullptr, nullptr, 1, 0, 0, 0, 1, 0, G, st_, launches);   // G = g(t_n, u_n)
    tucker(G, Gh, true);
    form_Fhat(Uh, Gh, Fh);
    // S = tau P1 o F^ ;  a^ = U^ + S ;  a = u + bwd(S)
    SpecArgs<T> a;
    a.nx = 1; a.nf = 1; a.X[0] = Fh; a.F[0] = F(FCGLE_F_PHI, 1, tau); a.fkind[0] = F_TENSOR; a.W[0][0] = tau;
    a.out = S; a.base = Uh; a.out2 = Uh;
    spec_combo<T>(s_, lv_, a, st_, launches);
    tucker(S, W, false);
    add(U, W, U);
    // D^ = fwd(g(t + tau, a) - G)
    gcombo<T>(s_, gp_, t + tau, U, nullptr, G, 1, 0, 0, 0, 1, -1, D, st_, launches);
    tucker(D, D, true);
    SpecArgs<T> b;
    b.nx = 1; b.nf = 1; b.X[0] = D; b.F[0] = F(FCGLE_F_PHI, 2, tau); b.fkind[0] = F_TENSOR; b.W[0][0] = tau;
    b.out = S; b.base = Uh; b.out2 = Uh;
    spec_combo<T>(s_, lv_, b, st_, launches);
    tucker(S, W, false);
    add(U, W, U);
  }

  void krogstad_step(double tau, double t) {
    T *U = B(kU), *Uh = B(kUh), *G = B(kG), *Fh = B(kFh), *S = B(kS), *W = B(kW);
    T *D2 = B(kD2), *D3 = B(kD3), *D4 = B(kD4), *Us = B(kGh);
    T* P1h = F(FCGLE_F_PHI, 1, tau / 2);
    T* P2h = F(FCGLE_F_PHI, 2, tau / 2);
    T* P1 = F(FCGLE_F_PHI, 1, tau);
    T* P2 = F(FCGLE_F_PHI, 2, tau);
    T* P3 = F(FCGLE_F_PHI, 3, tau);
    // G = g(t_n, u_n), F^ = Lam o U^ + fwd(G)
    gcombo<T>(s_, gp_, t, U, nullptr, nullptr, 1, 0, 0, 0, 1, 0, G, st_, launches);
    tucker(G, Fh, true);
    form_Fhat(Uh, Fh, Fh);
    auto stage = [&](const SpecArgs<T>& a, double tc, T* Dh) {
      // S = combination; U_s = u_n + bwd(S); D^ = fwd(g(tc, U_s) - G)
      spec_combo<T>(s_, lv_, a, st_, launches);
      tucker(S, W, false);
      add(U, W, Us);
      gcombo<T>(s_, gp_, tc, Us, nullptr, G, 1, 0, 0, 0, 1, -1, Dh, st_, launches);
      tucker(Dh, Dh, true);
    };
    {  // U_n2 = u_n + tau/2 phi_1(tau/2 K) f_n
      SpecArgs<T> a;
      a.nx = 1; a.nf = 1; a.X[0] = Fh; a.F[0] = P1h; a.fkind[0] = F_TENSOR; a.W[0][0] = tau / 2; a.out = S;
      stage(a, t + tau / 2, D2);
    }
    {  // U_n3 = u_n + tau (1/2 phi_1(tau/2 K) f_n + phi_2(tau/2 K) d_n2)
      SpecArgs<T> a;
      a.nx = 2; a.nf = 2; a.X[0] = Fh; a.X[1] = D2;
      a.F[0] = P1h; a.fkind[0] = F_TENSOR; a.W[0][0] = tau / 2;
      a.F[1] = P2h; a.fkind[1] = F_TENSOR; a.W[1][1] = tau;
      a.out = S;
      stage(a, t + tau / 2, D3);
    }
    {  // U_n4 = u_n + tau (phi_1(tau K) f_n + 2 phi_2(tau K) d_n3)
      SpecArgs<T> a;
      a.nx = 2; a.nf = 2; a.X[0] = Fh; a.X[1] = D3;
      a.F[0] = P1; a.fkind[0] = F_TENSOR; a.W[0][0] = tau;
      a.F[1] = P2; a.fkind[1] = F_TENSOR; a.W[1][1] = 2 * tau;
      a.out = S;
      stage(a, t + tau, D4);
    }
    {  // u_{n+1} = u_n + tau (P1 f + P2 (2 d2 + 2 d3 - d4) + P3 (-4 d2 - 4 d3 + 4 d4))
      SpecArgs<T> a;
      a.nx = 4; a.nf = 3; a.X[0] = Fh; a.X[1] = D2; a.X[2] = D3; a.X[3] = D4;
      a.F[0] = P1; a.fkind[0] = F_TENSOR; a.W[0][0] = tau;
      a.F[1] = P2; a.fkind[1] = F_TENSOR; a.W[1][1] = 2 * tau; a.W[1][2] = 2 * tau; a.W[1][3] = -tau;
      a.F[2] = P3; a.fkind[2] = F_TENSOR; a.W[2][1] = -4 * tau; a.W[2][2] = -4 * tau; a.W[2][3] = 4 * tau;
      a.out = S; a.base = Uh; a.out2 = Uh;
      spec_combo<T>(s_, lv_, a, st_, launches);
      tucker(S, W, false);
      add(U, W, U);
    }
  }

  void lbdf2_step(double tau, double t) {
    // Eq. lbdf2-v: rhs = 4/3 u_n - 1/3 u_{n-1} + 2 tau/3 g(t_{n+1}, 2 u_n - u_{n-1})
    T *U = B(kU), *Up = B(kG), *V = B(kW);
    gcombo<T>(s_, gp_, t + tau, U, Up, nullptr, 2, -1, 4.0 / 3.0, -1.0 / 3.0, 2.0 * tau / 3.0, 0, V, st_, launches);
    FCGLE_CUDA(cudaMemcpyAsync(Up, U, 2 * s_.P * sizeof(T), cudaMemcpyDeviceToDevice, st_));
    tucker(V, V, true);
    scale(F(FCGLE_F_INV, 0, 2.0 * tau / 3.0), V, V);
    tucker(V, U, false);
  }

  fcgle_params prm_;
  cudaStream_t st_;
  Shape s_;
  int rs_scheme_ = 0;
  double rs_tau_ = 0.0, rs_t0_ = 0.0;
  Direction dir_[kMaxDim];
  std::unique_ptr<DevBuf<double>> lam_[kMaxDim];
  std::unique_ptr<DevBuf<double>> mf64_[kMaxDim][2];
  LamVecs lv_{};
  GParams gp_{};
  std::unique_ptr<DevBuf<T>> buf_[kNumBuf];
  std::unique_ptr<DevBuf<T>> src_[kMaxSrc];
  std::unique_ptr<DevBuf<T>> host_stage_;
  std::unique_ptr<DevBuf<double>> scratch_;
  std::unique_ptr<DevBuf<int>> err_;
  std::map<std::tuple<int, int, uint64_t>, std::unique_ptr<DevBuf<T>>> fcache_;
  std::map<uint64_t, std::vector<std::unique_ptr<DevBuf<double>>>> ecache_;
  std::vector<std::unique_ptr<DevBuf<T>>> adj_mem_;
};

Direction spectral_direction(const fcgle_params& prm, int mu) {
  Direction D;
  D.n = prm.n[mu];
  D.p = D.n;
  D.h = (prm.b[mu] - prm.a[mu]) / (prm.n[mu] + 1);
  std::vector<double> A = build_D(D.n, prm.alpha[mu], D.h, prm.fd_order);
  D.Q.resize((size_t)D.n * D.n);
  D.lam.resize(D.n);
  if (!sym_eig(D.n, A.data(), D.lam.data(), D.Q.data())) throw NumericError("eigendecomposition did not converge");
  check_eig(A, D);
  return D;
}

std::unique_ptr<EngineBase> make_engine(const fcgle_params& prm, cudaStream_t st) {
  if (prm.precision == FCGLE_FP64) return std::unique_ptr<EngineBase>(new Engine<double>(prm, st));
  if (prm.precision == FCGLE_BF16X3) return make_engine_b3(prm, st);
  throw InvalidArg("unknown precision");
}

}  // namespace fcgle
