// FP64 symmetric eigendecomposition on the host, for the per-direction
// matrices D_mu = Q_mu Lam_mu Q_mu^T (paper Eq. diag; the paper also
// diagonalises on the CPU and ships the factors to the GPU once, Sec. 4.2).
//
// Method (textbook, Golub & Van Loan Sec. 8.3):
//  1. Householder reduction A = U T U^T, T symmetric tridiagonal.
//  2. Implicit symmetric QR sweeps with the Wilkinson shift on T, deflating
//     negligible off-diagonals; each sweep is a sequence of Givens
//     rotations that is recorded and, at the end, applied to U in parallel
//     over blocks of rows (Z = U * G_1 * G_2 * ...).
#include <algorithm>
#include <cmath>
#include <numeric>
#include <thread>
#include <vector>

#include "common.h"

namespace fcgle {

namespace {

struct Rot {
  int k;
  double c, s;
};

// Applies the recorded rotations to rows [r0, r1) of Z (row-major n x n):
// Z[:, k] <- c Z[:, k] + s Z[:, k+1];  Z[:, k+1] <- -s Z[:, k] + c Z[:, k+1].
void apply_rotations(int n, double* Z, const std::vector<Rot>& rots, int r0, int r1) {
  constexpr int B = 8;
  std::vector<double> buf((size_t)n * B);
  for (int rb = r0; rb < r1; rb += B) {
    int nb = std::min(B, r1 - rb);
    for (int j = 0; j < n; ++j)
      for (int i = 0; i < B; ++i) buf[(size_t)j * B + i] = i < nb ? Z[(size_t)(rb + i) * n + j] : 0.0;
    for (const Rot& g : rots) {
      double* a = &buf[(size_t)g.k * B];
      double* b = a + B;
      for (int i = 0; i < B; ++i) {
        double x = a[i], y = b[i];
        a[i] = g.c * x + g.s * y;
        b[i] = -g.s * x + g.c * y;
      }
    }
    for (int i = 0; i < nb; ++i)
      for (int j = 0; j < n; ++j) Z[(size_t)(rb + i) * n + j] = buf[(size_t)j * B + i];
  }
}

}  // namespace

bool sym_eig(int n, const double* Ain, double* w, double* Zout) {
  std::vector<double> A(Ain, Ain + (size_t)n * n);
  std::vector<double> d(n), e(std::max(n - 1, 1), 0.0);
  std::vector<double> V((size_t)n * n, 0.0);   // Householder vectors, row k = v_k (entries k+1..n-1)
  std::vector<double> beta(n, 0.0);
  std::vector<double> p(n), wv(n);

  // ---- 1. Householder tridiagonalisation
  for (int k = 0; k + 2 < n; ++k) {
    const int m = n - k - 1;               // length of x = A[k+1.., k]
    double* v = &V[(size_t)k * n + k + 1];
    double xnorm = 0.0;
    for (int i = 0; i < m; ++i) {
      double x = A[(size_t)(k + 1 + i) * n + k];
      v[i] = x;
      xnorm += x * x;
    }
    xnorm = std::sqrt(xnorm);
    double tail = xnorm * xnorm - v[0] * v[0];
    if (xnorm == 0.0 || tail <= 0.0) {   // already reduced
      e[k] = v[0];
      beta[k] = 0.0;
      continue;
    }
    double alpha = v[0] > 0 ? -xnorm : xnorm;      // H x = alpha e_1
    v[0] -= alpha;
    double vtv = 0.0;
    for (int i = 0; i < m; ++i) vtv += v[i] * v[i];
    double bt = 2.0 / vtv;
    beta[k] = bt;
    e[k] = alpha;
    // p = bt * B v with B = A[k+1.., k+1..]
    for (int i = 0; i < m; ++i) {
      const double* row = &A[(size_t)(k + 1 + i) * n + k + 1];
      double acc = 0.0;
      for (int j = 0; j < m; ++j) acc += row[j] * v[j];
      p[i] = bt * acc;
    }
    double ptv = 0.0;
    for (int i = 0; i < m; ++i) ptv += p[i] * v[i];
    const double K = 0.5 * bt * ptv;
    for (int i = 0; i < m; ++i) wv[i] = p[i] - K * v[i];
    // B <- B - v w^T - w v^T
    for (int i = 0; i < m; ++i) {
      double* row = &A[(size_t)(k + 1 + i) * n + k + 1];
      const double vi = v[i], wi = wv[i];
      for (int j = 0; j < m; ++j) row[j] -= vi * wv[j] + wi * v[j];
    }
  }
  for (int k = 0; k < n; ++k) d[k] = A[(size_t)k * n + k];
  if (n >= 2) e[n - 2] = A[(size_t)(n - 1) * n + n - 2];

  // U = H_0 H_1 ... H_{n-3}, accumulated backwards into Zout (row-major).
  double* Z = Zout;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) Z[(size_t)i * n + j] = (i == j) ? 1.0 : 0.0;
  std::vector<double> t(n);
  for (int k = n - 3; k >= 0; --k) {
    if (beta[k] == 0.0) continue;
    const int m = n - k - 1;
    const double* v = &V[(size_t)k * n + k + 1];
    // Z_sub = Z[k+1.., k+1..];  Z_sub <- Z_sub - beta v (v^T Z_sub)
    std::fill(t.begin(), t.begin() + m, 0.0);
    for (int i = 0; i < m; ++i) {
      const double* row = &Z[(size_t)(k + 1 + i) * n + k + 1];
      const double vi = v[i];
      for (int j = 0; j < m; ++j) t[j] += vi * row[j];
    }
    for (int i = 0; i < m; ++i) {
      double* row = &Z[(size_t)(k + 1 + i) * n + k + 1];
      const double f = beta[k] * v[i];
      for (int j = 0; j < m; ++j) row[j] -= f * t[j];
    }
  }

  // ---- 2. implicit QR with Wilkinson shift on (d, e)
  std::vector<Rot> rots;
  rots.reserve((size_t)n * 8);
  const double eps = 2.220446049250313e-16;
  long long iters = 0;
  const long long max_iters = 60LL * n + 100;
  int m = n - 1;
  while (m > 0) {
    for (int i = 0; i < m; ++i)
      if (std::fabs(e[i]) <= eps * (std::fabs(d[i]) + std::fabs(d[i + 1]))) e[i] = 0.0;
    while (m > 0 && e[m - 1] == 0.0) --m;
    if (m == 0) break;
    int l = m - 1;
    while (l > 0 && e[l - 1] != 0.0) --l;
    if (++iters > max_iters) return false;
    // Wilkinson shift from the trailing 2 x 2 block of T[l..m]
    const double delta = 0.5 * (d[m - 1] - d[m]);
    const double em = e[m - 1];
    const double sgn = delta >= 0.0 ? 1.0 : -1.0;
    const double mu = d[m] - em * em / (delta + sgn * std::hypot(delta, em));
    double x = d[l] - mu, z = e[l];
    double bulge = 0.0;
    for (int k = l; k < m; ++k) {
      // rotation G = [[c, -s], [s, c]] on coordinates (k, k+1)
      double r = std::hypot(x, z);
      double c = 1.0, s = 0.0;
      if (r != 0.0) {
        c = x / r;
        s = z / r;
      }
      if (k > l) e[k - 1] = r;    // bulge at (k-1, k+1) annihilated
      const double a = d[k], b = e[k], a2 = d[k + 1];
      d[k] = c * c * a + 2.0 * c * s * b + s * s * a2;
      d[k + 1] = s * s * a - 2.0 * c * s * b + c * c * a2;
      e[k] = c * s * (a2 - a) + (c * c - s * s) * b;
      if (k + 1 < m) {
        const double b2 = e[k + 1];
        bulge = s * b2;
        e[k + 1] = c * b2;
        x = e[k];
        z = bulge;
      }
      rots.push_back({k, c, s});
    }
  }

  // ---- apply the rotations to U in parallel row blocks
  unsigned hw = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
  int nthreads = (int)std::min<unsigned>(hw, (unsigned)std::max(1, n / 32));
  if (nthreads <= 1 || rots.size() < 1000) {
    apply_rotations(n, Z, rots, 0, n);
  } else {
    std::vector<std::thread> th;
    int chunk = ((n + nthreads - 1) / nthreads + 7) / 8 * 8;
    for (int t0 = 0; t0 < n; t0 += chunk)
      th.emplace_back(apply_rotations, n, Z, std::cref(rots), t0, std::min(n, t0 + chunk));
    for (auto& x : th) x.join();
  }

  // ---- sort ascending
  std::vector<int> idx(n);
  std::iota(idx.begin(), idx.end(), 0);
  std::sort(idx.begin(), idx.end(), [&](int a, int b) { return d[a] < d[b]; });
  std::vector<double> Zs((size_t)n * n);
  for (int j = 0; j < n; ++j) {
    w[j] = d[idx[j]];
    for (int i = 0; i < n; ++i) Zs[(size_t)i * n + j] = Z[(size_t)i * n + idx[j]];
  }
  std::copy(Zs.begin(), Zs.end(), Z);
  return true;
}

}  // namespace fcgle
