// Internal declarations of the FCGLE native library (not part of the C ABI).
//
// Internal tensor layout ("planar padded"): a complex tensor of logical
// shape (n_d, ..., n_1) is stored as two real planes (re, then im), each of
// P = p_1 * ... * p_d elements, p_mu = n_mu rounded up to a multiple of 4 so
// that every row is 16-byte aligned.  Padding entries are exactly zero and
// every kernel keeps them zero.  Within a plane the order is the paper's vec
// order (j_1 fastest, Eq. indexj) on the padded extents ("standard order").
//
// Mode products use a rotating order: a mode product always contracts the
// fastest index and writes its output index as the slowest one, so after
// the d mode products of a Tucker operator (directions 1, 2, .., d) the
// tensor is back in standard order.  Every mode product is then the same
// GEMM:  Y[c][i][r] = sum_k M[i][k] X[c][r][k]  (r = all other indices).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>

#include <string>

namespace fcgle {

constexpr int kMaxDim = 3;
constexpr int kMaxSrc = 4;
// Device error word codes: 1..99 name the bounded wait that gave up (a
// timeout); kErrNonFinite marks a NaN or Inf found in a result state.
constexpr int kErrNonFinite = 100;

struct Shape {
  int d = 0;
  int n[kMaxDim] = {1, 1, 1};   // interior points per direction
  int p[kMaxDim] = {1, 1, 1};   // padded extents (multiple of 4)
  size_t P = 0;                 // prod p  (elements per plane)
  size_t N = 0;                 // prod n  (complex elements of a user tensor)
};

inline int pad4(int n) { return (n + 3) & ~3; }

// ---------------------------------------------------------------- errors
struct CudaError {
  cudaError_t err;
  std::string where;
};
void throw_cuda(cudaError_t e, const char* where);
#define FCGLE_CUDA(call)                                    \
  do {                                                      \
    cudaError_t e__ = (call);                               \
    if (e__ != cudaSuccess) ::fcgle::throw_cuda(e__, #call); \
  } while (0)
#define FCGLE_LAUNCHED(ctr)                                         \
  do {                                                              \
    ++(ctr);                                                        \
    cudaError_t e__ = cudaGetLastError();                           \
    if (e__ != cudaSuccess) ::fcgle::throw_cuda(e__, "kernel launch"); \
  } while (0)

// ------------------------------------------------------- pointwise kernels
// Layout conversion between the user layout (interleaved complex, dense,
// vec order) and the internal planar padded layout.
template <typename T>
void pack(const Shape& s, const T* user, T* internal, cudaStream_t st, long long& nl);
// With `nonfinite` set, a NaN or Inf among the unpacked values records
// kErrNonFinite in that device error word (unless it already holds a code).
template <typename T>
void unpack(const Shape& s, const T* internal, T* user, cudaStream_t st, long long& nl, int* nonfinite = nullptr);

// g(t, u) = gamma u - (kappa + i zeta)|u|^2 u + sum_k exp(sigma_k t) S_k.
struct GParams {
  double gamma, kappa, zeta;
  int nsrc;
  double sig_re[kMaxSrc], sig_im[kMaxSrc];
  const void* S[kMaxSrc];   // internal-layout tensors of the handle's type
};

// out = a0 X0 + a1 X1 + b g(t, c0 X0 + c1 X1) + e X2   (X1, X2 may be null)
template <typename T>
void gcombo(const Shape& s, const GParams& gp, double t, const T* X0, const T* X1, const T* X2,
            double c0, double c1, double a0, double a1, double b, double e, T* out,
            cudaStream_t st, long long& nl);

// Spectral-space combination  out = sum_f F_f o (sum_x W[f][x] X_x),
// F_f one of: a stored complex tensor, the identity, or Lam (the
// eigenvalues of K, computed from the lam_mu vectors).  If base != null, also
// out2 = base + out.
enum FKind { F_TENSOR = 0, F_ONE = 1, F_LAM = 2 };
template <typename T>
struct SpecArgs {
  int nx = 0, nf = 0;
  const T* X[4] = {nullptr, nullptr, nullptr, nullptr};
  const T* F[4] = {nullptr, nullptr, nullptr, nullptr};
  int fkind[4] = {F_ONE, F_ONE, F_ONE, F_ONE};
  double W[4][4] = {};
  T* out = nullptr;
  const T* base = nullptr;
  T* out2 = nullptr;
};
struct LamVecs {
  const double* lam[kMaxDim];   // device, padded with zeros
  double c_re, c_im;            // nu + i eta
};
template <typename T>
void spec_combo(const Shape& s, const LamVecs& lv, const SpecArgs<T>& a, cudaStream_t st, long long& nl);

// F = f(theta (nu + i eta) sum_mu lam_mu) for f in {1/(1-z), e^z, phi_ell},
// evaluated in FP64 (phi_ell by its power series for |z| < 1, by the
// recurrence of Eq. phi otherwise), stored as T; zero on the padding.
template <typename T>
void fill_F(const Shape& s, const LamVecs& lv, int func, int ell, double theta, T* F,
            cudaStream_t st, long long& nl);

// The same FP64 evaluation on a device list of real eigenvalue sums s_j:
// out[2 j] + i out[2 j + 1] = f(theta (c_re + i c_im) s_j).
void spectral_scalars_f64(int n, const double* s_dev, double c_re, double c_im, int func, int ell, double theta,
                          double* out_dev, cudaStream_t st, long long& nl);

// Exact flow of w' = gamma w - (kappa + i zeta)|w|^2 w over time t (Sec. 4).
template <typename T>
void exact_flow(const Shape& s, double gamma, double kappa, double zeta, double t, const T* X, T* Y,
                cudaStream_t st, long long& nl);

// sum |X|^2 over the tensor, FP64 accumulation, written to a device double.
template <typename T>
void sumsq(const Shape& s, const T* X, double* out_dev, cudaStream_t st, long long& nl);

// ------------------------------------------------------------ mode products
// FP64, real matrix:    Y[c][i][r] = sum_k M[i][k] X[c][r][k], M p x p.
// FP64, complex matrix: Y[c'][i][r] = sum_{c,k} B[(c',i)][(c,k)] X[c][r][k], B 2p x 2p.
void mp_f64(const double* X, double* Y, const double* M, int p, size_t R, bool cplx,
            cudaStream_t st, long long& nl);
// FP32 real mu-mode product (same layout and kernel as mp_f64, REAL mode)
void mp_f32(const float* X, float* Y, const float* M, int p, size_t R, cudaStream_t st, long long& nl);

// ------------------------------------------------------------ host setup
// FP64 symmetric eigendecomposition A = Z diag(w) Z^T (A row-major n x n).
// Z row-major, column j = eigenvector of w[j]; w ascending.  Returns false if
// the QL iteration does not converge.
bool sym_eig(int n, const double* A, double* w, double* Z);

}  // namespace fcgle
