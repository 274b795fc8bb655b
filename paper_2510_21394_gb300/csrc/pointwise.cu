// Pointwise kernels of the FCGLE step (paper Sec. 4.2: "CUDA kernels for
// massive parallelization" of the nonlinearity, the Hadamard products with
// the spectral scalar tensors and the stage combinations).
//
// All kernels work on the internal planar padded layout (common.h): element
// q of plane 0 is the real part, element P + q of plane 1 the imaginary part.
// Grid-stride loops; each thread handles 4 consecutive elements so that
// every global access is a 16-byte (float) or 32-byte (double) vector.
#include <cmath>

#include "common.h"

namespace fcgle {

namespace {

inline int grid_for(size_t work, int block) {
  size_t g = (work + block - 1) / block;
  static const int sms = [] {   // thread-safe one-time initialisation
    int dev = 0, m = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&m, cudaDevAttrMultiProcessorCount, dev);
    return m > 0 ? m : 132;
  }();
  size_t cap = (size_t)sms * 16;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (int)g;
}

struct alignas(16) F4 {
  float x, y, z, w;
};
struct alignas(32) D4 {
  double x, y, z, w;
};
template <typename T>
struct Vec4;
template <>
struct Vec4<float> {
  using type = F4;
};
template <>
struct Vec4<double> {
  using type = D4;
};

template <typename T>
__device__ __forceinline__ void ld4(const T* p, T (&v)[4]) {
  using V = typename Vec4<T>::type;
  V x = *reinterpret_cast<const V*>(p);
  v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w;
}
template <typename T>
__device__ __forceinline__ void st4(T* p, const T (&v)[4]) {
  using V = typename Vec4<T>::type;
  V x;
  x.x = v[0]; x.y = v[1]; x.z = v[2]; x.w = v[3];
  *reinterpret_cast<V*>(p) = x;
}

// ----------------------------------------------------------------- pack
// One thread per 4 consecutive internal elements of a row of direction 1 (all
// P of them, padding included: p_1 is a multiple of 4), so that the index
// arithmetic is one division per 4 elements and the planar stores are 4-wide.
// Row rho = j_2 + p_2 j_3 of the internal layout holds user row
// (j_2 + n_2 j_3) when j_2 < n_2 and j_3 < n_3.
struct RowMap {
  size_t user_row;   // first user element of the row (valid rows)
  bool valid;
};
__device__ __forceinline__ RowMap row_map(const Shape& s, size_t rho) {
  RowMap m{0, true};
  if (s.d >= 2) {
    const int j2 = (int)(rho % (size_t)s.p[1]);
    const int j3 = (int)(rho / (size_t)s.p[1]);
    m.valid = j2 < s.n[1] && j3 < s.n[2];
    m.user_row = ((size_t)j2 + (size_t)s.n[1] * (size_t)j3) * (size_t)s.n[0];
  }
  return m;
}

template <typename T>
__global__ void pack_kernel(Shape s, const T* __restrict__ user, T* __restrict__ X) {
  const size_t P = s.P, quads_per_row = (size_t)s.p[0] / 4, nq = P / 4;
  const int n1 = s.n[0];
  for (size_t q4 = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q4 < nq; q4 += (size_t)gridDim.x * blockDim.x) {
    const size_t rho = q4 / quads_per_row;
    const int j1 = (int)(q4 - rho * quads_per_row) * 4;
    const RowMap m = row_map(s, rho);
    T re[4] = {0, 0, 0, 0}, im[4] = {0, 0, 0, 0};
    if (m.valid) {
      const T* src = user + 2 * (m.user_row + (size_t)j1);
      if (j1 + 4 <= n1 && (reinterpret_cast<uintptr_t>(src) & 15) == 0) {
        if constexpr (sizeof(T) == 4) {
          const float4 a = reinterpret_cast<const float4*>(src)[0], b = reinterpret_cast<const float4*>(src)[1];
          re[0] = a.x; im[0] = a.y; re[1] = a.z; im[1] = a.w;
          re[2] = b.x; im[2] = b.y; re[3] = b.z; im[3] = b.w;
        } else {
#pragma unroll
          for (int v = 0; v < 4; ++v) {
            const double2 a = reinterpret_cast<const double2*>(src)[v];
            re[v] = a.x;
            im[v] = a.y;
          }
        }
      } else {
#pragma unroll
        for (int v = 0; v < 4; ++v)
          if (j1 + v < n1) {
            re[v] = src[2 * v];
            im[v] = src[2 * v + 1];
          }
      }
    }
    st4<T>(X + 4 * q4, re);
    st4<T>(X + P + 4 * q4, im);
  }
}

template <typename T>
__global__ void unpack_kernel(Shape s, const T* __restrict__ X, T* __restrict__ user, int* __restrict__ nonfinite) {
  const size_t P = s.P, quads_per_row = (size_t)s.p[0] / 4, nq = P / 4;
  const int n1 = s.n[0];
  bool bad = false;
  for (size_t q4 = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q4 < nq; q4 += (size_t)gridDim.x * blockDim.x) {
    const size_t rho = q4 / quads_per_row;
    const int j1 = (int)(q4 - rho * quads_per_row) * 4;
    const RowMap m = row_map(s, rho);
    if (!m.valid || j1 >= n1) continue;
    T re[4], im[4];
    ld4<T>(X + 4 * q4, re);
    ld4<T>(X + P + 4 * q4, im);
    T* dst = user + 2 * (m.user_row + (size_t)j1);
#pragma unroll
    for (int v = 0; v < 4; ++v) bad |= (j1 + v < n1) && !(isfinite(re[v]) && isfinite(im[v]));
    if (j1 + 4 <= n1 && (reinterpret_cast<uintptr_t>(dst) & 15) == 0) {
      // 4 whole complex values, 16-byte aligned: vector stores of (re, im) pairs
      if constexpr (sizeof(T) == 4) {
        reinterpret_cast<float4*>(dst)[0] = make_float4(re[0], im[0], re[1], im[1]);
        reinterpret_cast<float4*>(dst)[1] = make_float4(re[2], im[2], re[3], im[3]);
      } else {
#pragma unroll
        for (int v = 0; v < 4; ++v) reinterpret_cast<double2*>(dst)[v] = make_double2(re[v], im[v]);
      }
    } else {
#pragma unroll
      for (int v = 0; v < 4; ++v)
        if (j1 + v < n1) {
          dst[2 * v] = re[v];
          dst[2 * v + 1] = im[v];
        }
    }
  }
  // a non-finite entry is recorded unless an earlier device error is already there
  if (bad && nonfinite) atomicCAS(nonfinite, 0, kErrNonFinite);
}

// ------------------------------------------------------------- g(t, u)
struct GDev {
  double gamma, kappa, zeta;
  int nsrc;
  double e_re[kMaxSrc], e_im[kMaxSrc];   // exp(sigma_k t), evaluated on the host in FP64
  const void* S[kMaxSrc];
};

template <typename T>
__global__ void gcombo_kernel(size_t P, GDev g, const T* __restrict__ X0, const T* __restrict__ X1,
                              const T* __restrict__ X2, double c0, double c1, double a0, double a1, double b,
                              double e, T* __restrict__ out) {
  const size_t nv = P / 4;
  for (size_t v = blockIdx.x * (size_t)blockDim.x + threadIdx.x; v < nv; v += (size_t)gridDim.x * blockDim.x) {
    const size_t q = v * 4;
    T x0r[4], x0i[4], x1r[4] = {0, 0, 0, 0}, x1i[4] = {0, 0, 0, 0}, x2r[4] = {0, 0, 0, 0}, x2i[4] = {0, 0, 0, 0};
    ld4(X0 + q, x0r);
    ld4(X0 + P + q, x0i);
    if (X1) { ld4(X1 + q, x1r); ld4(X1 + P + q, x1i); }
    if (X2) { ld4(X2 + q, x2r); ld4(X2 + P + q, x2i); }
    T src_r[4] = {0, 0, 0, 0}, src_i[4] = {0, 0, 0, 0};
    for (int k = 0; k < g.nsrc; ++k) {
      const T* S = reinterpret_cast<const T*>(g.S[k]);
      T sr[4], si[4];
      ld4(S + q, sr);
      ld4(S + P + q, si);
      const T er = (T)g.e_re[k], ei = (T)g.e_im[k];
#pragma unroll
      for (int l = 0; l < 4; ++l) {
        src_r[l] += er * sr[l] - ei * si[l];
        src_i[l] += er * si[l] + ei * sr[l];
      }
    }
    T o_r[4], o_i[4];
#pragma unroll
    for (int l = 0; l < 4; ++l) {
      const T ur = (T)c0 * x0r[l] + (T)c1 * x1r[l];
      const T ui = (T)c0 * x0i[l] + (T)c1 * x1i[l];
      const T m2 = ur * ur + ui * ui;
      // gamma u - (kappa + i zeta) |u|^2 u + s
      const T gr = (T)g.gamma * ur - m2 * ((T)g.kappa * ur - (T)g.zeta * ui) + src_r[l];
      const T gi = (T)g.gamma * ui - m2 * ((T)g.kappa * ui + (T)g.zeta * ur) + src_i[l];
      o_r[l] = (T)a0 * x0r[l] + (T)a1 * x1r[l] + (T)b * gr + (T)e * x2r[l];
      o_i[l] = (T)a0 * x0i[l] + (T)a1 * x1i[l] + (T)b * gi + (T)e * x2i[l];
    }
    st4(out + q, o_r);
    st4(out + P + q, o_i);
  }
}

// ------------------------------------------------------ spectral combos
struct LamDev {
  const double* lam[kMaxDim];
  int p[kMaxDim];
  int d;
  double c_re, c_im;
};

__device__ __forceinline__ void lam_at(const LamDev& L, size_t q, double& re, double& im) {
  double s = 0.0;
  size_t rem = q;
  for (int mu = 0; mu < L.d; ++mu) {
    int j = (int)(rem % L.p[mu]);
    rem /= L.p[mu];
    s += L.lam[mu][j];
  }
  re = L.c_re * s;
  im = L.c_im * s;
}

template <typename T>
struct SpecDev {
  int nx, nf;
  const T* X[4];
  const T* F[4];
  int fkind[4];
  double W[4][4];
  T* out;
  const T* base;
  T* out2;
};

template <typename T>
__global__ void spec_kernel(size_t P, LamDev L, SpecDev<T> a) {
  const size_t nv = P / 4;
  for (size_t v = blockIdx.x * (size_t)blockDim.x + threadIdx.x; v < nv; v += (size_t)gridDim.x * blockDim.x) {
    const size_t q = v * 4;
    T xr[4][4], xi[4][4];
#pragma unroll
    for (int x = 0; x < 4; ++x) {
      if (x < a.nx) {
        ld4(a.X[x] + q, xr[x]);
        ld4(a.X[x] + P + q, xi[x]);
      }
    }
    T o_r[4] = {0, 0, 0, 0}, o_i[4] = {0, 0, 0, 0};
#pragma unroll
    for (int f = 0; f < 4; ++f) {
      if (f >= a.nf) break;
      T sr[4] = {0, 0, 0, 0}, si[4] = {0, 0, 0, 0};
#pragma unroll
      for (int x = 0; x < 4; ++x) {
        if (x < a.nx && a.W[f][x] != 0.0) {
          const T w = (T)a.W[f][x];
#pragma unroll
          for (int l = 0; l < 4; ++l) {
            sr[l] += w * xr[x][l];
            si[l] += w * xi[x][l];
          }
        }
      }
      if (a.fkind[f] == F_ONE) {
#pragma unroll
        for (int l = 0; l < 4; ++l) { o_r[l] += sr[l]; o_i[l] += si[l]; }
      } else {
        T fr[4], fi[4];
        if (a.fkind[f] == F_TENSOR) {
          ld4(a.F[f] + q, fr);
          ld4(a.F[f] + P + q, fi);
        } else {
#pragma unroll
          for (int l = 0; l < 4; ++l) {
            double lr, li;
            lam_at(L, q + l, lr, li);
            fr[l] = (T)lr;
            fi[l] = (T)li;
          }
        }
#pragma unroll
        for (int l = 0; l < 4; ++l) {
          o_r[l] += fr[l] * sr[l] - fi[l] * si[l];
          o_i[l] += fr[l] * si[l] + fi[l] * sr[l];
        }
      }
    }
    if (a.out) {
      st4(a.out + q, o_r);
      st4(a.out + P + q, o_i);
    }
    if (a.out2) {
      T br[4], bi[4];
      ld4(a.base + q, br);
      ld4(a.base + P + q, bi);
#pragma unroll
      for (int l = 0; l < 4; ++l) { br[l] += o_r[l]; bi[l] += o_i[l]; }
      st4(a.out2 + q, br);
      st4(a.out2 + P + q, bi);
    }
  }
}

// --------------------------------------------------------- F = f(theta lam)
__device__ void phi_eval(int ell, double zr, double zi, double& fr, double& fi) {
  // phi_ell(z): power series sum_m z^m/(m+ell)! for |z| < 1, recurrence (Eq. phi) otherwise.
  const double az = hypot(zr, zi);
  if (az < 1.0) {
    double inv_fact = 1.0;
    for (int m = 2; m <= ell; ++m) inv_fact /= m;
    double tr = inv_fact, ti = 0.0, sr = tr, si = 0.0;
    for (int m = 1; m < 40; ++m) {
      const double nr = (tr * zr - ti * zi) / (m + ell);
      const double ni = (tr * zi + ti * zr) / (m + ell);
      tr = nr;
      ti = ni;
      sr += tr;
      si += ti;
      if (fabs(tr) + fabs(ti) < 1e-18 * (fabs(sr) + fabs(si))) break;
    }
    fr = sr;
    fi = si;
    return;
  }
  const double ex = exp(zr);
  double s, c;
  sincos(zi, &s, &c);
  double pr = ex * c, pi = ex * s;
  const double den = zr * zr + zi * zi;
  double inv_fact = 1.0;   // 1/(l-1)!
  for (int l = 1; l <= ell; ++l) {
    if (l >= 2) inv_fact /= (l - 1);
    const double ar = pr - inv_fact, ai = pi;
    // (ar + i ai) / (zr + i zi)
    pr = (ar * zr + ai * zi) / den;
    pi = (ai * zr - ar * zi) / den;
  }
  fr = pr;
  fi = pi;
}

// f(z) for func 0: 1/(1 - z), 1: e^z, 2: phi_ell (FP64)
__device__ __forceinline__ void f_eval64(int func, int ell, double zr, double zi, double& fr, double& fi) {
  if (func == 0) {
    const double ar = 1.0 - zr, ai = -zi, den = ar * ar + ai * ai;
    fr = ar / den;
    fi = -ai / den;
  } else if (func == 1) {
    double sn, cs;
    sincos(zi, &sn, &cs);
    const double ex = exp(zr);
    fr = ex * cs;
    fi = ex * sn;
  } else {
    phi_eval(ell, zr, zi, fr, fi);
  }
}

// out[2 j], out[2 j + 1] = f(theta (c_re + i c_im) s_j)
__global__ void scalars_f64_kernel(int n, const double* __restrict__ sv, double c_re, double c_im, int func,
                                   int ell, double theta, double* __restrict__ out) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
    double fr, fi;
    f_eval64(func, ell, theta * c_re * sv[j], theta * c_im * sv[j], fr, fi);
    out[2 * j] = fr;
    out[2 * j + 1] = fi;
  }
}

template <typename T>
__global__ void fill_F_kernel(size_t P, LamDev L, Shape s, int func, int ell, double theta, T* __restrict__ F) {
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < P; q += (size_t)gridDim.x * blockDim.x) {
    size_t rem = q;
    bool valid = true;
    double sum = 0.0;
    for (int mu = 0; mu < s.d; ++mu) {
      int j = (int)(rem % s.p[mu]);
      rem /= s.p[mu];
      valid = valid && j < s.n[mu];
      sum += L.lam[mu][j];
    }
    double fr = 0.0, fi = 0.0;
    if (valid) f_eval64(func, ell, theta * L.c_re * sum, theta * L.c_im * sum, fr, fi);
    F[q] = (T)fr;
    F[P + q] = (T)fi;
  }
}

// ------------------------------------------------------------ exact flow
template <typename T>
__global__ void exact_flow_kernel(size_t P, double gamma, double kappa, double zeta, double t, double tp1,
                                  const T* __restrict__ X, T* __restrict__ Y) {
  // w(t) = exp(t gamma - (kappa + i zeta)/(2 kappa) log(1 + 2 t phi_1(2 gamma t) kappa |w0|^2)) w0
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < P; q += (size_t)gridDim.x * blockDim.x) {
    const double wr = X[q], wi = X[P + q];
    const double L = log1p(2.0 * t * tp1 * kappa * (wr * wr + wi * wi));
    const double er = t * gamma - 0.5 * L, ei = -zeta / (2.0 * kappa) * L;
    double sn, cs;
    sincos(ei, &sn, &cs);
    const double m = exp(er);
    Y[q] = (T)(m * (cs * wr - sn * wi));
    Y[P + q] = (T)(m * (cs * wi + sn * wr));
  }
}

// ------------------------------------------------------------ sum |x|^2
template <typename T>
__global__ void sumsq_kernel(size_t P2, const T* __restrict__ X, double* out) {
  double acc = 0.0;
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < P2; q += (size_t)gridDim.x * blockDim.x) {
    const double x = X[q];
    acc += x * x;
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  __shared__ double red[32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) red[wid] = acc;
  __syncthreads();
  if (wid == 0) {
    acc = lane < (int)(blockDim.x >> 5) ? red[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) atomicAdd(out, acc);
  }
}

LamDev lamdev(const Shape& s, const LamVecs& lv) {
  LamDev L;
  for (int mu = 0; mu < kMaxDim; ++mu) {
    L.lam[mu] = lv.lam[mu];
    L.p[mu] = s.p[mu];
  }
  L.d = s.d;
  L.c_re = lv.c_re;
  L.c_im = lv.c_im;
  return L;
}

}  // namespace

// ===================================================================== host
template <typename T>
void pack(const Shape& s, const T* user, T* X, cudaStream_t st, long long& nl) {
  pack_kernel<T><<<grid_for(s.P / 4, 256), 256, 0, st>>>(s, user, X);
  FCGLE_LAUNCHED(nl);
}
template <typename T>
void unpack(const Shape& s, const T* X, T* user, cudaStream_t st, long long& nl, int* nonfinite) {
  unpack_kernel<T><<<grid_for(s.P / 4, 256), 256, 0, st>>>(s, X, user, nonfinite);
  FCGLE_LAUNCHED(nl);
}

template <typename T>
void gcombo(const Shape& s, const GParams& gp, double t, const T* X0, const T* X1, const T* X2, double c0,
            double c1, double a0, double a1, double b, double e, T* out, cudaStream_t st, long long& nl) {
  GDev g;
  g.gamma = gp.gamma;
  g.kappa = gp.kappa;
  g.zeta = gp.zeta;
  g.nsrc = (b != 0.0) ? gp.nsrc : 0;
  for (int k = 0; k < kMaxSrc; ++k) {
    g.S[k] = gp.S[k];
    if (k < gp.nsrc) {
      const double m = std::exp(gp.sig_re[k] * t);
      g.e_re[k] = m * std::cos(gp.sig_im[k] * t);
      g.e_im[k] = m * std::sin(gp.sig_im[k] * t);
    } else {
      g.e_re[k] = g.e_im[k] = 0.0;
    }
  }
  gcombo_kernel<T><<<grid_for(s.P / 4, 256), 256, 0, st>>>(s.P, g, X0, X1, X2, c0, c1, a0, a1, b, e, out);
  FCGLE_LAUNCHED(nl);
}

template <typename T>
void spec_combo(const Shape& s, const LamVecs& lv, const SpecArgs<T>& a, cudaStream_t st, long long& nl) {
  SpecDev<T> d;
  d.nx = a.nx;
  d.nf = a.nf;
  for (int i = 0; i < 4; ++i) {
    d.X[i] = a.X[i];
    d.F[i] = a.F[i];
    d.fkind[i] = a.fkind[i];
    for (int j = 0; j < 4; ++j) d.W[i][j] = a.W[i][j];
  }
  d.out = a.out;
  d.base = a.base;
  d.out2 = a.out2;
  spec_kernel<T><<<grid_for(s.P / 4, 256), 256, 0, st>>>(s.P, lamdev(s, lv), d);
  FCGLE_LAUNCHED(nl);
}

void spectral_scalars_f64(int n, const double* s_dev, double c_re, double c_im, int func, int ell, double theta,
                          double* out_dev, cudaStream_t st, long long& nl) {
  scalars_f64_kernel<<<grid_for((size_t)n, 256), 256, 0, st>>>(n, s_dev, c_re, c_im, func, ell, theta, out_dev);
  FCGLE_LAUNCHED(nl);
}

template <typename T>
void fill_F(const Shape& s, const LamVecs& lv, int func, int ell, double theta, T* F, cudaStream_t st,
            long long& nl) {
  fill_F_kernel<T><<<grid_for(s.P, 256), 256, 0, st>>>(s.P, lamdev(s, lv), s, func, ell, theta, F);
  FCGLE_LAUNCHED(nl);
}

template <typename T>
void exact_flow(const Shape& s, double gamma, double kappa, double zeta, double t, const T* X, T* Y,
                cudaStream_t st, long long& nl) {
  // t phi_1(2 gamma t), in FP64 on the host
  const double z = 2.0 * gamma * t;
  const double p1 = std::fabs(z) < 1e-8 ? 1.0 + z / 2.0 : std::expm1(z) / z;
  exact_flow_kernel<T><<<grid_for(s.P, 256), 256, 0, st>>>(s.P, gamma, kappa, zeta, t, p1, X, Y);
  FCGLE_LAUNCHED(nl);
}

template <typename T>
void sumsq(const Shape& s, const T* X, double* out_dev, cudaStream_t st, long long& nl) {
  FCGLE_CUDA(cudaMemsetAsync(out_dev, 0, sizeof(double), st));
  sumsq_kernel<T><<<grid_for(2 * s.P, 256), 256, 0, st>>>(2 * s.P, X, out_dev);
  FCGLE_LAUNCHED(nl);
}

#define INST(T)                                                                                           \
  template void pack<T>(const Shape&, const T*, T*, cudaStream_t, long long&);                           \
  template void unpack<T>(const Shape&, const T*, T*, cudaStream_t, long long&, int*);                         \
  template void gcombo<T>(const Shape&, const GParams&, double, const T*, const T*, const T*, double,     \
                          double, double, double, double, double, T*, cudaStream_t, long long&);         \
  template void spec_combo<T>(const Shape&, const LamVecs&, const SpecArgs<T>&, cudaStream_t, long long&); \
  template void fill_F<T>(const Shape&, const LamVecs&, int, int, double, T*, cudaStream_t, long long&);  \
  template void exact_flow<T>(const Shape&, double, double, double, double, const T*, T*, cudaStream_t,   \
                              long long&);                                                               \
  template void sumsq<T>(const Shape&, const T*, double*, cudaStream_t, long long&);
INST(float)
INST(double)
#undef INST

}  // namespace fcgle
