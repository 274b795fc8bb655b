// Pointwise kernels and reductions of the discrete adjoint (adjoint.h).
// Planar internal layout (common.h); FP64 accumulation of every reduction
// (warp shuffles, one atomic per block and slot).
#include <cmath>
#include <type_traits>

#include "adjoint.h"

namespace fcgle {

namespace {

int grid_of(size_t n) {
  static const int sms = [] {   // thread-safe one-time initialisation
    int dev = 0, m = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&m, cudaDevAttrMultiProcessorCount, dev);
    return m > 0 ? m : 132;
  }();
  size_t g = (n + 255) / 256;
  if (g > (size_t)sms * 8) g = (size_t)sms * 8;
  return (int)(g < 1 ? 1 : g);
}

// block-reduce NV values and atomically add them to acc[slot0 + k]
template <int NV>
__device__ void block_acc(double (&v)[NV], double* acc, int slot0) {
  __shared__ double red[NV][32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    double x = v[k];
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (lane == 0) red[k][wid] = x;
  }
  __syncthreads();
  if (wid == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double x = lane < nw ? red[k][lane] : 0.0;
      for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
      if (lane == 0) atomicAdd(acc + slot0 + k, x);
    }
  }
}

// g source term sum_k e^{sigma_k t} S_k is independent of u: its derivative vanishes.
struct GP {
  double gamma, kappa, zeta;
};

template <typename T>
__global__ void misfit_kernel(size_t P, const T* __restrict__ u, const T* __restrict__ tg, T* __restrict__ lam,
                              double* acc) {
  double v[1] = {0.0};
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < P; q += (size_t)gridDim.x * blockDim.x) {
    const double dr = (double)u[q] - (double)tg[q], di = (double)u[P + q] - (double)tg[P + q];
    lam[q] = (T)dr;
    lam[P + q] = (T)di;
    v[0] += 0.5 * (dr * dr + di * di);
  }
  block_acc<1>(v, acc, ADJ_LOSS);
}

// (D_z g)^* w = conj(alpha) w + beta conj(w),  alpha = gamma - 2 c |z|^2, beta = -c z^2, c = kappa + i zeta
__device__ __forceinline__ void gadj(const GP& g, double zr, double zi, double wr, double wi, double& orr,
                                     double& oi) {
  const double m2 = zr * zr + zi * zi;
  const double ar = g.gamma - 2.0 * g.kappa * m2, ai = -2.0 * g.zeta * m2;   // alpha
  const double z2r = zr * zr - zi * zi, z2i = 2.0 * zr * zi;
  const double br = -(g.kappa * z2r - g.zeta * z2i), bi = -(g.kappa * z2i + g.zeta * z2r);   // beta
  // conj(alpha) w + beta conj(w)
  orr = ar * wr + ai * wi + br * wr + bi * wi;
  oi = ar * wi - ai * wr + bi * wr - br * wi;
}
// Re<w, dg/dp(z)> for p = gamma, kappa, zeta
__device__ __forceinline__ void gpar(double zr, double zi, double wr, double wi, double (&v)[3]) {
  const double m2 = zr * zr + zi * zi;
  v[0] += wr * zr + wi * zi;                 // Re(conj(w) z)
  v[1] += -m2 * (wr * zr + wi * zi);         // Re(conj(w) (-|z|^2 z))
  v[2] += -m2 * (wr * (-zi) + wi * zr);      // Re(conj(w) (-i |z|^2 z)),  -i z = (zi, -zr) * (-1)
}

template <typename T>
__global__ void gv_kernel(size_t P, GP g, const T* __restrict__ z, const T* __restrict__ w, double c,
                          T* __restrict__ mu, double* acc) {
  double v[3] = {0.0, 0.0, 0.0};
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < P; q += (size_t)gridDim.x * blockDim.x) {
    const double zr = z[q], zi = z[P + q], wr = c * (double)w[q], wi = c * (double)w[P + q];
    double orr, oi;
    gadj(g, zr, zi, wr, wi, orr, oi);
    mu[q] = (T)orr;
    mu[P + q] = (T)oi;
    gpar(zr, zi, wr, wi, v);
  }
  block_acc<3>(v, acc, ADJ_GAMMA);
}

template <typename T>
__global__ void gu_kernel(size_t P, GP g, const T* __restrict__ u, const T* __restrict__ la,
                          const T* __restrict__ lb, double ca, double cb, T* __restrict__ out, double* acc) {
  double v[3] = {0.0, 0.0, 0.0};
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < P; q += (size_t)gridDim.x * blockDim.x) {
    const double ar = la[q], ai = la[P + q], br = lb[q], bi = lb[P + q];
    const double kr = ca * ar + cb * br, ki = ca * ai + cb * bi;
    const double zr = u[q], zi = u[P + q];
    double orr, oi;
    gadj(g, zr, zi, kr, ki, orr, oi);
    out[q] = (T)(ar + br + orr);
    out[P + q] = (T)(ai + bi + oi);
    gpar(zr, zi, kr, ki, v);
  }
  block_acc<3>(v, acc, ADJ_GAMMA);
}

struct LD {
  const double* lam[kMaxDim];
  int p[kMaxDim];
  int n[kMaxDim];
  int d;
};
__device__ __forceinline__ bool lam_sum(const LD& L, size_t q, double& s) {
  s = 0.0;
  bool valid = true;
  size_t rem = q;
  for (int mu = 0; mu < L.d; ++mu) {
    const int j = (int)(rem % L.p[mu]);
    rem /= L.p[mu];
    valid = valid && j < L.n[mu];
    s += L.lam[mu][j];
  }
  return valid;
}

template <typename T>
__global__ void spec_dot_kernel(size_t P, LD L, const T* __restrict__ x, const T* __restrict__ y, double* acc) {
  double v[2] = {0.0, 0.0};
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < P; q += (size_t)gridDim.x * blockDim.x) {
    double s;
    if (!lam_sum(L, q, s)) continue;
    const double xr = x[q], xi = x[P + q], yr = y[q], yi = y[P + q];
    v[0] += s * (xr * yr + xi * yi);   // Re conj(x) y
    v[1] += s * (xr * yi - xi * yr);   // Im conj(x) y
  }
  block_acc<2>(v, acc, ADJ_Z_RE);
}

template <typename T>
__global__ void axpby_kernel(size_t n, double a, const T* __restrict__ x1, double b, const T* __restrict__ x2,
                             T* __restrict__ y) {
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < n; q += (size_t)gridDim.x * blockDim.x)
    y[q] = (T)(a * (double)x1[q] + (x2 ? b * (double)x2[q] : 0.0));
}

// e^{z} with z = (cre + i cim) s at an element (0 on padding)
__device__ __forceinline__ void exp_z(const LD& L, size_t q, double cre, double cim, double& er, double& ei) {
  double s;
  er = ei = 0.0;
  if (lam_sum(L, q, s)) {
    double sn, cs;
    sincos(cim * s, &sn, &cs);
    const double m = exp(cre * s);
    er = m * cs;
    ei = m * sn;
  }
}

// y1 = e^z (x + c1 k), y2 = e^z (x + c2 k): the two stage values of a
// Lawson-RK2 step (V^ and W^), one pass over x and k
template <typename T>
__global__ void exp_pair_kernel(size_t P, LD L, double cre, double cim, const T* __restrict__ x,
                                const T* __restrict__ k, double c1, double c2, T* __restrict__ y1, T* __restrict__ y2) {
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < P; q += (size_t)gridDim.x * blockDim.x) {
    double er, ei;
    exp_z(L, q, cre, cim, er, ei);
    const double xr = x[q], xi = x[P + q], kr = k[q], ki = k[P + q];
    double ur = xr + c1 * kr, ui = xi + c1 * ki;
    y1[q] = (T)(er * ur - ei * ui);
    y1[P + q] = (T)(er * ui + ei * ur);
    ur = xr + c2 * kr;
    ui = xi + c2 * ki;
    y2[q] = (T)(er * ur - ei * ui);
    y2[P + q] = (T)(er * ui + ei * ur);
  }
}

// a = e^{z} x, b = e^{z} m (z already conjugated by the caller):
// y = ca a + cb b and sum = a + b, one pass; y may alias x
template <typename T>
__global__ void exp_combo_kernel(size_t P, LD L, double cre, double cim, const T* x, const T* __restrict__ m,
                                 double ca, double cb, T* y, T* __restrict__ sum) {
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < P; q += (size_t)gridDim.x * blockDim.x) {
    double er, ei;
    exp_z(L, q, cre, cim, er, ei);
    const double xr = x[q], xi = x[P + q], mr = m[q], mi = m[P + q];
    const double ar = er * xr - ei * xi, ai = er * xi + ei * xr;
    const double br = er * mr - ei * mi, bi = er * mi + ei * mr;
    y[q] = (T)(ca * ar + cb * br);
    y[P + q] = (T)(ca * ai + cb * bi);
    sum[q] = (T)(ar + br);
    sum[P + q] = (T)(ai + bi);
  }
}

// ---- FP32 forms (split-BF16 engine): per-element arithmetic in FP32 with
// 32-bit indices (2 P < 2^32 there), 4 consecutive elements of a row of
// direction 1 per thread step (p_1 is a multiple of 8), 16-byte accesses;
// reductions are summed in FP32 over a thread's few elements and accumulated
// in FP64 across threads and blocks.
struct Quad {
  float s[4];      // eigenvalue sums (without the factor nu + i eta)
  bool valid[4];   // interior (not padding)
};
// the 4 elements q .. q + 3 (q % 4 == 0, all in one row of direction 1)
__device__ __forceinline__ Quad quad_lam(const LD& L, uint32_t q) {
  Quad o;
  const uint32_t p1 = (uint32_t)L.p[0];
  const uint32_t j1 = q % p1;
  uint32_t rem = q / p1;
  float base = 0.f;
  bool ok = true;
  for (int mu = 1; mu < L.d; ++mu) {
    const uint32_t p = (uint32_t)L.p[mu];
    const uint32_t j = rem % p;
    rem /= p;
    ok = ok && (int)j < L.n[mu];
    base += (float)L.lam[mu][j];
  }
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    o.valid[v] = ok && (int)(j1 + v) < L.n[0];
    o.s[v] = base + (float)L.lam[0][j1 + v];
  }
  return o;
}
__device__ __forceinline__ void ld4f(const float* p, float (&v)[4]) {
  const float4 x = *reinterpret_cast<const float4*>(p);
  v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w;
}
__device__ __forceinline__ void st4f(float* p, const float (&v)[4]) {
  *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}

__device__ __forceinline__ void gadj_f(float gam, float kap, float zet, float zr, float zi, float wr, float wi,
                                       float& orr, float& oi) {
  const float m2 = zr * zr + zi * zi;
  const float ar = gam - 2.f * kap * m2, ai = -2.f * zet * m2;
  const float z2r = zr * zr - zi * zi, z2i = 2.f * zr * zi;
  const float br = -(kap * z2r - zet * z2i), bi = -(kap * z2i + zet * z2r);
  orr = ar * wr + ai * wi + br * wr + bi * wi;
  oi = ar * wi - ai * wr + bi * wr - br * wi;
}

__global__ void gv_kernel_f(uint32_t P, GP g, const float* __restrict__ z, const float* __restrict__ w, float c,
                            float* __restrict__ mu, double* acc) {
  float f[3] = {0.f, 0.f, 0.f};
  const float gam = (float)g.gamma, kap = (float)g.kappa, zet = (float)g.zeta;
  for (uint32_t q = 4 * (blockIdx.x * blockDim.x + threadIdx.x); q < P; q += 4 * gridDim.x * blockDim.x) {
    float zr[4], zi[4], wr[4], wi[4], orr[4], oi[4];
    ld4f(z + q, zr);
    ld4f(z + P + q, zi);
    ld4f(w + q, wr);
    ld4f(w + P + q, wi);
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      wr[v] *= c;
      wi[v] *= c;
      gadj_f(gam, kap, zet, zr[v], zi[v], wr[v], wi[v], orr[v], oi[v]);
      // Re<w, dg/dp(z)> for p = gamma, kappa, zeta
      const float m2 = zr[v] * zr[v] + zi[v] * zi[v];
      const float dd = wr[v] * zr[v] + wi[v] * zi[v], ee = wi[v] * zr[v] - wr[v] * zi[v];
      f[0] += dd;
      f[1] -= m2 * dd;
      f[2] -= m2 * ee;
    }
    st4f(mu + q, orr);
    st4f(mu + P + q, oi);
  }
  double v[3] = {(double)f[0], (double)f[1], (double)f[2]};
  block_acc<3>(v, acc, ADJ_GAMMA);
}

// e^z - 1 = mr + i mi at element v of a quad, z = (ar + i ai) s:
// expm1(Re z) cos(Im z) - 2 sin^2(Im z / 2) + i e^{Re z} sin(Im z), so that a
// product e^z x is formed as x + (e^z - 1) x and the FP32 rounding falls on the
// correction, not on a factor that the sweeps apply again every step.
// Padding (j >= n): e^z = 0, i.e. mr = -1, mi = 0.
__device__ __forceinline__ void expm1_z_f(const Quad& Q, int v, float ar, float ai, float& mr, float& mi) {
  mr = -1.f;
  mi = 0.f;
  if (Q.valid[v]) {
    const float a = ar * Q.s[v], b = ai * Q.s[v];
    float sn, cs, sh, ch;
    sincosf(b, &sn, &cs);
    sincosf(0.5f * b, &sh, &ch);
    const float em = expm1f(a);
    mr = em * cs - 2.f * sh * sh;
    mi = (1.f + em) * sn;
  }
}

// y1 = e^z (x + c1 k), y2 = e^z (x + c2 k) (FP32 form of exp_pair_kernel)
__global__ void exp_pair_kernel_f(uint32_t P, LD L, float ar, float ai, const float* __restrict__ x,
                                  const float* __restrict__ k, float c1, float c2, float* __restrict__ y1,
                                  float* __restrict__ y2) {
  for (uint32_t q = 4 * (blockIdx.x * blockDim.x + threadIdx.x); q < P; q += 4 * gridDim.x * blockDim.x) {
    const Quad Q = quad_lam(L, q);
    float xr[4], xi[4], kr[4], ki[4], pr[4], pi[4], wr[4], wi[4];
    ld4f(x + q, xr);
    ld4f(x + P + q, xi);
    ld4f(k + q, kr);
    ld4f(k + P + q, ki);
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      float mr, mi;
      expm1_z_f(Q, v, ar, ai, mr, mi);
      const float ur = xr[v] + c1 * kr[v], ui = xi[v] + c1 * ki[v];
      pr[v] = ur + (mr * ur - mi * ui);
      pi[v] = ui + (mr * ui + mi * ur);
      const float vr = xr[v] + c2 * kr[v], vi = xi[v] + c2 * ki[v];
      wr[v] = vr + (mr * vr - mi * vi);
      wi[v] = vi + (mr * vi + mi * vr);
    }
    st4f(y1 + q, pr);
    st4f(y1 + P + q, pi);
    st4f(y2 + q, wr);
    st4f(y2 + P + q, wi);
  }
}

// a = e^z x, b = e^z m; y = ca a + cb b, sum = a + b (FP32 form of exp_combo_kernel; y may alias x)
__global__ void exp_combo_kernel_f(uint32_t P, LD L, float ar, float ai, const float* x, const float* __restrict__ m,
                                   float ca, float cb, float* y, float* __restrict__ sum) {
  for (uint32_t q = 4 * (blockIdx.x * blockDim.x + threadIdx.x); q < P; q += 4 * gridDim.x * blockDim.x) {
    const Quad Q = quad_lam(L, q);
    float xr[4], xi[4], nr[4], ni[4], yr[4], yi[4], sr[4], si[4];
    ld4f(x + q, xr);
    ld4f(x + P + q, xi);
    ld4f(m + q, nr);
    ld4f(m + P + q, ni);
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      float mr, mi;
      expm1_z_f(Q, v, ar, ai, mr, mi);
      const float a_r = xr[v] + (mr * xr[v] - mi * xi[v]), a_i = xi[v] + (mr * xi[v] + mi * xr[v]);
      const float b_r = nr[v] + (mr * nr[v] - mi * ni[v]), b_i = ni[v] + (mr * ni[v] + mi * nr[v]);
      yr[v] = ca * a_r + cb * b_r;
      yi[v] = ca * a_i + cb * b_i;
      sr[v] = a_r + b_r;
      si[v] = a_i + b_i;
    }
    st4f(y + q, yr);
    st4f(y + P + q, yi);
    st4f(sum + q, sr);
    st4f(sum + P + q, si);
  }
}

__global__ void spec_dot_kernel_f(uint32_t P, LD L, const float* __restrict__ x, const float* __restrict__ y,
                                  double* acc) {
  float f[2] = {0.f, 0.f};
  for (uint32_t q = 4 * (blockIdx.x * blockDim.x + threadIdx.x); q < P; q += 4 * gridDim.x * blockDim.x) {
    const Quad Q = quad_lam(L, q);
    float xr[4], xi[4], yr[4], yi[4];
    ld4f(x + q, xr);
    ld4f(x + P + q, xi);
    ld4f(y + q, yr);
    ld4f(y + P + q, yi);
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      if (!Q.valid[v]) continue;
      f[0] += Q.s[v] * (xr[v] * yr[v] + xi[v] * yi[v]);   // Re conj(x) y
      f[1] += Q.s[v] * (xr[v] * yi[v] - xi[v] * yr[v]);   // Im conj(x) y
    }
  }
  double v[2] = {(double)f[0], (double)f[1]};
  block_acc<2>(v, acc, ADJ_Z_RE);
}

__global__ void axpby_kernel_f(uint32_t n, float a, const float* __restrict__ x1, float b,
                               const float* __restrict__ x2, float* __restrict__ y) {
  for (uint32_t q = 4 * (blockIdx.x * blockDim.x + threadIdx.x); q < n; q += 4 * gridDim.x * blockDim.x) {
    float u[4], w[4] = {0.f, 0.f, 0.f, 0.f};
    ld4f(x1 + q, u);
    if (x2) ld4f(x2 + q, w);
#pragma unroll
    for (int v = 0; v < 4; ++v) u[v] = a * u[v] + b * w[v];
    st4f(y + q, u);
  }
}

LD make_ld(const Shape& s, const LamVecs& lv) {
  LD L;
  for (int mu = 0; mu < kMaxDim; ++mu) {
    L.lam[mu] = lv.lam[mu];
    L.p[mu] = s.p[mu];
    L.n[mu] = s.n[mu];
  }
  L.d = s.d;
  return L;
}

}  // namespace

template <typename T>
void adj_misfit(const Shape& s, const T* u, const T* target, T* lam, double* acc, cudaStream_t st, long long& nl) {
  misfit_kernel<T><<<grid_of(s.P), 256, 0, st>>>(s.P, u, target, lam, acc);
  FCGLE_LAUNCHED(nl);
}
template <typename T>
void adj_gv(const Shape& s, const GParams& gp, const T* z, const T* w, double c, T* mu, double* acc, cudaStream_t st,
            long long& nl) {
  if constexpr (std::is_same<T, float>::value)
    gv_kernel_f<<<grid_of(s.P / 4), 256, 0, st>>>((uint32_t)s.P, GP{gp.gamma, gp.kappa, gp.zeta}, z, w, (float)c,
                                                   mu, acc);
  else
    gv_kernel<T><<<grid_of(s.P), 256, 0, st>>>(s.P, GP{gp.gamma, gp.kappa, gp.zeta}, z, w, c, mu, acc);
  FCGLE_LAUNCHED(nl);
}
template <typename T>
void adj_gu(const Shape& s, const GParams& gp, const T* u, const T* la, const T* lb, double ca, double cb, T* out,
            double* acc, cudaStream_t st, long long& nl) {
  gu_kernel<T><<<grid_of(s.P), 256, 0, st>>>(s.P, GP{gp.gamma, gp.kappa, gp.zeta}, u, la, lb, ca, cb, out, acc);
  FCGLE_LAUNCHED(nl);
}
template <typename T>
void adj_spec_dot(const Shape& s, const LamVecs& lv, const T* x, const T* y, double* acc, cudaStream_t st,
                  long long& nl) {
  if constexpr (std::is_same<T, float>::value)
    spec_dot_kernel_f<<<grid_of(s.P / 4), 256, 0, st>>>((uint32_t)s.P, make_ld(s, lv), x, y, acc);
  else
    spec_dot_kernel<T><<<grid_of(s.P), 256, 0, st>>>(s.P, make_ld(s, lv), x, y, acc);
  FCGLE_LAUNCHED(nl);
}
template <typename T>
void adj_axpby(const Shape& s, double a, const T* x1, double b, const T* x2, T* y, cudaStream_t st, long long& nl) {
  if constexpr (std::is_same<T, float>::value)
    axpby_kernel_f<<<grid_of(2 * s.P / 4), 256, 0, st>>>((uint32_t)(2 * s.P), (float)a, x1, (float)b, x2, y);
  else
    axpby_kernel<T><<<grid_of(2 * s.P), 256, 0, st>>>(2 * s.P, a, x1, b, x2, y);
  FCGLE_LAUNCHED(nl);
}

template <typename T>
void adj_exp_pair(const Shape& s, const LamVecs& lv, double theta, const T* x, const T* k, double c1, double c2,
                  T* y1, T* y2, cudaStream_t st, long long& nl) {
  if constexpr (std::is_same<T, float>::value)
    exp_pair_kernel_f<<<grid_of(s.P / 4), 256, 0, st>>>((uint32_t)s.P, make_ld(s, lv), (float)(theta * lv.c_re),
                                                     (float)(theta * lv.c_im), x, k, (float)c1, (float)c2, y1, y2);
  else
    exp_pair_kernel<T><<<grid_of(s.P), 256, 0, st>>>(s.P, make_ld(s, lv), theta * lv.c_re, theta * lv.c_im, x, k,
                                                       c1, c2, y1, y2);
  FCGLE_LAUNCHED(nl);
}
template <typename T>
void adj_exp_h_combo(const Shape& s, const LamVecs& lv, double theta, const T* x, const T* m, double ca, double cb,
                     T* y, T* sum, cudaStream_t st, long long& nl) {
  if constexpr (std::is_same<T, float>::value)
    exp_combo_kernel_f<<<grid_of(s.P / 4), 256, 0, st>>>((uint32_t)s.P, make_ld(s, lv), (float)(theta * lv.c_re),
                                                      (float)(-theta * lv.c_im), x, m, (float)ca, (float)cb, y, sum);
  else
    exp_combo_kernel<T><<<grid_of(s.P), 256, 0, st>>>(s.P, make_ld(s, lv), theta * lv.c_re, -theta * lv.c_im, x, m,
                                                        ca, cb, y, sum);
  FCGLE_LAUNCHED(nl);
}

#define INST(T)                                                                                                  \
  template void adj_misfit<T>(const Shape&, const T*, const T*, T*, double*, cudaStream_t, long long&);          \
  template void adj_gv<T>(const Shape&, const GParams&, const T*, const T*, double, T*, double*, cudaStream_t,  \
                          long long&);                                                                          \
  template void adj_gu<T>(const Shape&, const GParams&, const T*, const T*, const T*, double, double, T*,       \
                          double*, cudaStream_t, long long&);                                                   \
  template void adj_spec_dot<T>(const Shape&, const LamVecs&, const T*, const T*, double*, cudaStream_t,        \
                                long long&);                                                                    \
  template void adj_axpby<T>(const Shape&, double, const T*, double, const T*, T*, cudaStream_t, long long&);    \
  template void adj_exp_pair<T>(const Shape&, const LamVecs&, double, const T*, const T*, double, double, T*, T*, \
                                cudaStream_t, long long&);                                                       \
  template void adj_exp_h_combo<T>(const Shape&, const LamVecs&, double, const T*, const T*, double, double, T*,  \
                                   T*, cudaStream_t, long long&);
INST(float)
INST(double)
#undef INST

}  // namespace fcgle
