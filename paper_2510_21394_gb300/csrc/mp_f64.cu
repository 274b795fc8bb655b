// FP64 mu-mode products (paper Sec. 3.2: "each [mode product] realized in
// practice with a single BLAS call") in the rotating layout of common.h.
//
// GEMM view: C[row][col] = sum_kk A(row, kk) * B[col][kk], written with the
// output index `col` as the slowest one.
//   real matrix M (p x p):        row = (c, r), 2R rows; kk = k, K = p;
//     A(row, k) = X[row * p + k];  Y[c][i][r] = C[(c, r)][i].
//   complex matrix in real block form B = [[Re E, -Im E], [Im E, Re E]]
//   (2p x 2p):                    row = r, R rows; kk = (c, k), K = 2p;
//     A(r, (c, k)) = X[c][r][k];   Y[c'][i][r] = C[r][(c', i)].
// GB300's FP64 rate is a small fraction of its tensor-core rate, so this
// is a plain shared-memory tiled SIMT GEMM (64 x 64 tile, 4 x 4 per thread):
// it is FP64-ALU bound by a wide margin at every size used here.  The same
// kernel in FP32 (real matrices only) serves the split-BF16 engine for the
// few transforms per solve that must not carry the split-BF16 error (the
// first forward and the last backward Tucker operator of a time integration).
#include "common.h"

namespace fcgle {

namespace {

constexpr int BM = 64, BN = 64, BK = 16, NT = 256;

template <typename T, bool CPLX>
__global__ void __launch_bounds__(NT) mp_simt_kernel(const T* __restrict__ X, T* __restrict__ Y,
                                                     const T* __restrict__ B, int p, long long R) {
  __shared__ T As[BK][BM + 2];
  __shared__ T Bs[BK][BN + 2];
  const long long rows = CPLX ? R : 2 * R;
  const int K = CPLX ? 2 * p : p;
  const int Ncol = CPLX ? 2 * p : p;
  const long long Rp = R * (long long)p;

  const long long row0 = (long long)blockIdx.x * BM;
  const int col0 = blockIdx.y * BN;
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;   // rows tx*4.., cols ty*4..

  T acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = T(0);

  const int lk = tid & 15, lr = tid >> 4;   // loader: k offset, row offset (+16 j)
  for (int k0 = 0; k0 < K; k0 += BK) {
    const int kk = k0 + lk;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const long long row = row0 + lr + 16 * j;
      T a = T(0);
      if (row < rows && kk < K) {
        if (CPLX) {
          const int c = kk >= p ? 1 : 0;
          a = X[c * Rp + row * p + (kk - c * p)];
        } else {
          a = X[row * p + kk];
        }
      }
      As[lk][lr + 16 * j] = a;
      const int col = col0 + lr + 16 * j;
      Bs[lk][lr + 16 * j] = (col < Ncol && kk < K) ? B[(long long)col * K + kk] : T(0);
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < BK; ++k) {
      T a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[k][tx * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[k][ty * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }

#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int col = col0 + ty * 4 + j;
    if (col >= Ncol) continue;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const long long row = row0 + tx * 4 + i;
      if (row >= rows) continue;
      long long dst;
      if (CPLX) {
        const int c = col >= p ? 1 : 0;
        dst = c * Rp + (long long)(col - c * p) * R + row;
      } else {
        const long long c = row >= R ? 1 : 0;
        dst = c * Rp + (long long)col * R + (row - c * R);
      }
      Y[dst] = acc[i][j];
    }
  }
}

}  // namespace

void mp_f64(const double* X, double* Y, const double* M, int p, size_t R, bool cplx, cudaStream_t st,
            long long& nl) {
  const long long rows = cplx ? (long long)R : 2 * (long long)R;
  const int ncol = cplx ? 2 * p : p;
  dim3 grid((unsigned)((rows + BM - 1) / BM), (unsigned)((ncol + BN - 1) / BN));
  if (cplx)
    mp_simt_kernel<double, true><<<grid, NT, 0, st>>>(X, Y, M, p, (long long)R);
  else
    mp_simt_kernel<double, false><<<grid, NT, 0, st>>>(X, Y, M, p, (long long)R);
  FCGLE_LAUNCHED(nl);
}

// FP32 REAL mode with larger register tiles: 128 x 128 block tile, 8 x 8
// outputs per thread, K in steps of 8 through double-buffered shared memory.
// Needs p % 8 == 0 and R % 8 == 0 (then a thread's 8 rows never straddle the
// re/im plane boundary and its stores are 16-byte vectors).
constexpr int FM = 128, FN = 128, FK = 8, FT = 256;

__global__ void __launch_bounds__(FT) mp_f32_kernel(const float* __restrict__ X, float* __restrict__ Y,
                                                    const float* __restrict__ B, int p, long long R) {
  __shared__ __align__(16) float As[2][FK][FM];
  __shared__ __align__(16) float Bs[2][FK][FN];
  const long long rows = 2 * R;
  const long long Rp = R * (long long)p;
  const long long row0 = (long long)blockIdx.x * FM;
  const int col0 = blockIdx.y * FN;
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;   // cols tx*8.., rows ty*8..
  const int lrow = tid >> 1, lk = (tid & 1) * 4;   // loader: one float4 of A and one of B

  float acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;

  auto load = [&](int k0, float4& a, float4& b) {
    const long long row = row0 + lrow;
    const int col = col0 + lrow;
    a = row < rows ? *reinterpret_cast<const float4*>(X + row * p + k0 + lk) : make_float4(0.f, 0.f, 0.f, 0.f);
    b = col < p ? *reinterpret_cast<const float4*>(B + (long long)col * p + k0 + lk) : make_float4(0.f, 0.f, 0.f, 0.f);
  };
  auto stash = [&](int buf, const float4& a, const float4& b) {
    As[buf][lk + 0][lrow] = a.x;
    As[buf][lk + 1][lrow] = a.y;
    As[buf][lk + 2][lrow] = a.z;
    As[buf][lk + 3][lrow] = a.w;
    Bs[buf][lk + 0][lrow] = b.x;
    Bs[buf][lk + 1][lrow] = b.y;
    Bs[buf][lk + 2][lrow] = b.z;
    Bs[buf][lk + 3][lrow] = b.w;
  };
  float4 ra, rb;
  load(0, ra, rb);
  stash(0, ra, rb);
  __syncthreads();
  int buf = 0;
  for (int k0 = 0; k0 < p; k0 += FK) {
    const bool more = k0 + FK < p;
    if (more) load(k0 + FK, ra, rb);
#pragma unroll
    for (int k = 0; k < FK; ++k) {
      float a[8], b[8];
      const float4 a0 = *reinterpret_cast<const float4*>(&As[buf][k][ty * 8]);
      const float4 a1 = *reinterpret_cast<const float4*>(&As[buf][k][ty * 8 + 4]);
      const float4 b0 = *reinterpret_cast<const float4*>(&Bs[buf][k][tx * 8]);
      const float4 b1 = *reinterpret_cast<const float4*>(&Bs[buf][k][tx * 8 + 4]);
      a[0] = a0.x; a[1] = a0.y; a[2] = a0.z; a[3] = a0.w; a[4] = a1.x; a[5] = a1.y; a[6] = a1.z; a[7] = a1.w;
      b[0] = b0.x; b[1] = b0.y; b[2] = b0.z; b[3] = b0.w; b[4] = b1.x; b[5] = b1.y; b[6] = b1.z; b[7] = b1.w;
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    if (more) {
      stash(buf ^ 1, ra, rb);
      __syncthreads();
      buf ^= 1;
    }
  }

  const long long r0 = row0 + ty * 8;
  if (r0 >= rows) return;
  const long long c = r0 >= R ? 1 : 0;
  const long long rr = r0 - c * R;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const int col = col0 + tx * 8 + j;
    if (col >= p) continue;
    float* dst = Y + c * Rp + (long long)col * R + rr;
    *reinterpret_cast<float4*>(dst) = make_float4(acc[0][j], acc[1][j], acc[2][j], acc[3][j]);
    *reinterpret_cast<float4*>(dst + 4) = make_float4(acc[4][j], acc[5][j], acc[6][j], acc[7][j]);
  }
}

void mp_f32(const float* X, float* Y, const float* M, int p, size_t R, cudaStream_t st, long long& nl) {
  const long long rows = 2 * (long long)R;
  if (p % 8 == 0 && R % 8 == 0) {
    dim3 grid((unsigned)((rows + FM - 1) / FM), (unsigned)((p + FN - 1) / FN));
    mp_f32_kernel<<<grid, FT, 0, st>>>(X, Y, M, p, (long long)R);
  } else {
    dim3 grid((unsigned)((rows + BM - 1) / BM), (unsigned)((p + BN - 1) / BN));
    mp_simt_kernel<float, false><<<grid, NT, 0, st>>>(X, Y, M, p, (long long)R);
  }
  FCGLE_LAUNCHED(nl);
}

}  // namespace fcgle
