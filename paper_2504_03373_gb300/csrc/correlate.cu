// Correlation, eq. 2-3 (AddCorrelation + NormalizeCorrelation, block-wise):
//   R[k][w] = (1/T) sum_{f<T} x_f x_f^H,  x_f = X[k][f][w][:].
// One CTA per (bin, block).  Frames are staged through shared memory in
// chunks of 32; each of the 256 threads owns a (MT/16) x (MT/16) register
// tile of R, so every staged element is reused MT/16 times from registers.
#include "ssl_internal.cuh"

namespace ssl {
namespace {

constexpr int kThreads = 256;
constexpr int kFrameChunk = 32;

template <int MT>
__global__ void __launch_bounds__(kThreads)
correlate_kernel(const float2* __restrict__ X, int T, int B, int M, float2* __restrict__ R,
                 float invT, const float2* const* __restrict__ X_items) {
  constexpr int RPT = MT / 16;  // rows (and columns) per thread
  __shared__ float2 xs[kFrameChunk][MT];
  const int b = blockIdx.x;
  const int k = blockIdx.y;
  const int tid = threadIdx.x;
  const int ti = tid / 16, tj = tid % 16;
  const float2* Xk = X_items ? X_items[k] : X + (size_t)k * T * B * M;

  float accr[RPT][RPT], acci[RPT][RPT];
#pragma unroll
  for (int a = 0; a < RPT; ++a)
#pragma unroll
    for (int c = 0; c < RPT; ++c) accr[a][c] = acci[a][c] = 0.f;

  for (int t0 = 0; t0 < T; t0 += kFrameChunk) {
    const int tc = min(kFrameChunk, T - t0);
    for (int e = tid; e < kFrameChunk * MT; e += kThreads) {
      const int f = e / MT, m = e % MT;
      float2 v = make_float2(0.f, 0.f);
      if (f < tc && m < M) v = Xk[((size_t)(t0 + f) * B + b) * M + m];
      xs[f][m] = v;
    }
    __syncthreads();
    for (int f = 0; f < tc; ++f) {
      float2 xi[RPT], xj[RPT];
#pragma unroll
      for (int a = 0; a < RPT; ++a) {
        xi[a] = xs[f][ti + 16 * a];
        xj[a] = xs[f][tj + 16 * a];
      }
#pragma unroll
      for (int a = 0; a < RPT; ++a)
#pragma unroll
        for (int c = 0; c < RPT; ++c) {
          // x_i * conj(x_j)
          accr[a][c] = fmaf(xi[a].x, xj[c].x, fmaf(xi[a].y, xj[c].y, accr[a][c]));
          acci[a][c] = fmaf(xi[a].y, xj[c].x, fmaf(-xi[a].x, xj[c].y, acci[a][c]));
        }
    }
    __syncthreads();
  }
  float2* Rb = R + ((size_t)k * B + b) * M * M;
#pragma unroll
  for (int a = 0; a < RPT; ++a)
#pragma unroll
    for (int c = 0; c < RPT; ++c) {
      const int i = ti + 16 * a, j = tj + 16 * c;
      if (i < M && j < M) Rb[i * M + j] = make_float2(accr[a][c] * invT, acci[a][c] * invT);
    }
}

}  // namespace

cudaError_t launch_correlate(const float2* X, int nblk, int T, int B, int M, float2* R,
                             cudaStream_t s, const float2* const* X_items) {
  dim3 grid(B, nblk);
  const float invT = 1.0f / (float)T;
  if (M <= 16)
    correlate_kernel<16><<<grid, kThreads, 0, s>>>(X, T, B, M, R, invT, X_items);
  else if (M <= 32)
    correlate_kernel<32><<<grid, kThreads, 0, s>>>(X, T, B, M, R, invT, X_items);
  else
    correlate_kernel<64><<<grid, kThreads, 0, s>>>(X, T, B, M, R, invT, X_items);
  return cudaGetLastError();
}

}  // namespace ssl
