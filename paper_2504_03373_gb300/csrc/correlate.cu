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

// R of bin b from the frames Xk [T][B][M] into Rb [M][M]; MT = M rounded up
// to 16, 32 or 64.
template <int MT>
__device__ __forceinline__ void correlate_bin(const float2* __restrict__ Xk, int T, int B, int M,
                                              int b, float2* __restrict__ Rb, float invT,
                                              float2 (*xs)[MT]) {
  constexpr int RPT = MT / 16;  // rows (and columns) per thread
  const int tid = threadIdx.x;
  const int ti = tid / 16, tj = tid % 16;

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
#pragma unroll
  for (int a = 0; a < RPT; ++a)
#pragma unroll
    for (int c = 0; c < RPT; ++c) {
      const int i = ti + 16 * a, j = tj + 16 * c;
      if (i < M && j < M) Rb[i * M + j] = make_float2(accr[a][c] * invT, acci[a][c] * invT);
    }
}

template <int MT>
__global__ void __launch_bounds__(kThreads)
correlate_kernel(const float2* __restrict__ X, int T, int B, int M, float2* __restrict__ R,
                 float invT, const float2* const* __restrict__ X_items) {
  __shared__ float2 xs[kFrameChunk][MT];
  const int b = blockIdx.x, k = blockIdx.y;
  const float2* Xk = X_items ? X_items[k] : X + (size_t)k * T * B * M;
  correlate_bin<MT>(Xk, T, B, M, b, R + ((size_t)k * B + b) * M * M, invT, xs);
}

// Mixed batch: one CTA per (item, bin), the size class chosen per CTA.
__global__ void __launch_bounds__(kThreads)
correlate_mixed_kernel(const MixedItem* __restrict__ items, const int2* __restrict__ ctab) {
  __shared__ float2 xs[kFrameChunk][64];
  const int2 cb = ctab[blockIdx.x];
  const MixedItem& it = items[cb.x];
  const int M = it.M, T = it.T, B = it.B, b = cb.y;
  const float invT = 1.0f / (float)T;
  float2* Rb = it.R + (size_t)b * M * M;
  if (M <= 16)
    correlate_bin<16>(it.X, T, B, M, b, Rb, invT, reinterpret_cast<float2(*)[16]>(&xs[0][0]));
  else if (M <= 32)
    correlate_bin<32>(it.X, T, B, M, b, Rb, invT, reinterpret_cast<float2(*)[32]>(&xs[0][0]));
  else
    correlate_bin<64>(it.X, T, B, M, b, Rb, invT, xs);
}

}  // namespace

cudaError_t launch_correlate_mixed(const MixedItem* items, const int2* ctab, int n_ctab,
                                   cudaStream_t s) {
  if (n_ctab <= 0) return cudaSuccess;
  correlate_mixed_kernel<<<n_ctab, kThreads, 0, s>>>(items, ctab);
  return cudaGetLastError();
}

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
