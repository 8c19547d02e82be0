// Batched complex M x M products C[k][b] = op(A) op(B), op = identity or
// conjugate transpose, each factor either per (block, bin) or shared by the
// blocks of a bin.  Used around the decomposition: E_prev^H K^{-1} (warm
// start of a stream), R W^H and W^H Y (the generalised eigenproblem, with
// W = L^{-1} from the Cholesky factor of K).  One CTA per (bin, block); both
// factors staged in shared memory (stride MT + 1) in the orientation the
// product reads; each of the 256 threads owns an (MT/16)^2 register tile.
#include "ssl_internal.cuh"

namespace ssl {
namespace {

constexpr int kThreads = 256;

template <int MT>
__global__ void __launch_bounds__(kThreads)
cgemm_kernel(const float2* __restrict__ A, int a_item, int a_h, const float2* __restrict__ Bm,
             int b_item, int b_h, int B, int M, float2* __restrict__ C) {
  constexpr int RPT = MT / 16, LD = MT + 1;
  extern __shared__ float2 sm[];
  float2* As = sm;            // As[i][m] = op(A)[i][m]
  float2* Bs = sm + MT * LD;  // Bs[m][j] = op(B)[m][j]
  const int b = blockIdx.x, k = blockIdx.y;
  const size_t mm = (size_t)M * M;
  const size_t item = (size_t)k * B + b;
  const float2* Ab = A + (a_item ? item : (size_t)b) * mm;
  const float2* Bb = Bm + (b_item ? item : (size_t)b) * mm;
  for (int e = threadIdx.x; e < M * M; e += kThreads) {
    const int r = e / M, c = e % M;
    const float2 a = Ab[e], bb = Bb[e];
    if (a_h)
      As[c * LD + r] = make_float2(a.x, -a.y);
    else
      As[r * LD + c] = a;
    if (b_h)
      Bs[c * LD + r] = make_float2(bb.x, -bb.y);
    else
      Bs[r * LD + c] = bb;
  }
  __syncthreads();
  const int ti = threadIdx.x / 16, tj = threadIdx.x % 16;
  float2 acc[RPT][RPT];
#pragma unroll
  for (int a = 0; a < RPT; ++a)
#pragma unroll
    for (int c = 0; c < RPT; ++c) acc[a][c] = make_float2(0.f, 0.f);
  for (int m = 0; m < M; ++m) {
    float2 x[RPT], y[RPT];
#pragma unroll
    for (int a = 0; a < RPT; ++a) {
      const int i = ti + 16 * a, j = tj + 16 * a;
      x[a] = i < M ? As[i * LD + m] : make_float2(0.f, 0.f);
      y[a] = j < M ? Bs[m * LD + j] : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int a = 0; a < RPT; ++a)
#pragma unroll
      for (int c = 0; c < RPT; ++c) {
        acc[a][c].x = fmaf(x[a].x, y[c].x, fmaf(-x[a].y, y[c].y, acc[a][c].x));
        acc[a][c].y = fmaf(x[a].x, y[c].y, fmaf(x[a].y, y[c].x, acc[a][c].y));
      }
  }
  float2* Cb = C + item * mm;
#pragma unroll
  for (int a = 0; a < RPT; ++a)
#pragma unroll
    for (int c = 0; c < RPT; ++c) {
      const int i = ti + 16 * a, j = tj + 16 * c;
      if (i < M && j < M) Cb[(size_t)i * M + j] = acc[a][c];
    }
}

template <int MT>
cudaError_t launch_mt(const float2* A, bool a_item, bool a_h, const float2* Bm, bool b_item,
                      bool b_h, int nblk, int B, int M, float2* C, cudaStream_t s) {
  const size_t smem = 2 * (size_t)MT * (MT + 1) * sizeof(float2);
  cudaError_t e = cudaFuncSetAttribute(cgemm_kernel<MT>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  cgemm_kernel<MT><<<dim3(B, nblk), kThreads, smem, s>>>(A, a_item, a_h, Bm, b_item, b_h, B, M,
                                                          C);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_cgemm(const float2* A, bool a_item, bool a_h, const float2* Bm, bool b_item,
                         bool b_h, int nblk, int B, int M, float2* C, cudaStream_t s) {
  if (M <= 16) return launch_mt<16>(A, a_item, a_h, Bm, b_item, b_h, nblk, B, M, C, s);
  if (M <= 32) return launch_mt<32>(A, a_item, a_h, Bm, b_item, b_h, nblk, B, M, C, s);
  return launch_mt<64>(A, a_item, a_h, Bm, b_item, b_h, nblk, B, M, C, s);
}

}  // namespace ssl
