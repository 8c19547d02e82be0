// The whitening product of eq. 4, A = K^{-1} R, for every (block, bin), as a
// batched complex GEMM on the FP32 SIMT cores, written column by column
// (A_cm[c][r] = A[r][c]) for the decompositions that work on A's columns.
//
// With R and K^{-1} Hermitian, A_cm = conj(R K^{-1}) as a row-major matrix:
//   conj(R K^{-1})[c][r] = sum_k conj(R[c][k]) conj(K^{-1}[k][r])
//                        = sum_k K^{-1}[r][k] R[k][c] = A[r][c],
// and C = R K^{-1} reads row k of both factors at step k
// (C[c][r] = sum_k conj(R[k][c]) K^{-1}[k][r]), so both operands come from
// shared memory as 32-byte row segments.
//
// One CTA per (bin, group of blocks): K^{-1} of the bin is staged once and
// serves the group; each R is staged in turn.  256 threads, each a 4 x 4 tile
// of C (16 x 16 tiles cover M <= 64): per step 4 complex values of each
// operand and 16 complex multiply-adds (64 FMA for 4 shared-memory loads).
#include "ssl_internal.cuh"

namespace ssl {
namespace {

constexpr int kWhitenThreads = 256;
constexpr int kWhitenGroup = 4;  // blocks per CTA sharing the bin's K^{-1}

// row stride (complex elements) of the staged matrices: a multiple of 4 >= M
__host__ __device__ inline int whiten_ld(int M) { return (M + 3) & ~3; }

__global__ void __launch_bounds__(kWhitenThreads)
whiten_kernel(const float2* __restrict__ R, const float2* __restrict__ Kinv,
              const float2* const* __restrict__ kinv_items, int nblk, int B, int M,
              float2* __restrict__ Acm) {
  extern __shared__ float4 wsm[];
  const int ld = whiten_ld(M);
  float2* Ks = reinterpret_cast<float2*>(wsm);
  float2* Rs = Ks + (size_t)M * ld;
  const int b = blockIdx.x, k0 = blockIdx.y * kWhitenGroup;
  const int tid = threadIdx.x;
  const int mt = ld / 4;                       // tiles per dimension
  const int tc = tid / 16, tr = tid % 16;      // tile: rows 4 tc.. of C, columns 4 tr..
  const bool active = tc < mt && tr < mt;
  const float2 zero = make_float2(0.f, 0.f);
  for (int kk = 0; kk < kWhitenGroup && k0 + kk < nblk; ++kk) {
    const int k = k0 + kk;
    const float2* Kb = kinv_items ? kinv_items[k] + (size_t)b * M * M
                                  : Kinv + (size_t)b * M * M;
    const size_t item = (size_t)k * B + b;
    const float2* Rb = R + item * M * M;
    __syncthreads();  // the previous item's reads of Rs (and Ks) are done
    if (kk == 0 || kinv_items)
      for (int e = tid; e < M * ld; e += kWhitenThreads) {
        const int r = e / ld, c = e - r * ld;
        Ks[e] = c < M ? __ldg(Kb + (size_t)r * M + c) : zero;
      }
    for (int e = tid; e < M * ld; e += kWhitenThreads) {
      const int r = e / ld, c = e - r * ld;
      Rs[e] = c < M ? __ldg(Rb + (size_t)r * M + c) : zero;
    }
    __syncthreads();
    if (active) {
      float2 acc[4][4];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = zero;
      const float4* rrow = reinterpret_cast<const float4*>(Rs) + 2 * tc;
      const float4* krow = reinterpret_cast<const float4*>(Ks) + 2 * tr;
      const int step = ld / 2;  // float4 per row
#pragma unroll 4
      for (int s = 0; s < M; ++s) {
        const float4 ra = rrow[(size_t)s * step], rb = rrow[(size_t)s * step + 1];
        const float4 ka = krow[(size_t)s * step], kb = krow[(size_t)s * step + 1];
        // conj(R[s][4 tc + i]) and K^{-1}[s][4 tr + j]
        const float2 rv[4] = {make_float2(ra.x, -ra.y), make_float2(ra.z, -ra.w),
                              make_float2(rb.x, -rb.y), make_float2(rb.z, -rb.w)};
        const float2 kv[4] = {make_float2(ka.x, ka.y), make_float2(ka.z, ka.w),
                              make_float2(kb.x, kb.y), make_float2(kb.z, kb.w)};
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            acc[i][j].x = fmaf(rv[i].x, kv[j].x, fmaf(-rv[i].y, kv[j].y, acc[i][j].x));
            acc[i][j].y = fmaf(rv[i].x, kv[j].y, fmaf(rv[i].y, kv[j].x, acc[i][j].y));
          }
      }
      // A_cm[c][r] = conj(C[c][r])
      float2* Ab = Acm + item * M * M;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int c = 4 * tc + i;
        if (c < M) {
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const int r = 4 * tr + j;
            if (r < M) Ab[(size_t)c * M + r] = make_float2(acc[i][j].x, -acc[i][j].y);
          }
        }
      }
    }
  }
}

}  // namespace

cudaError_t launch_whiten(const float2* R, const float2* Kinv, const float2* const* kinv_items,
                          int nblk, int B, int M, float2* Acm, cudaStream_t s) {
  if (nblk < 1 || B < 1 || M < 1 || M > SSL_MAX_M || (!Kinv && !kinv_items))
    return cudaErrorInvalidValue;
  const size_t smem = (size_t)2 * M * whiten_ld(M) * sizeof(float2);
  cudaError_t e = cudaFuncSetAttribute(whiten_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  const dim3 grid(B, (nblk + kWhitenGroup - 1) / kWhitenGroup);
  whiten_kernel<<<grid, kWhitenThreads, smem, s>>>(R, Kinv, kinv_items, nblk, B, M, Acm);
  return cudaGetLastError();
}

}  // namespace ssl
