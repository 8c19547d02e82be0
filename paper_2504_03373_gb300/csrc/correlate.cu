// Correlation, eq. 2-3 (AddCorrelation + NormalizeCorrelation, block-wise):
//   R[k][w] = (1/T) sum_{f<T} x_f x_f^H,  x_f = X[k][f][w][:].
// One CTA of 128 threads per (bin, block).  R is Hermitian, so only its
// 4 x 4 tiles on and above the diagonal are accumulated (ceil(M/4) (ceil(M/4)
// + 1) / 2 of them: 120 at M = 60, one per thread), and R is written from
// their upper triangles, mirrored (exactly Hermitian, real diagonal).  The
// frames stream through a two-stage shared-memory ring of 16-frame chunks
// filled by asynchronous copies, so the next chunk's loads overlap this
// chunk's products (16-byte copies when M is even and X 16-byte aligned, so
// that every frame row starts on a 16-byte boundary); each thread reads its 4 + 4 staged values
// per frame as 16-byte loads.  A staged row keeps the two halves of each
// 4-element group apart (elements 4g, 4g + 1 at 2g; 4g + 2, 4g + 3 at
// 32 + 2g), so the 16-byte loads of 8 lanes for 8 consecutive groups fall in
// 32 different banks.  When every tile fits one round (M <= 60), R leaves
// through the same shared memory in passes of whole rows, so that the
// mirrored lower triangle is stored coalesced too.
#include "ssl_internal.cuh"

namespace ssl {
namespace {

constexpr int kThreads = 128;
constexpr int kChunk = 16;  // frames per stage
constexpr int kLD = 64;     // staged row length (float2), M <= 64
constexpr int kHalf = kLD / 2;

// staged position of element m of a frame row
__device__ __forceinline__ int spos(int m) {
  return ((m >> 1) & 1) * kHalf + ((m >> 2) << 1) + (m & 1);
}

__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(
                   static_cast<uint32_t>(__cvta_generic_to_shared(dst))),
               "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(
                   static_cast<uint32_t>(__cvta_generic_to_shared(dst))),
               "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// (ti, tj), ti <= tj, of upper-triangle tile q (column-packed)
__device__ __forceinline__ void tile_index(int q, int& ti, int& tj) {
  int r = (int)((sqrtf(8.f * (float)q + 1.f) - 1.f) * 0.5f);
  if (r * (r + 1) / 2 > q) --r;
  if ((r + 1) * (r + 2) / 2 <= q) ++r;
  tj = r;
  ti = q - r * (r + 1) / 2;
}

// R of bin b from the frames Xk [T][B][M] into Rb [M][M].
__device__ __forceinline__ void correlate_bin(const float2* __restrict__ Xk, int T, int B, int M,
                                              int b, float2* __restrict__ Rb, float invT,
                                              float2 (*xs)[kChunk][kLD]) {
  const int tid = threadIdx.x;
  const int nt = (M + 3) / 4;
  const int ntiles = nt * (nt + 1) / 2;
  // rows M .. 4 nt - 1 of the staged frames are read by edge tiles: zero
  for (int e = tid; e < 2 * kChunk * kLD; e += kThreads) {
    const int m = e % kLD;
    if (m >= M) (&xs[0][0][0])[e - m + spos(m)] = make_float2(0.f, 0.f);
  }
  const int nchunks = (T + kChunk - 1) / kChunk;
  // thread t copies element m = t % 64 of frames t / 64, t / 64 + 2, ...
  // (16 bytes, elements m and m + 1, when every row is 16-byte aligned; else
  // 8 bytes)
  const bool even = (M & 1) == 0 && (reinterpret_cast<uintptr_t>(Xk) & 15) == 0;
  auto stage = [&](int c) {
    const int t0 = c * kChunk, tc = min(kChunk, T - t0);
    float2(*dst)[kLD] = xs[c & 1];
    if (even) {
      const int m = 2 * (tid & 31);
      if (m < M)
        for (int f = tid >> 5; f < tc; f += kThreads / 32)
          cp_async16(&dst[f][spos(m)], Xk + ((size_t)(t0 + f) * B + b) * M + m);
    } else {
      const int m = tid & 63;
      if (m < M)
        for (int f = tid >> 6; f < tc; f += kThreads / 64)
          cp_async8(&dst[f][spos(m)], Xk + ((size_t)(t0 + f) * B + b) * M + m);
    }
    cp_async_commit();
  };
  stage(0);
  for (int q0 = 0; q0 < ntiles; q0 += kThreads) {
    const int q = q0 + tid;
    const bool act = q < ntiles;
    int ti = 0, tj = 0;
    if (act) tile_index(q, ti, tj);
    float2 acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[a][c] = make_float2(0.f, 0.f);
    for (int c = 0; c < nchunks; ++c) {
      if (q0 > 0 && c == 0) {
        // a second tile round (M > 60) restarts the frame stream
        __syncthreads();
        stage(0);
      }
      if (c + 1 < nchunks) {
        stage(c + 1);
        cp_async_wait<1>();
      } else {
        cp_async_wait<0>();
      }
      __syncthreads();
      const int tc = min(kChunk, T - c * kChunk);
      const float2(*x)[kLD] = xs[c & 1];
      if (act) {
        for (int f = 0; f < tc; ++f) {
          const float4 i01 = *reinterpret_cast<const float4*>(&x[f][2 * ti]);
          const float4 i23 = *reinterpret_cast<const float4*>(&x[f][kHalf + 2 * ti]);
          const float4 j01 = *reinterpret_cast<const float4*>(&x[f][2 * tj]);
          const float4 j23 = *reinterpret_cast<const float4*>(&x[f][kHalf + 2 * tj]);
          const float2 xi[4] = {make_float2(i01.x, i01.y), make_float2(i01.z, i01.w),
                                make_float2(i23.x, i23.y), make_float2(i23.z, i23.w)};
          const float2 xj[4] = {make_float2(j01.x, j01.y), make_float2(j01.z, j01.w),
                                make_float2(j23.x, j23.y), make_float2(j23.z, j23.w)};
#pragma unroll
          for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int cc = 0; cc < 4; ++cc) {
              // x_i * conj(x_j)
              acc[a][cc].x = fmaf(xi[a].x, xj[cc].x, fmaf(xi[a].y, xj[cc].y, acc[a][cc].x));
              acc[a][cc].y = fmaf(xi[a].y, xj[cc].x, fmaf(-xi[a].x, xj[cc].y, acc[a][cc].y));
            }
        }
      }
      __syncthreads();  // stage c & 1 is refilled by the next iteration
    }
    if (ntiles <= kThreads) {
      // one tile round: R leaves through the ring in passes of P whole rows
      // (row stride M + 2), each pass stored as one contiguous range of Rb
      float2* rs = &xs[0][0][0];
      const int RLD = M + 2, P = (2 * kChunk * kLD) / RLD;
      for (int r0 = 0; r0 < M; r0 += P) {
        const int r1 = min(M, r0 + P);
        __syncthreads();  // the frame loop's reads, or the previous pass's copy, are done
        if (act) {
#pragma unroll
          for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int cc = 0; cc < 4; ++cc) {
              const int i = 4 * ti + a, j = 4 * tj + cc;
              if (i > j || j >= M) continue;  // i <= j < M from here
              const float re = acc[a][cc].x * invT, im = i == j ? 0.f : acc[a][cc].y * invT;
              if (i >= r0 && i < r1) rs[(i - r0) * RLD + j] = make_float2(re, im);
              if (i != j && j >= r0 && j < r1) rs[(j - r0) * RLD + i] = make_float2(re, -im);
            }
        }
        __syncthreads();
        const int n = (r1 - r0) * M;
        for (int e = tid; e < n; e += kThreads) {
          const int r = e / M, c = e - r * M;
          Rb[r0 * M + e] = rs[r * RLD + c];
        }
      }
    } else if (act) {
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int cc = 0; cc < 4; ++cc) {
          const int i = 4 * ti + a, j = 4 * tj + cc;
          if (i > j || j >= M) continue;  // i <= j < M from here
          const float re = acc[a][cc].x * invT, im = i == j ? 0.f : acc[a][cc].y * invT;
          Rb[i * M + j] = make_float2(re, im);
          if (i != j) Rb[j * M + i] = make_float2(re, -im);
        }
    }
  }
}

__global__ void __launch_bounds__(kThreads)
correlate_kernel(const float2* __restrict__ X, int T, int B, int M, float2* __restrict__ R,
                 float invT, const float2* const* __restrict__ X_items) {
  __shared__ __align__(16) float2 xs[2][kChunk][kLD];
  const int b = blockIdx.x, k = blockIdx.y;
  const float2* Xk = X_items ? X_items[k] : X + (size_t)k * T * B * M;
  correlate_bin(Xk, T, B, M, b, R + ((size_t)k * B + b) * M * M, invT, xs);
}

// Mixed batch: one CTA per (item, bin).
__global__ void __launch_bounds__(kThreads)
correlate_mixed_kernel(const MixedItem* __restrict__ items, const int2* __restrict__ ctab) {
  __shared__ __align__(16) float2 xs[2][kChunk][kLD];
  const int2 cb = ctab[blockIdx.x];
  const MixedItem& it = items[cb.x];
  const int M = it.M, T = it.T, B = it.B, b = cb.y;
  correlate_bin(it.X, T, B, M, b, it.R + (size_t)b * M * M, 1.0f / (float)T, xs);
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
  if (nblk <= 0 || B <= 0) return cudaSuccess;
  dim3 grid(B, nblk);
  correlate_kernel<<<grid, kThreads, 0, s>>>(X, T, B, M, R, 1.0f / (float)T, X_items);
  return cudaGetLastError();
}

}  // namespace ssl
