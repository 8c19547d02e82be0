// MUSIC spectrum (eq. 5) on the SIMT cores in FP32, bin sum (eq. 6), and
// the steering norms |h^H h|.
//
//   y_i(d) = h_d^H e_i,  i = Ns..M-1           (the contraction H^H E_n)
//   P(d)   = |h_d|^2 / sum_i |y_i(d)|    (ABS)  or  / sum_i |y_i(d)|^2  (SQ)
//
// One CTA per (128 directions, bin, block).  E_n and the CTA's 128 steering
// rows are staged in shared memory (steering transposed so that the 128
// threads, one per direction, read consecutive words); each thread keeps 16
// running y_i in registers and folds them into the denominator chunk by chunk.
#include <float.h>

#include "ssl_internal.cuh"

namespace ssl {
namespace {

constexpr int kDirs = 128;   // directions per CTA = threads
constexpr int kChunk = 16;   // noise vectors per register chunk

// P of directions d0 .. d0 + 127 of one bin: Eb [M][M], Hb [D][M] and hn [D]
// of that bin, Pb [D].
__device__ __forceinline__ void spectrum_tile(const float2* __restrict__ Eb, int M, int Ns,
                                              const float2* __restrict__ Hb0,
                                              const float* __restrict__ hn, int D, int d0,
                                              int form, float* __restrict__ Pb, float2* sm) {
  float2* En = sm;             // [M][kLD]: En[m * kLD + i] = E[m][Ns + i]
  float2* Ht = sm + kLD * kLD; // [M][kDirs]: Ht[m * kDirs + t] = H[d0 + t][m]
  const int tid = threadIdx.x;
  const int N = M - Ns;
  for (int e = tid; e < M * N; e += kDirs) {
    const int m = e / N, i = e % N;
    En[m * kLD + i] = Eb[m * M + Ns + i];
  }
  const float2* Hb = Hb0 + (size_t)d0 * M;
  const int nd = min(kDirs, D - d0);
  for (int e = tid; e < kDirs * M; e += kDirs) {
    const int t = e / M, m = e % M;
    Ht[m * kDirs + t] = t < nd ? Hb[(size_t)t * M + m] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  float den = 0.f;
  for (int i0 = 0; i0 < N; i0 += kChunk) {
    float yr[kChunk], yi[kChunk];
#pragma unroll
    for (int c = 0; c < kChunk; ++c) yr[c] = yi[c] = 0.f;
    for (int m = 0; m < M; ++m) {
      const float2 h = Ht[m * kDirs + tid];
#pragma unroll
      for (int c = 0; c < kChunk; ++c) {
        const float2 e = En[m * kLD + i0 + c];  // broadcast
        // conj(h) * e
        yr[c] = fmaf(h.x, e.x, fmaf(h.y, e.y, yr[c]));
        yi[c] = fmaf(h.x, e.y, fmaf(-h.y, e.x, yi[c]));
      }
    }
#pragma unroll
    for (int c = 0; c < kChunk; ++c) {
      if (i0 + c < N) {
        const float s = yr[c] * yr[c] + yi[c] * yi[c];
        den += form == SSL_FORM_SQ ? s : sqrtf(s);
      }
    }
  }
  if (tid < nd) {
    const int d = d0 + tid;
    Pb[d] = hn[d] / fmaxf(den, FLT_MIN);
  }
}

__global__ void __launch_bounds__(kDirs)
spectrum_simt_kernel(const float2* __restrict__ E, int B, int M, int Ns,
                     const float2* __restrict__ H, const float* __restrict__ hnorm2, int D,
                     int form, float* __restrict__ P, const float2* const* __restrict__ H_items,
                     const float* const* __restrict__ hn_items) {
  extern __shared__ float2 sm[];
  const int w = blockIdx.y, k = blockIdx.z;
  const float2* Hb = (H_items ? H_items[k] : H) + (size_t)w * D * M;
  const float* hn = (hn_items ? hn_items[k] : hnorm2) + (size_t)w * D;
  spectrum_tile(E + ((size_t)k * B + w) * M * M, M, Ns, Hb, hn, D, blockIdx.x * kDirs, form,
                P + ((size_t)k * B + w) * D, sm);
}

// Mixed batch: blockIdx.y indexes the (item, bin) table.
__global__ void __launch_bounds__(kDirs)
spectrum_simt_mixed_kernel(const MixedItem* __restrict__ items, const int2* __restrict__ ctab,
                           int form) {
  extern __shared__ float2 sm[];
  const int2 cb = ctab[blockIdx.y];
  const MixedItem& it = items[cb.x];
  const int d0 = blockIdx.x * kDirs;
  if (d0 >= it.D) return;
  const int M = it.M, D = it.D, w = cb.y;
  spectrum_tile(it.E + (size_t)w * M * M, M, it.Ns, it.H + (size_t)w * D * M,
                it.hn + (size_t)w * D, D, d0, form, it.P + (size_t)w * D, sm);
}

__global__ void bin_sum_mixed_kernel(const MixedItem* __restrict__ items) {
  const MixedItem& it = items[blockIdx.y];
  const int d = blockIdx.x * blockDim.x + threadIdx.x;
  if (d >= it.D) return;
  const float* Pk = it.P + d;
  float s = 0.f;
  for (int w = 0; w < it.B; ++w) s += Pk[(size_t)w * it.D];
  it.Pbar[d] = s;
}

__global__ void bin_sum_kernel(const float* __restrict__ P, int B, int D,
                               float* __restrict__ Pbar) {
  const int d = blockIdx.x * blockDim.x + threadIdx.x;
  const int k = blockIdx.y;
  if (d >= D) return;
  const float* Pk = P + (size_t)k * B * D + d;
  float s = 0.f;
  for (int w = 0; w < B; ++w) s += Pk[(size_t)w * D];
  Pbar[(size_t)k * D + d] = s;
}

__global__ void hnorm2_kernel(const float2* __restrict__ H, int BD, int M,
                              float* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= BD) return;
  const float2* h = H + (size_t)i * M;
  float s = 0.f;
  for (int m = 0; m < M; ++m) s = fmaf(h[m].x, h[m].x, fmaf(h[m].y, h[m].y, s));
  out[i] = s;
}

}  // namespace

cudaError_t launch_spectrum_simt_mixed(const MixedItem* items, const int2* ctab, int n_ctab,
                                       int d_max, int form, cudaStream_t s) {
  if (n_ctab <= 0) return cudaSuccess;
  const size_t smem = ((size_t)kLD * kLD + (size_t)SSL_MAX_M * kDirs) * sizeof(float2);
  cudaError_t e = cudaFuncSetAttribute(spectrum_simt_mixed_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid(ceil_div(d_max, kDirs), n_ctab);
  spectrum_simt_mixed_kernel<<<grid, kDirs, smem, s>>>(items, ctab, form);
  return cudaGetLastError();
}

cudaError_t launch_bin_sum_mixed(const MixedItem* items, int n, int d_max, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  dim3 grid(ceil_div(d_max, 256), n);
  bin_sum_mixed_kernel<<<grid, 256, 0, s>>>(items);
  return cudaGetLastError();
}

cudaError_t launch_spectrum_simt(const float2* E, int nblk, int B, int M, int Ns, const float2* H,
                                 const float* hnorm2, int D, int form, float* P, cudaStream_t s,
                                 const float2* const* H_items, const float* const* hn_items) {
  const size_t smem = ((size_t)kLD * kLD + (size_t)M * kDirs) * sizeof(float2);
  cudaError_t e = cudaFuncSetAttribute(spectrum_simt_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid(ceil_div(D, kDirs), B, nblk);
  spectrum_simt_kernel<<<grid, kDirs, smem, s>>>(E, B, M, Ns, H, hnorm2, D, form, P,
                                                                 H_items, hn_items);
  return cudaGetLastError();
}

cudaError_t launch_bin_sum(const float* P, int nblk, int B, int D, float* Pbar, cudaStream_t s) {
  dim3 grid(ceil_div(D, 256), nblk);
  bin_sum_kernel<<<grid, 256, 0, s>>>(P, B, D, Pbar);
  return cudaGetLastError();
}

cudaError_t launch_hnorm2(const float2* H, int B, int D, int M, float* out, cudaStream_t s) {
  const int BD = B * D;
  hnorm2_kernel<<<ceil_div(BD, 256), 256, 0, s>>>(H, BD, M, out);
  return cudaGetLastError();
}

}  // namespace ssl
