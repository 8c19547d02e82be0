// Peak search over the direction grid (Sec. III-A, last step).
//
// Grid: n_el rows x n_az columns, d = e * n_az + a.  Neighbours: the 8
// surrounding points, azimuth wrapping around, elevation rows outside the
// grid dropped.  d is a peak iff for every neighbour n: Pbar[d] > Pbar[n],
// or Pbar[d] == Pbar[n] and d < n (a plateau yields its lowest index).  The
// Ns largest peaks are returned, ties to the lower index, missing ones as
// (-1, 0).  One CTA per block; the spectrum and the peak flags stay in
// shared memory and each selection is a block-wide arg-max.
#include "ssl_internal.cuh"

namespace ssl {
namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ bool better(float v1, int d1, float v2, int d2) {
  return v1 > v2 || (v1 == v2 && d1 < d2);
}

// The Ns largest peaks of Pk [n_el][n_az] into idx [Ns], val [Ns].
__device__ __forceinline__ void peaks_block(const float* __restrict__ Pk, int n_az, int n_el,
                                            int Ns, int32_t* __restrict__ idx,
                                            float* __restrict__ val, float* ps) {
  const int D = n_az * n_el;
  unsigned char* flag = reinterpret_cast<unsigned char*>(ps + D);
  __shared__ float wv[kThreads / 32];
  __shared__ int wd[kThreads / 32];
  const int tid = threadIdx.x;
  for (int d = tid; d < D; d += kThreads) ps[d] = Pk[d];
  __syncthreads();
  for (int d = tid; d < D; d += kThreads) {
    const int e = d / n_az, a = d % n_az;
    const float v = ps[d];
    bool ok = true;
    for (int de = -1; de <= 1 && ok; ++de) {
      const int ee = e + de;
      if (ee < 0 || ee >= n_el) continue;
      for (int da = -1; da <= 1; ++da) {
        const int aa = (a + da + n_az) % n_az;
        const int n = ee * n_az + aa;
        if (n == d) continue;
        if (!better(v, d, ps[n], n)) {
          ok = false;
          break;
        }
      }
    }
    flag[d] = ok ? 1 : 0;
  }
  __syncthreads();
  for (int s = 0; s < Ns; ++s) {
    float bv = 0.f;
    int bd = -1;
    for (int d = tid; d < D; d += kThreads)
      if (flag[d] && (bd < 0 || better(ps[d], d, bv, bd))) {
        bv = ps[d];
        bd = d;
      }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float ov = __shfl_xor_sync(0xffffffffu, bv, o);
      const int od = __shfl_xor_sync(0xffffffffu, bd, o);
      if (od >= 0 && (bd < 0 || better(ov, od, bv, bd))) {
        bv = ov;
        bd = od;
      }
    }
    if ((tid & 31) == 0) {
      wv[tid / 32] = bv;
      wd[tid / 32] = bd;
    }
    __syncthreads();
    if (tid == 0) {
      float fv = 0.f;
      int fd = -1;
      for (int w = 0; w < kThreads / 32; ++w)
        if (wd[w] >= 0 && (fd < 0 || better(wv[w], wd[w], fv, fd))) {
          fv = wv[w];
          fd = wd[w];
        }
      idx[s] = fd;
      val[s] = fd >= 0 ? fv : 0.f;
      if (fd >= 0) flag[fd] = 0;
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kThreads)
peaks_kernel(const float* __restrict__ Pbar, int n_az, int n_el, int Ns,
             int32_t* __restrict__ idx, float* __restrict__ val) {
  extern __shared__ float ps[];
  const int k = blockIdx.x;
  peaks_block(Pbar + (size_t)k * n_az * n_el, n_az, n_el, Ns, idx + (size_t)k * Ns,
              val + (size_t)k * Ns, ps);
}

// Mixed batch: one CTA per item; also the item's status (largest bin status).
__global__ void __launch_bounds__(kThreads)
peaks_mixed_kernel(const MixedItem* __restrict__ items) {
  extern __shared__ float ps[];
  const MixedItem& it = items[blockIdx.x];
  peaks_block(it.Pbar, it.n_az, it.n_el, it.Ns, it.idx, it.val, ps);
  if (it.status && threadIdx.x < 32) {
    int32_t m = 0;
    for (int w = threadIdx.x; w < it.B; w += 32) m = max(m, it.bst[w]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (threadIdx.x == 0) *it.status = m;
  }
}

__global__ void status_max_kernel(const int32_t* __restrict__ st, int nblk, int B,
                                  int32_t* __restrict__ out) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nblk) return;
  int32_t m = 0;
  for (int w = 0; w < B; ++w) m = max(m, st[(size_t)k * B + w]);
  out[k] = m;
}

}  // namespace

cudaError_t launch_peaks_mixed(const MixedItem* items, int n, int d_max, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const size_t smem = (size_t)d_max * sizeof(float) + (size_t)d_max;
  cudaError_t e = cudaFuncSetAttribute(peaks_mixed_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  peaks_mixed_kernel<<<n, kThreads, smem, s>>>(items);
  return cudaGetLastError();
}

cudaError_t launch_status_max(const int32_t* bin_status, int nblk, int B, int32_t* out,
                              cudaStream_t s) {
  status_max_kernel<<<ceil_div(nblk, 128), 128, 0, s>>>(bin_status, nblk, B, out);
  return cudaGetLastError();
}

cudaError_t launch_peaks(const float* Pbar, int nblk, int n_az, int n_el, int Ns, int32_t* idx,
                         float* val, cudaStream_t s) {
  const int D = n_az * n_el;
  const size_t smem = (size_t)D * sizeof(float) + (size_t)D;
  cudaError_t e =
      cudaFuncSetAttribute(peaks_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  peaks_kernel<<<nblk, kThreads, smem, s>>>(Pbar, n_az, n_el, Ns, idx, val);
  return cudaGetLastError();
}

}  // namespace ssl
