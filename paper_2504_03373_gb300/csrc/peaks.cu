// Peak search over the direction grid (Sec. III-A, last step), or over a
// direction set with explicit neighbour lists (the same rule, any set).
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

template <class T>
__device__ __forceinline__ bool better(T v1, int d1, T v2, int d2) {
  return v1 > v2 || (v1 == v2 && d1 < d2);
}

// The Ns largest peaks of Pk [D] into idx [Ns], val [Ns]; is_peak(d, ps)
// decides the peak rule from the spectrum staged in shared memory.  With a
// search range `in` (Sec. III-A: peaks are searched between theta_min and
// theta_max; in[d] != 0 inside it), only directions inside it may be peaks;
// their test still sees every neighbour.
template <class T, class IsPeak>
__device__ __forceinline__ void peaks_block(const T* __restrict__ Pk, int D, int Ns,
                                            int32_t* __restrict__ idx, T* __restrict__ val,
                                            T* ps, IsPeak is_peak,
                                            const uint8_t* __restrict__ in = nullptr) {
  unsigned char* flag = reinterpret_cast<unsigned char*>(ps + D);
  __shared__ T wv[kThreads / 32];
  __shared__ int wd[kThreads / 32];
  const int tid = threadIdx.x;
  for (int d = tid; d < D; d += kThreads) ps[d] = Pk[d];
  __syncthreads();
  for (int d = tid; d < D; d += kThreads)
    flag[d] = (in == nullptr || in[d] != 0) && is_peak(d, ps) ? 1 : 0;
  __syncthreads();
  for (int s = 0; s < Ns; ++s) {
    T bv = 0;
    int bd = -1;
    for (int d = tid; d < D; d += kThreads)
      if (flag[d] && (bd < 0 || better(ps[d], d, bv, bd))) {
        bv = ps[d];
        bd = d;
      }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const T ov = __shfl_xor_sync(0xffffffffu, bv, o);
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
      T fv = 0;
      int fd = -1;
      for (int w = 0; w < kThreads / 32; ++w)
        if (wd[w] >= 0 && (fd < 0 || better(wv[w], wd[w], fv, fd))) {
          fv = wv[w];
          fd = wd[w];
        }
      idx[s] = fd;
      val[s] = fd >= 0 ? fv : T(0);
      if (fd >= 0) flag[fd] = 0;
    }
    __syncthreads();
  }
}

// Grid rule: the 8 surrounding points, azimuth wrapping, rows outside the
// grid dropped.
struct GridPeak {
  int n_az, n_el;
  template <class T>
  __device__ __forceinline__ bool operator()(int d, const T* ps) const {
    const int e = d / n_az, a = d % n_az;
    const T v = ps[d];
    for (int de = -1; de <= 1; ++de) {
      const int ee = e + de;
      if (ee < 0 || ee >= n_el) continue;
      for (int da = -1; da <= 1; ++da) {
        const int n = ee * n_az + (a + da + n_az) % n_az;
        if (n != d && !better(v, d, ps[n], n)) return false;
      }
    }
    return true;
  }
};

// Neighbour lists (compressed rows, indices checked on the host when the
// lists were attached): every listed neighbour n != d.
struct ListPeak {
  const int32_t* ptr;
  const int32_t* nbr;
  int D;
  unsigned* flags;  // bounds-checked build: raised by an index outside [0, D)
  template <class T>
  __device__ __forceinline__ bool operator()(int d, const T* ps) const {
    const T v = ps[d];
    for (int j = __ldg(ptr + d), end = __ldg(ptr + d + 1); j < end; ++j) {
      const int n = __ldg(nbr + j);
      if (!SSL_IN_BOUNDS(n >= 0 && n < D, flags)) continue;
      if (n != d && !better(v, d, ps[n], n)) return false;
    }
    return true;
  }
};

template <class T>
__global__ void __launch_bounds__(kThreads)
peaks_kernel(const T* __restrict__ Pbar, int n_az, int n_el, int Ns, int32_t* __restrict__ idx,
             T* __restrict__ val, const uint8_t* __restrict__ in) {
  extern __shared__ __align__(16) unsigned char peaks_smem[];
  T* ps = reinterpret_cast<T*>(peaks_smem);
  const int k = blockIdx.x;
  const int D = n_az * n_el;
  peaks_block(Pbar + (size_t)k * D, D, Ns, idx + (size_t)k * Ns, val + (size_t)k * Ns, ps,
              GridPeak{n_az, n_el}, in);
}

template <class T>
__global__ void __launch_bounds__(kThreads)
peaks_nbr_kernel(const T* __restrict__ Pbar, int D, const int32_t* __restrict__ ptr,
                 const int32_t* __restrict__ nbr, int Ns, int32_t* __restrict__ idx,
                 T* __restrict__ val, unsigned* flags, const uint8_t* __restrict__ in) {
  extern __shared__ __align__(16) unsigned char peaks_smem[];
  T* ps = reinterpret_cast<T*>(peaks_smem);
  const int k = blockIdx.x;
  peaks_block(Pbar + (size_t)k * D, D, Ns, idx + (size_t)k * Ns, val + (size_t)k * Ns, ps,
              ListPeak{ptr, nbr, D, flags}, in);
}

// Per-item neighbour lists and search ranges (serving: the items of one shape
// class may belong to arrays with different direction sets of the same size,
// or different ranges).  ptrs == nullptr: the n_el x n_az grid for every item.
__global__ void __launch_bounds__(kThreads)
peaks_items_kernel(const float* __restrict__ Pbar, int D, int n_az, int n_el,
                   const int32_t* const* __restrict__ ptrs,
                   const int32_t* const* __restrict__ idxs,
                   const uint8_t* const* __restrict__ ranges, int Ns,
                   int32_t* __restrict__ idx, float* __restrict__ val, unsigned* flags) {
  extern __shared__ __align__(16) unsigned char peaks_smem[];
  float* ps = reinterpret_cast<float*>(peaks_smem);
  const int k = blockIdx.x;
  const uint8_t* in = ranges ? ranges[k] : nullptr;
  if (ptrs)
    peaks_block(Pbar + (size_t)k * D, D, Ns, idx + (size_t)k * Ns, val + (size_t)k * Ns, ps,
                ListPeak{ptrs[k], idxs[k], D, flags}, in);
  else
    peaks_block(Pbar + (size_t)k * D, D, Ns, idx + (size_t)k * Ns, val + (size_t)k * Ns, ps,
                GridPeak{n_az, n_el}, in);
}

// Mixed batch: one CTA per item; also the item's status (largest bin status).
__global__ void __launch_bounds__(kThreads)
peaks_mixed_kernel(const MixedItem* __restrict__ items) {
  extern __shared__ __align__(16) unsigned char peaks_smem[];
  float* ps = reinterpret_cast<float*>(peaks_smem);
  const MixedItem& it = items[blockIdx.x];
  if (it.n_el == 0)  // a direction set with neighbour lists
    peaks_block(it.Pbar, it.D, it.Ns, it.idx, it.val, ps,
                ListPeak{it.nbr_ptr, it.nbr_idx, it.D, nullptr}, it.range);
  else
    peaks_block(it.Pbar, it.D, it.Ns, it.idx, it.val, ps, GridPeak{it.n_az, it.n_el}, it.range);
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

cudaError_t launch_peaks_items(const float* Pbar, int nblk, int D, int n_az, int n_el,
                               const int32_t* const* nbr_ptrs, const int32_t* const* nbr_idxs,
                               const uint8_t* const* ranges, int Ns, int32_t* idx, float* val,
                               cudaStream_t s, unsigned* flags) {
  if (nblk <= 0) return cudaSuccess;
  const size_t smem = (size_t)D * sizeof(float) + (size_t)D;
  cudaError_t e = cudaFuncSetAttribute(peaks_items_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  peaks_items_kernel<<<nblk, kThreads, smem, s>>>(Pbar, D, n_az, n_el, nbr_ptrs, nbr_idxs, ranges,
                                                  Ns, idx, val, flags);
  return cudaGetLastError();
}

cudaError_t launch_status_max(const int32_t* bin_status, int nblk, int B, int32_t* out,
                              cudaStream_t s) {
  status_max_kernel<<<ceil_div(nblk, 128), 128, 0, s>>>(bin_status, nblk, B, out);
  return cudaGetLastError();
}

namespace {
template <class T>
cudaError_t peaks_grid(const T* Pbar, int nblk, int n_az, int n_el, int Ns, int32_t* idx, T* val,
                       cudaStream_t s, const uint8_t* in) {
  const int D = n_az * n_el;
  const size_t smem = (size_t)D * sizeof(T) + (size_t)D;
  cudaError_t e = cudaFuncSetAttribute(peaks_kernel<T>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  peaks_kernel<T><<<nblk, kThreads, smem, s>>>(Pbar, n_az, n_el, Ns, idx, val, in);
  return cudaGetLastError();
}
template <class T>
cudaError_t peaks_list(const T* Pbar, int nblk, int D, const int32_t* nbr_ptr,
                       const int32_t* nbr_idx, int Ns, int32_t* idx, T* val, cudaStream_t s,
                       unsigned* flags, const uint8_t* in) {
  const size_t smem = (size_t)D * sizeof(T) + (size_t)D;
  cudaError_t e = cudaFuncSetAttribute(peaks_nbr_kernel<T>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  peaks_nbr_kernel<T><<<nblk, kThreads, smem, s>>>(Pbar, D, nbr_ptr, nbr_idx, Ns, idx, val,
                                                     flags, in);
  return cudaGetLastError();
}
}  // namespace

cudaError_t launch_peaks(const float* Pbar, int nblk, int n_az, int n_el, int Ns, int32_t* idx,
                         float* val, cudaStream_t s, const uint8_t* in) {
  return peaks_grid(Pbar, nblk, n_az, n_el, Ns, idx, val, s, in);
}
cudaError_t launch_peaks(const double* Pbar, int nblk, int n_az, int n_el, int Ns, int32_t* idx,
                         double* val, cudaStream_t s, const uint8_t* in) {
  return peaks_grid(Pbar, nblk, n_az, n_el, Ns, idx, val, s, in);
}

cudaError_t launch_peaks_nbr(const float* Pbar, int nblk, int D, const int32_t* nbr_ptr,
                             const int32_t* nbr_idx, int Ns, int32_t* idx, float* val,
                             cudaStream_t s, unsigned* flags, const uint8_t* in) {
  return peaks_list(Pbar, nblk, D, nbr_ptr, nbr_idx, Ns, idx, val, s, flags, in);
}
cudaError_t launch_peaks_nbr(const double* Pbar, int nblk, int D, const int32_t* nbr_ptr,
                             const int32_t* nbr_idx, int Ns, int32_t* idx, double* val,
                             cudaStream_t s, unsigned* flags, const uint8_t* in) {
  return peaks_list(Pbar, nblk, D, nbr_ptr, nbr_idx, Ns, idx, val, s, flags, in);
}

}  // namespace ssl
