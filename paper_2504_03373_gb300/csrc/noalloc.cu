// ssl_gsvd_noalloc: the generalised SVD of ssl_gsvd for callers that must not
// allocate device memory.
//
// Who needs it: a real-time audio thread (a robot's or an array's audition
// loop) cannot afford cudaMalloc on its per-block path, because an allocation
// may synchronise the whole device and take far longer than the block's
// deadline; and a host framework that loads this library as a plug-in may
// own the device memory budget itself and forbid libraries from allocating
// behind its back.  Such callers still pass their own inputs and outputs; the
// scratch the decomposition needs, the per-bin inverse of the noise
// correlation and the per-bin outcome of that inversion, lives here in a
// fixed array compiled into the library.
//
// The array holds kMaxElems complex values (8 MiB) and is resident on every
// GPU that loads the library until the process exits.  Every call on a device
// shares it and it keeps the last call's contents; nothing in it has to start
// at zero (K^{-1} and the per-bin inversion status are fully written before
// they are read).  Calls whose work overlaps on the GPU, e.g. on two streams
// at once, race on the array.
//
// There is no context here, hence no sticky flag word a caller could read:
// the caller's per-(block, bin) status array is the only error channel, so it
// is required, and a bin whose K could not be inverted reports that outcome
// (SSL_E_NOT_PD or SSL_E_NONFINITE) there in every block.
#include <mutex>

#include "ssl_internal.cuh"

namespace {

// K^{-1} (B * M * M complex values) followed by the per-bin inversion status
// (B int32, two to a complex slot) must fit in kMaxElems complex values.
constexpr size_t kMaxElems = size_t(1) << 20;
constexpr int kMaxDevices = 64;

// The scratch, followed by one word for the kernels' sticky flags (written by
// the kernels, never read: the per-bin status carries every outcome).
static __device__ __align__(256) float2 g_noalloc_scratch[kMaxElems + 32];

// Complex slots a request needs: K^{-1} and the per-bin status words.
size_t scratch_elems(int B, int M) { return (size_t)B * M * M + ((size_t)B + 1) / 2; }

// A bin whose K^{-1} failed carries that status in every block (it replaces
// the decomposition's status, which describes a zeroed matrix).
__global__ void fold_inverse_status(const int32_t* __restrict__ kinv_status, int nblk, int B,
                                    int32_t* __restrict__ status) {
  const size_t n = (size_t)nblk * B;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    const int32_t k = kinv_status[i % B];
    if (k != 0) status[i] = k;
  }
}

std::mutex g_mu;
float2* g_dev_ptr[kMaxDevices] = {};  // device address of the array, per device

}  // namespace

extern "C" ssl_status ssl_gsvd_noalloc(const float* R, const float* K, int nblk, int B, int M,
                                       const ssl_jacobi_opts* opts, float* sigma, float* E,
                                       int32_t* status, void* stream) {
  if (!R || !K || !sigma || !E || !status || nblk < 1 || B < 1 || M < 1 || M > SSL_MAX_M)
    return SSL_E_INVALID_ARG;
  if (scratch_elems(B, M) > kMaxElems) return SSL_E_CAPACITY;
  ssl::JacobiOpts jo;
  if (!ssl::ctx_jacobi(opts, &jo)) return SSL_E_INVALID_ARG;  // the checks of ssl_gsvd
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return SSL_E_CUDA;
  }
  float2* base = nullptr;
  {
    // First call on this device (which must be current): look up where the
    // array lives on it.  In host code the array's name is not a device
    // address, so the kernels are only ever handed this looked-up pointer.
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_dev_ptr[dev]) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
        cudaGetLastError();
        return SSL_E_CUDA;
      }
      g_dev_ptr[dev] = static_cast<float2*>(p);
    }
    base = g_dev_ptr[dev];
  }
  float2* kinv = base;
  int32_t* kinv_status = reinterpret_cast<int32_t*>(base + (size_t)B * M * M);
  unsigned* flags = reinterpret_cast<unsigned*>(base + kMaxElems);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = ssl::launch_noise_inverse(reinterpret_cast<const float2*>(K), B, M, kinv,
                                            kinv_status, flags, s);
  if (e == cudaSuccess)
    e = ssl::launch_gsvd(reinterpret_cast<const float2*>(R), kinv, nblk, B, M, jo, sigma,
                         reinterpret_cast<float2*>(E), status, nullptr, flags, s);
  if (e == cudaSuccess) {
    const size_t n = (size_t)nblk * B;
    const int blocks = (int)((n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024);
    fold_inverse_status<<<blocks, 256, 0, s>>>(kinv_status, nblk, B, status);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    return SSL_E_CUDA;
  }
  return SSL_OK;
}
