// ssl_gsvd_noalloc: the generalised SVD of ssl_gsvd for callers that must not
// allocate device memory.
//
// Who needs it: a real-time audio thread (a robot's or an array's audition
// loop) cannot afford cudaMalloc on its per-block path, because an allocation
// may synchronise the whole device and take far longer than the block's
// deadline; and a host framework that loads this library as a plug-in may
// own the device memory budget itself and forbid libraries from allocating
// behind its back.  Such callers still pass their own inputs and outputs; the
// one piece of scratch the decomposition needs, the per-bin inverse of the
// noise correlation, lives here in a fixed array compiled into the library.
//
// The array holds kMaxElems complex values (8 MiB) and is resident on every
// GPU that loads the library until the process exits.  Every call on a device
// shares it and it keeps the last call's contents; nothing in it has to start
// at zero (K^{-1} is fully written before it is read).  Calls whose work
// overlaps on the GPU, e.g. on two streams at once, race on the array.
#include <mutex>

#include "ssl_internal.cuh"

namespace {

constexpr size_t kMaxElems = size_t(1) << 20;  // K^{-1}: B * M * M complex values at most
constexpr int kMaxDevices = 64;

// K^{-1} scratch followed by one word for the kernels' sticky flags.
static __device__ __align__(256) float2 g_noalloc_scratch[kMaxElems + 32];

std::mutex g_mu;
float2* g_dev_ptr[kMaxDevices] = {};  // device address of the array, per device

}  // namespace

extern "C" ssl_status ssl_gsvd_noalloc(const float* R, const float* K, int nblk, int B, int M,
                                       const ssl_jacobi_opts* opts, float* sigma, float* E,
                                       int32_t* status, void* stream) {
  if (!R || !K || !sigma || !E || nblk < 1 || B < 1 || M < 1 || M > SSL_MAX_M)
    return SSL_E_INVALID_ARG;
  if ((size_t)B * M * M > kMaxElems) return SSL_E_CAPACITY;
  ssl::JacobiOpts jo{30, 0.f, 0.f, true};
  if (opts) {
    if (opts->angles != SSL_ANGLES_F64 && opts->angles != SSL_ANGLES_F32) return SSL_E_INVALID_ARG;
    if (!(opts->rel_tol < 1.f) || !(opts->abs_tol < 1.f)) return SSL_E_INVALID_ARG;
    if (opts->method != SSL_SVD_JACOBI && opts->method != SSL_SVD_BIDIAG) return SSL_E_INVALID_ARG;
    jo.method = opts->method;
    jo.max_sweeps = opts->max_sweeps > 0 ? opts->max_sweeps : 30;
    jo.rel_tol = opts->rel_tol;
    jo.abs_tol = opts->abs_tol;
    jo.angles_f64 = opts->angles == SSL_ANGLES_F64;
  }
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
  unsigned* flags = reinterpret_cast<unsigned*>(base + kMaxElems);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = ssl::launch_noise_inverse(reinterpret_cast<const float2*>(K), B, M, kinv,
                                            nullptr, flags, s);
  if (e == cudaSuccess)
    e = ssl::launch_gsvd(reinterpret_cast<const float2*>(R), kinv, nblk, B, M, jo, sigma,
                         reinterpret_cast<float2*>(E), status, nullptr, flags, s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return SSL_E_CUDA;
  }
  return SSL_OK;
}
