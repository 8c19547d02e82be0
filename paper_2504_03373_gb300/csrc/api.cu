// C ABI of the GSVD-MUSIC library: argument checks, the context (device,
// sticky device flags, growable workspace), host<->device staging, and the
// sequencing of the kernels of the hot path on the caller's stream.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <new>

#include "ssl_internal.cuh"

struct ssl_ctx {
  int device;
  unsigned* dflags;     // sticky SSL_FLAG_* word on the device
  void* ws;             // workspace
  size_t ws_bytes;
  // a second stream for work of a call that is independent of the caller's
  // stream's current work (forked and joined by events inside the call)
  cudaStream_t aux;
  cudaEvent_t ev_fork, ev_join;
  // ssl_localize with host X: staging copy landed; staging buffer b read
  cudaEvent_t ev_xcopy, ev_xfree[2];
  // the workspace's last use: recorded on a call's stream after its work, and
  // waited for by the next call that uses the workspace, on whatever stream
  cudaEvent_t ev_ws;
  unsigned xcall;  // calls with host X so far (selects the staging buffer)
  // the two staging buffers of host X (apart from the workspace, so that the
  // copy of one call's X may run while the previous call still computes)
  void* xs;
  size_t xs_bytes;  // bytes of each
  uint64_t wait_ns;  // limit of each bounded device wait (0: the kernels' default)
  int test_stall;    // ssl_set_test_stall: spectrum launches withhold their operand loads
  char err[512];
};

struct ssl_steering {
  ssl_ctx* ctx;
  int B, D, M;
  float2* H;       // [B][D][M] c64
  float* hnorm2;   // [B][D]
  // tensor-core A-operand images, index 0 = TF32, 1 = BF16, 2 = the TF32
  // rounding residuals (3xTF32's low part); each built on first use
  void* img[3];
  CUtensorMap tm[3];
  // neighbour lists of a direction set that is not a grid (device CSR), or null
  int32_t* nbr_ptr;  // [D + 1]
  int32_t* nbr_idx;  // [n_edges]
  // search range of the peak search (Sec. III-A, last step): [D] bytes on the
  // device, nonzero inside; null: every direction
  uint8_t* range;
  // analytic form: geometry on the device (positions, directions, f/c) and a
  // device copy of its Geo descriptor; H and hnorm2 are then built only when
  // a path needs a table (the BF16/TF32 tensor-core spectrum generates its
  // tiles from the geometry)
  bool analytic;
  float* geo_buf;
  ssl::Geo* geo;
};

namespace {

constexpr int kDefaultSweeps = 30;

ssl_status fail(ssl_ctx* ctx, ssl_status st, const char* fmt, ...) {
  if (ctx) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(ctx->err, sizeof(ctx->err), fmt, ap);
    va_end(ap);
  }
  return st;
}

ssl_status cuda_fail(ssl_ctx* ctx, cudaError_t e, const char* what) {
  return fail(ctx, SSL_E_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

// Makes ctx->device current for the scope of an API call and restores the
// caller's device afterwards.
struct DeviceGuard {
  int prev = -1;
  bool ok = false;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    ok = (prev == dev) || (cudaSetDevice(dev) == cudaSuccess);
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

// Sub-allocator over the context workspace: offsets are 256-byte aligned.
struct Carve {
  size_t off = 0;
  size_t take(size_t bytes) {
    const size_t o = off;
    off += (bytes + 255) & ~(size_t)255;
    return o;
  }
};

bool capturing(cudaStream_t s) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return cs != cudaStreamCaptureStatusNone;
}

// Workspace of a call on stream s: ordered after the previous call that used
// it (any stream), grown if needed.  Pair with a WsUse once it succeeded.
ssl_status ws_reserve(ssl_ctx* ctx, size_t bytes, cudaStream_t s) {
  // (inside a stream capture the caller orders the captured work)
  if (!capturing(s)) {
    const cudaError_t w = cudaStreamWaitEvent(s, ctx->ev_ws, 0);
    if (w != cudaSuccess) return cuda_fail(ctx, w, "workspace: order after its last use");
  }
  if (bytes <= ctx->ws_bytes) return SSL_OK;
  // Kernels still in flight, on any stream, may use the old buffer.
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(ctx, e, "workspace: device synchronize");
  if (ctx->ws) cudaFree(ctx->ws);
  ctx->ws = nullptr;
  ctx->ws_bytes = 0;
  const size_t want = bytes + bytes / 4;
  e = cudaMalloc(&ctx->ws, want);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(ctx, SSL_E_OOM, "workspace: cudaMalloc(%zu) failed: %s", want,
                cudaGetErrorString(e));
  }
  ctx->ws_bytes = want;
  return SSL_OK;
}

char* ws_ptr(ssl_ctx* ctx, size_t off) { return static_cast<char*>(ctx->ws) + off; }

// Marks the end of a call's workspace use on stream s (the work enqueued on s
// so far), whatever path the call returns by.
struct WsUse {
  ssl_ctx* ctx;
  cudaStream_t s;
  ~WsUse() {
    if (!capturing(s) && cudaEventRecord(ctx->ev_ws, s) != cudaSuccess) cudaGetLastError();
  }
};

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

bool dims_ok(int B, int M) { return B >= 1 && M >= 1 && M <= SSL_MAX_M; }

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    else
      cudaGetLastError();
  }
  return fn;
}

}  // namespace

namespace ssl {

// 3-D tiled tensor map over a row-major [d2][d1][d0] array, 128-byte swizzle,
// box {b0, b1, 1}; out-of-range rows read as zero.
bool encode_tmap_3d(CUtensorMap* tm, void* base, int esz, uint64_t d0, uint64_t d1, uint64_t d2,
                    uint32_t b0, uint32_t b1) {
  PFN_cuTensorMapEncodeTiled_v12000 fn = tensor_map_encoder();
  if (!fn) return false;
  cuuint64_t dims[3] = {d0, d1, d2};
  cuuint64_t strides[2] = {d0 * esz, d0 * d1 * esz};
  cuuint32_t box[3] = {b0, b1, 1};
  cuuint32_t es[3] = {1, 1, 1};
  return fn(tm, esz == 2 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3,
            base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

unsigned* ctx_flags(ssl_ctx* ctx) { return ctx->dflags; }
uint64_t ctx_wait_ns(const ssl_ctx* ctx) { return ctx->wait_ns; }
int ctx_test_stall(const ssl_ctx* ctx) { return ctx->test_stall; }
ssl_status ctx_error(ssl_ctx* ctx, ssl_status st, const char* msg) {
  if (ctx && msg) snprintf(ctx->err, sizeof(ctx->err), "%s", msg);
  return st;
}
bool ctx_jacobi(const ssl_jacobi_opts* o, JacobiOpts* out);
int ctx_device(const ssl_ctx* ctx) { return ctx->device; }
bool steering_matches(const ssl_steering* st, int B, int D, int M) {
  return st && st->B == B && st->D == D && st->M == M;
}
bool steering_is_analytic(const ssl_steering* st) { return st && st->analytic; }
const uint8_t* steering_range(const ssl_steering* st) { return st ? st->range : nullptr; }
bool steering_lists(const ssl_steering* st, const int32_t** ptr, const int32_t** idx) {
  if (!st || !st->nbr_ptr) return false;
  *ptr = st->nbr_ptr;
  *idx = st->nbr_idx;
  return true;
}

}  // namespace ssl

namespace {

bool jacobi_opts(const ssl_jacobi_opts* o, ssl::JacobiOpts* out) {
  ssl::JacobiOpts j{kDefaultSweeps, 0.f, 0.f, true, SSL_SVD_JACOBI};
  if (o) {
    if (o->angles != SSL_ANGLES_F64 && o->angles != SSL_ANGLES_F32) return false;
    if (o->method != SSL_SVD_JACOBI && o->method != SSL_SVD_BIDIAG && o->method != SSL_SVD_SPLIT)
      return false;
    j.method = o->method;
    j.split_ns = o->split_ns;
    if (!(o->rel_tol < 1.f) || !(o->abs_tol < 1.f)) return false;  // also rejects NaN
    j.max_sweeps = o->max_sweeps > 0 ? o->max_sweeps : kDefaultSweeps;
    j.rel_tol = o->rel_tol;
    j.abs_tol = o->abs_tol;
    j.angles_f64 = o->angles == SSL_ANGLES_F64;
  }
  *out = j;
  return true;
}

}  // namespace

extern "C" {

ssl_status ssl_create(ssl_ctx** out, int device) {
  if (!out) return SSL_E_INVALID_ARG;
  *out = nullptr;
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) {
    cudaGetLastError();
    return SSL_E_INVALID_ARG;
  }
  ssl_ctx* ctx = new (std::nothrow) ssl_ctx();
  if (!ctx) return SSL_E_OOM;
  ctx->device = device;
  DeviceGuard g(device);
  if (!g.ok) {
    delete ctx;
    return SSL_E_CUDA;
  }
  if (cudaMalloc(&ctx->dflags, sizeof(unsigned)) != cudaSuccess ||
      cudaMemset(ctx->dflags, 0, sizeof(unsigned)) != cudaSuccess) {
    cudaGetLastError();
    delete ctx;
    return SSL_E_OOM;
  }
  if (cudaStreamCreateWithFlags(&ctx->aux, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->ev_join, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    if (ctx->aux) cudaStreamDestroy(ctx->aux);
    if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
    cudaFree(ctx->dflags);
    delete ctx;
    return SSL_E_CUDA;
  }
  if (cudaEventCreateWithFlags(&ctx->ev_xcopy, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->ev_xfree[0], cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->ev_xfree[1], cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->ev_ws, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    if (ctx->ev_xcopy) cudaEventDestroy(ctx->ev_xcopy);
    if (ctx->ev_xfree[0]) cudaEventDestroy(ctx->ev_xfree[0]);
    if (ctx->ev_xfree[1]) cudaEventDestroy(ctx->ev_xfree[1]);
    cudaEventDestroy(ctx->ev_fork);
    cudaEventDestroy(ctx->ev_join);
    cudaStreamDestroy(ctx->aux);
    cudaFree(ctx->dflags);
    delete ctx;
    return SSL_E_CUDA;
  }
  *out = ctx;
  return SSL_OK;
}

ssl_status ssl_destroy(ssl_ctx* ctx) {
  if (!ctx) return SSL_OK;
  {
    DeviceGuard g(ctx->device);
    cudaDeviceSynchronize();
    if (ctx->ws) cudaFree(ctx->ws);
    if (ctx->xs) cudaFree(ctx->xs);
    if (ctx->dflags) cudaFree(ctx->dflags);
    if (ctx->aux) cudaStreamDestroy(ctx->aux);
    if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
    if (ctx->ev_join) cudaEventDestroy(ctx->ev_join);
    if (ctx->ev_xcopy) cudaEventDestroy(ctx->ev_xcopy);
    for (int b = 0; b < 2; ++b)
      if (ctx->ev_xfree[b]) cudaEventDestroy(ctx->ev_xfree[b]);
    if (ctx->ev_ws) cudaEventDestroy(ctx->ev_ws);
  }
  delete ctx;
  return SSL_OK;
}

ssl_status ssl_last_error(const ssl_ctx* ctx, char* buf, size_t len) {
  if (!ctx || !buf || len == 0) return SSL_E_INVALID_ARG;
  snprintf(buf, len, "%s", ctx->err);
  return SSL_OK;
}

ssl_status ssl_device_flags(ssl_ctx* ctx, void* stream, uint32_t* flags) {
  if (!ctx || !flags) return SSL_E_INVALID_ARG;
  DeviceGuard g(ctx->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  unsigned h = 0;
  cudaError_t e = cudaMemcpyAsync(&h, ctx->dflags, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = cudaMemsetAsync(ctx->dflags, 0, sizeof(unsigned), s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "ssl_device_flags");
  *flags = h;
  return SSL_OK;
}

ssl_status ssl_set_wait_limit(ssl_ctx* ctx, uint64_t ns) {
  if (!ctx) return SSL_E_INVALID_ARG;
  ctx->wait_ns = ns;
  return SSL_OK;
}

ssl_status ssl_set_test_stall(ssl_ctx* ctx, int on) {
  if (!ctx) return SSL_E_INVALID_ARG;
  ctx->test_stall = on != 0;
  return SSL_OK;
}

ssl_status ssl_correlate(ssl_ctx* ctx, const float* X, int nblk, int T, int B, int M, float* R,
                         void* stream) {
  ssl::Range nvtx("ssl_correlate");
  if (!ctx) return SSL_E_INVALID_ARG;
  if (!X || !R || nblk < 1 || T < 1 || !dims_ok(B, M))
    return fail(ctx, SSL_E_INVALID_ARG, "ssl_correlate: bad arguments");
  DeviceGuard g(ctx->device);
  cudaError_t e = ssl::launch_correlate(reinterpret_cast<const float2*>(X), nblk, T, B, M,
                                        reinterpret_cast<float2*>(R),
                                        static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? SSL_OK : cuda_fail(ctx, e, "ssl_correlate");
}

ssl_status ssl_noise_inverse(ssl_ctx* ctx, const float* K, int B, int M, float* Kinv,
                             int32_t* status, void* stream) {
  ssl::Range nvtx("ssl_noise_inverse");
  if (!ctx) return SSL_E_INVALID_ARG;
  if (!K || !Kinv || !dims_ok(B, M))
    return fail(ctx, SSL_E_INVALID_ARG, "ssl_noise_inverse: bad arguments");
  DeviceGuard g(ctx->device);
  cudaError_t e = ssl::launch_noise_inverse(reinterpret_cast<const float2*>(K), B, M,
                                            reinterpret_cast<float2*>(Kinv), status, ctx->dflags,
                                            static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? SSL_OK : cuda_fail(ctx, e, "ssl_noise_inverse");
}

namespace {

// Workspace of the split iteration: A by columns, and a status array when the
// caller passes none.
void split_carve(Carve& cv, int nblk, int B, int M, bool need_status, size_t* o_a,
                 size_t* o_st) {
  *o_a = cv.take((size_t)nblk * B * M * M * sizeof(float2));
  *o_st = need_status ? cv.take((size_t)nblk * B * sizeof(int32_t)) : 0;
}

// eq. 4 with K^{-1} given; workspace from byte offset ws_off on (the part
// below belongs to the caller).  The split iteration takes a status array (the
// workspace's when the caller passes none) and a buffer for A.
ssl_status gsvd_kinv_impl(ssl_ctx* ctx, const float2* R, const float2* Kinv, int nblk, int B,
                          int M, const ssl::JacobiOpts& jo, float* sigma, float2* E,
                          int32_t* status, int32_t* stats, cudaStream_t s, size_t ws_off) {
  float2* abuf = nullptr;
  if (jo.method == SSL_SVD_SPLIT) {
    Carve cv;
    cv.off = ws_off;
    size_t o_a, o_st;
    split_carve(cv, nblk, B, M, !status, &o_a, &o_st);
    const ssl_status st = ws_reserve(ctx, cv.off, s);
    if (st != SSL_OK) return st;
    abuf = reinterpret_cast<float2*>(ws_ptr(ctx, o_a));
    if (!status) status = reinterpret_cast<int32_t*>(ws_ptr(ctx, o_st));
  }
  const cudaError_t e = ssl::launch_gsvd(R, Kinv, nblk, B, M, jo, sigma, E, status, stats,
                                         ctx->dflags, s, nullptr, nullptr, nullptr, abuf);
  return e == cudaSuccess ? SSL_OK : cuda_fail(ctx, e, "ssl_gsvd");
}

}  // namespace

ssl_status ssl_gsvd_kinv(ssl_ctx* ctx, const float* R, const float* Kinv, int nblk, int B, int M,
                         const ssl_jacobi_opts* opts, float* sigma, float* E, int32_t* status,
                         int32_t* stats, void* stream) {
  ssl::Range nvtx("ssl_gsvd_kinv");
  if (!ctx) return SSL_E_INVALID_ARG;
  ssl::JacobiOpts jo;
  if (!R || !Kinv || !sigma || !E || nblk < 1 || !dims_ok(B, M) || !jacobi_opts(opts, &jo) ||
      (jo.method == SSL_SVD_SPLIT && (jo.split_ns < 1 || jo.split_ns >= M)))
    return fail(ctx, SSL_E_INVALID_ARG, "ssl_gsvd: bad arguments");
  DeviceGuard g(ctx->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  WsUse ws_use{ctx, s};
  return gsvd_kinv_impl(ctx, reinterpret_cast<const float2*>(R),
                        reinterpret_cast<const float2*>(Kinv), nblk, B, M, jo, sigma,
                        reinterpret_cast<float2*>(E), status, stats, s, 0);
}

ssl_status ssl_gsvd(ssl_ctx* ctx, const float* R, const float* K, int nblk, int B, int M,
                    const ssl_jacobi_opts* opts, float* sigma, float* E, int32_t* status,
                    void* stream) {
  ssl::Range nvtx("ssl_gsvd");
  if (!ctx) return SSL_E_INVALID_ARG;
  ssl::JacobiOpts jo;
  if (!R || !K || !sigma || !E || nblk < 1 || !dims_ok(B, M) || !jacobi_opts(opts, &jo) ||
      (jo.method == SSL_SVD_SPLIT && (jo.split_ns < 1 || jo.split_ns >= M)))
    return fail(ctx, SSL_E_INVALID_ARG, "ssl_gsvd: bad arguments");
  DeviceGuard g(ctx->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  Carve cv;
  const size_t o_kinv = cv.take((size_t)B * M * M * sizeof(float2));
  const size_t rest = cv.off;
  if (jo.method == SSL_SVD_SPLIT) {  // reserve gsvd_kinv_impl's part too: K^{-1} must stay put
    size_t o_a, o_st;
    split_carve(cv, nblk, B, M, !status, &o_a, &o_st);
  }
  ssl_status st = ws_reserve(ctx, cv.off, s);
  if (st != SSL_OK) return st;
  WsUse ws_use{ctx, s};
  float2* Kinv = reinterpret_cast<float2*>(ws_ptr(ctx, o_kinv));
  cudaError_t e = ssl::launch_noise_inverse(reinterpret_cast<const float2*>(K), B, M, Kinv,
                                            nullptr, ctx->dflags, s);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "ssl_gsvd: noise inverse");
  return gsvd_kinv_impl(ctx, reinterpret_cast<const float2*>(R), Kinv, nblk, B, M, jo, sigma,
                        reinterpret_cast<float2*>(E), status, nullptr, s, rest);
}

ssl_status ssl_sevd(ssl_ctx* ctx, const float* R, int nblk, int B, int M,
                    const ssl_jacobi_opts* opts, float* lambda, float* E, int32_t* status,
                    void* stream) {
  ssl::Range nvtx("ssl_sevd");
  if (!ctx) return SSL_E_INVALID_ARG;
  ssl::JacobiOpts jo;
  if (!R || !lambda || !E || nblk < 1 || !dims_ok(B, M) || !jacobi_opts(opts, &jo))
    return fail(ctx, SSL_E_INVALID_ARG, "ssl_sevd: bad arguments");
  if (jo.method == SSL_SVD_SPLIT)
    return fail(ctx, SSL_E_UNSUPPORTED, "ssl_sevd: the split iteration serves ssl_gsvd and the SQ spectrum");
  DeviceGuard g(ctx->device);
  // whitening by the identity: one-sided Jacobi on R^H = R
  cudaError_t e = ssl::launch_gsvd(reinterpret_cast<const float2*>(R), nullptr, nblk, B, M, jo,
                                   lambda, reinterpret_cast<float2*>(E), status, nullptr,
                                   ctx->dflags, static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? SSL_OK : cuda_fail(ctx, e, "ssl_sevd");
}

ssl_status ssl_gevd(ssl_ctx* ctx, const float* R, const float* K, int nblk, int B, int M,
                    const ssl_jacobi_opts* opts, float* lambda, float* E, int32_t* status,
                    void* stream) {
  ssl::Range nvtx("ssl_gevd");
  if (!ctx) return SSL_E_INVALID_ARG;
  ssl::JacobiOpts jo;
  if (!R || !K || !lambda || !E || nblk < 1 || !dims_ok(B, M) || !jacobi_opts(opts, &jo))
    return fail(ctx, SSL_E_INVALID_ARG, "ssl_gevd: bad arguments");
  if (jo.method == SSL_SVD_SPLIT)
    return fail(ctx, SSL_E_UNSUPPORTED, "ssl_gevd: the split iteration serves ssl_gsvd and the SQ spectrum");
  DeviceGuard g(ctx->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t mm = (size_t)B * M * M * sizeof(float2);
  Carve cv;
  const size_t o_kinv = cv.take(mm), o_w = cv.take(mm);
  const size_t o_rw = cv.take(mm * nblk), o_y = cv.take(mm * nblk);
  ssl_status st = ws_reserve(ctx, cv.off, s);
  if (st != SSL_OK) return st;
  WsUse ws_use{ctx, s};
  float2* Kinv = reinterpret_cast<float2*>(ws_ptr(ctx, o_kinv));
  float2* W = reinterpret_cast<float2*>(ws_ptr(ctx, o_w));
  float2* RW = reinterpret_cast<float2*>(ws_ptr(ctx, o_rw));
  float2* Y = reinterpret_cast<float2*>(ws_ptr(ctx, o_y));
  // K = L L^H, W = L^{-1}; B = W R W^H is Hermitian PSD with the eigenvalues
  // of K^{-1} R; its eigenvectors Y give the right eigenvectors E = W^H Y.
  cudaError_t e = ssl::launch_noise_inverse(reinterpret_cast<const float2*>(K), B, M, Kinv,
                                            nullptr, ctx->dflags, s, W);
  if (e == cudaSuccess)
    e = ssl::launch_cgemm(reinterpret_cast<const float2*>(R), true, false, W, false, true, nblk, B,
                          M, RW, s);
  if (e == cudaSuccess)
    e = ssl::launch_gsvd(RW, W, nblk, B, M, jo, lambda, Y, status, nullptr, ctx->dflags, s);
  if (e == cudaSuccess)
    e = ssl::launch_cgemm(W, false, true, Y, true, false, nblk, B, M,
                          reinterpret_cast<float2*>(E), s);
  return e == cudaSuccess ? SSL_OK : cuda_fail(ctx, e, "ssl_gevd");
}

ssl_status ssl_steering_create(ssl_ctx* ctx, const float* H, int B, int D, int M,
                               ssl_steering** out) {
  ssl::Range nvtx("ssl_steering_create");
  if (!ctx) return SSL_E_INVALID_ARG;
  if (!H || !out || !dims_ok(B, M) || D < 1 || D > SSL_MAX_D)
    return fail(ctx, SSL_E_INVALID_ARG, "ssl_steering_create: bad arguments");
  *out = nullptr;
  DeviceGuard g(ctx->device);
  ssl_steering* st = new (std::nothrow) ssl_steering();
  if (!st) return SSL_E_OOM;
  st->ctx = ctx;
  st->B = B;
  st->D = D;
  st->M = M;
  const size_t hb = (size_t)B * D * M * sizeof(float2);
  if (cudaMalloc(&st->H, hb) != cudaSuccess ||
      cudaMalloc(&st->hnorm2, (size_t)B * D * sizeof(float)) != cudaSuccess) {
    cudaGetLastError();
    if (st->H) cudaFree(st->H);
    delete st;
    return fail(ctx, SSL_E_OOM, "ssl_steering_create: out of device memory");
  }
  cudaError_t e = cudaMemcpy(st->H, H, hb, cudaMemcpyDefault);
  if (e == cudaSuccess) e = ssl::launch_hnorm2(st->H, B, D, M, st->hnorm2, 0);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    cudaFree(st->H);
    cudaFree(st->hnorm2);
    delete st;
    return cuda_fail(ctx, e, "ssl_steering_create");
  }
  *out = st;
  return SSL_OK;
}

ssl_status ssl_steering_destroy(ssl_steering* st) {
  if (!st) return SSL_OK;
  {
    DeviceGuard g(st->ctx->device);
    cudaDeviceSynchronize();
    if (st->H) cudaFree(st->H);
    if (st->hnorm2) cudaFree(st->hnorm2);
    for (int i = 0; i < 3; ++i)
      if (st->img[i]) cudaFree(st->img[i]);
    if (st->nbr_ptr) cudaFree(st->nbr_ptr);
    if (st->nbr_idx) cudaFree(st->nbr_idx);
    if (st->range) cudaFree(st->range);
    if (st->geo_buf) cudaFree(st->geo_buf);
  }
  delete st;
  return SSL_OK;
}

ssl_status ssl_steering_create_analytic(ssl_ctx* ctx, const float* pos, const float* dirs,
                                        const float* freqs, float c, int B, int D, int M,
                                        ssl_steering** out) {
  ssl::Range nvtx("ssl_steering_create_analytic");
  if (!ctx) return SSL_E_INVALID_ARG;
  if (!pos || !dirs || !freqs || !out || !dims_ok(B, M) || D < 1 || D > SSL_MAX_D || !(c > 0.f))
    return fail(ctx, SSL_E_INVALID_ARG, "ssl_steering_create_analytic: bad arguments");
  *out = nullptr;
  DeviceGuard g(ctx->device);
  // one host image of the inputs (host or device pointers): positions,
  // directions, then f / c per bin
  const size_t nf = 3 * (size_t)M + 3 * (size_t)D + (size_t)B;
  float* hbuf = new (std::nothrow) float[nf];
  if (!hbuf) return SSL_E_OOM;
  cudaError_t e = cudaMemcpy(hbuf, pos, 3 * (size_t)M * sizeof(float), cudaMemcpyDefault);
  if (e == cudaSuccess)
    e = cudaMemcpy(hbuf + 3 * M, dirs, 3 * (size_t)D * sizeof(float), cudaMemcpyDefault);
  if (e == cudaSuccess)
    e = cudaMemcpy(hbuf + 3 * M + 3 * D, freqs, (size_t)B * sizeof(float), cudaMemcpyDefault);
  if (e != cudaSuccess) {
    delete[] hbuf;
    return cuda_fail(ctx, e, "ssl_steering_create_analytic: read the geometry");
  }
  const char* bad = nullptr;
  for (size_t i = 0; i < nf && !bad; ++i)
    if (!isfinite(hbuf[i]))
      bad = i < 3 * (size_t)M ? "position" : i < 3 * (size_t)(M + D) ? "direction" : "frequency";
  if (bad) {
    delete[] hbuf;
    return fail(ctx, SSL_E_INVALID_ARG, "analytic steering: non-finite %s", bad);
  }
  for (int w = 0; w < B; ++w) hbuf[3 * M + 3 * D + w] /= c;
  ssl_steering* st = new (std::nothrow) ssl_steering();
  if (!st) {
    delete[] hbuf;
    return SSL_E_OOM;
  }
  st->ctx = ctx;
  st->B = B;
  st->D = D;
  st->M = M;
  st->analytic = true;
  // one device buffer: the Geo descriptor (256-byte slot), then hbuf
  const size_t bytes = 256 + nf * sizeof(float);
  char* dbuf = nullptr;
  e = cudaMalloc(&dbuf, bytes);
  if (e == cudaSuccess) {
    const float* fd = reinterpret_cast<const float*>(dbuf + 256);
    ssl::Geo geo{fd, fd + 3 * M, fd + 3 * M + 3 * D, M, D, B};
    e = cudaMemcpy(dbuf, &geo, sizeof(geo), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
      e = cudaMemcpy(dbuf + 256, hbuf, nf * sizeof(float), cudaMemcpyHostToDevice);
  }
  delete[] hbuf;
  if (e != cudaSuccess) {
    cudaGetLastError();
    if (dbuf) cudaFree(dbuf);
    delete st;
    return cuda_fail(ctx, e, "ssl_steering_create_analytic");
  }
  st->geo_buf = reinterpret_cast<float*>(dbuf);
  st->geo = reinterpret_cast<ssl::Geo*>(dbuf);
  *out = st;
  return SSL_OK;
}

ssl_status ssl_steering_set_neighbours(ssl_steering* st, const int32_t* nbr_ptr,
                                       const int32_t* nbr_idx, int n_edges) {
  ssl::Range nvtx("ssl_steering_set_neighbours");
  if (!st || !nbr_ptr || n_edges < 0 || (n_edges > 0 && !nbr_idx)) return SSL_E_INVALID_ARG;
  ssl_ctx* ctx = st->ctx;
  DeviceGuard g(ctx->device);
  const int D = st->D;
  // checked on the host once, so the peak kernel may trust every index
  int32_t* hp = new (std::nothrow) int32_t[D + 1];
  int32_t* hi = new (std::nothrow) int32_t[n_edges > 0 ? n_edges : 1];
  if (!hp || !hi) {
    delete[] hp;
    delete[] hi;
    return SSL_E_OOM;
  }
  cudaError_t e = cudaMemcpy(hp, nbr_ptr, (size_t)(D + 1) * sizeof(int32_t), cudaMemcpyDefault);
  if (e == cudaSuccess && n_edges > 0)
    e = cudaMemcpy(hi, nbr_idx, (size_t)n_edges * sizeof(int32_t), cudaMemcpyDefault);
  bool ok = e == cudaSuccess && hp[0] == 0 && hp[D] == n_edges;
  for (int d = 0; ok && d < D; ++d) ok = hp[d] <= hp[d + 1];
  for (int j = 0; ok && j < n_edges; ++j) ok = hi[j] >= 0 && hi[j] < D;
  ssl_status r = SSL_OK;
  if (e != cudaSuccess) {
    cudaGetLastError();
    r = cuda_fail(ctx, e, "ssl_steering_set_neighbours: copy");
  } else if (!ok) {
    r = fail(ctx, SSL_E_INVALID_ARG,
             "ssl_steering_set_neighbours: lists must start at 0, not decrease, end at "
             "n_edges and hold indices in [0, D)");
  }
  int32_t *dp = nullptr, *di = nullptr;
  if (r == SSL_OK &&
      (cudaMalloc(&dp, (size_t)(D + 1) * sizeof(int32_t)) != cudaSuccess ||
       cudaMalloc(&di, (size_t)(n_edges > 0 ? n_edges : 1) * sizeof(int32_t)) != cudaSuccess)) {
    cudaGetLastError();
    r = fail(ctx, SSL_E_OOM, "ssl_steering_set_neighbours: out of device memory");
  }
  if (r == SSL_OK) {
    e = cudaMemcpy(dp, hp, (size_t)(D + 1) * sizeof(int32_t), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && n_edges > 0)
      e = cudaMemcpy(di, hi, (size_t)n_edges * sizeof(int32_t), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) r = cuda_fail(ctx, e, "ssl_steering_set_neighbours: upload");
  }
  delete[] hp;
  delete[] hi;
  if (r != SSL_OK) {
    if (dp) cudaFree(dp);
    if (di) cudaFree(di);
    return r;
  }
  cudaDeviceSynchronize();  // no kernel may still read the lists replaced here
  if (st->nbr_ptr) cudaFree(st->nbr_ptr);
  if (st->nbr_idx) cudaFree(st->nbr_idx);
  st->nbr_ptr = dp;
  st->nbr_idx = di;
  return SSL_OK;
}

ssl_status ssl_steering_set_search_range(ssl_steering* st, const uint8_t* in_range) {
  ssl::Range nvtx("ssl_steering_set_search_range");
  if (!st) return SSL_E_INVALID_ARG;
  ssl_ctx* ctx = st->ctx;
  DeviceGuard g(ctx->device);
  uint8_t* d = nullptr;
  if (in_range) {
    if (cudaMalloc(&d, (size_t)st->D) != cudaSuccess) {
      cudaGetLastError();
      return fail(ctx, SSL_E_OOM, "ssl_steering_set_search_range: out of device memory");
    }
    const cudaError_t e = cudaMemcpy(d, in_range, (size_t)st->D, cudaMemcpyDefault);
    if (e != cudaSuccess) {
      cudaFree(d);
      return cuda_fail(ctx, e, "ssl_steering_set_search_range: copy");
    }
  }
  cudaDeviceSynchronize();  // no kernel may still read the range replaced here
  if (st->range) cudaFree(st->range);
  st->range = d;
  return SSL_OK;
}

// Builds (once) tensor-core A image `which` of a steering table (0 TF32,
// 1 BF16, 2 TF32 residuals).
static ssl_status steering_image_one(ssl_ctx* ctx, ssl_steering* st, int which) {
  if (st->img[which]) return SSL_OK;
  const int precision = which == 1 ? SSL_PREC_BF16 : which == 0 ? SSL_PREC_TF32 : ssl::kPrecTf32Lo;
  const int esz = which == 1 ? 2 : 4;
  const int KP = ssl::tc_kp(st->M);
  void* img = nullptr;
  const size_t bytes = (size_t)st->B * st->D * KP * esz;
  if (cudaMalloc(&img, bytes) != cudaSuccess) {
    cudaGetLastError();
    return fail(ctx, SSL_E_OOM, "steering image: cudaMalloc(%zu) failed", bytes);
  }
  cudaError_t e = ssl::launch_pack_h(st->H, st->B, st->D, st->M, precision, img, 0);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    cudaFree(img);
    return cuda_fail(ctx, e, "steering image");
  }
  if (!ssl::encode_tmap_3d(&st->tm[which], img, esz, KP, st->D, st->B, 128 / esz, 128)) {
    cudaFree(img);
    return fail(ctx, SSL_E_CUDA, "steering image: tensor map encoding failed");
  }
  st->img[which] = img;
  return SSL_OK;
}

// The A images `precision` reads (3xTF32: the TF32 image and its residuals).
// The c64 table and |h|^2 of an analytic steering object, built on first use
// by a path that reads a table (FP32 SIMT and FP64 spectra, 3xTF32 images,
// mixed plans and streams).
static ssl_status ensure_table(ssl_ctx* ctx, ssl_steering* st) {
  if (st->H) return SSL_OK;
  const size_t hb = (size_t)st->B * st->D * st->M * sizeof(float2);
  float2* H = nullptr;
  float* hn = nullptr;
  if (cudaMalloc(&H, hb) != cudaSuccess ||
      cudaMalloc(&hn, (size_t)st->B * st->D * sizeof(float)) != cudaSuccess) {
    cudaGetLastError();
    if (H) cudaFree(H);
    return fail(ctx, SSL_E_OOM, "analytic steering: table: out of device memory");
  }
  cudaError_t e = ssl::launch_steering_table(st->geo, st->B, st->D, st->M, H, 0);
  if (e == cudaSuccess) e = ssl::launch_hnorm2(H, st->B, st->D, st->M, hn, 0);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    cudaFree(H);
    cudaFree(hn);
    return cuda_fail(ctx, e, "analytic steering: table");
  }
  st->H = H;
  st->hnorm2 = hn;
  return SSL_OK;
}

static ssl_status steering_image(ssl_ctx* ctx, ssl_steering* st, int precision) {
  if (st->analytic) {
    ssl_status r = ensure_table(ctx, st);
    if (r != SSL_OK) return r;
  }
  if (precision == SSL_PREC_BF16) return steering_image_one(ctx, st, 1);
  ssl_status r = steering_image_one(ctx, st, 0);
  if (r == SSL_OK && precision == SSL_PREC_TF32X3) r = steering_image_one(ctx, st, 2);
  return r;
}

static bool precision_ok(int p) {
  return p == SSL_PREC_FP32 || p == SSL_PREC_TF32 || p == SSL_PREC_BF16 || p == SSL_PREC_TF32X3;
}

// Workspace bytes of the spectrum step beyond P: the tensor-core B image.
// (3xTF32: the TF32 image followed by its residual image.)
static size_t spectrum_image_bytes(int nblk, int B, int M, int Ns, int precision) {
  if (precision == SSL_PREC_FP32) return 0;
  const int esz = precision == SSL_PREC_BF16 ? 2 : 4;
  const size_t one = (size_t)nblk * B * ssl::tc_np(M, Ns) * ssl::tc_kp(M) * esz;
  return precision == SSL_PREC_TF32X3 ? 2 * one : one;
}

// eq. 5 + eq. 6 with every buffer already in place (no allocation here).
// With `packed` the decomposition already wrote the tensor-core image into img
// (E is then not read).
static ssl_status spectrum_run(ssl_ctx* ctx, const float2* E, int nblk, int B, int M, int Ns,
                               const ssl_steering* cst, int form, int precision, float* Pw,
                               void* img, float* Pbar, cudaStream_t s, bool packed = false) {
  ssl_steering* st = const_cast<ssl_steering*>(cst);
  const int D = st->D;
  cudaError_t e = cudaSuccess;
  // analytic steering on the BF16 / TF32 tensor cores: tiles generated in the
  // kernel, no table
  const bool gen = st->analytic && (precision == SSL_PREC_BF16 || precision == SSL_PREC_TF32);
  if (precision == SSL_PREC_FP32) {
    if (st->analytic) {
      ssl_status r = ensure_table(ctx, st);
      if (r != SSL_OK) return r;
    }
    e = ssl::launch_spectrum_simt(E, nblk, B, M, Ns, st->H, st->hnorm2, D, form, Pw, s);
  } else {
    ssl_status r = gen ? SSL_OK : steering_image(ctx, st, precision);
    if (r != SSL_OK) return r;
    const int esz = precision == SSL_PREC_BF16 ? 2 : 4;
    const int KP = ssl::tc_kp(M), NP = ssl::tc_np(M, Ns);
    const bool x3 = precision == SSL_PREC_TF32X3;
    void* img_lo = x3 ? static_cast<char*>(img) + spectrum_image_bytes(nblk, B, M, Ns, precision) / 2
                      : nullptr;
    if (!packed) {
      e = ssl::launch_pack_e(E, nblk * B, M, Ns, precision, img, s, img_lo);
      if (e != cudaSuccess) return cuda_fail(ctx, e, "spectrum: operand image");
    }
    CUtensorMap tmE, tmElo;
    if (!ssl::encode_tmap_3d(&tmE, img, esz, KP, NP, (uint64_t)nblk * B, 128 / esz, NP) ||
        (x3 && !ssl::encode_tmap_3d(&tmElo, img_lo, esz, KP, NP, (uint64_t)nblk * B, 128 / esz,
                                    NP)))
      return fail(ctx, SSL_E_CUDA, "spectrum: tensor map encoding failed");
    if (x3)
      e = ssl::launch_spectrum_tc3(st->tm[0], st->tm[2], tmE, tmElo, nblk, B, D, M, Ns, form,
                                   st->hnorm2, Pw, ctx->dflags, s, ctx->wait_ns, ctx->test_stall);
    else
      e = ssl::launch_spectrum_tc(st->tm[precision == SSL_PREC_BF16 ? 1 : 0], tmE, nblk, B, D, M,
                                  Ns, precision, form, st->hnorm2, Pw, ctx->dflags, s, nullptr,
                                  nullptr, ctx->wait_ns, gen ? st->geo : nullptr, nullptr,
                                  ctx->test_stall);
  }
  if (e != cudaSuccess) return cuda_fail(ctx, e, "spectrum");
  e = ssl::launch_bin_sum(Pw, nblk, B, D, Pbar, s);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "bin sum");
  return SSL_OK;
}

ssl_status ssl_music_spectrum(ssl_ctx* ctx, const float* E, int nblk, int B, int M, int Ns,
                              const ssl_steering* st, int form, int precision, float* P,
                              float* Pbar, void* stream) {
  ssl::Range nvtx("ssl_music_spectrum");
  if (!ctx) return SSL_E_INVALID_ARG;
  if (!E || !st || !Pbar || nblk < 1 || !dims_ok(B, M) || Ns < 1 || Ns >= M || st->B != B ||
      st->M != M || (form != SSL_FORM_ABS && form != SSL_FORM_SQ))
    return fail(ctx, SSL_E_INVALID_ARG, "ssl_music_spectrum: bad arguments");
  if (!precision_ok(precision))
    return fail(ctx, SSL_E_INVALID_ARG, "ssl_music_spectrum: unknown precision %d", precision);
  DeviceGuard g(ctx->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  Carve cv;
  const size_t o_p = P ? 0 : cv.take((size_t)nblk * B * st->D * sizeof(float));
  const size_t o_img = cv.take(spectrum_image_bytes(nblk, B, M, Ns, precision));
  ssl_status r = ws_reserve(ctx, cv.off, s);
  if (r != SSL_OK) return r;
  WsUse ws_use{ctx, s};
  float* Pw = P ? P : reinterpret_cast<float*>(ws_ptr(ctx, o_p));
  return spectrum_run(ctx, reinterpret_cast<const float2*>(E), nblk, B, M, Ns, st, form,
                      precision, Pw, ws_ptr(ctx, o_img), Pbar, s);
}

ssl_status ssl_peaks(ssl_ctx* ctx, const float* Pbar, int nblk, int n_az, int n_el, int Ns,
                     int32_t* idx, float* val, void* stream) {
  ssl::Range nvtx("ssl_peaks");
  if (!ctx) return SSL_E_INVALID_ARG;
  if (!Pbar || !idx || !val || nblk < 1 || n_az < 1 || n_el < 1 || Ns < 1 || Ns > SSL_MAX_NS ||
      (long)n_az * n_el > SSL_MAX_D)
    return fail(ctx, SSL_E_INVALID_ARG, "ssl_peaks: bad arguments");
  DeviceGuard g(ctx->device);
  cudaError_t e = ssl::launch_peaks(Pbar, nblk, n_az, n_el, Ns, idx, val,
                                    static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? SSL_OK : cuda_fail(ctx, e, "ssl_peaks");
}

ssl_status ssl_peaks_nbr(ssl_ctx* ctx, const float* Pbar, int nblk, const ssl_steering* st, int Ns,
                         int32_t* idx, float* val, void* stream) {
  ssl::Range nvtx("ssl_peaks_nbr");
  if (!ctx) return SSL_E_INVALID_ARG;
  if (!Pbar || !st || !idx || !val || nblk < 1 || Ns < 1 || Ns > SSL_MAX_NS)
    return fail(ctx, SSL_E_INVALID_ARG, "ssl_peaks_nbr: bad arguments");
  if (!st->nbr_ptr)
    return fail(ctx, SSL_E_INVALID_ARG, "ssl_peaks_nbr: the steering object has no neighbour lists");
  DeviceGuard g(ctx->device);
  cudaError_t e = ssl::launch_peaks_nbr(Pbar, nblk, st->D, st->nbr_ptr, st->nbr_idx, Ns, idx, val,
                                        static_cast<cudaStream_t>(stream), ctx->dflags,
                                        st->range);
  return e == cudaSuccess ? SSL_OK : cuda_fail(ctx, e, "ssl_peaks_nbr");
}

}  // extern "C"

// The whole path; with k_is_inverse, K already holds K^{-1} (no FP64
// Cholesky in this call).
static ssl_status localize_impl(ssl_ctx* ctx, const float* X, int nblk, const float* K,
                                bool k_is_inverse, const ssl_steering* st, const ssl_config* cfg,
                                int32_t* peak_idx, float* peak_val, float* Pbar, void* stream) {
  ssl::Range nvtx(k_is_inverse ? "ssl_localize_kinv" : "ssl_localize");
  if (!ctx) return SSL_E_INVALID_ARG;
  if (!X || !K || !st || !cfg || !peak_idx || !peak_val || nblk < 1)
    return fail(ctx, SSL_E_INVALID_ARG, "ssl_localize: null argument");
  const int M = cfg->M, T = cfg->T, B = cfg->B, Ns = cfg->Ns;
  // n_el == 0: a direction set of n_az directions with the steering object's
  // neighbour lists
  const bool lists = cfg->n_el == 0;
  const int D = lists ? cfg->n_az : cfg->n_az * cfg->n_el;
  ssl::JacobiOpts jo;
  if (!dims_ok(B, M) || T < 1 || Ns < 1 || Ns >= M || Ns > SSL_MAX_NS || cfg->n_az < 1 ||
      cfg->n_el < 0 || (lists && !st->nbr_ptr) || D != st->D || st->B != B || st->M != M ||
      (cfg->form != SSL_FORM_ABS && cfg->form != SSL_FORM_SQ) || !jacobi_opts(&cfg->jacobi, &jo) ||
      !precision_ok(cfg->precision))
    return fail(ctx, SSL_E_INVALID_ARG, "ssl_localize: inconsistent configuration");
  if (jo.method == SSL_SVD_SPLIT && cfg->form != SSL_FORM_SQ)
    return fail(ctx, SSL_E_UNSUPPORTED,
                "ssl_localize: the split iteration gives the noise subspace, the ABS form needs "
                "its individual vectors");
  jo.split_ns = Ns;
  DeviceGuard g(ctx->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const bool x_dev = is_device_ptr(X), k_dev = is_device_ptr(K);
  const bool idx_dev = is_device_ptr(peak_idx), val_dev = is_device_ptr(peak_val);
  const bool pb_dev = Pbar && is_device_ptr(Pbar);

  const size_t mm = (size_t)M * M * sizeof(float2);
  Carve cv;
  const size_t x_bytes = (size_t)nblk * T * B * M * sizeof(float2);
  const size_t o_k = k_dev ? 0 : cv.take((size_t)B * mm);
  const size_t o_kinv = cv.take((size_t)B * mm);
  const size_t o_r = cv.take((size_t)nblk * B * mm);
  const size_t o_e = cv.take((size_t)nblk * B * mm);
  // the split iteration's A: E's space with the tensor-core spectrum (E is not
  // formed then), its own otherwise
  const bool split_a = jo.method == SSL_SVD_SPLIT;
  const size_t o_a = !split_a ? 0 : cfg->precision != SSL_PREC_FP32 ? o_e
                                                                    : cv.take((size_t)nblk * B * mm);
  const size_t o_sig = cv.take((size_t)nblk * B * M * sizeof(float));
  const size_t o_st = cv.take((size_t)nblk * B * sizeof(int32_t));
  const size_t o_pbar = pb_dev ? 0 : cv.take((size_t)nblk * D * sizeof(float));
  const size_t o_idx = idx_dev ? 0 : cv.take((size_t)nblk * Ns * sizeof(int32_t));
  const size_t o_val = val_dev ? 0 : cv.take((size_t)nblk * Ns * sizeof(float));
  const size_t o_p = cv.take((size_t)nblk * B * D * sizeof(float));
  const size_t o_img = cv.take(spectrum_image_bytes(nblk, B, M, Ns, cfg->precision));
  ssl_status r = ws_reserve(ctx, cv.off, s);
  if (r != SSL_OK) return r;
  WsUse ws_use{ctx, s};

  cudaError_t e = cudaSuccess;
  float2* Kinv = reinterpret_cast<float2*>(ws_ptr(ctx, o_kinv));  // K^{-1} used below
  float2* Rw = reinterpret_cast<float2*>(ws_ptr(ctx, o_r));
  float2* Ew = reinterpret_cast<float2*>(ws_ptr(ctx, o_e));
  float* sig = reinterpret_cast<float*>(ws_ptr(ctx, o_sig));
  int32_t* bst = reinterpret_cast<int32_t*>(ws_ptr(ctx, o_st));
  float* Pb = pb_dev ? Pbar : reinterpret_cast<float*>(ws_ptr(ctx, o_pbar));
  int32_t* id = idx_dev ? peak_idx : reinterpret_cast<int32_t*>(ws_ptr(ctx, o_idx));
  float* vl = val_dev ? peak_val : reinterpret_cast<float*>(ws_ptr(ctx, o_val));
  float* Pw = reinterpret_cast<float*>(ws_ptr(ctx, o_p));
  void* img = ws_ptr(ctx, o_img);

  const float2* Xd = reinterpret_cast<const float2*>(X);
  if (!x_dev) {
    // Host X goes through one of two staging buffers, alternating from call
    // to call, and is copied on the auxiliary stream: the copy waits only
    // until the correlation of the call two back has read that buffer, so
    // back-to-back calls copy the next block batch while this one computes.
    if (x_bytes > ctx->xs_bytes) {
      // every earlier copy into, and read of, the old buffers is finished
      e = cudaDeviceSynchronize();
      if (e != cudaSuccess) return cuda_fail(ctx, e, "ssl_localize: staging synchronize");
      if (ctx->xs) cudaFree(ctx->xs);
      ctx->xs = nullptr;
      ctx->xs_bytes = 0;
      if (cudaMalloc(&ctx->xs, 2 * x_bytes) != cudaSuccess) {
        cudaGetLastError();
        return fail(ctx, SSL_E_OOM, "ssl_localize: staging buffers: cudaMalloc(%zu) failed",
                    2 * x_bytes);
      }
      ctx->xs_bytes = x_bytes;
    }
    const int xb = ctx->xcall++ & 1;
    float2* dst = reinterpret_cast<float2*>(static_cast<char*>(ctx->xs) + xb * ctx->xs_bytes);
    e = cudaStreamWaitEvent(ctx->aux, ctx->ev_xfree[xb], 0);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(dst, X, (size_t)nblk * T * B * M * sizeof(float2),
                          cudaMemcpyHostToDevice, ctx->aux);
    if (e == cudaSuccess) e = cudaEventRecord(ctx->ev_xcopy, ctx->aux);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "ssl_localize: copy X");
    Xd = dst;
    const float2* Kd = reinterpret_cast<const float2*>(K);
    if (!k_dev) {
      float2* kdst = reinterpret_cast<float2*>(ws_ptr(ctx, o_k));
      e = cudaMemcpyAsync(kdst, K, (size_t)B * mm, cudaMemcpyHostToDevice, s);
      if (e != cudaSuccess) return cuda_fail(ctx, e, "ssl_localize: copy K");
      Kd = kdst;
    }
    if (k_is_inverse)
      Kinv = const_cast<float2*>(Kd);
    else
      e = ssl::launch_noise_inverse(Kd, B, M, Kinv, nullptr, ctx->dflags, s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "ssl_localize: noise inverse");
    e = cudaStreamWaitEvent(s, ctx->ev_xcopy, 0);
    if (e == cudaSuccess) e = ssl::launch_correlate(Xd, nblk, T, B, M, Rw, s);
    if (e == cudaSuccess) e = cudaEventRecord(ctx->ev_xfree[xb], s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "ssl_localize: correlate");
  } else {
    // K^{-1} (FP64, few CTAs) on the auxiliary stream beside the correlation
    // (memory-side, many CTAs): the two are independent, and the caller's
    // stream waits for both before the decomposition.
    e = cudaEventRecord(ctx->ev_fork, s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->aux, ctx->ev_fork, 0);
    const float2* Kd = reinterpret_cast<const float2*>(K);
    if (e == cudaSuccess && !k_dev) {
      float2* kdst = reinterpret_cast<float2*>(ws_ptr(ctx, o_k));
      e = cudaMemcpyAsync(kdst, K, (size_t)B * mm, cudaMemcpyHostToDevice, ctx->aux);
      Kd = kdst;
    }
    if (e == cudaSuccess && k_is_inverse)
      Kinv = const_cast<float2*>(Kd);  // (a host K^{-1} is copied on the auxiliary stream)
    else if (e == cudaSuccess)
      e = ssl::launch_noise_inverse(Kd, B, M, Kinv, nullptr, ctx->dflags, ctx->aux);
    if (e == cudaSuccess) e = cudaEventRecord(ctx->ev_join, ctx->aux);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "ssl_localize: noise inverse");
    e = ssl::launch_correlate(Xd, nblk, T, B, M, Rw, s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, ctx->ev_join, 0);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "ssl_localize: correlate");
  }
  // With the tensor-core spectrum the decomposition writes the noise-subspace
  // image itself (E is not needed then).
  const bool tc = cfg->precision != SSL_PREC_FP32;
  void* img_lo = cfg->precision == SSL_PREC_TF32X3
                     ? static_cast<char*>(img) +
                           spectrum_image_bytes(nblk, B, M, Ns, cfg->precision) / 2
                     : nullptr;
  const ssl::ImgOut io{img, cfg->precision == SSL_PREC_BF16 ? 2 : 4, Ns, ssl::tc_kp(M),
                       ssl::tc_np(M, Ns), img_lo};
  e = ssl::launch_gsvd(Rw, Kinv, nblk, B, M, jo, sig, tc ? nullptr : Ew, bst, nullptr,
                       ctx->dflags, s, nullptr, nullptr, tc ? &io : nullptr,
                       split_a ? reinterpret_cast<float2*>(ws_ptr(ctx, o_a)) : nullptr);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "ssl_localize: gsvd");
  r = spectrum_run(ctx, Ew, nblk, B, M, Ns, st, cfg->form, cfg->precision, Pw, img, Pb, s, tc);
  if (r != SSL_OK) return r;
  e = lists ? ssl::launch_peaks_nbr(Pb, nblk, D, st->nbr_ptr, st->nbr_idx, Ns, id, vl, s,
                                    ctx->dflags, st->range)
            : ssl::launch_peaks(Pb, nblk, cfg->n_az, cfg->n_el, Ns, id, vl, s, st->range);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "ssl_localize: peaks");
  if (!idx_dev)
    e = cudaMemcpyAsync(peak_idx, id, (size_t)nblk * Ns * sizeof(int32_t),
                        cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && !val_dev)
    e = cudaMemcpyAsync(peak_val, vl, (size_t)nblk * Ns * sizeof(float), cudaMemcpyDeviceToHost,
                        s);
  if (e == cudaSuccess && Pbar && !pb_dev)
    e = cudaMemcpyAsync(Pbar, Pb, (size_t)nblk * D * sizeof(float), cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "ssl_localize: copy out");
  return SSL_OK;
}

extern "C" {

ssl_status ssl_localize(ssl_ctx* ctx, const float* X, int nblk, const float* K,
                        const ssl_steering* st, const ssl_config* cfg, int32_t* peak_idx,
                        float* peak_val, float* Pbar, void* stream) {
  return localize_impl(ctx, X, nblk, K, false, st, cfg, peak_idx, peak_val, Pbar, stream);
}

ssl_status ssl_localize_kinv(ssl_ctx* ctx, const float* X, int nblk, const float* Kinv,
                             const ssl_steering* st, const ssl_config* cfg, int32_t* peak_idx,
                             float* peak_val, float* Pbar, void* stream) {
  return localize_impl(ctx, X, nblk, Kinv, true, st, cfg, peak_idx, peak_val, Pbar, stream);
}

// ---- the FP64 path ------------------------------------------------------------

ssl_status ssl_gsvd_f64(ssl_ctx* ctx, const double* R, const float* K, int nblk, int B, int M,
                        const ssl_jacobi_opts* opts, double* sigma, double* E, int32_t* status,
                        int32_t* stats, void* stream) {
  ssl::Range nvtx("ssl_gsvd_f64");
  if (!ctx) return SSL_E_INVALID_ARG;
  ssl::JacobiOpts jo;
  if (!R || !K || !sigma || !E || nblk < 1 || !dims_ok(B, M) || !jacobi_opts(opts, &jo))
    return fail(ctx, SSL_E_INVALID_ARG, "ssl_gsvd_f64: bad arguments");
  if (jo.method != SSL_SVD_JACOBI)
    return fail(ctx, SSL_E_UNSUPPORTED, "ssl_gsvd_f64: one-sided Jacobi only");
  DeviceGuard g(ctx->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  Carve cv;
  const size_t o_kinv = cv.take((size_t)B * M * M * sizeof(double2));
  ssl_status r = ws_reserve(ctx, cv.off, s);
  if (r != SSL_OK) return r;
  WsUse ws_use{ctx, s};
  double2* Kinv = reinterpret_cast<double2*>(ws_ptr(ctx, o_kinv));
  cudaError_t e = ssl::launch_noise_inverse_f64(reinterpret_cast<const float2*>(K), B, M, Kinv,
                                                nullptr, ctx->dflags, s);
  if (e == cudaSuccess)
    e = ssl::launch_gsvd_f64(reinterpret_cast<const double2*>(R), Kinv, nblk, B, M,
                             jo.max_sweeps, opts ? opts->rel_tol : 0.0, jo.abs_tol, sigma,
                             reinterpret_cast<double2*>(E), status, stats, ctx->dflags, s);
  return e == cudaSuccess ? SSL_OK : cuda_fail(ctx, e, "ssl_gsvd_f64");
}

ssl_status ssl_localize_f64(ssl_ctx* ctx, const float* X, int nblk, const float* K,
                            const ssl_steering* st, const ssl_config* cfg, int32_t* peak_idx,
                            double* peak_val, double* Pbar, void* stream) {
  ssl::Range nvtx("ssl_localize_f64");
  if (!ctx) return SSL_E_INVALID_ARG;
  if (!X || !K || !st || !cfg || !peak_idx || !peak_val || nblk < 1)
    return fail(ctx, SSL_E_INVALID_ARG, "ssl_localize_f64: null argument");
  const int M = cfg->M, T = cfg->T, B = cfg->B, Ns = cfg->Ns;
  const bool lists = cfg->n_el == 0;
  const int D = lists ? cfg->n_az : cfg->n_az * cfg->n_el;
  ssl::JacobiOpts jo;
  if (!dims_ok(B, M) || T < 1 || Ns < 1 || Ns >= M || Ns > SSL_MAX_NS || cfg->n_az < 1 ||
      cfg->n_el < 0 || (lists && !st->nbr_ptr) || D != st->D || st->B != B || st->M != M ||
      (cfg->form != SSL_FORM_ABS && cfg->form != SSL_FORM_SQ) || !jacobi_opts(&cfg->jacobi, &jo))
    return fail(ctx, SSL_E_INVALID_ARG, "ssl_localize_f64: inconsistent configuration");
  if (jo.method != SSL_SVD_JACOBI)
    return fail(ctx, SSL_E_UNSUPPORTED, "ssl_localize_f64: one-sided Jacobi only");
  DeviceGuard g(ctx->device);
  if (!is_device_ptr(X) || !is_device_ptr(K) || !is_device_ptr(peak_idx) ||
      !is_device_ptr(peak_val) || (Pbar && !is_device_ptr(Pbar)))
    return fail(ctx, SSL_E_INVALID_ARG, "ssl_localize_f64: device pointers only");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t mm = (size_t)M * M * sizeof(double2);
  Carve cv;
  const size_t o_kinv = cv.take((size_t)B * mm);
  const size_t o_r = cv.take((size_t)nblk * B * mm);
  const size_t o_e = cv.take((size_t)nblk * B * mm);
  const size_t o_sig = cv.take((size_t)nblk * B * M * sizeof(double));
  const size_t o_p = cv.take((size_t)nblk * B * D * sizeof(double));
  const size_t o_pbar = Pbar ? 0 : cv.take((size_t)nblk * D * sizeof(double));
  ssl_status r = st->analytic ? ensure_table(ctx, const_cast<ssl_steering*>(st)) : SSL_OK;
  if (r == SSL_OK) r = ws_reserve(ctx, cv.off, s);
  if (r != SSL_OK) return r;
  WsUse ws_use{ctx, s};
  double2* Kinv = reinterpret_cast<double2*>(ws_ptr(ctx, o_kinv));
  double2* Rw = reinterpret_cast<double2*>(ws_ptr(ctx, o_r));
  double2* Ew = reinterpret_cast<double2*>(ws_ptr(ctx, o_e));
  double* sig = reinterpret_cast<double*>(ws_ptr(ctx, o_sig));
  double* Pw = reinterpret_cast<double*>(ws_ptr(ctx, o_p));
  double* Pb = Pbar ? Pbar : reinterpret_cast<double*>(ws_ptr(ctx, o_pbar));
  cudaError_t e = ssl::launch_noise_inverse_f64(reinterpret_cast<const float2*>(K), B, M, Kinv,
                                                nullptr, ctx->dflags, s);
  if (e == cudaSuccess)
    e = ssl::launch_correlate_f64(reinterpret_cast<const float2*>(X), nblk, T, B, M, Rw, s);
  if (e == cudaSuccess)
    e = ssl::launch_gsvd_f64(Rw, Kinv, nblk, B, M, jo.max_sweeps, cfg->jacobi.rel_tol,
                             jo.abs_tol, sig, Ew, nullptr, nullptr, ctx->dflags, s);
  if (e == cudaSuccess)
    e = ssl::launch_spectrum_f64(Ew, nblk, B, M, Ns, st->H, D, cfg->form, Pw, s);
  if (e == cudaSuccess) e = ssl::launch_bin_sum_f64(Pw, nblk, B, D, Pb, s);
  if (e == cudaSuccess)
    e = lists ? ssl::launch_peaks_nbr(Pb, nblk, D, st->nbr_ptr, st->nbr_idx, Ns, peak_idx,
                                      peak_val, s, ctx->dflags, st->range)
              : ssl::launch_peaks(Pb, nblk, cfg->n_az, cfg->n_el, Ns, peak_idx, peak_val, s,
                                  st->range);
  return e == cudaSuccess ? SSL_OK : cuda_fail(ctx, e, "ssl_localize_f64");
}

}  // extern "C"

namespace ssl {
bool ctx_jacobi(const ssl_jacobi_opts* o, JacobiOpts* out) { return jacobi_opts(o, out); }
ssl_status steering_tables(ssl_ctx* ctx, const ssl_steering* cst, int precision, const float2** H,
                           const float** hnorm2, const CUtensorMap** tm, const Geo** geo) {
  ssl_steering* st = const_cast<ssl_steering*>(cst);
  *tm = nullptr;
  if (geo) *geo = nullptr;
  const bool tc = precision == SSL_PREC_TF32 || precision == SSL_PREC_BF16;
  if (st->analytic && tc && geo) {  // the caller's kernels generate the tiles
    *geo = st->geo;
    *H = nullptr;
    *hnorm2 = nullptr;
    return SSL_OK;
  }
  if (st->analytic) {
    ssl_status r = ensure_table(ctx, st);
    if (r != SSL_OK) return r;
  }
  *H = st->H;
  *hnorm2 = st->hnorm2;
  if (tc) {
    ssl_status r = steering_image(ctx, st, precision);
    if (r != SSL_OK) return r;
    *tm = &st->tm[precision == SSL_PREC_BF16 ? 1 : 0];
  }
  return SSL_OK;
}
}  // namespace ssl

