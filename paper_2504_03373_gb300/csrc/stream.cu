// Stream (per-frame) processing: the sliding form of eq. 3 with a
// warm-started decomposition.
//
// A stream is one array that delivers `hop` new frames at a time.  It keeps
// the last T frames in a device ring, K^{-1} (FP64 Cholesky at creation), and
// the previous decomposition's E.  Each push overwrites the oldest frames,
// recomputes R over the window (the sum of eq. 3 does not depend on the
// frames' order), and continues the Jacobi iteration from the previous E:
// with G0 = A^H E_prev (whitening with E_prev^H K^{-1}, see cgemm.cu) and
// V0 = E_prev, consecutive windows that share T - hop frames need a fraction
// of the rotations of a cold start.  Spectrum, bin sum and peaks follow as in
// the block path.
#include <cuda.h>
#include <cuda_runtime.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "ssl_internal.cuh"

struct ssl_stream {
  ssl_ctx* ctx = nullptr;
  int device = 0;
  ssl_config cfg{};
  int hop = 0;
  const ssl_steering* st = nullptr;
  ssl::JacobiOpts jo{};
  void* arena = nullptr;
  float2* kinv = nullptr;  // [B][M][M]
  float2* ring = nullptr;  // [T][B][M]
  float2* E[2] = {nullptr, nullptr};
  float2* R = nullptr;
  float2* KE = nullptr;
  float* sig = nullptr;
  int32_t* bst = nullptr;
  void* img = nullptr;
  float* P = nullptr;
  float* Pbar = nullptr;
  int32_t* idx = nullptr;
  float* val = nullptr;
  int pos = 0;        // ring frame the next push starts at
  int cur = 0;        // E[cur] holds the last decomposition
  bool warm = false;  // E[cur] is valid
};

namespace {

size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

struct Guard {
  int prev = -1;
  explicit Guard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~Guard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

ssl_status cuda_err(ssl_ctx* ctx, const char* what) {
  cudaGetLastError();
  return ssl::ctx_error(ctx, SSL_E_CUDA, what);
}

}  // namespace

extern "C" {

ssl_status ssl_stream_create(ssl_ctx* ctx, const ssl_config* cfg, int hop, const float* K,
                             const ssl_steering* st, ssl_stream** out) {
  ssl::Range nvtx("ssl_stream_create");
  if (!ctx || !cfg || !K || !st || !out) return SSL_E_INVALID_ARG;
  *out = nullptr;
  const ssl_config& c = *cfg;
  // n_el == 0: a direction set of n_az directions with the steering object's
  // neighbour lists
  const int D = c.n_el == 0 ? c.n_az : c.n_az * c.n_el;
  ssl::JacobiOpts jo{};
  const int32_t *lp = nullptr, *li = nullptr;
  if (c.M < 2 || c.M > SSL_MAX_M || c.T < 1 || c.B < 1 || c.Ns < 1 || c.Ns >= c.M ||
      c.Ns > SSL_MAX_NS || c.n_az < 1 || c.n_el < 0 || D > SSL_MAX_D || hop < 1 || hop > c.T ||
      (c.n_el == 0 && !ssl::steering_lists(st, &lp, &li)) ||
      (c.form != SSL_FORM_ABS && c.form != SSL_FORM_SQ) ||
      (c.precision != SSL_PREC_FP32 && c.precision != SSL_PREC_TF32 &&
       c.precision != SSL_PREC_BF16) ||
      !ssl::ctx_jacobi(&c.jacobi, &jo) || !ssl::steering_matches(st, c.B, D, c.M))
    return ssl::ctx_error(ctx, SSL_E_INVALID_ARG, "ssl_stream_create: bad arguments");
  if (jo.method == SSL_SVD_SPLIT && c.form != SSL_FORM_SQ)
    return ssl::ctx_error(ctx, SSL_E_UNSUPPORTED,
                          "ssl_stream_create: the split iteration gives the noise subspace, the "
                          "ABS form needs its individual vectors");
  jo.split_ns = c.Ns;  // (the split iteration starts cold at every push)
  Guard g(ssl::ctx_device(ctx));
  {
    // build the steering table / tensor-core image now (a build synchronises
    // the device), not in the first push
    const float2* H = nullptr;
    const float* hn = nullptr;
    const CUtensorMap* tm = nullptr;
    const ssl_status r = ssl::steering_tables(ctx, st, c.precision, &H, &hn, &tm);
    if (r != SSL_OK) return r;
  }
  ssl_stream* s = new (std::nothrow) ssl_stream();
  if (!s) return SSL_E_OOM;
  s->ctx = ctx;
  s->device = ssl::ctx_device(ctx);
  s->cfg = c;
  s->hop = hop;
  s->st = st;
  s->jo = jo;
  const size_t mm = (size_t)c.B * c.M * c.M * sizeof(float2);
  const int esz = c.precision == SSL_PREC_BF16 ? 2 : 4;
  const size_t img = c.precision == SSL_PREC_FP32
                         ? 0
                         : (size_t)c.B * ssl::tc_np(c.M, c.Ns) * ssl::tc_kp(c.M) * esz;
  size_t off = 0;
  auto take = [&](size_t n) {
    const size_t o = off;
    off += a256(n);
    return o;
  };
  const size_t o_kinv = take(mm), o_ring = take((size_t)c.T * c.B * c.M * sizeof(float2));
  const size_t o_e0 = take(mm), o_e1 = take(mm), o_r = take(mm), o_ke = take(mm);
  const size_t o_sig = take((size_t)c.B * c.M * 4), o_bst = take((size_t)c.B * 4);
  const size_t o_img = take(img), o_p = take((size_t)c.B * D * 4);
  const size_t o_pbar = take((size_t)D * 4), o_idx = take((size_t)c.Ns * 4);
  const size_t o_val = take((size_t)c.Ns * 4), o_k = take(mm), o_kst = take((size_t)c.B * 4);
  if (cudaMalloc(&s->arena, off) != cudaSuccess) {
    delete s;
    return cuda_err(ctx, "ssl_stream_create: device memory");
  }
  char* b = static_cast<char*>(s->arena);
  s->kinv = reinterpret_cast<float2*>(b + o_kinv);
  s->ring = reinterpret_cast<float2*>(b + o_ring);
  s->E[0] = reinterpret_cast<float2*>(b + o_e0);
  s->E[1] = reinterpret_cast<float2*>(b + o_e1);
  s->R = reinterpret_cast<float2*>(b + o_r);
  s->KE = reinterpret_cast<float2*>(b + o_ke);
  s->sig = reinterpret_cast<float*>(b + o_sig);
  s->bst = reinterpret_cast<int32_t*>(b + o_bst);
  s->img = img ? b + o_img : nullptr;
  s->P = reinterpret_cast<float*>(b + o_p);
  s->Pbar = reinterpret_cast<float*>(b + o_pbar);
  s->idx = reinterpret_cast<int32_t*>(b + o_idx);
  s->val = reinterpret_cast<float*>(b + o_val);
  float2* Kd = reinterpret_cast<float2*>(b + o_k);
  int32_t* kst = reinterpret_cast<int32_t*>(b + o_kst);
  // K (host or device) -> K^{-1} by FP64 Cholesky; the window starts empty
  cudaStream_t cs = nullptr;
  bool ok = cudaMemcpy(Kd, K, mm, cudaMemcpyDefault) == cudaSuccess &&
            cudaMemset(s->ring, 0, (size_t)c.T * c.B * c.M * sizeof(float2)) == cudaSuccess &&
            ssl::launch_noise_inverse(Kd, c.B, c.M, s->kinv, kst, ssl::ctx_flags(ctx), cs) ==
                cudaSuccess;
  int32_t worst = 0;
  if (ok) {
    std::vector<int32_t> h(c.B);
    ok = cudaMemcpy(h.data(), kst, (size_t)c.B * 4, cudaMemcpyDeviceToHost) == cudaSuccess;
    for (int32_t v : h) worst = v > worst ? v : worst;
  }
  if (!ok) {
    cudaFree(s->arena);
    delete s;
    return cuda_err(ctx, "ssl_stream_create: K^{-1}");
  }
  if (worst != 0) {
    cudaFree(s->arena);
    delete s;
    return ssl::ctx_error(ctx, worst, "ssl_stream_create: K is not positive definite");
  }
  *out = s;
  return SSL_OK;
}

ssl_status ssl_stream_push(ssl_stream* s, const float* X, int32_t* peak_idx, float* peak_val,
                           float* Pbar, int32_t* stats, void* stream) {
  if (!s || !X || !peak_idx || !peak_val) return SSL_E_INVALID_ARG;
  ssl::Range nvtx("ssl_stream_push");
  Guard g(s->device);
  const ssl_config& c = s->cfg;
  cudaStream_t cs = static_cast<cudaStream_t>(stream);
  const size_t frame = (size_t)c.B * c.M;
  const int D = c.n_el == 0 ? c.n_az : c.n_az * c.n_el;
  // the hop new frames replace the oldest ones (one or two copies)
  const int first = std::min(s->hop, c.T - s->pos);
  cudaError_t e = cudaMemcpyAsync(s->ring + (size_t)s->pos * frame, X,
                                  (size_t)first * frame * sizeof(float2), cudaMemcpyDefault, cs);
  if (e == cudaSuccess && first < s->hop)
    e = cudaMemcpyAsync(s->ring, reinterpret_cast<const float2*>(X) + (size_t)first * frame,
                        (size_t)(s->hop - first) * frame * sizeof(float2), cudaMemcpyDefault, cs);
  if (e != cudaSuccess) return cuda_err(s->ctx, "ssl_stream_push: frame copy");
  s->pos = (s->pos + s->hop) % c.T;
  // eq. 2-3 over the window
  e = ssl::launch_correlate(s->ring, 1, c.T, c.B, c.M, s->R, cs);
  // eq. 4, continuing from the previous E when there is one
  unsigned* flags = ssl::ctx_flags(s->ctx);
  float2* Eout = s->E[s->warm ? 1 - s->cur : s->cur];
  if (e == cudaSuccess) {
    if (s->warm && s->jo.method == SSL_SVD_JACOBI) {
      // E_prev^H K^{-1}
      e = ssl::launch_cgemm(s->E[s->cur], true, true, s->kinv, false, false, 1, c.B, c.M, s->KE,
                            cs);
      if (e == cudaSuccess)
        e = ssl::launch_gsvd(s->R, s->KE, 1, c.B, c.M, s->jo, s->sig, Eout, s->bst, stats, flags,
                             cs, nullptr, s->E[s->cur]);
    } else {
      // (the split iteration forms A in KE's space, unused without the warm start)
      e = ssl::launch_gsvd(s->R, s->kinv, 1, c.B, c.M, s->jo, s->sig, Eout, s->bst, stats, flags,
                           cs, nullptr, nullptr, nullptr,
                           s->jo.method == SSL_SVD_SPLIT ? s->KE : nullptr);
    }
  }
  // eq. 5-6 and the peaks
  if (e == cudaSuccess) {
    const float2* H = nullptr;
    const float* hn = nullptr;
    const CUtensorMap* tm = nullptr;
    if (ssl::steering_tables(s->ctx, s->st, c.precision, &H, &hn, &tm) != SSL_OK)
      return cuda_err(s->ctx, "ssl_stream_push: steering tables");
    if (c.precision == SSL_PREC_FP32) {
      e = ssl::launch_spectrum_simt(Eout, 1, c.B, c.M, c.Ns, H, hn, D, c.form, s->P, cs);
    } else {
      const int esz = c.precision == SSL_PREC_BF16 ? 2 : 4;
      const int KP = ssl::tc_kp(c.M), NP = ssl::tc_np(c.M, c.Ns);
      e = ssl::launch_pack_e(Eout, c.B, c.M, c.Ns, c.precision, s->img, cs);
      CUtensorMap tmE;
      if (e == cudaSuccess &&
          !ssl::encode_tmap_3d(&tmE, s->img, esz, KP, NP, (uint64_t)c.B, 128 / esz, NP))
        return cuda_err(s->ctx, "ssl_stream_push: tensor map");
      if (e == cudaSuccess)
        e = ssl::launch_spectrum_tc(*tm, tmE, 1, c.B, D, c.M, c.Ns, c.precision, c.form, hn,
                                    s->P, flags, cs, nullptr, nullptr, ssl::ctx_wait_ns(s->ctx));
    }
  }
  if (e == cudaSuccess) e = ssl::launch_bin_sum(s->P, 1, c.B, D, s->Pbar, cs);
  if (e == cudaSuccess) {
    const int32_t *lp = nullptr, *li = nullptr;
    const uint8_t* in = ssl::steering_range(s->st);
    e = c.n_el == 0 && ssl::steering_lists(s->st, &lp, &li)
            ? ssl::launch_peaks_nbr(s->Pbar, 1, D, lp, li, c.Ns, s->idx, s->val, cs, flags, in)
            : ssl::launch_peaks(s->Pbar, 1, c.n_az, c.n_el, c.Ns, s->idx, s->val, cs, in);
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(peak_idx, s->idx, (size_t)c.Ns * 4, cudaMemcpyDefault, cs);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(peak_val, s->val, (size_t)c.Ns * 4, cudaMemcpyDefault, cs);
  if (e == cudaSuccess && Pbar)
    e = cudaMemcpyAsync(Pbar, s->Pbar, (size_t)D * 4, cudaMemcpyDefault, cs);
  if (e != cudaSuccess) return cuda_err(s->ctx, "ssl_stream_push: launch");
  if (s->warm) s->cur = 1 - s->cur;
  s->warm = true;
  return SSL_OK;
}

ssl_status ssl_stream_destroy(ssl_stream* s) {
  if (!s) return SSL_OK;
  Guard g(s->device);
  cudaDeviceSynchronize();
  cudaFree(s->arena);
  delete s;
  return SSL_OK;
}

}  // extern "C"
