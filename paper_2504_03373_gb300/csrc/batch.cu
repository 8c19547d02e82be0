// Mixed batches: many arrays of different sizes, one launch per stage.
//
// A plan owns a device arena with the per-array scratch (R, E, singular
// values, bin status, tensor-core E images, spectra) and the tables the
// mixed kernels read: one MixedItem per array, the (array, bin) list, one
// GsvdProblem per (array, bin) and the Jacobi work units.  A run enqueues
//   correlation -> whitening + Jacobi (persistent) -> [E image] -> spectrum
//   -> bin sum -> peaks + status
// over every (array, bin) pair at once, or replays the CUDA graph captured
// from that sequence at creation.  The optional autotuner times each Jacobi
// size class an M admits (16, 32 or 64 rows per matrix, i.e. one, two or
// four warps per matrix) on the plan's own data and keeps the fastest.
#include <cuda.h>
#include <cuda_runtime.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <new>
#include <vector>

#include "ssl_internal.cuh"

struct ssl_plan {
  ssl_ctx* ctx = nullptr;
  int device = 0;
  int n = 0;
  int form = 0, precision = 0;
  ssl::JacobiOpts jo{};
  void* arena = nullptr;
  ssl::MixedItem* items_d = nullptr;
  int2* ctab_d = nullptr;
  ssl::GsvdProblem* probs_d = nullptr;
  ssl::GsvdUnit* units_d = nullptr;
  int* counter_d = nullptr;
  int n_ctab = 0, n_units = 0, d_max = 0, grid = 0, launches = 0;
  std::vector<int> prob_m;  // M of every problem (host copy, for the unit lists)
  int class_of_m[SSL_MAX_M + 1] = {};
  double autotune_ms = 0.0;
  cudaStream_t cap = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

namespace {

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

struct DevGuard {
  int prev = -1;
  explicit DevGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DevGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

// Directions of an array: its grid, or (n_el == 0) a direction set of n_az
// directions whose peak search uses the steering object's neighbour lists.
int n_dirs(const ssl_config& c) { return c.n_el == 0 ? c.n_az : c.n_az * c.n_el; }

bool cfg_valid(const ssl_config& c) {
  const int D = n_dirs(c);
  return c.M >= 2 && c.M <= SSL_MAX_M && c.T >= 1 && c.B >= 1 && c.Ns >= 1 && c.Ns < c.M &&
         c.Ns <= SSL_MAX_NS && c.n_az >= 1 && c.n_el >= 0 && D <= SSL_MAX_D &&
         (c.form == SSL_FORM_ABS || c.form == SSL_FORM_SQ) &&
         (c.precision == SSL_PREC_FP32 || c.precision == SSL_PREC_TF32 ||
          c.precision == SSL_PREC_BF16);
}

bool same_jacobi(const ssl_jacobi_opts& a, const ssl_jacobi_opts& b) {
  return a.max_sweeps == b.max_sweeps && a.rel_tol == b.rel_tol && a.abs_tol == b.abs_tol &&
         a.angles == b.angles && a.method == b.method;
}

int default_class(int M) { return M <= 16 ? 16 : (M <= 32 ? 32 : 64); }

// Work units for the problems whose M is accepted by `want`, with the size
// class of each M from cls: the 64 class first (longest), then 32, then 16.
template <class Want>
std::vector<ssl::GsvdUnit> make_units(const std::vector<int>& prob_m, const int* cls, Want want) {
  std::vector<ssl::GsvdUnit> out;
  for (int mp : {64, 32, 16}) {
    const int per = 64 / mp;
    ssl::GsvdUnit u{mp, 0, {0, 0, 0, 0}};
    for (int i = 0; i < (int)prob_m.size(); ++i) {
      if (!want(prob_m[i]) || cls[prob_m[i]] != mp) continue;
      u.prob[u.n++] = i;
      if (u.n == per) {
        out.push_back(u);
        u = ssl::GsvdUnit{mp, 0, {0, 0, 0, 0}};
      }
    }
    if (u.n > 0) out.push_back(u);
  }
  return out;
}

cudaError_t enqueue(ssl_plan* p, cudaStream_t s) {
  const bool tc = p->precision != SSL_PREC_FP32;
  unsigned* flags = ssl::ctx_flags(p->ctx);
  cudaError_t e = ssl::launch_correlate_mixed(p->items_d, p->ctab_d, p->n_ctab, s);
  if (e == cudaSuccess)
    e = p->jo.method == SSL_SVD_BIDIAG
            ? ssl::launch_gsvd_bidiag(nullptr, nullptr, 0, 0, 0, p->jo, nullptr, nullptr, nullptr,
                                      nullptr, flags, s, nullptr, p->probs_d, p->n_ctab)
            : ssl::launch_gsvd_mixed(p->units_d, p->n_units, p->probs_d, p->counter_d, p->grid,
                                     p->jo, flags, s);
  if (e == cudaSuccess) {
    if (tc) {  // the decomposition wrote the operand images of E_n
      e = ssl::launch_spectrum_tc_mixed(p->items_d, p->ctab_d, p->n_ctab, p->precision, p->form,
                                        flags, s, ssl::ctx_wait_ns(p->ctx));
    } else {
      e = ssl::launch_spectrum_simt_mixed(p->items_d, p->ctab_d, p->n_ctab, p->d_max, p->form, s);
    }
  }
  if (e == cudaSuccess) e = ssl::launch_bin_sum_mixed(p->items_d, p->n, p->d_max, s);
  if (e == cudaSuccess) e = ssl::launch_peaks_mixed(p->items_d, p->n, p->d_max, s);
  return e;
}

void release(ssl_plan* p) {
  if (p->exec) cudaGraphExecDestroy(p->exec);
  if (p->graph) cudaGraphDestroy(p->graph);
  if (p->cap) cudaStreamDestroy(p->cap);
  if (p->arena) cudaFree(p->arena);
  delete p;
}

ssl_status plan_fail(ssl_plan* p, ssl_ctx* ctx, ssl_status st, const char* msg) {
  cudaGetLastError();
  if (p) release(p);
  return ssl::ctx_error(ctx, st, msg);
}

// Milliseconds of the Jacobi stage over `units` (best of three after one
// warm-up run), on the plan's capture stream.
float time_units(ssl_plan* p, const std::vector<ssl::GsvdUnit>& units, ssl::GsvdUnit* dev_units,
                 int grid) {
  if (units.empty()) return 0.f;
  if (cudaMemcpy(dev_units, units.data(), units.size() * sizeof(ssl::GsvdUnit),
                 cudaMemcpyHostToDevice) != cudaSuccess)
    return -1.f;
  cudaEvent_t a = nullptr, b = nullptr;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  float best = -1.f;
  for (int r = 0; r < 4; ++r) {
    cudaEventRecord(a, p->cap);
    cudaError_t e = ssl::launch_gsvd_mixed(dev_units, (int)units.size(), p->probs_d, p->counter_d,
                                           grid, p->jo, ssl::ctx_flags(p->ctx), p->cap);
    cudaEventRecord(b, p->cap);
    if (e != cudaSuccess || cudaEventSynchronize(b) != cudaSuccess) {
      best = -1.f;
      break;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    if (r > 0 && (best < 0.f || ms < best)) best = ms;
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return best;
}

}  // namespace

extern "C" {

ssl_status ssl_plan_create(ssl_ctx* ctx, int n, const ssl_batch_item* items, unsigned flags,
                           ssl_plan** out) {
  ssl::Range nvtx("ssl_plan_create");
  if (!ctx || !out || n < 1 || !items || (flags & ~(SSL_PLAN_GRAPH | SSL_PLAN_AUTOTUNE)))
    return ssl::ctx_error(ctx, SSL_E_INVALID_ARG, "ssl_plan_create: bad arguments");
  *out = nullptr;
  const ssl_config& c0 = items[0].cfg;
  ssl::JacobiOpts jo{};
  if (!ssl::ctx_jacobi(&c0.jacobi, &jo))
    return ssl::ctx_error(ctx, SSL_E_INVALID_ARG, "ssl_plan_create: bad Jacobi options");
  if (jo.method == SSL_SVD_SPLIT)
    return ssl::ctx_error(ctx, SSL_E_UNSUPPORTED,
                          "ssl_plan_create: plans run the one-sided Jacobi or the paper's route");
  for (int i = 0; i < n; ++i) {
    const ssl_batch_item& it = items[i];
    const ssl_config& c = it.cfg;
    const int32_t *lp = nullptr, *li = nullptr;
    if (!cfg_valid(c) || c.form != c0.form || c.precision != c0.precision ||
        !same_jacobi(c.jacobi, c0.jacobi) || !it.X || !it.Kinv || !it.peak_idx || !it.peak_val ||
        !ssl::steering_matches(it.steering, c.B, n_dirs(c), c.M) ||
        (c.n_el == 0 && !ssl::steering_lists(it.steering, &lp, &li)))
      return ssl::ctx_error(ctx, SSL_E_INVALID_ARG,
                            "ssl_plan_create: invalid item or items that disagree on form, "
                            "precision or Jacobi options");
  }
  DevGuard dg(ssl::ctx_device(ctx));
  ssl_plan* p = new (std::nothrow) ssl_plan();
  if (!p) return ssl::ctx_error(ctx, SSL_E_OOM, "ssl_plan_create: host allocation");
  p->ctx = ctx;
  p->device = ssl::ctx_device(ctx);
  p->n = n;
  p->form = c0.form;
  p->precision = c0.precision;
  p->jo = jo;
  const bool tc = p->precision != SSL_PREC_FP32;
  const int esz = p->precision == SSL_PREC_BF16 ? 2 : 4;

  // ---- arena layout ----
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off += align256(bytes);
    return o;
  };
  struct Offs {
    size_t R, E, sig, bst, img, P, Pbar;
  };
  std::vector<Offs> o(n);
  for (int i = 0; i < n; ++i) {
    const ssl_config& c = items[i].cfg;
    const int D = n_dirs(c);
    const size_t mm = (size_t)c.M * c.M * sizeof(float2);
    o[i].R = take((size_t)c.B * mm);
    o[i].E = tc ? 0 : take((size_t)c.B * mm);  // E_n is only formed for the FP32 spectrum
    o[i].sig = take((size_t)c.B * c.M * sizeof(float));
    o[i].bst = take((size_t)c.B * sizeof(int32_t));
    o[i].img = tc ? take((size_t)c.B * ssl::tc_np(c.M, c.Ns) * ssl::tc_kp(c.M) * esz) : 0;
    o[i].P = take((size_t)c.B * D * sizeof(float));
    o[i].Pbar = items[i].Pbar ? 0 : take((size_t)D * sizeof(float));
    p->n_ctab += c.B;
    p->d_max = std::max(p->d_max, D);
  }
  const size_t o_items = take((size_t)n * sizeof(ssl::MixedItem));
  const size_t o_ctab = take((size_t)p->n_ctab * sizeof(int2));
  const size_t o_probs = take((size_t)p->n_ctab * sizeof(ssl::GsvdProblem));
  const size_t o_units = take((size_t)p->n_ctab * sizeof(ssl::GsvdUnit));
  const size_t o_tune = take((size_t)p->n_ctab * sizeof(ssl::GsvdUnit));
  const size_t o_counter = take(sizeof(int));
  if (cudaMalloc(&p->arena, off) != cudaSuccess)
    return plan_fail(p, ctx, SSL_E_OOM, "ssl_plan_create: device arena");
  char* base = static_cast<char*>(p->arena);

  // ---- tables ----
  std::vector<ssl::MixedItem> mi(n);
  std::vector<int2> ctab;
  std::vector<ssl::GsvdProblem> probs;
  ctab.reserve(p->n_ctab);
  probs.reserve(p->n_ctab);
  for (int i = 0; i < n; ++i) {
    const ssl_batch_item& it = items[i];
    const ssl_config& c = it.cfg;
    ssl::MixedItem& m = mi[i];
    memset(&m, 0, sizeof(m));
    const float2* H = nullptr;
    const float* hn = nullptr;
    const CUtensorMap* tm = nullptr;
    if (ssl::steering_tables(ctx, it.steering, p->precision, &H, &hn, &tm) != SSL_OK)
      return plan_fail(p, ctx, SSL_E_CUDA, "ssl_plan_create: steering tables");
    m.X = reinterpret_cast<const float2*>(it.X);
    m.Kinv = reinterpret_cast<const float2*>(it.Kinv);
    m.H = H;
    m.hn = hn;
    m.R = reinterpret_cast<float2*>(base + o[i].R);
    m.E = tc ? nullptr : reinterpret_cast<float2*>(base + o[i].E);
    m.sig = reinterpret_cast<float*>(base + o[i].sig);
    m.bst = reinterpret_cast<int32_t*>(base + o[i].bst);
    m.eimg = tc ? base + o[i].img : nullptr;
    m.P = reinterpret_cast<float*>(base + o[i].P);
    m.Pbar = it.Pbar ? it.Pbar : reinterpret_cast<float*>(base + o[i].Pbar);
    m.idx = it.peak_idx;
    m.val = it.peak_val;
    m.status = it.status;
    m.M = c.M;
    m.T = c.T;
    m.B = c.B;
    m.Ns = c.Ns;
    m.n_az = c.n_az;
    m.n_el = c.n_el;
    m.D = n_dirs(c);
    m.nbr_ptr = m.nbr_idx = nullptr;
    if (c.n_el == 0) ssl::steering_lists(it.steering, &m.nbr_ptr, &m.nbr_idx);
    m.range = ssl::steering_range(it.steering);
    m.KP = ssl::tc_kp(c.M);
    m.NP = ssl::tc_np(c.M, c.Ns);
    if (tc) {
      m.tmH = *tm;
      if (!ssl::encode_tmap_3d(&m.tmE, m.eimg, esz, m.KP, m.NP, c.B, 128 / esz, m.NP))
        return plan_fail(p, ctx, SSL_E_CUDA, "ssl_plan_create: E image tensor map");
    }
    const size_t mm = (size_t)c.M * c.M;
    const size_t img_bin = (size_t)m.NP * m.KP * esz;  // image bytes per bin
    for (int w = 0; w < c.B; ++w) {
      ctab.push_back(make_int2(i, w));
      // with the tensor-core spectrum the decomposition writes the operand
      // image of E_n itself (E is not formed)
      void* img = tc ? static_cast<char*>(m.eimg) + w * img_bin : nullptr;
      probs.push_back(ssl::GsvdProblem{m.R + w * mm, m.Kinv + w * mm, m.sig + (size_t)w * c.M,
                                       tc ? nullptr : m.E + w * mm, m.bst + w, c.M, w, img, esz,
                                       c.Ns, m.KP, m.NP});
      p->prob_m.push_back(c.M);
    }
  }
  p->items_d = reinterpret_cast<ssl::MixedItem*>(base + o_items);
  p->ctab_d = reinterpret_cast<int2*>(base + o_ctab);
  p->probs_d = reinterpret_cast<ssl::GsvdProblem*>(base + o_probs);
  p->units_d = reinterpret_cast<ssl::GsvdUnit*>(base + o_units);
  ssl::GsvdUnit* tune_d = reinterpret_cast<ssl::GsvdUnit*>(base + o_tune);
  p->counter_d = reinterpret_cast<int*>(base + o_counter);
  if (cudaMemcpy(p->items_d, mi.data(), (size_t)n * sizeof(ssl::MixedItem),
                 cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(p->ctab_d, ctab.data(), ctab.size() * sizeof(int2), cudaMemcpyHostToDevice) !=
          cudaSuccess ||
      cudaMemcpy(p->probs_d, probs.data(), probs.size() * sizeof(ssl::GsvdProblem),
                 cudaMemcpyHostToDevice) != cudaSuccess)
    return plan_fail(p, ctx, SSL_E_CUDA, "ssl_plan_create: table upload");
  if (cudaStreamCreateWithFlags(&p->cap, cudaStreamNonBlocking) != cudaSuccess)
    return plan_fail(p, ctx, SSL_E_CUDA, "ssl_plan_create: stream");

  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->device);
  p->grid = std::max(1, sms) * ssl::gsvd_mixed_ctas_per_sm();
  std::vector<bool> present(SSL_MAX_M + 1, false);
  for (int m : p->prob_m) present[m] = true;
  for (int m = 0; m <= SSL_MAX_M; ++m) p->class_of_m[m] = present[m] ? default_class(m) : 0;

  // ---- autotuner: Jacobi size class per M, timed on this plan's matrices ----
  if ((flags & SSL_PLAN_AUTOTUNE) && jo.method == SSL_SVD_JACOBI) {
    const auto t0 = std::chrono::steady_clock::now();
    if (ssl::launch_correlate_mixed(p->items_d, p->ctab_d, p->n_ctab, p->cap) != cudaSuccess ||
        cudaStreamSynchronize(p->cap) != cudaSuccess)
      return plan_fail(p, ctx, SSL_E_CUDA, "ssl_plan_create: autotune correlation");
    for (int m = 2; m <= SSL_MAX_M; ++m) {
      if (!present[m] || m > 32) continue;
      float best = -1.f;
      int best_cls = default_class(m);
      for (int cls : {16, 32, 64}) {
        if (cls < m) continue;
        int cl[SSL_MAX_M + 1];
        std::copy(p->class_of_m, p->class_of_m + SSL_MAX_M + 1, cl);
        cl[m] = cls;
        const auto units = make_units(p->prob_m, cl, [m](int mm) { return mm == m; });
        const float ms = time_units(p, units, tune_d, p->grid);
        if (ms < 0.f) return plan_fail(p, ctx, SSL_E_CUDA, "ssl_plan_create: autotune launch");
        if (best < 0.f || ms < best) {
          best = ms;
          best_cls = cls;
        }
      }
      p->class_of_m[m] = best_cls;
    }
    p->autotune_ms =
        std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  }
  const auto units = make_units(p->prob_m, p->class_of_m, [](int) { return true; });
  p->n_units = (int)units.size();
  if (cudaMemcpy(p->units_d, units.data(), units.size() * sizeof(ssl::GsvdUnit),
                 cudaMemcpyHostToDevice) != cudaSuccess)
    return plan_fail(p, ctx, SSL_E_CUDA, "ssl_plan_create: unit upload");
  p->launches = 5;  // correlation, decomposition (+ E_n image), spectrum, bin sum, peaks

  // ---- CUDA graph of one run ----
  if (flags & SSL_PLAN_GRAPH) {
    // one plain run first: kernel attributes are set outside the capture
    if (enqueue(p, p->cap) != cudaSuccess || cudaStreamSynchronize(p->cap) != cudaSuccess)
      return plan_fail(p, ctx, SSL_E_CUDA, "ssl_plan_create: first run");
    if (cudaStreamBeginCapture(p->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
      return plan_fail(p, ctx, SSL_E_CUDA, "ssl_plan_create: begin capture");
    const cudaError_t e = enqueue(p, p->cap);
    const cudaError_t e2 = cudaStreamEndCapture(p->cap, &p->graph);
    if (e != cudaSuccess || e2 != cudaSuccess ||
        cudaGraphInstantiate(&p->exec, p->graph, 0) != cudaSuccess)
      return plan_fail(p, ctx, SSL_E_CUDA, "ssl_plan_create: graph capture");
  }
  if (cudaDeviceSynchronize() != cudaSuccess)
    return plan_fail(p, ctx, SSL_E_CUDA, "ssl_plan_create: synchronise");
  *out = p;
  return SSL_OK;
}

ssl_status ssl_plan_run(ssl_plan* p, void* stream) {
  if (!p) return SSL_E_INVALID_ARG;
  ssl::Range nvtx("ssl_plan_run");
  DevGuard dg(p->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const cudaError_t e = p->exec ? cudaGraphLaunch(p->exec, s) : enqueue(p, s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return ssl::ctx_error(p->ctx, SSL_E_CUDA, "ssl_plan_run: launch failed");
  }
  return SSL_OK;
}

ssl_status ssl_plan_get_info(const ssl_plan* p, ssl_plan_info* out) {
  if (!p || !out) return SSL_E_INVALID_ARG;
  memset(out, 0, sizeof(*out));
  out->n_items = p->n;
  out->n_bins = p->n_ctab;
  out->gsvd_units = p->n_units;
  out->gsvd_grid = std::min(p->grid, p->n_units);
  out->launches = p->launches;
  out->graph = p->exec ? 1 : 0;
  std::copy(p->class_of_m, p->class_of_m + SSL_MAX_M + 1, out->class_of_m);
  out->autotune_ms = p->autotune_ms;
  return SSL_OK;
}

ssl_status ssl_plan_destroy(ssl_plan* p) {
  if (!p) return SSL_OK;
  DevGuard dg(p->device);
  if (p->cap) cudaStreamSynchronize(p->cap);
  release(p);
  return SSL_OK;
}

}  // extern "C"
