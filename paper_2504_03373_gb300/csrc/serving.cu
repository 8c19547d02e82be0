// Sessions and serving: many arrays, each sending blocks of T frames, served
// by continuous batching on one GPU.
//
// A session is one microphone array: its K^{-1} (FP64 Cholesky, computed once
// at creation), a caller-owned steering table, and a ring of device slots for
// blocks in flight.  ssl_session_submit copies a block into a free slot on the
// server's copy stream and queues it.  ssl_server_run_step
//   1. retires every batch whose completion event has fired: results move to
//      their sessions (with the latency t_done - t_arrival), slots are freed;
//   2. if fewer than kInFlight batches are on the GPU, launches one batch made
//      of every queued block: blocks are grouped by shape class (M, T, B, Ns,
//      grid, form, precision, Jacobi options) and each class runs the whole
//      hot path as one launch per stage, every block with its own array's
//      K^{-1} and steering through per-item pointer tables.
// Blocks submitted while a batch is on the GPU wait only for the next step,
// not for the batch to finish, so their copies and computation overlap the
// running batch.  Admission: a session is accepted only if its device
// footprint (K^{-1} and its input slots) fits the server's HBM budget; a
// submit to a full ring is refused (SSL_E_ADMISSION) until a slot frees.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <map>
#include <new>
#include <tuple>
#include <unordered_map>
#include <vector>

#include "ssl_internal.cuh"

namespace {

constexpr int kInFlight = 2;

uint64_t now_ns() {
  return (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(
             std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

struct ClassKey {
  int M, T, B, Ns, n_az, n_el, form, precision, sweeps, angles, method;
  float rel_tol, abs_tol;
  int analytic;  // generated steering tiles (analytic steering, TF32/BF16)
  bool operator<(const ClassKey& o) const {
    return std::tie(M, T, B, Ns, n_az, n_el, form, precision, sweeps, angles, method, rel_tol,
                    abs_tol, analytic) < std::tie(o.M, o.T, o.B, o.Ns, o.n_az, o.n_el, o.form,
                                                  o.precision, o.sweeps, o.angles, o.method,
                                                  o.rel_tol, o.abs_tol, o.analytic);
  }
};

ClassKey key_of(const ssl_config& c, bool analytic) {
  return ClassKey{c.M, c.T, c.B, c.Ns, c.n_az, c.n_el, c.form, c.precision,
                  c.jacobi.max_sweeps, c.jacobi.angles, c.jacobi.method, c.jacobi.rel_tol,
                  c.jacobi.abs_tol, analytic ? 1 : 0};
}

struct Item {
  ssl_session* s;
  int slot;
  ssl_ticket ticket;
  uint64_t t_arrival;
  cudaEvent_t copied;
};

// Device/pinned memory of one batch in flight (grown on demand).
struct BatchMem {
  void* dev = nullptr;
  size_t dev_bytes = 0;
  void* host = nullptr;  // pinned: pointer tables out, results back
  size_t host_bytes = 0;
};

struct Batch {
  bool active = false;
  cudaEvent_t done = nullptr;
  std::vector<Item> items;
  // per item, where its results land in the pinned buffer
  std::vector<int32_t*> idx;
  std::vector<float*> val;
  std::vector<int32_t*> status;
  BatchMem mem;
  uint64_t t_launch = 0;
};

}  // namespace

struct ssl_server {
  ssl_ctx* ctx = nullptr;
  int device = 0;
  size_t budget = 0, used = 0;
  int max_batch = 0;
  cudaStream_t stream = nullptr, copy_stream = nullptr;
  std::vector<ssl_session*> sessions;
  std::vector<Item> pending;
  Batch batch[kInFlight];
  std::vector<double> lat_ms;
  uint64_t blocks_done = 0, batches = 0, refused_sessions = 0, refused_blocks = 0;
  // wall time with at least one batch in flight: closed intervals summed in
  // busy_ms, the open one started at busy_since while in_flight > 0
  double busy_ms = 0.0;
  uint64_t busy_since = 0;
  int in_flight = 0;
  std::vector<cudaEvent_t> free_events;
};

struct ssl_session {
  ssl_server* srv = nullptr;
  ssl_config cfg{};
  int qdepth = 0;
  const ssl_steering* st = nullptr;
  float2* kinv = nullptr;
  float2* slots = nullptr;
  size_t slot_elems = 0;
  std::vector<int> free_slots;
  std::unordered_map<ssl_ticket, ssl_result> results;
  size_t footprint = 0;
  ssl_ticket next_ticket = 1;
  int inflight = 0;
};

namespace {

// Directions of an array: its grid, or (n_el == 0) a direction set of n_az
// directions whose peak search uses the steering object's neighbour lists.
int n_dirs(const ssl_config& c) { return c.n_el == 0 ? c.n_az : c.n_az * c.n_el; }

bool is_dev(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

cudaEvent_t get_event(ssl_server* s) {
  if (!s->free_events.empty()) {
    cudaEvent_t e = s->free_events.back();
    s->free_events.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return e;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

bool ensure(BatchMem& m, size_t dev_bytes, size_t host_bytes) {
  if (dev_bytes > m.dev_bytes) {
    if (m.dev) cudaFree(m.dev);
    m.dev = nullptr;
    m.dev_bytes = 0;
    if (cudaMalloc(&m.dev, dev_bytes) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    m.dev_bytes = dev_bytes;
  }
  if (host_bytes > m.host_bytes) {
    if (m.host) cudaFreeHost(m.host);
    m.host = nullptr;
    m.host_bytes = 0;
    if (cudaMallocHost(&m.host, host_bytes) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    m.host_bytes = host_bytes;
  }
  return true;
}

// Retire the finished batch b: results to their sessions, slots freed.
void retire(ssl_server* s, Batch& b) {
  const uint64_t t = now_ns();
  for (size_t i = 0; i < b.items.size(); ++i) {
    Item& it = b.items[i];
    ssl_session* se = it.s;
    ssl_result r{};
    r.done = 1;
    r.status = b.status[i][0];
    for (int k = 0; k < se->cfg.Ns && k < SSL_MAX_NS; ++k) {
      r.peak_idx[k] = b.idx[i][k];
      r.peak_val[k] = b.val[i][k];
    }
    r.t_arrival_ns = it.t_arrival;
    r.t_done_ns = t;
    se->results[it.ticket] = r;
    se->free_slots.push_back(it.slot);
    se->inflight--;
    s->lat_ms.push_back((double)(t - it.t_arrival) * 1e-6);
    s->free_events.push_back(it.copied);
  }
  s->blocks_done += b.items.size();
  b.items.clear();
  b.active = false;
}

// A batch found finished: the busy-time bookkeeping, then retire().
void retire_batch(ssl_server* s, Batch& b) {
  if (--s->in_flight == 0) s->busy_ms += (double)(now_ns() - s->busy_since) * 1e-6;
  retire(s, b);
}

// Run one shape class of items on the server stream.  `dev` and `host`
// point into the batch's arenas at this class's offsets.
ssl_status launch_class(ssl_server* s, Batch& b, const std::vector<int>& which, char* dev,
                        char* host, size_t& dev_off, size_t& host_off) {
  const ssl_session* s0 = b.items[which[0]].s;
  const ssl_config& c = s0->cfg;
  const int n = (int)which.size();
  const int M = c.M, T = c.T, B = c.B, Ns = c.Ns, D = n_dirs(c);
  const bool lists = c.n_el == 0;
  const size_t mm = (size_t)M * M * sizeof(float2);
  auto take_d = [&](size_t bytes) {
    char* p = dev + dev_off;
    dev_off += align256(bytes);
    return p;
  };
  auto take_h = [&](size_t bytes) {
    char* p = host + host_off;
    host_off += align256(bytes);
    return p;
  };
  // pointer tables, staged in pinned memory and copied in one go
  const size_t tab_bytes = (size_t)n * (8 * sizeof(void*)) + (size_t)n * sizeof(CUtensorMap);
  char* tab_h = take_h(tab_bytes + 128);
  char* tab_d = take_d(tab_bytes + 128);
  // CUtensorMap entries first (128-byte aligned), then the pointer arrays
  CUtensorMap* tm_h = reinterpret_cast<CUtensorMap*>(tab_h);
  const float2** x_h = reinterpret_cast<const float2**>(tab_h + (size_t)n * sizeof(CUtensorMap));
  const float2** k_h = x_h + n;
  const float2** H_h = k_h + n;
  const float** hn_h = reinterpret_cast<const float**>(H_h + n);
  const ssl::Geo** geo_h = reinterpret_cast<const ssl::Geo**>(hn_h + n);
  const int32_t** nptr_h = reinterpret_cast<const int32_t**>(geo_h + n);
  const int32_t** nidx_h = nptr_h + n;
  const uint8_t** rng_h = reinterpret_cast<const uint8_t**>(nidx_h + n);
  const bool tc = c.precision != SSL_PREC_FP32;
  bool gen = false;  // analytic steering: the spectrum kernel generates the tiles
  for (int i = 0; i < n; ++i) {
    const Item& it = b.items[which[i]];
    const float2* H = nullptr;
    const float* hn = nullptr;
    const CUtensorMap* tm = nullptr;
    const ssl::Geo* geo = nullptr;
    ssl_status r = ssl::steering_tables(s->ctx, it.s->st, c.precision, &H, &hn, &tm, &geo);
    if (r != SSL_OK) return r;
    x_h[i] = it.s->slots + (size_t)it.slot * it.s->slot_elems;
    k_h[i] = it.s->kinv;
    H_h[i] = H;
    hn_h[i] = hn;
    geo_h[i] = geo;
    nptr_h[i] = nidx_h[i] = nullptr;
    if (lists && !ssl::steering_lists(it.s->st, &nptr_h[i], &nidx_h[i])) return SSL_E_INVALID_ARG;
    rng_h[i] = ssl::steering_range(it.s->st);
    gen = geo != nullptr;  // the same for every item of a class
    if (tc && tm) tm_h[i] = *tm;
  }
  cudaError_t e = cudaMemcpyAsync(tab_d, tab_h, tab_bytes, cudaMemcpyHostToDevice, s->stream);
  if (e != cudaSuccess) return SSL_E_CUDA;
  const CUtensorMap* tm_d = reinterpret_cast<const CUtensorMap*>(tab_d);
  const float2* const* x_d =
      reinterpret_cast<const float2* const*>(tab_d + (size_t)n * sizeof(CUtensorMap));
  const float2* const* k_d = x_d + n;
  const float2* const* H_d = k_d + n;
  const float* const* hn_d = reinterpret_cast<const float* const*>(H_d + n);
  const ssl::Geo* const* geo_d = reinterpret_cast<const ssl::Geo* const*>(hn_d + n);
  const int32_t* const* nptr_d = reinterpret_cast<const int32_t* const*>(geo_d + n);
  const int32_t* const* nidx_d = nptr_d + n;
  const uint8_t* const* rng_d = reinterpret_cast<const uint8_t* const*>(nidx_d + n);

  float2* R = reinterpret_cast<float2*>(take_d((size_t)n * B * mm));
  float2* E = reinterpret_cast<float2*>(take_d((size_t)n * B * mm));
  float* sig = reinterpret_cast<float*>(take_d((size_t)n * B * M * sizeof(float)));
  int32_t* bst = reinterpret_cast<int32_t*>(take_d((size_t)n * B * sizeof(int32_t)));
  float* P = reinterpret_cast<float*>(take_d((size_t)n * B * D * sizeof(float)));
  float* Pbar = reinterpret_cast<float*>(take_d((size_t)n * D * sizeof(float)));
  int32_t* idx = reinterpret_cast<int32_t*>(take_d((size_t)n * Ns * sizeof(int32_t)));
  float* val = reinterpret_cast<float*>(take_d((size_t)n * Ns * sizeof(float)));
  int32_t* bstat = reinterpret_cast<int32_t*>(take_d((size_t)n * sizeof(int32_t)));
  const int esz = c.precision == SSL_PREC_BF16 ? 2 : 4;
  const int KP = ssl::tc_kp(M), NP = ssl::tc_np(M, Ns);
  void* img = tc ? take_d((size_t)n * B * NP * KP * esz) : nullptr;
  // the split iteration's A: E's space with the tensor-core spectrum, its own otherwise
  const bool split = c.jacobi.method == SSL_SVD_SPLIT;
  float2* abuf = !split ? nullptr : tc ? E : reinterpret_cast<float2*>(take_d((size_t)n * B * mm));

  ssl::JacobiOpts jo{c.jacobi.max_sweeps > 0 ? c.jacobi.max_sweeps : 30, c.jacobi.rel_tol,
                     c.jacobi.abs_tol, c.jacobi.angles == SSL_ANGLES_F64, c.jacobi.method, Ns};
  unsigned* flags = ssl::ctx_flags(s->ctx);
  e = ssl::launch_correlate(nullptr, n, T, B, M, R, s->stream, x_d);
  // with the tensor-core spectrum the decomposition writes its operand image
  // (E itself is not needed then)
  const ssl::ImgOut io{img, esz, Ns, KP, NP};
  if (e == cudaSuccess)
    e = ssl::launch_gsvd(R, nullptr, n, B, M, jo, sig, tc ? nullptr : E, bst, nullptr, flags,
                         s->stream, k_d, nullptr, tc ? &io : nullptr, abuf);
  if (e == cudaSuccess) {
    if (tc) {
      CUtensorMap tmE;
      if (e == cudaSuccess &&
          !ssl::encode_tmap_3d(&tmE, img, esz, KP, NP, (uint64_t)n * B, 128 / esz, NP))
        return SSL_E_CUDA;
      if (e == cudaSuccess)
        e = ssl::launch_spectrum_tc(tm_h[0], tmE, n, B, D, M, Ns, c.precision, c.form, nullptr,
                                    P, flags, s->stream, gen ? nullptr : tm_d,
                                    gen ? nullptr : hn_d, ssl::ctx_wait_ns(s->ctx), nullptr,
                                    gen ? geo_d : nullptr);
    } else {
      e = ssl::launch_spectrum_simt(E, n, B, M, Ns, nullptr, nullptr, D, c.form, P, s->stream,
                                    H_d, hn_d);
    }
  }
  if (e == cudaSuccess) e = ssl::launch_bin_sum(P, n, B, D, Pbar, s->stream);
  if (e == cudaSuccess)  // each item with its own lists (direction sets) and search range
    e = ssl::launch_peaks_items(Pbar, n, D, c.n_az, c.n_el, lists ? nptr_d : nullptr,
                                lists ? nidx_d : nullptr, rng_d, Ns, idx, val, s->stream, flags);
  if (e == cudaSuccess) e = ssl::launch_status_max(bst, n, B, bstat, s->stream);
  // results back to pinned memory
  int32_t* idx_h = reinterpret_cast<int32_t*>(take_h((size_t)n * Ns * sizeof(int32_t)));
  float* val_h = reinterpret_cast<float*>(take_h((size_t)n * Ns * sizeof(float)));
  int32_t* st_h = reinterpret_cast<int32_t*>(take_h((size_t)n * sizeof(int32_t)));
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(idx_h, idx, (size_t)n * Ns * sizeof(int32_t), cudaMemcpyDeviceToHost,
                        s->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(val_h, val, (size_t)n * Ns * sizeof(float), cudaMemcpyDeviceToHost,
                        s->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(st_h, bstat, (size_t)n * sizeof(int32_t), cudaMemcpyDeviceToHost,
                        s->stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return SSL_E_CUDA;
  }
  for (int i = 0; i < n; ++i) {
    b.idx[which[i]] = idx_h + (size_t)i * Ns;
    b.val[which[i]] = val_h + (size_t)i * Ns;
    b.status[which[i]] = st_h + i;
  }
  return SSL_OK;
}

// Bytes of device and pinned memory one class of n items needs.
void class_bytes(const ssl_config& c, int n, size_t& dev, size_t& host) {
  const int M = c.M, B = c.B, Ns = c.Ns, D = n_dirs(c);
  const size_t mm = (size_t)M * M * sizeof(float2);
  const int esz = c.precision == SSL_PREC_BF16 ? 2 : 4;
  // the pointer tables of launch_class: X, K^{-1}, H, |h|^2, geometry, the
  // two neighbour-list arrays and the search range per item, after the
  // tensor maps
  const size_t tab = (size_t)n * (8 * sizeof(void*)) + (size_t)n * sizeof(CUtensorMap) + 128;
  dev += align256(tab) + 2 * align256((size_t)n * B * mm) +
         align256((size_t)n * B * M * sizeof(float)) + align256((size_t)n * B * 4) +
         align256((size_t)n * B * D * sizeof(float)) + align256((size_t)n * D * sizeof(float)) +
         2 * align256((size_t)n * Ns * 4) + align256((size_t)n * 4) +
         (c.precision != SSL_PREC_FP32
              ? align256((size_t)n * B * ssl::tc_np(M, Ns) * ssl::tc_kp(M) * esz)
              : 0) +
         // the split iteration's A with the FP32 spectrum (else it uses E's space)
         (c.jacobi.method == SSL_SVD_SPLIT && c.precision == SSL_PREC_FP32
              ? align256((size_t)n * B * mm)
              : 0);
  host += align256(tab) + 2 * align256((size_t)n * Ns * 4) + align256((size_t)n * 4);
}

}  // namespace

extern "C" {

ssl_status ssl_now_ns(uint64_t* out) {
  if (!out) return SSL_E_INVALID_ARG;
  *out = now_ns();
  return SSL_OK;
}

ssl_status ssl_server_create(ssl_ctx* ctx, size_t hbm_budget_bytes, int max_batch,
                             ssl_server** out) {
  ssl::Range nvtx("ssl_server_create");
  if (!ctx || !out || max_batch < 1 || hbm_budget_bytes == 0) return SSL_E_INVALID_ARG;
  *out = nullptr;
  ssl_server* s = new (std::nothrow) ssl_server();
  if (!s) return SSL_E_OOM;
  s->ctx = ctx;
  s->device = ssl::ctx_device(ctx);
  s->budget = hbm_budget_bytes;
  s->max_batch = max_batch;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(s->device);
  bool ok = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) == cudaSuccess &&
            cudaStreamCreateWithFlags(&s->copy_stream, cudaStreamNonBlocking) == cudaSuccess;
  for (int i = 0; ok && i < kInFlight; ++i)
    ok = cudaEventCreateWithFlags(&s->batch[i].done, cudaEventDisableTiming) == cudaSuccess;
  cudaSetDevice(prev);
  if (!ok) {
    cudaGetLastError();
    delete s;
    return SSL_E_CUDA;
  }
  *out = s;
  return SSL_OK;
}

ssl_status ssl_server_destroy(ssl_server* s) {
  if (!s) return SSL_OK;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(s->device);
  cudaStreamSynchronize(s->copy_stream);
  cudaStreamSynchronize(s->stream);
  for (ssl_session* se : s->sessions) {
    cudaFree(se->kinv);
    cudaFree(se->slots);
    delete se;
  }
  for (auto& it : s->pending) cudaEventDestroy(it.copied);
  for (int i = 0; i < kInFlight; ++i) {
    for (auto& it : s->batch[i].items) cudaEventDestroy(it.copied);
    if (s->batch[i].mem.dev) cudaFree(s->batch[i].mem.dev);
    if (s->batch[i].mem.host) cudaFreeHost(s->batch[i].mem.host);
    cudaEventDestroy(s->batch[i].done);
  }
  for (cudaEvent_t e : s->free_events) cudaEventDestroy(e);
  cudaStreamDestroy(s->stream);
  cudaStreamDestroy(s->copy_stream);
  cudaSetDevice(prev);
  delete s;
  return SSL_OK;
}

}  // extern "C"

namespace {

// Validation, steering build, admission and device memory of a new session
// (K^{-1} not yet filled); on success *out is ready for session_commit.
ssl_status session_prepare(ssl_server* srv, const ssl_array_desc* desc, const ssl_steering* st,
                           ssl_session** out) {
  *out = nullptr;
  const ssl_config& c = desc->cfg;
  const int D = n_dirs(c);
  const int32_t *lp = nullptr, *li = nullptr;
  if (desc->queue_depth < 1 || c.M < 2 || c.M > SSL_MAX_M || c.T < 1 || c.B < 1 || c.Ns < 1 ||
      c.Ns >= c.M || c.Ns > SSL_MAX_NS || c.n_az < 1 || c.n_el < 0 || D > SSL_MAX_D ||
      (c.n_el == 0 && !ssl::steering_lists(st, &lp, &li)) ||
      (c.form != SSL_FORM_ABS && c.form != SSL_FORM_SQ) ||
      (c.precision != SSL_PREC_FP32 && c.precision != SSL_PREC_TF32 &&
       c.precision != SSL_PREC_BF16) ||
      !ssl::steering_matches(st, c.B, D, c.M))
    return SSL_E_INVALID_ARG;
  // the Jacobi options pass the checks of the stateless calls (method, angle
  // mode, finite tolerances below 1): a NaN tolerance would otherwise reach
  // the ordering of the server's shape classes
  ssl::JacobiOpts jo;
  if (!ssl::ctx_jacobi(&c.jacobi, &jo)) return SSL_E_INVALID_ARG;
  // the split iteration gives the noise subspace, not the ABS form's vectors
  if (jo.method == SSL_SVD_SPLIT && c.form != SSL_FORM_SQ) return SSL_E_UNSUPPORTED;
  // the steering object's table and tensor-core image for this precision are
  // built now (a build synchronises the device), not in the first server
  // step that uses them
  {
    const float2* H = nullptr;
    const float* hn = nullptr;
    const CUtensorMap* tm = nullptr;
    const ssl::Geo* geo = nullptr;
    const ssl_status r = ssl::steering_tables(srv->ctx, st, c.precision, &H, &hn, &tm, &geo);
    if (r != SSL_OK) return r;
  }
  const size_t kin = (size_t)c.B * c.M * c.M * sizeof(float2);
  const size_t slot_elems = (size_t)c.T * c.B * c.M;
  const size_t foot = kin + (size_t)desc->queue_depth * slot_elems * sizeof(float2);
  if (srv->used + foot > srv->budget) {
    srv->refused_sessions++;
    return SSL_E_ADMISSION;
  }
  ssl_session* se = new (std::nothrow) ssl_session();
  if (!se) return SSL_E_OOM;
  se->srv = srv;
  se->cfg = c;
  se->qdepth = desc->queue_depth;
  se->st = st;
  se->slot_elems = slot_elems;
  se->footprint = foot;
  if (cudaMalloc(&se->kinv, kin) != cudaSuccess ||
      cudaMalloc(&se->slots, (size_t)se->qdepth * slot_elems * sizeof(float2)) != cudaSuccess) {
    cudaGetLastError();
    if (se->kinv) cudaFree(se->kinv);
    delete se;
    return SSL_E_OOM;
  }
  *out = se;
  return SSL_OK;
}

void session_discard(ssl_session* se) {
  if (se->kinv) cudaFree(se->kinv);
  if (se->slots) cudaFree(se->slots);
  delete se;
}

void session_commit(ssl_server* srv, ssl_session* se) {
  for (int i = se->qdepth - 1; i >= 0; --i) se->free_slots.push_back(i);
  srv->used += se->footprint;
  srv->sessions.push_back(se);
}

}  // namespace

extern "C" {

ssl_status ssl_session_create(ssl_server* srv, const ssl_array_desc* desc, const float* K,
                              const ssl_steering* st, ssl_session** out) {
  ssl::Range nvtx("ssl_session_create");
  if (!srv || !desc || !K || !st || !out) return SSL_E_INVALID_ARG;
  *out = nullptr;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(srv->device);
  ssl_session* se = nullptr;
  ssl_status r = session_prepare(srv, desc, st, &se);
  if (r != SSL_OK) {
    cudaSetDevice(prev);
    return r;
  }
  const ssl_config& c = desc->cfg;
  const size_t kin = (size_t)c.B * c.M * c.M * sizeof(float2);
  float2* Kd = nullptr;
  // A device K may still be in production on any stream of the caller:
  // creation is synchronous and rare, so it waits for all device work first.
  if (is_dev(K) && cudaDeviceSynchronize() != cudaSuccess) {
    cudaGetLastError();
    r = SSL_E_CUDA;
  }
  if (r == SSL_OK && !is_dev(K)) {
    if (cudaMalloc(&Kd, kin) != cudaSuccess ||
        cudaMemcpy(Kd, K, kin, cudaMemcpyHostToDevice) != cudaSuccess) {
      cudaGetLastError();
      r = SSL_E_OOM;
    }
  }
  if (r == SSL_OK) {
    const float2* Ks = Kd ? Kd : reinterpret_cast<const float2*>(K);
    int32_t* kst = nullptr;
    if (cudaMalloc(&kst, (size_t)c.B * sizeof(int32_t)) != cudaSuccess) {
      cudaGetLastError();
      r = SSL_E_OOM;
    } else {
      cudaError_t e = ssl::launch_noise_inverse(Ks, c.B, c.M, se->kinv, kst,
                                                ssl::ctx_flags(srv->ctx), srv->stream);
      std::vector<int32_t> h(c.B);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(h.data(), kst, (size_t)c.B * sizeof(int32_t),
                            cudaMemcpyDeviceToHost, srv->stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(srv->stream);
      if (e != cudaSuccess) {
        cudaGetLastError();
        r = SSL_E_CUDA;
      } else {
        for (int b = 0; b < c.B; ++b)
          if (h[b] != 0) r = h[b];
      }
      cudaFree(kst);
    }
  }
  if (Kd) cudaFree(Kd);
  if (r != SSL_OK) {
    session_discard(se);
    cudaSetDevice(prev);
    return r;
  }
  session_commit(srv, se);
  cudaSetDevice(prev);
  *out = se;
  return SSL_OK;
}

}  // extern "C"

namespace {

// Saved session state: this header, then K^{-1} (c64 [B][M][M]).
constexpr uint32_t kStateMagic = 0x53534c53u;  // "SSLS"
constexpr uint32_t kStateVersion = 2;  // 2: the Jacobi options carry split_ns
struct SessionState {
  uint32_t magic;
  uint32_t version;
  ssl_config cfg;
  int32_t queue_depth;
  int32_t reserved;
  uint64_t kinv_bytes;
};

size_t kinv_bytes(const ssl_config& c) { return (size_t)c.B * c.M * c.M * sizeof(float2); }

}  // namespace

extern "C" {

ssl_status ssl_session_state_size(const ssl_session* se, size_t* bytes) {
  if (!se || !bytes) return SSL_E_INVALID_ARG;
  *bytes = sizeof(SessionState) + kinv_bytes(se->cfg);
  return SSL_OK;
}

ssl_status ssl_session_save(const ssl_session* se, void* buf, size_t len) {
  ssl::Range nvtx("ssl_session_save");
  if (!se || !buf) return SSL_E_INVALID_ARG;
  const size_t kin = kinv_bytes(se->cfg);
  if (len < sizeof(SessionState) + kin) return SSL_E_INVALID_ARG;
  SessionState h{};
  h.magic = kStateMagic;
  h.version = kStateVersion;
  h.cfg = se->cfg;
  h.queue_depth = se->qdepth;
  h.kinv_bytes = kin;
  std::memcpy(buf, &h, sizeof(h));
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(se->srv->device);
  // K^{-1} does not change after creation (which synchronised its stream)
  const cudaError_t e = cudaMemcpy(static_cast<char*>(buf) + sizeof(h), se->kinv, kin,
                                   cudaMemcpyDeviceToHost);
  cudaSetDevice(prev);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return SSL_E_CUDA;
  }
  return SSL_OK;
}

ssl_status ssl_session_restore(ssl_server* srv, const void* buf, size_t len,
                               const ssl_steering* st, ssl_session** out) {
  ssl::Range nvtx("ssl_session_restore");
  if (!srv || !buf || !st || !out || len < sizeof(SessionState)) return SSL_E_INVALID_ARG;
  *out = nullptr;
  SessionState h;
  std::memcpy(&h, buf, sizeof(h));
  if (h.magic != kStateMagic || h.version != kStateVersion || h.cfg.B < 1 || h.cfg.M < 1 ||
      h.cfg.M > SSL_MAX_M || h.kinv_bytes != kinv_bytes(h.cfg) ||
      len != sizeof(h) + h.kinv_bytes)
    return SSL_E_INVALID_ARG;
  const float* kv = reinterpret_cast<const float*>(static_cast<const char*>(buf) + sizeof(h));
  for (size_t i = 0; i < h.kinv_bytes / sizeof(float); ++i)
    if (!std::isfinite(kv[i])) return SSL_E_INVALID_ARG;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(srv->device);
  const ssl_array_desc desc{h.cfg, h.queue_depth};
  ssl_session* se = nullptr;
  ssl_status r = session_prepare(srv, &desc, st, &se);
  if (r == SSL_OK && cudaMemcpy(se->kinv, kv, h.kinv_bytes, cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaGetLastError();
    session_discard(se);
    r = SSL_E_CUDA;
  }
  if (r == SSL_OK) {
    session_commit(srv, se);
    *out = se;
  }
  cudaSetDevice(prev);
  return r;
}

ssl_status ssl_session_destroy(ssl_session* se) {
  ssl::Range nvtx("ssl_session_destroy");
  if (!se) return SSL_OK;
  ssl_server* s = se->srv;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(s->device);
  // A session may go while its blocks are in flight (its client went away):
  // queued blocks are dropped; batches on the GPU that hold some of its blocks
  // are waited for and retired (every block in them, of any session, gets
  // its result as usual; this session's are discarded with it).
  if (se->inflight > 0) {
    std::vector<Item> keep;
    keep.reserve(s->pending.size());
    for (const Item& it : s->pending) {
      if (it.s == se) {
        s->free_events.push_back(it.copied);
        se->free_slots.push_back(it.slot);
        se->inflight--;
      } else {
        keep.push_back(it);
      }
    }
    s->pending.swap(keep);
    for (int i = 0; i < kInFlight && se->inflight > 0; ++i) {
      Batch& b = s->batch[i];
      if (!b.active) continue;
      bool mine = false;
      for (const Item& it : b.items) mine |= it.s == se;
      if (!mine) continue;
      if (cudaEventSynchronize(b.done) != cudaSuccess) {
        cudaGetLastError();
        cudaSetDevice(prev);
        return SSL_E_CUDA;
      }
      retire_batch(s, b);
    }
  }
  cudaStreamSynchronize(s->copy_stream);
  cudaFree(se->kinv);
  cudaFree(se->slots);
  s->used -= se->footprint;
  s->sessions.erase(std::remove(s->sessions.begin(), s->sessions.end(), se), s->sessions.end());
  delete se;
  cudaSetDevice(prev);
  return SSL_OK;
}

namespace {

// Queue one block; with `order`, the copy first waits for the work already
// issued to `after` (the stream that produced X).
ssl_status submit_block(ssl_session* se, const float* X, uint64_t t_arrival_ns, bool order,
                        cudaStream_t after, ssl_ticket* out) {
  if (!se || !X || !out) return SSL_E_INVALID_ARG;
  ssl_server* s = se->srv;
  if (se->free_slots.empty()) {
    s->refused_blocks++;
    return SSL_E_ADMISSION;
  }
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(s->device);
  const int slot = se->free_slots.back();
  float2* dst = se->slots + (size_t)slot * se->slot_elems;
  cudaEvent_t ev = get_event(s);
  cudaError_t e = ev ? cudaSuccess : cudaErrorMemoryAllocation;
  if (e == cudaSuccess && order) {
    // the wait takes the event's state now, so the event can go straight
    // back to the pool
    cudaEvent_t ready = get_event(s);
    e = ready ? cudaEventRecord(ready, after) : cudaErrorMemoryAllocation;
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s->copy_stream, ready, 0);
    if (ready) s->free_events.push_back(ready);
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(dst, X, se->slot_elems * sizeof(float2), cudaMemcpyDefault,
                        s->copy_stream);
  if (e == cudaSuccess) e = cudaEventRecord(ev, s->copy_stream);
  cudaSetDevice(prev);
  if (e != cudaSuccess) {
    cudaGetLastError();
    if (ev) s->free_events.push_back(ev);
    return SSL_E_CUDA;
  }
  se->free_slots.pop_back();
  const ssl_ticket t = se->next_ticket++;
  se->inflight++;
  s->pending.push_back(Item{se, slot, t, t_arrival_ns, ev});
  *out = t;
  return SSL_OK;
}

}  // namespace

ssl_status ssl_session_submit(ssl_session* se, const float* X, uint64_t t_arrival_ns,
                              ssl_ticket* out) {
  ssl::Range nvtx("ssl_session_submit");
  return submit_block(se, X, t_arrival_ns, false, nullptr, out);
}

ssl_status ssl_session_submit_after(ssl_session* se, const float* X, uint64_t t_arrival_ns,
                                    void* stream, ssl_ticket* out) {
  ssl::Range nvtx("ssl_session_submit_after");
  return submit_block(se, X, t_arrival_ns, true, static_cast<cudaStream_t>(stream), out);
}

ssl_status ssl_session_poll(ssl_session* se, ssl_ticket t, ssl_result* out) {
  if (!se || !out) return SSL_E_INVALID_ARG;
  auto it = se->results.find(t);
  if (it == se->results.end()) {
    std::memset(out, 0, sizeof(*out));
    return SSL_OK;
  }
  *out = it->second;
  se->results.erase(it);
  return SSL_OK;
}

ssl_status ssl_server_run_step(ssl_server* s, int* launched, int* retired) {
  ssl::Range nvtx("ssl_server_run_step");
  if (!s) return SSL_E_INVALID_ARG;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(s->device);
  int nret = 0, nlaunch = 0;
  for (int i = 0; i < kInFlight; ++i) {
    Batch& b = s->batch[i];
    if (!b.active) continue;
    cudaError_t q = cudaEventQuery(b.done);
    if (q == cudaSuccess) {
      nret += (int)b.items.size();
      retire_batch(s, b);
    } else if (q != cudaErrorNotReady) {
      cudaGetLastError();
      cudaSetDevice(prev);
      return SSL_E_CUDA;
    }
  }
  ssl_status r = SSL_OK;
  Batch* b = nullptr;
  for (int i = 0; i < kInFlight; ++i)
    if (!s->batch[i].active) b = &s->batch[i];
  if (b && !s->pending.empty()) {
    // take up to max_batch queued blocks, oldest first
    const size_t n = std::min(s->pending.size(), (size_t)s->max_batch);
    b->items.assign(s->pending.begin(), s->pending.begin() + n);
    s->pending.erase(s->pending.begin(), s->pending.begin() + n);
    b->idx.assign(n, nullptr);
    b->val.assign(n, nullptr);
    b->status.assign(n, nullptr);
    std::map<ClassKey, std::vector<int>> classes;
    for (size_t i = 0; i < n; ++i) {
      const ssl_session* se = b->items[i].s;
      const bool gen = ssl::steering_is_analytic(se->st) &&
                       (se->cfg.precision == SSL_PREC_TF32 || se->cfg.precision == SSL_PREC_BF16);
      classes[key_of(se->cfg, gen)].push_back((int)i);
    }
    size_t dev_bytes = 0, host_bytes = 0;
    for (auto& kv : classes) class_bytes(b->items[kv.second[0]].s->cfg, (int)kv.second.size(),
                                         dev_bytes, host_bytes);
    if (!ensure(b->mem, dev_bytes, host_bytes)) r = SSL_E_OOM;
    for (auto& it : b->items)
      if (r == SSL_OK && cudaStreamWaitEvent(s->stream, it.copied, 0) != cudaSuccess) r = SSL_E_CUDA;
    size_t doff = 0, hoff = 0;
    for (auto& kv : classes) {
      if (r != SSL_OK) break;
      r = launch_class(s, *b, kv.second, static_cast<char*>(b->mem.dev),
                       static_cast<char*>(b->mem.host), doff, hoff);
    }
    if (r == SSL_OK && cudaEventRecord(b->done, s->stream) != cudaSuccess) r = SSL_E_CUDA;
    if (r == SSL_OK) {
      b->active = true;
      b->t_launch = now_ns();
      if (s->in_flight++ == 0) s->busy_since = b->t_launch;
      s->batches++;
      nlaunch = (int)n;
    } else {
      // give the blocks back to the queue, untouched
      s->pending.insert(s->pending.begin(), b->items.begin(), b->items.end());
      b->items.clear();
      cudaGetLastError();
    }
  }
  cudaSetDevice(prev);
  if (launched) *launched = nlaunch;
  if (retired) *retired = nret;
  return r;
}

ssl_status ssl_session_wait(ssl_session* se, ssl_ticket t, uint64_t timeout_ns, ssl_result* out) {
  if (!se || !out) return SSL_E_INVALID_ARG;
  const uint64_t t0 = now_ns();
  for (;;) {
    ssl_status r = ssl_session_poll(se, t, out);
    if (r != SSL_OK || out->done) return r;
    r = ssl_server_run_step(se->srv, nullptr, nullptr);
    if (r != SSL_OK) return r;
    if (now_ns() - t0 > timeout_ns) return SSL_E_TIMEOUT;
  }
}

ssl_status ssl_server_stats(ssl_server* s, ssl_stats* out) {
  if (!s || !out) return SSL_E_INVALID_ARG;
  std::memset(out, 0, sizeof(*out));
  out->blocks_done = s->blocks_done;
  out->batches = s->batches;
  out->sessions = s->sessions.size();
  out->sessions_refused = s->refused_sessions;
  out->blocks_refused = s->refused_blocks;
  out->blocks_pending = s->pending.size();
  out->hbm_budget = s->budget;
  out->hbm_used = s->used;
  size_t work = 0;
  for (int i = 0; i < kInFlight; ++i) work += s->batch[i].mem.dev_bytes;
  out->hbm_work = work;
  out->busy_ms = s->busy_ms;
  if (s->in_flight > 0) out->busy_ms += (double)(now_ns() - s->busy_since) * 1e-6;
  if (!s->lat_ms.empty()) {
    std::vector<double> v = s->lat_ms;
    std::sort(v.begin(), v.end());
    auto q = [&](double p) { return v[std::min(v.size() - 1, (size_t)(p * (v.size() - 1) + 0.5))]; };
    out->latency_p50_ms = q(0.50);
    out->latency_p99_ms = q(0.99);
    out->latency_max_ms = v.back();
  }
  return SSL_OK;
}

ssl_status ssl_server_reset_stats(ssl_server* s) {
  if (!s) return SSL_E_INVALID_ARG;
  s->lat_ms.clear();
  s->blocks_done = s->batches = s->refused_blocks = 0;
  s->busy_ms = 0.0;
  if (s->in_flight > 0) s->busy_since = now_ns();  // the open interval restarts now
  return SSL_OK;
}

}  // extern "C"
