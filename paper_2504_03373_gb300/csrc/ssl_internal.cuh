// Internal declarations shared by the kernels and the C-ABI host code.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/ssl_gsvd_music.h"
#include <nvtx3/nvToolsExt.h>

// Index checks of the bounds-checked debug build (-DSSL_DEBUG_BOUNDS): a
// failed check raises SSL_FLAG_BOUNDS in the launch's flag word and the guarded
// access is skipped; in the release build every check is a constant `true`.
#ifdef SSL_DEBUG_BOUNDS
#define SSL_IN_BOUNDS(cond, flags) \
  ((cond) ? true : (atomicOr((flags), (unsigned)SSL_FLAG_BOUNDS), false))
#else
#define SSL_IN_BOUNDS(cond, flags) true
#endif

namespace ssl {

// A named range on the host timeline (NVTX) for the scope of an API call, so
// that a profiler attributes the launches it issues; a no-op without one.
struct Range {
  explicit Range(const char* name) { nvtxRangePushA(name); }
  ~Range() { nvtxRangePop(); }
  Range(const Range&) = delete;
  Range& operator=(const Range&) = delete;
};

// Column stride (in complex elements) of the shared-memory matrices of the
// per-bin kernels; SSL_MAX_M rounded to the warp-friendly 64.
constexpr int kLD = 64;

__host__ __device__ inline int ceil_div(int a, int b) { return (a + b - 1) / b; }

// ---- launchers (all asynchronous on `s`; return the launch error) ----

// Optional per-item pointer tables (device arrays of nblk entries) let one
// launch serve blocks of different arrays (sessions) of the same shape:
// X_items[k] -> [T][B][M], kinv_items[k] -> [B][M][M], H_items[k] -> [B][D][M],
// hn_items[k] -> [B][D], tmH_items[k] = tensor map of that array's A image.
// NULL tables mean "one shared array" (the stateless calls).

// eq. 2-3: R[k][w] = (1/T) sum_f x_f x_f^H.
cudaError_t launch_correlate(const float2* X, int nblk, int T, int B, int M, float2* R,
                             cudaStream_t s, const float2* const* X_items = nullptr);

// K^{-1} through an FP64 Cholesky factorisation, one CTA per bin; W (optional)
// receives L^{-1} (lower triangular, K = L L^H).
cudaError_t launch_noise_inverse(const float2* K, int B, int M, float2* Kinv, int32_t* status,
                                 unsigned* flags, cudaStream_t s, float2* W = nullptr);

// The tensor-core spectrum's noise-subspace operand (the real embedding of
// E_n, NP rows x KP columns per (block, bin), BF16 or TF32-rounded FP32),
// written by the decomposition kernels straight from their shared-memory E
// when img is set (instead of E followed by a packing pass).
struct ImgOut {
  void* img;  // [items][NP][KP] of esz-byte elements; nullptr: none
  int esz, Ns, KP, NP;
  void* lo;   // TF32 only: residual image x - tf32(x) for 3xTF32; nullptr: none
};

// Row n = 2i (+1) of item `item`'s image from E (e_at(m, r) = E[m][r]):
//   B[2i][k]   = Re E[k][Ns+i] (k < M),  Im E[k-M][Ns+i] (M <= k < 2M)
//   B[2i+1][k] = Im E[k][Ns+i] (k < M), -Re E[k-M][Ns+i] (M <= k < 2M)
// and zero elsewhere; 16-byte stores by `nt` threads from thread `t`.
template <class EAt>
__device__ __forceinline__ void write_noise_image(const ImgOut& io, size_t item, int M, EAt e_at,
                                                  int t, int nt) {
  const int N = M - io.Ns, V = 16 / io.esz, chunks = io.KP / V;
  uint4* base = reinterpret_cast<uint4*>(static_cast<char*>(io.img) +
                                         item * (size_t)io.NP * io.KP * io.esz);
  for (int e = t; e < io.NP * chunks; e += nt) {
    const int n = e / chunks, k0 = (e % chunks) * V, i = n >> 1;
    float x[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int k = k0 + u;
      float v = 0.f;
      if (u < V && i < N && k < 2 * M) {
        const float2 w = e_at(k < M ? k : k - M, io.Ns + i);
        v = (n & 1) == 0 ? (k < M ? w.x : w.y) : (k < M ? w.y : -w.x);
      }
      x[u] = v;
    }
    uint32_t r[4];
    if (io.esz == 2) {
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(x[2 * u], x[2 * u + 1]);
        r[u] = *reinterpret_cast<const uint32_t*>(&h);
      }
    } else {
#pragma unroll
      for (int u = 0; u < 4; ++u) asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r[u]) : "f"(x[u]));
      if (io.lo) {  // 3xTF32: the rounding residuals, themselves rounded to TF32
        uint32_t l[4];
#pragma unroll
        for (int u = 0; u < 4; ++u)
          asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(l[u]) : "f"(x[u] - __uint_as_float(r[u])));
        reinterpret_cast<uint4*>(static_cast<char*>(io.lo) +
                                 item * (size_t)io.NP * io.KP * io.esz)[e] =
            make_uint4(l[0], l[1], l[2], l[3]);
      }
    }
    base[e] = make_uint4(r[0], r[1], r[2], r[3]);
  }
}

// Jacobi controls (see ssl_jacobi_opts in the public header).
struct JacobiOpts {
  int max_sweeps;
  float rel_tol;   // <= 0: M * 2^-24
  float abs_tol;   // <= 0: no absolute criterion
  bool angles_f64;
  int method;      // SSL_SVD_JACOBI, SSL_SVD_BIDIAG or SSL_SVD_SPLIT
  int split_ns;    // SSL_SVD_SPLIT: the signal dimension Ns
};

// Per-bin status the split iteration leaves on a matrix it hands back
// (never returned to callers: the bidiagonalisation route, launched next in
// its retry mode, solves the matrix and overwrites it).
constexpr int32_t kSplitRetry = 0x53504c54;

// Whether the split iteration takes an M x M problem with Ns signal vectors
// (otherwise launch_gsvd runs the full iteration for it).
__host__ __device__ inline bool split_applies(int M, int Ns) {
  return Ns >= 1 && Ns <= 8 && 3 * Ns <= M;
}

// A = K^{-1} R and its SVD by one-sided Jacobi (eq. 4), one CTA per (block, bin).
// stats (optional, int32 [nblk][B][2]): pairs tested and rotations applied.
// V0 (optional, [nblk][B][M][M]): warm start; Kinv must then hold V0^H K^{-1}
// so that the iteration continues from A^H V0.  Kinv == nullptr (and no
// kinv_items) means K^{-1} = I: the eigendecomposition of R (SEVD).
// io (optional): also write the spectrum's noise-subspace image; E may then be
// nullptr (not written).
// abuf (optional): scratch the split iteration uses for A (launch_gsvd_split).
cudaError_t launch_gsvd(const float2* R, const float2* Kinv, int nblk, int B, int M,
                        const JacobiOpts& o, float* sigma, float2* E, int32_t* status,
                        int32_t* stats, unsigned* flags, cudaStream_t s,
                        const float2* const* kinv_items = nullptr,
                        const float2* V0 = nullptr, const ImgOut* io = nullptr,
                        float2* abuf = nullptr);
// The noise subspace of eq. 4 for the SQ spectrum by the split one-sided
// Jacobi (pivot-partner pairs only; o.split_ns = Ns), E = [E_s | basis of the
// complement of E_s], sigma = [sigma_s | norms of the other columns of A V];
// matrices that do not converge within its sweep limit are solved again by the
// full iteration on the same stream.  status is required.
// abuf (optional, [nblk][B][M][M]): scratch for A = K^{-1} R by columns, formed
// by one batched GEMM launch before the iteration (else each warp forms its
// matrix's A itself).
cudaError_t launch_gsvd_split(const float2* R, const float2* Kinv, int nblk, int B, int M,
                              const JacobiOpts& o, float* sigma, float2* E, int32_t* status,
                              int32_t* stats, unsigned* flags, cudaStream_t s,
                              const float2* const* kinv_items, const ImgOut* io,
                              float2* abuf = nullptr);
// A = K^{-1} R for every (block, bin), stored by columns: Acm[k][b][c][r] =
// A[r][c] (a batched FP32 complex GEMM; K^{-1} shared by the blocks of a bin
// unless kinv_items gives one per block).  With 0 < Ns <= 8, A Q instead: Q
// unitary with its first Ns columns spanning A^H A_top (one power step from
// the Ns columns of largest norm), the split iteration's preconditioner.
cudaError_t launch_whiten(const float2* R, const float2* Kinv, const float2* const* kinv_items,
                          int nblk, int B, int M, int Ns, float2* Acm, cudaStream_t s);
struct GsvdProblem;
// The paper's route (bidiagonalisation + implicit QR), one CTA per (bin,
// block), or per entry of probs[0..n_probs) when probs is given.  retry: only
// the (bin, block) items whose status is kSplitRetry (status required, no
// probs); the others are left as they are.
cudaError_t launch_gsvd_bidiag(const float2* R, const float2* Kinv, int nblk, int B, int M,
                               const JacobiOpts& o, float* sigma, float2* E, int32_t* status,
                               int32_t* stats, unsigned* flags, cudaStream_t s,
                               const float2* const* kinv_items = nullptr,
                               const GsvdProblem* probs = nullptr, int n_probs = 0,
                               const ImgOut* io = nullptr, bool retry = false);
// C[k][b] = op(A) op(B) for M x M complex matrices in FP32; a_item / b_item:
// the factor is [nblk][B][M][M] (else [B][M][M], shared by the blocks);
// a_h / b_h: conjugate transpose.
cudaError_t launch_cgemm(const float2* A, bool a_item, bool a_h, const float2* Bm, bool b_item,
                         bool b_h, int nblk, int B, int M, float2* C, cudaStream_t s);

// eq. 5 on the SIMT cores in FP32: P[k][w][d].
cudaError_t launch_spectrum_simt(const float2* E, int nblk, int B, int M, int Ns, const float2* H,
                                 const float* hnorm2, int D, int form, float* P, cudaStream_t s,
                                 const float2* const* H_items = nullptr,
                                 const float* const* hn_items = nullptr);

// eq. 6: Pbar[k][d] = sum_w P[k][w][d] in bin order.
cudaError_t launch_bin_sum(const float* P, int nblk, int B, int D, float* Pbar, cudaStream_t s);

// Peak search on the direction grid; `in` (device [D], nonzero inside, or
// null) restricts the reported peaks to a search range.
cudaError_t launch_peaks(const float* Pbar, int nblk, int n_az, int n_el, int Ns, int32_t* idx,
                         float* val, cudaStream_t s, const uint8_t* in = nullptr);
// Peak search over a direction set with neighbour lists (device CSR arrays
// whose indices are in [0, D)).
cudaError_t launch_peaks_nbr(const float* Pbar, int nblk, int D, const int32_t* nbr_ptr,
                             const int32_t* nbr_idx, int Ns, int32_t* idx, float* val,
                             cudaStream_t s, unsigned* flags, const uint8_t* in = nullptr);
// Each item with its own lists (nbr_ptrs == null: the n_el x n_az grid for
// all) and its own search range (ranges == null or an entry null: all
// directions); device arrays of nblk pointers.
cudaError_t launch_peaks_items(const float* Pbar, int nblk, int D, int n_az, int n_el,
                               const int32_t* const* nbr_ptrs, const int32_t* const* nbr_idxs,
                               const uint8_t* const* ranges, int Ns, int32_t* idx, float* val,
                               cudaStream_t s, unsigned* flags);

// ---- the FP64 path (eq. 2-6 in double precision), see fp64_path.cu ----
cudaError_t launch_peaks(const double* Pbar, int nblk, int n_az, int n_el, int Ns, int32_t* idx,
                         double* val, cudaStream_t s, const uint8_t* in = nullptr);
cudaError_t launch_peaks_nbr(const double* Pbar, int nblk, int D, const int32_t* nbr_ptr,
                             const int32_t* nbr_idx, int Ns, int32_t* idx, double* val,
                             cudaStream_t s, unsigned* flags, const uint8_t* in = nullptr);
// K^{-1} kept in FP64.
cudaError_t launch_noise_inverse_f64(const float2* K, int B, int M, double2* Kinv,
                                     int32_t* status, unsigned* flags, cudaStream_t s);
// eq. 2-3 with FP64 sums: R[k][w] (double) from FP32 frames X.
cudaError_t launch_correlate_f64(const float2* X, int nblk, int T, int B, int M, double2* R,
                                 cudaStream_t s);
// eq. 4 in FP64: A = K^{-1} R and its SVD by one-sided Jacobi on complex
// doubles (FP64 data, angles and tests); tol <= 0: M 2^-53.
cudaError_t launch_gsvd_f64(const double2* R, const double2* Kinv, int nblk, int B, int M,
                            int max_sweeps, double tol, double abs_tol, double* sigma, double2* E,
                            int32_t* status, int32_t* stats, unsigned* flags, cudaStream_t s);
// eq. 5 in FP64 on the SIMT cores (h from the FP32 table, widened): P[k][w][d].
cudaError_t launch_spectrum_f64(const double2* E, int nblk, int B, int M, int Ns, const float2* H,
                                int D, int form, double* P, cudaStream_t s);
// eq. 6 in FP64, fixed bin order.
cudaError_t launch_bin_sum_f64(const double* P, int nblk, int B, int D, double* Pbar,
                               cudaStream_t s);

// Analytic (free-field, far-field) steering of one array: h_m(d, w) =
// exp(+j 2 pi f_w (u_d . p_m) / c), generated where it is used instead of
// read from a table.  Plain device pointers; the struct itself lives in
// device memory so that kernels can take a pointer to it.
struct Geo {
  const float* pos;   // [M][3] microphone positions (m)
  const float* dirs;  // [D][3] direction unit vectors
  const float* fc;    // [B] f_w / c (1/m)
  int M, D, B;
};

// ---- tensor-core spectrum (tcgen05), see spectrum_tc.cu ----
int tc_kp(int M);            // padded K of the real-embedded operands (64 or 128)
int tc_np(int M, int Ns);    // padded N = 2 (M - Ns) rounded up to 16
size_t tc_smem_bytes(int M, int Ns, int precision);
// H [B][D][M] -> A image [B][D][KP] (bf16 or tf32-rounded f32).
cudaError_t launch_pack_h(const float2* H, int B, int D, int M, int precision, void* out,
                          cudaStream_t s);
// H [B][D][M] -> the A image's TF32 residuals (3xTF32's low part).
constexpr int kPrecTf32Lo = -1;
// E [nmat][M][M] -> B image [nmat][NP][KP]; out_lo (TF32 only): the image of
// the TF32 rounding residuals (3xTF32's low part).
cudaError_t launch_pack_e(const float2* E, int nmat, int M, int Ns, int precision, void* out,
                          cudaStream_t s, void* out_lo = nullptr);
// With geo (one array) or geo_items (per block, device array of device
// pointers) the A tiles are generated from the analytic steering in the
// kernel (tmH and the norms are then unused; |h|^2 = M).
cudaError_t launch_spectrum_tc(const CUtensorMap& tmH, const CUtensorMap& tmE, int nblk, int B,
                               int D, int M, int Ns, int precision, int form,
                               const float* hnorm2, float* P, unsigned* flags, cudaStream_t s,
                               const CUtensorMap* tmH_items = nullptr,
                               const float* const* hn_items = nullptr, uint64_t wait_ns = 0,
                               const Geo* geo = nullptr, const Geo* const* geo_items = nullptr,
                               int stall = 0);
// The c64 table H [B][D][M] of an analytic steering (phases in FP64).
cudaError_t launch_steering_table(const Geo* geo, int B, int D, int M, float2* H, cudaStream_t s);

// 3xTF32 (FP32-class) spectrum: hi/lo images of both operands, one (block,
// bin) per item.
cudaError_t launch_spectrum_tc3(const CUtensorMap& tmH, const CUtensorMap& tmHlo,
                                const CUtensorMap& tmE, const CUtensorMap& tmElo, int nblk, int B,
                                int D, int M, int Ns, int form, const float* hnorm2, float* P,
                                unsigned* flags, cudaStream_t s, uint64_t wait_ns = 0,
                                int stall = 0);

// ---- mixed batches: arrays of different sizes in one launch per stage ----

// One array of a mixed batch (device-resident table entry).  The tensor maps
// come first so that the 64-byte alignment of CUtensorMap holds.
struct alignas(128) MixedItem {
  CUtensorMap tmH;      // steering image of the array (tensor-core spectrum)
  CUtensorMap tmE;      // E_n image [B][NP][KP] (tensor-core spectrum)
  const float2* X;      // [T][B][M]
  const float2* Kinv;   // [B][M][M]
  const float2* H;      // [B][D][M]
  const float* hn;      // [B][D]
  float2* R;            // [B][M][M]
  float2* E;            // [B][M][M] (FP32 spectrum only; null with the tensor-core spectrum)
  float* sig;           // [B][M]
  int32_t* bst;         // [B] per-bin status
  void* eimg;           // [B][NP][KP]
  float* P;             // [B][D]
  float* Pbar;          // [D]
  int32_t* idx;         // [Ns]
  float* val;           // [Ns]
  int32_t* status;      // [1] or null
  const int32_t* nbr_ptr;  // neighbour lists of a direction set (n_el == 0), else null
  const int32_t* nbr_idx;
  const uint8_t* range;    // search range [D] (nonzero inside), or null: all directions
  int M, T, B, Ns, n_az, n_el, D, KP, NP;
};

// The generalised SVD of one (array, bin) in the mixed kernel.
struct GsvdProblem {
  const float2* R;      // [M][M]
  const float2* Kinv;   // [M][M]
  float* sig;           // [M]
  float2* E;            // [M][M], or null when img is written instead
  int32_t* status;      // [1]
  int M;
  int salt;
  // the spectrum's operand image of this problem's E_n ([NP][KP] of esz-byte
  // elements, see ImgOut), or null
  void* img;
  int esz, Ns, KP, NP;
};

// One work unit of the mixed Jacobi kernel (a 128-thread CTA): one matrix
// of the 64 class, two of the 32 class or four of the 16 class.
struct GsvdUnit {
  int mp, n;
  int prob[4];
};

// Persistent launch over `units` (grid CTAs take units from *counter, which
// the launcher zeroes first).
cudaError_t launch_gsvd_mixed(const GsvdUnit* units, int n_units, const GsvdProblem* probs,
                              int* counter, int grid, const JacobiOpts& o, unsigned* flags,
                              cudaStream_t s);
// Largest grid worth launching: resident CTAs per SM of the mixed kernel.
int gsvd_mixed_ctas_per_sm();

// One CTA per (item, bin) of ctab = {item, bin}.
cudaError_t launch_correlate_mixed(const MixedItem* items, const int2* ctab, int n_ctab,
                                   cudaStream_t s);
cudaError_t launch_spectrum_tc_mixed(const MixedItem* items, const int2* ctab, int n_ctab,
                                     int precision, int form, unsigned* flags, cudaStream_t s,
                                     uint64_t wait_ns = 0);
cudaError_t launch_spectrum_simt_mixed(const MixedItem* items, const int2* ctab, int n_ctab,
                                       int d_max, int form, cudaStream_t s);
// Per item: Pbar (eq. 6), peaks, and the item status (largest bin status).
cudaError_t launch_bin_sum_mixed(const MixedItem* items, int n, int d_max, cudaStream_t s);
cudaError_t launch_peaks_mixed(const MixedItem* items, int n, int d_max, cudaStream_t s);

// Per-block status = the largest per-bin status of the block.
cudaError_t launch_status_max(const int32_t* bin_status, int nblk, int B, int32_t* out,
                              cudaStream_t s);

// ---- host-side helpers shared by the C-ABI translation units ----
unsigned* ctx_flags(ssl_ctx* ctx);
// Limit of each bounded device wait of the context's tensor-core kernels (ns;
// 0 = the kernels' default), see ssl_set_wait_limit.
uint64_t ctx_wait_ns(const ssl_ctx* ctx);
// Test hook of ssl_set_test_stall: nonzero makes the context's tensor-core
// spectrum launches withhold their operand loads.
int ctx_test_stall(const ssl_ctx* ctx);
// Stores msg as the context's last error and returns st.
ssl_status ctx_error(ssl_ctx* ctx, ssl_status st, const char* msg);
// Validated Jacobi controls with the library defaults filled in.
bool ctx_jacobi(const ssl_jacobi_opts* o, JacobiOpts* out);
int ctx_device(const ssl_ctx* ctx);
bool steering_matches(const ssl_steering* st, int B, int D, int M);
bool steering_is_analytic(const ssl_steering* st);
// The neighbour lists attached to st (device CSR), or false if it has none.
bool steering_lists(const ssl_steering* st, const int32_t** ptr, const int32_t** idx);
// The search range attached to st (device [D], nonzero inside), or null.
const uint8_t* steering_range(const ssl_steering* st);
// Device table, norms and (for TF32/BF16, built on first use) the tensor map
// of the tensor-core A image of a steering object; with `geo`, an analytic
// object used at TF32/BF16 returns its geometry instead (the kernels generate
// the tiles) and nothing else.
ssl_status steering_tables(ssl_ctx* ctx, const ssl_steering* st, int precision, const float2** H,
                           const float** hnorm2, const CUtensorMap** tm,
                           const Geo** geo = nullptr);
// 3-D tiled tensor map over a row-major [d2][d1][d0] array, 128-byte swizzle.
bool encode_tmap_3d(CUtensorMap* tm, void* base, int esz, uint64_t d0, uint64_t d1, uint64_t d2,
                    uint32_t b0, uint32_t b1);

// |h|^2 per (bin, direction) of a c64 table.
cudaError_t launch_hnorm2(const float2* H, int B, int D, int M, float* out, cudaStream_t s);

}  // namespace ssl
