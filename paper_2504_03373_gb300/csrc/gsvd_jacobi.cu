// Whitening and generalised SVD, eq. 4 (Sec. III-A/B):
//   A = K^{-1} R = E Lambda E_r^H,   E = left singular vectors (columns).
//
// One CTA of MP / 16 warps per (bin, block); the matrix is padded to MP x MP
// with MP = 16, 32 or 64 (the description below is for MP = 64).  The 64-size
// class keeps shared memory near 52 KB and registers at 128 so that four
// CTAs share an SM.
//
//  1. G = A^H = (K^{-1} R)^H in FP32: each warp forms its own 16 columns of G
//     in registers from R (staged in shared memory) and K^{-1} (read from
//     global memory, passed between lanes by shuffles).
//  2. One-sided (Hestenes) Jacobi on G: pairs of columns (p, q) are rotated
//     by a unitary 2x2 J until all columns are mutually orthogonal; the
//     product V of the rotations gives G V = U Sigma, i.e. A = V Sigma U^H, so
//     E = V and the singular values are the column norms of G V.
//  3. G stays in registers: each warp owns 16 columns (two blocks of 8; lane
//     l holds rows l and l + 32).  V lives in shared memory at a fixed place
//     per column and is touched only when a pair is actually rotated; a
//     per-slot column index travels with G.  A sweep is a block-level
//     round-robin over the 8 blocks: in the first block round every warp
//     visits all 120 pairs among its own 16 columns (circle method, columns
//     shifted between register slots), in the 6 following ones the 64 pairs
//     across its two blocks (slot k against slot 8 + k while the bottom block
//     rotates through its slots; register indices stay static and the round
//     body exists once, which keeps the code inside the instruction cache),
//     after which blocks move to the next warp through shared memory.  63 inner rounds of 32 disjoint
//     pairs visit each of the 2016 pairs once.
//  4. Per inner round a warp forms gamma = g_p^H g_q for its 8 pairs in FP32
//     (a transposing butterfly reduces 16 values over 32 lanes in 16
//     shuffles); the squared column norms are carried along
//     (alpha' = alpha - t|gamma|, beta' = beta + t|gamma|) and recomputed
//     exactly at every block round.
//  5. Convergence (the Jacobi counterpart of Sec. III-B's tolerance): a pair
//     is rotated only if |gamma| > tol * sqrt(alpha * beta), tol = M 2^-24
//     (relative test) and |gamma| > abs_tol * max_c |g_c|^2 (the paper's
//     tolerance taken from the global maximum; abs_tol = 0 disables it),
//     the latter only for pairs of small columns (larger squared norm at most
//     sqrt(abs_tol) max_c |g_c|^2), so that it cannot leave a large column
//     unrotated against a small one.  The
//     iteration stops once a full sweep's worth of consecutive rounds (63)
//     has rotated nothing, wherever that window starts.
//  6. Angles.  FP64 (default): the CTA's 32 pairs are gathered so that one
//     warp (a different one each round) computes them one pair per lane,
//     because on this part an FP64 warp instruction costs the same with one
//     active lane as with 32; the decision and the rotation are evaluated in
//     FP64 (FP32 estimates refined by one Newton-Raphson step each, 14 FP64
//     operations per pair, results rounded to FP32 to nearest).
//     Before that, every warp screens its own 8 pairs in FP32 (a slightly
//     wider band than the FP64 warp's), and the first of the round's two
//     barriers reduces the screens: a round in which no pair may rotate
//     skips the FP64 warp, the second barrier and the updates.
//     FP32: each warp computes its own 8 pairs and the warps run without
//     block barriers between exchanges.
//  7. Singular values = column norms, sorted descending (Alg. 1's sort step);
//     E's columns (V's, renormalised) are permuted accordingly.
#include <float.h>

#include "jacobi_rot.cuh"
#include "ssl_internal.cuh"

namespace ssl {
namespace {

constexpr int kCols = 16;  // columns per warp (two blocks of 8)
constexpr int kBlk = 8;
using namespace jrot;

// Size class of the padded matrix (MP = 16, 32 or 64 rows and columns):
// MP / 16 warps of 16 columns each, MP / 32 rows per lane (one row on the
// first 16 lanes for MP = 16), 2 W block positions in the round-robin.
template <int MP>
struct Shape {
  static constexpr int W = MP / 16;
  static constexpr int RPL = MP >= 64 ? 2 : 1;
  static constexpr int NPOS = 2 * W;
  static constexpr int THREADS = 32 * W;
  // V is stored column by column with a stride of MP + 1 complex values, so
  // that reading one row across columns is free of bank conflicts.
  static constexpr int VLD = MP + 1;
};

// Barriers of the group of warps that solves one matrix: the whole CTA
// (per-bin kernel, and the 64 class of the mixed kernel), a named barrier
// over two warps (32 class of the mixed kernel) or the warp itself.
// any(p): the same barrier, returning whether p held in any thread.
struct CtaSync {
  __device__ __forceinline__ void operator()() const { __syncthreads(); }
  __device__ __forceinline__ bool any(bool p) const { return __syncthreads_or(p) != 0; }
};
struct BarSync {
  int id, n;
  __device__ __forceinline__ void operator()() const {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
  }
  __device__ __forceinline__ bool any(bool p) const {
    unsigned r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\t"
        "bar.red.or.pred q, %2, %3, p;\n\tselp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"((unsigned)p), "r"(id), "r"(n)
        : "memory");
    return r != 0;
  }
};
struct WarpSync {
  __device__ __forceinline__ void operator()() const { __syncwarp(); }
  __device__ __forceinline__ bool any(bool p) const {
    __syncwarp();
    return __any_sync(0xffffffffu, p);
  }
};

template <int MP>
struct SmemJ {
  static constexpr int W = Shape<MP>::W;
  float gram[W * 16];    // [warp][pair][re, im]
  float4 rot[W * 8];     // [warp][pair]
  float nrm[W * kCols];  // squared norms per (warp, slot)
  int colid[W * kCols];  // logical column per (warp, slot)
  float red[W];
  float sig[MP];
  int rnk[MP];
  int inv[MP];     // rank -> logical column
  float vinv[MP];  // 1 / |V column|
  int rot_count[3];
  int visits;
  int bad;
};

// Rotate V's columns p, q (logical ids) in shared memory.
template <int MP>
__device__ __forceinline__ void rot_v(float2* Vs, int p, int q, int lane, float c, float sr,
                                      float si) {
#pragma unroll
  for (int h = 0; h < Shape<MP>::RPL; ++h) {
    const int row = lane + 32 * h;
    if (row < MP) {
      float2 a = Vs[p * Shape<MP>::VLD + row], d = Vs[q * Shape<MP>::VLD + row];
      rot1(a, d, c, sr, si);
      Vs[p * Shape<MP>::VLD + row] = a;
      Vs[q * Shape<MP>::VLD + row] = d;
    }
  }
}

// Slot of pair k's second column: intra rounds (KIND 0) pair slot k with
// slot 15 - k, cross rounds (KIND 1) with slot 8 + k.
template <int KIND>
__host__ __device__ constexpr int partner(int k) {
  return KIND == 0 ? 15 - k : kBlk + k;
}

// One inner round over the warp's 8 pairs (k, partner<KIND>(k)).  With FP64
// angles, warp fw computes all of the CTA's pairs; fw changes from round to
// round so that the FP64 work of the CTAs sharing an SM spreads over its
// sub-partitions.
template <bool kF64, int MP, int KIND, class Sync>
__device__ __forceinline__ void inner_round(const Sync& sync, float2 (&g)[kCols][Shape<MP>::RPL],
                                            SmemJ<MP>& S, float2* Vs, int warp, int lane,
                                            float tol, float2 abs_thr, int& wrot, int fw,
                                            unsigned* flags) {
  constexpr int RPL = Shape<MP>::RPL;
  float x[16];
#pragma unroll
  for (int k = 0; k < 8; ++k) dot_partial<RPL>(g[k], g[partner<KIND>(k)], x[2 * k], x[2 * k + 1]);
  const float v = transpose_reduce16(x, lane);
  if ((lane & 1) == 0) S.gram[warp * 16 + (lane >> 1)] = v;
  if (kF64) {
    // every warp screens its own pairs in FP32; the first barrier also
    // tells whether any pair of the CTA may rotate, and a round in which
    // none may skips the FP64 warp, the second barrier and the updates
    __syncwarp();
    bool may = false;
    if (lane < 8) {
      const float2 gm = reinterpret_cast<const float2*>(S.gram)[warp * 8 + lane];
      may = may_rotate(S.nrm[warp * kCols + lane], S.nrm[warp * kCols + partner<KIND>(lane)],
                       gm.x, gm.y, tol, abs_thr);
    }
    if (!sync.any(may)) return;
    if (warp == fw) {
      const int w = lane >> 3, k = lane & 7;
      bool did = false;
      if (w < Shape<MP>::W) {
        const int sp = w * kCols + k, sq = w * kCols + partner<KIND>(k);
        const float2 gm = reinterpret_cast<const float2*>(S.gram)[w * 8 + k];
        float4 o = make_float4(1.f, 0.f, 0.f, 0.f);
        float na = 0.f, nb = 0.f;
        did = rotation<true>(S.nrm[sp], S.nrm[sq], gm.x, gm.y, tol, abs_thr, o, na, nb);
        S.rot[lane] = o;
        if (did) {
          S.nrm[sp] = na;
          S.nrm[sq] = nb;
        }
      }
      wrot += __popc(__ballot_sync(kFull, did));
    }
    sync();
  } else {
    __syncwarp();
    bool did = false;
    if (lane < 8) {
      const int sp = warp * kCols + lane, sq = warp * kCols + partner<KIND>(lane);
      const float2 gm = reinterpret_cast<const float2*>(S.gram)[warp * 8 + lane];
      float4 o = make_float4(1.f, 0.f, 0.f, 0.f);
      float na = 0.f, nb = 0.f;
      did = rotation<false>(S.nrm[sp], S.nrm[sq], gm.x, gm.y, tol, abs_thr, o, na, nb);
      S.rot[warp * 8 + lane] = o;
      if (did) {
        S.nrm[sp] = na;
        S.nrm[sq] = nb;
      }
    }
    wrot += __popc(__ballot_sync(kFull, did));
    __syncwarp();
  }
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const float4 cs = S.rot[warp * 8 + k];
    if (cs.w != 0.f) {
#pragma unroll
      for (int h = 0; h < RPL; ++h) rot1(g[k][h], g[partner<KIND>(k)][h], cs.x, cs.y, cs.z);
      const int vp = S.colid[warp * kCols + k], vq = S.colid[warp * kCols + partner<KIND>(k)];
      if (SSL_IN_BOUNDS(vp >= 0 && vp < MP && vq >= 0 && vq < MP, flags))
        rot_v<MP>(Vs, vp, vq, lane, cs.x, cs.y, cs.z);
    }
  }
}

// Move slot columns: slot i takes slot nxt(i)'s column for i in [lo, 16) and
// slot 15 takes slot `wrap`'s (circle over the 16 slots with lo = 1, wrap = 1;
// bottom block rotation with lo = 8, wrap = 8).  Ids and norms move along.
template <int MP>
__device__ __forceinline__ void shift_slots(float2 (&g)[kCols][Shape<MP>::RPL], SmemJ<MP>& S,
                                            int warp, int lane, int lo) {
  constexpr int RPL = Shape<MP>::RPL;
  float2 t[RPL];
#pragma unroll
  for (int h = 0; h < RPL; ++h) t[h] = g[lo][h];
  if (lo == 1) {
#pragma unroll
    for (int i = 1; i < 15; ++i)
#pragma unroll
      for (int h = 0; h < RPL; ++h) g[i][h] = g[i + 1][h];
  } else {
#pragma unroll
    for (int i = kBlk; i < 15; ++i)
#pragma unroll
      for (int h = 0; h < RPL; ++h) g[i][h] = g[i + 1][h];
  }
#pragma unroll
  for (int h = 0; h < RPL; ++h) g[15][h] = t[h];
  int id = 0;
  float nr = 0.f;
  if (lane >= lo && lane < 16) {
    const int src = warp * kCols + (lane == 15 ? lo : lane + 1);
    id = S.colid[src];
    nr = S.nrm[src];
  }
  __syncwarp();
  if (lane >= lo && lane < 16) {
    S.colid[warp * kCols + lane] = id;
    S.nrm[warp * kCols + lane] = nr;
  }
  __syncwarp();
}

// Exact squared norms of the warp's 16 columns into S.nrm.
template <int MP>
__device__ __forceinline__ void refresh_norms(const float2 (&g)[kCols][Shape<MP>::RPL],
                                              SmemJ<MP>& S, int warp, int lane) {
  float x[16];
#pragma unroll
  for (int c = 0; c < kCols; ++c) x[c] = norm2<Shape<MP>::RPL>(g[c]);
  const float v = transpose_reduce16(x, lane);
  if ((lane & 1) == 0) S.nrm[warp * kCols + (lane >> 1)] = v;
  __syncwarp();
}

// Block exchange between block rounds: circle method over 2W block positions,
// warp s holding positions s (top) and 2W - 1 - s (bottom), position 0 fixed.
// A position's block moves one position down; position 1's wraps to 2W - 1.
template <int MP>
__device__ __forceinline__ void store_block(const float2 (&g)[kCols][Shape<MP>::RPL],
                                            const SmemJ<MP>& S, int half, float2* xg, int* xid,
                                            int slot, int warp, int lane) {
#pragma unroll
  for (int c = 0; c < kBlk; ++c)
#pragma unroll
    for (int h = 0; h < Shape<MP>::RPL; ++h)
      if (lane + 32 * h < MP) xg[(slot * kBlk + c) * MP + lane + 32 * h] = g[half * kBlk + c][h];
  if (lane < kBlk) xid[slot * kBlk + lane] = S.colid[warp * kCols + half * kBlk + lane];
}
template <int MP>
__device__ __forceinline__ void load_block(float2 (&g)[kCols][Shape<MP>::RPL], SmemJ<MP>& S,
                                           int half, const float2* xg, const int* xid, int slot,
                                           int warp, int lane) {
#pragma unroll
  for (int c = 0; c < kBlk; ++c)
#pragma unroll
    for (int h = 0; h < Shape<MP>::RPL; ++h)
      if (lane + 32 * h < MP) g[half * kBlk + c][h] = xg[(slot * kBlk + c) * MP + lane + 32 * h];
  if (lane < kBlk) S.colid[warp * kCols + half * kBlk + lane] = xid[slot * kBlk + lane];
}

// The exchange goes through W slots of 8 columns in four steps: tops out
// (warp s -> slot s - 1), tops in, bottoms out (warp s -> slot s + 1),
// bottoms in.  Warp 0's new bottom is warp 1's old top (slot 0, still intact
// after the third step) and the last warp's bottom becomes its own top.
template <int MP, class Sync>
__device__ __forceinline__ void exchange(const Sync& sync, float2 (&g)[kCols][Shape<MP>::RPL],
                                         SmemJ<MP>& S, float2* xg, int* xid, int warp, int lane) {
  constexpr int W = Shape<MP>::W;
  constexpr int RPL = Shape<MP>::RPL;
  if (warp >= 1) store_block<MP>(g, S, 0, xg, xid, warp - 1, warp, lane);
  sync();
  if (warp == W - 1) {
    int id = 0;
    if (lane < kBlk) id = S.colid[warp * kCols + kBlk + lane];
#pragma unroll
    for (int c = 0; c < kBlk; ++c)
#pragma unroll
      for (int h = 0; h < RPL; ++h) g[c][h] = g[kBlk + c][h];
    __syncwarp();
    if (lane < kBlk) S.colid[warp * kCols + lane] = id;
  } else if (warp >= 1) {
    load_block<MP>(g, S, 0, xg, xid, warp, warp, lane);
  }
  sync();
  if (warp <= W - 2) store_block<MP>(g, S, 1, xg, xid, warp + 1, warp, lane);
  sync();
  load_block<MP>(g, S, 1, xg, xid, warp, warp, lane);
  sync();
}

// Whitening and Jacobi SVD of one matrix by one group of MP / 16 warps: tid is
// the thread's index within the group, Vs / xg / xid / S the group's shared
// memory, `salt` varies the angle warp's rotation between matrices.  Outputs:
// sigma [M] (descending), E [M][M] (columns = left singular vectors), the
// status word and optionally the statistics {pairs tested, rotations}.
template <bool kF64, int MP, class Sync>
__device__ __forceinline__ void gsvd_solve(const Sync& sync, int tid, const float2* __restrict__ Rb,
                                           const float2* __restrict__ Kb, int M, int max_sweeps,
                                           float tol, float abs_tol, float* __restrict__ sig_out,
                                           float2* __restrict__ E_out, int32_t* status_out,
                                           int32_t* stats_out, unsigned* flags, int salt,
                                           float2* Vs, float2* xg, int* xid, SmemJ<MP>& S,
                                           const float2* __restrict__ V0 = nullptr,
                                           const ImgOut io = ImgOut{nullptr, 0, 0, 0, 0},
                                           size_t item = 0) {
  using Sh = Shape<MP>;
  constexpr int W = Sh::W, RPL = Sh::RPL, NT = Sh::THREADS;
  const int warp = tid / 32, lane = tid % 32;
  const int b = salt;

  if (tid == 0) {
    S.bad = 0;
    S.rot_count[0] = S.rot_count[1] = S.rot_count[2] = 0;
    S.visits = 0;
  }
  // ---- G = A^H, A = K^{-1} R; each warp forms its own 16 columns (top block
  // = position warp, bottom = 2W-1-warp):
  //   G[j][i] = conj(A[i][j]) = sum_m conj(Kinv[i][m]) conj(R[m][j]).
  // R is staged in V's space; K^{-1} is read from global memory.
  float2 g[kCols][RPL];
  {
    float2* Rs = Vs;
    for (int e = tid; e < M * M; e += NT) Rs[e] = Rb[e];
#pragma unroll
    for (int half = 0; half < 2; ++half) {
      const int blk = half == 0 ? warp : Sh::NPOS - 1 - warp;
      if (lane < kBlk) S.colid[warp * kCols + half * kBlk + lane] = blk * kBlk + lane;
    }
#pragma unroll
    for (int c = 0; c < kCols; ++c)
#pragma unroll
      for (int h = 0; h < RPL; ++h) g[c][h] = make_float2(0.f, 0.f);
    // lane l fetches K^{-1}[col(l % 16)][m0 + l / 16]; the values reach the
    // other lanes by shuffles
    const int lc = lane & 15;
    const int lcol = (lc < kBlk ? warp : Sh::NPOS - 1 - warp) * kBlk + (lc & 7);
    const float2* kp = Kb ? Kb + (size_t)lcol * M + (lane >> 4) : nullptr;
    sync();
#pragma unroll 1
    for (int m0 = 0; m0 < M; m0 += 2) {
      const bool in = lcol < M && m0 + (lane >> 4) < M;
      // Kb == nullptr: K^{-1} = I (the eigendecomposition of R)
      const float2 kl = !in ? make_float2(0.f, 0.f)
                            : Kb ? __ldg(kp + m0)
                                 : make_float2(lcol == m0 + (lane >> 4) ? 1.f : 0.f, 0.f);
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int m = min(m0 + u, M - 1);  // a repeated row meets zero K^{-1} values
        float2 rv[RPL];
#pragma unroll
        for (int h = 0; h < RPL; ++h) {
          const int j = lane + 32 * h;
          rv[h] = j < M ? Rs[m * M + j] : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int c = 0; c < kCols; ++c) {
          const float kx = __shfl_sync(kFull, kl.x, c + 16 * u);
          const float ky = __shfl_sync(kFull, kl.y, c + 16 * u);
#pragma unroll
          for (int h = 0; h < RPL; ++h) {
            g[c][h].x = fmaf(kx, rv[h].x, fmaf(-ky, rv[h].y, g[c][h].x));
            g[c][h].y = fmaf(-kx, rv[h].y, fmaf(-ky, rv[h].x, g[c][h].y));
          }
        }
      }
    }
    bool finite = true;
#pragma unroll
    for (int c = 0; c < kCols; ++c)
#pragma unroll
      for (int h = 0; h < RPL; ++h) finite &= isfinite(g[c][h].x) && isfinite(g[c][h].y);
    if (!finite) atomicExch(&S.bad, 1);
    sync();
    // V = I, or the warm start V0 (the caller then passes E0^H K^{-1} for
    // K^{-1}, so that G = A^H V0 and the rotations continue from V0)
    for (int e = tid; e < MP * Sh::VLD; e += NT) {
      const int c = e / Sh::VLD, r = e % Sh::VLD;
      float2 v = make_float2(c == r ? 1.f : 0.f, 0.f);
      if (V0 && c < M) v = r < M ? V0[(size_t)r * M + c] : make_float2(0.f, 0.f);
      Vs[e] = v;
    }
    sync();
  }

  // Convergence: the schedule repeats every sweep of MP - 1 rounds, so once
  // MP - 1 consecutive rounds have rotated nothing, every pair has passed its
  // test (against the threshold of the sweep it ran in) with G as it now is,
  // whether or not that window started at a sweep boundary.  Rotations are
  // counted per block round in a triple-buffered counter that is read after
  // the barriers of the next block exchange.
  int rotations = 0, wrot = 0, wvis = 0, quiet = 0, t = 0, nr_prev = 0;
  bool converged = S.bad != 0;
  float2 abs_thr = make_float2(0.f, 0.f);  // absolute level and its gate, per sweep
  for (int sw = 0; sw < max_sweeps && !converged; ++sw) {
#pragma unroll 1
    for (int br = 0; br < Sh::NPOS - 1; ++br) {
      if (W > 1 && (br > 0 || sw > 0))
        exchange<MP>(sync, g, S, xg, xid, warp, lane);
      else
        sync();
      if (t > 0) {  // verdict on the block round before the exchange
        const int rc = S.rot_count[(t - 1) % 3];
        if (tid == 0) S.rot_count[(t + 1) % 3] = 0;
        rotations += rc;
        quiet = rc != 0 ? 0 : quiet + nr_prev;
        if (quiet >= MP - 1) {
          converged = true;
          break;
        }
      }
      refresh_norms<MP>(g, S, warp, lane);
      {  // pairs of real (unpadded) columns this block round tests in this warp
        const unsigned real =
            __ballot_sync(kFull, lane < kCols && S.colid[warp * kCols + (lane & 15)] < M);
        const int nt = __popc(real & 0xffu), nb = __popc(real & 0xff00u);
        wvis += br == 0 ? (nt + nb) * (nt + nb - 1) / 2 : nt * nb;
      }
      if (br == 0) {
        if (abs_tol > 0.f) {
          float mx = lane < kCols ? S.nrm[warp * kCols + lane] : 0.f;
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(kFull, mx, o));
          if (lane == 0) S.red[warp] = mx;
          sync();
          float amax = 0.f;
#pragma unroll
          for (int w = 0; w < W; ++w) amax = fmaxf(amax, S.red[w]);
          abs_thr = make_float2(abs_tol * amax, sqrtf(abs_tol) * amax);
        }
        sync();
        // all pairs among the warp's 16 columns
#pragma unroll 1
        for (int r = 0; r < 15; ++r) {
          inner_round<kF64, MP, 0>(sync, g, S, Vs, warp, lane, tol, abs_thr, wrot,
                                   (r + b) & (W - 1), flags);
          shift_slots<MP>(g, S, warp, lane, 1);
        }
        nr_prev = 15;
      } else {
        if (kF64) sync();
        // pairs across the warp's two blocks
#pragma unroll 1
        for (int j = 0; j < kBlk; ++j) {
          inner_round<kF64, MP, 1>(sync, g, S, Vs, warp, lane, tol, abs_thr, wrot,
                                   (j + br + b) & (W - 1), flags);
          shift_slots<MP>(g, S, warp, lane, kBlk);
        }
        nr_prev = kBlk;
      }
      if (lane == 0 && wrot != 0) atomicAdd(&S.rot_count[t % 3], wrot);
      wrot = 0;
      ++t;
    }
  }
  if (lane == 0 && wvis != 0) atomicAdd(&S.visits, wvis);
  sync();
  if (!converged && t > 0) {  // the sweep limit ended the loop: last verdict
    const int rc = S.rot_count[(t - 1) % 3];
    rotations += rc;
    converged = rc == 0 && quiet + nr_prev >= MP - 1;
  }

  // ---- singular values: column norms of G, by logical column ----
  {
    float x[16];
#pragma unroll
    for (int c = 0; c < kCols; ++c) x[c] = norm2<RPL>(g[c]);
    const float v = transpose_reduce16(x, lane);
    if ((lane & 1) == 0) {
      const int id = S.colid[warp * kCols + (lane >> 1)];
      S.sig[id] = id < M ? sqrtf(v) : -1.f;
    }
  }
  sync();
  if (tid < MP) {
    // ranks by value, ties by column; a NaN (non-finite input) ranks after
    // the real columns and before the padding, so the ranks stay a
    // permutation and every index derived from them stays in range
    const float v0 = S.sig[tid], v = v0 == v0 ? v0 : -0.5f;
    int rk = 0;
    for (int c = 0; c < MP; ++c) {
      const float w0 = S.sig[c], w = w0 == w0 ? w0 : -0.5f;
      rk += (w > v) || (w == v && c < tid);
    }
    S.rnk[tid] = rk;
  }
  sync();
  // 1 / |V column| per logical column, and rank -> column
  for (int c = warp; c < MP; c += W) {
    float n2 = 0.f;
#pragma unroll
    for (int h = 0; h < RPL; ++h) {
      const int row = lane + 32 * h;
      if (row < MP) {
        const float2 v = Vs[c * Shape<MP>::VLD + row];
        n2 = fmaf(v.x, v.x, fmaf(v.y, v.y, n2));
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) n2 += __shfl_xor_sync(kFull, n2, o);
    if (lane == 0) S.vinv[c] = n2 > 0.f ? __frsqrt_rn(n2) : 1.f;
  }
  if (tid < MP) S.inv[S.rnk[tid]] = tid;
  sync();
  // E[row][rk] = V[row][c] / |V[:, c]| with c the column of rank rk: rows of E
  // leave in coalesced stores, V is read across its columns.
  if (E_out)
    for (int e = tid; e < M * M; e += NT) {
      const int row = e / M, rk = e % M;
      const int c = S.inv[rk];
      if (!SSL_IN_BOUNDS(c >= 0 && c < MP, flags)) continue;
      const float2 v = Vs[c * Shape<MP>::VLD + row];
      const float sc = S.vinv[c];
      E_out[e] = make_float2(v.x * sc, v.y * sc);
    }
  if (io.img)  // the spectrum's operand image, from V's columns directly
    write_noise_image(
        io, item, M,
        [&](int row, int rk) {
          const int c = S.inv[rk];
          const float2 v = Vs[c * Shape<MP>::VLD + row];
          const float sc = S.vinv[c];
          return make_float2(v.x * sc, v.y * sc);
        },
        tid, NT);
  if (tid < M) sig_out[S.rnk[tid]] = S.sig[tid];
  if (tid == 0) {
    int st = 0;
    if (S.bad != 0)
      st = SSL_E_NONFINITE;
    else if (!converged)
      st = SSL_E_NO_CONVERGENCE;
    if (status_out) *status_out = st;
    if (stats_out) {
      stats_out[0] = S.visits;
      stats_out[1] = rotations;
    }
    if (st == SSL_E_NONFINITE) atomicOr(flags, SSL_FLAG_NONFINITE);
    if (st == SSL_E_NO_CONVERGENCE) atomicOr(flags, SSL_FLAG_NO_CONVERGENCE);
  }
}

template <bool kF64, int MP>
__global__ void __launch_bounds__(Shape<MP>::THREADS, MP >= 64 ? 4 : 8)
gsvd_jacobi_kernel(const float2* __restrict__ R, const float2* __restrict__ Kinv, int B, int M,
                   int max_sweeps, float tol, float abs_tol, float* __restrict__ sigma,
                   float2* __restrict__ E, int32_t* __restrict__ status,
                   int32_t* __restrict__ stats, unsigned* flags,
                   const float2* const* __restrict__ kinv_items, const float2* __restrict__ V0,
                   const ImgOut io) {
  extern __shared__ float2 dsm[];
  __shared__ int xid[Shape<MP>::W * kBlk];
  __shared__ SmemJ<MP> S;
  const int b = blockIdx.x, k = blockIdx.y;
  const size_t item = (size_t)k * B + b;
  const float2* Kb = kinv_items ? kinv_items[k] + (size_t)b * M * M
                               : Kinv ? Kinv + (size_t)b * M * M : nullptr;
  gsvd_solve<kF64, MP>(CtaSync{}, threadIdx.x, R + item * M * M, Kb, M, max_sweeps, tol, abs_tol,
                       sigma + item * M, E ? E + item * M * M : nullptr,
                       status ? status + item : nullptr, stats ? stats + item * 2 : nullptr,
                       flags, b, dsm, dsm + MP * Shape<MP>::VLD, xid, S,
                       V0 ? V0 + item * M * M : nullptr, io, item);
}

template <bool kF64, int MP>
cudaError_t launch_mp(const float2* R, const float2* Kinv, int nblk, int B, int M, int sweeps,
                      float tol, float abs_tol, float* sigma, float2* E, int32_t* status,
                      int32_t* stats, unsigned* flags, cudaStream_t s,
                      const float2* const* kinv_items, const float2* V0, const ImgOut& io) {
  const size_t smem = ((size_t)MP * Shape<MP>::VLD + (size_t)Shape<MP>::W * kBlk * MP) * sizeof(float2);
  cudaError_t e = cudaFuncSetAttribute(gsvd_jacobi_kernel<kF64, MP>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid(B, nblk);
  gsvd_jacobi_kernel<kF64, MP><<<grid, Shape<MP>::THREADS, smem, s>>>(
      R, Kinv, B, M, sweeps, tol, abs_tol, sigma, E, status, stats, flags, kinv_items, V0, io);
  return cudaGetLastError();
}

// ---- mixed sizes: one persistent launch ------------------------------------
// Shared memory per group: V [MP][MP + 1] and W exchange slots [8][MP].
template <int MP>
__host__ __device__ constexpr int group_smem_elems() {
  return MP * Shape<MP>::VLD + Shape<MP>::W * kBlk * MP;
}
constexpr int kMixedThreads = 128;
constexpr size_t kMixedSmem = (size_t)group_smem_elems<64>() * sizeof(float2);
static_assert(2 * group_smem_elems<32>() <= group_smem_elems<64>(), "32-class groups fit");
static_assert(4 * group_smem_elems<16>() <= group_smem_elems<64>(), "16-class groups fit");

template <bool kF64, int MP>
__device__ __forceinline__ void solve_problem(const GsvdProblem& p, int tid, int max_sweeps,
                                              float rel_tol, float abs_tol, unsigned* flags,
                                              float2* base, int* xid, SmemJ<MP>& S, int g) {
  const float tol = rel_tol > 0.f ? rel_tol : (float)p.M * 5.9604644775390625e-8f;
  float2* Vs = base;
  float2* xg = base + MP * Shape<MP>::VLD;
  const ImgOut io{p.img, p.esz, p.Ns, p.KP, p.NP, nullptr};
  if (MP == 64)
    gsvd_solve<kF64, MP>(CtaSync{}, tid, p.R, p.Kinv, p.M, max_sweeps, tol, abs_tol, p.sig, p.E,
                         p.status, nullptr, flags, p.salt, Vs, xg, xid, S, nullptr, io, 0);
  else if (MP == 32)
    gsvd_solve<kF64, MP>(BarSync{1 + g, 64}, tid, p.R, p.Kinv, p.M, max_sweeps, tol, abs_tol,
                         p.sig, p.E, p.status, nullptr, flags, p.salt, Vs, xg, xid, S, nullptr,
                         io, 0);
  else
    gsvd_solve<kF64, MP>(WarpSync{}, tid, p.R, p.Kinv, p.M, max_sweeps, tol, abs_tol, p.sig,
                         p.E, p.status, nullptr, flags, p.salt, Vs, xg, xid, S, nullptr, io, 0);
}

// Every CTA takes units from a global counter until none is left: a unit is
// one matrix of the 64 class (four warps), two of the 32 class (two warps
// each, named barriers 1 and 2) or four of the 16 class (one warp each), so
// arrays of every size share the launch and the SMs stay busy to the end.
template <bool kF64>
__global__ void __launch_bounds__(kMixedThreads, 4)
gsvd_mixed_kernel(const GsvdUnit* __restrict__ units, int n_units,
                  const GsvdProblem* __restrict__ probs, int* counter, int max_sweeps,
                  float rel_tol, float abs_tol, unsigned* flags) {
  extern __shared__ float2 dsm[];
  __shared__ union {
    struct {
      int xid[4 * kBlk];
      SmemJ<64> S;
    } c64;
    struct {
      int xid[2][2 * kBlk];
      SmemJ<32> S[2];
    } c32;
    struct {
      int xid[4][kBlk];
      SmemJ<16> S[4];
    } c16;
  } U;
  __shared__ int unit_sh;
  const int tid = threadIdx.x;
  for (;;) {
    if (tid == 0) unit_sh = atomicAdd(counter, 1);
    __syncthreads();
    const int u = unit_sh;
    if (u >= n_units) break;
    const GsvdUnit un = units[u];
    if (un.mp == 64) {
      solve_problem<kF64, 64>(probs[un.prob[0]], tid, max_sweeps, rel_tol, abs_tol, flags, dsm,
                              U.c64.xid, U.c64.S, 0);
    } else if (un.mp == 32) {
      const int g = tid >> 6;
      if (g < un.n)
        solve_problem<kF64, 32>(probs[un.prob[g]], tid & 63, max_sweeps, rel_tol, abs_tol, flags,
                                dsm + g * group_smem_elems<32>(), U.c32.xid[g], U.c32.S[g], g);
    } else {
      const int g = tid >> 5;
      if (g < un.n)
        solve_problem<kF64, 16>(probs[un.prob[g]], tid & 31, max_sweeps, rel_tol, abs_tol, flags,
                                dsm + g * group_smem_elems<16>(), U.c16.xid[g], U.c16.S[g], g);
    }
    __syncthreads();
  }
}

}  // namespace

cudaError_t launch_gsvd(const float2* R, const float2* Kinv, int nblk, int B, int M,
                        const JacobiOpts& o, float* sigma, float2* E, int32_t* status,
                        int32_t* stats, unsigned* flags, cudaStream_t s,
                        const float2* const* kinv_items, const float2* V0,
                        const ImgOut* iop, float2* abuf) {
  if (o.method == SSL_SVD_BIDIAG)  // the paper's route; no warm start
    return launch_gsvd_bidiag(R, Kinv, nblk, B, M, o, sigma, E, status, stats, flags, s,
                              kinv_items, nullptr, 0, iop);
  if (o.method == SSL_SVD_SPLIT)  // the noise subspace only; no warm start
    return launch_gsvd_split(R, Kinv, nblk, B, M, o, sigma, E, status, stats, flags, s,
                             kinv_items, iop, abuf);
  const ImgOut io = iop ? *iop : ImgOut{nullptr, 0, 0, 0, 0};
  const float tol = o.rel_tol > 0.f ? o.rel_tol : (float)M * 5.9604644775390625e-8f;
  const float abs_tol = o.abs_tol > 0.f ? o.abs_tol : 0.f;
  const int sw = o.max_sweeps;
  if (o.angles_f64) {
    if (M <= 16)
      return launch_mp<true, 16>(R, Kinv, nblk, B, M, sw, tol, abs_tol, sigma, E, status, stats,
                                 flags, s, kinv_items, V0, io);
    if (M <= 32)
      return launch_mp<true, 32>(R, Kinv, nblk, B, M, sw, tol, abs_tol, sigma, E, status, stats,
                                 flags, s, kinv_items, V0, io);
    return launch_mp<true, 64>(R, Kinv, nblk, B, M, sw, tol, abs_tol, sigma, E, status, stats,
                               flags, s, kinv_items, V0, io);
  }
  if (M <= 16)
    return launch_mp<false, 16>(R, Kinv, nblk, B, M, sw, tol, abs_tol, sigma, E, status, stats,
                                flags, s, kinv_items, V0, io);
  if (M <= 32)
    return launch_mp<false, 32>(R, Kinv, nblk, B, M, sw, tol, abs_tol, sigma, E, status, stats,
                                flags, s, kinv_items, V0, io);
  return launch_mp<false, 64>(R, Kinv, nblk, B, M, sw, tol, abs_tol, sigma, E, status, stats,
                              flags, s, kinv_items, V0, io);
}

int gsvd_mixed_ctas_per_sm() {
  int n = 0;
  // the dynamic shared memory above 48 KB has to be allowed before the query
  if (cudaFuncSetAttribute(gsvd_mixed_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)kMixedSmem) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, gsvd_mixed_kernel<true>, kMixedThreads,
                                                    kMixedSmem) != cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  return n > 0 ? n : 1;
}

cudaError_t launch_gsvd_mixed(const GsvdUnit* units, int n_units, const GsvdProblem* probs,
                              int* counter, int grid, const JacobiOpts& o, unsigned* flags,
                              cudaStream_t s) {
  if (n_units <= 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  const float rel = o.rel_tol > 0.f ? o.rel_tol : 0.f;
  const float abs_tol = o.abs_tol > 0.f ? o.abs_tol : 0.f;
  grid = grid < 1 ? 1 : (grid > n_units ? n_units : grid);
  if (o.angles_f64) {
    e = cudaFuncSetAttribute(gsvd_mixed_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kMixedSmem);
    if (e != cudaSuccess) return e;
    gsvd_mixed_kernel<true><<<grid, kMixedThreads, kMixedSmem, s>>>(
        units, n_units, probs, counter, o.max_sweeps, rel, abs_tol, flags);
  } else {
    e = cudaFuncSetAttribute(gsvd_mixed_kernel<false>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMixedSmem);
    if (e != cudaSuccess) return e;
    gsvd_mixed_kernel<false><<<grid, kMixedThreads, kMixedSmem, s>>>(
        units, n_units, probs, counter, o.max_sweeps, rel, abs_tol, flags);
  }
  return cudaGetLastError();
}

}  // namespace ssl
