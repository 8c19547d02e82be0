// Whitening and generalised SVD, eq. 4 (Sec. III-A/B):
//   A = K^{-1} R = E Lambda E_r^H,   E = left singular vectors (columns).
//
// One CTA of 4 warps per (bin, block); the matrix is padded to 64 x 64.
//
//  1. A = K^{-1} R in FP32 (register-tiled complex product through shared
//     memory), kept as G = A^H.
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
//     tolerance taken from the global maximum; abs_tol = 0 disables it).  The
//     sweep loop stops after the first sweep that rotates nothing.
//  6. Angles.  FP64 (default): the CTA's 32 pairs are gathered so that warp 0
//     computes them one pair per lane, because on this part an FP64 warp
//     instruction costs the same with one active lane as with 32; the
//     decision and the rotation are evaluated in FP64 (FP32 estimates refined
//     by one Newton-Raphson step each).  FP32: each warp computes its own 8
//     pairs and the warps run without block barriers between exchanges.
//  7. Singular values = column norms, sorted descending (Alg. 1's sort step);
//     E's columns (V's, renormalised) are permuted accordingly.
#include <float.h>

#include "ssl_internal.cuh"

namespace ssl {
namespace {

constexpr int kThreads = 128;
constexpr int kWarps = 4;
constexpr int kCols = 16;  // columns per warp (two blocks of 8)
constexpr int kBlk = 8;
constexpr unsigned kFull = 0xffffffffu;

// Transposing butterfly over 16 values: on exit lanes 2i and 2i + 1 hold the
// warp-wide sum of value i (16 shuffles instead of 5 per value).
__device__ __forceinline__ float transpose_reduce16(float (&x)[16], int lane) {
#pragma unroll
  for (int w = 16, n = 8; w >= 2; w >>= 1, n >>= 1) {
    const bool hi = (lane & w) != 0;
#pragma unroll
    for (int k = 0; k < n; ++k) {
      const float send = hi ? x[k] : x[k + n];
      const float keep = hi ? x[k + n] : x[k];
      x[k] = keep + __shfl_xor_sync(kFull, send, w);
    }
  }
  return x[0] + __shfl_xor_sync(kFull, x[0], 1);
}

__device__ __forceinline__ float norm2(const float2 (&x)[2]) {
  return fmaf(x[0].x, x[0].x, fmaf(x[0].y, x[0].y, fmaf(x[1].x, x[1].x, x[1].y * x[1].y)));
}

// conj(x) . y over the lane's two rows
__device__ __forceinline__ void dot_partial(const float2 (&x)[2], const float2 (&y)[2], float& gr,
                                            float& gi) {
  gr = fmaf(x[0].x, y[0].x, fmaf(x[0].y, y[0].y, fmaf(x[1].x, y[1].x, x[1].y * y[1].y)));
  gi = fmaf(x[0].x, y[0].y, fmaf(-x[0].y, y[0].x, fmaf(x[1].x, y[1].y, -x[1].y * y[1].x)));
}

// x' = c x - conj(se) y ;  y' = se x + c y
__device__ __forceinline__ void rot1(float2& x, float2& y, float c, float sr, float si) {
  const float2 a = x, d = y;
  x = make_float2(fmaf(c, a.x, -fmaf(sr, d.x, si * d.y)), fmaf(c, a.y, -fmaf(sr, d.y, -si * d.x)));
  y = make_float2(fmaf(c, d.x, fmaf(sr, a.x, -si * a.y)), fmaf(c, d.y, fmaf(sr, a.y, si * a.x)));
}

// ---- rotation for one pair --------------------------------------------------
// In: alpha, beta (squared norms), gamma = (gr, gi), thresholds.
// Out: o = (c, sr, si, 1) with s e = sr + i si, e = gamma/|gamma|, and the new
// squared norms.  Returns false for "converged" (o, norms untouched).
// Inputs are scaled by a power of two so that max(alpha, beta) is in [1, 2):
// the rotation is scale-invariant and all intermediates stay well inside the
// FP32 range of the hardware estimates.  A pair whose norm ratio is below
// 2^-60 is left alone (its rotation would change V by less than 2^-30).
//
// With d = beta - alpha the rotation's tangent solves t^2 + (d/|gamma|) t = 1;
// the smaller root is t = sign(d) 2|gamma| / (|d| + sqrt(d^2 + 4|gamma|^2)).
// With den = |d| + sqrt(d^2 + 4|gamma|^2) and q = den^2 + 4|gamma|^2:
//   c = den / sqrt(q),   s e = sign(d) 2 gamma / sqrt(q),
//   alpha' = alpha - t |gamma|,  beta' = beta + t |gamma|,
//   t |gamma| = sign(d) 2 |gamma|^2 / den = sign(d) (sqrt(d^2 + 4|gamma|^2) - |d|) / 2.

__device__ __forceinline__ float pow2_scale(float m) {  // 2^-floor(log2 m), m normal
  const int e = min((__float_as_int(m) >> 23) & 0xff, 253);
  return __int_as_float((254 - e) << 23);
}

// Newton-Raphson step for 1/sqrt(x) from an FP32 estimate y0:
// y <- y (3 - x y^2) / 2 roughly doubles the number of correct bits.
__device__ __forceinline__ double rsqrt_nr(double x, float y0) {
  const double y = (double)y0;
  const double h = x * y * y;
  return y * fma(-0.5, h, 1.5);
}

template <bool kF64>
__device__ __forceinline__ bool rotation(float al, float be, float gr, float gi, float tol,
                                         float abs_thr, float4& o, float& al_out,
                                         float& be_out) {
  const float m = fmaxf(al, be);
  if (!(m >= FLT_MIN)) return false;  // zero (padding) or non-finite
  const float sc = pow2_scale(m);
  const float a = al * sc, b = be * sc, x = gr * sc, y = gi * sc;
  if (!(fminf(a, b) >= 8.67361738e-19f)) return false;  // norm ratio below 2^-60
  const float at = abs_thr * sc;
  if (kF64) {
    // Decision: |gamma|^2 against max(tol^2 alpha beta, at^2).  The FP32
    // evaluation is within a few ulp of the exact one, so outside a 2^-18
    // band around the threshold it already gives the FP64 answer; inside the
    // band the comparison is redone in FP64.
    const float g4s = fmaf(2.f * x, 2.f * x, 4.f * y * y);
    const float lims = fmaxf(4.f * tol * tol * (a * b), 4.f * at * at);
    if (!(g4s > lims * 0.99999619f)) return false;  // below the band: converged
    const double ad = a, bd = b, xd = 2.0 * (double)x, yd = 2.0 * (double)y;
    const double g4 = fma(xd, xd, yd * yd);  // 4 |gamma|^2
    if (!(g4s > lims * 1.00000381f)) {        // inside the band: exact test
      const double td = tol, atd = at;
      const double lim = fmax(4.0 * td * td * (ad * bd), 4.0 * atd * atd);
      if (!(g4 > lim)) return false;
    }
    const double d = bd - ad;
    const double w = fma(d, d, g4);
    // FP32 estimates of the same chain seed the FP64 Newton steps
    const float g4f = g4s;
    const float df = b - a;
    const float wf = fmaf(df, df, g4f);
    const float denf = fabsf(df) + sqrtf(wf);
    const double sw = w * rsqrt_nr(w, rsqrtf(wf));
    const double den = fabs(d) + sw;
    const double q = fma(den, den, g4);
    const double rq = rsqrt_nr(q, rsqrtf(fmaf(denf, denf, g4f)));
    const float c = (float)(den * rq);
    const float f = (float)(d < 0.0 ? -rq : rq);
    o = make_float4(c, f * (2.f * x), f * (2.f * y), 1.f);
    // t |gamma| (signed with t) in the caller's scale; g4 / den = sw - |d|
    // because den (sw - |d|) = sw^2 - d^2 = g4.
    const double tg = 0.5 * (sw - fabs(d));
    const float tgf = (float)(d < 0.0 ? -tg : tg) / sc;
    al_out = fmaxf(al - tgf, 0.f);
    be_out = fmaxf(be + tgf, 0.f);
    return true;
  } else {
    const float g4 = fmaf(2.f * x, 2.f * x, 4.f * y * y);
    if (!(g4 > 4.f * tol * tol * (a * b)) || !(g4 > 4.f * at * at)) return false;
    const float d = b - a;
    const float sw = sqrtf(fmaf(d, d, g4));
    const float den = fabsf(d) + sw;
    const float rq = __frsqrt_rn(fmaf(den, den, g4));
    const float c = den * rq;
    const float f = d < 0.f ? -rq : rq;
    o = make_float4(c, f * (2.f * x), f * (2.f * y), 1.f);
    const float tgf = (d < 0.f ? -0.5f : 0.5f) * (sw - fabsf(d)) / sc;  // signed t |gamma|
    al_out = fmaxf(al - tgf, 0.f);
    be_out = fmaxf(be + tgf, 0.f);
    return true;
  }
}

struct SmemJ {
  float gram[kWarps * 16];    // [warp][pair][re, im]
  float4 rot[kWarps * 8];     // [warp][pair]
  float nrm[kWarps * kCols];  // squared norms per (warp, slot)
  int colid[kWarps * kCols];  // logical column per (warp, slot)
  float red[kWarps];
  float sig[64];
  int rnk[64];
  int rot_count;
  int bad;
};

// Rotate V's columns p, q (logical ids) in shared memory.
__device__ __forceinline__ void rot_v(float2* Vs, int p, int q, int lane, float c, float sr,
                                      float si) {
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    float2 a = Vs[p * 64 + lane + 32 * h], d = Vs[q * 64 + lane + 32 * h];
    rot1(a, d, c, sr, si);
    Vs[p * 64 + lane + 32 * h] = a;
    Vs[q * 64 + lane + 32 * h] = d;
  }
}

// Slot of pair k's second column: intra rounds (KIND 0) pair slot k with
// slot 15 - k, cross rounds (KIND 1) with slot 8 + k.
template <int KIND>
__host__ __device__ constexpr int partner(int k) {
  return KIND == 0 ? 15 - k : kBlk + k;
}

// One inner round over the warp's 8 pairs (k, partner<KIND>(k)).
template <bool kF64, int KIND>
__device__ __forceinline__ void inner_round(float2 (&g)[kCols][2], SmemJ& S, float2* Vs, int warp,
                                            int lane, float tol, float abs_thr, int& wrot) {
  float x[16];
#pragma unroll
  for (int k = 0; k < 8; ++k) dot_partial(g[k], g[partner<KIND>(k)], x[2 * k], x[2 * k + 1]);
  const float v = transpose_reduce16(x, lane);
  if ((lane & 1) == 0) S.gram[warp * 16 + (lane >> 1)] = v;
  if (kF64) {
    __syncthreads();
    if (warp == 0) {
      const int w = lane >> 3, k = lane & 7;
      const int sp = w * kCols + k, sq = w * kCols + partner<KIND>(k);
      const float2 gm = reinterpret_cast<const float2*>(S.gram)[w * 8 + k];
      float4 o = make_float4(1.f, 0.f, 0.f, 0.f);
      float na = 0.f, nb = 0.f;
      const bool did = rotation<true>(S.nrm[sp], S.nrm[sq], gm.x, gm.y, tol, abs_thr, o, na, nb);
      S.rot[lane] = o;
      if (did) {
        S.nrm[sp] = na;
        S.nrm[sq] = nb;
      }
      wrot += __popc(__ballot_sync(kFull, did));
    }
    __syncthreads();
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
      rot1(g[k][0], g[partner<KIND>(k)][0], cs.x, cs.y, cs.z);
      rot1(g[k][1], g[partner<KIND>(k)][1], cs.x, cs.y, cs.z);
      rot_v(Vs, S.colid[warp * kCols + k], S.colid[warp * kCols + partner<KIND>(k)], lane, cs.x,
            cs.y, cs.z);
    }
  }
}

// Circle method over the warp's 16 slots: after a round, slot i takes slot
// i + 1's column (i = 1..14) and slot 15 takes slot 1's; the column ids and
// norms move with the registers.  After 15 rounds every local pair has met.
__device__ __forceinline__ void shift_circle16(float2 (&g)[kCols][2], SmemJ& S, int warp,
                                               int lane) {
  const float2 t0 = g[1][0], t1 = g[1][1];
#pragma unroll
  for (int i = 1; i < 15; ++i) {
    g[i][0] = g[i + 1][0];
    g[i][1] = g[i + 1][1];
  }
  g[15][0] = t0;
  g[15][1] = t1;
  int id = 0;
  float nr = 0.f;
  if (lane >= 1 && lane < 16) {
    const int src = warp * kCols + (lane == 15 ? 1 : lane + 1);
    id = S.colid[src];
    nr = S.nrm[src];
  }
  __syncwarp();
  if (lane >= 1 && lane < 16) {
    S.colid[warp * kCols + lane] = id;
    S.nrm[warp * kCols + lane] = nr;
  }
  __syncwarp();
}

// Cross rounds: after a round the bottom block rotates by one slot (slot
// 8 + i takes slot 8 + i + 1's column, slot 15 takes slot 8's), so that after
// 8 rounds every top/bottom pair has met; ids and norms move along.
__device__ __forceinline__ void shift_bottom8(float2 (&g)[kCols][2], SmemJ& S, int warp,
                                              int lane) {
  const float2 t0 = g[kBlk][0], t1 = g[kBlk][1];
#pragma unroll
  for (int i = kBlk; i < 15; ++i) {
    g[i][0] = g[i + 1][0];
    g[i][1] = g[i + 1][1];
  }
  g[15][0] = t0;
  g[15][1] = t1;
  int id = 0;
  float nr = 0.f;
  if (lane >= kBlk && lane < 16) {
    const int src = warp * kCols + (lane == 15 ? kBlk : lane + 1);
    id = S.colid[src];
    nr = S.nrm[src];
  }
  __syncwarp();
  if (lane >= kBlk && lane < 16) {
    S.colid[warp * kCols + lane] = id;
    S.nrm[warp * kCols + lane] = nr;
  }
  __syncwarp();
}

// Exact squared norms of the warp's 16 columns into S.nrm.
__device__ __forceinline__ void refresh_norms(const float2 (&g)[kCols][2], SmemJ& S, int warp,
                                              int lane) {
  float x[16];
#pragma unroll
  for (int c = 0; c < kCols; ++c) x[c] = norm2(g[c]);
  const float v = transpose_reduce16(x, lane);
  if ((lane & 1) == 0) S.nrm[warp * kCols + (lane >> 1)] = v;
  __syncwarp();
}

// Block exchange between block rounds (circle method over 8 block positions,
// warp s holding positions s (top) and 7 - s (bottom); position 0 fixed).
__device__ __forceinline__ void store_block(const float2 (&g)[kCols][2], const SmemJ& S, int half,
                                            float2* xg, int* xid, int slot, int warp, int lane) {
#pragma unroll
  for (int c = 0; c < kBlk; ++c)
#pragma unroll
    for (int h = 0; h < 2; ++h) xg[(slot * kBlk + c) * 64 + lane + 32 * h] = g[half * kBlk + c][h];
  if (lane < kBlk) xid[slot * kBlk + lane] = S.colid[warp * kCols + half * kBlk + lane];
}
__device__ __forceinline__ void load_block(float2 (&g)[kCols][2], SmemJ& S, int half,
                                           const float2* xg, const int* xid, int slot, int warp,
                                           int lane) {
#pragma unroll
  for (int c = 0; c < kBlk; ++c)
#pragma unroll
    for (int h = 0; h < 2; ++h) g[half * kBlk + c][h] = xg[(slot * kBlk + c) * 64 + lane + 32 * h];
  if (lane < kBlk) S.colid[warp * kCols + half * kBlk + lane] = xid[slot * kBlk + lane];
}
__device__ __forceinline__ int slot_of(int w, int half) { return 2 * w + half; }

__device__ __forceinline__ void exchange(float2 (&g)[kCols][2], SmemJ& S, float2* xg, int* xid,
                                         int warp, int lane) {
  if (warp == 0) {
    store_block(g, S, 1, xg, xid, slot_of(1, 1), warp, lane);
  } else if (warp == 1) {
    store_block(g, S, 0, xg, xid, slot_of(0, 1), warp, lane);
    store_block(g, S, 1, xg, xid, slot_of(2, 1), warp, lane);
  } else if (warp == 2) {
    store_block(g, S, 0, xg, xid, slot_of(1, 0), warp, lane);
    store_block(g, S, 1, xg, xid, slot_of(3, 1), warp, lane);
  } else {
    store_block(g, S, 0, xg, xid, slot_of(2, 0), warp, lane);
  }
  __syncthreads();
  if (warp == 0) {
    load_block(g, S, 1, xg, xid, slot_of(0, 1), warp, lane);
  } else if (warp == 1) {
    load_block(g, S, 0, xg, xid, slot_of(1, 0), warp, lane);
    load_block(g, S, 1, xg, xid, slot_of(1, 1), warp, lane);
  } else if (warp == 2) {
    load_block(g, S, 0, xg, xid, slot_of(2, 0), warp, lane);
    load_block(g, S, 1, xg, xid, slot_of(2, 1), warp, lane);
  } else {
    // the bottom block becomes the top block in place
    int id = 0;
    if (lane < kBlk) id = S.colid[warp * kCols + kBlk + lane];
#pragma unroll
    for (int c = 0; c < kBlk; ++c)
#pragma unroll
      for (int h = 0; h < 2; ++h) g[c][h] = g[kBlk + c][h];
    __syncwarp();
    if (lane < kBlk) S.colid[warp * kCols + lane] = id;
    load_block(g, S, 1, xg, xid, slot_of(3, 1), warp, lane);
  }
  __syncthreads();
}

template <bool kF64>
__global__ void __launch_bounds__(kThreads, 3)
gsvd_jacobi_kernel(const float2* __restrict__ R, const float2* __restrict__ Kinv, int B, int M,
                   int max_sweeps, float tol, float abs_tol, float* __restrict__ sigma,
                   float2* __restrict__ E, int32_t* __restrict__ status,
                   int32_t* __restrict__ stats, unsigned* flags,
                   const float2* const* __restrict__ kinv_items) {
  extern __shared__ float2 dsm[];
  float2* Vs = dsm;            // [64 columns][64 rows]
  float2* xg = dsm + 64 * 64;  // [8 slots][8 columns][64 rows]: exchange and staging
  __shared__ int xid[8 * kBlk];
  __shared__ SmemJ S;

  const int b = blockIdx.x, k = blockIdx.y;
  const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
  const size_t mat = ((size_t)k * B + b) * M * M;

  if (tid == 0) {
    S.bad = 0;
    S.rot_count = 0;
  }
  // ---- A = K^{-1} R: stage K^{-1} (in Vs) and R (in xg), dense row-major ----
  {
    float2* Ks = Vs;
    float2* Rs = xg;
    const float2* Kb = (kinv_items ? kinv_items[k] : Kinv) + (size_t)b * M * M;
    const float2* Rb = R + mat;
    for (int e = tid; e < M * M; e += kThreads) {
      Ks[e] = Kb[e];
      Rs[e] = Rb[e];
    }
    __syncthreads();
    // thread tile: rows i = tid/16 + 8a (a < 8), cols j = tid%16 + 16c (c < 4)
    const int ti = tid / 16, tj = tid % 16;
    float2 acc[8][4];
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[a][c] = make_float2(0.f, 0.f);
    for (int m = 0; m < M; ++m) {
      float2 kv[8], rv[4];
#pragma unroll
      for (int a = 0; a < 8; ++a) {
        const int i = ti + 8 * a;
        kv[a] = i < M ? Ks[i * M + m] : make_float2(0.f, 0.f);
      }
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int j = tj + 16 * c;
        rv[c] = j < M ? Rs[m * M + j] : make_float2(0.f, 0.f);
      }
#pragma unroll
      for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          acc[a][c].x = fmaf(kv[a].x, rv[c].x, fmaf(-kv[a].y, rv[c].y, acc[a][c].x));
          acc[a][c].y = fmaf(kv[a].x, rv[c].y, fmaf(kv[a].y, rv[c].x, acc[a][c].y));
        }
    }
    bool finite = true;
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
      for (int c = 0; c < 4; ++c) finite &= isfinite(acc[a][c].x) && isfinite(acc[a][c].y);
    if (!finite) atomicExch(&S.bad, 1);
    __syncthreads();
    // G = A^H, column-major in xg: column i of G = conj(row i of A); V = I.
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int i = ti + 8 * a, j = tj + 16 * c;
        xg[i * 64 + j] = (i < M && j < M) ? make_float2(acc[a][c].x, -acc[a][c].y)
                                          : make_float2(0.f, 0.f);
      }
    for (int e = tid; e < 64 * 64; e += kThreads)
      Vs[e] = make_float2((e / 64) == (e % 64) ? 1.f : 0.f, 0.f);
    __syncthreads();
  }

  // ---- the warp's 16 columns: top block = position warp, bottom = 7 - warp
  float2 g[kCols][2];
#pragma unroll
  for (int half = 0; half < 2; ++half) {
    const int blk = half == 0 ? warp : 7 - warp;
#pragma unroll
    for (int c = 0; c < kBlk; ++c)
#pragma unroll
      for (int h = 0; h < 2; ++h) g[half * kBlk + c][h] = xg[(blk * kBlk + c) * 64 + lane + 32 * h];
    if (lane < kBlk) S.colid[warp * kCols + half * kBlk + lane] = blk * kBlk + lane;
  }
  __syncthreads();

  int sweeps = 0, rotations = 0, wrot = 0;
  bool converged = S.bad != 0;
  for (int sw = 0; sw < max_sweeps && !converged; ++sw) {
    float abs_thr = 0.f;
    refresh_norms(g, S, warp, lane);
    if (abs_tol > 0.f) {
      float mx = lane < kCols ? S.nrm[warp * kCols + lane] : 0.f;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(kFull, mx, o));
      if (lane == 0) S.red[warp] = mx;
      __syncthreads();
      abs_thr = abs_tol * fmaxf(fmaxf(S.red[0], S.red[1]), fmaxf(S.red[2], S.red[3]));
    }
    __syncthreads();
    // block round 0: all pairs among the warp's 16 columns
#pragma unroll 1
    for (int r = 0; r < 15; ++r) {
      inner_round<kF64, 0>(g, S, Vs, warp, lane, tol, abs_thr, wrot);
      shift_circle16(g, S, warp, lane);
    }
    // block rounds 1..6: pairs across the two blocks, after a block exchange
#pragma unroll 1
    for (int br = 1; br < 7; ++br) {
      exchange(g, S, xg, xid, warp, lane);
      refresh_norms(g, S, warp, lane);
      if (kF64) __syncthreads();
#pragma unroll 1
      for (int j = 0; j < kBlk; ++j) {
        inner_round<kF64, 1>(g, S, Vs, warp, lane, tol, abs_thr, wrot);
        shift_bottom8(g, S, warp, lane);
      }
    }
    if (lane == 0 && wrot != 0) atomicAdd(&S.rot_count, wrot);
    wrot = 0;
    exchange(g, S, xg, xid, warp, lane);  // back to the starting positions
    ++sweeps;
    const int rc = S.rot_count;
    rotations += rc;
    converged = (rc == 0);
    __syncthreads();
    if (tid == 0) S.rot_count = 0;
  }

  // ---- singular values: column norms of G, by logical column ----
  {
    float x[16];
#pragma unroll
    for (int c = 0; c < kCols; ++c) x[c] = norm2(g[c]);
    const float v = transpose_reduce16(x, lane);
    if ((lane & 1) == 0) {
      const int id = S.colid[warp * kCols + (lane >> 1)];
      S.sig[id] = id < M ? sqrtf(v) : -1.f;
    }
  }
  __syncthreads();
  if (tid < 64) {
    const float v = S.sig[tid];
    int rk = 0;
    for (int c = 0; c < 64; ++c) {
      const float w = S.sig[c];
      rk += (w > v) || (w == v && c < tid);
    }
    S.rnk[tid] = rk;
  }
  __syncthreads();
  // E[:, rank(c)] = V[:, c] / |V[:, c]|, staged row-major in xg, copied out.
  float2* Es = xg;
  for (int c = warp; c < M; c += kWarps) {
    const float2 v0 = Vs[c * 64 + lane], v1 = Vs[c * 64 + lane + 32];
    float n2 = fmaf(v0.x, v0.x, fmaf(v0.y, v0.y, fmaf(v1.x, v1.x, v1.y * v1.y)));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) n2 += __shfl_xor_sync(kFull, n2, o);
    const float inv = n2 > 0.f ? __frsqrt_rn(n2) : 1.f;
    const int rk = S.rnk[c];
    if (lane < M) Es[lane * M + rk] = make_float2(v0.x * inv, v0.y * inv);
    if (lane + 32 < M) Es[(lane + 32) * M + rk] = make_float2(v1.x * inv, v1.y * inv);
  }
  __syncthreads();
  for (int e = tid; e < M * M; e += kThreads) E[mat + e] = Es[e];
  if (tid < M) sigma[((size_t)k * B + b) * M + S.rnk[tid]] = S.sig[tid];
  if (tid == 0) {
    int st = 0;
    if (S.bad != 0)
      st = SSL_E_NONFINITE;
    else if (!converged)
      st = SSL_E_NO_CONVERGENCE;
    if (status) status[(size_t)k * B + b] = st;
    if (stats) {
      stats[((size_t)k * B + b) * 2 + 0] = sweeps;
      stats[((size_t)k * B + b) * 2 + 1] = rotations;
    }
    if (st == SSL_E_NONFINITE) atomicOr(flags, SSL_FLAG_NONFINITE);
    if (st == SSL_E_NO_CONVERGENCE) atomicOr(flags, SSL_FLAG_NO_CONVERGENCE);
  }
}

}  // namespace

cudaError_t launch_gsvd(const float2* R, const float2* Kinv, int nblk, int B, int M,
                        const JacobiOpts& o, float* sigma, float2* E, int32_t* status,
                        int32_t* stats, unsigned* flags, cudaStream_t s,
                        const float2* const* kinv_items) {
  const size_t smem = 2 * 64 * 64 * sizeof(float2);
  const float tol = o.rel_tol > 0.f ? o.rel_tol : (float)M * 5.9604644775390625e-8f;
  const float abs_tol = o.abs_tol > 0.f ? o.abs_tol : 0.f;
  dim3 grid(B, nblk);
  cudaError_t e;
  if (o.angles_f64) {
    e = cudaFuncSetAttribute(gsvd_jacobi_kernel<true>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    gsvd_jacobi_kernel<true><<<grid, kThreads, smem, s>>>(R, Kinv, B, M, o.max_sweeps, tol,
                                                           abs_tol, sigma, E, status, stats,
                                                           flags, kinv_items);
  } else {
    e = cudaFuncSetAttribute(gsvd_jacobi_kernel<false>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    gsvd_jacobi_kernel<false><<<grid, kThreads, smem, s>>>(R, Kinv, B, M, o.max_sweeps, tol,
                                                            abs_tol, sigma, E, status, stats,
                                                            flags, kinv_items);
  }
  return cudaGetLastError();
}

}  // namespace ssl
