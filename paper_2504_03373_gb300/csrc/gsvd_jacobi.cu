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
//  3. Data stay in registers.  Each warp owns 16 columns of G and of V (two
//     blocks of 8; lane l holds rows l and l + 32).  A sweep is a block-level
//     round-robin over the 8 blocks: in the first block round every warp
//     rotates all 120 pairs among its own 16 columns, in the 6 following ones
//     only the 64 pairs across its two blocks, after which blocks move to the
//     next warp through shared memory (circle method on block positions).
//     Each "inner round" rotates 32 disjoint pairs, 8 per warp; 63 inner
//     rounds visit each of the 2016 pairs once.
//  4. Per inner round: the Gram entries alpha = |g_p|^2, beta = |g_q|^2 and
//     gamma = g_p^H g_q of a warp's 8 pairs are formed in FP32 and reduced
//     with a transposing butterfly (32 values over 32 lanes in 31 shuffles);
//     warp 0 then computes all 32 rotations, one pair per lane, because FP64
//     issue is the scarce resource on this part and a warp instruction costs
//     the same with one active lane as with 32; all warps apply the rotations
//     to their registers.
//  5. Convergence (the Jacobi counterpart of Sec. III-B's tolerance): a pair
//     is rotated only if |gamma| > tol * sqrt(alpha * beta), tol = M 2^-24
//     (relative test) and |gamma| > abs_tol * max_c |g_c|^2 (the paper's
//     tolerance taken from the global maximum; abs_tol = 0 disables it).  The
//     sweep loop stops after the first sweep that rotates nothing.
//  6. Angles: with ANGLES_F64 the decision and tan(theta) are computed in
//     FP64 from the FP32 Gram entries (hardware FP32 estimates refined by
//     Newton-Raphson steps in FP64); with ANGLES_F32 everything stays FP32.
//  7. Singular values = column norms, sorted descending (Alg. 1's sort step);
//     E's columns are permuted accordingly.
#include <float.h>

#include "ssl_internal.cuh"

namespace ssl {
namespace {

constexpr int kThreads = 128;
constexpr int kWarps = 4;
constexpr int kCols = 16;    // columns per warp (two blocks of 8)
constexpr int kBlk = 8;
constexpr unsigned kFull = 0xffffffffu;

struct Cols {
  float2 g[kCols][2];  // G columns, rows lane and lane + 32
  float2 v[kCols][2];  // V columns
};

// Transposing butterfly: on entry every lane holds 32 partial values; on exit
// lane l holds the warp-wide sum of value l.  31 shuffles instead of 5 per
// value.
__device__ __forceinline__ float transpose_reduce32(float (&x)[32], int lane) {
#pragma unroll
  for (int w = 16; w >= 1; w >>= 1) {
    const bool hi = (lane & w) != 0;
#pragma unroll
    for (int k = 0; k < w; ++k) {
      const float send = hi ? x[k] : x[k + w];
      const float keep = hi ? x[k + w] : x[k];
      x[k] = keep + __shfl_xor_sync(kFull, send, w);
    }
  }
  return x[0];
}

__device__ __forceinline__ void gram_partial(const float2 (&x)[2], const float2 (&y)[2], float& a,
                                             float& b, float& gr, float& gi) {
  a = fmaf(x[0].x, x[0].x, fmaf(x[0].y, x[0].y, fmaf(x[1].x, x[1].x, x[1].y * x[1].y)));
  b = fmaf(y[0].x, y[0].x, fmaf(y[0].y, y[0].y, fmaf(y[1].x, y[1].x, y[1].y * y[1].y)));
  // conj(x) . y
  gr = fmaf(x[0].x, y[0].x, fmaf(x[0].y, y[0].y, fmaf(x[1].x, y[1].x, x[1].y * y[1].y)));
  gi = fmaf(x[0].x, y[0].y, fmaf(-x[0].y, y[0].x, fmaf(x[1].x, y[1].y, -x[1].y * y[1].x)));
}

// x' = c x - conj(se) y ;  y' = se x + c y
__device__ __forceinline__ void rotate2(float2 (&x)[2], float2 (&y)[2], float c, float sr,
                                        float si) {
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const float2 a = x[h], d = y[h];
    x[h] = make_float2(fmaf(c, a.x, -fmaf(sr, d.x, si * d.y)),
                       fmaf(c, a.y, -fmaf(sr, d.y, -si * d.x)));
    y[h] = make_float2(fmaf(c, d.x, fmaf(sr, a.x, -si * a.y)),
                       fmaf(c, d.y, fmaf(sr, a.y, si * a.x)));
  }
}

// ---- rotation angle for one pair --------------------------------------------
// In: alpha, beta, gamma (FP32 Gram entries), thresholds.  Out: (c, sr, si)
// with s e = sr + i si, e = gamma / |gamma|; returns false for "converged".
// Inputs are first scaled by a power of two so that max(alpha, beta) is in
// [1, 2): the rotation is scale-invariant and every intermediate stays well
// inside the FP32 range used for the hardware estimates.  Pairs whose norm
// ratio is below 2^-60 are left alone (their rotation would change V by less
// than 2^-30).

__device__ __forceinline__ float pow2_scale(float m) {  // 2^-floor(log2 m), m normal
  const int e = min((__float_as_int(m) >> 23) & 0xff, 253);
  return __int_as_float((254 - e) << 23);
}

// Newton-Raphson refinement of FP32 estimates (each step roughly doubles the
// number of correct bits; the estimates come from the same quantities
// computed in FP32, so no FP64 -> FP32 conversion is needed):
//   1/sqrt(x):  y <- y (3 - x y^2) / 2        1/x:  y <- y (2 - x y)
__device__ __forceinline__ double rsqrt_nr(double x, float y0) {
  const double y = (double)y0;
  const double h = x * y * y;
  return y * fma(-0.5, h, 1.5);
}
__device__ __forceinline__ double rcp_nr(double x, float y0) {
  const double y = (double)y0;
  return y * fma(-x, y, 2.0);
}

template <bool kF64>
__device__ __forceinline__ bool rotation(float al, float be, float gr, float gi, float tol,
                                         float abs_thr, float4& out) {
  const float m = fmaxf(al, be);
  if (!(m >= FLT_MIN)) return false;  // zero (padding) or non-finite
  const float sc = pow2_scale(m);
  al *= sc;
  be *= sc;
  gr *= sc;
  gi *= sc;
  const float mn = fminf(al, be);
  if (!(mn >= 8.67361738e-19f)) return false;  // 2^-60
  // absolute (global-maximum) criterion, scaled the same way
  const float at = abs_thr * sc;
  if (kF64) {
    // Exact decision and tan(theta) in FP64.
    const double a = al, b = be, x = gr, y = gi;
    const double g2 = fma(x, x, y * y);
    const double t2 = (double)tol * (double)tol;
    const double atd = at;
    if (!(g2 > t2 * (a * b)) || !(g2 > atd * atd)) return false;
    // FP32 estimates of the same chain seed the FP64 Newton steps.
    const float g2f = fmaf(gr, gr, gi * gi);
    const float rgf = rsqrtf(g2f);
    const float zf = fabsf((be - al) * (0.5f * rgf));
    const float uf = fmaf(zf, zf, 1.0f);
    const float ruf = rsqrtf(uf);
    const float df = fmaf(uf, ruf, zf);
    const double rg = rsqrt_nr(g2, rgf);        // 1 / |gamma|
    const double zeta = (b - a) * (0.5 * rg);   // (beta - alpha) / (2 |gamma|)
    const double z = fabs(zeta);
    const double u = fma(z, z, 1.0);
    const double su = u * rsqrt_nr(u, ruf);     // sqrt(1 + zeta^2)
    double t = rcp_nr(z + su, __frcp_rn(df));   // |tan(theta)|, the smaller root
    t = zeta < 0.0 ? -t : t;
    // c and s e are rounded once each from accurate values, so that the
    // applied 2x2 matrix is unitary to within rounding, without bias.
    const float tf = (float)t;
    const float c = __frsqrt_rn(fmaf(tf, tf, 1.0f));
    const float sg = c * tf * (float)rg;
    out = make_float4(c, sg * gr, sg * gi, 1.0f);
    return true;
  } else {
    const float g2f = fmaf(gr, gr, gi * gi);
    if (!(g2f > tol * tol * (al * be)) || !(g2f > at * at)) return false;
    const float rg = __frsqrt_rn(g2f);
    const float zeta = (be - al) * (0.5f * rg);
    const float z = fabsf(zeta);
    float t = 1.0f / (z + sqrtf(fmaf(z, z, 1.0f)));
    t = zeta < 0.0f ? -t : t;
    const float c = __frsqrt_rn(fmaf(t, t, 1.0f));
    const float sg = c * t * rg;
    out = make_float4(c, sg * gr, sg * gi, 1.0f);
    return true;
  }
}

// ---- one inner round: 8 pairs per warp ---------------------------------------
struct SmemJ {
  float gram[kWarps * 32];  // [pair][alpha, beta, gr, gi]
  float4 rot[kWarps * 8];
  float colnorm[kWarps * kCols];
  float padmass[kWarps * kCols];
  float sig[64];
  int rnk[64];
  int rot_count;
  int bad;
};

// Pairs are always register slots (k, Q0 + k*QS) so that every register index
// is a compile-time constant; the round-robin order is realised by moving
// columns between slots (shift_* below) instead of by indexing.
// FP64 angles: the 32 pairs of the CTA are gathered so that warp 0 computes
// them one per lane (FP64 issue costs the same for 1 or 32 active lanes).
// FP32 angles: each warp computes its own 8 pairs (lanes 0..7) and the warps
// run independently between block exchanges.  wrot counts the rotations this
// warp applied (FP32 path) or the CTA applied (FP64 path, warp 0).
template <bool kF64, int Q0, int QS>
__device__ __forceinline__ void inner_round(Cols& C, SmemJ& S, int warp, int lane, float tol,
                                            float abs_thr, int& wrot) {
  float x[32];
#pragma unroll
  for (int k = 0; k < 8; ++k)
    gram_partial(C.g[k], C.g[Q0 + QS * k], x[4 * k + 0], x[4 * k + 1], x[4 * k + 2],
                 x[4 * k + 3]);
  const float mine = transpose_reduce32(x, lane);
  S.gram[warp * 32 + lane] = mine;
  if (kF64) {
    __syncthreads();
    if (warp == 0) {
      const float4 g = reinterpret_cast<const float4*>(S.gram)[lane];
      float4 o = make_float4(1.f, 0.f, 0.f, 0.f);
      const bool did = rotation<true>(g.x, g.y, g.z, g.w, tol, abs_thr, o);
      S.rot[lane] = o;
      wrot += __popc(__ballot_sync(kFull, did));
    }
    __syncthreads();
  } else {
    __syncwarp();
    bool did = false;
    if (lane < 8) {
      const float4 g = reinterpret_cast<const float4*>(S.gram)[warp * 8 + lane];
      float4 o = make_float4(1.f, 0.f, 0.f, 0.f);
      did = rotation<false>(g.x, g.y, g.z, g.w, tol, abs_thr, o);
      S.rot[warp * 8 + lane] = o;
    }
    wrot += __popc(__ballot_sync(kFull, did));
    __syncwarp();
  }
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const float4 cs = S.rot[warp * 8 + k];
    if (cs.w != 0.f) {
      rotate2(C.g[k], C.g[Q0 + QS * k], cs.x, cs.y, cs.z);
      rotate2(C.v[k], C.v[Q0 + QS * k], cs.x, cs.y, cs.z);
    }
  }
}

__device__ __forceinline__ void move_col(Cols& C, int dst, int src) {
  C.g[dst][0] = C.g[src][0];
  C.g[dst][1] = C.g[src][1];
  C.v[dst][0] = C.v[src][0];
  C.v[dst][1] = C.v[src][1];
}

// Circle method over the 16 local slots: pairs (k, 15 - k); afterwards slot i
// takes slot i + 1's column (i = 1..14) and slot 15 takes slot 1's.  After 15
// rounds every local pair has met once and the slots are back in place.
__device__ __forceinline__ void shift_circle16(Cols& C) {
  float2 g0 = C.g[1][0], g1 = C.g[1][1], v0 = C.v[1][0], v1 = C.v[1][1];
#pragma unroll
  for (int i = 1; i < 15; ++i) move_col(C, i, i + 1);
  C.g[15][0] = g0;
  C.g[15][1] = g1;
  C.v[15][0] = v0;
  C.v[15][1] = v1;
}
// Cross rounds pair top slot k with bottom slot 8 + k; afterwards the bottom
// block rotates by one slot.  After 8 rounds every top/bottom pair has met.
__device__ __forceinline__ void shift_bottom8(Cols& C) {
  float2 g0 = C.g[8][0], g1 = C.g[8][1], v0 = C.v[8][0], v1 = C.v[8][1];
#pragma unroll
  for (int i = 8; i < 15; ++i) move_col(C, i, i + 1);
  C.g[15][0] = g0;
  C.g[15][1] = g1;
  C.v[15][0] = v0;
  C.v[15][1] = v1;
}

// Block exchange between block rounds (circle method over 8 block positions,
// warp s holding positions s (top) and 7 - s (bottom); position 0 fixed).
__device__ __forceinline__ void store_block(const Cols& C, int half, float2* xg, float2* xv,
                                            int slot, int lane) {
#pragma unroll
  for (int c = 0; c < kBlk; ++c)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      xg[(slot * kBlk + c) * 64 + lane + 32 * h] = C.g[half * kBlk + c][h];
      xv[(slot * kBlk + c) * 64 + lane + 32 * h] = C.v[half * kBlk + c][h];
    }
}
__device__ __forceinline__ void load_block(Cols& C, int half, const float2* xg, const float2* xv,
                                           int slot, int lane) {
#pragma unroll
  for (int c = 0; c < kBlk; ++c)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      C.g[half * kBlk + c][h] = xg[(slot * kBlk + c) * 64 + lane + 32 * h];
      C.v[half * kBlk + c][h] = xv[(slot * kBlk + c) * 64 + lane + 32 * h];
    }
}
// slot index of (warp, half) where half 0 = top, 1 = bottom
__device__ __forceinline__ int slot_of(int w, int half) { return 2 * w + half; }

__device__ __forceinline__ void exchange(Cols& C, float2* xg, float2* xv, int warp, int lane) {
  // senders
  if (warp == 0) {
    store_block(C, 1, xg, xv, slot_of(1, 1), lane);
  } else if (warp == 1) {
    store_block(C, 0, xg, xv, slot_of(0, 1), lane);
    store_block(C, 1, xg, xv, slot_of(2, 1), lane);
  } else if (warp == 2) {
    store_block(C, 0, xg, xv, slot_of(1, 0), lane);
    store_block(C, 1, xg, xv, slot_of(3, 1), lane);
  } else {
    store_block(C, 0, xg, xv, slot_of(2, 0), lane);
  }
  __syncthreads();
  if (warp == 0) {
    load_block(C, 1, xg, xv, slot_of(0, 1), lane);
  } else if (warp == 1) {
    load_block(C, 0, xg, xv, slot_of(1, 0), lane);
    load_block(C, 1, xg, xv, slot_of(1, 1), lane);
  } else if (warp == 2) {
    load_block(C, 0, xg, xv, slot_of(2, 0), lane);
    load_block(C, 1, xg, xv, slot_of(2, 1), lane);
  } else {
#pragma unroll
    for (int c = 0; c < kBlk; ++c)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        C.g[c][h] = C.g[kBlk + c][h];
        C.v[c][h] = C.v[kBlk + c][h];
      }
    load_block(C, 1, xg, xv, slot_of(3, 1), lane);
  }
  __syncthreads();
}

template <bool kF64>
__global__ void __launch_bounds__(kThreads, 2)
gsvd_jacobi_kernel(const float2* __restrict__ R, const float2* __restrict__ Kinv, int B, int M,
                   int max_sweeps, float tol, float abs_tol, float* __restrict__ sigma,
                   float2* __restrict__ E, int32_t* __restrict__ status,
                   int32_t* __restrict__ stats, unsigned* flags) {
  extern __shared__ float2 xbuf[];  // 2 x [8 slots][8 cols][64 rows] (64 KB)
  float2* xg = xbuf;
  float2* xv = xbuf + 8 * kBlk * 64;
  __shared__ SmemJ S;

  const int b = blockIdx.x, k = blockIdx.y;
  const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
  const size_t mat = ((size_t)k * B + b) * M * M;

  if (tid == 0) {
    S.bad = 0;
    S.rot_count = 0;
  }
  // ---- A = K^{-1} R: stage K^{-1} and R (dense row-major) in xbuf ----
  {
    float2* Ks = xg;
    float2* Rs = xv;
    const float2* Kb = Kinv + (size_t)b * M * M;
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
    // G = A^H, column-major in xg: column i of G = conj(row i of A).
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int i = ti + 8 * a, j = tj + 16 * c;
        xg[i * 64 + j] = (i < M && j < M) ? make_float2(acc[a][c].x, -acc[a][c].y)
                                          : make_float2(0.f, 0.f);
      }
    __syncthreads();
  }

  // ---- load the warp's 16 columns: top block = position warp, bottom = 7 - warp
  Cols C;
#pragma unroll
  for (int half = 0; half < 2; ++half) {
    const int blk = half == 0 ? warp : 7 - warp;
#pragma unroll
    for (int c = 0; c < kBlk; ++c) {
      const int col = blk * kBlk + c;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int row = lane + 32 * h;
        C.g[half * kBlk + c][h] = xg[col * 64 + row];
        C.v[half * kBlk + c][h] = make_float2(row == col && col < M ? 1.f : 0.f, 0.f);
      }
    }
  }
  __syncthreads();

  int sweeps = 0, rotations = 0, wrot = 0;
  bool converged = S.bad != 0;
  for (int sw = 0; sw < max_sweeps && !converged; ++sw) {
    // global maximum column norm^2 for the absolute criterion
    float abs_thr = 0.f;
    if (abs_tol > 0.f) {
      float x[32];
#pragma unroll
      for (int c = 0; c < kCols; ++c) {
        x[c] = fmaf(C.g[c][0].x, C.g[c][0].x, fmaf(C.g[c][0].y, C.g[c][0].y,
               fmaf(C.g[c][1].x, C.g[c][1].x, C.g[c][1].y * C.g[c][1].y)));
        x[16 + c] = 0.f;
      }
      float n2 = transpose_reduce32(x, lane);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) n2 = fmaxf(n2, __shfl_xor_sync(kFull, n2, o));
      if (lane == 0) S.colnorm[warp] = n2;
      __syncthreads();
      const float amax = fmaxf(fmaxf(S.colnorm[0], S.colnorm[1]),
                               fmaxf(S.colnorm[2], S.colnorm[3]));
      abs_thr = abs_tol * amax;
      __syncthreads();
    }
    // block round 0: all pairs among the warp's 16 columns
#pragma unroll 1
    for (int r = 0; r < 15; ++r) {
      inner_round<kF64, 15, -1>(C, S, warp, lane, tol, abs_thr, wrot);
      shift_circle16(C);
    }
    // block rounds 1..6: pairs across the two blocks, after a block exchange
#pragma unroll 1
    for (int br = 1; br < 7; ++br) {
      exchange(C, xg, xv, warp, lane);
#pragma unroll 1
      for (int k0 = 0; k0 < 8; ++k0) {
        inner_round<kF64, 8, 1>(C, S, warp, lane, tol, abs_thr, wrot);
        shift_bottom8(C);
      }
    }
    if (lane == 0 && wrot != 0) atomicAdd(&S.rot_count, wrot);
    wrot = 0;
    exchange(C, xg, xv, warp, lane);  // back to the starting positions
    ++sweeps;
    const int rc = S.rot_count;
    rotations += rc;
    converged = (rc == 0);
    __syncthreads();
    if (tid == 0) S.rot_count = 0;
  }

  // ---- renormalise V's columns (unit singular vectors) ----
  {
    float x[32];
#pragma unroll
    for (int c = 0; c < kCols; ++c) {
      x[c] = fmaf(C.v[c][0].x, C.v[c][0].x, fmaf(C.v[c][0].y, C.v[c][0].y,
             fmaf(C.v[c][1].x, C.v[c][1].x, C.v[c][1].y * C.v[c][1].y)));
      x[16 + c] = 0.f;
    }
    const float r = transpose_reduce32(x, lane);
    // lane c (< 16) holds |v_c|^2; broadcast and scale
#pragma unroll
    for (int c = 0; c < kCols; ++c) {
      const float n2 = __shfl_sync(kFull, r, c);
      const float inv = n2 > 0.f ? __frsqrt_rn(n2) : 1.f;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        C.v[c][h].x *= inv;
        C.v[c][h].y *= inv;
      }
    }
  }
  // ---- column norms (singular values) and padding detection ----
  {
    float x[32];
#pragma unroll
    for (int c = 0; c < kCols; ++c) {
      x[c] = fmaf(C.g[c][0].x, C.g[c][0].x, fmaf(C.g[c][0].y, C.g[c][0].y,
             fmaf(C.g[c][1].x, C.g[c][1].x, C.g[c][1].y * C.g[c][1].y)));
      float pm = 0.f;
#pragma unroll
      for (int h = 0; h < 2; ++h)
        if (lane + 32 * h >= M) pm = fmaf(C.v[c][h].x, C.v[c][h].x, fmaf(C.v[c][h].y, C.v[c][h].y, pm));
      x[16 + c] = pm;
    }
    const float r = transpose_reduce32(x, lane);
    if (lane < 16)
      S.colnorm[warp * kCols + lane] = r;
    else
      S.padmass[warp * kCols + lane - 16] = r;
  }
  __syncthreads();
  if (tid < 64) S.sig[tid] = S.padmass[tid] > 0.5f ? -1.f : sqrtf(S.colnorm[tid]);
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
  // stage E (row-major M x M) in xbuf, then copy out coalesced
  float2* Es = xbuf;
#pragma unroll
  for (int c = 0; c < kCols; ++c) {
    const int gc = warp * kCols + c;
    const int rk = S.rnk[gc];
    if (rk < M) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int row = lane + 32 * h;
        if (row < M) Es[row * M + rk] = C.v[c][h];
      }
    }
  }
  __syncthreads();
  for (int e = tid; e < M * M; e += kThreads) E[mat + e] = Es[e];
  if (tid < 64 && S.rnk[tid] < M) sigma[((size_t)k * B + b) * M + S.rnk[tid]] = S.sig[tid];
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
                        int32_t* stats, unsigned* flags, cudaStream_t s) {
  const size_t smem = 2 * 8 * kBlk * 64 * sizeof(float2);
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
                                                           flags);
  } else {
    e = cudaFuncSetAttribute(gsvd_jacobi_kernel<false>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    gsvd_jacobi_kernel<false><<<grid, kThreads, smem, s>>>(R, Kinv, B, M, o.max_sweeps, tol,
                                                            abs_tol, sigma, E, status, stats,
                                                            flags);
  }
  return cudaGetLastError();
}

}  // namespace ssl
