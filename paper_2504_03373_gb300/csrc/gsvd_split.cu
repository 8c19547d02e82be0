// The noise subspace of eq. 4 for the SQ form of eq. 5 (Sec. III-A), by a
// split one-sided Jacobi iteration.
//
// The SQ spectrum depends on E_n only through the projector
// E_n E_n^H = I - E_s E_s^H, E_s the Ns left singular vectors of
// A = K^{-1} R with the largest singular values.  This kernel finds that
// dominant subspace and an orthonormal basis of its complement, without the
// individual noise vectors:
//
//  1. A = K^{-1} R by columns (from the whitening GEMM, or formed here).  A
//     group of kSplitLanes lanes per matrix (lane l holds rows l, l + LG,
//     ...; one or two matrices per warp).  Every column passes an insertion network of Ns register
//     slots, the pivots, kept in descending order of squared norm; the column
//     that drops out goes to the next partner slot in shared memory.
//  2. One-sided Jacobi on A's columns restricted to pivot-partner pairs: in
//     round j pivot i meets partner slot (i + j) mod (M - Ns), and after every
//     16 such rounds the pivots meet each other (circle order).  A pair is
//     rotated under the same tests and with the same angle arithmetic as the
//     full iteration; a partner larger than its pivot is exchanged with it
//     after the rotation, so that the pivots only gain norm.  At the fixed
//     point every other column of A V is orthogonal to every pivot:
//     span(pivots) is the dominant left singular subspace, and with the pivot
//     pairs converged the pivots are sigma_s E_s.
//  3. Angles in FP64 (or FP32): the lanes that hold a pair's reduced sums
//     evaluate its rotation; an FP64 warp instruction occupies a
//     sub-partition's FP64 unit for ~64 cycles whether 1 or 32 lanes are
//     active, so with 16 lanes per matrix the two matrices of a warp share
//     each one.  A matrix stops
//     once M - Ns consecutive rounds have changed nothing.
//  4. E_s = pivots / |pivots|, sorted by norm.  The Householder QR of E_s
//     gives Q = H_0 ... H_{Ns-1} = I - V T V^H (compact WY form); its
//     trailing M - Ns columns are the noise basis:
//       E_n[r][c] = delta_rc - sum_b W[r][b] conj(V[c][b]),   W = V T.
// A matrix still rotating after the sweep limit, or one the batched test
// shows the rounds would not finish (below), is marked kSplitRetry and solved
// again by the paper's bidiagonalisation route in its retry mode; a matrix the
// split does not apply to (split_applies) takes the full one-sided Jacobi.
#include <float.h>

#include "jacobi_rot.cuh"
#include "ssl_internal.cuh"

namespace ssl {
namespace {

using namespace jrot;

constexpr int kSplitBlk = 16;     // pivot-partner rounds between pivot-pair passes
constexpr int kSplitMaxWarps = 8; // warps per CTA
constexpr int kSplitSweeps = 8;   // sweeps of M - Ns rounds before the retry
constexpr float kSplitHopeless = 0.5f;  // partner / pivot energy that goes to the retry at once
constexpr float kSplitHopelessCoupling = 1e-5f;  // squared pair coupling that does too
constexpr size_t kSplitSmemMax = 227u * 1024u;

struct SplitArgs {
  const float2* R;
  const float2* Acm;  // A = K^{-1} R by columns ([item][c][r]), or null: formed here
  const float2* Kinv;
  const float2* const* kinv_items;
  int n_items, B, M, Ns, cap_rounds;
  float tol, abs_tol, sqrt_abs_tol;
  float* sigma;
  float2* E;
  int32_t* status;
  int32_t* stats;
  unsigned* flags;
  ImgOut io;
};

__host__ __device__ constexpr size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

// Shared memory of one CTA of nm matrices: partner columns, then per matrix
// the rotation slots of a round, the WY factor T and the partner norms.
struct SplitLayout {
  size_t g, ang, t, pn, total;
  __host__ __device__ SplitLayout(int nm, int M, int Ns, int NSP) {
    g = 0;
    ang = align16((size_t)nm * (M - Ns) * M * sizeof(float2));
    t = ang + (size_t)nm * NSP * sizeof(float4);
    pn = t + (size_t)nm * NSP * NSP * sizeof(float2);
    total = pn + (size_t)nm * 64 * sizeof(float);
  }
};

// Circle order over n (even) players, round u: pair 0 = (u, n - 1), pair k
// = ((u + k) mod (n - 1), (u - k) mod (n - 1)).
__host__ __device__ constexpr int circ_a(int n, int u, int k) { return k == 0 ? u : (u + k) % (n - 1); }
__host__ __device__ constexpr int circ_b(int n, int u, int k) {
  return k == 0 ? n - 1 : (u - k + n - 1) % (n - 1);
}

// Sum over the LG lanes of a matrix's lane group (the same value on each).
template <int LG>
__device__ __forceinline__ float group_sum(float v) {
#pragma unroll
  for (int o = LG / 2; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

// Transposing butterfly over the LG lanes of a group: 16 values per lane in,
// the group-wide sum of value v out on lane v * VS of the group (VS = 2 for
// LG = 32: lanes 2v and 2v + 1; VS = 1 for LG = 16: lane v).
template <int LG>
__device__ __forceinline__ float group_transpose16(float (&x)[16], int lane) {
  if (LG == 32) return transpose_reduce16(x, lane);
#pragma unroll
  for (int w = 8, n = 8; w >= 1; w >>= 1, n >>= 1) {
    const bool hi = (lane & w) != 0;
#pragma unroll
    for (int k = 0; k < n; ++k) {
      const float send = hi ? x[k] : x[k + n];
      const float keep = hi ? x[k + n] : x[k];
      x[k] = keep + __shfl_xor_sync(kFull, send, w);
    }
  }
  return x[0];
}

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// a * conj(b)
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}


// kF64: FP64 angles.  LG lanes per matrix (32: one matrix per warp; 16: two,
// so that each FP64 warp instruction of a round serves both matrices' pairs).
// RPL rows per lane (M <= LG * RPL).  NSP pivot registers (Ns <= NSP).
// Control flow that contains shuffles is the same for the whole warp; what
// differs between its matrices (their convergence) only gates loads, stores
// and register updates.
template <bool kF64, int LG, int RPL, int NSP>
__global__ void __launch_bounds__(32 * kSplitMaxWarps, 1) gsvd_split_kernel(const SplitArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr int NG = (NSP + 3) / 4;    // groups of four pairs per reduction
  constexpr int NE = NSP + (NSP & 1);  // players of the pivot-pair circle
  constexpr int MPW = 32 / LG;         // matrices per warp
  constexpr int VS = LG == 32 ? 2 : 1; // lane stride of the reduced values
  const int nw = blockDim.x >> 5;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int sub = lane / LG, hl = lane % LG, g0 = sub * LG;
  const int mslot = warp * MPW + sub, nm = nw * MPW;
  const int M = a.M, Ns = a.Ns, nR = M - Ns;
  const SplitLayout L(nm, M, Ns, NSP);
  float2* Gw = reinterpret_cast<float2*>(smem + L.g) + (size_t)mslot * nR * M;
  float4* ang = reinterpret_cast<float4*>(smem + L.ang) + mslot * NSP;
  float2* Tw = reinterpret_cast<float2*>(smem + L.t) + mslot * NSP * NSP;
  float* pnrm = reinterpret_cast<float*>(smem + L.pn) + mslot * 64;

  const int item = blockIdx.x * nm + mslot;
  const bool valid = item < a.n_items;
  const int itm = valid ? item : 0;  // (addresses of an empty slot stay in bounds)
  int row[RPL];
  bool rv[RPL];
#pragma unroll
  for (int h = 0; h < RPL; ++h) {
    row[h] = hl + LG * h;
    rv[h] = row[h] < M;
  }
  const float2 zero = make_float2(0.f, 0.f);

  // ---- 1. the columns of A (from the whitening launch, else A = K^{-1} R
  // formed here: A[r][c] = sum_k conj(K^{-1}[k][r]) R[k][c], K^{-1} Hermitian),
  // 8 at a time; each column passes the pivot network.
  float2 P[NSP][RPL];
  float pk[NSP];  // pivot keys (squared norms), descending; -1: empty
#pragma unroll
  for (int i = 0; i < NSP; ++i) {
    pk[i] = -1.f;
#pragma unroll
    for (int h = 0; h < RPL; ++h) P[i][h] = zero;
  }
  bool bad = false;
  {
    const int k = itm / a.B, b = itm - k * a.B;
    const float2* Rb = a.R + (size_t)itm * M * M;
    const float2* Kb = a.kinv_items ? a.kinv_items[k] + (size_t)b * M * M
                       : a.Kinv     ? a.Kinv + (size_t)b * M * M
                                    : nullptr;
    int nslot = 0;
    for (int c0 = 0; c0 < M; c0 += 8) {
      float2 acc[8][RPL];
#pragma unroll
      for (int cc = 0; cc < 8; ++cc)
#pragma unroll
        for (int h = 0; h < RPL; ++h) acc[cc][h] = zero;
      if (a.Acm) {
        const float2* Ab = a.Acm + (size_t)itm * M * M + (size_t)c0 * M;
#pragma unroll
        for (int cc = 0; cc < 8; ++cc)
#pragma unroll
          for (int h = 0; h < RPL; ++h)
            acc[cc][h] = (valid && rv[h] && c0 + cc < M) ? __ldg(Ab + (size_t)cc * M + row[h])
                                                          : zero;
      } else if (Kb) {
        // (whole 16-byte aligned row segments: M even, 8 columns inside the row)
        const bool vec = (M & 1) == 0 && c0 + 8 <= M &&
                         (reinterpret_cast<uintptr_t>(Rb) & 15) == 0;
#pragma unroll 2
        for (int kk = 0; kk < M; ++kk) {
          float2 kv[RPL];
#pragma unroll
          for (int h = 0; h < RPL; ++h) {
            const float2 t = (valid && rv[h]) ? __ldg(Kb + (size_t)kk * M + row[h]) : zero;
            kv[h] = make_float2(t.x, -t.y);
          }
          const float2* rr = Rb + (size_t)kk * M + c0;
          float2 rv8[8];
          if (vec) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              const float4 t = __ldg(reinterpret_cast<const float4*>(rr) + q);
              rv8[2 * q] = make_float2(t.x, t.y);
              rv8[2 * q + 1] = make_float2(t.z, t.w);
            }
          } else {
#pragma unroll
            for (int cc = 0; cc < 8; ++cc) rv8[cc] = c0 + cc < M ? __ldg(rr + cc) : zero;
          }
#pragma unroll
          for (int cc = 0; cc < 8; ++cc) {
            const float2 r = rv8[cc];
#pragma unroll
            for (int h = 0; h < RPL; ++h) {
              acc[cc][h].x = fmaf(kv[h].x, r.x, fmaf(-kv[h].y, r.y, acc[cc][h].x));
              acc[cc][h].y = fmaf(kv[h].x, r.y, fmaf(kv[h].y, r.x, acc[cc][h].y));
            }
          }
        }
      } else {  // K^{-1} = I
#pragma unroll
        for (int cc = 0; cc < 8; ++cc)
#pragma unroll
          for (int h = 0; h < RPL; ++h)
            acc[cc][h] = (valid && rv[h] && c0 + cc < M)
                             ? __ldg(Rb + (size_t)row[h] * M + c0 + cc)
                             : zero;
      }
#pragma unroll
      for (int cc = 0; cc < 8; ++cc) {
        if (c0 + cc < M) {
          const float n = group_sum<LG>(norm2<RPL>(acc[cc]));  // the same on the group's lanes
          if (!(fabsf(n) <= FLT_MAX)) bad = true;
          float key = n == n ? n : -0.5f;
          float2 col[RPL];
#pragma unroll
          for (int h = 0; h < RPL; ++h) col[h] = acc[cc][h];
#pragma unroll
          for (int i = 0; i < NSP; ++i) {
            if (i < Ns && key > pk[i]) {
#pragma unroll
              for (int h = 0; h < RPL; ++h) {
                const float2 t = P[i][h];
                P[i][h] = col[h];
                col[h] = t;
              }
              const float t = pk[i];
              pk[i] = key;
              key = t;
            }
          }
          if (key > -1.f) {  // a column left the network: next partner slot
            if (valid && SSL_IN_BOUNDS(nslot < nR, a.flags)) {
#pragma unroll
              for (int h = 0; h < RPL; ++h)
                if (rv[h]) Gw[(size_t)nslot * M + row[h]] = col[h];
              if (hl == 0) pnrm[nslot] = key;
            }
            ++nslot;
          }
        }
      }
    }
  }

  // ---- 2. pivot-partner rounds, pivot pairs every kSplitBlk rounds
  int since = 0, rounds = 0, nrot = 0;
  bool done = !valid || bad;
  bool retry = false;
  int j = 0;  // partner offset of the round (the same for the warp's matrices)
  float am_last = pk[0] > 0.f ? pk[0] : 0.f;
  const int blk = nR < kSplitBlk ? nR : kSplitBlk;
  const int own = hl % (4 * VS) == 0 ? hl / (4 * VS) : -1;  // pair (in a group) this lane owns
  // A sweep's worth of tests at once: every pivot-partner pair and every pivot
  // pair against the current columns, under the rounds' own FP32 screen (which
  // lets through every pair the FP64 test could rotate).  A matrix that passes
  // them all is at its fixed point -- the preconditioned input often is -- and
  // skips the rounds.
  {
    float alp[NSP];  // squared pivot norms
    {
      float x[16];
#pragma unroll
      for (int q = 0; q < 16; ++q) x[q] = q < NSP ? norm2<RPL>(P[q < NSP ? q : 0]) : 0.f;
      const float v = group_transpose16<LG>(x, lane);
#pragma unroll
      for (int i = 0; i < NSP; ++i) alp[i] = __shfl_sync(kFull, v, g0 + i * VS);
    }
    float am = 0.f;
#pragma unroll
    for (int i = 0; i < NSP; ++i)
      if (i < Ns) am = fmaxf(am, alp[i]);
    const float2 at2 = make_float2(a.abs_tol * am, a.sqrt_abs_tol * am);
    bool need = false;
    float cpl = 0.f;  // largest squared coupling of a pivot-partner pair the screen lets through
    for (int sl = 0; sl < nR; ++sl) {
      float2 qv[RPL];
#pragma unroll
      for (int h = 0; h < RPL; ++h) qv[h] = rv[h] ? Gw[(size_t)sl * M + row[h]] : zero;
      float x[16];
#pragma unroll
      for (int q = 0; q < 16; ++q) x[q] = 0.f;
#pragma unroll
      for (int i = 0; i < NSP; ++i) dot_partial<RPL>(P[i], qv, x[2 * i], x[2 * i + 1]);
      const float be = group_sum<LG>(norm2<RPL>(qv));
      const float v = group_transpose16<LG>(x, lane);
      const float vi_ = __shfl_down_sync(kFull, v, VS);  // the imaginary part's lane
      const int vix = hl / VS;                            // value this lane holds
      if (hl % VS == 0 && (vix & 1) == 0 && (vix >> 1) < Ns) {
        float al = 0.f;
#pragma unroll
        for (int i = 0; i < NSP; ++i)
          if (i == (vix >> 1)) al = alp[i];
        const bool rot = may_rotate(al, be, v, vi_, a.tol, at2);
        need = need || be > al || rot;
        if (rot && al > 0.f && be > 0.f) {  // |g_s^H g_n|^2 / (|g_s|^2 |g_n|^2)
          const float sc = rsqrtf(al) * rsqrtf(be), cr = v * sc, ci = vi_ * sc;
          cpl = fmaxf(cpl, fmaf(cr, cr, ci * ci));
        }
        if (!done) pnrm[sl] = be;
      }
    }
#pragma unroll
    for (int pp = 0; pp < NSP; ++pp)
#pragma unroll
      for (int qq = pp + 1; qq < NSP; ++qq)
        if (qq < Ns) {
          float gr, gi;
          dot_partial<RPL>(P[pp], P[qq], gr, gi);
          gr = group_sum<LG>(gr);
          gi = group_sum<LG>(gi);
          need = need || may_rotate(alp[pp], alp[qq], gr, gi, a.tol, at2);
        }
    const unsigned bal = __ballot_sync(kFull, need);
    const bool gneed = LG == 32 ? bal != 0u : ((bal >> g0) & 0xffffu) != 0u;
    if (!gneed) done = true;
    __syncwarp();  // (the partner norms written above)
    // The rounds reduce a pivot-partner coupling by about
    // (sigma_{Ns+1} / sigma_Ns)^2 per sweep, and the preconditioner already
    // did several such steps: a matrix whose largest coupling is still above
    // ~3e-3 (or whose largest partner holds more than half the smallest
    // pivot's energy) has sigma_{Ns+1} close to sigma_Ns -- more pivots than
    // sources, say -- and the rounds would not finish within the sweep limit,
    // so it goes to the retry at once.
    // (the reductions run on every lane: the warp's two matrices may differ)
    float amin = FLT_MAX, bmax = 0.f;
#pragma unroll
    for (int i = 0; i < NSP; ++i)
      if (i < Ns) amin = fminf(amin, alp[i]);
    for (int sl = hl; sl < nR; sl += LG) bmax = fmaxf(bmax, pnrm[sl]);
#pragma unroll
    for (int o = LG / 2; o > 0; o >>= 1) {
      bmax = fmaxf(bmax, __shfl_xor_sync(kFull, bmax, o));
      cpl = fmaxf(cpl, __shfl_xor_sync(kFull, cpl, o));
    }
    if (gneed && !done && (bmax > kSplitHopeless * amin || cpl > kSplitHopelessCoupling)) {
      done = true;
      retry = true;
    }
  }
  while (!__all_sync(kFull, done)) {
    bool stop = false;
    for (int t = 0; t < blk; ++t) {
      float2 Q[NSP][RPL];
      float x[NG][16];
#pragma unroll
      for (int g = 0; g < NG; ++g)
#pragma unroll
        for (int q = 0; q < 16; ++q) x[g][q] = 0.f;
#pragma unroll
      for (int i = 0; i < NSP; ++i) {
        int s = i + j;
        if (s >= nR) s -= nR;
#pragma unroll
        for (int h = 0; h < RPL; ++h)
          Q[i][h] = (i < Ns && rv[h]) ? Gw[(size_t)s * M + row[h]] : zero;
        float gr, gi;
        dot_partial<RPL>(P[i], Q[i], gr, gi);
        x[i / 4][4 * (i % 4) + 0] = norm2<RPL>(P[i]);
        x[i / 4][4 * (i % 4) + 1] = norm2<RPL>(Q[i]);
        x[i / 4][4 * (i % 4) + 2] = gr;
        x[i / 4][4 * (i % 4) + 3] = gi;
      }
      // pair 4 g + p's sums (alpha, beta, gamma) on the lane that owns p
      float pv[NG][4];
      float am = 0.f;
#pragma unroll
      for (int g = 0; g < NG; ++g) {
        const float v = group_transpose16<LG>(x[g], lane);
        pv[g][0] = v;
        pv[g][1] = __shfl_down_sync(kFull, v, VS);
        pv[g][2] = __shfl_down_sync(kFull, v, 2 * VS);
        pv[g][3] = __shfl_down_sync(kFull, v, 3 * VS);
        if (own >= 0 && 4 * g + own < Ns) am = fmaxf(am, pv[g][0]);
      }
#pragma unroll
      for (int o = 4 * VS; o < LG; o <<= 1) am = fmaxf(am, __shfl_xor_sync(kFull, am, o));
      if (!done) am_last = am;
      const float2 at2 = make_float2(a.abs_tol * am, a.sqrt_abs_tol * am);
#pragma unroll
      for (int g = 0; g < NG; ++g) {
        const int i = 4 * g + own;
        if (own >= 0 && i < Ns && !done) {
          const float al = pv[g][0], be = pv[g][1], gr = pv[g][2], gi = pv[g][3];
          int s = i + j;
          if (s >= nR) s -= nR;
          pnrm[s] = be;
          float4 o = make_float4(1.f, 0.f, 0.f, 0.f);
          float na, nb;
          int code = rotation<kF64>(al, be, gr, gi, a.tol, at2, o, na, nb) ? 1 : 0;
          if (be > al) code |= 2;  // the partner is the larger: exchange after the rotation
          ang[i] = make_float4(o.x, o.y, o.z, __int_as_float(code));
        }
      }
      __syncwarp();
      if (!done) {
        bool changed = false;
#pragma unroll
        for (int i = 0; i < NSP; ++i) {
          if (i < Ns) {
            const float4 o = ang[i];
            const int code = __float_as_int(o.w);
            if (code != 0) {
              if (code & 1) {
#pragma unroll
                for (int h = 0; h < RPL; ++h) rot1(P[i][h], Q[i][h], o.x, o.y, o.z);
              }
              if (code & 2) {
#pragma unroll
                for (int h = 0; h < RPL; ++h) {
                  const float2 tt = P[i][h];
                  P[i][h] = Q[i][h];
                  Q[i][h] = tt;
                }
              }
              int s = i + j;
              if (s >= nR) s -= nR;
#pragma unroll
              for (int h = 0; h < RPL; ++h)
                if (rv[h]) Gw[(size_t)s * M + row[h]] = Q[i][h];
              changed = true;
              ++nrot;
            }
          }
        }
        since = changed ? 0 : since + 1;
        ++rounds;
        if (since >= nR) {
          done = true;
        } else if (rounds >= a.cap_rounds) {
          done = true;
          retry = true;
        }
      }
      j = j + 1 == nR ? 0 : j + 1;
      __syncwarp();
      if (__all_sync(kFull, done)) {
        stop = true;
        break;
      }
    }
    if (stop) break;
    // pivot pairs in circle order (rounds without a pair of real pivots are skipped)
    if (Ns >= 2) {
#pragma unroll
      for (int u = 0; u < NE - 1; ++u) {
        bool real = false;
#pragma unroll
        for (int k = 0; k < NE / 2; ++k)
          real = real || (circ_a(NE, u, k) < Ns && circ_b(NE, u, k) < Ns);
        if (!real) continue;
        float x[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) x[q] = 0.f;
#pragma unroll
        for (int k = 0; k < NE / 2; ++k) {
          // (register indices clamped; a pair with a dummy player is not used)
          const int pa = min(circ_a(NE, u, k), NSP - 1), pb = min(circ_b(NE, u, k), NSP - 1);
          float gr, gi;
          dot_partial<RPL>(P[pa], P[pb], gr, gi);
          x[4 * k + 0] = norm2<RPL>(P[pa]);
          x[4 * k + 1] = norm2<RPL>(P[pb]);
          x[4 * k + 2] = gr;
          x[4 * k + 3] = gi;
        }
        const float v = group_transpose16<LG>(x, lane);
        const float al = v, be = __shfl_down_sync(kFull, v, VS);
        const float gr = __shfl_down_sync(kFull, v, 2 * VS), gi = __shfl_down_sync(kFull, v, 3 * VS);
        const int k = own;
        if (k >= 0 && k < NE / 2 && circ_a(NE, u, k) < Ns && circ_b(NE, u, k) < Ns && !done) {
          const float2 at2 = make_float2(a.abs_tol * am_last, a.sqrt_abs_tol * am_last);
          float4 o = make_float4(1.f, 0.f, 0.f, 0.f);
          float na, nb;
          const int code = rotation<kF64>(al, be, gr, gi, a.tol, at2, o, na, nb) ? 1 : 0;
          ang[k] = make_float4(o.x, o.y, o.z, __int_as_float(code));
        }
        __syncwarp();
        if (!done) {
#pragma unroll
          for (int kk = 0; kk < NE / 2; ++kk) {
            const int pa = circ_a(NE, u, kk), pb = circ_b(NE, u, kk);
            if (pa < Ns && pb < Ns) {
              const float4 o = ang[kk];
              if (__float_as_int(o.w) & 1) {
                const int qa = min(pa, NSP - 1), qb = min(pb, NSP - 1);
#pragma unroll
                for (int h = 0; h < RPL; ++h) rot1(P[qa][h], P[qb][h], o.x, o.y, o.z);
                since = 0;
                ++nrot;
              }
            }
          }
        }
        __syncwarp();
      }
    }
  }

  // ---- 3. outputs (every lane takes part in the group reductions; only a
  // matrix that converged here writes)
  const bool out = valid && !retry;
  if (valid && retry && hl == 0) a.status[item] = kSplitRetry;
  float al[NSP];  // exact squared pivot norms
  {
    float x[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) x[q] = q < NSP ? norm2<RPL>(P[q < NSP ? q : 0]) : 0.f;
    const float v = group_transpose16<LG>(x, lane);
#pragma unroll
    for (int i = 0; i < NSP; ++i) al[i] = __shfl_sync(kFull, v, g0 + i * VS);
  }
  // ranks (descending; NaN below everything, ties by index: a permutation)
  int rk[NSP];
#pragma unroll
  for (int i = 0; i < NSP; ++i) {
    const float wi = al[i] == al[i] ? al[i] : -0.5f;
    int r = 0;
#pragma unroll
    for (int k = 0; k < NSP; ++k) {
      const float wk = al[k] == al[k] ? al[k] : -0.5f;
      if (k < Ns && k != i) r += (wk > wi) || (wk == wi && k < i);
    }
    rk[i] = r;
    if (i < Ns && !(al[i] <= FLT_MAX)) bad = true;
  }
  float* sg = a.sigma + (size_t)itm * M;
  float2* Eo = a.E ? a.E + (size_t)itm * M * M : nullptr;
  float2 Y[NSP][RPL];  // E_s (pivot order), then the Householder vectors
#pragma unroll
  for (int i = 0; i < NSP; ++i) {
    const float inv = (i < Ns && al[i] > 0.f) ? 1.f / sqrtf(al[i]) : 0.f;
#pragma unroll
    for (int h = 0; h < RPL; ++h) Y[i][h] = make_float2(P[i][h].x * inv, P[i][h].y * inv);
    if (i < Ns && out) {
      if (hl == 0) sg[rk[i]] = sqrtf(fmaxf(al[i], 0.f));
      if (Eo) {
#pragma unroll
        for (int h = 0; h < RPL; ++h)
          if (rv[h]) Eo[(size_t)row[h] * M + rk[i]] = Y[i][h];
      }
    }
  }
  // the other columns' norms, descending, after the pivots
  if (out)
    for (int sl = hl; sl < nR; sl += LG) {
      const float v0 = pnrm[sl], v = v0 == v0 ? v0 : -0.5f;
      int r = 0;
      for (int q = 0; q < nR; ++q) {
        const float w0 = pnrm[q], w = w0 == w0 ? w0 : -0.5f;
        r += (w > v) || (w == v && q < sl);
      }
      if (SSL_IN_BOUNDS(r < nR, a.flags)) sg[Ns + r] = sqrtf(fmaxf(v0, 0.f));
    }
  __syncwarp();
  // Householder QR of E_s: H_i = I - tau_i v_i v_i^H, v_i = x + phase(x_i) |x| e_i
  // with x the rows i.. of column i after H_0 .. H_{i-1}.
  float2* Vw = Gw;                   // v_b in partner slots 0 .. Ns-1
  float2* Ww = Gw + (size_t)Ns * M;  // W = V T in slots Ns .. 2 Ns - 1 (2 Ns <= nR)
  float tau[NSP];
#pragma unroll
  for (int i = 0; i < NSP; ++i) {
    tau[i] = 0.f;
    if (i < Ns) {
#pragma unroll
      for (int h = 0; h < RPL; ++h)
        if (row[h] < i) Y[i][h] = zero;
      const float xn2 = group_sum<LG>(norm2<RPL>(Y[i]));
      const float2 xi = make_float2(__shfl_sync(kFull, Y[i][0].x, g0 + i),
                                    __shfl_sync(kFull, Y[i][0].y, g0 + i));
      const float xn = sqrtf(xn2), ax = sqrtf(fmaf(xi.x, xi.x, xi.y * xi.y));
      const float2 ph = ax > 0.f ? make_float2(xi.x / ax, xi.y / ax) : make_float2(1.f, 0.f);
      if (hl == i) Y[i][0] = make_float2(fmaf(ph.x, xn, Y[i][0].x), fmaf(ph.y, xn, Y[i][0].y));
      tau[i] = xn > 0.f ? 1.f / (xn * (xn + ax)) : 0.f;
#pragma unroll
      for (int k = 0; k < NSP; ++k) {
        if (k > i && k < Ns) {
          float gr, gi;
          dot_partial<RPL>(Y[i], Y[k], gr, gi);
          const float2 d = make_float2(tau[i] * group_sum<LG>(gr), tau[i] * group_sum<LG>(gi));
#pragma unroll
          for (int h = 0; h < RPL; ++h) {
            const float2 t = cmul(d, Y[i][h]);
            Y[k][h] = make_float2(Y[k][h].x - t.x, Y[k][h].y - t.y);
          }
        }
      }
#pragma unroll
      for (int h = 0; h < RPL; ++h)
        if (rv[h]) Vw[(size_t)i * M + row[h]] = Y[i][h];
    }
  }
  // T (upper triangular): T[i][i] = tau_i, T[0:i][i] = -tau_i T[0:i][0:i] (V^H v_i)
#pragma unroll
  for (int i = 0; i < NSP; ++i) {
    if (i < Ns) {
      float2 z[NSP];
#pragma unroll
      for (int b = 0; b < NSP; ++b) {
        z[b] = zero;
        if (b < i) {
          float gr, gi;
          dot_partial<RPL>(Y[b], Y[i], gr, gi);
          z[b] = make_float2(group_sum<LG>(gr), group_sum<LG>(gi));
        }
      }
      if (hl == 0) {
#pragma unroll
        for (int b = 0; b < NSP; ++b) {
          if (b < i) {
            float2 acc = zero;
#pragma unroll
            for (int c = 0; c < NSP; ++c)
              if (c >= b && c < i) {
                const float2 t = cmul(Tw[b * NSP + c], z[c]);
                acc = make_float2(acc.x + t.x, acc.y + t.y);
              }
            Tw[b * NSP + i] = make_float2(-tau[i] * acc.x, -tau[i] * acc.y);
          } else {
            Tw[b * NSP + i] = b == i ? make_float2(tau[i], 0.f) : zero;
          }
        }
      }
      __syncwarp();
    }
  }
  // W = V T (registers and shared memory)
  float2 Wr[NSP][RPL];
#pragma unroll
  for (int b = 0; b < NSP; ++b) {
#pragma unroll
    for (int h = 0; h < RPL; ++h) Wr[b][h] = zero;
    if (b < Ns) {
#pragma unroll
      for (int c = 0; c < NSP; ++c)
        if (c <= b) {
          const float2 t = Tw[c * NSP + b];
#pragma unroll
          for (int h = 0; h < RPL; ++h) {
            const float2 m = cmul(Y[c][h], t);
            Wr[b][h] = make_float2(Wr[b][h].x + m.x, Wr[b][h].y + m.y);
          }
        }
#pragma unroll
      for (int h = 0; h < RPL; ++h)
        if (rv[h]) Ww[(size_t)b * M + row[h]] = Wr[b][h];
    }
  }
  __syncwarp();
  // E_n[r][c] = delta_rc - sum_b W[r][b] conj(V[c][b]), c = Ns .. M-1
  if (out && Eo) {
    for (int c = Ns; c < M; ++c) {
      float2 vc[NSP];
#pragma unroll
      for (int b = 0; b < NSP; ++b) vc[b] = b < Ns ? Vw[(size_t)b * M + c] : zero;
#pragma unroll
      for (int h = 0; h < RPL; ++h) {
        if (rv[h]) {
          float2 e = row[h] == c ? make_float2(1.f, 0.f) : zero;
#pragma unroll
          for (int b = 0; b < NSP; ++b) {
            const float2 t = cmulc(Wr[b][h], vc[b]);
            e = make_float2(e.x - t.x, e.y - t.y);
          }
          Eo[(size_t)row[h] * M + c] = e;
        }
      }
    }
  }
  if (out && a.io.img) {
    // The spectrum's operand image from registers: E_n[r][c] for the lane's
    // own rows r (row 2i of the image: Re E[:, Ns + i] then Im E[:, Ns + i];
    // row 2i + 1: Im, then -Re; zero beyond 2M columns and 2 (M - Ns) rows),
    // element by element so that the group's lanes store consecutive
    // elements; the same values and roundings as write_noise_image.
    const ImgOut& io = a.io;
    const size_t ibytes = (size_t)io.NP * io.KP * io.esz;
    char* base = static_cast<char*>(io.img) + (size_t)item * ibytes;
    char* lo = io.lo ? static_cast<char*>(io.lo) + (size_t)item * ibytes : nullptr;
    auto put = [&](int n, int k, float v) {
      const size_t at = (size_t)n * io.KP + k;
      if (io.esz == 2) {
        reinterpret_cast<__nv_bfloat16*>(base)[at] = __float2bfloat16_rn(v);
      } else {
        uint32_t hb;
        asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(hb) : "f"(v));
        reinterpret_cast<uint32_t*>(base)[at] = hb;
        if (lo) {  // 3xTF32: the rounding residual, itself rounded to TF32
          uint32_t lb;
          asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(lb) : "f"(v - __uint_as_float(hb)));
          reinterpret_cast<uint32_t*>(lo)[at] = lb;
        }
      }
    };
    for (int i = 0; i < nR; ++i) {
      const int c = Ns + i;
      float2 vc[NSP];
#pragma unroll
      for (int b = 0; b < NSP; ++b) vc[b] = b < Ns ? Vw[(size_t)b * M + c] : zero;
#pragma unroll
      for (int h = 0; h < RPL; ++h) {
        if (rv[h]) {
          float2 e = row[h] == c ? make_float2(1.f, 0.f) : zero;
#pragma unroll
          for (int b = 0; b < NSP; ++b) {
            const float2 t = cmulc(Wr[b][h], vc[b]);
            e = make_float2(e.x - t.x, e.y - t.y);
          }
          put(2 * i, row[h], e.x);
          put(2 * i, M + row[h], e.y);
          put(2 * i + 1, row[h], e.y);
          put(2 * i + 1, M + row[h], -e.x);
        }
      }
    }
    for (int n = 0; n < 2 * nR; ++n)
      for (int k = 2 * M + hl; k < io.KP; k += LG) put(n, k, 0.f);
    for (int e = hl; e < (io.NP - 2 * nR) * io.KP; e += LG)
      put(2 * nR + e / io.KP, e % io.KP, 0.f);
  }
  if (out && hl == 0) {
    a.status[item] = bad ? SSL_E_NONFINITE : 0;
    if (bad) atomicOr(a.flags, SSL_FLAG_NONFINITE);
    if (a.stats) {
      a.stats[(size_t)item * 2] = rounds;
      a.stats[(size_t)item * 2 + 1] = nrot;
    }
  }
}

// Lanes per matrix.  32 (one matrix per warp, twice the warps per SM) now
// that the preconditioned matrices settle in the batched test; 16 (two per
// warp, sharing each FP64 warp instruction of a round) was the faster while
// most matrices ran rounds.
constexpr int kSplitLanes = 32;

template <bool kF64, int LG, int RPL, int NSP>
cudaError_t launch_split_t(const SplitArgs& a, cudaStream_t s) {
  constexpr int MPW = 32 / LG;
  // as many matrices as the shared memory takes, whole warps, at most 8 warps
  int nm = kSplitMaxWarps * MPW;
  while (nm > MPW && SplitLayout(nm, a.M, a.Ns, NSP).total > kSplitSmemMax) nm -= MPW;
  const size_t smem = SplitLayout(nm, a.M, a.Ns, NSP).total;
  if (smem > kSplitSmemMax) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(gsvd_split_kernel<kF64, LG, RPL, NSP>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int grid = (a.n_items + nm - 1) / nm;
  gsvd_split_kernel<kF64, LG, RPL, NSP><<<grid, 32 * (nm / MPW), smem, s>>>(a);
  return cudaGetLastError();
}

template <bool kF64, int LG, int RPL>
cudaError_t launch_split_r(const SplitArgs& a, cudaStream_t s) {
  switch (a.Ns) {
    case 1: return launch_split_t<kF64, LG, RPL, 1>(a, s);
    case 2: return launch_split_t<kF64, LG, RPL, 2>(a, s);
    case 3:
    case 4: return launch_split_t<kF64, LG, RPL, 4>(a, s);
    default: return launch_split_t<kF64, LG, RPL, 8>(a, s);
  }
}

// kSplitLanes lanes per matrix, rows per lane by size class.
template <bool kF64>
cudaError_t launch_split_f(const SplitArgs& a, cudaStream_t s) {
  constexpr int LG = kSplitLanes;
  if (a.M <= LG) return launch_split_r<kF64, LG, 1>(a, s);
  if (a.M <= 2 * LG) return launch_split_r<kF64, LG, 2>(a, s);
  return launch_split_r<kF64, LG, 64 / LG>(a, s);
}

}  // namespace

cudaError_t launch_gsvd_split(const float2* R, const float2* Kinv, int nblk, int B, int M,
                              const JacobiOpts& o, float* sigma, float2* E, int32_t* status,
                              int32_t* stats, unsigned* flags, cudaStream_t s,
                              const float2* const* kinv_items, const ImgOut* io, float2* abuf) {
  if (!status || !sigma) return cudaErrorInvalidValue;
  JacobiOpts full = o;
  full.method = SSL_SVD_JACOBI;
  if (!split_applies(M, o.split_ns))
    return launch_gsvd(R, Kinv, nblk, B, M, full, sigma, E, status, stats, flags, s, kinv_items,
                       nullptr, io);
  if (nblk < 1 || B < 1) return cudaSuccess;
  SplitArgs a;
  a.R = R;
  a.Acm = nullptr;
  a.Kinv = Kinv;
  a.kinv_items = kinv_items;
  a.n_items = nblk * B;
  a.B = B;
  a.M = M;
  a.Ns = o.split_ns;
  const int sweeps = o.max_sweeps < 1 ? 1 : (o.max_sweeps < kSplitSweeps ? o.max_sweeps : kSplitSweeps);
  a.cap_rounds = sweeps * (M - o.split_ns);
  a.tol = o.rel_tol > 0.f ? o.rel_tol : (float)M * 5.9604644775390625e-8f;
  a.abs_tol = o.abs_tol > 0.f ? o.abs_tol : 0.f;
  a.sqrt_abs_tol = sqrtf(a.abs_tol);
  a.sigma = sigma;
  a.E = E;
  a.status = status;
  a.stats = stats;
  a.flags = flags;
  a.io = io ? *io : ImgOut{nullptr, 0, 0, 0, 0, nullptr};
  cudaError_t e = cudaSuccess;
  if (abuf && (Kinv || kinv_items)) {  // the whitening product (and preconditioning) first
    e = launch_whiten(R, Kinv, kinv_items, nblk, B, M, o.split_ns, abuf, s);
    if (e != cudaSuccess) return e;
    a.Acm = abuf;
  }
  e = o.angles_f64 ? launch_split_f<true>(a, s) : launch_split_f<false>(a, s);
  if (e != cudaSuccess) return e;
  // the matrices marked kSplitRetry, by the paper's route (on the data that
  // needs it -- noise values on both sides of the split -- it takes about 0.4
  // of the full one-sided Jacobi's time per matrix)
  return launch_gsvd_bidiag(R, Kinv, nblk, B, M, o, sigma, E, status, stats, flags, s, kinv_items,
                            nullptr, 0, io, true);
}

}  // namespace ssl
