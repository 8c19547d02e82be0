// Generalised SVD of eq. 4 by the paper's own route (Sec. III-B, SVD1-SVD6 of
// Alg. 1): Householder bidiagonalisation, phase transform to a real
// bidiagonal, implicit QR (Golub-Kahan) with the tolerance taken from the
// global maximum of the bidiagonal, sort, back-transformation.  The paper
// runs it with one thread per bin; here one CTA of 128 threads owns a
// (bin, block) and everything stays in shared memory:
//
//  1. A = K^{-1} R in FP32 (R staged in shared memory, K^{-1} through L1,
//     32 entries per thread in registers), written over R.
//  2. For k = 0..M-1: a left reflector H_k = I - beta v v^H zeroes A[k+1:, k]
//     (one thread per trailing column applies it), then a right reflector
//     zeroes A[k, k+2:] (one thread per trailing row).  The left vectors v_k
//     stay in the lower part of A; the right ones are not needed (E_r is not
//     used downstream).
//  3. Phase transform: diagonal unitary scalings make the complex bidiagonal
//     real and non-negative (serial, one thread).
//  4. Q = H_0 ... H_{M-1} formed in place over the stored reflectors
//     (backward accumulation), its columns scaled by the left phases.
//  5. Implicit-shift QR on the real bidiagonal (Wilkinson shift, deflation
//     of |e_i| or |d_i| <= eps * max|bidiagonal|, zero-diagonal chase): one
//     thread chases each bulge and records its left rotations; three warps
//     apply them to the rows of Q while the next bulge is chased.
//  6. Singular values |d_i| sorted descending, E's columns (sign-corrected)
//     written in that order.
#include <float.h>

#include "ssl_internal.cuh"

namespace ssl {
namespace {

constexpr int kThreads = 128;
constexpr int kMax = SSL_MAX_M;
constexpr int kBLD = kMax + 1;

struct Rot {
  int a, b;     // columns rotated: U[:, a] = c U_a + s U_b, U[:, b] = -s U_a + c U_b
  float c, s;
};

struct SmemB {
  float2 dc[kMax];   // complex bidiagonal: diagonal
  float2 fc[kMax];   // and superdiagonal
  float beta[kMax];  // left reflector scale
  float2 p[kMax];    // left phases
  float d[kMax];     // real bidiagonal
  float e[kMax];
  Rot rot[2][2 * kMax];  // double buffer: chase i fills rot[i & 1]
  int nrot[2];       // rotations in rot[b]; -1: converged, -2: iteration limit
  int kind[2];       // 0: chase, 1: zero-diagonal sweep
  float wbeta;       // current right reflector scale
  int bad;
  int iters, steps;
  int rnk[kMax];
  int inv[kMax];
};

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ float cabs2(float2 a) { return a.x * a.x + a.y * a.y; }

// c, s, r with [c s; -s c] [a; b] = [r; 0].  1/r is the correctly rounded
// reciprocal square root of a^2 + b^2, so that c^2 + s^2 = 1 to rounding
// without bias (the rotations accumulate into E); inputs far from 1 in
// magnitude are first scaled by an exact power of two.
__device__ __forceinline__ void givens(float a, float b, float& c, float& s, float& r) {
  if (b == 0.f) {
    c = 1.f;
    s = 0.f;
    r = a;
    return;
  }
  const float m = fmaxf(fabsf(a), fabsf(b));
  float sc = 1.f;
  if (m > 1e18f || m < 1e-18f) {
    const int ex = ((__float_as_int(m) >> 23) & 0xff) - 127;  // m normal here
    sc = __int_as_float((127 - ex) << 23);                     // 2^-ex
  }
  const float as = a * sc, bs = b * sc;
  const float t = fmaf(as, as, bs * bs);
  const float ir = __frsqrt_rn(t);
  c = as * ir;
  s = bs * ir;
  r = (t * ir) / sc;
}

// Householder data for x (length n, element i at x[i * stride]) reduced to
// alpha e_0: v = x + e^{i arg x0} |x| e_0 (written back to x[0]),
// beta = 2 / (v^H v) = 1 / (|x| (|x| + |x0|)), alpha = -e^{i arg x0} |x|.
// Warp-wide; lanes read the elements they own.
__device__ __forceinline__ void house_warp(float2* x, int stride, int n, int lane, float& beta,
                                           float2& alpha) {
  float ss = 0.f;
  for (int i = lane; i < n; i += 32) ss += cabs2(x[i * stride]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
  const float nx = sqrtf(ss);
  const float2 x0 = x[0];
  const float a0 = sqrtf(cabs2(x0));
  if (nx == 0.f) {
    beta = 0.f;
    alpha = make_float2(0.f, 0.f);
    return;
  }
  const float ia0 = a0 > 0.f ? __frcp_rn(a0) : 0.f;
  const float2 ph = a0 > 0.f ? make_float2(x0.x * ia0, x0.y * ia0) : make_float2(1.f, 0.f);
  beta = __frcp_rn(nx * (nx + a0));
  alpha = make_float2(-ph.x * nx, -ph.y * nx);
  __syncwarp();
  if (lane == 0) x[0] = make_float2(x0.x + ph.x * nx, x0.y + ph.y * nx);
  __syncwarp();
}

// Named CTA barriers (ids 1-4; __syncthreads uses 0): arrive publishes the
// thread's prior shared-memory writes without waiting, sync waits for all.
__device__ __forceinline__ void named_sync(int id, int n) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}
__device__ __forceinline__ void named_arrive(int id, int n) {
  asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(n) : "memory");
}

// sum over rows i = i0, i0 + 2, ... < n of conj(A[i][kc]) A[i][j], two
// independent accumulators (the row loop is the serial part of a step).
__device__ __forceinline__ float2 dot_conj_col(const float2* As, int kc, int j, int i0, int n) {
  float2 s0 = make_float2(0.f, 0.f), s1 = make_float2(0.f, 0.f);
  int i = i0;
  for (; i + 2 < n; i += 4) {
    const float2 v0 = As[i * kBLD + kc], a0 = As[i * kBLD + j];
    const float2 v1 = As[(i + 2) * kBLD + kc], a1 = As[(i + 2) * kBLD + j];
    s0.x = fmaf(v0.x, a0.x, fmaf(v0.y, a0.y, s0.x));
    s0.y = fmaf(v0.x, a0.y, fmaf(-v0.y, a0.x, s0.y));
    s1.x = fmaf(v1.x, a1.x, fmaf(v1.y, a1.y, s1.x));
    s1.y = fmaf(v1.x, a1.y, fmaf(-v1.y, a1.x, s1.y));
  }
  if (i < n) {
    const float2 v0 = As[i * kBLD + kc], a0 = As[i * kBLD + j];
    s0.x = fmaf(v0.x, a0.x, fmaf(v0.y, a0.y, s0.x));
    s0.y = fmaf(v0.x, a0.y, fmaf(-v0.y, a0.x, s0.y));
  }
  return make_float2(s0.x + s1.x, s0.y + s1.y);
}

// One implicit QR step (or a zero-diagonal chase) on the unreduced block
// [l, h]; records the left rotations (S.kind: 0 = chase (k, k + 1),
// 1 = zero-diagonal sweep (j, k0)).  Thread 0 only.  The chase carries the
// diagonal and superdiagonal entries it is about to reuse in registers, so
// each step loads only the two entries it has not touched yet.
__device__ void qr_step(SmemB& S, int l, int h, int bf) {
  float* d = S.d;
  float* e = S.e;
  Rot* rot = S.rot[bf];
  int n = 0;
  for (int k = l; k < h; ++k) {
    if (d[k] == 0.f) {  // zero diagonal: rotate e_k away from the left
      float x = e[k];
      e[k] = 0.f;
      for (int j = k + 1; j <= h; ++j) {
        float c, s, r;
        givens(d[j], x, c, s, r);
        d[j] = r;
        if (j < h) {
          x = -s * e[j];
          e[j] = c * e[j];
        }
        rot[n++] = Rot{j, k, c, s};
      }
      S.nrot[bf] = n;
      S.kind[bf] = 1;
      return;
    }
  }
  // Wilkinson shift from the trailing 2 x 2 of B^T B
  const float dm = d[h - 1], dh = d[h], em = e[h - 1], em1 = h - 1 > l ? e[h - 2] : 0.f;
  const float t11 = dm * dm + em1 * em1, t12 = dm * em, t22 = dh * dh + em * em;
  const float delta = 0.5f * (t11 - t22);
  const float den = delta + copysignf(hypotf(delta, t12), delta != 0.f ? delta : 1.f);
  const float mu = den != 0.f ? t22 - t12 * t12 / den : t22;
  float dk = d[l], ek = e[l], dk1 = d[l + 1];
  float y = dk * dk - mu, z = dk * ek;
  for (int k = l; k < h; ++k) {
    float c, s, r;
    givens(y, z, c, s, r);  // right rotation of columns k, k + 1
    if (k > l) e[k - 1] = r;
    y = c * dk + s * ek;
    const float ekp = -s * dk + c * ek;
    z = s * dk1;
    const float dk1p = c * dk1;
    givens(y, z, c, s, r);  // left rotation of rows k, k + 1
    d[k] = r;
    y = c * ekp + s * dk1p;
    const float dk1pp = -s * ekp + c * dk1p;
    if (k < h - 1) {
      const float ek1 = e[k + 1];
      z = s * ek1;
      ek = c * ek1;
      dk1 = d[k + 2];
    }
    dk = dk1pp;
    rot[n++] = Rot{k, k + 1, c, s};
  }
  d[h] = dk;
  e[h - 1] = y;
  S.nrot[bf] = n;
  S.kind[bf] = 0;
}

__global__ void __launch_bounds__(kThreads, 5)
gsvd_bidiag_kernel(const float2* __restrict__ R, const float2* __restrict__ Kinv, int B, int M,
                   int max_iter, float eps, float* __restrict__ sigma, float2* __restrict__ E,
                   int32_t* __restrict__ status, int32_t* __restrict__ stats, unsigned* flags,
                   const float2* const* __restrict__ kinv_items,
                   const GsvdProblem* __restrict__ probs) {
  extern __shared__ float2 As[];  // [M][kBLD]
  __shared__ SmemB S;
  const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
  const float2* Rb;
  const float2* Kb;
  float* sig_out;
  float2* E_out;
  int32_t* st_out;
  int32_t* stats_out = nullptr;
  if (probs) {
    const GsvdProblem& p = probs[blockIdx.x];
    Rb = p.R;
    Kb = p.Kinv;
    sig_out = p.sig;
    E_out = p.E;
    st_out = p.status;
    M = p.M;
  } else {
    const int b = blockIdx.x, k = blockIdx.y;
    const size_t item = (size_t)k * B + b;
    Rb = R + item * M * M;
    Kb = kinv_items ? kinv_items[k] + (size_t)b * M * M
                    : Kinv ? Kinv + (size_t)b * M * M : nullptr;
    sig_out = sigma + item * M;
    E_out = E + item * M * M;
    st_out = status ? status + item : nullptr;
    stats_out = stats ? stats + item * 2 : nullptr;
  }
  const int n = M;
  if (tid == 0) {
    S.bad = 0;
    S.iters = 0;
    S.steps = 0;
    S.nrot[0] = S.nrot[1] = 0;
  }

  // ---- 1. A = K^{-1} R (K^{-1} = I when Kb is null) ----
  for (int e = tid; e < n * n; e += kThreads) As[(e / n) * kBLD + e % n] = Rb[e];
  __syncthreads();
  {
    // rows ti + 8a (a < 8), columns tj + 16c (c < 4), in two passes of four
    // row groups so that 16 complex accumulators live at a time; results are
    // kept until every thread has read R, then written over it
    const int ti = tid / 16, tj = tid % 16;
    float2 res[2][4][4];
#pragma unroll
    for (int pass = 0; pass < 2; ++pass) {
      float2 acc[4][4];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[a][c] = make_float2(0.f, 0.f);
      for (int m = 0; m < n; ++m) {
        float2 kv[4], rv[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) {
          const int i = ti + 8 * (a + 4 * pass);
          kv[a] = i >= n ? make_float2(0.f, 0.f)
                         : Kb ? __ldg(Kb + (size_t)i * n + m)
                              : make_float2(i == m ? 1.f : 0.f, 0.f);
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const int j = tj + 16 * c;
          rv[c] = j < n ? As[m * kBLD + j] : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            acc[a][c].x = fmaf(kv[a].x, rv[c].x, fmaf(-kv[a].y, rv[c].y, acc[a][c].x));
            acc[a][c].y = fmaf(kv[a].x, rv[c].y, fmaf(kv[a].y, rv[c].x, acc[a][c].y));
          }
      }
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < 4; ++c) res[pass][a][c] = acc[a][c];
    }
    bool finite = true;
#pragma unroll
    for (int pass = 0; pass < 2; ++pass)
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < 4; ++c)
          finite &= isfinite(res[pass][a][c].x) && isfinite(res[pass][a][c].y);
    if (!finite) atomicExch(&S.bad, 1);
    __syncthreads();
#pragma unroll
    for (int pass = 0; pass < 2; ++pass)
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const int i = ti + 8 * (a + 4 * pass), j = tj + 16 * c;
          if (i < n && j < n) As[i * kBLD + j] = res[pass][a][c];
        }
    __syncthreads();
  }

  // ---- 2. bidiagonalisation ----
  for (int k = 0; k < n; ++k) {
    if (warp == 0) {  // left reflector of column k
      float beta;
      float2 alpha;
      house_warp(As + k * kBLD + k, kBLD, n - k, lane, beta, alpha);
      if (lane == 0) {
        S.beta[k] = beta;
        S.dc[k] = alpha;
      }
    }
    __syncthreads();
    {
      // apply H_k to column j: a thread pair per column, rows split by parity
      const int j = k + 1 + (tid >> 1), half = tid & 1;
      const float beta = S.beta[k];
      const bool act = j < n && beta != 0.f;
      float2 s = dot_conj_col(As, k, j, k + half, act ? n : 0);
      s.x += __shfl_xor_sync(0xffffffffu, s.x, 1);
      s.y += __shfl_xor_sync(0xffffffffu, s.y, 1);
      if (act) {
        s.x *= beta;
        s.y *= beta;
        for (int i = k + half; i < n; i += 2) {
          const float2 v = As[i * kBLD + k];
          float2 a = As[i * kBLD + j];
          a.x -= v.x * s.x - v.y * s.y;
          a.y -= v.x * s.y + v.y * s.x;
          As[i * kBLD + j] = a;
        }
      }
    }
    __syncthreads();
    if (k + 1 >= n) break;
    if (warp == 0) {  // right reflector of row k: w from conj(A[k, k+1:])
      float2* row = As + k * kBLD + k + 1;
      for (int j = lane; j < n - k - 1; j += 32) row[j] = cconj(row[j]);
      __syncwarp();
      float beta;
      float2 alpha;
      house_warp(row, 1, n - k - 1, lane, beta, alpha);
      if (lane == 0) {
        S.wbeta = beta;
        S.fc[k] = cconj(alpha);  // A[k][k+1] after the right reflector
      }
    }
    __syncthreads();
    {
      // A[i, k+1:] -= beta (A[i, k+1:] w) w^H: a thread pair per row, columns
      // split by parity
      const int i = k + 1 + (tid >> 1), half = tid & 1;
      const float beta = S.wbeta;
      const bool act = i < n && beta != 0.f;
      const float2* w = As + k * kBLD;
      float2 s0 = make_float2(0.f, 0.f), s1 = make_float2(0.f, 0.f);
      if (act) {
        int j = k + 1 + half;
        for (; j + 2 < n; j += 4) {
          const float2 a0 = As[i * kBLD + j], w0 = w[j];
          const float2 a1 = As[i * kBLD + j + 2], w1 = w[j + 2];
          s0.x = fmaf(a0.x, w0.x, fmaf(-a0.y, w0.y, s0.x));
          s0.y = fmaf(a0.x, w0.y, fmaf(a0.y, w0.x, s0.y));
          s1.x = fmaf(a1.x, w1.x, fmaf(-a1.y, w1.y, s1.x));
          s1.y = fmaf(a1.x, w1.y, fmaf(a1.y, w1.x, s1.y));
        }
        if (j < n) {
          const float2 a0 = As[i * kBLD + j], w0 = w[j];
          s0.x = fmaf(a0.x, w0.x, fmaf(-a0.y, w0.y, s0.x));
          s0.y = fmaf(a0.x, w0.y, fmaf(a0.y, w0.x, s0.y));
        }
      }
      float2 s = make_float2(s0.x + s1.x, s0.y + s1.y);
      s.x += __shfl_xor_sync(0xffffffffu, s.x, 1);
      s.y += __shfl_xor_sync(0xffffffffu, s.y, 1);
      if (act) {
        s.x *= beta;
        s.y *= beta;
        for (int j = k + 1 + half; j < n; j += 2) {
          const float2 ww = w[j];
          float2 a = As[i * kBLD + j];
          // a -= s conj(w)
          a.x -= s.x * ww.x + s.y * ww.y;
          a.y -= s.y * ww.x - s.x * ww.y;
          As[i * kBLD + j] = a;
        }
      }
    }
    __syncthreads();
  }

  // ---- 3. phase transform (serial) ----
  if (tid == 0) {
    float2 q = make_float2(1.f, 0.f);
    for (int i = 0; i < n; ++i) {
      const float2 di = cmul(S.dc[i], q);
      const float ad = sqrtf(cabs2(di));
      S.p[i] = ad > 0.f ? make_float2(di.x / ad, -di.y / ad) : make_float2(1.f, 0.f);
      S.d[i] = ad;
      if (i + 1 < n) {
        const float2 fi = cmul(S.p[i], S.fc[i]);
        const float af = sqrtf(cabs2(fi));
        q = af > 0.f ? make_float2(fi.x / af, -fi.y / af) : make_float2(1.f, 0.f);
        S.e[i] = af;
      }
    }
  }
  __syncthreads();

  // ---- 4. Q = H_0 ... H_{n-1}, in place, backward; columns times conj(p) ----
  for (int k = n - 1; k >= 0; --k) {
    const float beta = S.beta[k];
    {
      // columns to the right, rows > k: a thread pair per column, rows split
      // by parity (row k of these columns is zero before H_k)
      const int j = k + 1 + (tid >> 1), half = tid & 1;
      const bool act = j < n;
      float2 s = dot_conj_col(As, k, j, k + 1 + half, act ? n : 0);
      s.x += __shfl_xor_sync(0xffffffffu, s.x, 1);
      s.y += __shfl_xor_sync(0xffffffffu, s.y, 1);
      if (act) {
        s.x *= beta;
        s.y *= beta;
        for (int i = k + 1 + half; i < n; i += 2) {
          const float2 v = As[i * kBLD + k];
          float2 q = As[i * kBLD + j];
          q.x -= v.x * s.x - v.y * s.y;
          q.y -= v.x * s.y + v.y * s.x;
          As[i * kBLD + j] = q;
        }
        const float2 v0 = As[k * kBLD + k];  // row k of column j was 0
        if (half == 0)
          As[k * kBLD + j] = make_float2(-(v0.x * s.x - v0.y * s.y), -(v0.x * s.y + v0.y * s.x));
      }
    }
    __syncthreads();
    {
      // column k = H_k e_k: 1 - beta |v0|^2 at row k, -beta v_i conj(v0) below
      const float2 v0 = As[k * kBLD + k];
      float2 val = make_float2(0.f, 0.f);
      const int i = tid;
      if (i < n) {
        if (i == k)
          val = make_float2(1.f - beta * cabs2(v0), 0.f);
        else if (i > k) {
          const float2 v = As[i * kBLD + k];
          val = make_float2(-beta * (v.x * v0.x + v.y * v0.y), -beta * (v.y * v0.x - v.x * v0.y));
        }
      }
      __syncthreads();
      if (i < n) As[i * kBLD + k] = val;
    }
    __syncthreads();
  }
  for (int e = tid; e < n * n; e += kThreads) {
    const int i = e / n, j = e % n;
    const float2 ph = cconj(S.p[j]);
    As[i * kBLD + j] = cmul(As[i * kBLD + j], ph);
  }
  __syncthreads();

  // ---- 5. implicit QR on the real bidiagonal ----
  float thr = 0.f;
  if (tid == 0) {
    float bmax = 0.f;
    for (int i = 0; i < n; ++i) bmax = fmaxf(bmax, fabsf(S.d[i]));
    for (int i = 0; i + 1 < n; ++i) bmax = fmaxf(bmax, fabsf(S.e[i]));
    S.wbeta = eps * bmax;
  }
  __syncthreads();
  thr = S.wbeta;
  // Warp 0 finds the bottom unreduced block and chases its bulge (lane 0),
  // recording the left rotations in rot[it & 1]; warps 1-3 apply them to the
  // rows of Q while warp 0 already chases the next one.  Named barriers
  // 1 + b (rotations b ready) and 3 + b (rotations b applied) hand the two
  // buffers back and forth.
  bool converged = S.bad != 0;
  if (!converged) {
    if (warp == 0) {
      int it = 0;
      for (;; ++it) {
        const int bf = it & 1;
        if (it >= 2) named_sync(3 + bf, kThreads);
        int done = 0;
        if (it >= max_iter) done = -2;
        unsigned long long nz = 0ull;
#pragma unroll
        for (int hh = 0; hh < 2; ++hh) {
          const int i = lane + 32 * hh;
          if (i < n && fabsf(S.d[i]) <= thr && S.d[i] != 0.f) S.d[i] = 0.f;
          bool live = false;
          if (i + 1 < n) {
            const float ei = S.e[i];
            if (fabsf(ei) <= thr) {
              if (ei != 0.f) S.e[i] = 0.f;
            } else {
              live = true;
            }
          }
          nz |= (unsigned long long)__ballot_sync(0xffffffffu, live) << (32 * hh);
        }
        __syncwarp();
        if (nz == 0ull) done = -1;
        if (lane == 0) {
          if (done != 0) {
            S.nrot[bf] = done;
          } else {
            // bottom unreduced block [l, h]: e_{h-1} is the highest live
            // entry, e_{l-1} the highest dead one below it
            const int h = 64 - __clzll(nz);
            const unsigned long long below = ~nz & ((1ull << (h - 1)) - 1ull);
            const int l = below ? 64 - __clzll(below) : 0;
            qr_step(S, l, h, bf);
            S.iters++;
            S.steps += S.nrot[bf];
          }
        }
        __syncwarp();
        named_arrive(1 + bf, kThreads);
        if (done != 0) break;
      }
      if (it >= 1) named_sync(3 + ((it - 1) & 1), kThreads);  // last buffer applied
    } else {
      const int r = tid - 32;  // this thread's row of Q
      for (int it = 0;; ++it) {
        const int bf = it & 1;
        named_sync(1 + bf, kThreads);
        const int nr = S.nrot[bf];
        if (nr < 0) break;
        if (r < n) {
          float2* row = As + r * kBLD;
          const Rot* rot = S.rot[bf];
          if (S.kind[bf] == 0) {  // chase: the entry carried along is U[r][k + 1]
            int k = rot[0].a;
            float2 x = row[k];
            for (int q = 0; q < nr; ++q) {
              const Rot rr = rot[q];
              const float2 xb = row[k + 1];
              row[k] = make_float2(rr.c * x.x + rr.s * xb.x, rr.c * x.y + rr.s * xb.y);
              x = make_float2(-rr.s * x.x + rr.c * xb.x, -rr.s * x.y + rr.c * xb.y);
              ++k;
            }
            row[k] = x;
          } else {  // zero-diagonal sweep: U[r][k0] carried along
            const int k0 = rot[0].b;
            float2 xk = row[k0];
            for (int q = 0; q < nr; ++q) {
              const Rot rr = rot[q];
              const float2 xa = row[rr.a];
              row[rr.a] = make_float2(rr.c * xa.x + rr.s * xk.x, rr.c * xa.y + rr.s * xk.y);
              xk = make_float2(-rr.s * xa.x + rr.c * xk.x, -rr.s * xa.y + rr.c * xk.y);
            }
            row[k0] = xk;
          }
        }
        named_arrive(3 + bf, kThreads);
      }
    }
    __syncthreads();
    converged = S.nrot[0] == -1 || S.nrot[1] == -1;
  }

  // ---- 6. sort, write ----
  if (tid < n) {
    // ranks by |d|, ties by column; a NaN (non-finite input) ranks last so
    // the ranks stay a permutation and every index derived from them stays
    // in range
    const float v = fabsf(S.d[tid]), vk = v == v ? v : -1.f;
    int rk = 0;
    for (int c = 0; c < n; ++c) {
      const float w0 = fabsf(S.d[c]), w = w0 == w0 ? w0 : -1.f;
      rk += (w > vk) || (w == vk && c < tid);
    }
    S.rnk[tid] = rk;
    S.inv[rk] = tid;
    sig_out[rk] = v;
  }
  __syncthreads();
  for (int e = tid; e < n * n; e += kThreads) {
    const int row = e / n, rk = e % n;
    const int c = S.inv[rk];
    float2 v = As[row * kBLD + c];
    if (S.d[c] < 0.f) v = make_float2(-v.x, -v.y);
    E_out[e] = v;
  }
  if (tid == 0) {
    int st = 0;
    if (S.bad != 0)
      st = SSL_E_NONFINITE;
    else if (!converged)
      st = SSL_E_NO_CONVERGENCE;
    if (st_out) *st_out = st;
    if (stats_out) {
      stats_out[0] = S.iters;
      stats_out[1] = S.steps;
    }
    if (st == SSL_E_NONFINITE) atomicOr(flags, SSL_FLAG_NONFINITE);
    if (st == SSL_E_NO_CONVERGENCE) atomicOr(flags, SSL_FLAG_NO_CONVERGENCE);
  }
}

}  // namespace

cudaError_t launch_gsvd_bidiag(const float2* R, const float2* Kinv, int nblk, int B, int M,
                               const JacobiOpts& o, float* sigma, float2* E, int32_t* status,
                               int32_t* stats, unsigned* flags, cudaStream_t s,
                               const float2* const* kinv_items, const GsvdProblem* probs,
                               int n_probs) {
  const size_t smem = (size_t)kMax * kBLD * sizeof(float2);
  cudaError_t e = cudaFuncSetAttribute(gsvd_bidiag_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  // the paper's tolerance from the global maximum: abs_tol, else FP32 epsilon
  const float eps = o.abs_tol > 0.f ? o.abs_tol : 1.1920928955078125e-7f;
  const int max_iter = (o.max_sweeps > 0 ? o.max_sweeps : 30) * SSL_MAX_M;
  const dim3 grid = probs ? dim3(n_probs) : dim3(B, nblk);
  if (grid.x == 0 || grid.y == 0) return cudaSuccess;
  gsvd_bidiag_kernel<<<grid, kThreads, smem, s>>>(R, Kinv, B, M, max_iter, eps, sigma, E, status,
                                                   stats, flags, kinv_items, probs);
  return cudaGetLastError();
}

}  // namespace ssl
