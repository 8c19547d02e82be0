// Generalised SVD of eq. 4 by the paper's own route (Sec. III-B, SVD1-SVD6 of
// Alg. 1): Householder bidiagonalisation, phase transform to a real
// bidiagonal, implicit QR (Golub-Kahan) with the tolerance taken from the
// global maximum of the bidiagonal's column sums, sort, back-transformation.
// The paper runs it with one thread per bin; here one CTA of 128 threads owns
// a (bin, block) and everything stays in shared memory (six CTAs per SM):
//
//  1. A = K^{-1} R in FP32, two passes of 32 columns (K^{-1} through L1, R
//     staged in shared memory), each written over its own columns of R.
//  2. For k = 0..M-1: a left reflector H_k = I - beta v v^H zeroes A[k+1:, k],
//     then a right reflector zeroes A[k, k+2:].  Every thread forms the
//     reflector's scalars from per-warp partial sums of the squared norm that
//     the previous update left behind; a thread pair per trailing column (row)
//     applies it.  Two CTA barriers per step.  The left vectors v_k stay in
//     the lower part of A; the right ones are not kept (E_r is not used
//     downstream).
//  3. Phase transform: diagonal unitary scalings make the complex bidiagonal
//     real and non-negative; the tolerance (SVD2) comes out of the same
//     serial pass.
//  4. Q = H_0 ... H_{M-1} (the back-transformation, SVD6) formed in place over
//     the stored reflectors by backward accumulation, one barrier per step,
//     its columns scaled by the left phases.  The QR rotations then act on Q
//     directly, so E needs no transformation after the sort.
//  5. Implicit-shift QR on the real bidiagonal (SVD4: Wilkinson shift,
//     deflation of |e_i| or |d_i| <= tolerance, zero-diagonal chase): one
//     lane chases each bulge and records its left rotations; three warps
//     apply them to the rows of Q while the next bulge is chased.
//  6. Singular values |d_i| sorted descending (SVD5), E's columns
//     (sign-corrected) written in that order.
// With `retry` set, a CTA whose (bin, block) status is not kSplitRetry exits
// at once: the split decomposition hands its unresolved matrices to this
// route that way, and the hardware hands the grid's slots to the marked ones
// as the others leave.
#include <float.h>

#include "ssl_internal.cuh"

namespace ssl {
namespace {

constexpr int kThreads = 128;
constexpr int kMax = SSL_MAX_M;
constexpr int kBLD = kMax + 1;

struct SmemB {
  float2 dc[kMax];   // complex bidiagonal: diagonal
  float2 fc[kMax];   // and superdiagonal
  float beta[kMax];  // left reflector scale
  float2 p[kMax];    // left phases
  float d[kMax];     // real bidiagonal
  float e[kMax];
  // double buffer of left rotations (c, s): chase i fills rot[i & 1].
  // kind 0 (chase from r0): rotation q acts on columns (a, b) = (r0 + q,
  // r0 + q + 1); kind 1 (zero-diagonal sweep of r0): on (r0 + 1 + q, r0).
  // Columns a, b become c U_a + s U_b and -s U_a + c U_b.
  float2 rot[2][kMax];
  int nrot[2];       // rotations in rot[b]; -1: converged, -2: iteration limit
  int kind[2];
  int r0[2];
  float2 F[2][kMax];  // H_k e_k for the backward accumulation of Q
  float p1[4], p2[4];  // per-warp partial sums of squared norms
  float thr;         // deflation threshold
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

// 1 / sqrt(t) for t in the normal range: the hardware estimate refined by one
// Newton-Raphson step (about an ulp).
__device__ __forceinline__ float rsqrt_nr(float t) {
  const float r0 = rsqrtf(t);
  const float h = t * r0;
  return fmaf(0.5f * r0, fmaf(-h, r0, 1.f), r0);
}

// c, s, r with [c s; -s c] [a; b] = [r; 0].  1/r is the hardware estimate of
// 1/sqrt(a^2 + b^2) refined by one Newton-Raphson step, so that c^2 + s^2 = 1
// to about an ulp (the rotations accumulate into E).  a^2 + b^2 outside
// [1e-36, 1e36] (or not finite, or zero) takes the careful path: inputs
// scaled by an exact power of two, b = 0 giving the identity.
__device__ __forceinline__ void givens(float a, float b, float& c, float& s, float& r) {
  const float t = fmaf(a, a, b * b);
  if (t >= 1e-36f && t <= 1e36f) {
    const float r0 = rsqrtf(t);
    const float h = t * r0;
    const float ir = fmaf(0.5f * r0, fmaf(-h, r0, 1.f), r0);
    c = a * ir;
    s = b * ir;
    r = t * ir;
    return;
  }
  if (b == 0.f) {
    c = 1.f;
    s = 0.f;
    r = a;
    return;
  }
  // 2^-ex with ex the exponent of max(|a|, |b|), at most 126 so that 2^-ex
  // stays normal (a subnormal reads as 2^-127)
  const float m = fmaxf(fabsf(a), fabsf(b));
  const int ex = min(((__float_as_int(m) >> 23) & 0xff) - 127, 126);
  const float sc = __int_as_float((127 - ex) << 23);
  const float as = a * sc, bs = b * sc;
  const float ts = fmaf(as, as, bs * bs);
  const float ir = __frsqrt_rn(ts);
  c = as * ir;
  s = bs * ir;
  r = (ts * ir) / sc;
}

// Householder data for x = (x0, ...) with ss = |x|^2, reduced to alpha e_0:
// v = x + e^{i arg x0} |x| e_0 (v0 returned), beta = 2 / (v^H v)
// = 1 / (|x| (|x| + |x0|)), alpha = -e^{i arg x0} |x|.  x = 0 gives beta = 0.
__device__ __forceinline__ void house_scalars(float ss, float2 x0, float& beta, float2& alpha,
                                              float2& v0) {
  const float nx = sqrtf(ss);
  const float a0 = sqrtf(cabs2(x0));
  if (nx == 0.f) {
    beta = 0.f;
    alpha = make_float2(0.f, 0.f);
    v0 = x0;
    return;
  }
  const float ia0 = a0 > 0.f ? __frcp_rn(a0) : 0.f;
  const float2 ph = a0 > 0.f ? make_float2(x0.x * ia0, x0.y * ia0) : make_float2(1.f, 0.f);
  beta = __frcp_rn(nx * (nx + a0));
  alpha = make_float2(-ph.x * nx, -ph.y * nx);
  v0 = make_float2(x0.x + ph.x * nx, x0.y + ph.y * nx);
}

// K^{-1}[i][m] (the identity when Kb is null); zero outside the matrix
__device__ __forceinline__ float2 kinv_at(const float2* __restrict__ Kb, int i, int m, int n) {
  if (i >= n || m >= n) return make_float2(0.f, 0.f);
  return Kb ? __ldg(Kb + (size_t)i * n + m) : make_float2(i == m ? 1.f : 0.f, 0.f);
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Named CTA barriers (ids 1-4; __syncthreads uses 0): arrive publishes the
// thread's prior shared-memory writes without waiting, sync waits for all.
// The ids are immediates so that the kernel reserves five hardware barriers
// (a register id reserves all sixteen, which caps residency at four CTAs).
template <int ID>
__device__ __forceinline__ void named_sync() {
  asm volatile("bar.sync %0, %1;" ::"n"(ID), "n"(kThreads) : "memory");
}
template <int ID>
__device__ __forceinline__ void named_arrive() {
  asm volatile("bar.arrive %0, %1;" ::"n"(ID), "n"(kThreads) : "memory");
}
// barrier 1 + b (rotations of buffer b ready), 3 + b (buffer b applied)
__device__ __forceinline__ void ready_arrive(int b) { b ? named_arrive<2>() : named_arrive<1>(); }
__device__ __forceinline__ void ready_sync(int b) { b ? named_sync<2>() : named_sync<1>(); }
__device__ __forceinline__ void done_arrive(int b) { b ? named_arrive<4>() : named_arrive<3>(); }
__device__ __forceinline__ void done_sync(int b) { b ? named_sync<4>() : named_sync<3>(); }

// One implicit QR step (or, when zk >= 0 is a zero diagonal in [l, h), the
// chase that rotates e_zk away from the left) on the unreduced block [l, h];
// records the left rotations (S.kind: 0 = chase (k, k + 1), 1 = zero-diagonal
// sweep (j, k0)).  Thread 0 only.  The chase carries the diagonal and
// superdiagonal entries it is about to reuse in registers and loads the two
// it has not touched yet one step ahead.
__device__ void qr_step(SmemB& S, int l, int h, int zk, int bf) {
  float* d = S.d;
  float* e = S.e;
  float2* rot = S.rot[bf];
  int n = 0;
  if (zk >= 0) {
    float x = e[zk];
    e[zk] = 0.f;
    for (int j = zk + 1; j <= h; ++j) {
      float c, s, r;
      givens(d[j], x, c, s, r);
      d[j] = r;
      if (j < h) {
        x = -s * e[j];
        e[j] = c * e[j];
      }
      rot[n++] = make_float2(c, s);
    }
    S.nrot[bf] = n;
    S.kind[bf] = 1;
    S.r0[bf] = zk;
    return;
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
    const bool more = k < h - 1;
    const float ek1 = more ? e[k + 1] : 0.f, dk2 = more ? d[k + 2] : 0.f;
    // The right rotation of columns k, k + 1 is (c1, s1) = (y, z) / r1 and
    // the left one of rows k, k + 1 normalises (c1 dk + s1 ek, s1 dk1).
    // Scaling that pair by r1 leaves the left rotation unchanged, so both
    // reciprocal square roots are taken from the unnormalised products at
    // once (t1 = y^2 + z^2 and n2 = |(y dk + z ek, z dk1)|^2), which halves
    // the dependent chain of the step; 1 / r1 then rescales what the left
    // rotation produces.
    const float t1 = fmaf(y, y, z * z);
    const float y2 = fmaf(y, dk, z * ek), z2 = z * dk1;  // r1 (c1 dk + s1 ek), r1 s1 dk1
    const float n2 = fmaf(y2, y2, z2 * z2);
    float c, s;
    if (t1 >= 1e-36f && t1 <= 1e36f && n2 >= 1e-36f && n2 <= 1e36f) {
      const float ekp = fmaf(y, ek, -z * dk), dk1p = y * dk1;  // r1 (-s1 dk + c1 ek), r1 c1 dk1
      const float ir1 = rsqrt_nr(t1), ir2 = rsqrt_nr(n2);
      if (k > l) e[k - 1] = t1 * ir1;
      c = y2 * ir2;
      s = z2 * ir2;
      const float g = ir2 * ir1;
      d[k] = n2 * g;
      y = fmaf(y2, ekp, z2 * dk1p) * g;
      dk = fmaf(y2, dk1p, -z2 * ekp) * g;
    } else {  // magnitudes near the FP32 range: the scaled Givens helper
      float r;
      givens(y, z, c, s, r);  // right rotation of columns k, k + 1
      if (k > l) e[k - 1] = r;
      y = c * dk + s * ek;
      const float ekp = -s * dk + c * ek;
      z = s * dk1;
      const float dk1p = c * dk1;
      givens(y, z, c, s, r);  // left rotation of rows k, k + 1
      d[k] = r;
      y = c * ekp + s * dk1p;
      dk = -s * ekp + c * dk1p;
    }
    if (more) {
      z = s * ek1;
      ek = c * ek1;
      dk1 = dk2;
    }
    rot[n++] = make_float2(c, s);
  }
  d[h] = dk;
  e[h - 1] = y;
  S.nrot[bf] = n;
  S.kind[bf] = 0;
  S.r0[bf] = l;
}

__global__ void __launch_bounds__(kThreads, 6)
gsvd_bidiag_kernel(const float2* __restrict__ R, const float2* __restrict__ Kinv, int B, int M,
                   int max_iter, float eps, float* __restrict__ sigma, float2* __restrict__ E,
                   int32_t* __restrict__ status, int32_t* __restrict__ stats, unsigned* flags,
                   const float2* const* __restrict__ kinv_items,
                   const GsvdProblem* __restrict__ probs, const ImgOut io, int retry) {
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
    E_out = E ? E + item * M * M : nullptr;
    st_out = status ? status + item : nullptr;
    stats_out = stats ? stats + item * 2 : nullptr;
    // (every thread reads the same word: the whole CTA leaves or stays; the
    // word is rewritten only at the end, after every thread's barriers)
    if (retry && *st_out != kSplitRetry) return;
  }
  const int n = M;
  if (tid == 0) {
    S.bad = 0;
    S.iters = 0;
    S.steps = 0;
    S.nrot[0] = S.nrot[1] = 0;
  }

  // ---- 1. A = K^{-1} R (K^{-1} = I when Kb is null) ----
  // Column j of A depends only on column j of R, so A is formed in two passes
  // of 32 columns, each written over its own columns of R once every thread
  // has read them.  The threads holding column 0 also leave the partial sums
  // of |A[i][0]|^2 for the first left reflector.
  for (int e = tid; e < n * n; e += kThreads) As[(e / n) * kBLD + e % n] = Rb[e];
  __syncthreads();
  {
    const int ti = tid / 8, tj = tid % 8;  // rows ti + 16a, columns J0 + tj + 8c
    const bool vec = Kb && (n & 1) == 0 && (reinterpret_cast<uintptr_t>(Kb) & 15) == 0;
    bool finite = true;
    float c0 = 0.f;
    if (!Kb) {  // K^{-1} = I: A = R as staged
      for (int e = tid; e < n * n; e += kThreads) {
        const float2 v = As[(e / n) * kBLD + e % n];
        finite &= isfinite(v.x) && isfinite(v.y);
      }
      for (int i = tid; i < n; i += kThreads) c0 += cabs2(As[i * kBLD]);
    }
    for (int J0 = 0; Kb && J0 < n; J0 += 32) {
      float2 acc[4][4];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[a][c] = make_float2(0.f, 0.f);
      if (vec) {
        // two K^{-1} columns per 16-byte load (n even, rows 16-byte aligned)
        for (int m = 0; m < n; m += 2) {
          float4 kv[4];
          float2 rv0[4], rv1[4];
#pragma unroll
          for (int a = 0; a < 4; ++a) {
            const int i = ti + 16 * a;
            kv[a] = i < n ? __ldg(reinterpret_cast<const float4*>(Kb + (size_t)i * n + m))
                          : make_float4(0.f, 0.f, 0.f, 0.f);
          }
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            const int j = J0 + tj + 8 * c;
            rv0[c] = j < n ? As[m * kBLD + j] : make_float2(0.f, 0.f);
            rv1[c] = j < n ? As[(m + 1) * kBLD + j] : make_float2(0.f, 0.f);
          }
#pragma unroll
          for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int c = 0; c < 4; ++c) {
              float2 t = acc[a][c];
              t.x = fmaf(kv[a].x, rv0[c].x, fmaf(-kv[a].y, rv0[c].y, t.x));
              t.y = fmaf(kv[a].x, rv0[c].y, fmaf(kv[a].y, rv0[c].x, t.y));
              t.x = fmaf(kv[a].z, rv1[c].x, fmaf(-kv[a].w, rv1[c].y, t.x));
              t.y = fmaf(kv[a].z, rv1[c].y, fmaf(kv[a].w, rv1[c].x, t.y));
              acc[a][c] = t;
            }
        }
      } else {
        for (int m = 0; m < n; ++m) {
          float2 kv[4], rv[4];
#pragma unroll
          for (int a = 0; a < 4; ++a) kv[a] = kinv_at(Kb, ti + 16 * a, m, n);
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            const int j = J0 + tj + 8 * c;
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
      }
      __syncthreads();  // columns J0 .. J0 + 31 of R are read
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const int i = ti + 16 * a, j = J0 + tj + 8 * c;
          if (i < n && j < n) {
            finite &= isfinite(acc[a][c].x) && isfinite(acc[a][c].y);
            As[i * kBLD + j] = acc[a][c];
            if (j == 0) c0 += cabs2(acc[a][c]);
          }
        }
    }
    if (!finite) atomicExch(&S.bad, 1);
    c0 = warp_sum(c0);
    if (lane == 0) S.p2[warp] = c0;
    __syncthreads();
  }

  // ---- 2. bidiagonalisation ----
  // Step k: every thread forms the left reflector of column k from the
  // partial sums of |A[k:, k]|^2, a thread pair per column j > k applies it
  // and stores the conjugated new row-k entry (the right reflector's vector)
  // with its |.|^2; after one barrier every thread forms the right reflector,
  // a thread pair per row i > k applies it and leaves |A[i][k + 1]|^2 for the
  // next step.  Two barriers per step.  The thread pairs are (lane,
  // lane + 16) of a warp, index pq, splitting their elements by parity: each
  // half-warp then touches 16 consecutive columns of one row (or rows of one
  // column) per access, 16 distinct 8-byte bank pairs.
  const int pq = warp * 16 + (lane & 15), half = lane >> 4;
  for (int k = 0; k < n; ++k) {
    float beta;
    float2 alpha, v0;
    house_scalars(S.p2[0] + S.p2[1] + S.p2[2] + S.p2[3], As[k * kBLD + k], beta, alpha, v0);
    if (tid == 0) {
      S.beta[k] = beta;
      S.dc[k] = alpha;
    }
    if (k + 1 == n) {
      __syncthreads();  // every thread has read A[k][k]
      if (tid == 0) As[k * kBLD + k] = v0;
      break;
    }
    float r1 = 0.f;
    {
      // H_k on column j: v = (v0, A[k+1:, k]); half 0 takes rows k, k+2, ...
      const int j = k + 1 + pq;
      const bool act = j < n;
      float2 s0 = make_float2(0.f, 0.f), s1 = make_float2(0.f, 0.f), akj = s0;
      if (act) {
        if (half == 0) {
          akj = As[k * kBLD + j];
          s0.x = fmaf(v0.x, akj.x, v0.y * akj.y);
          s0.y = fmaf(v0.x, akj.y, -v0.y * akj.x);
        }
        int i = k + 2 - half;
        for (; i + 2 < n; i += 4) {
          const float2 va = As[i * kBLD + k], aa = As[i * kBLD + j];
          const float2 vb = As[(i + 2) * kBLD + k], ab = As[(i + 2) * kBLD + j];
          s0.x = fmaf(va.x, aa.x, fmaf(va.y, aa.y, s0.x));
          s0.y = fmaf(va.x, aa.y, fmaf(-va.y, aa.x, s0.y));
          s1.x = fmaf(vb.x, ab.x, fmaf(vb.y, ab.y, s1.x));
          s1.y = fmaf(vb.x, ab.y, fmaf(-vb.y, ab.x, s1.y));
        }
        if (i < n) {
          const float2 va = As[i * kBLD + k], aa = As[i * kBLD + j];
          s0.x = fmaf(va.x, aa.x, fmaf(va.y, aa.y, s0.x));
          s0.y = fmaf(va.x, aa.y, fmaf(-va.y, aa.x, s0.y));
        }
      }
      float2 s = make_float2(s0.x + s1.x, s0.y + s1.y);
      s.x += __shfl_xor_sync(0xffffffffu, s.x, 16);
      s.y += __shfl_xor_sync(0xffffffffu, s.y, 16);
      if (act) {
        s.x *= beta;
        s.y *= beta;
#pragma unroll 4
        for (int i = k + 2 - half; i < n; i += 2) {
          const float2 v = As[i * kBLD + k];
          float2 a = As[i * kBLD + j];
          a.x -= v.x * s.x - v.y * s.y;
          a.y -= v.x * s.y + v.y * s.x;
          As[i * kBLD + j] = a;
        }
        if (half == 0) {
          akj.x -= v0.x * s.x - v0.y * s.y;
          akj.y -= v0.x * s.y + v0.y * s.x;
          As[k * kBLD + j] = cconj(akj);
          r1 = cabs2(akj);
        }
      }
    }
    r1 = warp_sum(r1);
    if (lane == 0) S.p1[warp] = r1;
    __syncthreads();
    if (tid == 0) As[k * kBLD + k] = v0;  // reflector head, read again only by step 4
    float wbeta;
    float2 walpha, w0;
    house_scalars(S.p1[0] + S.p1[1] + S.p1[2] + S.p1[3], As[k * kBLD + k + 1], wbeta, walpha,
                  w0);
    if (tid == 0) S.fc[k] = cconj(walpha);  // A[k][k+1] after the right reflector
    float r2 = 0.f;
    {
      // A[i, k+1:] -= wbeta (A[i, k+1:] w) w^H, w = (w0, row k of As from
      // column k + 2); half 0 takes columns k + 1, k + 3, ...
      const int i = k + 1 + pq;
      const bool act = i < n;
      const float2* w = As + k * kBLD;
      float2 s0 = make_float2(0.f, 0.f), s1 = make_float2(0.f, 0.f), aik = s0;
      if (act) {
        if (half == 0) {
          aik = As[i * kBLD + k + 1];
          s0.x = fmaf(aik.x, w0.x, -aik.y * w0.y);
          s0.y = fmaf(aik.x, w0.y, aik.y * w0.x);
        }
        int j = k + 3 - half;
        for (; j + 2 < n; j += 4) {
          const float2 a0 = As[i * kBLD + j], wa = w[j];
          const float2 a1 = As[i * kBLD + j + 2], wb = w[j + 2];
          s0.x = fmaf(a0.x, wa.x, fmaf(-a0.y, wa.y, s0.x));
          s0.y = fmaf(a0.x, wa.y, fmaf(a0.y, wa.x, s0.y));
          s1.x = fmaf(a1.x, wb.x, fmaf(-a1.y, wb.y, s1.x));
          s1.y = fmaf(a1.x, wb.y, fmaf(a1.y, wb.x, s1.y));
        }
        if (j < n) {
          const float2 a0 = As[i * kBLD + j], wa = w[j];
          s0.x = fmaf(a0.x, wa.x, fmaf(-a0.y, wa.y, s0.x));
          s0.y = fmaf(a0.x, wa.y, fmaf(a0.y, wa.x, s0.y));
        }
      }
      float2 s = make_float2(s0.x + s1.x, s0.y + s1.y);
      s.x += __shfl_xor_sync(0xffffffffu, s.x, 16);
      s.y += __shfl_xor_sync(0xffffffffu, s.y, 16);
      if (act) {
        s.x *= wbeta;
        s.y *= wbeta;
#pragma unroll 4
        for (int j = k + 3 - half; j < n; j += 2) {
          const float2 ww = w[j];
          float2 a = As[i * kBLD + j];
          a.x -= s.x * ww.x + s.y * ww.y;  // a -= s conj(w)
          a.y -= s.y * ww.x - s.x * ww.y;
          As[i * kBLD + j] = a;
        }
        if (half == 0) {
          aik.x -= s.x * w0.x + s.y * w0.y;
          aik.y -= s.y * w0.x - s.x * w0.y;
          As[i * kBLD + k + 1] = aik;
          r2 = cabs2(aik);
        }
      }
    }
    r2 = warp_sum(r2);
    if (lane == 0) S.p2[warp] = r2;
    __syncthreads();
  }

  // ---- 3. phase transform (serial) and the tolerance (SVD2) ----
  // The tolerance is eps times the largest column sum |d_i| + |e_{i-1}| of
  // the real bidiagonal (e_{i-1} is the off-diagonal entry of column i).
  if (tid == 0) {
    float2 q = make_float2(1.f, 0.f);
    float anorm = 0.f, eprev = 0.f;
    for (int i = 0; i < n; ++i) {
      const float2 di = cmul(S.dc[i], q);
      const float ad = sqrtf(cabs2(di));
      S.p[i] = ad > 0.f ? make_float2(di.x / ad, -di.y / ad) : make_float2(1.f, 0.f);
      S.d[i] = ad;
      anorm = fmaxf(anorm, ad + eprev);
      if (i + 1 < n) {
        const float2 fi = cmul(S.p[i], S.fc[i]);
        const float af = sqrtf(cabs2(fi));
        q = af > 0.f ? make_float2(fi.x / af, -fi.y / af) : make_float2(1.f, 0.f);
        S.e[i] = af;
        eprev = af;
      }
    }
    S.thr = eps * anorm;
    // H_{n-1} e_{n-1}, the last column of Q before the backward loop
    const float2 vl = As[(n - 1) * kBLD + n - 1];
    S.F[(n - 1) & 1][n - 1] = make_float2(1.f - S.beta[n - 1] * cabs2(vl), 0.f);
  }
  __syncthreads();

  // ---- 4. Q = H_0 ... H_{n-1}, in place, backward; columns times conj(p) ----
  // Step k applies H_k to columns j > k (rows > k; row k of these columns is
  // zero before H_k).  Column k + 1 enters as H_{k+1} e_{k+1}, which the
  // threads of rows >= k + 1 wrote into F[(k + 1) & 1] during the previous
  // step (its reflector is still being read then); one barrier per step.
  for (int k = n - 2; k >= 0; --k) {
    const float beta = S.beta[k];
    const float2 v0 = As[k * kBLD + k];
    {
      const int j = k + 1 + pq;
      const bool act = j < n;
      const bool fresh = j == k + 1;
      const float2* src = fresh ? S.F[(k + 1) & 1] : As + j;  // row i at src[i * ss]
      const int ss = fresh ? 1 : kBLD;
      float2 s0 = make_float2(0.f, 0.f), s1 = make_float2(0.f, 0.f);
      int i = k + 1 + half;
      if (act) {
        for (; i + 2 < n; i += 4) {
          const float2 va = As[i * kBLD + k], qa = src[i * ss];
          const float2 vb = As[(i + 2) * kBLD + k], qb = src[(i + 2) * ss];
          s0.x = fmaf(va.x, qa.x, fmaf(va.y, qa.y, s0.x));
          s0.y = fmaf(va.x, qa.y, fmaf(-va.y, qa.x, s0.y));
          s1.x = fmaf(vb.x, qb.x, fmaf(vb.y, qb.y, s1.x));
          s1.y = fmaf(vb.x, qb.y, fmaf(-vb.y, qb.x, s1.y));
        }
        if (i < n) {
          const float2 va = As[i * kBLD + k], qa = src[i * ss];
          s0.x = fmaf(va.x, qa.x, fmaf(va.y, qa.y, s0.x));
          s0.y = fmaf(va.x, qa.y, fmaf(-va.y, qa.x, s0.y));
        }
      }
      float2 s = make_float2(s0.x + s1.x, s0.y + s1.y);
      s.x += __shfl_xor_sync(0xffffffffu, s.x, 16);
      s.y += __shfl_xor_sync(0xffffffffu, s.y, 16);
      if (act) {
        s.x *= beta;
        s.y *= beta;
#pragma unroll 4
        for (int i = k + 1 + half; i < n; i += 2) {
          const float2 v = As[i * kBLD + k];
          float2 q = src[i * ss];
          q.x -= v.x * s.x - v.y * s.y;
          q.y -= v.x * s.y + v.y * s.x;
          As[i * kBLD + j] = q;
        }
        if (half == 0)
          As[k * kBLD + j] = make_float2(-(v0.x * s.x - v0.y * s.y), -(v0.x * s.y + v0.y * s.x));
      }
    }
    // H_k e_k: 1 - beta |v0|^2 at row k, -beta v_i conj(v0) below
    if (tid >= k && tid < n) {
      float2 val;
      if (tid == k) {
        val = make_float2(1.f - beta * cabs2(v0), 0.f);
      } else {
        const float2 v = As[tid * kBLD + k];
        val = make_float2(-beta * (v.x * v0.x + v.y * v0.y), -beta * (v.y * v0.x - v.x * v0.y));
      }
      S.F[k & 1][tid] = val;
    }
    __syncthreads();
  }
  // column 0 from F[0]; every column times conj(p)
  for (int e = tid; e < n * n; e += kThreads) {
    const int i = e / n, j = e % n;
    const float2 q = j == 0 ? S.F[0][i] : As[i * kBLD + j];
    As[i * kBLD + j] = cmul(q, cconj(S.p[j]));
  }
  __syncthreads();

  // ---- 5. implicit QR on the real bidiagonal ----
  const float thr = S.thr;
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
        if (it >= 2) done_sync(bf);
        int done = 0;
        if (it >= max_iter) done = -2;
        unsigned long long nz = 0ull, zd = 0ull;
#pragma unroll
        for (int hh = 0; hh < 2; ++hh) {
          const int i = lane + 32 * hh;
          bool zero = false;
          if (i < n) {
            const float di = S.d[i];
            zero = fabsf(di) <= thr;
            if (zero && di != 0.f) S.d[i] = 0.f;
          }
          zd |= (unsigned long long)__ballot_sync(0xffffffffu, zero) << (32 * hh);
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
            // first zero diagonal in [l, h), if any
            const unsigned long long zr = zd & ((1ull << h) - 1ull) & ~((1ull << l) - 1ull);
            qr_step(S, l, h, zr ? __ffsll((long long)zr) - 1 : -1, bf);
            S.iters++;
            S.steps += S.nrot[bf];
          }
        }
        __syncwarp();
        ready_arrive(bf);
        if (done != 0) break;
      }
      if (it >= 1) done_sync((it - 1) & 1);  // last buffer applied
    } else {
      const int r = tid - 32;  // this thread's row of Q
      for (int it = 0;; ++it) {
        const int bf = it & 1;
        ready_sync(bf);
        const int nr = S.nrot[bf];
        if (nr < 0) break;
        if (r < n) {
          float2* row = As + r * kBLD;
          const float2* rot = S.rot[bf];
          const int k0 = S.r0[bf];
          if (S.kind[bf] == 0) {  // chase: the entry carried along is U[r][k + 1]
            int k = k0;
            float2 x = row[k];
#pragma unroll 4
            for (int q = 0; q < nr; ++q) {
              const float2 cs = rot[q];
              const float2 xb = row[k + 1];
              row[k] = make_float2(cs.x * x.x + cs.y * xb.x, cs.x * x.y + cs.y * xb.y);
              x = make_float2(-cs.y * x.x + cs.x * xb.x, -cs.y * x.y + cs.x * xb.y);
              ++k;
            }
            row[k] = x;
          } else {  // zero-diagonal sweep: U[r][k0] carried along
            float2 xk = row[k0];
            for (int q = 0; q < nr; ++q) {
              const float2 cs = rot[q];
              const int a = k0 + 1 + q;
              const float2 xa = row[a];
              row[a] = make_float2(cs.x * xa.x + cs.y * xk.x, cs.x * xa.y + cs.y * xk.y);
              xk = make_float2(-cs.y * xa.x + cs.x * xk.x, -cs.y * xa.y + cs.x * xk.y);
            }
            row[k0] = xk;
          }
        }
        done_arrive(bf);
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
  if (E_out)
    for (int e = tid; e < n * n; e += kThreads) {
      const int row = e / n, rk = e % n;
      const int c = S.inv[rk];
      float2 v = As[row * kBLD + c];
      if (S.d[c] < 0.f) v = make_float2(-v.x, -v.y);
      E_out[e] = v;
    }
  // the spectrum's operand image, from E's columns directly (a problem list
  // carries its own image per problem)
  const ImgOut pio = probs ? ImgOut{probs[blockIdx.x].img, probs[blockIdx.x].esz,
                                    probs[blockIdx.x].Ns, probs[blockIdx.x].KP,
                                    probs[blockIdx.x].NP, nullptr}
                           : io;
  if (pio.img)
    write_noise_image(
        pio, probs ? 0 : (size_t)blockIdx.y * B + blockIdx.x, n,
        [&](int row, int rk) {
          const int c = S.inv[rk];
          const float2 v = As[row * kBLD + c];
          return S.d[c] < 0.f ? make_float2(-v.x, -v.y) : v;
        },
        tid, kThreads);
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
                               int n_probs, const ImgOut* iop, bool retry) {
  // rows of the working matrix: M, or the largest size for a problem table
  const size_t smem = (size_t)(M > 0 ? M : kMax) * kBLD * sizeof(float2);
  cudaError_t e = cudaFuncSetAttribute(gsvd_bidiag_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  // the largest shared-memory carveout, so that the register limit (six
  // CTAs per SM) and not the carveout bounds residency at M <= 60
  e = cudaFuncSetAttribute(gsvd_bidiag_kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                           cudaSharedmemCarveoutMaxShared);
  if (e != cudaSuccess) return e;
  // the paper's tolerance from the global maximum: abs_tol, else FP32 epsilon
  const float eps = o.abs_tol > 0.f ? o.abs_tol : 1.1920928955078125e-7f;
  const int max_iter = (o.max_sweeps > 0 ? o.max_sweeps : 30) * SSL_MAX_M;
  if (retry && (probs || !status)) return cudaErrorInvalidValue;
  const dim3 grid = probs ? dim3(n_probs) : dim3(B, nblk);
  if (grid.x == 0 || grid.y == 0) return cudaSuccess;
  gsvd_bidiag_kernel<<<grid, kThreads, smem, s>>>(R, Kinv, B, M, max_iter, eps, sigma, E, status,
                                                   stats, flags, kinv_items, probs,
                                                   iop ? *iop : ImgOut{nullptr, 0, 0, 0, 0},
                                                   retry ? 1 : 0);
  return cudaGetLastError();
}

}  // namespace ssl
