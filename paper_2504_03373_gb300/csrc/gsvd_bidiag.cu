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
//     thread chases each bulge and records its left rotations; then every
//     thread applies the recorded rotations to its row of Q.
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
  Rot rot[2 * kMax];
  int nrot;          // rotations in rot[]; < 0: done
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

// c, s, r with [c s; -s c] [a; b] = [r; 0]
__device__ __forceinline__ void givens(float a, float b, float& c, float& s, float& r) {
  if (b == 0.f) {
    c = 1.f;
    s = 0.f;
    r = a;
    return;
  }
  r = hypotf(a, b);
  const float ir = 1.f / r;
  c = a * ir;
  s = b * ir;
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
  const float2 ph = a0 > 0.f ? make_float2(x0.x / a0, x0.y / a0) : make_float2(1.f, 0.f);
  beta = 1.f / (nx * (nx + a0));
  alpha = make_float2(-ph.x * nx, -ph.y * nx);
  __syncwarp();
  if (lane == 0) x[0] = make_float2(x0.x + ph.x * nx, x0.y + ph.y * nx);
  __syncwarp();
}

// One implicit QR step (or a zero-diagonal chase) on the unreduced block
// [l, h]; records the left rotations.  Thread 0 only.
__device__ void qr_step(SmemB& S, int l, int h) {
  float* d = S.d;
  float* e = S.e;
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
        S.rot[n++] = Rot{j, k, c, s};
      }
      S.nrot = n;
      return;
    }
  }
  // Wilkinson shift from the trailing 2 x 2 of B^T B
  const float dm = d[h - 1], dh = d[h], em = e[h - 1], em1 = h - 1 > l ? e[h - 2] : 0.f;
  const float t11 = dm * dm + em1 * em1, t12 = dm * em, t22 = dh * dh + em * em;
  const float delta = 0.5f * (t11 - t22);
  const float den = delta + copysignf(hypotf(delta, t12), delta != 0.f ? delta : 1.f);
  const float mu = den != 0.f ? t22 - t12 * t12 / den : t22;
  float y = d[l] * d[l] - mu, z = d[l] * e[l];
  for (int k = l; k < h; ++k) {
    float c, s, r;
    givens(y, z, c, s, r);  // right rotation of columns k, k + 1
    if (k > l) e[k - 1] = r;
    y = c * d[k] + s * e[k];
    e[k] = -s * d[k] + c * e[k];
    z = s * d[k + 1];
    d[k + 1] = c * d[k + 1];
    givens(y, z, c, s, r);  // left rotation of rows k, k + 1
    d[k] = r;
    y = c * e[k] + s * d[k + 1];
    d[k + 1] = -s * e[k] + c * d[k + 1];
    if (k < h - 1) {
      z = s * e[k + 1];
      e[k + 1] = c * e[k + 1];
    }
    S.rot[n++] = Rot{k, k + 1, c, s};
  }
  e[h - 1] = y;
  S.nrot = n;
}

__global__ void __launch_bounds__(kThreads)
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
  }

  // ---- 1. A = K^{-1} R (K^{-1} = I when Kb is null) ----
  for (int e = tid; e < n * n; e += kThreads) As[(e / n) * kBLD + e % n] = Rb[e];
  __syncthreads();
  {
    const int ti = tid / 16, tj = tid % 16;  // rows ti + 8a, columns tj + 16c
    float2 acc[8][4];
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[a][c] = make_float2(0.f, 0.f);
    for (int m = 0; m < n; ++m) {
      float2 kv[8], rv[4];
#pragma unroll
      for (int a = 0; a < 8; ++a) {
        const int i = ti + 8 * a;
        kv[a] = i >= n ? make_float2(0.f, 0.f)
                       : Kb ? __ldg(Kb + (size_t)i * n + m) : make_float2(i == m ? 1.f : 0.f, 0.f);
      }
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int j = tj + 16 * c;
        rv[c] = j < n ? As[m * kBLD + j] : make_float2(0.f, 0.f);
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
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int i = ti + 8 * a, j = tj + 16 * c;
        if (i < n && j < n) As[i * kBLD + j] = acc[a][c];
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
      const int j = k + 1 + tid;  // apply H_k to column j
      const float beta = S.beta[k];
      if (j < n && beta != 0.f) {
        float2 s = make_float2(0.f, 0.f);
        for (int i = k; i < n; ++i) {
          const float2 v = As[i * kBLD + k], a = As[i * kBLD + j];
          s.x = fmaf(v.x, a.x, fmaf(v.y, a.y, s.x));  // conj(v) a
          s.y = fmaf(v.x, a.y, fmaf(-v.y, a.x, s.y));
        }
        s.x *= beta;
        s.y *= beta;
        for (int i = k; i < n; ++i) {
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
      const int i = k + 1 + tid;  // A[i, k+1:] -= beta (A[i, k+1:] w) w^H
      const float beta = S.wbeta;
      if (i < n && beta != 0.f) {
        const float2* w = As + k * kBLD;
        float2 s = make_float2(0.f, 0.f);
        for (int j = k + 1; j < n; ++j) {
          const float2 a = As[i * kBLD + j], ww = w[j];
          s.x = fmaf(a.x, ww.x, fmaf(-a.y, ww.y, s.x));
          s.y = fmaf(a.x, ww.y, fmaf(a.y, ww.x, s.y));
        }
        s.x *= beta;
        s.y *= beta;
        for (int j = k + 1; j < n; ++j) {
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
      const int j = k + 1 + tid;  // columns to the right: rows >= k
      if (j < n) {
        float2 s = make_float2(0.f, 0.f);
        for (int i = k + 1; i < n; ++i) {
          const float2 v = As[i * kBLD + k], q = As[i * kBLD + j];
          s.x = fmaf(v.x, q.x, fmaf(v.y, q.y, s.x));
          s.y = fmaf(v.x, q.y, fmaf(-v.y, q.x, s.y));
        }
        s.x *= beta;
        s.y *= beta;
        for (int i = k + 1; i < n; ++i) {
          const float2 v = As[i * kBLD + k];
          float2 q = As[i * kBLD + j];
          q.x -= v.x * s.x - v.y * s.y;
          q.y -= v.x * s.y + v.y * s.x;
          As[i * kBLD + j] = q;
        }
        const float2 v0 = As[k * kBLD + k];  // row k of column j was 0
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
  bool converged = S.bad != 0;
  for (int it = 0; it < max_iter && !converged; ++it) {
    if (tid == 0) {
      float* d = S.d;
      float* e = S.e;
      for (int i = 0; i + 1 < n; ++i)
        if (fabsf(e[i]) <= thr) e[i] = 0.f;
      for (int i = 0; i < n; ++i)
        if (fabsf(d[i]) <= thr) d[i] = 0.f;
      int h = n - 1;
      while (h > 0 && e[h - 1] == 0.f) --h;
      if (h == 0) {
        S.nrot = -1;
      } else {
        int l = h - 1;
        while (l > 0 && e[l - 1] != 0.f) --l;
        qr_step(S, l, h);
        S.iters++;
        S.steps += S.nrot;
      }
    }
    __syncthreads();
    const int nr = S.nrot;
    if (nr < 0) {
      converged = true;
      break;
    }
    if (tid < n) {  // this thread's row of Q
      float2* row = As + tid * kBLD;
      for (int q = 0; q < nr; ++q) {
        const Rot r = S.rot[q];
        const float2 xa = row[r.a], xb = row[r.b];
        row[r.a] = make_float2(r.c * xa.x + r.s * xb.x, r.c * xa.y + r.s * xb.y);
        row[r.b] = make_float2(-r.s * xa.x + r.c * xb.x, -r.s * xa.y + r.c * xb.y);
      }
    }
    __syncthreads();
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
