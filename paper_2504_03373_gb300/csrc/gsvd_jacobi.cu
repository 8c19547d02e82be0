// Whitening and generalised SVD, eq. 4 (Sec. III-A/B):
//   A = K^{-1} R = E Lambda E_r^H,   E = left singular vectors (columns).
//
// One CTA per (bin, block), everything resident in shared memory.
//  1. A = K^{-1} R in FP32 (register-tiled complex GEMM), stored as
//     G = A^H column-major.
//  2. One-sided (Hestenes) Jacobi on G: columns p, q are rotated by a
//     unitary 2x2 J until all pairs are orthogonal; the product V of the
//     rotations gives G V = U Sigma, i.e. A = V Sigma U^H, so E = V and the
//     singular values are the column norms of G V.  Pairs are visited in the
//     round-robin (circle) order: each round has M/2 disjoint pairs, M-1
//     rounds form a sweep, every pair once per sweep.
//  3. Per round: each warp forms the Gram entries (alpha = |g_p|^2,
//     beta = |g_q|^2, gamma = g_p^H g_q) of its pairs in FP32 with warp-shuffle
//     reductions; warp 0 then computes every pair's rotation in FP64, one
//     lane per pair (FP64 issue is the scarce resource on this part, so it is
//     never replicated across a warp); all warps apply the rotations to G and
//     V in FP32.
//  4. Convergence (FP64): a pair is rotated only if
//     |gamma| > tol * sqrt(alpha * beta), tol = M * 2^-24; the sweep loop stops
//     after the first sweep that rotates nothing.
//  5. Singular values = column norms, sorted descending; E's columns are
//     permuted accordingly (Alg. 1's sort step).
#include "ssl_internal.cuh"

namespace ssl {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kMaxPairs = kLD / 2;            // 32
constexpr int kSlotsPerWarp = kMaxPairs / kWarps;  // 4

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Circle-method schedule: position 0 is fixed, the others rotate by one per
// round; slot s pairs positions s and n-1-s.
__device__ __forceinline__ int circle_pos(int i, int r, int n) {
  return i == 0 ? 0 : 1 + (i - 1 + r) % (n - 1);
}

// FP64 rotation for one pair.  In: alpha, beta, gamma = (gr, gi).
// Out: c (real) and s*e (complex, e = gamma/|gamma|) such that
//   g_p' = c g_p - conj(s e) g_q,   g_q' = (s e) g_p + c g_q
// makes g_p'^H g_q' = 0.  Returns false if the pair is already orthogonal to
// within tol (or degenerate).
__device__ __forceinline__ bool rotation_f64(float4 in, double tol, float4& out) {
  const double a = in.x, bb = in.y, gr = in.z, gi = in.w;
  const double g2 = gr * gr + gi * gi;
  if (!(g2 > tol * tol * a * bb) || !(g2 > 0.0)) return false;
  const double g = sqrt(g2);
  const double zeta = (bb - a) / (2.0 * g);
  const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
  const double c = 1.0 / sqrt(1.0 + t * t);
  const double sg = c * t / g;
  out = make_float4((float)c, (float)(sg * gr), (float)(sg * gi), 1.0f);
  return true;
}

__global__ void __launch_bounds__(kThreads)
gsvd_jacobi_kernel(const float2* __restrict__ R, const float2* __restrict__ Kinv, int B, int M,
                   int max_sweeps, float tol, float* __restrict__ sigma, float2* __restrict__ E,
                   int32_t* __restrict__ status, int32_t* __restrict__ stats, unsigned* flags) {
  extern __shared__ float2 sm[];
  float2* G = sm;              // column c of G at G + c * kLD
  float2* V = sm + kLD * kLD;  // column c of V at V + c * kLD
  __shared__ float4 gram[kMaxPairs];
  __shared__ float4 rot[kMaxPairs];
  __shared__ int rot_count;
  __shared__ int bad;
  __shared__ float sig[kLD];
  __shared__ int rnk[kLD];

  const int b = blockIdx.x, k = blockIdx.y;
  const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
  const size_t mat = ((size_t)k * B + b) * M * M;
  const float2* Rb = R + mat;
  const float2* Kb = Kinv + (size_t)b * M * M;

  if (tid == 0) {
    bad = 0;
    rot_count = 0;
  }
  // Stage K^{-1} (into G's space) and R (into V's space), dense row-major.
  for (int e = tid; e < M * M; e += kThreads) {
    G[e] = Kb[e];
    V[e] = Rb[e];
  }
  __syncthreads();

  // A = K^{-1} R, 4x4 register tile per thread over a 64x64 frame.
  const int ti = tid / 16, tj = tid % 16;
  float2 acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[a][c] = make_float2(0.f, 0.f);
  for (int m = 0; m < M; ++m) {
    float2 kv[4], rv[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const int i = ti + 16 * a, j = tj + 16 * a;
      kv[a] = i < M ? G[i * M + m] : make_float2(0.f, 0.f);
      rv[a] = j < M ? V[m * M + j] : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        acc[a][c].x = fmaf(kv[a].x, rv[c].x, fmaf(-kv[a].y, rv[c].y, acc[a][c].x));
        acc[a][c].y = fmaf(kv[a].x, rv[c].y, fmaf(kv[a].y, rv[c].x, acc[a][c].y));
      }
  }
  bool finite = true;
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int c = 0; c < 4; ++c) finite &= isfinite(acc[a][c].x) && isfinite(acc[a][c].y);
  if (!finite) atomicExch(&bad, 1);
  __syncthreads();
  // G = A^H: column i of G is conj(row i of A).  Zero padding outside M x M.
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int i = ti + 16 * a, j = tj + 16 * c;  // A[i][j] -> G[row j][col i]
      G[i * kLD + j] = (i < M && j < M) ? make_float2(acc[a][c].x, -acc[a][c].y)
                                        : make_float2(0.f, 0.f);
    }
  for (int e = tid; e < kLD * kLD; e += kThreads) {
    const int c = e / kLD, r = e % kLD;
    V[e] = make_float2((r == c && c < M) ? 1.f : 0.f, 0.f);
  }
  __syncthreads();

  const int n = (M + 1) & ~1;  // even number of circle positions
  const int npair = n / 2;
  int sweeps = 0, rotations = 0;
  bool converged = (bad != 0);
  for (int sw = 0; sw < max_sweeps && !converged; ++sw) {
    for (int r = 0; r < n - 1; ++r) {
      float2 gp[kSlotsPerWarp][2], gq[kSlotsPerWarp][2];
      int pp[kSlotsPerWarp], qq[kSlotsPerWarp];
#pragma unroll
      for (int j = 0; j < kSlotsPerWarp; ++j) {
        const int slot = warp + kWarps * j;
        pp[j] = qq[j] = -1;
        if (slot < npair) {
          const int p = circle_pos(slot, r, n), q = circle_pos(n - 1 - slot, r, n);
          if (p < M && q < M) {
            pp[j] = p;
            qq[j] = q;
            gp[j][0] = G[p * kLD + lane];
            gp[j][1] = G[p * kLD + lane + 32];
            gq[j][0] = G[q * kLD + lane];
            gq[j][1] = G[q * kLD + lane + 32];
            float al = 0.f, be = 0.f, gr = 0.f, gi = 0.f;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              al = fmaf(gp[j][h].x, gp[j][h].x, fmaf(gp[j][h].y, gp[j][h].y, al));
              be = fmaf(gq[j][h].x, gq[j][h].x, fmaf(gq[j][h].y, gq[j][h].y, be));
              // conj(gp) * gq
              gr = fmaf(gp[j][h].x, gq[j][h].x, fmaf(gp[j][h].y, gq[j][h].y, gr));
              gi = fmaf(gp[j][h].x, gq[j][h].y, fmaf(-gp[j][h].y, gq[j][h].x, gi));
            }
            al = warp_sum(al);
            be = warp_sum(be);
            gr = warp_sum(gr);
            gi = warp_sum(gi);
            if (lane == 0) gram[slot] = make_float4(al, be, gr, gi);
          } else if (lane == 0) {
            gram[slot] = make_float4(-1.f, -1.f, 0.f, 0.f);
          }
        }
      }
      __syncthreads();
      if (warp == 0) {
        float4 o = make_float4(1.f, 0.f, 0.f, 0.f);
        bool did = false;
        if (lane < npair) {
          const float4 g = gram[lane];
          if (g.x >= 0.f) did = rotation_f64(g, (double)tol, o);
          rot[lane] = o;
        }
        const unsigned m = __ballot_sync(0xffffffffu, did);
        if (lane == 0) rot_count += __popc(m);
      }
      __syncthreads();
#pragma unroll
      for (int j = 0; j < kSlotsPerWarp; ++j) {
        const int slot = warp + kWarps * j;
        if (pp[j] < 0) continue;
        const float4 cs = rot[slot];
        if (cs.w == 0.f) continue;
        const float c = cs.x, sr = cs.y, si = cs.z;  // s e = sr + i si
        const int p = pp[j], q = qq[j];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const float2 a = gp[j][h], d = gq[j][h];
          // p' = c a - conj(se) d ; q' = se a + c d
          G[p * kLD + lane + 32 * h] = make_float2(c * a.x - (sr * d.x + si * d.y),
                                                   c * a.y - (sr * d.y - si * d.x));
          G[q * kLD + lane + 32 * h] = make_float2(c * d.x + (sr * a.x - si * a.y),
                                                   c * d.y + (sr * a.y + si * a.x));
          const float2 va = V[p * kLD + lane + 32 * h], vd = V[q * kLD + lane + 32 * h];
          V[p * kLD + lane + 32 * h] = make_float2(c * va.x - (sr * vd.x + si * vd.y),
                                                   c * va.y - (sr * vd.y - si * vd.x));
          V[q * kLD + lane + 32 * h] = make_float2(c * vd.x + (sr * va.x - si * va.y),
                                                   c * vd.y + (sr * va.y + si * va.x));
        }
      }
      __syncthreads();
    }
    ++sweeps;
    const int rc = rot_count;
    rotations += rc;
    converged = (rc == 0);
    __syncthreads();
    if (tid == 0) rot_count = 0;
  }

  // Column norms -> singular values.
  for (int c = warp; c < M; c += kWarps) {
    const float2 x0 = G[c * kLD + lane], x1 = G[c * kLD + lane + 32];
    float s = x0.x * x0.x + x0.y * x0.y + x1.x * x1.x + x1.y * x1.y;
    s = warp_sum(s);
    if (lane == 0) sig[c] = sqrtf(s);
  }
  __syncthreads();
  if (tid < M) {
    const float v = sig[tid];
    int rk = 0;
    for (int c = 0; c < M; ++c) {
      const float w = sig[c];
      rk += (w > v) || (w == v && c < tid);
    }
    rnk[tid] = rk;
  }
  __syncthreads();
  const size_t vec = ((size_t)k * B + b) * M;
  for (int e = tid; e < M * M; e += kThreads) {
    const int r = e / M, c = e % M;
    E[mat + (size_t)r * M + rnk[c]] = V[c * kLD + r];
  }
  if (tid < M) sigma[vec + rnk[tid]] = sig[tid];
  if (tid == 0) {
    int st = 0;
    if (bad != 0)
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
                        int max_sweeps, float* sigma, float2* E, int32_t* status, int32_t* stats,
                        unsigned* flags, cudaStream_t s) {
  const size_t smem = 2 * (size_t)kLD * kLD * sizeof(float2);
  cudaError_t e = cudaFuncSetAttribute(gsvd_jacobi_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const float tol = (float)M * 5.9604644775390625e-8f;  // M * 2^-24
  dim3 grid(B, nblk);
  gsvd_jacobi_kernel<<<grid, kThreads, smem, s>>>(R, Kinv, B, M, max_sweeps, tol, sigma, E,
                                                   status, stats, flags);
  return cudaGetLastError();
}

}  // namespace ssl
