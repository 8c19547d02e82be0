// The whitening product of eq. 4, A = K^{-1} R, for every (block, bin), as a
// batched complex GEMM on the FP32 SIMT cores, written column by column
// (A_cm[c][r] = A[r][c]) for the decompositions that work on A's columns.
//
// With R and K^{-1} Hermitian, A_cm = conj(R K^{-1}) as a row-major matrix:
//   conj(R K^{-1})[c][r] = sum_k conj(R[c][k]) conj(K^{-1}[k][r])
//                        = sum_k K^{-1}[r][k] R[k][c] = A[r][c],
// and C = R K^{-1} reads row k of both factors at step k
// (C[c][r] = sum_k conj(R[k][c]) K^{-1}[k][r]), so both operands come from
// shared memory as 32-byte row segments.
//
// One CTA per (bin, group of blocks): K^{-1} of the bin is staged once and
// serves the group; each R is staged in turn.  256 threads, each a 4 x 4 tile
// of C (16 x 16 tiles cover M <= 64): per step 4 complex values of each
// operand and 16 complex multiply-adds (64 FMA for 4 shared-memory loads).
//
// With Ns > 0 the columns are then rotated toward the split iteration's
// fixed point (a right-multiplication by a unitary Q, which leaves the left
// singular vectors of A unchanged): Y = A^H A_top, A_top the Ns columns of
// largest norm, is one power step toward the dominant right singular
// subspace; Q = H_0 .. H_{Ns-1} is the Householder basis whose first Ns
// columns span Y (compact WY, Q = I - V T V^H), and A Q = A - (A V T) V^H is
// written instead of A.  Its first Ns columns carry most of the signal
// energy, so the split iteration starts near its fixed point.
#include "ssl_internal.cuh"

namespace ssl {
namespace {

constexpr int kWhitenThreads = 256;
constexpr int kWhitenGroup = 2;  // blocks per CTA sharing the bin's K^{-1} (small: a short last wave)
constexpr int kPrecMaxNs = 8;    // preconditioning for Ns <= 8 (the split's range)
static_assert(kPrecMaxNs * 64 <= 2 * kWhitenThreads, "two rotated-pivot elements per thread");

__device__ __forceinline__ float2 cmad(float2 acc, float2 a, float2 b) {  // acc + a b
  return make_float2(fmaf(a.x, b.x, fmaf(-a.y, b.y, acc.x)), fmaf(a.x, b.y, fmaf(a.y, b.x, acc.y)));
}
__device__ __forceinline__ float2 cmadc(float2 acc, float2 a, float2 b) {  // acc + conj(a) b
  return make_float2(fmaf(a.x, b.x, fmaf(a.y, b.y, acc.x)), fmaf(a.x, b.y, fmaf(-a.y, b.x, acc.y)));
}
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}

// Eigenvectors of the n x n Hermitian H (stride kPrecMaxNs, n <= kPrecMaxNs)
// by cyclic Jacobi, run by one warp: every lane forms each rotation from
// H[p][p], H[q][q], H[p][q], then lane t < 2n updates row t % n of the
// columns p, q of H (t < n) or V (t >= n), and lane k < n the row pair
// p, q of H in column k.  V receives the eigenvectors as columns, sorted by
// eigenvalue descending, lam the eigenvalues.  H is overwritten.
__device__ void herm_eig_warp(float2* H, float2* V, float* lam, int n, int lane) {
  constexpr int S = kPrecMaxNs;
  for (int e = lane; e < n * n; e += 32) {
    const int i = e / n, j = e - i * n;
    V[i * S + j] = make_float2(i == j ? 1.f : 0.f, 0.f);
  }
  __syncwarp();
  for (int sweep = 0; sweep < 12; ++sweep) {
    float off = 0.f, dia = 0.f;
    for (int e = lane; e < n * n; e += 32) {
      const int i = e / n, j = e - i * n;
      const float2 h = H[i * S + j];
      if (i == j) dia += fabsf(h.x);
      else if (j > i) off += fabsf(h.x) + fabsf(h.y);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      off += __shfl_xor_sync(0xffffffffu, off, o);
      dia += __shfl_xor_sync(0xffffffffu, dia, o);
    }
    if (!(off > 1e-7f * dia)) break;  // (FP32: converged to rounding level; uniform)
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) {
        const float2 hpq = H[p * S + q];
        const float g = sqrtf(fmaf(hpq.x, hpq.x, hpq.y * hpq.y));
        if (!(g > 0.f)) continue;  // (uniform: every lane read the same word)
        const float a = H[p * S + p].x, b = H[q * S + q].x;
        const float2 e = make_float2(hpq.x / g, hpq.y / g);  // phase of H[p][q]
        // J = [[c, s], [-s conj(e), c conj(e)]] zeroes H[p][q] (t = s / c)
        const float zeta = (b - a) / (2.f * g);
        const float t = (zeta >= 0.f ? 1.f : -1.f) / (fabsf(zeta) + sqrtf(fmaf(zeta, zeta, 1.f)));
        const float c = 1.f / sqrtf(fmaf(t, t, 1.f)), sn = t * c;
        __syncwarp();  // every lane has read H[p][q], H[p][p], H[q][q]
        if (lane < 2 * n) {  // columns p, q of H and V: X <- X J
          float2* X = lane < n ? H : V;
          const int k = lane < n ? lane : lane - n;
          const float2 xp = X[k * S + p], xq = X[k * S + q];
          const float2 xqe = cmul(xq, make_float2(e.x, -e.y));
          X[k * S + p] = make_float2(c * xp.x - sn * xqe.x, c * xp.y - sn * xqe.y);
          X[k * S + q] = make_float2(sn * xp.x + c * xqe.x, sn * xp.y + c * xqe.y);
        }
        __syncwarp();
        if (lane < n) {  // rows p, q of H: H <- J^H H
          const int k = lane;
          const float2 hp = H[p * S + k], hq = H[q * S + k];
          const float2 hqe = cmul(hq, e);  // conj(conj(e)) = e on the row side
          H[p * S + k] = make_float2(c * hp.x - sn * hqe.x, c * hp.y - sn * hqe.y);
          H[q * S + k] = make_float2(sn * hp.x + c * hqe.x, sn * hp.y + c * hqe.y);
        }
        __syncwarp();
      }
  }
  if (lane == 0) {
    for (int i = 0; i < n; ++i) lam[i] = H[i * S + i].x;
    for (int i = 0; i < n; ++i) {  // selection sort, descending
      int m = i;
      for (int j = i + 1; j < n; ++j)
        if (lam[j] > lam[m]) m = j;
      if (m != i) {
        const float tl = lam[i];
        lam[i] = lam[m];
        lam[m] = tl;
        for (int k = 0; k < n; ++k) {
          const float2 tv = V[k * S + i];
          V[k * S + i] = V[k * S + m];
          V[k * S + m] = tv;
        }
      }
    }
  }
}

// Inverse of the n x n Hermitian positive definite D (stride kPrecMaxNs) by
// Gauss-Jordan without pivoting (D = I + Z Z^H: its pivots are >= 1), run by
// one warp over the n x 2n elements of [D | Di]; D is overwritten.
__device__ void hpd_inv_warp(float2* D, float2* Di, int n, int lane) {
  constexpr int S = kPrecMaxNs;
  for (int e = lane; e < n * n; e += 32) {
    const int i = e / n, j = e - i * n;
    Di[i * S + j] = make_float2(i == j ? 1.f : 0.f, 0.f);
  }
  __syncwarp();
  const int w = 2 * n;
  for (int k = 0; k < n; ++k) {
    const float2 pv = D[k * S + k];
    const float den = fmaf(pv.x, pv.x, pv.y * pv.y);
    const float2 ip = make_float2(pv.x / den, -pv.y / den);
    float2 nv[4];  // new values of this lane's elements (n x 2n <= 128 = 4 per lane)
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int e = lane + 32 * u;
      if (e < n * w) {
        const int i = e / w, j = e - i * w;
        float2* row_k = j < n ? D + k * S + j : Di + k * S + (j - n);
        const float2 pk = cmul(*row_k, ip);  // row k scaled by the pivot's inverse
        if (i == k) {
          nv[u] = pk;
        } else {
          const float2 f = D[i * S + k], x = j < n ? D[i * S + j] : Di[i * S + (j - n)];
          const float2 fp = cmul(f, pk);
          nv[u] = make_float2(x.x - fp.x, x.y - fp.y);
        }
      }
    }
    __syncwarp();  // every element of step k read before any is written
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int e = lane + 32 * u;
      if (e < n * w) {
        const int i = e / w, j = e - i * w;
        if (j < n) D[i * S + j] = nv[u];
        else Di[i * S + (j - n)] = nv[u];
      }
    }
    __syncwarp();
  }
}

// Row stride (complex elements) of the staged matrices: even (16-byte rows for
// the GEMM's float4 loads) and >= 4 ceil(M / 4) (the tiles' zero padding);
// 2 more than that multiple of 4 where three CTAs per SM still fit (M <= 60),
// which halves the bank conflicts of the phases whose threads walk across
// columns (a stride of 2 mod 4 float4s instead of 0 mod 4).
__host__ __device__ inline int whiten_ld(int M) {
  return M <= 60 ? ((M + 3) & ~3) + 2 : (M + 3) & ~3;
}

__global__ void __launch_bounds__(kWhitenThreads, 3)
whiten_kernel(const float2* __restrict__ R, const float2* __restrict__ Kinv,
              const float2* const* __restrict__ kinv_items, int nblk, int B, int M, int Ns,
              float2* __restrict__ Acm) {
  extern __shared__ float4 wsm[];
  const int ld = whiten_ld(M);
  float2* Ks = reinterpret_cast<float2*>(wsm);
  float2* Rs = Ks + (size_t)M * ld;             // R, then A by columns: Rs[c ld + r]
  float2* Ys = Rs + (size_t)M * ld;             // Y, then V, then G: [kPrecMaxNs][64]
  float2* Ws = Ys + kPrecMaxNs * 64;            // A V T, then A_n Z^H: [kPrecMaxNs][64]
  float2* Zs = Ws + kPrecMaxNs * 64;            // Z = Theta / 2: [kPrecMaxNs][64]
  float2* Ts = Zs + kPrecMaxNs * 64;            // T, then the pivots' eigenvectors
  float2* Ps = Ts + kPrecMaxNs * kPrecMaxNs;    // pivot Gram, then D = I + Z Z^H
  float2* Di = Ps + kPrecMaxNs * kPrecMaxNs;    // D^{-1}
  float* nrm = reinterpret_cast<float*>(Di + kPrecMaxNs * kPrecMaxNs);  // [64]
  float* lam = nrm + 64;                        // [kPrecMaxNs]
  __shared__ int top[kPrecMaxNs];
  __shared__ float tau_s[kPrecMaxNs];
  const int b = blockIdx.x, k0 = blockIdx.y * kWhitenGroup;
  const int tid = threadIdx.x;
  const int mt = (M + 3) / 4;                  // tiles per dimension
  const int tc = tid / 16, tr = tid % 16;      // tile: rows 4 tc.. of C, columns 4 tr..
  const bool active = tc < mt && tr < mt;
  const float2 zero = make_float2(0.f, 0.f);
  __shared__ float2 zs[kPrecMaxNs];
  for (int kk = 0; kk < kWhitenGroup && k0 + kk < nblk; ++kk) {
    const int k = k0 + kk;
    const float2* Kb = kinv_items ? kinv_items[k] + (size_t)b * M * M
                                  : Kinv + (size_t)b * M * M;
    const size_t item = (size_t)k * B + b;
    const float2* Rb = R + item * M * M;
    float2* Ab = Acm + item * M * M;
    __syncthreads();  // the previous item's reads of Rs (and Ks) are done
    // K^{-1} (first item, or every item with per-block inverses), then R:
    // eight loads in flight per thread before their shared-memory stores
    for (int pass = (kk == 0 || kinv_items) ? 0 : 1; pass < 2; ++pass) {
      const float2* src = pass == 0 ? Kb : Rb;
      float2* dst = pass == 0 ? Ks : Rs;
      for (int e0 = tid; e0 < M * ld; e0 += 8 * kWhitenThreads) {
        float2 v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int e = e0 + u * kWhitenThreads;
          v[u] = zero;
          if (e < M * ld) {
            const int r = e / ld, c = e - r * ld;
            if (c < M) v[u] = __ldg(src + (size_t)r * M + c);
          }
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int e = e0 + u * kWhitenThreads;
          if (e < M * ld) dst[e] = v[u];
        }
      }
    }
    __syncthreads();
    float2 acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = zero;
    if (active) {
      const float4* rrow = reinterpret_cast<const float4*>(Rs) + 2 * tc;
      const float4* krow = reinterpret_cast<const float4*>(Ks) + 2 * tr;
      const int step = ld / 2;  // float4 per row
#pragma unroll 4
      for (int s = 0; s < M; ++s) {
        const float4 ra = rrow[(size_t)s * step], rb = rrow[(size_t)s * step + 1];
        const float4 ka = krow[(size_t)s * step], kb = krow[(size_t)s * step + 1];
        // conj(R[s][4 tc + i]) and K^{-1}[s][4 tr + j]
        const float2 rv[4] = {make_float2(ra.x, -ra.y), make_float2(ra.z, -ra.w),
                              make_float2(rb.x, -rb.y), make_float2(rb.z, -rb.w)};
        const float2 kv[4] = {make_float2(ka.x, ka.y), make_float2(ka.z, ka.w),
                              make_float2(kb.x, kb.y), make_float2(kb.z, kb.w)};
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            acc[i][j].x = fmaf(rv[i].x, kv[j].x, fmaf(-rv[i].y, kv[j].y, acc[i][j].x));
            acc[i][j].y = fmaf(rv[i].x, kv[j].y, fmaf(rv[i].y, kv[j].x, acc[i][j].y));
          }
      }
    }
    if (Ns == 0) {  // A_cm[c][r] = conj(C[c][r]) straight out
      if (active)
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int c = 4 * tc + i;
          if (c < M)
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              const int r = 4 * tr + j;
              if (r < M) Ab[(size_t)c * M + r] = make_float2(acc[i][j].x, -acc[i][j].y);
            }
        }
      continue;
    }
    // ---- preconditioning: A by columns in shared memory (over R)
    float2* As = Rs;
    // squared column norms of A from the tiles: the 16 threads of a half-warp
    // share tc and hold rows 4 tr .. 4 tr + 3 of its four columns (zero
    // outside the matrix)
    float cn[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      float v = 0.f;
#pragma unroll
      for (int j = 0; j < 4; ++j) v = fmaf(acc[i][j].x, acc[i][j].x, fmaf(acc[i][j].y, acc[i][j].y, v));
#pragma unroll
      for (int o = 8; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      cn[i] = v;
    }
    __syncthreads();  // every tile has finished reading R
    if (active)
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int c = 4 * tc + i;
        if (c < M) {
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const int r = 4 * tr + j;
            if (r < M) As[(size_t)c * ld + r] = make_float2(acc[i][j].x, -acc[i][j].y);
          }
          if (tr == 0) nrm[c] = cn[i] == cn[i] ? cn[i] : -0.5f;
        }
      }
    __syncthreads();
    if (tid < 32) {  // the Ns columns of largest norm (ties: the lower index)
      const int lane = tid;
      for (int i = 0; i < Ns; ++i) {
        float best = -2.f;
        int bi = 0;
        for (int c = lane; c < M; c += 32)
          if (nrm[c] > best) {
            best = nrm[c];
            bi = c;
          }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          const float ob = __shfl_xor_sync(0xffffffffu, best, o);
          const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
          if (ob > best || (ob == best && oi < bi)) {
            best = ob;
            bi = oi;
          }
        }
        if (lane == 0) {
          top[i] = bi;
          nrm[bi] = -1.f;  // (taken)
        }
        __syncwarp();
      }
    }
    __syncthreads();
    // Y = A^H A_top (one power step), Ys[i][c]
    for (int e = tid; e < Ns * M; e += kWhitenThreads) {
      const int i = e / M, c = e - i * M;
      const float2* ac = As + (size_t)c * ld;
      const float2* at = As + (size_t)top[i] * ld;
      float2 y = zero;
      for (int r = 0; r < M; ++r) y = cmadc(y, ac[r], at[r]);
      Ys[i * 64 + c] = y;
    }
    __syncthreads();
    if (tid < 32) {  // Householder QR of Y: V over Y (rows < i zero), tau, then T
      const int lane = tid;
      for (int i = 0; i < Ns; ++i) {
        float2* v = Ys + i * 64;
        float2 x0 = lane >= i && lane < M ? v[lane] : zero;
        float2 x1 = lane + 32 < M ? v[lane + 32] : zero;
        float n2 = fmaf(x0.x, x0.x, fmaf(x0.y, x0.y, fmaf(x1.x, x1.x, x1.y * x1.y)));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) n2 += __shfl_xor_sync(0xffffffffu, n2, o);
        const float2 xi = make_float2(__shfl_sync(0xffffffffu, x0.x, i),
                                      __shfl_sync(0xffffffffu, x0.y, i));
        const float xn = sqrtf(n2), ax = sqrtf(fmaf(xi.x, xi.x, xi.y * xi.y));
        const float2 ph = ax > 0.f ? make_float2(xi.x / ax, xi.y / ax) : make_float2(1.f, 0.f);
        if (lane == i) x0 = make_float2(fmaf(ph.x, xn, x0.x), fmaf(ph.y, xn, x0.y));
        const float tau = xn > 0.f ? 1.f / (xn * (xn + ax)) : 0.f;
        if (lane < M) v[lane] = x0;
        if (lane + 32 < M) v[lane + 32] = x1;
        for (int q = i + 1; q < Ns; ++q) {  // H_i on the later columns
          float2* y = Ys + q * 64;
          const float2 y0 = lane < M ? y[lane] : zero, y1 = lane + 32 < M ? y[lane + 32] : zero;
          float2 d = cmadc(cmadc(zero, x0, y0), x1, y1);
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) {
            d.x += __shfl_xor_sync(0xffffffffu, d.x, o);
            d.y += __shfl_xor_sync(0xffffffffu, d.y, o);
          }
          const float2 td = make_float2(tau * d.x, tau * d.y);
          if (lane < M) y[lane] = cmad(y0, make_float2(-td.x, -td.y), x0);
          if (lane + 32 < M) y[lane + 32] = cmad(y1, make_float2(-td.x, -td.y), x1);
        }
        if (lane == 0) tau_s[i] = tau;
        __syncwarp();
      }
      // T[i][i] = tau_i, T[0:i][i] = -tau_i T[0:i][0:i] (V^H v_i)
      for (int i = 0; i < Ns; ++i) {
        const float2* vi = Ys + i * 64;
        for (int bq = 0; bq < i; ++bq) {
          const float2* vb = Ys + bq * 64;
          float2 d = zero;
          if (lane < M) d = cmadc(d, vb[lane], vi[lane]);
          if (lane + 32 < M) d = cmadc(d, vb[lane + 32], vi[lane + 32]);
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) {
            d.x += __shfl_xor_sync(0xffffffffu, d.x, o);
            d.y += __shfl_xor_sync(0xffffffffu, d.y, o);
          }
          if (lane == 0) zs[bq] = d;
        }
        __syncwarp();
        if (lane == 0) {
          const float ti = tau_s[i];
          for (int a = 0; a < Ns; ++a) {
            float2 t = zero;
            if (a < i) {
              for (int c = a; c < i; ++c) t = cmad(t, Ts[a * kPrecMaxNs + c], zs[c]);
              t = make_float2(-ti * t.x, -ti * t.y);
            } else if (a == i) {
              t = make_float2(ti, 0.f);
            }
            Ts[a * kPrecMaxNs + i] = t;
          }
        }
        __syncwarp();
      }
    }
    __syncthreads();
    // A V, then (A V) T, Ws[b][r]
    for (int e = tid; e < Ns * M; e += kWhitenThreads) {
      const int bq = e / M, r = e - bq * M;
      const float2* vb = Ys + bq * 64;
      float2 w = zero;
      for (int c = 0; c < M; ++c) w = cmad(w, As[(size_t)c * ld + r], vb[c]);
      Ws[bq * 64 + r] = w;
    }
    __syncthreads();
    for (int r = tid; r < M; r += kWhitenThreads) {
      float2 w[kPrecMaxNs];
#pragma unroll
      for (int q = 0; q < kPrecMaxNs; ++q) w[q] = q < Ns ? Ws[q * 64 + r] : zero;
#pragma unroll
      for (int q = 0; q < kPrecMaxNs; ++q) {
        if (q < Ns) {
          float2 t = zero;
#pragma unroll
          for (int a = 0; a < kPrecMaxNs; ++a)
            if (a <= q) t = cmad(t, w[a], Ts[a * kPrecMaxNs + q]);
          Ws[q * 64 + r] = t;
        }
      }
    }
    __syncthreads();
    // A Q = A - (A V T) V^H, by columns, in place (each element once)
    for (int e = tid; e < M * M; e += kWhitenThreads) {
      const int c = e / M, r = e - c * M;
      float2 v = As[(size_t)c * ld + r];
#pragma unroll
      for (int q = 0; q < kPrecMaxNs; ++q)
        if (q < Ns) {
          const float2 w = Ws[q * 64 + r], vc = Ys[q * 64 + c];
          // v -= w conj(vc)
          v.x -= fmaf(w.x, vc.x, w.y * vc.y);
          v.y -= fmaf(w.y, vc.x, -w.x * vc.y);
        }
      As[(size_t)c * ld + r] = v;
    }
    // Two block steps toward the fixed point, each: the pivots (first Ns
    // columns) rotated by the eigenvectors of their Gram matrix, so that they
    // are mutually orthogonal, then the Cayley transform U = (I + S/2)(I - S/2)^{-1}
    // of S = [[0, -Theta], [Theta^H, 0]], theta_sn = g_s^H g_n / (|g_s|^2 - |g_n|^2)
    // (the first-order rotation of each pivot-partner pair, at most 1/2 in size):
    // U is unitary for any Theta, and with Z = Theta / 2, D = I + Z Z^H,
    // G = (A_s + A_n Z^H) D^{-1}:  A_s <- 2 G - A_s,  A_n <- A_n - 2 G Z.
    const int nR = M - Ns;
    for (int step = 0; step < 2; ++step) {
      __syncthreads();
      for (int e = tid; e < Ns * Ns; e += kWhitenThreads) {  // pivot Gram
        const int a = e / Ns, c = e - a * Ns;
        float2 g = zero;
        for (int r = 0; r < M; ++r) g = cmadc(g, As[(size_t)a * ld + r], As[(size_t)c * ld + r]);
        Ps[a * kPrecMaxNs + c] = g;
      }
      for (int n = tid; n < nR; n += kWhitenThreads) {  // partner norms
        float v = 0.f;
        for (int r = 0; r < M; ++r) {
          const float2 x = As[(size_t)(Ns + n) * ld + r];
          v = fmaf(x.x, x.x, fmaf(x.y, x.y, v));
        }
        nrm[n] = v;
      }
      __syncthreads();
      if (tid < 32) herm_eig_warp(Ps, Ts, lam, Ns, tid);
      __syncthreads();
      float2 xr[2];  // the rotated pivots (Ns M <= 2 kWhitenThreads elements)
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int e = tid + u * kWhitenThreads;
        if (e < Ns * M) {
          const int t = e / M, r = e - t * M;
          float2 x = zero;
          for (int a = 0; a < Ns; ++a) x = cmad(x, As[(size_t)a * ld + r], Ts[a * kPrecMaxNs + t]);
          xr[u] = x;
        }
      }
      __syncthreads();
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int e = tid + u * kWhitenThreads;
        if (e < Ns * M) {
          const int t = e / M, r = e - t * M;
          As[(size_t)t * ld + r] = xr[u];
        }
      }
      __syncthreads();
      for (int e = tid; e < Ns * nR; e += kWhitenThreads) {  // Z = Theta / 2
        const int a = e / nR, n = e - a * nR;
        float2 g = zero;
        for (int r = 0; r < M; ++r)
          g = cmadc(g, As[(size_t)a * ld + r], As[(size_t)(Ns + n) * ld + r]);
        const float den = lam[a] - nrm[n];
        float2 th = den > 0.f ? make_float2(g.x / den, g.y / den) : zero;
        const float m = sqrtf(fmaf(th.x, th.x, th.y * th.y));
        if (!(m <= 0.5f)) th = m > 0.5f ? make_float2(th.x * (0.5f / m), th.y * (0.5f / m)) : zero;
        Zs[a * 64 + n] = make_float2(0.5f * th.x, 0.5f * th.y);
      }
      __syncthreads();
      for (int e = tid; e < Ns * M; e += kWhitenThreads) {  // A_n Z^H -> Ws
        const int a = e / M, r = e - a * M;
        float2 w = zero;
        for (int n = 0; n < nR; ++n) {
          const float2 x = As[(size_t)(Ns + n) * ld + r], z = Zs[a * 64 + n];
          w = make_float2(fmaf(x.x, z.x, fmaf(x.y, z.y, w.x)), fmaf(x.y, z.x, fmaf(-x.x, z.y, w.y)));
        }
        Ws[a * 64 + r] = w;
      }
      for (int e = tid; e < Ns * Ns; e += kWhitenThreads) {  // D = I + Z Z^H
        const int a = e / Ns, c = e - a * Ns;
        float2 d = make_float2(a == c ? 1.f : 0.f, 0.f);
        for (int n = 0; n < nR; ++n) d = cmadc(d, Zs[c * 64 + n], Zs[a * 64 + n]);
        Ps[a * kPrecMaxNs + c] = d;
      }
      __syncthreads();
      if (tid < 32) hpd_inv_warp(Ps, Di, Ns, tid);
      __syncthreads();
      for (int e = tid; e < Ns * M; e += kWhitenThreads) {  // G -> Ys
        const int a = e / M, r = e - a * M;
        float2 g = zero;
        for (int t = 0; t < Ns; ++t) {
          const float2 x = As[(size_t)t * ld + r], w = Ws[t * 64 + r];
          g = cmad(g, make_float2(x.x + w.x, x.y + w.y), Di[t * kPrecMaxNs + a]);
        }
        Ys[a * 64 + r] = g;
      }
      __syncthreads();
      for (int e = tid; e < M * M; e += kWhitenThreads) {
        const int c = e / M, r = e - c * M;
        float2 v = As[(size_t)c * ld + r];
        if (c < Ns) {
          const float2 g = Ys[c * 64 + r];
          v = make_float2(2.f * g.x - v.x, 2.f * g.y - v.y);
        } else {
          for (int a = 0; a < Ns; ++a) {
            const float2 u = cmul(Ys[a * 64 + r], Zs[a * 64 + (c - Ns)]);
            v = make_float2(fmaf(-2.f, u.x, v.x), fmaf(-2.f, u.y, v.y));
          }
        }
        As[(size_t)c * ld + r] = v;
      }
    }
    __syncthreads();
    for (int e = tid; e < M * M; e += kWhitenThreads) {
      const int c = e / M, r = e - c * M;
      Ab[(size_t)c * M + r] = As[(size_t)c * ld + r];
    }
  }
}

}  // namespace

cudaError_t launch_whiten(const float2* R, const float2* Kinv, const float2* const* kinv_items,
                          int nblk, int B, int M, int Ns, float2* Acm, cudaStream_t s) {
  if (nblk < 1 || B < 1 || M < 1 || M > SSL_MAX_M || (!Kinv && !kinv_items))
    return cudaErrorInvalidValue;
  if (Ns < 0 || Ns > kPrecMaxNs || Ns > M) Ns = 0;
  const size_t smem = (size_t)2 * M * whiten_ld(M) * sizeof(float2) +
                      (size_t)(3 * kPrecMaxNs * 64 + 3 * kPrecMaxNs * kPrecMaxNs) * sizeof(float2) +
                      (64 + kPrecMaxNs) * sizeof(float);
  cudaError_t e = cudaFuncSetAttribute(whiten_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  const dim3 grid(B, (nblk + kWhitenGroup - 1) / kWhitenGroup);
  whiten_kernel<<<grid, kWhitenThreads, smem, s>>>(R, Kinv, kinv_items, nblk, B, M, Ns, Acm);
  return cudaGetLastError();
}

}  // namespace ssl
