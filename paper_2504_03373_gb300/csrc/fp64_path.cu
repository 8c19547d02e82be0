// The hot path in double precision: eq. 2-6 and the peak search, every sum,
// product and decision in FP64 (inputs are the FP32 frames X, the FP32 noise
// correlation K and the FP32 steering table, widened).  It is the accuracy
// reference on the GPU: with the FP32 path's inputs it agrees with the FP64
// oracle to rounding, so the FP32 path's own error can be split from the
// method's on the device.
//
//  * correlate_f64_kernel  eq. 2-3: R = (1/T) sum_f x x^H with FP64 sums, one
//    CTA per (bin, block), frames staged in shared memory in chunks, each
//    thread owning entries of the upper triangle (R is written mirrored).
//  * gsvd_f64_kernel  eq. 4: A = K^{-1} R (K^{-1} from the FP64 Cholesky,
//    kept in FP64) and the SVD of A by one-sided (Hestenes) Jacobi on
//    G = A^H with complex-double columns in shared memory: the circle method
//    pairs the MP (padded) columns into MP / 2 disjoint pairs per round, a
//    warp takes a pair at a time (lanes over rows), forms alpha = |g_p|^2,
//    beta = |g_q|^2, gamma = g_p^H g_q, and rotates both columns of G and of
//    V by the unitary that zeroes gamma; V accumulates E.  A pair rotates while
//    |gamma| > tol sqrt(alpha beta) (tol = M 2^-53 by default) and, for pairs
//    of small columns (larger |g|^2 at most sqrt(abs_tol) max |g|^2), while
//    |gamma| > abs_tol max |g|^2; the iteration ends after a sweep without a
//    rotation.  Singular values are the column norms, sorted descending.
//  * spectrum_f64_kernel  eq. 5 on the SIMT cores: y_i = h^H e_i for the noise
//    columns in chunks of eight (E_n staged in shared memory), den = sum |y|^2
//    (SQ) or sum |y| (ABS), P = |h|^2 / den.
//  * bin_sum_f64_kernel  eq. 6 in fixed bin order.
#include <float.h>

#include "ssl_internal.cuh"

namespace ssl {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr double kDenFloor = 1e-300;  // a zero denominator of eq. 5

// ---- eq. 2-3 ----------------------------------------------------------------
constexpr int kCorrThreads = 256;
constexpr int kCorrChunk = 32;                                  // frames per stage
constexpr int kCorrAcc = (SSL_MAX_M * (SSL_MAX_M + 1) / 2 + kCorrThreads - 1) / kCorrThreads;

__global__ void __launch_bounds__(kCorrThreads)
correlate_f64_kernel(const float2* __restrict__ X, int T, int B, int M, double2* __restrict__ R) {
  __shared__ double2 xs[kCorrChunk * SSL_MAX_M];
  const int w = blockIdx.x, k = blockIdx.y, tid = threadIdx.x;
  const int ntri = M * (M + 1) / 2;
  double2 acc[kCorrAcc];
  int ii[kCorrAcc], jj[kCorrAcc];
#pragma unroll
  for (int u = 0; u < kCorrAcc; ++u) {
    acc[u] = make_double2(0.0, 0.0);
    // entry e of the row-packed upper triangle: (i, j), i <= j
    int e = tid + u * kCorrThreads, i = 0;
    while (e >= M - i && i < M) {
      e -= M - i;
      ++i;
    }
    ii[u] = i;
    jj[u] = i + e;
  }
  for (int f0 = 0; f0 < T; f0 += kCorrChunk) {
    const int nf = min(kCorrChunk, T - f0);
    __syncthreads();
    for (int e = tid; e < nf * M; e += kCorrThreads) {
      const int f = e / M, m = e % M;
      const float2 v = X[(((size_t)k * T + f0 + f) * B + w) * M + m];
      xs[f * M + m] = make_double2(v.x, v.y);
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < kCorrAcc; ++u) {
      if (tid + u * kCorrThreads >= ntri) continue;
      double re = acc[u].x, im = acc[u].y;
      for (int f = 0; f < nf; ++f) {
        const double2 a = xs[f * M + ii[u]], b = xs[f * M + jj[u]];
        re = fma(a.x, b.x, fma(a.y, b.y, re));   // x_i conj(x_j)
        im = fma(a.y, b.x, fma(-a.x, b.y, im));
      }
      acc[u] = make_double2(re, im);
    }
  }
  double2* Rb = R + ((size_t)k * B + w) * M * M;
  const double s = 1.0 / T;
#pragma unroll
  for (int u = 0; u < kCorrAcc; ++u) {
    if (tid + u * kCorrThreads >= ntri) continue;
    const int i = ii[u], j = jj[u];
    const double re = acc[u].x * s, im = i == j ? 0.0 : acc[u].y * s;
    Rb[(size_t)i * M + j] = make_double2(re, im);
    if (i != j) Rb[(size_t)j * M + i] = make_double2(re, -im);
  }
}

// ---- eq. 4 --------------------------------------------------------------------
constexpr int kJThreads = 256;
constexpr int kJWarps = kJThreads / 32;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

// Column of round-robin position `pos` in round r (circle method over MP
// positions: position 0 fixed, the others shifted by one per round).
__device__ __forceinline__ int rr_col(int pos, int r, int MP) {
  return pos == 0 ? 0 : 1 + (pos - 1 + r) % (MP - 1);
}

template <int MP>
__global__ void __launch_bounds__(kJThreads)
gsvd_f64_kernel(const double2* __restrict__ R, const double2* __restrict__ Kinv, int B, int M,
                int max_sweeps, double tol, double abs_tol, double* __restrict__ sigma,
                double2* __restrict__ E, int32_t* __restrict__ status,
                int32_t* __restrict__ stats, unsigned* flags) {
  constexpr int LD = MP + 1;  // column stride of G and V (complex doubles)
  constexpr int RPL = MP / 32 > 0 ? MP / 32 : 1;
  extern __shared__ double2 jsm[];
  double2* G = jsm;            // [MP][LD]: column c at G + c * LD
  double2* V = jsm + MP * LD;  // [MP][LD]
  __shared__ double nrm[MP];
  __shared__ double sig[MP];
  __shared__ int rnk[MP], inv[MP];
  __shared__ int bad, rot_sweep, tested_all, rot_all;
  const int w = blockIdx.x, k = blockIdx.y, tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  const size_t item = (size_t)k * B + w;
  const double2* Rb = R + item * M * M;
  const double2* Kb = Kinv + (size_t)w * M * M;

  if (tid == 0) {
    bad = 0;
    tested_all = rot_all = 0;
  }
  // R staged in V's space; G[c][r] = conj(A[c][r]) with A = K^{-1} R
  for (int e = tid; e < M * M; e += kJThreads) V[e] = Rb[e];
  __syncthreads();
  for (int e = tid; e < MP * MP; e += kJThreads) {
    const int c = e / MP, r = e % MP;
    double re = 0.0, im = 0.0;
    if (c < M && r < M)
      for (int m = 0; m < M; ++m) {
        const double2 a = __ldg(Kb + (size_t)c * M + m), b = V[m * M + r];
        re = fma(a.x, b.x, fma(-a.y, b.y, re));
        im = fma(a.x, b.y, fma(a.y, b.x, im));
      }
    if (!isfinite(re) || !isfinite(im)) bad = 1;
    G[c * LD + r] = make_double2(re, -im);
  }
  __syncthreads();
  for (int e = tid; e < MP * MP; e += kJThreads) {
    const int c = e / MP, r = e % MP;
    V[c * LD + r] = make_double2(c == r ? 1.0 : 0.0, 0.0);
  }
  __syncthreads();

  bool converged = bad != 0;
  int tested = 0, rotated = 0;
  for (int sw = 0; sw < max_sweeps && !converged; ++sw) {
    // squared column norms at the sweep start: the absolute level and its gate
    for (int c = warp; c < MP; c += kJWarps) {
      double s = 0.0;
#pragma unroll
      for (int h = 0; h < RPL; ++h) {
        const int r = lane + 32 * h;
        if (r < MP) {
          const double2 g = G[c * LD + r];
          s = fma(g.x, g.x, fma(g.y, g.y, s));
        }
      }
      s = warp_sum(s);
      if (lane == 0) nrm[c] = s;
    }
    if (tid == 0) rot_sweep = 0;
    __syncthreads();
    double amax = 0.0;
    for (int c = 0; c < MP; ++c) amax = fmax(amax, nrm[c]);
    const double abs_thr = abs_tol * amax, gate = sqrt(abs_tol) * amax;
    int wrot = 0;
    for (int r = 0; r < MP - 1; ++r) {
      for (int pk = warp; pk < MP / 2; pk += kJWarps) {
        const int p = rr_col(pk, r, MP), q = rr_col(MP - 1 - pk, r, MP);
        double2 x[RPL], y[RPL];
        double al = 0.0, be = 0.0, gr = 0.0, gi = 0.0;
#pragma unroll
        for (int h = 0; h < RPL; ++h) {
          const int row = lane + 32 * h;
          x[h] = row < MP ? G[p * LD + row] : make_double2(0.0, 0.0);
          y[h] = row < MP ? G[q * LD + row] : make_double2(0.0, 0.0);
          al = fma(x[h].x, x[h].x, fma(x[h].y, x[h].y, al));
          be = fma(y[h].x, y[h].x, fma(y[h].y, y[h].y, be));
          gr = fma(x[h].x, y[h].x, fma(x[h].y, y[h].y, gr));   // conj(x) y
          gi = fma(x[h].x, y[h].y, fma(-x[h].y, y[h].x, gi));
        }
        al = warp_sum(al);
        be = warp_sum(be);
        gr = warp_sum(gr);
        gi = warp_sum(gi);
        const bool real = p < M && q < M;
        tested += real && lane == 0;
        const double g2 = fma(gr, gr, gi * gi);
        const double mx = fmax(al, be);
        bool rot = real && al > 0.0 && be > 0.0 && g2 > tol * tol * al * be;
        if (rot && mx <= gate) rot = g2 > abs_thr * abs_thr;
        if (!rot) continue;  // warp-uniform: every lane holds the same sums
        const double d = be - al;
        const double wq = sqrt(fma(d, d, 4.0 * g2));
        const double den = fabs(d) + wq;
        const double rq = 1.0 / sqrt(fma(den, den, 4.0 * g2));
        const double c = den * rq, f = d < 0.0 ? -rq : rq;
        const double sr = 2.0 * f * gr, si = 2.0 * f * gi;  // s e = sign(d) 2 gamma / sqrt(q)
        // x' = c x - conj(se) y,  y' = se x + c y  (columns of G and of V)
#pragma unroll
        for (int h = 0; h < RPL; ++h) {
          const int row = lane + 32 * h;
          if (row < MP) {
            const double2 a = x[h], b = y[h];
            G[p * LD + row] = make_double2(fma(c, a.x, -fma(sr, b.x, si * b.y)),
                                           fma(c, a.y, -fma(sr, b.y, -si * b.x)));
            G[q * LD + row] = make_double2(fma(c, b.x, fma(sr, a.x, -si * a.y)),
                                           fma(c, b.y, fma(sr, a.y, si * a.x)));
            const double2 va = V[p * LD + row], vb = V[q * LD + row];
            V[p * LD + row] = make_double2(fma(c, va.x, -fma(sr, vb.x, si * vb.y)),
                                           fma(c, va.y, -fma(sr, vb.y, -si * vb.x)));
            V[q * LD + row] = make_double2(fma(c, vb.x, fma(sr, va.x, -si * va.y)),
                                           fma(c, vb.y, fma(sr, va.y, si * va.x)));
          }
        }
        wrot += lane == 0;
      }
      __syncthreads();
    }
    if (lane == 0 && wrot) atomicAdd(&rot_sweep, wrot);
    __syncthreads();
    rotated += rot_sweep;
    converged = rot_sweep == 0;
    __syncthreads();
  }
  if (lane == 0 && tested) atomicAdd(&tested_all, tested);
  // ---- singular values and E ----
  for (int c = warp; c < MP; c += kJWarps) {
    double s = 0.0, v2 = 0.0;
#pragma unroll
    for (int h = 0; h < RPL; ++h) {
      const int r = lane + 32 * h;
      if (r < MP) {
        const double2 g = G[c * LD + r], v = V[c * LD + r];
        s = fma(g.x, g.x, fma(g.y, g.y, s));
        v2 = fma(v.x, v.x, fma(v.y, v.y, v2));
      }
    }
    s = warp_sum(s);
    v2 = warp_sum(v2);
    if (lane == 0) {
      sig[c] = c < M ? sqrt(s) : -1.0;
      nrm[c] = v2 > 0.0 ? 1.0 / sqrt(v2) : 1.0;
    }
  }
  __syncthreads();
  if (tid < MP) {
    // ranks by value, ties by column; NaN after the real columns, before the
    // padding, so the ranks stay a permutation
    const double v0 = sig[tid], v = v0 == v0 ? v0 : -0.5;
    int rk = 0;
    for (int c = 0; c < MP; ++c) {
      const double u0 = sig[c], u = u0 == u0 ? u0 : -0.5;
      rk += (u > v) || (u == v && c < tid);
    }
    rnk[tid] = rk;
  }
  __syncthreads();
  if (tid < MP) inv[rnk[tid]] = tid;
  __syncthreads();
  double2* Eb = E + item * M * M;
  for (int e = tid; e < M * M; e += kJThreads) {
    const int row = e / M, rk = e % M, c = inv[rk];
    const double2 v = V[c * LD + row];
    Eb[e] = make_double2(v.x * nrm[c], v.y * nrm[c]);
  }
  if (tid < M) sigma[item * M + rnk[tid]] = sig[tid];
  if (tid == 0) {
    int st = 0;
    if (bad)
      st = SSL_E_NONFINITE;
    else if (!converged)
      st = SSL_E_NO_CONVERGENCE;
    if (status) status[item] = st;
    if (stats) {
      stats[2 * item] = tested_all;
      stats[2 * item + 1] = rotated;
    }
    if (st == SSL_E_NONFINITE) atomicOr(flags, SSL_FLAG_NONFINITE);
    if (st == SSL_E_NO_CONVERGENCE) atomicOr(flags, SSL_FLAG_NO_CONVERGENCE);
  }
}

// ---- eq. 5 --------------------------------------------------------------------
constexpr int kSpecThreads = 256;
constexpr int kSpecChunk = 8;  // noise columns per pass over h

__global__ void __launch_bounds__(kSpecThreads)
spectrum_f64_kernel(const double2* __restrict__ E, int B, int M, int Ns,
                    const float2* __restrict__ H, int D, int form, double* __restrict__ P) {
  extern __shared__ double2 en[];  // [M][N]: E_n of this (block, bin)
  const int w = blockIdx.x, k = blockIdx.y, tid = threadIdx.x;
  const int N = M - Ns;
  const size_t item = (size_t)k * B + w;
  const double2* Eb = E + item * M * M;
  for (int e = tid; e < M * N; e += kSpecThreads) {
    const int m = e / N, i = e % N;
    en[e] = Eb[(size_t)m * M + Ns + i];
  }
  __syncthreads();
  for (int d = tid; d < D; d += kSpecThreads) {
    const float2* h = H + ((size_t)w * D + d) * M;
    double hh = 0.0;
    for (int m = 0; m < M; ++m) {
      const float2 v = __ldg(h + m);
      hh = fma((double)v.x, (double)v.x, fma((double)v.y, (double)v.y, hh));
    }
    double den = 0.0;
    for (int i0 = 0; i0 < N; i0 += kSpecChunk) {
      double yr[kSpecChunk], yi[kSpecChunk];
#pragma unroll
      for (int u = 0; u < kSpecChunk; ++u) yr[u] = yi[u] = 0.0;
      for (int m = 0; m < M; ++m) {
        const float2 hv = __ldg(h + m);
        const double hx = hv.x, hy = hv.y;
#pragma unroll
        for (int u = 0; u < kSpecChunk; ++u) {
          if (i0 + u < N) {
            const double2 e = en[m * N + i0 + u];
            yr[u] = fma(hx, e.x, fma(hy, e.y, yr[u]));   // conj(h) e
            yi[u] = fma(hx, e.y, fma(-hy, e.x, yi[u]));
          }
        }
      }
#pragma unroll
      for (int u = 0; u < kSpecChunk; ++u) {
        if (i0 + u < N) {
          const double a2 = fma(yr[u], yr[u], yi[u] * yi[u]);
          den += form == SSL_FORM_SQ ? a2 : sqrt(a2);
        }
      }
    }
    P[item * D + d] = hh / fmax(den, kDenFloor);
  }
}

// ---- eq. 6 --------------------------------------------------------------------
__global__ void bin_sum_f64_kernel(const double* __restrict__ P, int B, int D,
                                   double* __restrict__ Pbar) {
  const int d = blockIdx.x * blockDim.x + threadIdx.x;
  const int k = blockIdx.y;
  if (d >= D) return;
  const double* Pk = P + (size_t)k * B * D + d;
  double s = 0.0;
  for (int w = 0; w < B; ++w) s += Pk[(size_t)w * D];
  Pbar[(size_t)k * D + d] = s;
}

template <int MP>
cudaError_t gsvd_f64_mp(const double2* R, const double2* Kinv, int nblk, int B, int M,
                        int max_sweeps, double tol, double abs_tol, double* sigma, double2* E,
                        int32_t* status, int32_t* stats, unsigned* flags, cudaStream_t s) {
  const size_t smem = 2 * (size_t)MP * (MP + 1) * sizeof(double2);
  cudaError_t e = cudaFuncSetAttribute(gsvd_f64_kernel<MP>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  gsvd_f64_kernel<MP><<<dim3(B, nblk), kJThreads, smem, s>>>(R, Kinv, B, M, max_sweeps, tol,
                                                             abs_tol, sigma, E, status, stats,
                                                             flags);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_correlate_f64(const float2* X, int nblk, int T, int B, int M, double2* R,
                                 cudaStream_t s) {
  correlate_f64_kernel<<<dim3(B, nblk), kCorrThreads, 0, s>>>(X, T, B, M, R);
  return cudaGetLastError();
}

cudaError_t launch_gsvd_f64(const double2* R, const double2* Kinv, int nblk, int B, int M,
                            int max_sweeps, double tol, double abs_tol, double* sigma, double2* E,
                            int32_t* status, int32_t* stats, unsigned* flags, cudaStream_t s) {
  if (tol <= 0.0) tol = (double)M * 1.1102230246251565e-16;  // M 2^-53
  if (abs_tol < 0.0) abs_tol = 0.0;
  if (M <= 16)
    return gsvd_f64_mp<16>(R, Kinv, nblk, B, M, max_sweeps, tol, abs_tol, sigma, E, status,
                           stats, flags, s);
  if (M <= 32)
    return gsvd_f64_mp<32>(R, Kinv, nblk, B, M, max_sweeps, tol, abs_tol, sigma, E, status,
                           stats, flags, s);
  return gsvd_f64_mp<64>(R, Kinv, nblk, B, M, max_sweeps, tol, abs_tol, sigma, E, status, stats,
                         flags, s);
}

cudaError_t launch_spectrum_f64(const double2* E, int nblk, int B, int M, int Ns, const float2* H,
                                int D, int form, double* P, cudaStream_t s) {
  const size_t smem = (size_t)M * (M - Ns) * sizeof(double2);
  cudaError_t e = cudaFuncSetAttribute(spectrum_f64_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  spectrum_f64_kernel<<<dim3(B, nblk), kSpecThreads, smem, s>>>(E, B, M, Ns, H, D, form, P);
  return cudaGetLastError();
}

cudaError_t launch_bin_sum_f64(const double* P, int nblk, int B, int D, double* Pbar,
                               cudaStream_t s) {
  bin_sum_f64_kernel<<<dim3(ceil_div(D, 256), nblk), 256, 0, s>>>(P, B, D, Pbar);
  return cudaGetLastError();
}

}  // namespace ssl
