// Inverse of the preset noise correlation K (eq. 4, Sec. III-B) in FP64.
//
// The paper inverts K by Gaussian elimination.  K is Hermitian positive
// definite, so this kernel factors K = L L^H (Cholesky, right-looking),
// inverts the triangular factor W = L^{-1} by forward substitution, and forms
// K^{-1} = W^H W; the product with R is the same A = K^{-1} R.  One CTA per
// bin, the whole matrix resident in shared memory as complex doubles.
//
// FP64 issues at a small fraction of the FP32 rate on this part and a warp
// instruction costs the same however many of its lanes are active, so the
// loops keep the lanes full: the trailing update and W^H W run over the
// packed lower triangle (not the square with half the lanes idle), each
// subtraction is folded into FMAs, and four lanes share each column of the
// substitution so that its longest serial chain is a quarter of a column.
#include "ssl_internal.cuh"

namespace ssl {
namespace {

constexpr int kThreads = 256;

struct cd {
  double x, y;
};

// (i, j), j <= i, of entry e of the row-packed lower triangle
__device__ __forceinline__ void tri_index(int e, int& i, int& j) {
  int r = (int)((sqrtf(8.f * (float)e + 1.f) - 1.f) * 0.5f);
  if (r * (r + 1) / 2 > e) --r;
  if ((r + 1) * (r + 2) / 2 <= e) ++r;
  i = r;
  j = e - r * (r + 1) / 2;
}

// Output element: FP32 complex (the FP32 path) or FP64 complex (the FP64 path).
__device__ __forceinline__ void store(float2* p, double x, double y) {
  *p = make_float2((float)x, (float)y);
}
__device__ __forceinline__ void store(double2* p, double x, double y) { *p = make_double2(x, y); }

template <class OutT>
__global__ void __launch_bounds__(kThreads)
noise_inverse_kernel(const float2* __restrict__ K, int M, OutT* __restrict__ Kinv,
                     int32_t* __restrict__ status, unsigned* flags, float2* __restrict__ Wout) {
  extern __shared__ cd sm[];
  const int LD = M + 1;
  cd* L = sm;           // [M][LD], lower triangle holds the factor
  cd* W = sm + M * LD;  // [M][LD], W = L^{-1} (lower triangular)
  __shared__ double invd[SSL_MAX_M];  // 1 / L_ii
  __shared__ int bad;
  const int b = blockIdx.x, tid = threadIdx.x;
  const float2* Kb = K + (size_t)b * M * M;
  if (tid == 0) bad = 0;
  __syncthreads();
  for (int e = tid; e < M * M; e += kThreads) {
    const int i = e / M, j = e % M;
    const float2 v = Kb[e];
    if (!isfinite(v.x) || !isfinite(v.y)) atomicExch(&bad, SSL_E_NONFINITE);
    L[i * LD + j] = {(double)v.x, (double)v.y};
  }
  __syncthreads();

  // Cholesky, column by column; the trailing update L_ij -= L_ik conj(L_jk)
  // over the packed lower triangle of rows and columns k + 1 .. M - 1.
  for (int k = 0; k < M && bad == 0; ++k) {
    if (tid == 0) {
      const double d = L[k * LD + k].x;
      if (!(d > 0.0)) {
        bad = SSL_E_NOT_PD;
      } else {
        const double r = sqrt(d);
        L[k * LD + k] = {r, 0.0};
        invd[k] = 1.0 / r;
      }
    }
    __syncthreads();
    if (bad != 0) break;
    const double inv = invd[k];
    for (int i = k + 1 + tid; i < M; i += kThreads) {
      L[i * LD + k].x *= inv;
      L[i * LD + k].y *= inv;
    }
    __syncthreads();
    const int n = M - k - 1;
    for (int e = tid; e < n * (n + 1) / 2; e += kThreads) {
      int ii, jj;
      tri_index(e, ii, jj);
      const int i = k + 1 + ii, j = k + 1 + jj;
      const cd a = L[i * LD + k], c = L[j * LD + k];
      cd& t = L[i * LD + j];
      t.x = fma(-a.x, c.x, fma(-a.y, c.y, t.x));
      t.y = fma(-a.y, c.x, fma(a.x, c.y, t.y));
    }
    __syncthreads();
  }

  OutT* Ob = Kinv + (size_t)b * M * M;
  if (bad != 0) {
    for (int e = tid; e < M * M; e += kThreads) {
      store(Ob + e, 0.0, 0.0);
      if (Wout) Wout[(size_t)b * M * M + e] = make_float2(0.f, 0.f);
    }
    if (tid == 0) {
      if (status) status[b] = bad;
      atomicOr(flags, bad == SSL_E_NOT_PD ? SSL_FLAG_NOT_PD : SSL_FLAG_NONFINITE);
    }
    return;
  }

  // W = L^{-1} by forward substitution, column c: W_cc = 1 / L_cc and
  // W_ic = -(sum_{c <= m < i} L_im W_mc) / L_ii.  Four lanes of a warp own
  // column c (thread 4c .. 4c + 3) and split each dot product by m mod 4, so
  // the serial chain of the longest column is a quarter of its length; the
  // upper triangle of W is zero.
  for (int e = tid; e < M * M; e += kThreads) {
    const int i = e / M, j = e % M;
    if (j > i) W[i * LD + j] = {0.0, 0.0};
  }
  {
    const int c = tid >> 2, part = tid & 3;
    const int c0 = (tid & ~31) >> 2;  // first column of this warp
    if (c < M && part == 0) W[c * LD + c] = {invd[c], 0.0};
    __syncwarp();
    for (int i = c0 + 1; i < M; ++i) {  // warp-uniform: the shuffles below
      double sx = 0.0, sy = 0.0;
      if (c < i && c < M)
        for (int m = c + part; m < i; m += 4) {
          const cd a = L[i * LD + m], w = W[m * LD + c];
          sx = fma(a.x, w.x, fma(-a.y, w.y, sx));
          sy = fma(a.x, w.y, fma(a.y, w.x, sy));
        }
      sx += __shfl_xor_sync(0xffffffffu, sx, 1);
      sy += __shfl_xor_sync(0xffffffffu, sy, 1);
      sx += __shfl_xor_sync(0xffffffffu, sx, 2);
      sy += __shfl_xor_sync(0xffffffffu, sy, 2);
      if (c < i && c < M && part == 0) {
        const double r = -invd[i];
        W[i * LD + c] = {sx * r, sy * r};
      }
      __syncwarp();
    }
  }
  __syncthreads();
  if (Wout)
    for (int e = tid; e < M * M; e += kThreads) {
      const cd w = W[(e / M) * LD + e % M];
      Wout[(size_t)b * M * M + e] = make_float2((float)w.x, (float)w.y);
    }

  // K^{-1} = W^H W over the packed lower triangle:
  //   (K^{-1})_ij = sum_{m >= i} conj(W_mi) W_mj,  i >= j.
  for (int e = tid; e < M * (M + 1) / 2; e += kThreads) {
    int i, j;
    tri_index(e, i, j);
    double ax = 0.0, ay = 0.0;
    for (int m = i; m < M; ++m) {
      const cd p = W[m * LD + i], q = W[m * LD + j];
      ax = fma(p.x, q.x, fma(p.y, q.y, ax));
      ay = fma(p.x, q.y, fma(-p.y, q.x, ay));
    }
    if (j == i) ay = 0.0;  // Hermitian: a real diagonal
    store(Ob + i * M + j, ax, ay);
    if (j != i) store(Ob + j * M + i, ax, -ay);
  }
  if (tid == 0 && status) status[b] = 0;
}

template <class OutT>
cudaError_t launch_inverse(const float2* K, int B, int M, OutT* Kinv, int32_t* status,
                           unsigned* flags, cudaStream_t s, float2* W) {
  const size_t smem = 2 * (size_t)M * (M + 1) * sizeof(cd);
  cudaError_t e = cudaFuncSetAttribute(noise_inverse_kernel<OutT>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  noise_inverse_kernel<OutT><<<B, kThreads, smem, s>>>(K, M, Kinv, status, flags, W);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_noise_inverse(const float2* K, int B, int M, float2* Kinv, int32_t* status,
                                 unsigned* flags, cudaStream_t s, float2* W) {
  return launch_inverse(K, B, M, Kinv, status, flags, s, W);
}

cudaError_t launch_noise_inverse_f64(const float2* K, int B, int M, double2* Kinv,
                                     int32_t* status, unsigned* flags, cudaStream_t s) {
  return launch_inverse(K, B, M, Kinv, status, flags, s, nullptr);
}

}  // namespace ssl
