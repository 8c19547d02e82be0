// Inverse of the preset noise correlation K (eq. 4, Sec. III-B) in FP64.
//
// The paper inverts K by Gaussian elimination.  K is Hermitian positive
// definite, so this kernel factors K = L L^H (Cholesky, right-looking),
// inverts the triangular factor W = L^{-1} by forward substitution, and forms
// K^{-1} = W^H W; the product with R is the same A = K^{-1} R.  One CTA per
// bin, the whole matrix resident in shared memory as complex doubles.
#include "ssl_internal.cuh"

namespace ssl {
namespace {

constexpr int kThreads = 256;

struct cd {
  double x, y;
};

__device__ __forceinline__ cd cmul(cd a, cd b) { return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x}; }
__device__ __forceinline__ cd cmulc(cd a, cd b) {  // a * conj(b)
  return {a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y};
}
__device__ __forceinline__ cd cconjmul(cd a, cd b) {  // conj(a) * b
  return {a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x};
}

__global__ void __launch_bounds__(kThreads)
noise_inverse_kernel(const float2* __restrict__ K, int M, float2* __restrict__ Kinv,
                     int32_t* __restrict__ status, unsigned* flags, float2* __restrict__ Wout) {
  extern __shared__ cd sm[];
  const int LD = M + 1;
  cd* L = sm;           // [M][LD], lower triangle holds the factor
  cd* W = sm + M * LD;  // [M][LD], W = L^{-1} (lower triangular)
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

  // Cholesky, column by column.
  for (int k = 0; k < M && bad == 0; ++k) {
    if (tid == 0) {
      const double d = L[k * LD + k].x;
      if (!(d > 0.0))
        bad = SSL_E_NOT_PD;
      else
        L[k * LD + k] = {sqrt(d), 0.0};
    }
    __syncthreads();
    if (bad != 0) break;
    const double inv = 1.0 / L[k * LD + k].x;
    for (int i = k + 1 + tid; i < M; i += kThreads) {
      L[i * LD + k].x *= inv;
      L[i * LD + k].y *= inv;
    }
    __syncthreads();
    const int n = M - k - 1;
    for (int e = tid; e < n * n; e += kThreads) {
      const int i = k + 1 + e / n, j = k + 1 + e % n;
      if (j <= i) {
        const cd t = cmulc(L[i * LD + k], L[j * LD + k]);  // L_ik conj(L_jk)
        L[i * LD + j].x -= t.x;
        L[i * LD + j].y -= t.y;
      }
    }
    __syncthreads();
  }

  float2* Ob = Kinv + (size_t)b * M * M;
  if (bad != 0) {
    for (int e = tid; e < M * M; e += kThreads) {
      Ob[e] = make_float2(0.f, 0.f);
      if (Wout) Wout[(size_t)b * M * M + e] = make_float2(0.f, 0.f);
    }
    if (tid == 0) {
      if (status) status[b] = bad;
      atomicOr(flags, bad == SSL_E_NOT_PD ? SSL_FLAG_NOT_PD : SSL_FLAG_NONFINITE);
    }
    return;
  }

  // W = L^{-1}: thread c solves column c by forward substitution.
  for (int c = tid; c < M; c += kThreads) {
    for (int i = 0; i < c; ++i) W[i * LD + c] = {0.0, 0.0};
    W[c * LD + c] = {1.0 / L[c * LD + c].x, 0.0};
    for (int i = c + 1; i < M; ++i) {
      cd acc = {0.0, 0.0};
      for (int k = c; k < i; ++k) {
        const cd t = cmul(L[i * LD + k], W[k * LD + c]);
        acc.x += t.x;
        acc.y += t.y;
      }
      const double r = -1.0 / L[i * LD + i].x;
      W[i * LD + c] = {acc.x * r, acc.y * r};
    }
  }
  __syncthreads();
  if (Wout)
    for (int e = tid; e < M * M; e += kThreads) {
      const cd w = W[(e / M) * LD + e % M];
      Wout[(size_t)b * M * M + e] = make_float2((float)w.x, (float)w.y);
    }

  // K^{-1} = W^H W:  (K^{-1})_ij = sum_{k >= max(i,j)} conj(W_ki) W_kj.
  for (int e = tid; e < M * M; e += kThreads) {
    const int i = e / M, j = e % M;
    if (j > i) continue;
    cd acc = {0.0, 0.0};
    for (int k = i; k < M; ++k) {  // i >= j
      const cd t = cconjmul(W[k * LD + i], W[k * LD + j]);
      acc.x += t.x;
      acc.y += t.y;
    }
    Ob[i * M + j] = make_float2((float)acc.x, (float)acc.y);
    if (j != i) Ob[j * M + i] = make_float2((float)acc.x, (float)-acc.y);
  }
  if (tid == 0 && status) status[b] = 0;
}

}  // namespace

cudaError_t launch_noise_inverse(const float2* K, int B, int M, float2* Kinv, int32_t* status,
                                 unsigned* flags, cudaStream_t s, float2* W) {
  const size_t smem = 2 * (size_t)M * (M + 1) * sizeof(cd);
  cudaError_t e = cudaFuncSetAttribute(noise_inverse_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  noise_inverse_kernel<<<B, kThreads, smem, s>>>(K, M, Kinv, status, flags, W);
  return cudaGetLastError();
}

}  // namespace ssl
