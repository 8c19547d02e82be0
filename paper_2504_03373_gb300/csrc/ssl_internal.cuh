// Internal declarations shared by the kernels and the C-ABI host code.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/ssl_gsvd_music.h"

namespace ssl {

// Column stride (in complex elements) of the shared-memory matrices of the
// per-bin kernels; SSL_MAX_M rounded to the warp-friendly 64.
constexpr int kLD = 64;

__host__ __device__ inline int ceil_div(int a, int b) { return (a + b - 1) / b; }

// ---- launchers (all asynchronous on `s`; return the launch error) ----

// eq. 2-3: R[k][w] = (1/T) sum_f x_f x_f^H.
cudaError_t launch_correlate(const float2* X, int nblk, int T, int B, int M, float2* R,
                             cudaStream_t s);

// K^{-1} through an FP64 Cholesky factorisation, one CTA per bin.
cudaError_t launch_noise_inverse(const float2* K, int B, int M, float2* Kinv, int32_t* status,
                                 unsigned* flags, cudaStream_t s);

// Jacobi controls (see ssl_jacobi_opts in the public header).
struct JacobiOpts {
  int max_sweeps;
  float rel_tol;   // <= 0: M * 2^-24
  float abs_tol;   // <= 0: no absolute criterion
  bool angles_f64;
};

// A = K^{-1} R and its SVD by one-sided Jacobi (eq. 4), one CTA per (block, bin).
// stats (optional, int32 [nblk][B][2]): sweeps run and rotations applied.
cudaError_t launch_gsvd(const float2* R, const float2* Kinv, int nblk, int B, int M,
                        const JacobiOpts& o, float* sigma, float2* E, int32_t* status,
                        int32_t* stats, unsigned* flags, cudaStream_t s);

// eq. 5 on the SIMT cores in FP32: P[k][w][d].
cudaError_t launch_spectrum_simt(const float2* E, int nblk, int B, int M, int Ns, const float2* H,
                                 const float* hnorm2, int D, int form, float* P, cudaStream_t s);

// eq. 6: Pbar[k][d] = sum_w P[k][w][d] in bin order.
cudaError_t launch_bin_sum(const float* P, int nblk, int B, int D, float* Pbar, cudaStream_t s);

// Peak search on the direction grid.
cudaError_t launch_peaks(const float* Pbar, int nblk, int n_az, int n_el, int Ns, int32_t* idx,
                         float* val, cudaStream_t s);

// ---- tensor-core spectrum (tcgen05), see spectrum_tc.cu ----
int tc_kp(int M);            // padded K of the real-embedded operands (64 or 128)
int tc_np(int M, int Ns);    // padded N = 2 (M - Ns) rounded up to 16
size_t tc_smem_bytes(int M, int Ns, int precision);
// H [B][D][M] -> A image [B][D][KP] (bf16 or tf32-rounded f32).
cudaError_t launch_pack_h(const float2* H, int B, int D, int M, int precision, void* out,
                          cudaStream_t s);
// E [nmat][M][M] -> B image [nmat][NP][KP].
cudaError_t launch_pack_e(const float2* E, int nmat, int M, int Ns, int precision, void* out,
                          cudaStream_t s);
cudaError_t launch_spectrum_tc(const CUtensorMap& tmH, const CUtensorMap& tmE, int nblk, int B,
                               int D, int M, int Ns, int precision, int form,
                               const float* hnorm2, float* P, unsigned* flags, cudaStream_t s);

// |h|^2 per (bin, direction) of a c64 table.
cudaError_t launch_hnorm2(const float2* H, int B, int D, int M, float* out, cudaStream_t s);

}  // namespace ssl
