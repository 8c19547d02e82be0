// MUSIC spectrum (eq. 5) on the 5th-generation tensor cores (tcgen05).
//
// The complex contraction Y = H^H E_n of one bin is embedded in a real GEMM:
//   A[d][k]   = Re h_d[k]            (k < M)        Im h_d[k-M]      (M <= k < 2M)
//   B[2i][k]  = Re E[k][Ns+i]        (k < M)        Im E[k-M][Ns+i]  (M <= k < 2M)
//   B[2i+1][k]= Im E[k][Ns+i]        (k < M)       -Re E[k-M][Ns+i]  (M <= k < 2M)
// so that D = A B^T holds Re(h_d^H e_i) in column 2i and Im(h_d^H e_i) in
// column 2i+1.  Both operands are K-major, zero-padded to KP (64 or 128)
// columns and NP (a multiple of 16) rows, stored in BF16 (kind::f16) or in
// TF32-rounded FP32 (kind::tf32), with FP32 accumulation in tensor memory.
//
// One CTA of five warps per (block, bin), warp-specialised.  Lane 0 of
// warp 4 loads the block's B tile once and the bin's A tiles (128 directions
// each) through TMA with the 128-byte swizzle into a two-stage ring, and
// issues each tile's MMAs into one of two TMEM accumulators, committing them
// to mbarriers (accumulator full, A stage empty).  Warps 0-3 read their 32
// TMEM lanes of the finished accumulator (one direction per thread), fold
// the NP accumulator columns into the denominator of eq. 5 (sum of |y| or
// |y|^2), release the accumulator and write P; meanwhile the next tile's MMAs
// run into the other accumulator and the tile after that is being loaded.
// Every wait is bounded: on expiry the kernel raises SSL_FLAG_TIMEOUT, stops,
// waits (bounded) for its own copies and MMAs in flight, and still releases
// its tensor memory.
#include <cuda.h>
#include <cuda_bf16.h>
#include <float.h>
#include <string.h>

#include "ssl_internal.cuh"

namespace ssl {
namespace {

constexpr int kEpiThreads = 128;                 // warps 0-3: epilogue
constexpr int kThreads = kEpiThreads + 32;       // warp 4: loads and MMAs
constexpr int kTileM = 128;        // directions per MMA tile
constexpr uint32_t kWaitLimit = 1u << 22;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}
// Bounded wait on the given phase parity; false if the limit expired.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  for (uint32_t i = 0; i < kWaitLimit; ++i) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* tm, int c0, int c1,
                                            int c2, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(tm)), "r"(c0), "r"(c1), "r"(c2), "r"(bar)
      : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, 8-row
// core-matrix groups 1024 bytes apart (SBO), descriptor version 1.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFF) >> 4);          // start address
  d |= (uint64_t)1 << 16;                          // leading byte offset (unused here)
  d |= (uint64_t)(1024 >> 4) << 32;                // stride byte offset
  d |= (uint64_t)1 << 46;                          // version
  d |= (uint64_t)2 << 61;                          // 128-byte swizzle
  return d;
}

// Instruction descriptor: FP32 accumulator, A/B of format `fmt` (1 = BF16,
// 2 = TF32), both K-major, M = 128, N = n.
__device__ __forceinline__ uint32_t instr_desc(uint32_t fmt, uint32_t n) {
  return (1u << 4) | (fmt << 7) | (fmt << 10) | ((n >> 3) << 17) | ((uint32_t)(kTileM >> 4) << 24);
}

template <int ESZ>
__device__ __forceinline__ void mma(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc,
                                    uint32_t acc) {
  if (ESZ == 2) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
  } else {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
  }
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
      : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
        "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_wait_ld() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ float sqrt_approx(float x) {
  float r;
  asm("sqrt.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

template <int ESZ>
__global__ void __launch_bounds__(kThreads)
spectrum_tc_kernel(const __grid_constant__ CUtensorMap tmH, const __grid_constant__ CUtensorMap tmE,
                   int B, int D, int M, int Ns, int KP, int NP, uint32_t tmem_cols, int form,
                   const float* __restrict__ hnorm2, float* __restrict__ P, unsigned* flags,
                   const CUtensorMap* __restrict__ tmH_items,
                   const float* const* __restrict__ hn_items,
                   const MixedItem* __restrict__ mitems, const int2* __restrict__ mctab) {
  extern __shared__ uint8_t smem_raw[];
  constexpr int kAtomElems = 128 / ESZ;  // elements per 128-byte swizzle row
  constexpr int kKStep = 32 / ESZ;       // K per MMA instruction (32 bytes)
  uint8_t* smem = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  // a_full[2], a_empty[2], acc_full[2], acc_empty[2], b_full
  __shared__ __align__(8) uint64_t bars[9];
  __shared__ uint32_t tmem_sh;
  __shared__ int abort_sh;

  // blocks vary fastest so that the CTAs of one bin run together and its
  // steering tiles are served from L2
  int blk = blockIdx.x, bin = blockIdx.y;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // per-array steering (serving) or the shared one (stateless calls)
  const CUtensorMap* tmA = tmH_items ? tmH_items + blk : &tmH;
  const CUtensorMap* tmB = &tmE;
  const float* hn = hn_items ? hn_items[blk] : hnorm2;
  int ecoord = blk * B + bin;
  size_t prow = ((size_t)blk * B + bin) * D;
  if (mitems) {  // mixed batch: the CTA's (array, bin) and that array's shapes
    const int2 cb = mctab[blockIdx.x];
    const MixedItem& it = mitems[cb.x];
    bin = cb.y;
    tmA = &it.tmH;
    tmB = &it.tmE;
    hn = it.hn;
    P = it.P;
    D = it.D;
    M = it.M;
    Ns = it.Ns;
    KP = it.KP;
    NP = it.NP;
    ecoord = bin;
    prow = (size_t)bin * D;
    tmem_cols = 32;
    while ((int)tmem_cols < NP) tmem_cols <<= 1;
  }
  const int ndt = ceil_div(D, kTileM);
  const int N = M - Ns;
  const int natoms = KP / kAtomElems;
  const uint32_t a_bytes = natoms * kTileM * 128;
  const uint32_t b_bytes = natoms * NP * 128;
  // A stages at smem and smem + a_bytes (natoms x [128 rows][128 B] each),
  // then B (natoms x [NP rows][128 B])
  const uint32_t sA0 = smem_u32(smem);
  uint8_t* const sB = smem + 2 * a_bytes;
  const uint32_t bar0 = smem_u32(&bars[0]);
  auto a_full = [&](int st) { return bar0 + 8u * st; };
  auto a_empty = [&](int st) { return bar0 + 8u * (2 + st); };
  auto acc_full = [&](int st) { return bar0 + 8u * (4 + st); };
  auto acc_empty = [&](int st) { return bar0 + 8u * (6 + st); };
  const uint32_t b_full = bar0 + 8u * 8;

  // two accumulators of tmem_cols columns: tile dt accumulates into dt & 1
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_sh)),
                 "r"(2 * tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    for (int i = 0; i < 6; ++i) mbar_init(bar0 + 8u * i, 1);
    mbar_init(acc_empty(0), kEpiThreads);
    mbar_init(acc_empty(1), kEpiThreads);
    mbar_init(b_full, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    abort_sh = 0;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_sh;

  if (warp == kEpiThreads / 32) {
    // ---- producer: one lane loads the operands and issues the MMAs ----
    if (lane == 0 && ndt > 0) {
      // A tensor map read from global memory (per-array steering) is made
      // visible to the tensor-map proxy before its first use.
      if (tmH_items || mitems)
        asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(
                         reinterpret_cast<uint64_t>(tmA))
                     : "memory");
      if (mitems)
        asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(
                         reinterpret_cast<uint64_t>(tmB))
                     : "memory");
      mbar_expect_tx(b_full, b_bytes);
      for (int j = 0; j < natoms; ++j)
        tma_load_3d(smem_u32(sB + j * NP * 128), tmB, j * kAtomElems, 0, ecoord, b_full);
      mbar_expect_tx(a_full(0), a_bytes);
      for (int j = 0; j < natoms; ++j)
        tma_load_3d(sA0 + j * kTileM * 128, tmA, j * kAtomElems, 0, bin, a_full(0));
      const uint32_t idesc = instr_desc(ESZ == 2 ? 1u : 2u, (uint32_t)NP);
      const int ksteps = KP / kKStep;
      int a_issued = 1;   // A tiles whose loads were issued
      int mma_issued = 0;  // tiles whose MMAs were issued
      bool ok = mbar_wait(b_full, 0);
      for (int dt = 0; ok && dt < ndt; ++dt) {
        const int st = dt & 1;
        ok = mbar_wait(a_full(st), (dt >> 1) & 1) &&
             mbar_wait(acc_empty(st), ((dt >> 1) & 1) ^ 1) && !*(volatile int*)&abort_sh;
        if (!ok) break;
        tc_fence_after();
        for (int kk = 0; kk < ksteps; ++kk) {
          const int j = kk / 4, off = (kk % 4) * 32;
          const uint64_t a = smem_desc(sA0 + st * a_bytes + j * kTileM * 128 + off);
          const uint64_t b = smem_desc(smem_u32(sB + j * NP * 128) + off);
          mma<ESZ>(tmem + (uint32_t)st * tmem_cols, a, b, idesc, kk > 0 ? 1u : 0u);
        }
        mma_commit(acc_full(st));
        mma_commit(a_empty(st));
        mma_issued = dt + 1;
        // refill: A(dt + 1) goes to the stage MMA(dt - 1) read
        if (dt + 1 < ndt) {
          const int sn = (dt + 1) & 1;
          if (dt >= 1) ok = mbar_wait(a_empty(sn), ((dt - 1) >> 1) & 1);
          if (!ok) break;
          mbar_expect_tx(a_full(sn), a_bytes);
          for (int j = 0; j < natoms; ++j)
            tma_load_3d(sA0 + sn * a_bytes + j * kTileM * 128, tmA, j * kAtomElems,
                        (dt + 1) * kTileM, bin, a_full(sn));
          a_issued = dt + 2;
        }
      }
      // Drain before teardown: the last MMAs have signalled their stage
      // (so no tensor-core write to TMEM or read of shared memory is left),
      // and, after an abort, every issued A load has landed.
      if (mma_issued > 0) {
        const int t = mma_issued - 1;
        mbar_wait(a_empty(t & 1), (t >> 1) & 1);
      }
      if (!ok) {
        atomicExch(&abort_sh, 1);
        for (int t = mma_issued; t < a_issued; ++t) mbar_wait(a_full(t & 1), (t >> 1) & 1);
        if (mma_issued == 0) mbar_wait(b_full, 0);
      }
    }
  } else {
    // ---- epilogue: warp w reads TMEM lanes 32w .. 32w + 31, one direction
    // per thread, and folds the NP accumulator columns into eq. 5 ----
    for (int dt = 0; dt < ndt; ++dt) {
      const int st = dt & 1;
      if (!mbar_wait(acc_full(st), (dt >> 1) & 1) || *(volatile int*)&abort_sh) {
        atomicExch(&abort_sh, 1);
        break;
      }
      tc_fence_after();
      float den = 0.f;
      const uint32_t trow = tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)st * tmem_cols;
      for (int c0 = 0; c0 < NP; c0 += 64) {
        float v[4][16];
#pragma unroll
        for (int q = 0; q < 4; ++q)
          if (c0 + 16 * q < NP) tmem_ld16(trow + c0 + 16 * q, v[q]);
        tmem_wait_ld();
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const int i = (c0 + 16 * q) / 2 + j;
            if (c0 + 16 * q < NP && i < N) {
              const float s2 = fmaf(v[q][2 * j], v[q][2 * j], v[q][2 * j + 1] * v[q][2 * j + 1]);
              den += form == SSL_FORM_SQ ? s2 : sqrt_approx(s2);
            }
          }
      }
      tc_fence_before();
      mbar_arrive(acc_empty(st));  // this accumulator may be overwritten
      const int d = dt * kTileM + 32 * warp + lane;
      if (d < D) P[prow + d] = hn[(size_t)bin * D + d] / fmaxf(den, FLT_MIN);
    }
  }

  // Teardown: release the tensor memory once every warp is done with it.
  tc_fence_before();
  __syncthreads();
  if (tid == 0 && abort_sh) atomicOr(flags, SSL_FLAG_TIMEOUT);
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(2 * tmem_cols)
                 : "memory");
  }
}

// ---- operand images ---------------------------------------------------------

__device__ __forceinline__ float to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

template <int ESZ>
__device__ __forceinline__ void put(void* base, size_t i, float x) {
  if (ESZ == 2)
    reinterpret_cast<__nv_bfloat16*>(base)[i] = __float2bfloat16_rn(x);
  else
    reinterpret_cast<float*>(base)[i] = to_tf32(x);
}

// H [B][D][M] c64 -> A image [B][D][KP].
template <int ESZ>
__global__ void pack_h_kernel(const float2* __restrict__ H, int BD, int M, int KP, void* out) {
  const size_t n = (size_t)BD * KP;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n;
       e += (size_t)gridDim.x * blockDim.x) {
    const size_t row = e / KP;
    const int k = (int)(e % KP);
    float x = 0.f;
    if (k < M)
      x = H[row * M + k].x;
    else if (k < 2 * M)
      x = H[row * M + k - M].y;
    put<ESZ>(out, e, x);
  }
}

// E [nblk*B][M][M] c64 -> B image [nblk*B][NP][KP].
template <int ESZ>
__global__ void pack_e_kernel(const float2* __restrict__ E, int M, int Ns, int KP, int NP,
                              void* out) {
  const size_t mat = blockIdx.x;
  const float2* Eb = E + mat * M * M;
  const size_t base = mat * NP * KP;
  const int N = M - Ns;
  for (int e = threadIdx.x; e < NP * KP; e += blockDim.x) {
    const int n = e / KP, k = e % KP;
    const int i = n >> 1;
    float x = 0.f;
    if (i < N && k < 2 * M) {
      const int m = k < M ? k : k - M;
      const float2 v = Eb[m * M + Ns + i];
      if ((n & 1) == 0)
        x = k < M ? v.x : v.y;
      else
        x = k < M ? v.y : -v.x;
    }
    put<ESZ>(out, base + e, x);
  }
}

// Mixed batch: one CTA per (item, bin).
template <int ESZ>
__global__ void pack_e_mixed_kernel(const MixedItem* __restrict__ items,
                                    const int2* __restrict__ ctab) {
  const int2 cb = ctab[blockIdx.x];
  const MixedItem& it = items[cb.x];
  const int M = it.M, Ns = it.Ns, KP = it.KP, NP = it.NP;
  const float2* Eb = it.E + (size_t)cb.y * M * M;
  const size_t base = (size_t)cb.y * NP * KP;
  const int N = M - Ns;
  for (int e = threadIdx.x; e < NP * KP; e += blockDim.x) {
    const int n = e / KP, k = e % KP;
    const int i = n >> 1;
    float x = 0.f;
    if (i < N && k < 2 * M) {
      const int m = k < M ? k : k - M;
      const float2 v = Eb[m * M + Ns + i];
      if ((n & 1) == 0)
        x = k < M ? v.x : v.y;
      else
        x = k < M ? v.y : -v.x;
    }
    put<ESZ>(it.eimg, base + e, x);
  }
}

}  // namespace

int tc_kp(int M) { return 2 * M <= 64 ? 64 : 128; }
int tc_np(int M, int Ns) { return ((2 * (M - Ns) + 15) / 16) * 16; }

cudaError_t launch_pack_h(const float2* H, int B, int D, int M, int precision, void* out,
                          cudaStream_t s) {
  const int KP = tc_kp(M);
  const int BD = B * D;
  const int blocks = 1024;
  if (precision == SSL_PREC_BF16)
    pack_h_kernel<2><<<blocks, 256, 0, s>>>(H, BD, M, KP, out);
  else
    pack_h_kernel<4><<<blocks, 256, 0, s>>>(H, BD, M, KP, out);
  return cudaGetLastError();
}

cudaError_t launch_pack_e(const float2* E, int nmat, int M, int Ns, int precision, void* out,
                          cudaStream_t s) {
  const int KP = tc_kp(M), NP = tc_np(M, Ns);
  if (precision == SSL_PREC_BF16)
    pack_e_kernel<2><<<nmat, 256, 0, s>>>(E, M, Ns, KP, NP, out);
  else
    pack_e_kernel<4><<<nmat, 256, 0, s>>>(E, M, Ns, KP, NP, out);
  return cudaGetLastError();
}

size_t tc_smem_bytes(int M, int Ns, int precision) {
  const int esz = precision == SSL_PREC_BF16 ? 2 : 4;
  const int natoms = tc_kp(M) * esz / 128;
  return 1024 + (size_t)natoms * 128 * (2 * kTileM + tc_np(M, Ns));
}

cudaError_t launch_spectrum_tc(const CUtensorMap& tmH, const CUtensorMap& tmE, int nblk, int B,
                               int D, int M, int Ns, int precision, int form,
                               const float* hnorm2, float* P, unsigned* flags, cudaStream_t s,
                               const CUtensorMap* tmH_items, const float* const* hn_items) {
  const int KP = tc_kp(M), NP = tc_np(M, Ns);
  uint32_t cols = 32;
  while ((int)cols < NP) cols <<= 1;
  const size_t smem = tc_smem_bytes(M, Ns, precision);
  dim3 grid(nblk, B);
  cudaError_t e;
  if (precision == SSL_PREC_BF16) {
    e = cudaFuncSetAttribute(spectrum_tc_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
    if (e != cudaSuccess) return e;
    spectrum_tc_kernel<2><<<grid, kThreads, smem, s>>>(tmH, tmE, B, D, M, Ns, KP, NP, cols, form,
                                                        hnorm2, P, flags, tmH_items, hn_items, nullptr,
                                                        nullptr);
  } else {
    e = cudaFuncSetAttribute(spectrum_tc_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
    if (e != cudaSuccess) return e;
    spectrum_tc_kernel<4><<<grid, kThreads, smem, s>>>(tmH, tmE, B, D, M, Ns, KP, NP, cols, form,
                                                        hnorm2, P, flags, tmH_items, hn_items, nullptr,
                                                        nullptr);
  }
  return cudaGetLastError();
}

cudaError_t launch_pack_e_mixed(const MixedItem* items, const int2* ctab, int n_ctab,
                                int precision, cudaStream_t s) {
  if (n_ctab <= 0) return cudaSuccess;
  if (precision == SSL_PREC_BF16)
    pack_e_mixed_kernel<2><<<n_ctab, 256, 0, s>>>(items, ctab);
  else
    pack_e_mixed_kernel<4><<<n_ctab, 256, 0, s>>>(items, ctab);
  return cudaGetLastError();
}

// Mixed batch: one CTA per (item, bin), shapes and tensor maps from the
// item; shared memory sized for the largest operands (M = 64, Ns = 1).
cudaError_t launch_spectrum_tc_mixed(const MixedItem* items, const int2* ctab, int n_ctab,
                                     int precision, int form, unsigned* flags, cudaStream_t s) {
  if (n_ctab <= 0) return cudaSuccess;
  const size_t smem = tc_smem_bytes(SSL_MAX_M, 1, precision);
  CUtensorMap dummy;
  memset(&dummy, 0, sizeof(dummy));
  cudaError_t e;
  if (precision == SSL_PREC_BF16) {
    e = cudaFuncSetAttribute(spectrum_tc_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
    if (e != cudaSuccess) return e;
    spectrum_tc_kernel<2><<<n_ctab, kThreads, smem, s>>>(dummy, dummy, 0, 0, 0, 0, 0, 0, 32, form,
                                                         nullptr, nullptr, flags, nullptr,
                                                         nullptr, items, ctab);
  } else {
    e = cudaFuncSetAttribute(spectrum_tc_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
    if (e != cudaSuccess) return e;
    spectrum_tc_kernel<4><<<n_ctab, kThreads, smem, s>>>(dummy, dummy, 0, 0, 0, 0, 0, 0, 32, form,
                                                         nullptr, nullptr, flags, nullptr,
                                                         nullptr, items, ctab);
  }
  return cudaGetLastError();
}

}  // namespace ssl
