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
// Persistent and warp-specialised: one CTA of 18 warps per SM walks the
// items: with BF16 operands a bin and two blocks, whose noise images are
// stacked into one B operand of 2 NP rows so that each steering tile feeds
// both in one MMA (N = 2 NP); otherwise a (block, bin).  Lane 0 of warp 16
// streams each item's B image(s) and its A tiles (128 directions each)
// through TMA with the 128-byte swizzle into shared-memory rings (three A
// stages and two B stages for BF16, two and one for TF32); lane 0 of warp 17
// issues each tile's MMAs into one of the TMEM accumulators (two of 256
// columns, or four of 128) and commits them to mbarriers (accumulator full,
// stages empty); four epilogue warpgroups, one or two per accumulator (then
// one per block of the item), read their 32 TMEM lanes per warp (one
// direction per thread), fold their block's accumulator columns into the
// denominator of eq. 5 (sum of |y| or |y|^2), release the accumulator and
// write P.  Loads, MMAs and epilogues of
// different tiles overlap, across item boundaries too.  Every wait is
// bounded: on expiry the kernel raises SSL_FLAG_TIMEOUT, stops, waits
// (bounded) for its own copies and MMAs in flight, and still releases its
// tensor memory.
#include <cuda.h>
#include <cuda_bf16.h>
#include <float.h>
#include <string.h>

#include "ssl_internal.cuh"

namespace ssl {
namespace {

constexpr int kEpiWarps = 16;                    // warps 0-15: epilogue
constexpr int kEpiThreads = 32 * kEpiWarps;
constexpr int kThreads = kEpiThreads + 64;       // warp 16: loads, warp 17: MMAs
constexpr int kTileM = 128;        // directions per MMA tile
constexpr uint64_t kWaitNs = 250000000ull;  // 0.25 s per wait (default limit)
constexpr uint32_t kSuspendNs = 20000;        // suspend hint of one try_wait

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
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Bounded wait on the given phase parity: false once limit_ns have passed or
// another role of the CTA has raised *abort_flag (then the caller stops too).
// Each try_wait may suspend the warp for up to kSuspendNs, so that waiting
// warps do not take issue slots from the working ones.  The pipeline's waits
// take the launch's limit; the waits that drain a role's own copies and MMAs
// after an abort always take kWaitNs, so that nothing of the CTA is still in
// flight when it releases its tensor memory and exits.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity,
                                          const volatile int* abort_flag = nullptr,
                                          uint64_t limit_ns = kWaitNs) {
  const uint64_t t0 = global_ns();
  for (;;) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity), "n"(kSuspendNs)
        : "memory");
    if (done) return true;
    if (global_ns() - t0 > limit_ns) return false;
    if (abort_flag && *abort_flag) return false;
  }
}

// The same bounded wait without suspending: test_wait polls and returns at
// once, so the single-lane pipeline roles (loads, MMAs, tile generation) see a
// phase complete with no wake-up delay; the time limit and abort flag are
// checked every 32 polls.
__device__ __forceinline__ bool mbar_wait_spin(uint32_t bar, uint32_t parity,
                                               const volatile int* abort_flag = nullptr,
                                               uint64_t limit_ns = kWaitNs) {
  const uint64_t t0 = global_ns();
  for (uint32_t n = 1;; ++n) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
    if ((n & 31) == 0) {
      if (global_ns() - t0 > limit_ns) return false;
      if (abort_flag && *abort_flag) return false;
    }
  }
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
// acc + (a.x^2, a.y^2) as one packed two-lane FMA
__device__ __forceinline__ uint64_t fma_sq2(float ax, float ay, uint64_t acc) {
  uint64_t a, r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(a) : "f"(ax), "f"(ay));
  asm("fma.rn.f32x2 %0, %1, %1, %2;" : "=l"(r) : "l"(a), "l"(acc));
  return r;
}
__device__ __forceinline__ float sum2(uint64_t v) {
  float x, y;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(x), "=f"(y) : "l"(v));
  return x + y;
}
__device__ __forceinline__ void tmem_wait_ld() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// |y| from |y|^2 with one reciprocal-square-root estimate (zero stays zero)
__device__ __forceinline__ float sqrt_approx(float x) { return x * rsqrtf(fmaxf(x, FLT_MIN)); }

// The denominator of eq. 5 for the thread's direction (its TMEM lane) from
// the accumulator columns tg .. tg + NP - 1, which hold (Re, Im) of h^H e_i in
// columns (2i, 2i + 1); the zero rows that pad a noise image past 2N
// contribute 0 to either sum.  NP is a multiple of 16: chunks of 16 columns.
__device__ __forceinline__ float fold_den(uint32_t tg, int NP, int form) {
  if (form == SSL_FORM_SQ) {
    uint64_t acc2 = 0ull;  // (sum Re^2, sum Im^2)
    for (int c0 = 0; c0 < NP; c0 += 16) {
      float v[16];
      tmem_ld16(tg + c0, v);
      tmem_wait_ld();
#pragma unroll
      for (int j = 0; j < 8; ++j) acc2 = fma_sq2(v[2 * j], v[2 * j + 1], acc2);
    }
    return sum2(acc2);
  }
  float s0 = 0.f, s1 = 0.f;
  for (int c0 = 0; c0 < NP; c0 += 16) {
    float v[16];
    tmem_ld16(tg + c0, v);
    tmem_wait_ld();
#pragma unroll
    for (int j = 0; j < 8; j += 2) {
      s0 += sqrt_approx(fmaf(v[2 * j], v[2 * j], v[2 * j + 1] * v[2 * j + 1]));
      s1 += sqrt_approx(fmaf(v[2 * j + 2], v[2 * j + 2], v[2 * j + 3] * v[2 * j + 3]));
    }
  }
  return s0 + s1;
}

// Generator warps of the analytic-steering mode (after the load and MMA warps).
constexpr int kGenWarps = 8;
constexpr int kGenThreads = 32 * kGenWarps;
constexpr int kGenRows = kTileM / kGenWarps;  // rows per generator warp: gw + 8 q
static_assert(kGenRows * kGenWarps == kTileM && kGenRows <= 32 && kGenRows % 4 == 0,
              "each generator lane fetches one row's direction; rows go four at a time");
constexpr int kGenWarp0 = kEpiWarps + 2;

// Shared-memory byte address of element (r, k) of a 128-row K-major operand
// tile written the way a TMA load with the 128-byte swizzle writes it: K atoms
// of 128 bytes per row, atom j of the tile kTileM * 128 bytes after atom j - 1,
// and the 16-byte chunk c of row r of an atom stored at chunk c ^ (r % 8)
// (the tile bases are 1024-byte aligned).
template <int ESZ>
__device__ __forceinline__ uint32_t a_tile_addr(uint32_t base, int r, int k) {
  constexpr int kPer = 128 / ESZ;  // elements per 128-byte atom row
  const int j = k / kPer, byte = (k % kPer) * ESZ;
  return base + j * (kTileM * 128) + r * 128 + ((((byte >> 4) ^ (r & 7)) << 4) | (byte & 15));
}

template <int ESZ>
__device__ __forceinline__ void st_shared_zero(uint32_t addr) {
  if (ESZ == 2)
    asm volatile("st.shared.u16 [%0], %1;" ::"r"(addr), "h"((unsigned short)0) : "memory");
  else
    asm volatile("st.shared.u32 [%0], %1;" ::"r"(addr), "r"(0u) : "memory");
}

// Elements k and k + 1 (k = m or M + m, m even) of row r from two values; the
// second only when `two` (it falls past the last microphone otherwise).  BF16:
// one 32-bit store when k is even (M even), else two 16-bit stores; TF32: the
// values rounded to TF32, one 32-bit store each.
template <int ESZ>
__device__ __forceinline__ void st_pair(uint32_t base, int r, int k, int M, float a, float b,
                                        bool two) {
  if (ESZ == 2) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    const uint32_t w = *reinterpret_cast<const uint32_t*>(&h);
    if (two && (k & 1) == 0) {
      asm volatile("st.shared.u32 [%0], %1;" ::"r"(a_tile_addr<2>(base, r, k)), "r"(w)
                   : "memory");
    } else {
      asm volatile("st.shared.u16 [%0], %1;" ::"r"(a_tile_addr<2>(base, r, k)),
                   "h"((unsigned short)(w & 0xffffu))
                   : "memory");
      if (two)
        asm volatile("st.shared.u16 [%0], %1;" ::"r"(a_tile_addr<2>(base, r, k + 1)),
                     "h"((unsigned short)(w >> 16))
                     : "memory");
    }
  } else {
    uint32_t ta, tb;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(ta) : "f"(a));
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(tb) : "f"(b));
    asm volatile("st.shared.u32 [%0], %1;" ::"r"(a_tile_addr<4>(base, r, k)), "r"(ta) : "memory");
    if (two)
      asm volatile("st.shared.u32 [%0], %1;" ::"r"(a_tile_addr<4>(base, r, k + 1)), "r"(tb)
                   : "memory");
  }
  (void)M;
}

// cos and sin of 2 pi t for a phase t in turns: t is first reduced to
// [-1/2, 1/2] (exactly, t - rint(t)), so that the fast hardware sine and cosine
// see an argument in [-pi, pi], where their absolute error is about 2^-21 -
// below the TF32 (2^-11) and BF16 (2^-8) rounding the tile goes through.
__device__ __forceinline__ void steer_cs(float t, float& c, float& s) {
  const float tr = t - rintf(t);
  __sincosf(6.28318530717958647692f * tr, &s, &c);
}

// Pipeline depths: A stages (steering tiles), B stages (noise-subspace
// images), and the blocks per item (kG): with BF16 operands the stateless
// launch pairs two blocks of a bin, which share every steering tile, into one
// MMA of N = 2 NP columns (the tile is then read from shared memory once for
// both blocks, which halves the operand bandwidth per output).  TMEM holds
// 512 / (128 kG) accumulators of 128 kG columns.
template <int ESZ>
struct Pipe {
  static constexpr int kG = ESZ == 2 ? 2 : 1;
  static constexpr int kSA = ESZ == 2 ? 3 : 2;
  static constexpr int kSB = ESZ == 2 ? 2 : 1;
  static constexpr int kAtoms = 128 * ESZ / 128;                  // KP = 128
  static constexpr uint32_t kABytes = kAtoms * kTileM * 128;      // one A stage
  static constexpr uint32_t kBBytes = kG * kAtoms * 128 * 128;    // one B stage (NP <= 128)
  static constexpr int kAccCols = 128 * kG;
  static constexpr int kAcc = 512 / kAccCols;
  static constexpr size_t kSmem = 1024 + kSA * kABytes + kSB * kBBytes;
};

// One work item: G (1 or 2) blocks of one bin of the stateless and serving
// launches, or an (array, bin) of a mixed batch, with its operands' shapes.
struct Item {
  const CUtensorMap* tmA;
  const CUtensorMap* tmB;
  const Geo* geo;   // analytic steering (A tiles generated), else nullptr
  const float* hn;  // |h|^2, [D] of this bin (nullptr with geo: |h|^2 = M)
  float* P[2];      // [D] of each block
  int ecoord[2];    // noise-image coordinate of each block
  int D, N, KP, NP, bin, ndt, G, M;
};

// Items per launch: bins x ceil(nblk / G) (stateless), or the table's rows.
__device__ __host__ __forceinline__ int pair_count(int nblk, int G) { return (nblk + G - 1) / G; }

__device__ __forceinline__ Item item_of(int i, int G, const CUtensorMap* tmH,
                                        const CUtensorMap* tmE, int nblk, int B, int D, int M,
                                        int Ns, int KP, int NP, const float* hnorm2, float* P,
                                        const CUtensorMap* tmH_items,
                                        const float* const* hn_items, const MixedItem* mitems,
                                        const int2* mctab, const Geo* geo,
                                        const Geo* const* geo_items) {
  Item it;
  it.geo = nullptr;
  if (mitems) {
    const int2 cb = mctab[i];
    const MixedItem& m = mitems[cb.x];
    it.tmA = &m.tmH;
    it.tmB = &m.tmE;
    it.bin = cb.y;
    it.D = m.D;
    it.M = m.M;
    it.N = m.M - m.Ns;
    it.KP = m.KP;
    it.NP = m.NP;
    it.G = 1;
    it.ecoord[0] = it.ecoord[1] = cb.y;
    it.hn = m.hn + (size_t)cb.y * m.D;
    it.P[0] = it.P[1] = m.P + (size_t)cb.y * m.D;
  } else {
    // blocks vary fastest so that the items in flight share a bin and its
    // steering tiles are served from L2
    const int np = pair_count(nblk, G);
    const int blk = (i % np) * G, bin = i / np;
    it.G = blk + 1 < nblk ? G : 1;
    it.tmA = tmH_items ? tmH_items + blk : tmH;
    it.tmB = tmE;
    it.geo = geo_items ? geo_items[blk] : geo;
    it.bin = bin;
    it.D = D;
    it.M = M;
    it.N = M - Ns;
    it.KP = KP;
    it.NP = NP;
    it.hn = it.geo ? nullptr : (hn_items ? hn_items[blk] : hnorm2) + (size_t)bin * D;
    for (int g = 0; g < 2; ++g) {
      const int b = g < it.G ? blk + g : blk;
      it.ecoord[g] = b * B + bin;
      it.P[g] = P + ((size_t)b * B + bin) * D;
    }
  }
  it.ndt = ceil_div(it.D, kTileM);
  return it;
}

// Persistent, warp-specialised: one CTA per SM walks the items i = blockIdx.x,
// blockIdx.x + gridDim.x, ...  Warp 16 (one lane) streams the B image of each
// item and its A tiles into shared-memory rings; warp 17 (one lane) issues
// each tile's MMAs into one of the TMEM accumulators (tile g into g % kAcc);
// the epilogue warpgroups of that accumulator (warps 4 wg .. 4 wg + 3, warp w
// reading TMEM lanes 32 (w % 4) .. + 31, one direction per thread) read it,
// release it, and write P.  Four warpgroups keep several tiles' epilogues in
// flight, so their latency (TMEM reads, the |h|^2 load) overlaps.  All hand-offs are
// mbarriers; every wait is bounded.
template <int ESZ, bool kGen>
__global__ void __launch_bounds__(kThreads + kGenThreads, 1)
spectrum_tc_kernel(const __grid_constant__ CUtensorMap tmH, const __grid_constant__ CUtensorMap tmE,
                   int nitems, int nblk, int B, int D, int M, int Ns, int KP, int NP, int form,
                   const float* __restrict__ hnorm2, float* __restrict__ P, unsigned* flags,
                   const CUtensorMap* __restrict__ tmH_items,
                   const float* const* __restrict__ hn_items,
                   const MixedItem* __restrict__ mitems, const int2* __restrict__ mctab,
                   uint64_t wait_ns, const Geo* geo, const Geo* const* __restrict__ geo_items,
                   int stall) {
  using PP = Pipe<ESZ>;
  constexpr int kAtomElems = 128 / ESZ;  // elements per 128-byte swizzle row
  constexpr int kKStep = 32 / ESZ;       // K per MMA instruction (32 bytes)
  constexpr int SA = PP::kSA, SB = PP::kSB, kAcc = PP::kAcc;
  constexpr uint32_t kAccCols = PP::kAccCols;
  // two blocks per item only where they share the steering table
  const int G = (tmH_items || mitems || geo_items) ? 1 : PP::kG;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  // a_full[SA], a_empty[SA], b_full[SB], b_empty[SB], acc_full[4], acc_empty[4]
  __shared__ __align__(8) uint64_t bars[2 * SA + 2 * SB + 2 * kAcc];
  __shared__ uint32_t tmem_sh;
  __shared__ int abort_sh;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t bar0 = smem_u32(&bars[0]);
  auto a_full = [&](int st) { return bar0 + 8u * st; };
  auto a_empty = [&](int st) { return bar0 + 8u * (SA + st); };
  auto b_full = [&](int st) { return bar0 + 8u * (2 * SA + st); };
  auto b_empty = [&](int st) { return bar0 + 8u * (2 * SA + SB + st); };
  auto acc_full = [&](int st) { return bar0 + 8u * (2 * SA + 2 * SB + st); };
  auto acc_empty = [&](int st) { return bar0 + 8u * (2 * SA + 2 * SB + kAcc + st); };
  const uint32_t sA0 = smem_u32(smem);
  const uint32_t sB0 = sA0 + SA * PP::kABytes;
  const CUtensorMap* tmHp = &tmH;
  const CUtensorMap* tmEp = &tmE;
  auto item = [&](int i) {
    return item_of(i, G, tmHp, tmEp, nblk, B, D, M, Ns, KP, NP, hnorm2, P, tmH_items, hn_items,
                   mitems, mctab, geo, geo_items);
  };

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_sh)),
                 "r"(kAccCols * kAcc)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    for (int i = 0; i < 2 * SA + 2 * SB + kAcc; ++i) mbar_init(bar0 + 8u * i, 1);
    // generated A tiles: one arrival per generator warp
    if (kGen)
      for (int i = 0; i < SA; ++i) mbar_init(a_full(i), kGenWarps);
    for (int i = 0; i < kAcc; ++i) mbar_init(acc_empty(i), kEpiThreads / kAcc);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    abort_sh = 0;
  }
  if (kGen && warp >= kGenWarp0) {
    // the padding columns 2M .. KP - 1 of every A stage are zero and are
    // never written again
    for (int e = tid - kGenWarp0 * 32; e < SA * kTileM * (KP - 2 * M); e += kGenThreads) {
      const int sa = e / (kTileM * (KP - 2 * M)), rem = e % (kTileM * (KP - 2 * M));
      const int r = rem / (KP - 2 * M), k = 2 * M + rem % (KP - 2 * M);
      st_shared_zero<ESZ>(a_tile_addr<ESZ>(sA0 + sa * PP::kABytes, r, k));
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_sh;
  volatile int* abort_v = &abort_sh;

  if (kGen && warp >= kGenWarp0) {
    // ---- A tiles generated from the analytic steering: warp gw of the
    // generators writes rows gw, gw + 4, ... of each 128-direction tile; lane
    // l the microphone pair (2l, 2l + 1) ----
    const int gw = warp - kGenWarp0;
    int ia = 0;
    bool ok = true;
    // the geometry of the previous item stays in registers (the stateless
    // launch has one array; serving items change arrays)
    const Geo* last = nullptr;
    Geo g{};
    const int m0 = 2 * lane, m1 = 2 * lane + 1;
    bool has0 = false, has1 = false;
    float p0x = 0.f, p0y = 0.f, p0z = 0.f, p1x = 0.f, p1y = 0.f, p1z = 0.f;
    for (int i = blockIdx.x; ok && i < nitems; i += gridDim.x) {
      const Item it = item(i);
      if (it.geo != last) {
        last = it.geo;
        g = *it.geo;
        has0 = m0 < g.M;
        has1 = m1 < g.M;
        if (has0) {
          p0x = __ldg(g.pos + 3 * m0);
          p0y = __ldg(g.pos + 3 * m0 + 1);
          p0z = __ldg(g.pos + 3 * m0 + 2);
        }
        if (has1) {
          p1x = __ldg(g.pos + 3 * m1);
          p1y = __ldg(g.pos + 3 * m1 + 1);
          p1z = __ldg(g.pos + 3 * m1 + 2);
        }
      }
      const float fcw = __ldg(g.fc + it.bin);
      // lane l fetches the direction of row gw + kGenWarps l (the warp's rows)
      // of a tile; the next tile's are fetched while this one is generated
      auto fetch_u = [&](int dt, float& x, float& y, float& z) {
        const int r = gw + kGenWarps * lane;
        const int dl = dt * kTileM + r;
        x = y = z = 0.f;
        if (dt < it.ndt && lane < kGenRows && dl < it.D) {
          x = __ldg(g.dirs + 3 * dl);
          y = __ldg(g.dirs + 3 * dl + 1);
          z = __ldg(g.dirs + 3 * dl + 2);
        }
      };
      float nx, ny, nz;
      fetch_u(0, nx, ny, nz);
      for (int dt = 0; dt < it.ndt; ++dt) {
        const float uxl = nx, uyl = ny, uzl = nz;
        fetch_u(dt + 1, nx, ny, nz);
        const int sa = ia % SA;
        // warp-uniform outcome: every lane reaches the __syncwarp below
        ok = __all_sync(0xffffffffu,
                        mbar_wait_spin(a_empty(sa), ((ia / SA) & 1) ^ 1, abort_v, wait_ns));
        if (!ok) break;
        const uint32_t base = sA0 + sa * PP::kABytes;
        // four rows at a time: their phases, then their sines and cosines,
        // then their stores, so that the four chains overlap (the directions
        // arrive by shuffles)
#pragma unroll
        for (int q0 = 0; q0 < kGenRows; q0 += 4) {
          float ta[4], tb[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const float ux = __shfl_sync(0xffffffffu, uxl, q0 + u);
            const float uy = __shfl_sync(0xffffffffu, uyl, q0 + u);
            const float uz = __shfl_sync(0xffffffffu, uzl, q0 + u);
            ta[u] = fmaf(ux, p0x, fmaf(uy, p0y, uz * p0z)) * fcw;
            tb[u] = fmaf(ux, p1x, fmaf(uy, p1y, uz * p1z)) * fcw;
          }
          float ca[4], sa4[4], cb[4], sb4[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            steer_cs(ta[u], ca[u], sa4[u]);
            steer_cs(tb[u], cb[u], sb4[u]);
          }
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int r = gw + kGenWarps * (q0 + u);
            const bool in = dt * kTileM + r < it.D;  // rows past D are written as zero
            if (has0) {
              // Re h into column m, Im h into column M + m
              st_pair<ESZ>(base, r, m0, g.M, in ? ca[u] : 0.f, in ? cb[u] : 0.f, has1);
              st_pair<ESZ>(base, r, g.M + m0, g.M, in ? sa4[u] : 0.f, in ? sb4[u] : 0.f, has1);
            }
          }
        }
        // the tensor cores read the tile through the async proxy
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        if (lane == 0) mbar_arrive(a_full(sa));
        ++ia;
      }
    }
    if (!ok) atomicExch(&abort_sh, 1);
  } else if (warp == kEpiWarps) {
    // ---- loads ----
    if (lane == 0) {
      int ia = 0, ib = 0;
      bool ok = true;
      // test hook (ssl_set_test_stall): issue no operand load at all, so that
      // the MMA role's first wait can only end by running out
      for (int i = blockIdx.x; ok && !stall && i < nitems; i += gridDim.x) {
        const Item it = item(i);
        const int natoms = it.KP / kAtomElems;
        if (tmH_items || mitems)
          asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(
                           reinterpret_cast<uint64_t>(it.tmA))
                       : "memory");
        if (mitems)
          asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(
                           reinterpret_cast<uint64_t>(it.tmB))
                       : "memory");
        const int sb = ib % SB;
        ok = mbar_wait_spin(b_empty(sb), ((ib / SB) & 1) ^ 1, abort_v, wait_ns);
        if (!ok) break;
        // the G images stacked by rows: atom j holds rows g NP .. g NP + NP - 1
        // of image g
        mbar_expect_tx(b_full(sb), it.G * natoms * it.NP * 128);
        for (int j = 0; j < natoms; ++j)
          for (int gg = 0; gg < it.G; ++gg)
            tma_load_3d(sB0 + sb * PP::kBBytes + (j * it.G + gg) * it.NP * 128, it.tmB,
                        j * kAtomElems, 0, it.ecoord[gg], b_full(sb));
        ++ib;
        for (int dt = 0; !kGen && dt < it.ndt; ++dt) {
          const int sa = ia % SA;
          ok = mbar_wait_spin(a_empty(sa), ((ia / SA) & 1) ^ 1, abort_v, wait_ns);
          if (!ok) break;
          mbar_expect_tx(a_full(sa), natoms * kTileM * 128);
          for (int j = 0; j < natoms; ++j)
            tma_load_3d(sA0 + sa * PP::kABytes + j * kTileM * 128, it.tmA, j * kAtomElems,
                        dt * kTileM, it.bin, a_full(sa));
          ++ia;
        }
      }
      if (!ok) {
        atomicExch(&abort_sh, 1);
        // the loads still in flight are the last SA (SB) issued
        for (int k = max(0, ia - SA); k < ia; ++k) mbar_wait(a_full(k % SA), (k / SA) & 1);
        for (int k = max(0, ib - SB); k < ib; ++k) mbar_wait(b_full(k % SB), (k / SB) & 1);
      }
    }
  } else if (warp == kEpiWarps + 1) {
    // ---- MMAs ----
    if (lane == 0) {
      int ia = 0, ib = 0, g = 0;
      bool ok = true;
      uint32_t last_b = 0, last_bp = 0;
      for (int i = blockIdx.x; ok && i < nitems; i += gridDim.x) {
        const Item it = item(i);
        const int sb = ib % SB;
        ok = mbar_wait_spin(b_full(sb), (ib / SB) & 1, abort_v, wait_ns);
        if (!ok) break;
        const uint32_t idesc = instr_desc(ESZ == 2 ? 1u : 2u, (uint32_t)(it.G * it.NP));
        const int ksteps = it.KP / kKStep;
        for (int dt = 0; dt < it.ndt; ++dt) {
          const int sa = ia % SA, ac = g % kAcc;
          ok = mbar_wait_spin(a_full(sa), (ia / SA) & 1, abort_v, wait_ns) &&
               mbar_wait_spin(acc_empty(ac), ((g / kAcc) & 1) ^ 1, abort_v, wait_ns);
          if (!ok) break;
          tc_fence_after();
          for (int kk = 0; kk < ksteps; ++kk) {
            const int j = kk / 4, off = (kk % 4) * 32;
            const uint64_t a = smem_desc(sA0 + sa * PP::kABytes + j * kTileM * 128 + off);
            const uint64_t b =
                smem_desc(sB0 + sb * PP::kBBytes + j * it.G * it.NP * 128 + off);
            mma<ESZ>(tmem + kAccCols * ac, a, b, idesc, kk > 0 ? 1u : 0u);
          }
          mma_commit(acc_full(ac));
          mma_commit(a_empty(sa));
          ++ia;
          ++g;
        }
        if (!ok) break;
        mma_commit(b_empty(sb));
        last_b = b_empty(sb);
        last_bp = (ib / SB) & 1;
        ++ib;
      }
      // the last commit has landed: no MMA of ours is still running
      if (ib > 0) mbar_wait(last_b, last_bp);
      if (!ok) {
        atomicExch(&abort_sh, 1);
        if (ia > 0) mbar_wait(a_empty((ia - 1) % SA), ((ia - 1) / SA) & 1);
      }
    }
  } else {
    // ---- epilogue: warpgroup wg takes the tiles g with g % kAcc == wg % kAcc
    // (accumulator wg % kAcc) and, with two accumulators, the columns of
    // block wg / kAcc of each; a warpgroup thus waits on every phase of its
    // accumulator in turn ----
    const int wg = warp >> 2, q = warp & 3;
    const int r = wg % kAcc, part = wg / kAcc;
    int g = 0;
    bool ok = true;
    for (int i = blockIdx.x; ok && i < nitems; i += gridDim.x) {
      const Item it = item(i);
      for (int dt = 0; dt < it.ndt; ++dt, ++g) {
        if (g % kAcc != r) continue;
        const int ac = r;
        const int d = dt * kTileM + 32 * q + lane;
        // |h|^2, issued before the wait (analytic steering: unit modulus)
        const float hd = d >= it.D ? 0.f : it.hn ? __ldg(it.hn + d) : (float)it.M;
        // warp-uniform outcome: the TMEM loads below are .sync.aligned
        if (!__all_sync(0xffffffffu, mbar_wait(acc_full(ac), (g / kAcc) & 1, abort_v, wait_ns))) {
          atomicExch(&abort_sh, 1);
          ok = false;
          break;
        }
        tc_fence_after();
        // Columns g NP + (2i, 2i + 1) hold (Re, Im) of h^H e_i of block g; the
        // zero rows that pad each noise image past 2N contribute 0 to either
        // sum.  NP is a multiple of 16: chunks of 16 columns.
        const uint32_t trow = tmem + ((uint32_t)(32 * q) << 16) + kAccCols * ac;
        const bool mine = part < it.G;  // this warpgroup's block exists in the item
        const float den = mine ? fold_den(trow + part * it.NP, it.NP, form) : 0.f;
        tc_fence_before();
        mbar_arrive(acc_empty(ac));  // this accumulator may be overwritten
        float* const Pp = part ? it.P[1] : it.P[0];
        if (mine && d < it.D) Pp[d] = __fdividef(hd, fmaxf(den, FLT_MIN));
      }
    }
  }

  // Teardown: release the tensor memory once every warp is done with it.
  tc_fence_before();
  __syncthreads();
  if (tid == 0 && abort_sh) atomicOr(flags, SSL_FLAG_TIMEOUT);
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(kAccCols * kAcc)
                 : "memory");
  }
}

// ---- 3xTF32: FP32-class products on the TF32 tensor cores --------------------
// Each FP32 operand x is split into x_hi = tf32(x) and x_lo = tf32(x - x_hi)
// (22 significant bits together), and every K-step issues three kind::tf32
// MMAs into one FP32 accumulator: A_hi B_hi + A_hi B_lo + A_lo B_hi (the
// dropped A_lo B_lo term is below 2^-22 of the product).  The noise-subspace
// image of an item (hi and lo, 128 KB at NP = KP = 128) stays in shared
// memory for all of its direction tiles; the steering tiles stream through a
// ring of three stages, each one 32-element K atom of A_hi and A_lo (32 KB),
// so that both fit one CTA's shared memory.  One (block, bin) per item, items
// bin-major; roles, accumulators, epilogue and bounded waits as in
// spectrum_tc_kernel.
struct Pipe3 {
  static constexpr int kSA = 3;
  static constexpr uint32_t kAtomA = kTileM * 128;           // one K atom of one A tile
  static constexpr uint32_t kABytes = 2 * kAtomA;            // hi + lo
  static constexpr uint32_t kBBytes = 2 * 4 * 128 * 128;     // hi + lo, KP = NP = 128 at most
  static constexpr int kAccCols = 128;
  static constexpr int kAcc = 4;
  static constexpr size_t kSmem = 1024 + kSA * kABytes + kBBytes;
};
static_assert(Pipe3::kSmem <= 227 * 1024, "3xTF32 rings fit one CTA");

__global__ void __launch_bounds__(kThreads, 1)
spectrum_tc3_kernel(const __grid_constant__ CUtensorMap tmH, const __grid_constant__ CUtensorMap tmHlo,
                    const __grid_constant__ CUtensorMap tmE, const __grid_constant__ CUtensorMap tmElo,
                    int nitems, int nblk, int B, int D, int M, int Ns, int KP, int NP, int form,
                    const float* __restrict__ hnorm2, float* __restrict__ P, unsigned* flags,
                    uint64_t wait_ns, int stall) {
  using PP = Pipe3;
  constexpr int kAtomElems = 32;  // TF32 per 128-byte swizzle row
  constexpr int SA = PP::kSA, kAcc = PP::kAcc;
  constexpr uint32_t kAccCols = PP::kAccCols;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  // a_full[SA], a_empty[SA], b_full, b_empty, acc_full[kAcc], acc_empty[kAcc]
  __shared__ __align__(8) uint64_t bars[2 * SA + 2 + 2 * kAcc];
  __shared__ uint32_t tmem_sh;
  __shared__ int abort_sh;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t bar0 = smem_u32(&bars[0]);
  auto a_full = [&](int st) { return bar0 + 8u * st; };
  auto a_empty = [&](int st) { return bar0 + 8u * (SA + st); };
  const uint32_t b_full = bar0 + 8u * (2 * SA), b_empty = bar0 + 8u * (2 * SA + 1);
  auto acc_full = [&](int st) { return bar0 + 8u * (2 * SA + 2 + st); };
  auto acc_empty = [&](int st) { return bar0 + 8u * (2 * SA + 2 + kAcc + st); };
  const uint32_t sA0 = smem_u32(smem);
  const uint32_t sB0 = sA0 + SA * PP::kABytes;
  const int natoms = KP / kAtomElems;
  const int ndt = ceil_div(D, kTileM);

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_sh)),
                 "r"(kAccCols * kAcc)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    for (int i = 0; i < 2 * SA + 2 + kAcc; ++i) mbar_init(bar0 + 8u * i, 1);
    for (int i = 0; i < kAcc; ++i) mbar_init(acc_empty(i), kEpiThreads / kAcc);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    abort_sh = 0;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_sh;
  volatile int* abort_v = &abort_sh;
  // item i: bin i / nblk, block i % nblk (blocks fastest: the items in flight
  // share a bin's steering tiles in L2)
  auto bin_of = [&](int i) { return i / nblk; };
  auto ecoord_of = [&](int i) { return (i % nblk) * B + i / nblk; };

  if (warp == kEpiWarps) {
    // ---- loads ----
    if (lane == 0) {
      int ia = 0, ib = 0;
      bool ok = true;
      for (int i = blockIdx.x; ok && !stall && i < nitems; i += gridDim.x) {  // see the tc kernel
        ok = mbar_wait_spin(b_empty, (ib & 1) ^ 1, abort_v, wait_ns);
        if (!ok) break;
        mbar_expect_tx(b_full, 2 * natoms * NP * 128);
        for (int j = 0; j < natoms; ++j) {
          tma_load_3d(sB0 + j * NP * 128, &tmE, j * kAtomElems, 0, ecoord_of(i), b_full);
          tma_load_3d(sB0 + (natoms + j) * NP * 128, &tmElo, j * kAtomElems, 0, ecoord_of(i),
                      b_full);
        }
        ++ib;
        for (int dt = 0; ok && dt < ndt; ++dt)
          for (int j = 0; j < natoms; ++j) {
            const int sa = ia % SA;
            ok = mbar_wait_spin(a_empty(sa), ((ia / SA) & 1) ^ 1, abort_v, wait_ns);
            if (!ok) break;
            mbar_expect_tx(a_full(sa), PP::kABytes);
            tma_load_3d(sA0 + sa * PP::kABytes, &tmH, j * kAtomElems, dt * kTileM, bin_of(i),
                        a_full(sa));
            tma_load_3d(sA0 + sa * PP::kABytes + PP::kAtomA, &tmHlo, j * kAtomElems,
                        dt * kTileM, bin_of(i), a_full(sa));
            ++ia;
          }
      }
      if (!ok) {
        atomicExch(&abort_sh, 1);
        for (int k = max(0, ia - SA); k < ia; ++k) mbar_wait(a_full(k % SA), (k / SA) & 1);
        if (ib > 0) mbar_wait(b_full, (ib - 1) & 1);
      }
    }
  } else if (warp == kEpiWarps + 1) {
    // ---- MMAs ----
    if (lane == 0) {
      int ia = 0, ib = 0, g = 0;
      bool ok = true, issued = false;
      const uint32_t idesc = instr_desc(2u, (uint32_t)NP);
      for (int i = blockIdx.x; ok && i < nitems; i += gridDim.x) {
        ok = mbar_wait_spin(b_full, ib & 1, abort_v, wait_ns);
        if (!ok) break;
        for (int dt = 0; ok && dt < ndt; ++dt) {
          const int ac = g % kAcc;
          ok = mbar_wait_spin(acc_empty(ac), ((g / kAcc) & 1) ^ 1, abort_v, wait_ns);
          if (!ok) break;
          for (int j = 0; j < natoms; ++j) {
            const int sa = ia % SA;
            ok = mbar_wait_spin(a_full(sa), (ia / SA) & 1, abort_v, wait_ns);
            if (!ok) break;
            tc_fence_after();
            const uint32_t ah = sA0 + sa * PP::kABytes, al = ah + PP::kAtomA;
            const uint32_t bh = sB0 + j * NP * 128, bl = sB0 + (natoms + j) * NP * 128;
            for (int kk = 0; kk < 4; ++kk) {  // 8 TF32 (32 bytes) per MMA
              const uint32_t off = kk * 32;
              const uint32_t acc = (j > 0 || kk > 0) ? 1u : 0u;
              mma<4>(tmem + kAccCols * ac, smem_desc(ah + off), smem_desc(bh + off), idesc, acc);
              mma<4>(tmem + kAccCols * ac, smem_desc(ah + off), smem_desc(bl + off), idesc, 1u);
              mma<4>(tmem + kAccCols * ac, smem_desc(al + off), smem_desc(bh + off), idesc, 1u);
            }
            mma_commit(a_empty(sa));
            issued = true;
            ++ia;
          }
          if (!ok) break;
          mma_commit(acc_full(ac));
          ++g;
        }
        if (!ok) break;
        mma_commit(b_empty);
        ++ib;
      }
      // the last commit has landed: no MMA of ours is still running
      if (issued) mbar_wait(a_empty((ia - 1) % SA), ((ia - 1) / SA) & 1);
      if (!ok) atomicExch(&abort_sh, 1);
    }
  } else {
    // ---- epilogue: warpgroup wg takes the tiles g with g % 4 == wg ----
    const int wg = warp >> 2, q = warp & 3;
    int g = 0;
    bool ok = true;
    for (int i = blockIdx.x; ok && i < nitems; i += gridDim.x) {
      const float* hn = hnorm2 + (size_t)bin_of(i) * D;
      float* Pi = P + (size_t)ecoord_of(i) * D;
      for (int dt = 0; dt < ndt; ++dt, ++g) {
        if (g % kAcc != wg) continue;
        const int d = dt * kTileM + 32 * q + lane;
        const float hd = d < D ? __ldg(hn + d) : 0.f;
        if (!__all_sync(0xffffffffu, mbar_wait(acc_full(wg), (g / kAcc) & 1, abort_v, wait_ns))) {
          atomicExch(&abort_sh, 1);
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t trow = tmem + ((uint32_t)(32 * q) << 16) + kAccCols * wg;
        const float den = fold_den(trow, NP, form);
        tc_fence_before();
        mbar_arrive(acc_empty(wg));
        if (d < D) Pi[d] = __fdividef(hd, fmaxf(den, FLT_MIN));
      }
    }
  }

  tc_fence_before();
  __syncthreads();
  if (tid == 0 && abort_sh) atomicOr(flags, SSL_FLAG_TIMEOUT);
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(kAccCols * kAcc)
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

// H [B][D][M] c64 -> A image [B][D][KP]; with `lo` (TF32 only) the image of
// the residuals x - tf32(x), rounded to TF32 (the low part of 3xTF32).
template <int ESZ>
__global__ void pack_h_kernel(const float2* __restrict__ H, int BD, int M, int KP, void* out,
                              bool lo) {
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
    if (lo) x -= to_tf32(x);
    put<ESZ>(out, e, x);
  }
}

// E [nblk*B][M][M] c64 -> B image [nblk*B][NP][KP].
// One noise image: E [M][M] (row-major, columns are the singular vectors) ->
// B image [NP][KP] of the real embedding.  E is staged transposed in shared
// memory (row stride M + 1: the transposing writes of a half-warp fall on
// distinct bank pairs), so that each output row reads a contiguous column of
// E; every thread then writes 16 bytes (8 BF16 or 4 TF32 values) at a time.
template <int ESZ>
__device__ __forceinline__ void pack_e_one(const float2* __restrict__ Eb, int M, int Ns, int KP,
                                           int NP, void* __restrict__ out, float2* Et,
                                           void* __restrict__ out_lo = nullptr) {
  constexpr int V = 16 / ESZ;  // values per 16-byte store
  const int LT = M + 1;
  const int N = M - Ns;
  // eight loads in flight per thread before their transposing stores
  for (int e0 = threadIdx.x; e0 < M * M; e0 += 8 * blockDim.x) {
    float2 v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int e = e0 + u * blockDim.x;
      v[u] = e < M * M ? __ldg(Eb + e) : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int e = e0 + u * blockDim.x;
      if (e < M * M) Et[(e % M) * LT + e / M] = v[u];
    }
  }
  __syncthreads();
  const int chunks = KP / V;
  for (int e = threadIdx.x; e < NP * chunks; e += blockDim.x) {
    const int n = e / chunks, k0 = (e % chunks) * V;
    const int i = n >> 1;
    float x[V];
#pragma unroll
    for (int t = 0; t < V; ++t) {
      const int k = k0 + t;
      float v = 0.f;
      if (i < N && k < 2 * M) {
        const float2 w = Et[(Ns + i) * LT + (k < M ? k : k - M)];
        v = (n & 1) == 0 ? (k < M ? w.x : w.y) : (k < M ? w.y : -w.x);
      }
      x[t] = v;
    }
    uint4 pk;
    if (ESZ == 2) {
      uint32_t w[4];
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(x[2 * t], x[2 * t + 1]);
        w[t] = *reinterpret_cast<const uint32_t*>(&h);
      }
      pk = make_uint4(w[0], w[1], w[2], w[3]);
    } else {
      pk = make_uint4(__float_as_uint(to_tf32(x[0])), __float_as_uint(to_tf32(x[1 % V])),
                      __float_as_uint(to_tf32(x[2 % V])), __float_as_uint(to_tf32(x[3 % V])));
      if (out_lo)  // residuals of the TF32 rounding, themselves rounded to TF32
        reinterpret_cast<uint4*>(out_lo)[(size_t)n * chunks + e % chunks] = make_uint4(
            __float_as_uint(to_tf32(x[0] - __uint_as_float(pk.x))),
            __float_as_uint(to_tf32(x[1 % V] - __uint_as_float(pk.y))),
            __float_as_uint(to_tf32(x[2 % V] - __uint_as_float(pk.z))),
            __float_as_uint(to_tf32(x[3 % V] - __uint_as_float(pk.w))));
    }
    reinterpret_cast<uint4*>(out)[(size_t)n * chunks + e % chunks] = pk;
  }
}

template <int ESZ>
__global__ void pack_e_kernel(const float2* __restrict__ E, int M, int Ns, int KP, int NP,
                              void* out, void* out_lo) {
  __shared__ float2 Et[SSL_MAX_M * (SSL_MAX_M + 1)];
  const size_t mat = blockIdx.x;
  pack_e_one<ESZ>(E + mat * M * M, M, Ns, KP, NP,
                  static_cast<uint8_t*>(out) + mat * (size_t)NP * KP * ESZ, Et,
                  out_lo ? static_cast<uint8_t*>(out_lo) + mat * (size_t)NP * KP * ESZ : nullptr);
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
    pack_h_kernel<2><<<blocks, 256, 0, s>>>(H, BD, M, KP, out, false);
  else
    pack_h_kernel<4><<<blocks, 256, 0, s>>>(H, BD, M, KP, out, precision == kPrecTf32Lo);
  return cudaGetLastError();
}

cudaError_t launch_pack_e(const float2* E, int nmat, int M, int Ns, int precision, void* out,
                          cudaStream_t s, void* out_lo) {
  const int KP = tc_kp(M), NP = tc_np(M, Ns);
  if (precision == SSL_PREC_BF16)
    pack_e_kernel<2><<<nmat, 256, 0, s>>>(E, M, Ns, KP, NP, out, nullptr);
  else
    pack_e_kernel<4><<<nmat, 256, 0, s>>>(E, M, Ns, KP, NP, out, out_lo);
  return cudaGetLastError();
}

size_t tc_smem_bytes(int M, int Ns, int precision) {
  (void)M;
  (void)Ns;
  return precision == SSL_PREC_BF16    ? Pipe<2>::kSmem
         : precision == SSL_PREC_TF32X3 ? Pipe3::kSmem
                                        : Pipe<4>::kSmem;
}

namespace {

// One persistent CTA per SM (the shared memory of the rings admits one).
int spectrum_grid(int nitems) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
    sms = 1;
  return nitems < sms ? nitems : sms;
}

template <int ESZ, bool kGen>
cudaError_t launch_tc_mode(const CUtensorMap& tmH, const CUtensorMap& tmE, int nitems, int nblk,
                           int B, int D, int M, int Ns, int KP, int NP, int form,
                           const float* hnorm2, float* P, unsigned* flags, cudaStream_t s,
                           const CUtensorMap* tmH_items, const float* const* hn_items,
                           const MixedItem* mitems, const int2* mctab, uint64_t wait_ns,
                           const Geo* geo, const Geo* const* geo_items, int stall) {
  const size_t smem = Pipe<ESZ>::kSmem;
  cudaError_t e = cudaFuncSetAttribute(spectrum_tc_kernel<ESZ, kGen>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  spectrum_tc_kernel<ESZ, kGen><<<spectrum_grid(nitems), kThreads + (kGen ? kGenThreads : 0),
                                  smem, s>>>(
      tmH, tmE, nitems, nblk, B, D, M, Ns, KP, NP, form, hnorm2, P, flags, tmH_items, hn_items,
      mitems, mctab, wait_ns > 0 ? wait_ns : kWaitNs, geo, geo_items, stall);
  return cudaGetLastError();
}

template <int ESZ>
cudaError_t launch_tc(const CUtensorMap& tmH, const CUtensorMap& tmE, int nitems, int nblk, int B,
                      int D, int M, int Ns, int KP, int NP, int form, const float* hnorm2,
                      float* P, unsigned* flags, cudaStream_t s, const CUtensorMap* tmH_items,
                      const float* const* hn_items, const MixedItem* mitems, const int2* mctab,
                      uint64_t wait_ns, const Geo* geo = nullptr,
                      const Geo* const* geo_items = nullptr, int stall = 0) {
  if (nitems <= 0) return cudaSuccess;
  if (geo || geo_items)
    return launch_tc_mode<ESZ, true>(tmH, tmE, nitems, nblk, B, D, M, Ns, KP, NP, form, hnorm2,
                                     P, flags, s, tmH_items, hn_items, mitems, mctab, wait_ns,
                                     geo, geo_items, stall);
  return launch_tc_mode<ESZ, false>(tmH, tmE, nitems, nblk, B, D, M, Ns, KP, NP, form, hnorm2, P,
                                    flags, s, tmH_items, hn_items, mitems, mctab, wait_ns,
                                    nullptr, nullptr, stall);
}

}  // namespace

cudaError_t launch_spectrum_tc(const CUtensorMap& tmH, const CUtensorMap& tmE, int nblk, int B,
                               int D, int M, int Ns, int precision, int form,
                               const float* hnorm2, float* P, unsigned* flags, cudaStream_t s,
                               const CUtensorMap* tmH_items, const float* const* hn_items,
                               uint64_t wait_ns, const Geo* geo, const Geo* const* geo_items,
                               int stall) {
  const int KP = tc_kp(M), NP = tc_np(M, Ns);
  // items: bins x block groups (pairs of blocks where they share the steering)
  if (precision == SSL_PREC_BF16) {
    const int G = (tmH_items || geo_items) ? 1 : Pipe<2>::kG;
    return launch_tc<2>(tmH, tmE, B * pair_count(nblk, G), nblk, B, D, M, Ns, KP, NP, form,
                        hnorm2, P, flags, s, tmH_items, hn_items, nullptr, nullptr, wait_ns,
                        geo, geo_items, stall);
  }
  const int G = (tmH_items || geo_items) ? 1 : Pipe<4>::kG;
  return launch_tc<4>(tmH, tmE, B * pair_count(nblk, G), nblk, B, D, M, Ns, KP, NP, form, hnorm2,
                      P, flags, s, tmH_items, hn_items, nullptr, nullptr, wait_ns, geo,
                      geo_items, stall);
}

cudaError_t launch_spectrum_tc3(const CUtensorMap& tmH, const CUtensorMap& tmHlo,
                                const CUtensorMap& tmE, const CUtensorMap& tmElo, int nblk, int B,
                                int D, int M, int Ns, int form, const float* hnorm2, float* P,
                                unsigned* flags, cudaStream_t s, uint64_t wait_ns, int stall) {
  const int KP = tc_kp(M), NP = tc_np(M, Ns);
  const int nitems = nblk * B;
  if (nitems <= 0) return cudaSuccess;
  const size_t smem = Pipe3::kSmem;
  cudaError_t e = cudaFuncSetAttribute(spectrum_tc3_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  spectrum_tc3_kernel<<<spectrum_grid(nitems), kThreads, smem, s>>>(
      tmH, tmHlo, tmE, tmElo, nitems, nblk, B, D, M, Ns, KP, NP, form, hnorm2, P, flags,
      wait_ns > 0 ? wait_ns : kWaitNs, stall);
  return cudaGetLastError();
}

// Mixed batch: items are the (array, bin) pairs of the table, shapes and
// tensor maps from the array.
cudaError_t launch_spectrum_tc_mixed(const MixedItem* items, const int2* ctab, int n_ctab,
                                     int precision, int form, unsigned* flags, cudaStream_t s,
                                     uint64_t wait_ns) {
  if (n_ctab <= 0) return cudaSuccess;
  CUtensorMap dummy;
  memset(&dummy, 0, sizeof(dummy));
  if (precision == SSL_PREC_BF16)
    return launch_tc<2>(dummy, dummy, n_ctab, 1, 0, 0, 0, 0, 0, 0, form, nullptr, nullptr, flags,
                        s, nullptr, nullptr, items, ctab, wait_ns);
  return launch_tc<4>(dummy, dummy, n_ctab, 1, 0, 0, 0, 0, 0, 0, form, nullptr, nullptr, flags, s,
                      nullptr, nullptr, items, ctab, wait_ns);
}

namespace {
// H[w][d][m] = exp(+j 2 pi f_w (u_d . p_m) / c) with the phase formed and
// reduced in FP64 (the table is the reference the generated tiles are
// compared with; sincospi takes the phase in half turns).
__global__ void steering_table_kernel(const Geo* __restrict__ geo, int B, int D, int M,
                                      float2* __restrict__ H) {
  const Geo g = *geo;
  const size_t n = (size_t)B * D * M;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n;
       e += (size_t)gridDim.x * blockDim.x) {
    const int m = (int)(e % M), d = (int)((e / M) % D), w = (int)(e / ((size_t)M * D));
    const double s = (double)g.dirs[3 * d] * g.pos[3 * m] + (double)g.dirs[3 * d + 1] * g.pos[3 * m + 1] +
                     (double)g.dirs[3 * d + 2] * g.pos[3 * m + 2];
    double t = s * (double)g.fc[w];
    t -= rint(t);
    double sn, cs;
    sincospi(2.0 * t, &sn, &cs);
    H[e] = make_float2((float)cs, (float)sn);
  }
}
}  // namespace

cudaError_t launch_steering_table(const Geo* geo, int B, int D, int M, float2* H, cudaStream_t s) {
  steering_table_kernel<<<1024, 256, 0, s>>>(geo, B, D, M, H);
  return cudaGetLastError();
}

}  // namespace ssl
