// Rotation arithmetic shared by the one-sided Jacobi kernels (eq. 4): the
// warp reductions of a round, the 2x2 unitary that orthogonalises a pair of
// columns, and its FP32 / FP64 evaluation.
#pragma once

#include <float.h>

#include "ssl_internal.cuh"

namespace ssl {
namespace jrot {

constexpr unsigned kFull = 0xffffffffu;

// Transposing butterfly over 16 values: on exit lanes 2i and 2i + 1 hold the
// warp-wide sum of value i (16 shuffles instead of 5 per value).
__device__ __forceinline__ float transpose_reduce16(float (&x)[16], int lane) {
#pragma unroll
  for (int w = 16, n = 8; w >= 2; w >>= 1, n >>= 1) {
    const bool hi = (lane & w) != 0;
#pragma unroll
    for (int k = 0; k < n; ++k) {
      const float send = hi ? x[k] : x[k + n];
      const float keep = hi ? x[k + n] : x[k];
      x[k] = keep + __shfl_xor_sync(kFull, send, w);
    }
  }
  return x[0] + __shfl_xor_sync(kFull, x[0], 1);
}

template <int RPL>
__device__ __forceinline__ float norm2(const float2 (&x)[RPL]) {
  float s = 0.f;
#pragma unroll
  for (int h = 0; h < RPL; ++h) s = fmaf(x[h].x, x[h].x, fmaf(x[h].y, x[h].y, s));
  return s;
}

// conj(x) . y over the lane's rows
template <int RPL>
__device__ __forceinline__ void dot_partial(const float2 (&x)[RPL], const float2 (&y)[RPL],
                                            float& gr, float& gi) {
  gr = 0.f;
  gi = 0.f;
#pragma unroll
  for (int h = 0; h < RPL; ++h) {
    gr = fmaf(x[h].x, y[h].x, fmaf(x[h].y, y[h].y, gr));
    gi = fmaf(x[h].x, y[h].y, fmaf(-x[h].y, y[h].x, gi));
  }
}

// x' = c x - conj(se) y ;  y' = se x + c y
__device__ __forceinline__ void rot1(float2& x, float2& y, float c, float sr, float si) {
  const float2 a = x, d = y;
  x = make_float2(fmaf(c, a.x, -fmaf(sr, d.x, si * d.y)), fmaf(c, a.y, -fmaf(sr, d.y, -si * d.x)));
  y = make_float2(fmaf(c, d.x, fmaf(sr, a.x, -si * a.y)), fmaf(c, d.y, fmaf(sr, a.y, si * a.x)));
}

// ---- rotation for one pair --------------------------------------------------
// In: alpha, beta (squared norms), gamma = (gr, gi), thresholds.
// Out: o = (c, sr, si, 1) with s e = sr + i si, e = gamma/|gamma|, and the new
// squared norms.  Returns false for "converged" (o, norms untouched).
// Inputs are scaled by a power of two so that max(alpha, beta) is in [1, 2):
// the rotation is scale-invariant and all intermediates stay well inside the
// FP32 range of the hardware estimates.  A pair whose norm ratio is below
// 2^-60 is left alone (its rotation would change V by less than 2^-30).
//
// With d = beta - alpha the rotation's tangent solves t^2 + (d/|gamma|) t = 1;
// the smaller root is t = sign(d) 2|gamma| / (|d| + sqrt(d^2 + 4|gamma|^2)).
// With den = |d| + sqrt(d^2 + 4|gamma|^2) and q = den^2 + 4|gamma|^2:
//   c = den / sqrt(q),   s e = sign(d) 2 gamma / sqrt(q),
//   alpha' = alpha - t |gamma|,  beta' = beta + t |gamma|,
//   t |gamma| = sign(d) 2 |gamma|^2 / den = sign(d) (sqrt(d^2 + 4|gamma|^2) - |d|) / 2.

// sc = 2^-floor(log2 m) for a normal m; ex = floor(log2 m), capped at 126
__device__ __forceinline__ float pow2_scale(float m, int& ex) {
  const int e = min((__float_as_int(m) >> 23) & 0xff, 253);
  ex = e - 127;
  return __int_as_float((254 - e) << 23);
}

// Conversions between binary32 and binary64 on the integer pipes.  On this
// part an FP64 warp instruction, a conversion included, occupies its
// sub-partition's FP64 unit for ~64 cycles, so the rotation's FP64 chain keeps
// only the arithmetic there.  f2d: exact (IEEE 754: re-bias the exponent by
// 1023 - 127 and append 29 zero bits to the significand) for normal numbers;
// zero, subnormals, Inf and NaN take the conversion instruction.  d2f_rn:
// round to nearest even of a binary64 whose binary32 result is a normal
// number (the callers' values lie in [2^-64, 2^64]): keep the top 23 bits of
// the significand, add one when the 29 dropped bits exceed half an ulp or equal
// it with an odd kept part; a carry out of the significand moves into the
// exponent field by the same addition.
__device__ __forceinline__ double f2d(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned e = (u >> 23) & 0xffu;
  if (e == 0u || e == 0xffu) return (double)f;
  const unsigned hi = (u & 0x80000000u) | ((e + 896u) << 20) | ((u & 0x7fffffu) >> 3);
  return __hiloint2double((int)hi, (int)(u << 29));
}
__device__ __forceinline__ float d2f_rn(double d) {
  const unsigned hi = (unsigned)__double2hiint(d), lo = (unsigned)__double2loint(d);
  const unsigned e = ((hi >> 20) & 0x7ffu) - 896u;  // binary32 exponent field (1..254)
  unsigned m = ((hi & 0xfffffu) << 3) | (lo >> 29);
  const unsigned rest = lo & 0x1fffffffu;
  m += (rest > 0x10000000u || (rest == 0x10000000u && (m & 1u))) ? 1u : 0u;
  return __uint_as_float((hi & 0x80000000u) | ((e << 23) + m));
}

// FP64 refinements of FP32 estimates, one Newton-Raphson step each: with
// y0 = (1 + e) / sqrt(x), |e| <= 2^-21, the results carry a relative error
// of about 1.5 e^2 <= 2^-41.  Three FP64 operations apiece.
//   1/sqrt(x):  y0 + (y0 / 2) (1 - x y0^2)
//   sqrt(x):    s0 + (y0 / 2) (x - s0^2),  s0 = x y0
__device__ __forceinline__ double rsqrt_nr(double x, float y0) {
  const double y = f2d(y0);
  const double e = fma(-(x * y), y, 1.0);
  return fma(f2d(0.5f * y0), e, y);
}
__device__ __forceinline__ double sqrt_nr(double x, float y0) {
  const double s0 = x * f2d(y0);
  const double e = fma(-s0, s0, x);
  return fma(f2d(0.5f * y0), e, s0);
}

// 2^e as a float, for e within the normal exponent range
__device__ __forceinline__ float exp2i(int e) { return __int_as_float((e + 127) << 23); }

// The absolute test (at2.x = abs_tol max_c |g_c|^2) applies only to pairs
// whose larger squared norm is at most at2.y = sqrt(abs_tol) max_c |g_c|^2:
// a residual g_p^H g_q left by it moves the singular vectors by about
// |g_p^H g_q| / (|g_p|^2 - |g_q|^2), which stays below sqrt(abs_tol) on those
// pairs, while a pair with a column above that level (a signal column, say,
// against a noise column) is always held to the relative test, so that the
// absolute test cannot mix the large singular vectors with the small ones.
__device__ __forceinline__ float abs_level(float m, float2 at2) {
  return m <= at2.y ? at2.x : 0.f;
}

template <bool kF64>
__device__ __forceinline__ bool rotation(float al, float be, float gr, float gi, float tol,
                                         float2 at2, float4& o, float& al_out,
                                         float& be_out) {
  const float m = fmaxf(al, be);
  if (!(m >= FLT_MIN)) return false;  // zero (padding) or non-finite
  int ex;
  const float sc = pow2_scale(m, ex);
  const float a = al * sc, b = be * sc, x = gr * sc, y = gi * sc;
  if (!(fminf(a, b) >= 8.67361738e-19f)) return false;  // norm ratio below 2^-60
  const float at = abs_level(m, at2) * sc;
  if (kF64) {
    // Decision: |gamma|^2 against max(tol^2 alpha beta, at^2).  The FP32
    // evaluation is within a few ulp of the exact one, so outside a 2^-18
    // band around the threshold it already gives the FP64 answer; inside the
    // band the comparison is redone in FP64.
    const float g4s = fmaf(2.f * x, 2.f * x, 4.f * y * y);
    const float lims = fmaxf(4.f * tol * tol * (a * b), 4.f * at * at);
    if (!(g4s > lims * 0.99999619f)) return false;  // below the band: converged
    const double ad = f2d(a), bd = f2d(b), xd = f2d(2.f * x), yd = f2d(2.f * y);  // exact
    const double g4 = fma(xd, xd, yd * yd);                     // 4 |gamma|^2
    if (!(g4s > lims * 1.00000381f)) {        // inside the band: exact test
      const double td = tol, atd = at;
      const double lim = fmax(4.0 * td * td * (ad * bd), 4.0 * atd * atd);
      if (!(g4 > lim)) return false;
    }
    const double d = bd - ad;
    const double w = fma(d, d, g4);
    // FP32 estimates of the same chain seed the FP64 Newton steps
    const float g4f = g4s;
    const float df = b - a;
    const float wf = fmaf(df, df, g4f);
    const float denf = fabsf(df) + sqrtf(wf);
    const double sw = sqrt_nr(w, rsqrtf(wf));
    const double den = fabs(d) + sw;
    const double q = fma(den, den, g4);
    const double rq = rsqrt_nr(q, rsqrtf(fmaf(denf, denf, g4f)));
    const float c = d2f_rn(den * rq);
    const float f = d < 0.0 ? -d2f_rn(rq) : d2f_rn(rq);
    o = make_float4(c, f * (2.f * x), f * (2.f * y), 1.f);
    // t |gamma| (signed with t) in the caller's scale: (sw - |d|) / 2, since
    // g4 / den = sw - |d| (den (sw - |d|) = sw^2 - d^2 = g4); the halving and
    // the unscaling are one exact power-of-two factor.
    const float tgf = __double2float_rn(d < 0.0 ? fabs(d) - sw : sw - fabs(d)) * exp2i(ex) * 0.5f;
    al_out = fmaxf(al - tgf, 0.f);
    be_out = fmaxf(be + tgf, 0.f);
    return true;
  } else {
    const float g4 = fmaf(2.f * x, 2.f * x, 4.f * y * y);
    if (!(g4 > 4.f * tol * tol * (a * b)) || !(g4 > 4.f * at * at)) return false;
    const float d = b - a;
    const float sw = sqrtf(fmaf(d, d, g4));
    const float den = fabsf(d) + sw;
    const float rq = __frsqrt_rn(fmaf(den, den, g4));
    const float c = den * rq;
    const float f = d < 0.f ? -rq : rq;
    o = make_float4(c, f * (2.f * x), f * (2.f * y), 1.f);
    const float tgf = (d < 0.f ? -0.5f : 0.5f) * (sw - fabsf(d)) / sc;  // signed t |gamma|
    al_out = fmaxf(al - tgf, 0.f);
    be_out = fmaxf(be + tgf, 0.f);
    return true;
  }
}

// The FP32 part of rotation<true>'s decision with a slightly wider band:
// false only for pairs that rotation<true> leaves alone (same expressions,
// so the same values), so a round in which no pair of the CTA passes it is
// a round without rotations.
__device__ __forceinline__ bool may_rotate(float al, float be, float gr, float gi, float tol,
                                           float2 at2) {
  const float m = fmaxf(al, be);
  if (!(m >= FLT_MIN)) return false;
  int ex;
  const float sc = pow2_scale(m, ex);
  const float a = al * sc, b = be * sc, x = gr * sc, y = gi * sc;
  if (!(fminf(a, b) >= 8.67361738e-19f)) return false;
  const float at = abs_level(m, at2) * sc;
  const float g4s = fmaf(2.f * x, 2.f * x, 4.f * y * y);
  const float lims = fmaxf(4.f * tol * tol * (a * b), 4.f * at * at);
  return g4s > lims * 0.9999f;
}

}  // namespace jrot
}  // namespace ssl
