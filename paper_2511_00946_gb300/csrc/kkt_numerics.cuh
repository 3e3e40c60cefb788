// Device arithmetic helpers of the factor and residual kernels, in a header
// of their own so that a test can run them on the device against exact
// references: the pivot reciprocal square root and the truncated |v| used
// for the row sums of |Psi|.
#pragma once
#include <cuda_runtime.h>

namespace kkt {

// Rare path of pivot_rsqrt (zero, negative, NaN, infinite, subnormal or
// huge pivots), kept out of line: 1/sqrt(d) for a positive finite d, NaN
// otherwise.
static __device__ __noinline__ double pivot_rsqrt_slow(double d) {
  return (d > 0.0 && d <= 1.7976931348623157e308) ? 1.0 / sqrt(d) : __longlong_as_double(0x7ff8000000000000LL);
}

// True unless d is a positive finite number (integer test on the bits: an
// FP64 comparison would occupy the scarce FP64 pipe).
static __device__ __forceinline__ bool not_positive(double d) {
  const long long bits = __double_as_longlong(d);
  return bits <= 0 || bits >= 0x7ff0000000000000LL;
}

// 1/sqrt(d) for a pivot d > 0 in four dependent FP64 operations instead of a
// square root and a division (each several hundred cycles on this part).
// The exponent is split off with integer operations so that d' = d 4^-k lies
// in [1, 4); the single-precision hardware estimate r ~ 1/sqrt(d') (relative
// error below 2^-21) is formed from d' and converted back with bit
// manipulation only, then refined by one step of Halley's method for
// f(r) = r^-2 - d': with e = 1 - d' r^2, r <- r (1 + e/2 + 3 e^2 / 8), which
// leaves an error of order e^3 (below 2^-62), so the result is within a few
// units in the last place; finally r 2^-k. The step is evaluated as
// r + e (r/2 + (3r/8) e): r carries the estimate's 24 significant bits, so
// r/2 and 3r/8 are exact and are formed on the bits with integer operations,
// and the step costs two FP64 operations after e (a warp's FP64 instruction
// holds the sub-partition's FP64 pipe for 64 cycles, so every instruction on
// a pivot chain counts). Zero, negative, NaN, subnormal or huge d take an
// out-of-line path (NaN when d is not positive). The range tests are integer
// tests: FP64 comparisons would occupy the FP64 pipe.
static __device__ __forceinline__ double pivot_rsqrt(double d) {
  const long long bits = __double_as_longlong(d);
  const int ef = (int)((bits >> 52) & 0x7ff);  // biased exponent; sign handled by bits > 0
  if (bits <= 0 || ef <= 1 || ef >= 2046) return pivot_rsqrt_slow(d);
  const int k = (ef - 1023) >> 1;                            // floor(ex / 2)
  const long long dbits = bits - ((long long)(2 * k) << 52);  // d' in [1, 4)
  const double dp = __longlong_as_double(dbits);
  // d' truncated to single precision (exponent 0 or 1, top 23 mantissa bits)
  const int fbits = ((int)((dbits >> 52) & 0x7ff) - 1023 + 127) << 23 | (int)((dbits >> 29) & 0x7fffff);
  float rf;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(rf) : "f"(__int_as_float(fbits)));
  const int rb = __float_as_int(rf);  // in (0.5, 1]: normal
  double r = __longlong_as_double((long long)(((rb >> 23) & 0xff) - 127 + 1023) << 52 |
                                  (long long)(rb & 0x7fffff) << 29);
  const long long rbits = __double_as_longlong(r), re = (rbits >> 52) & 0x7ff;  // r in (1/2, 1]
  const double half_r = __longlong_as_double(rbits - (1LL << 52));
  // 3r/8: the 53-bit significand times 3 (its low 29 bits are zero, so the
  // renormalising shift by one or two places is exact)
  const long long sig3 = 3 * ((rbits & ((1LL << 52) - 1)) | (1LL << 52));
  const double c38_r = __longlong_as_double(sig3 >= (1LL << 54) ? ((re - 1) << 52) | ((sig3 >> 2) - (1LL << 52))
                                                                 : ((re - 2) << 52) | ((sig3 >> 1) - (1LL << 52)));
  const double e = fma(-dp * r, r, 1.0);
  r = fma(fma(c38_r, e, half_r), e, r);
  return __longlong_as_double(__double_as_longlong(r) - ((long long)k << 52));
}

// |v| as a float for the |Psi| row sums that scale eta: the exponent rebased
// and the mantissa cut to 20 bits with integer operations only (no FP64
// instruction), so never above |v|; 0 below the float range, the largest
// float above it. The sums then run in FP32: about 1e-6 relative, ample for
// the scale of a backward error.
static __device__ __forceinline__ float abs_lo(double v) {
  const int hi = __double2hiint(v) & 0x7fffffff;
  const int e = hi - (896 << 20);  // exponent bias 1023 -> 127
  if (e >= (255 << 20)) return 3.4028234e38f;
  return e > 0 ? __int_as_float(e << 3) : 0.0f;
}

}  // namespace kkt
