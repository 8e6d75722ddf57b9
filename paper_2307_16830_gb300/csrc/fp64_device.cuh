// FP64 helpers of the vector kernels (device code only).  On this part the
// FP64 unit is the scarce one (2 FMA per clock per SM), so operations that
// integer instructions can do, or that need not be correctly rounded, are
// kept off it: range tests on the bit pattern, a reciprocal in three FP64
// operations, and sums of logarithms as one logarithm of a product.
#pragma once

#include <cuda_runtime.h>

namespace acopf {

// |v| in [2^-500, 2^500) (a test on the exponent bits).
__device__ __forceinline__ bool fp64_mid_range(double v) {
  const unsigned e = static_cast<unsigned>(__double_as_longlong(v) >> 52) & 0x7ffu;
  return e - 523u < 1000u;
}

// 1/x for |x| in [2^-1000, 2^1000) to within one ulp, with three FP64
// operations: a single-precision seed and one Newton-Raphson step with its
// cubic correction (y <- y + y (e + e^2), e = 1 - x y: the relative error
// goes from d to d^3, Markstein's form of the reciprocal iteration).  The
// seed is the hardware's approximate reciprocal of x's significand (as a
// float in [1, 2), cut from x's bits with integer instructions), scaled by
// x's exponent on the integer pipe: |d| < 2^-21, so d^3 is far below an
// ulp and the result is the correctly rounded y0 (1 + e + e^2) of the last
// FMA.
__device__ __forceinline__ double recip_nr(double x) {
  const long long b = __double_as_longlong(x);
  const int ex = static_cast<int>((b >> 52) & 0x7ff);  // biased exponent of x
  const float m = __int_as_float(0x3f800000 | static_cast<int>((b >> 29) & 0x7fffff));
  float rm;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rm) : "f"(m));  // ~1/m, in (0.5, 1]
  const int fb = __float_as_int(rm);
  const long long ey = static_cast<long long>(((fb >> 23) & 0xff) - 127 + 2046 - ex);
  const double y0 = __longlong_as_double((b & static_cast<long long>(0x8000000000000000ULL)) |
                                         (ey << 52) |
                                         (static_cast<long long>(fb & 0x7fffff) << 29));
  const double e = fma(-x, y0, 1.0);
  return fma(y0, fma(e, e, e), y0);
}

// 1/x: the Newton-Raphson form in its range, else the library's.
__device__ __forceinline__ double recip(double x) {
  return fp64_mid_range(x) ? recip_nr(x) : __drcp_rn(x);
}

// A sum of logarithms kept as log(m) + e ln 2 of their product m 2^e: each
// term multiplies the significand product by the term's significand (one
// FP64 multiply) and adds the exponents on the integer pipe; the product's
// own exponent is moved into e after every term, so m stays in [1, 2).
// Terms that are not positive normal numbers go to `rest` as log(g), so
// zeros, negatives, infinities and NaNs give what a plain sum would.
struct LogSum {
  double m = 1.0;
  long long e = 0;
  double rest = 0.0;
  __device__ __forceinline__ void add(double g) {
    const long long b = __double_as_longlong(g);
    const long long eg = (b >> 52) & 0x7ff;
    if (b <= 0 || eg == 0 || eg == 0x7ff) {  // sign set, zero, subnormal, inf, NaN
      rest += log(g);
      return;
    }
    const double mg = __longlong_as_double((b & 0x000fffffffffffffLL) | 0x3ff0000000000000LL);
    const long long bm = __double_as_longlong(m * mg);  // in [1, 4)
    e += eg + ((bm >> 52) & 0x7ff) - 2046;
    m = __longlong_as_double((bm & 0x000fffffffffffffLL) | 0x3ff0000000000000LL);
  }
  __device__ __forceinline__ double value() const {
    return fma(static_cast<double>(e), 0.69314718055994530942, log(m)) + rest;
  }
};

}  // namespace acopf
