// Conversions between binary32 and binary64 by integer operations on the
// IEEE 754 fields (sign, biased exponent, fraction; biases 127 and 1023).
//
// On this GPU the FP64 instructions, the F2F conversions between float and
// double included, issue at about 1/64 of the FP32 rate.  The vector kernels
// of the mixed-precision outer iteration perform a few such conversions per
// element and, measured, were bound by the FP64 pipe rather than by memory.
// The functions below take the common cases (zeros and normal numbers in
// the handled exponent ranges) with integer instructions and leave every
// other case (subnormal, infinite, NaN, out of range) to the hardware
// conversion.  f2d and d2f_rn return bit-for-bit what the casts return;
// split_f2 defines its own split (truncation, see there).
#pragma once

namespace vps {

// The hardware conversions, out of line: called only by the lanes that need
// them (inlined, the compiler may evaluate them on every lane and select).
static __device__ __noinline__ double f2d_hw(float f) { return (double)f; }
static __device__ __noinline__ float d2f_hw(double d) { return (float)d; }
static __device__ __noinline__ void split_hw(double v, float& hi, float& lo) {
  hi = (float)v;
  lo = (float)(v - (double)hi);
}

// Exact float -> double (the value is unchanged).
__device__ __forceinline__ double f2d(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned e = (u >> 23) & 0xffu;
  const unsigned long long sign = (unsigned long long)(u & 0x80000000u) << 32;
  if (e - 1u < 254u)  // normal (1 <= e <= 254): rebias the exponent, widen the fraction
    return __longlong_as_double((long long)(sign | ((unsigned long long)(e + 896u) << 52) |
                                            ((unsigned long long)(u & 0x7fffffu) << 29)));
  if ((u << 1) == 0u) return __longlong_as_double((long long)sign);  // +-0
  return f2d_hw(f);                                                  // subnormal, inf, NaN
}

// double -> float rounded to nearest, ties to even (the rounding of the cast).
__device__ __forceinline__ float d2f_rn(double d) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(d);
  const unsigned top = (unsigned)(b >> 32);
  const unsigned E = (top >> 20) & 0x7ffu;
  if (E - 897u < 254u) {  // a normal float exponent: E - 1023 in [-126, 127]
    const unsigned long long frac = b & 0xfffffffffffffull;  // 52 fraction bits
    const unsigned m = (unsigned)(frac >> 29);                // the 23 kept
    const unsigned long long rest = frac & 0x1fffffffull;     // the 29 dropped
    unsigned r = ((E - 896u) << 23) | m;
    // up if the dropped part is above half an ulp, or exactly half and m is
    // odd; a carry out of the fraction increments the exponent (254 -> 255
    // with a zero fraction is infinity, the rounded overflow)
    if (rest > (1ull << 28) || (rest == (1ull << 28) && (m & 1u))) r += 1u;
    return __uint_as_float((top & 0x80000000u) | r);
  }
  if ((b << 1) == 0ull) return __uint_as_float(top & 0x80000000u);  // +-0
  return d2f_hw(d);  // below or above the normal float range, inf, NaN
}

// v = hi + lo + t with hi = v truncated to 24 significant bits and lo the
// next (up to) 24 bits of v, truncated: hi, lo and t carry the sign of v
// (or are zero), |lo| < ulp(hi) and |t| < 2^-47 |v|.  Zeros give signed
// zeros.  Outside E - 1023 in [-73, 127] (lo could be subnormal, or hi out
// of range) the pair is the rounded split hi = fl(v), lo = fl(v - hi).
__device__ __forceinline__ void split_f2(double v, float& hi, float& lo) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  const unsigned top = (unsigned)(b >> 32);
  const unsigned sign = top & 0x80000000u;
  if ((b << 1) == 0ull) {
    hi = lo = __uint_as_float(sign);
    return;
  }
  const unsigned E = (top >> 20) & 0x7ffu;
  if (E - 950u < 201u) {
    const unsigned long long frac = b & 0xfffffffffffffull;
    hi = __uint_as_float(sign | ((E - 896u) << 23) | (unsigned)(frac >> 29));
    const unsigned rest = (unsigned)(frac & 0x1fffffffull);  // weight of bit 0: 2^(E-1023-52)
    if (rest == 0u) {
      lo = __uint_as_float(sign);
      return;
    }
    const int lz = __clz(rest) - 3;      // leading zeros within the 29 bits (0 .. 28)
    const unsigned norm = rest << (lz + 3);  // leading one at bit 31
    // the leading one has weight 2^(E-1023-24-lz): biased exponent E-920-lz >= 1
    lo = __uint_as_float(sign | ((E - 920u - (unsigned)lz) << 23) | ((norm >> 8) & 0x7fffffu));
    return;
  }
  split_hw(v, hi, lo);
}

}  // namespace vps
