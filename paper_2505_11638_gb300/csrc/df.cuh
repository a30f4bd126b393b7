// Double-float ("FP32 pair") arithmetic: a value is the unevaluated sum hi + lo of two floats,
// which carries ~48 significant bits.  Products of FP32 numbers are made exact with fmaf
// (Dekker's product via fused multiply-add) and sums with Knuth's TwoSum, so FP64-accurate dot
// products run on the FP32 pipes; on GB300 these issue ~60x faster than FP64 arithmetic.
#pragma once
#include <cuda_runtime.h>

namespace ngd {

struct DF {
  float hi, lo;
};

// s = a + b exactly as s + e (TwoSum, no ordering assumption)
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float z = s - a;
  e = (a - (s - z)) + (b - z);
}

// s += a * (bh + bl), a exact FP32, (bh, bl) a double split into two floats
__device__ __forceinline__ void df_add_prod(DF& s, float a, float bh, float bl) {
  const float p = a * bh;
  const float pe = fmaf(a, bh, -p);      // exact error of the product
  float t, e;
  two_sum(s.hi, p, t, e);
  s.hi = t;
  s.lo += e + fmaf(a, bl, pe);
}

// s += (ah + al) * (bh + bl)   (al bl dropped: below the pair's precision)
__device__ __forceinline__ void df_add_prod2(DF& s, float ah, float al, float bh, float bl) {
  const float p = ah * bh;
  float pe = fmaf(ah, bh, -p);
  pe = fmaf(ah, bl, pe);
  pe = fmaf(al, bh, pe);
  float t, e;
  two_sum(s.hi, p, t, e);
  s.hi = t;
  s.lo += e + pe;
}

// (a.hi + a.lo) + (b.hi + b.lo), renormalised; symmetric in a and b
__device__ __forceinline__ DF df_add(DF a, DF b) {
  float s, e;
  two_sum(a.hi, b.hi, s, e);
  e += a.lo + b.lo;
  const float hi = s + e;
  return DF{hi, e - (hi - s)};
}

__device__ __forceinline__ DF df_neg(DF a) { return DF{-a.hi, -a.lo}; }

// (t.hi + t.lo) * (wh + wl), renormalised
__device__ __forceinline__ DF df_mul(DF t, float wh, float wl) {
  const float p = t.hi * wh;
  float pe = fmaf(t.hi, wh, -p);
  pe = fmaf(t.hi, wl, pe);
  pe = fmaf(t.lo, wh, pe);
  const float hi = p + pe;
  return DF{hi, pe - (hi - p)};
}

// FP64 <-> FP32 conversions by integer operations on the bit patterns.  GB300 executes the
// hardware conversions on its FP64 pipe (about two per cycle and SM, measured), so bulk splits
// and recombinations do them in the integer pipes instead; the results are the same bits as the
// hardware's round-to-nearest-even conversions.  Zeros stay in the integer path; other values
// outside FP32's normal range (subnormal, overflow, inf, NaN) take the hardware conversion.
__device__ __forceinline__ float f64_to_f32_rn(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int e = (int)((b >> 52) & 0x7ff) - 1023;
  if (e < -126 || e > 127) {
    if ((b << 1) == 0ull) return __uint_as_float((unsigned)(b >> 32));       // +-0
    return __double2float_rn(x);
  }
  const unsigned long long m = b & 0xfffffffffffffull;                 // 52-bit fraction
  const unsigned t = (unsigned)((m + 0xfffffffull + ((m >> 29) & 1ull)) >> 29);   // 23 bits, half to even
  // a rounding carry (t == 2^23) moves into the exponent field; 2^128 becomes inf as it should
  const unsigned bits = ((unsigned)(b >> 32) & 0x80000000u) | (((unsigned)(e + 127) << 23) + t);
  return __uint_as_float(bits);
}

__device__ __forceinline__ double f32_to_f64(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned ef = (u >> 23) & 0xffu;
  if (ef == 0u || ef == 255u) {
    if ((u & 0x7fffffffu) == 0u) return __longlong_as_double((long long)((unsigned long long)u << 32));  // +-0
    return (double)f;                                                  // subnormal, inf, NaN
  }
  const unsigned long long b = ((unsigned long long)(u & 0x80000000u) << 32) |
                               ((unsigned long long)(ef + (1023u - 127u)) << 52) |
                               ((unsigned long long)(u & 0x7fffffu) << 29);
  return __longlong_as_double((long long)b);
}

double f32_to_f64(double) = delete;     // a double argument would be narrowed first

// widening of a templated accumulator: FP32 by the integer path, FP64 unchanged
__device__ __forceinline__ double to_f64(float f) { return f32_to_f64(f); }
__device__ __forceinline__ double to_f64(double d) { return d; }

// x = hi + lo: hi = x rounded to FP32, lo = the rest rounded to FP32 (one FP64 subtraction)
__device__ __forceinline__ void split_df(double x, float& hi, float& lo) {
  hi = f64_to_f32_rn(x);
  lo = f64_to_f32_rn(x - f32_to_f64(hi));
}

__device__ __forceinline__ double df_to_double(DF a) { return f32_to_f64(a.hi) + f32_to_f64(a.lo); }

// warp-wide sum by an XOR butterfly: every lane ends with the same value
__device__ __forceinline__ DF warp_sum_df(DF a) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const DF b{__shfl_xor_sync(0xffffffffu, a.hi, o), __shfl_xor_sync(0xffffffffu, a.lo, o)};
    a = df_add(a, b);
  }
  return a;
}

}  // namespace ngd

namespace ngd {

__device__ __forceinline__ DF shfl_xor_df(DF a, int o) {
  return DF{__shfl_xor_sync(0xffffffffu, a.hi, o), __shfl_xor_sync(0xffffffffu, a.lo, o)};
}

// Reduce-scatter of two per-lane values over a warp: lane L returns the warp-wide sum of
// v[(L >> 4) & 1].  Five double-float additions per lane instead of ten for two butterflies.
__device__ __forceinline__ DF warp_reduce_scatter2(DF v0, DF v1) {
  const bool h = threadIdx.x & 16;
  DF s = df_add(h ? v1 : v0, shfl_xor_df(h ? v0 : v1, 16));
#pragma unroll
  for (int o = 8; o > 0; o >>= 1) s = df_add(s, shfl_xor_df(s, o));
  return s;
}

// Reduce-scatter of eight per-lane values over a warp: lane L returns the warp-wide sum of
// v[(L >> 2) & 7] (nine double-float additions per lane instead of forty).
__device__ __forceinline__ DF warp_reduce_scatter8(DF v[8]) {
  const int lane = threadIdx.x & 31;
  {
    const bool h = lane & 16;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const DF send = h ? v[i] : v[4 + i];
      const DF mine = h ? v[4 + i] : v[i];
      v[i] = df_add(mine, shfl_xor_df(send, 16));
    }
  }
  {
    const bool h = lane & 8;
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const DF send = h ? v[i] : v[2 + i];
      const DF mine = h ? v[2 + i] : v[i];
      v[i] = df_add(mine, shfl_xor_df(send, 8));
    }
  }
  {
    const bool h = lane & 4;
    const DF send = h ? v[0] : v[1];
    const DF mine = h ? v[1] : v[0];
    v[0] = df_add(mine, shfl_xor_df(send, 4));
  }
  v[0] = df_add(v[0], shfl_xor_df(v[0], 2));
  v[0] = df_add(v[0], shfl_xor_df(v[0], 1));
  return v[0];
}

// Packed pairs: two independent FP32 lanes in one 64-bit register, operated on by the f32x2
// arithmetic of sm_100-class GPUs (one instruction for both lanes, same IEEE rounding per lane).
typedef unsigned long long f2x;

__device__ __forceinline__ f2x pk2(float a, float b) {
  f2x d;
  asm("mov.b64 %0, {%1, %2};" : "=l"(d) : "f"(a), "f"(b));
  return d;
}
__device__ __forceinline__ void upk2(f2x v, float& a, float& b) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}
__device__ __forceinline__ f2x add2(f2x a, f2x b) {
  f2x d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f2x sub2(f2x a, f2x b) {
  f2x d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f2x mul2(f2x a, f2x b) {
  f2x d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f2x fma2(f2x a, f2x b, f2x c) {
  f2x d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}

// two double-float accumulators, lane-wise
struct DF2 {
  f2x hi, lo;
};

// s += a * (bh + bl) lane-wise; nbh = -bh.  The rounded product is formed negated (pn = a * nbh,
// exact negation) so that its exact error is one fused multiply-add, a * bh + pn; TwoSum adds
// p = -pn to the high word.
__device__ __forceinline__ void df2_add_prod(DF2& s, f2x a, f2x bh, f2x nbh, f2x bl) {
  const f2x pn = mul2(a, nbh);
  const f2x pe = fma2(a, bh, pn);
  const f2x t = sub2(s.hi, pn);
  const f2x z = sub2(t, s.hi);
  const f2x e = sub2(sub2(s.hi, sub2(t, z)), add2(pn, z));
  s.hi = t;
  s.lo = add2(add2(fma2(a, bl, s.lo), pe), e);
}

// the same with the negated product formed from a with both sign bits flipped (an integer
// operation off the FP32 pipe) instead of a stored -bh
__device__ __forceinline__ void df2_add_prod_nj(DF2& s, f2x a, f2x bh, f2x bl) {
  const f2x pn = mul2(a ^ 0x8000000080000000ull, bh);
  const f2x pe = fma2(a, bh, pn);
  const f2x t = sub2(s.hi, pn);
  const f2x z = sub2(t, s.hi);
  const f2x e = sub2(sub2(s.hi, sub2(t, z)), add2(pn, z));
  s.hi = t;
  s.lo = add2(add2(fma2(a, bl, s.lo), pe), e);
}

__device__ __forceinline__ void df2_split(DF2 s, DF& a, DF& b) {
  upk2(s.hi, a.hi, b.hi);
  upk2(s.lo, a.lo, b.lo);
}

}  // namespace ngd
