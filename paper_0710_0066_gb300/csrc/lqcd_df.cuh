// lqcd_df.cuh -- double-float ("df") arithmetic for the double-precision
// hopping sweeps of the mixed-precision path.
//
// GB300 runs FP64 at a small fraction of its FP32 rate, so a double hopping
// sweep is bound by the FP64 pipe, not by memory.  A df number is the
// unevaluated sum hi + lo of two floats (about 47 significant bits here);
// its sums and products use only FP32 adds and FMAs:
//   - Knuth's TwoSum: s + e = a + b exactly (six adds);
//   - the FMA product: p = a b, e = fma(a, b, -p), p + e = a b exactly.
// (T. J. Dekker, Numer. Math. 18 (1971) 224; D. E. Knuth, TAOCP vol. 2,
// Sec. 4.2.2; Y. Hida, X. S. Li, D. H. Bailey, ARITH-15 (2001) 155.)
//
// Doubles are split into df with integer operations only (no conversion
// through the FP64 pipe): hi takes the sign, the exponent and the leading
// 23 fraction bits; lo the next 23 of the remaining 29 fraction bits, so
// the split is exact to a relative 2^-46.  Values below 2^-126 in
// magnitude (and zeros) split to hi only; below 2^-80 lo is dropped.
// Results go back to double as (double) hi + (double) lo.
//
// Every function is host- and device-callable so that the host compiler
// can test them against long-double arithmetic.
#pragma once
#include <math.h>
#include <stdint.h>
#include <string.h>

#ifndef LQ_HD
#define LQ_HD __host__ __device__ __forceinline__
#endif

LQ_HD uint64_t df_bits64(double x)
{
#ifdef __CUDA_ARCH__
    return (uint64_t)__double_as_longlong(x);
#else
    uint64_t b;
    memcpy(&b, &x, 8);
    return b;
#endif
}

LQ_HD float df_f32(uint32_t b)
{
#ifdef __CUDA_ARCH__
    return __uint_as_float(b);
#else
    float x;
    memcpy(&x, &b, 4);
    return x;
#endif
}

// a * b and fma(a, b, c), each rounded once and never merged by the compiler
LQ_HD float df_mul_rn(float a, float b)
{
#ifdef __CUDA_ARCH__
    return __fmul_rn(a, b);
#else
    volatile float p = a * b;
    return p;
#endif
}

LQ_HD float df_fma_rn(float a, float b, float c)
{
#ifdef __CUDA_ARCH__
    return __fmaf_rn(a, b, c);
#else
    return fmaf(a, b, c);
#endif
}

struct df;
LQ_HD df df_split(double x);

struct df {
    float hi, lo;
    df() = default;
    LQ_HD constexpr df(float h, float l) : hi(h), lo(l) {}
    LQ_HD explicit df(int z) : hi((float)z), lo(0.f) {}
    LQ_HD explicit df(double x) { *this = df_split(x); }
};

// s + e = a + b exactly
LQ_HD void df_two_sum(float a, float b, float& s, float& e)
{
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// Sums and products leave the pair unnormalised (|lo| may exceed half an
// ulp of hi): no FastTwoSum after every operation, which cuts the sweep's
// instruction count by a third.  The value hi + lo keeps its ~2^-46
// accuracy relative to the operands' magnitudes (after a cancellation the
// small result sits partly in lo and carries float precision of itself,
// which is the same absolute accuracy).
LQ_HD df operator+(df a, df b)
{
    float s, e;
    df_two_sum(a.hi, b.hi, s, e);
    return df(s, e + (a.lo + b.lo));
}

LQ_HD df operator-(df a) { return df(-a.hi, -a.lo); }

LQ_HD df operator-(df a, df b) { return a + (-b); }

LQ_HD df operator*(df a, df b)
{
    const float p = df_mul_rn(a.hi, b.hi);
    float e = df_fma_rn(a.hi, b.hi, -p);
    e = df_fma_rn(a.hi, b.lo, e);
    e = df_fma_rn(a.lo, b.hi, e);
    return df(p, e);
}

// hi + lo as a normalised pair (|lo| <= half an ulp of hi)
LQ_HD df df_norm(df a)
{
    df r;
    df_two_sum(a.hi, a.lo, r.hi, r.lo);
    return r;
}

LQ_HD df df_split(double x)
{
    const uint64_t b = df_bits64(x);
    const uint32_t sign = (uint32_t)(b >> 32) & 0x80000000u;
    const int e = (int)((b >> 52) & 0x7ff);  // biased double exponent
    if (e == 0) return df(0.f, 0.f);        // zero (and double subnormals)
    const int ef = e - 1023 + 127;           // biased float exponent of hi
    if (ef <= 0 || ef >= 255) return df((float)x, 0.f);  // outside the float range, inf, nan
    const float h = df_f32(sign | ((uint32_t)ef << 23) | (uint32_t)((b >> 29) & 0x7fffffu));
    // remainder: the low 29 fraction bits m, worth m 2^(e - 1075); keep the
    // top 23 (m23 = m >> 6, worth m23 2^(e - 1069)).  float(m23) is exact:
    // 2^23 + m23 has the float bit pattern 0x4B000000 | m23.
    const uint32_t m23 = (uint32_t)(b & 0x1fffffffu) >> 6;
    float l = df_f32(0x4B000000u | m23) - 8388608.0f;
    const int es = e - 1069 + 127;  // biased float exponent of 2^(e - 1069)
    l = es > 0 ? l * df_f32((uint32_t)es << 23) : 0.f;
    return df(h, sign ? -l : l);
}

LQ_HD double df_to_double(df a) { return (double)a.hi + (double)a.lo; }
