// ln g table value types shared by the sampling kernels of librewl: the
// exact update value + n * ln f of one bin in each table format, and the
// float approximation the decision screens with.
#pragma once

#include "rewl_internal.cuh"

namespace rewl {
namespace tab {

// |x| rounded toward zero to float with integer operations only (no FP64
// instruction): relative error below 2^-23; 0 for |x| < 2^-126; +-inf for
// |x| >= 2^128.
__device__ __forceinline__ float trunc_f(double x)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const uint32_t hi = (uint32_t)(b >> 32);
    const int ex = (int)((hi >> 20) & 0x7FFu);
    if (ex < 897) return 0.0f;
    if (ex > 1150) return __uint_as_float((hi & 0x80000000u) | 0x7F800000u);
    return __uint_as_float((hi & 0x80000000u) | ((uint32_t)(ex - 896) << 23) | ((uint32_t)(b >> 29) & 0x7FFFFFu));
}

__device__ __forceinline__ double unit_open_d(uint32_t x) { return ((double)x + 0.5) * 0x1p-32; }

// (hi, lo) + x for a float x, compensated (Knuth's two-sum, then a fast
// renormalisation): exact while the result has at most ~48 significant bits
// and every addend is a multiple of the finest ln f.
__device__ __forceinline__ float2 add2(float2 a, float x)
{
    const float s = __fadd_rn(a.x, x);
    const float bb = __fsub_rn(s, a.x);
    const float err = __fadd_rn(__fsub_rn(a.x, __fsub_rn(s, bb)), __fsub_rn(x, bb));
    const float l2 = __fadd_rn(a.y, err);
    const float h2 = __fadd_rn(s, l2);
    const float l3 = __fsub_rn(l2, __fsub_rn(h2, s));
    return make_float2(h2, l3);
}

// Table value types.  Val: the value of one bin as kept in registers.
template <int PREC>
struct Tab;

template <>
struct Tab<REWL_FP64> {
    using Elem = double;
    using Val = double;
    __device__ static Val load(const Elem *t, int i) { return t[i]; }
    __device__ static float approx(Val v) { return trunc_f(v); }       // |err| < 2^-23 |v|
    __device__ static double exact(Val v) { return v; }
    // v + n * lnf (exact for the dyadic schedule)
    __device__ static Val add(Val v, int n, double lnf, float) { return fma((double)n, lnf, v); }
};

template <>
struct Tab<REWL_F32X2> {
    using Elem = float2;
    using Val = float2;
    __device__ static Val load(const Elem *t, int i) { return t[i]; }
    __device__ static float approx(Val v) { return v.x; }               // |err| <= 2^-24 |v|
    __device__ static double exact(Val v) { return (double)v.x + (double)v.y; }
    __device__ static Val add(Val v, int n, double, float lnf32) { return add2(v, __fmul_rn((float)n, lnf32)); }
};

// Plain float (demonstration of the precision loss the compensated pair
// avoids): each visit adds ln f to a single float and rounds.
template <>
struct Tab<REWL_F32> {
    using Elem = float;
    using Val = float;
    __device__ static Val load(const Elem *t, int i) { return t[i]; }
    __device__ static float approx(Val v) { return v; }
    __device__ static double exact(Val v) { return (double)v; }
    __device__ static Val add(Val v, int n, double, float lnf32)
    {
        for (int i = 0; i < n; ++i) v = __fadd_rn(v, lnf32);
        return v;
    }
};

}  // namespace tab
}  // namespace rewl
