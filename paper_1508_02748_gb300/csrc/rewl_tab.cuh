// ln g table formats shared by the kernels of librewl.
//
// Exact formats (REWL_FP64, REWL_F32X2) keep a base per bin and the
// iteration's visit count H beside it; ln g = base + max(H, 0) * ln f is
// formed only where a value is needed exactly.  With ln f = 2^-k every such
// value is a dyadic rational of at most ~44 significant bits in the
// workloads, so double arithmetic and the compensated float pair (hi, lo)
// hold it exactly.  REWL_F32 (plain float, the precision demonstration)
// keeps ln g itself and rounds at every visit.
#pragma once

#include "rewl_internal.cuh"

namespace rewl {
namespace tab {

__device__ __forceinline__ double unit_open_d(uint32_t x) { return ((double)x + 0.5) * 0x1p-32; }

template <int PREC>
struct Tab;

template <>
struct Tab<REWL_FP64> {
    using Elem = double;
    __device__ static double exact(Elem v) { return v; }
    __device__ static Elem from(double v) { return v; }
};

// (hi, lo) with hi = v rounded to float and lo = the rest: exact for values
// of at most 48 significant bits.
template <>
struct Tab<REWL_F32X2> {
    using Elem = float2;
    __device__ static double exact(Elem v) { return (double)v.x + (double)v.y; }
    __device__ static Elem from(double v)
    {
        const float hi = __double2float_rn(v);
        return make_float2(hi, __double2float_rn(v - (double)hi));
    }
};

template <>
struct Tab<REWL_F32> {
    using Elem = float;
    __device__ static double exact(Elem v) { return (double)v; }
    __device__ static Elem from(double v) { return __double2float_rn(v); }
};

// REWL_F32: n visits, each adding ln f and rounding to float
__device__ __forceinline__ float f32_visits(float v, int n, float lnf32)
{
    for (int i = 0; i < n; ++i) v = __fadd_rn(v, lnf32);
    return v;
}

}  // namespace tab
}  // namespace rewl
