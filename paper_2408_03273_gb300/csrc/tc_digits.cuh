// tc_digits.cuh -- exact BF16 digit planes of fixed-point numbers for the tensor-core sums
// (recip_tc.cu, mmrecip_tc.cu), and 2^61 fixed-point complex arithmetic on 32-bit halves.
//
// A 48-bit fixed-point value v (|v| <= 2^48) is written as seven balanced planes, a leading one
// and six base-128 digits: v 2^-48 = 2^-6 sum_{s<7} p_s with p_0 in [-64, 64] and
// p_s in [-64, 63] 2^-7s; every p_s has at most 7 significant bits, so it is exact in BF16 and
// products of two planes are exact in FP32.
#pragma once
#include <stdint.h>

namespace qmmm {
namespace tcd {

constexpr int ND = 7;                              // planes
constexpr double FIX61 = 2305843009213693952.0;    // 2^61

// Balanced digits: w = v + 64 sum_{k<6} 2^7k; plane 0 = w >> 42 (|.| <= 64), plane s >= 1 =
// (((w >> 7 (6 - s)) & 127) - 64) 2^-7s in [-64, 63] 2^-7s, so sum_s p_s = 2^-42 v exactly and the
// digit products have random signs (their sums do not drift).  Each plane is exact in BF16.
constexpr long long BAL = 64ll * (((1ll << 42) - 1) / 127);
struct Planes { float p[ND]; };
__device__ __forceinline__ Planes planes(long long w)
{
    Planes r;
    const uint32_t lo = (uint32_t)w, hi = (uint32_t)((unsigned long long)w >> 32);
    r.p[0] = (float)((int)hi >> 10);
    uint32_t u[ND - 1];  // u[k] = bits [7k, 7k + 7) of w (higher bits masked below)
    u[0] = lo;
    u[1] = lo >> 7;
    u[2] = lo >> 14;
    u[3] = lo >> 21;
    u[4] = __funnelshift_r(lo, hi, 28);
    u[5] = hi >> 3;
#pragma unroll
    for (int s = 1; s < ND; ++s) {
        const uint32_t mag = (uint32_t)(127 + 23 - 7 * s) << 23;  // 2^(23-7s): mantissa LSB 2^-7s
        r.p[s] = __uint_as_float(mag | (u[ND - 1 - s] & 127u)) - __uint_as_float(mag | 64u);
    }
    return r;
}
// (lo, hi) as BF16 (exact values) in one 32-bit word, lo at the lower K index
__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi)
{
    return __byte_perm(__float_as_uint(lo), __float_as_uint(hi), 0x7632);
}

// 2^61 fixed point split into 32-bit halves: x = h 2^31 + l, l in [0, 2^31), |h| <= 2^30; an int4
// holds (re h, re l, im h, im l)
__device__ __forceinline__ int4 split61(long long re, long long im)
{
    return make_int4((int)(re >> 31), (int)(re & 0x7fffffff), (int)(im >> 31), (int)(im & 0x7fffffff));
}
__device__ __forceinline__ long long join61(int h, int l) { return (long long)h * 2147483648ll + l; }
// (x y) / 2^62 for 2^61 values, within 1 unit: the low x low term is dropped
__device__ __forceinline__ long long mul61(long long x, long long y)
{
    const int xh = (int)(x >> 31), xl = (int)(x & 0x7fffffff), yh = (int)(y >> 31), yl = (int)(y & 0x7fffffff);
    return (long long)xh * yh + (((long long)xh * yl + (long long)xl * yh) >> 31);
}
// complex product of two split 2^61 values at 2^60 scale, within 2 units (six 32 x 32 -> 64
// products and four for the cross terms)
__device__ __forceinline__ void cmul61(const int4 x, const int4 y, long long &re, long long &im)
{
    const long long mr = (long long)x.x * y.y + (long long)x.y * y.x - (long long)x.z * y.w - (long long)x.w * y.z;
    const long long mi = (long long)x.x * y.w + (long long)x.y * y.z + (long long)x.z * y.y + (long long)x.w * y.x;
    re = (long long)x.x * y.x - (long long)x.z * y.z + (mr >> 31);
    im = (long long)x.x * y.z + (long long)x.z * y.x + (mi >> 31);
}
// balanced-digit input w of a value v at 2^(48 + shift) scale: rounded to 2^-48, offset by BAL
__device__ __forceinline__ long long fixw(long long v, int shift)
{
    return (v + (1ll << (shift - 1)) + (BAL << shift)) >> shift;
}

__device__ __forceinline__ long long fix61(double v) { return __double2ll_rn(v * FIX61); }

// The same balanced split with NP planes of a (6 + 7 (NP - 1))-bit value v: the leading plane
// w >> 7 (NP - 1) in [-64, 64] and NP - 1 base-128 digits; bal<NP>() is the offset that makes the
// digits balanced; NP = 7 is planes() above.
template <int NP>
__host__ __device__ constexpr long long bal()
{
    return 64ll * (((1ll << (7 * (NP - 1))) - 1) / 127);
}
template <int NP>
struct PlanesN { float p[NP]; };
template <int NP>
__device__ __forceinline__ PlanesN<NP> planes_n(long long w)
{
    PlanesN<NP> r;
    r.p[0] = (float)(int)(w >> (7 * (NP - 1)));
#pragma unroll
    for (int s = 1; s < NP; ++s) {
        const uint32_t u = (uint32_t)((unsigned long long)w >> (7 * (NP - 1 - s))) & 127u;
        const uint32_t mag = (uint32_t)(127 + 23 - 7 * s) << 23;  // 2^(23-7s): mantissa LSB 2^-7s
        r.p[s] = __uint_as_float(mag | u) - __uint_as_float(mag | 64u);
    }
    return r;
}

}  // namespace tcd
}  // namespace qmmm
