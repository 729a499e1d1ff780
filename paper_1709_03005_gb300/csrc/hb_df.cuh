// Double-float arithmetic on the FP32 pipes: a value is an unevaluated sum
// hi + lo of two floats (about 48 significant bits).  The error-free
// transformations are Knuth's TwoSum and the FMA product error
// (Dekker / Ogita-Rump-Oishi); the conversion back to FP64 uses integer
// operations only, because the FP64 pipe of this part is slow.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace hb {

// s + e = a + b exactly
__device__ __forceinline__ void df_two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    const float bp = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bp)), __fsub_rn(b, bp));
}

// (hi, lo) := (ah, al) + (bh, bl), renormalised
__device__ __forceinline__ void df_add2(float &hi, float &lo, float bh, float bl) {
    float s, e;
    df_two_sum(hi, bh, s, e);
    e = __fadd_rn(e, __fadd_rn(lo, bl));
    hi = __fadd_rn(s, e);
    lo = __fsub_rn(e, __fsub_rn(hi, s));
}

// hi + lo as a double, with integer operations only.  Both are aligned into a
// 64-bit integer with 38 bits of headroom below the larger exponent, added
// exactly, and the result is truncated to 53 bits (relative error below
// 2^-52).  FP32 subnormals are treated as zero.
__device__ __forceinline__ double df_to_double(float hi, float lo) {
    const uint32_t bh = __float_as_uint(hi), bl = __float_as_uint(lo);
    const int eh = (int)((bh >> 23) & 0xFF), el = (int)((bl >> 23) & 0xFF);
    long long mh = eh ? (long long)((bh & 0x7FFFFFu) | 0x800000u) : 0;
    long long ml = el ? (long long)((bl & 0x7FFFFFu) | 0x800000u) : 0;
    if (bh >> 31) mh = -mh;
    if (bl >> 31) ml = -ml;
    const int base = eh > el ? eh : el;
    // value = (mh 2^(eh-base) + ml 2^(el-base)) * 2^(base - 150)
    const int sh_h = 38 - (base - eh), sh_l = 38 - (base - el);
    long long acc = 0;
    if (mh) acc += sh_h >= 0 ? (mh << sh_h) : (sh_h > -63 ? (mh >> -sh_h) : 0);
    if (ml) acc += sh_l >= 0 ? (ml << sh_l) : (sh_l > -63 ? (ml >> -sh_l) : 0);
    if (acc == 0) return 0.0;
    const unsigned long long neg = acc < 0 ? 1ull : 0ull;
    unsigned long long u = neg ? (unsigned long long)(-acc) : (unsigned long long)acc;
    const int lz = __clzll((long long)u);            // leading zeros, u > 0
    const int top = 63 - lz;                          // position of the leading one
    // normalise to 53 bits: leading one at bit 52
    if (top > 52) u >>= (top - 52);
    else u <<= (52 - top);
    // exponent: value = u * 2^(top - 52) * 2^(base - 150 - 38), u in [2^52, 2^53)
    const int e2 = top + base - 150 - 38;             // unbiased exponent of the leading one
    const long long be = (long long)e2 + 1023;
    if (be <= 0) return 0.0;                          // below the FP64 normal range
    const unsigned long long bits = (neg << 63) | ((unsigned long long)be << 52) | (u & 0xFFFFFFFFFFFFFull);
    return __longlong_as_double((long long)bits);
}

// FP64 array -> (hi, lo) float pairs, hi = x rounded to float, lo = the rest
// rounded to float (|x - hi - lo| <= 2^-48 |x| for x in the float range).
void split_df(const double *x, int64_t n, float2 *out, cudaStream_t s);

}  // namespace hb
