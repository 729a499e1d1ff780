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

// Sum accumulators with one interface: add / subtract table entry i, where a
// table exists as FP64 and as (hi, lo) float pairs.  AccD sums the FP64 table
// on the FP64 pipe; AccF sums the float pairs in double-float.
struct AccD {
    double v = 0.0;
    __device__ __forceinline__ void add(const double *t, const float2 *, int64_t i) { v += __ldg(t + i); }
    __device__ __forceinline__ void sub(const double *t, const float2 *, int64_t i) { v -= __ldg(t + i); }
    __device__ __forceinline__ void neg() { v = -v; }
    __device__ __forceinline__ void add_const(double c) { v += c; }
    __device__ __forceinline__ double value() const { return v; }
};

struct AccF {
    float h = 0.0f, l = 0.0f;
    __device__ __forceinline__ void add(const double *, const float2 *t, int64_t i) {
        const float2 x = __ldg(t + i);
        df_add2(h, l, x.x, x.y);
    }
    __device__ __forceinline__ void sub(const double *, const float2 *t, int64_t i) {
        const float2 x = __ldg(t + i);
        df_add2(h, l, -x.x, -x.y);
    }
    __device__ __forceinline__ void neg() { h = -h; l = -l; }
    __device__ __forceinline__ void add_const(double c) {   // host-side constants only (e_core)
        const float ch = (float)c;
        df_add2(h, l, ch, (float)(c - (double)ch));
    }
    __device__ __forceinline__ double value() const { return df_to_double(h, l); }
};

// (hi, lo) += a * b for double-float a, b (products exact by FMA, TwoSum on the
// high words; the low words collect the rest)
__device__ __forceinline__ void df_fma(float &hi, float &lo, float ah, float al, float bh, float bl) {
    const float ph = ah * bh;
    const float pe = fmaf(ah, bh, -ph);
    const float pl = fmaf(ah, bl, fmaf(al, bh, pe));
    float s, e;
    df_two_sum(hi, ph, s, e);
    hi = s;
    lo = __fadd_rn(lo, __fadd_rn(e, pl));
}

// renormalise (hi, lo) so that |lo| <= ulp(hi) / 2
__device__ __forceinline__ void df_norm(float &hi, float &lo) {
    const float s = __fadd_rn(hi, lo);
    lo = __fsub_rn(lo, __fsub_rn(s, hi));
    hi = s;
}

// FP64 array -> (hi, lo) float pairs, hi = x rounded to float, lo = the rest
// rounded to float (|x - hi - lo| <= 2^-48 |x| for x in the float range).
void split_df(const double *x, int64_t n, float2 *out, cudaStream_t s);

}  // namespace hb
