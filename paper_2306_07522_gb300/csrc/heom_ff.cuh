// Float-float (double-single) arithmetic for the kernels that would otherwise spend GB300's
// scarce FP64 issue slots.
#pragma once

#include "heom_internal.h"

namespace heom {

// ---------------------------------------------------------------- float-float arithmetic
// GB300 issues FP64 at 1/64 of its FP32 rate, and the Gram-Schmidt loops are nothing but
// complex multiply-adds. They run in float-float instead: a value is an unevaluated sum
// hi + lo of two FP32 numbers (about 48 significant bits, unit roundoff 2^-48 ~ 3.6e-15),
// products by the FMA-based exact product of Dekker/Kahan (p = a*b, e = fma(a, b, -p)),
// sums by Knuth's two-sum. A complex value is a float4 {hi.re, hi.im, lo.re, lo.im}.
// Per-thread results are turned back into FP64 before any block or grid reduction.
__device__ __forceinline__ float4 ff_split(cx<double> a) {
    const float hr = __double2float_rn(a.re), hi = __double2float_rn(a.im);
    return make_float4(hr, hi, __double2float_rn(a.re - (double)hr), __double2float_rn(a.im - (double)hi));
}
__device__ __forceinline__ cx<double> ff_join(float4 f) {
    return cx<double>{(double)f.x + (double)f.z, (double)f.y + (double)f.w};
}
// (sh, sl) += (ah + al)(bh + bl), dropping al*bl (2^-48 relative)
__device__ __forceinline__ void ff_mac(float &sh, float &sl, float ah, float al, float bh, float bl) {
    const float p = ah * bh;
    float e = fmaf(ah, bh, -p);
    e = fmaf(ah, bl, e);
    e = fmaf(al, bh, e);
    const float s = sh + p;
    const float bb = s - sh;
    const float t = (sh - (s - bb)) + (p - bb);
    sh = s;
    sl += t + e;
}
// normalise (sh, sl) so that |sl| <= ulp(sh) / 2
__device__ __forceinline__ void ff_norm(float &sh, float &sl) {
    const float s = sh + sl;
    sl = sl - (s - sh);
    sh = s;
}

}  // namespace heom
