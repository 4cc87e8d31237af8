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

// Knuth's two-sum: s + e = a + b exactly
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}
// (h, l) * (sh + sl) for a float-float real scale, normalised
__device__ __forceinline__ void ff_scale(float &h, float &l, float sh, float sl) {
    const float p = h * sh;
    float e = fmaf(h, sh, -p);
    e = fmaf(h, sl, e);
    e = fmaf(l, sh, e);
    h = p + e;
    l = e - (h - p);
}

// (h, l) += (bh, bl), float-float sum by Knuth's two-sum, renormalised
__device__ __forceinline__ void ff_add(float &h, float &l, float bh, float bl) {
    const float s = h + bh;
    const float bb = s - h;
    const float t = (h - (s - bb)) + (bh - bb) + l + bl;
    h = s + t;
    l = t - (h - s);
}

// One Givens step of a rotation chain in float-float: h <- c a - conj(s) h, with c real
// {hi, lo}, s, a, h complex {re hi, im hi, re lo, im lo}.
__device__ __forceinline__ float4 ff_rot_step(float2 c, float4 s, float4 a, float4 h) {
    float rh = 0.f, rl = 0.f, ih = 0.f, il = 0.f;
    ff_mac(rh, rl, c.x, c.y, a.x, a.z);
    ff_mac(rh, rl, -s.x, -s.z, h.x, h.z);
    ff_mac(rh, rl, -s.y, -s.w, h.y, h.w);
    ff_mac(ih, il, c.x, c.y, a.y, a.w);
    ff_mac(ih, il, -s.x, -s.z, h.y, h.w);
    ff_mac(ih, il, s.y, s.w, h.x, h.z);
    ff_norm(rh, rl);
    ff_norm(ih, il);
    return make_float4(rh, ih, rl, il);
}

// acc += c x (complex float-float; acc = {re hi, im hi, re lo, im lo})
__device__ __forceinline__ void ff_cmac(float &rh, float &rl, float &ih, float &il, const float4 &c,
                                        const float4 &x) {
    ff_mac(rh, rl, c.x, c.z, x.x, x.z);
    ff_mac(rh, rl, -c.y, -c.w, x.y, x.w);
    ff_mac(ih, il, c.x, c.z, x.y, x.w);
    ff_mac(ih, il, c.y, c.w, x.x, x.z);
}

// ---------------------------------------------------------------- packed float-float pairs
// The same arithmetic on two values at once with GB300's packed FP32 instructions
// ({add,sub,mul,fma}.rn.f32x2): a float2 holds the high (or low) words of two float-float
// numbers, typically the real and imaginary parts of one complex value.
__device__ __forceinline__ float2 f2_add(float2 a, float2 b) {
    float2 d;
    asm("{\n\t.reg .b64 ra, rb, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
        "add.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(d.x), "=f"(d.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}
__device__ __forceinline__ float2 f2_sub(float2 a, float2 b) {
    float2 d;
    asm("{\n\t.reg .b64 ra, rb, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
        "sub.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(d.x), "=f"(d.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}
__device__ __forceinline__ float2 f2_mul(float2 a, float2 b) {
    float2 d;
    asm("{\n\t.reg .b64 ra, rb, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
        "mul.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(d.x), "=f"(d.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}
__device__ __forceinline__ float2 f2_fma(float2 a, float2 b, float2 c) {
    float2 d;
    asm("{\n\t.reg .b64 ra, rb, rc, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
        "mov.b64 rc, {%6, %7};\n\tfma.rn.f32x2 rd, ra, rb, rc;\n\tmov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(d.x), "=f"(d.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
    return d;
}
// (H, L) += (Ah + Al)(Bh + Bl) elementwise, dropping Al*Bl; nBh = -Bh is passed in (it is
// formed once per operand and reused) so that no separate negation is issued: -p = Ah * nBh
// exactly, the product error is fma(Ah, Bh, -p), and H + p = H - (-p) is Knuth's two-sum.
__device__ __forceinline__ void ff2_mac(float2 &H, float2 &L, float2 Ah, float2 Al, float2 Bh, float2 Bl,
                                        float2 nBh) {
    const float2 np = f2_mul(Ah, nBh);
    float2 e = f2_fma(Ah, Bh, np);
    e = f2_fma(Ah, Bl, e);
    e = f2_fma(Al, Bh, e);
    const float2 s = f2_sub(H, np);
    const float2 bb = f2_sub(s, H);
    const float2 t = f2_sub(f2_sub(H, f2_sub(s, bb)), f2_add(np, bb));
    H = s;
    L = f2_add(L, f2_add(t, e));
}

}  // namespace heom
