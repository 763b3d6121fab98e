// grape_num.cuh - the two complex number types the kernels are written over.
//
//  NumD   native FP64 complex (double2 storage).
//  NumF   double-float complex: every real part is an unevaluated sum hi + lo
//         of two FP32 numbers with |lo| <= ulp(hi)/2, about 48 significant
//         bits (float4 storage: re.hi, im.hi, re.lo, im.lo), computed on
//         FP32 pairs (re, im) with Blackwell's paired instructions.  Arithmetic
//         uses the error-free transformations TwoSum (Knuth), Fast2Sum
//         (Dekker) and TwoProduct through the fused multiply-add, all with
//         explicitly rounded intrinsics so the compiler can neither contract
//         nor reassociate them.  GB300 issues FP32 at ~67x its FP64 rate,
//         which is what makes the pair arithmetic the fast path.
//
// Both types are 16 bytes per complex entry, so every buffer of the path has
// the same size in either precision.  Accumulators (Acc) collect products of
// complex numbers; for NumF the high parts are summed with TwoSum and all
// rounding errors and cross terms gather in the low parts, normalised once
// at the end (lazy renormalisation).
#pragma once

#include <cuda_runtime.h>

namespace grape_num {

// ---------------------------------------------------------------- FP32 EFTs
struct ff {
    float h, l;
};

__device__ __forceinline__ ff two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}
// requires |a| >= |b| (or a == 0)
__device__ __forceinline__ ff fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ ff ff_mul(ff a, ff b) {
    const float p = __fmul_rn(a.h, b.h);
    float e = __fmaf_rn(a.h, b.h, -p);
    e = __fmaf_rn(a.h, b.l, e);
    e = __fmaf_rn(a.l, b.h, e);
    return fast_two_sum(p, e);
}
// x + s*w: the product's high part is exact (FMA) and its error joins the
// cross terms and the low parts, renormalised once.  One TwoSum instead of
// the accurate sum's two: the error is about 2^-47 (|x| + |s w|), an
// absolute bound on the scale of the operands, which is what the
// propagation needs (its tolerances are relative to the largest entry).
__device__ __forceinline__ ff ff_axpy(ff s, ff w, ff x) {
    const float p = __fmul_rn(s.h, w.h);
    float e = __fmaf_rn(s.h, w.h, -p);
    e = __fmaf_rn(s.h, w.l, e);
    e = __fmaf_rn(s.l, w.h, e);
    const ff t = two_sum(x.h, p);
    return fast_two_sum(t.h, __fadd_rn(t.l, __fadd_rn(x.l, e)));
}
// g*x + b*w, same error model
__device__ __forceinline__ ff ff_lin2(ff g, ff x, ff b, ff w) {
    const float p = __fmul_rn(g.h, x.h);
    float e = __fmaf_rn(g.h, x.h, -p);
    e = __fmaf_rn(g.h, x.l, e);
    e = __fmaf_rn(g.l, x.h, e);
    const float q = __fmul_rn(b.h, w.h);
    float f = __fmaf_rn(b.h, w.h, -q);
    f = __fmaf_rn(b.h, w.l, f);
    f = __fmaf_rn(b.l, w.h, f);
    const ff t = two_sum(p, q);
    return fast_two_sum(t.h, __fadd_rn(t.l, __fadd_rn(e, f)));
}
// a + b with one TwoSum (same error model as ff_axpy)
__device__ __forceinline__ ff ff_sum(ff a, ff b) {
    const ff t = two_sum(a.h, b.h);
    return fast_two_sum(t.h, __fadd_rn(t.l, __fadd_rn(a.l, b.l)));
}
__host__ __device__ __forceinline__ ff ff_from_double(double x) {
    const float h = (float)x;
    return {h, (float)(x - (double)h)};
}
__host__ __device__ __forceinline__ double ff_to_double(ff a) { return (double)a.h + (double)a.l; }

// lazy accumulator of one real part: acc += a*b (sign s = +1/-1)
struct lacc {
    float h, l;
};
__device__ __forceinline__ void lacc_fma(lacc &acc, float ah, float al, float bh, float bl) {
    const float p = __fmul_rn(ah, bh);
    float e = __fmaf_rn(ah, bh, -p);
    e = __fmaf_rn(ah, bl, e);
    e = __fmaf_rn(al, bh, e);
    const ff s = two_sum(acc.h, p);
    acc.h = s.h;
    acc.l = __fadd_rn(acc.l, __fadd_rn(s.l, e));
}
__device__ __forceinline__ void lacc_fms(lacc &acc, float ah, float al, float bh, float bl) {
    lacc_fma(acc, -ah, -al, bh, bl);
}
__device__ __forceinline__ ff lacc_done(lacc a) { return two_sum(a.h, a.l); }

// ------------------------------------------------------------ number types
struct NumD {
    using store_t = double2;
    using real_t = double;
    struct val { double re, im; };
    struct acc { double re, im; };

    static __device__ __forceinline__ val load(const store_t &s) { return {s.x, s.y}; }
    // the real part alone (8-byte load)
    static __device__ __forceinline__ real_t load_re(const store_t &s) { return s.x; }
    static __device__ __forceinline__ store_t store(val v) { return make_double2(v.re, v.im); }
    static __device__ __forceinline__ val zero() { return {0.0, 0.0}; }
    static __device__ __forceinline__ acc acc_zero() { return {0.0, 0.0}; }
    static __device__ __forceinline__ real_t real_const(double x) { return x; }
    // acc += a * b
    static __device__ __forceinline__ void mac(acc &c, val a, val b) {
        c.re = fma(a.re, b.re, fma(-a.im, b.im, c.re));
        c.im = fma(a.re, b.im, fma(a.im, b.re, c.im));
    }
    // acc -= conj(a) * b
    static __device__ __forceinline__ void mac_conj_neg(acc &c, val a, val b) {
        c.re = fma(-a.re, b.re, fma(-a.im, b.im, c.re));
        c.im = fma(-a.re, b.im, fma(a.im, b.re, c.im));
    }
    // acc += a * conj(b)
    static __device__ __forceinline__ void mac_conjb(acc &c, val a, val b) {
        c.re = fma(a.re, b.re, fma(a.im, b.im, c.re));
        c.im = fma(a.im, b.re, fma(-a.re, b.im, c.im));
    }
    static __device__ __forceinline__ val done(acc c) { return {c.re, c.im}; }
    static __device__ __forceinline__ val raw(acc c) { return {c.re, c.im}; }
    static __device__ __forceinline__ acc acc_minus_i(acc c) { return {c.im, -c.re}; }
    static __device__ __forceinline__ acc acc_add(acc a, acc b) { return {a.re + b.re, a.im + b.im}; }
    // a - conj(b), a + b, a + c (c real)
    static __device__ __forceinline__ val sub_conj(val a, val b) { return {a.re - b.re, a.im + b.im}; }
    static __device__ __forceinline__ val add(val a, val b) { return {a.re + b.re, a.im + b.im}; }
    static __device__ __forceinline__ val add_real(val a, real_t c) { return {a.re + c, a.im}; }
    // a * conj(b)
    static __device__ __forceinline__ val mul_conjb(val a, val b) {
        return {fma(a.re, b.re, a.im * b.im), fma(a.im, b.re, -a.re * b.im)};
    }
    static __device__ __forceinline__ val minus_i(val a) { return {a.im, -a.re}; }
    static __device__ __forceinline__ real_t re(val a) { return a.re; }
    static __device__ __forceinline__ real_t im(val a) { return a.im; }
    static __device__ __forceinline__ val conj(val a) { return {a.re, -a.im}; }
    static __device__ __forceinline__ real_t neg_real(real_t a) { return -a; }
    static __device__ __forceinline__ real_t real_mul(real_t a, real_t b) { return a * b; }
    // acc += c * b, c real
    static __device__ __forceinline__ void mac_real(acc &w, real_t c, val b) {
        w.re = fma(c, b.re, w.re);
        w.im = fma(c, b.im, w.im);
    }
    // x + s*w
    static __device__ __forceinline__ val axpy(real_t s, val w, val x) {
        return {fma(s, w.re, x.re), fma(s, w.im, x.im)};
    }
    // g*x + b*w
    static __device__ __forceinline__ val lin2(real_t g, val x, real_t b, val w) {
        return {fma(g, x.re, b * w.re), fma(g, x.im, b * w.im)};
    }
    static __device__ __forceinline__ val scale(real_t s, val a) { return {s * a.re, s * a.im}; }
    static __device__ __forceinline__ double2 to_double2(val v) { return make_double2(v.re, v.im); }
    static __device__ __forceinline__ val from_double2(double2 v) { return {v.x, v.y}; }
};

// ------------------------------------------------------- paired FP32 EFTs
// Blackwell issues two FP32 operations per instruction on a float2 operand
// pair (FADD2 / FMUL2 / FFMA2, at the same flop rate as scalar FP32 in half
// the issue slots; negated operands and a broadcast lane cost nothing extra).
// The complex double-float type keeps its real and imaginary high parts in
// one pair and its low parts in another, so each transformation below runs
// the scalar one's exact operation sequence on both lanes at once: the
// results are those of lane-wise scalar code, bit for bit.
__device__ __forceinline__ float2 p_add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 p_sub(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }
__device__ __forceinline__ float2 p_mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 p_fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 p_neg(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 p_bx(float2 a) { return make_float2(a.x, a.x); }     // lane x twice
__device__ __forceinline__ float2 p_by(float2 a) { return make_float2(a.y, a.y); }     // lane y twice
__device__ __forceinline__ float2 p_b(float a) { return make_float2(a, a); }

// TwoSum and Fast2Sum on both lanes (as two_sum / fast_two_sum)
__device__ __forceinline__ void p_two_sum(float2 a, float2 b, float2 &s, float2 &e) {
    s = p_add(a, b);
    const float2 bb = p_sub(s, a);
    e = p_add(p_sub(a, p_sub(s, bb)), p_sub(b, bb));
}
__device__ __forceinline__ void p_fast_two_sum(float2 a, float2 b, float2 &s, float2 &e) {
    s = p_add(a, b);
    e = p_sub(b, p_sub(s, a));
}
// lacc_fma on both lanes: (acc_h, acc_l) += (xh + xl)(yh + yl) lane by lane
__device__ __forceinline__ void p_lacc_fma(float2 &ah, float2 &al, float2 xh, float2 xl, float2 yh, float2 yl) {
    const float2 p = p_mul(xh, yh);
    float2 e = p_fma(xh, yh, p_neg(p));
    e = p_fma(xh, yl, e);
    e = p_fma(xl, yh, e);
    float2 s, t;
    p_two_sum(ah, p, s, t);
    ah = s;
    al = p_add(al, p_add(t, e));
}
// ff_axpy, ff_lin2, ff_sum, ff_mul on both lanes (s, g, b: lane-broadcast scalars)
__device__ __forceinline__ void p_axpy(float2 sh, float2 sl, float2 wh, float2 wl, float2 xh, float2 xl,
                                       float2 &oh, float2 &ol) {
    const float2 p = p_mul(sh, wh);
    float2 e = p_fma(sh, wh, p_neg(p));
    e = p_fma(sh, wl, e);
    e = p_fma(sl, wh, e);
    float2 th, tl;
    p_two_sum(xh, p, th, tl);
    p_fast_two_sum(th, p_add(tl, p_add(xl, e)), oh, ol);
}
__device__ __forceinline__ void p_lin2(float2 gh, float2 gl, float2 xh, float2 xl, float2 bh, float2 bl,
                                       float2 wh, float2 wl, float2 &oh, float2 &ol) {
    const float2 p = p_mul(gh, xh);
    float2 e = p_fma(gh, xh, p_neg(p));
    e = p_fma(gh, xl, e);
    e = p_fma(gl, xh, e);
    const float2 q = p_mul(bh, wh);
    float2 f = p_fma(bh, wh, p_neg(q));
    f = p_fma(bh, wl, f);
    f = p_fma(bl, wh, f);
    float2 th, tl;
    p_two_sum(p, q, th, tl);
    p_fast_two_sum(th, p_add(tl, p_add(e, f)), oh, ol);
}
__device__ __forceinline__ void p_sum(float2 ah, float2 al, float2 bh, float2 bl, float2 &oh, float2 &ol) {
    float2 th, tl;
    p_two_sum(ah, bh, th, tl);
    p_fast_two_sum(th, p_add(tl, p_add(al, bl)), oh, ol);
}
__device__ __forceinline__ void p_mulff(float2 sh, float2 sl, float2 ah, float2 al, float2 &oh, float2 &ol) {
    const float2 p = p_mul(sh, ah);
    float2 e = p_fma(sh, ah, p_neg(p));
    e = p_fma(sh, al, e);
    e = p_fma(sl, ah, e);
    p_fast_two_sum(p, e, oh, ol);
}

struct NumF {
    // storage: re.h, im.h, re.l, im.l (the high pair, then the low pair)
    using store_t = float4;
    using real_t = ff;
    struct val { float2 h, l; };    // h = (re.h, im.h), l = (re.l, im.l)
    struct acc { float2 h, l; };    // lazy: the low pair collects every error

    static __device__ __forceinline__ val load(const store_t &s) {
        return {make_float2(s.x, s.y), make_float2(s.z, s.w)};
    }
    static __device__ __forceinline__ real_t load_re(const store_t &s) { return {s.x, s.z}; }
    static __device__ __forceinline__ store_t store(val v) { return make_float4(v.h.x, v.h.y, v.l.x, v.l.y); }
    static __device__ __forceinline__ val zero() { return {make_float2(0.f, 0.f), make_float2(0.f, 0.f)}; }
    static __device__ __forceinline__ acc acc_zero() { return {make_float2(0.f, 0.f), make_float2(0.f, 0.f)}; }
    static __device__ __forceinline__ real_t real_const(double x) { return ff_from_double(x); }
    // acc += a b: re += a.re b.re - a.im b.im, im += a.re b.im + a.im b.re
    // (per lane, in that order)
    static __device__ __forceinline__ void mac(acc &c, val a, val b) {
        p_lacc_fma(c.h, c.l, p_bx(a.h), p_bx(a.l), b.h, b.l);
        p_lacc_fma(c.h, c.l, make_float2(-a.h.y, a.h.y), make_float2(-a.l.y, a.l.y),
                   make_float2(b.h.y, b.h.x), make_float2(b.l.y, b.l.x));
    }
    // acc -= conj(a) b: re -= a.re b.re + a.im b.im, im -= a.re b.im - a.im b.re
    static __device__ __forceinline__ void mac_conj_neg(acc &c, val a, val b) {
        p_lacc_fma(c.h, c.l, p_neg(p_bx(a.h)), p_neg(p_bx(a.l)), b.h, b.l);
        p_lacc_fma(c.h, c.l, make_float2(-a.h.y, a.h.y), make_float2(-a.l.y, a.l.y),
                   make_float2(b.h.y, b.h.x), make_float2(b.l.y, b.l.x));
    }
    // acc += a conj(b): re += a.re b.re + a.im b.im, im += a.im b.re - a.re b.im
    static __device__ __forceinline__ void mac_conjb(acc &c, val a, val b) {
        p_lacc_fma(c.h, c.l, a.h, a.l, p_bx(b.h), p_bx(b.l));
        p_lacc_fma(c.h, c.l, make_float2(a.h.y, -a.h.x), make_float2(a.l.y, -a.l.x), p_by(b.h), p_by(b.l));
    }
    static __device__ __forceinline__ val done(acc c) {
        val v;
        p_two_sum(c.h, c.l, v.h, v.l);
        return v;
    }
    // the accumulator's pairs as they stand (the low parts not renormalised;
    // consumers that multiply keep every cross term, so nothing is lost)
    static __device__ __forceinline__ val raw(acc c) { return {c.h, c.l}; }
    static __device__ __forceinline__ acc acc_minus_i(acc c) {
        return {make_float2(c.h.y, -c.h.x), make_float2(c.l.y, -c.l.x)};
    }
    // a + b of two accumulators: the high parts with TwoSum, every error in
    // the low part (still unnormalised)
    static __device__ __forceinline__ acc acc_add(acc a, acc b) {
        float2 s, t;
        p_two_sum(a.h, b.h, s, t);
        return {s, p_add(t, p_add(a.l, b.l))};
    }
    static __device__ __forceinline__ val sub_conj(val a, val b) {
        val v;
        p_sum(a.h, a.l, make_float2(-b.h.x, b.h.y), make_float2(-b.l.x, b.l.y), v.h, v.l);
        return v;
    }
    static __device__ __forceinline__ val add(val a, val b) {
        val v;
        p_sum(a.h, a.l, b.h, b.l, v.h, v.l);
        return v;
    }
    static __device__ __forceinline__ val add_real(val a, real_t c) {
        const ff r = ff_sum({a.h.x, a.l.x}, c);
        return {make_float2(r.h, a.h.y), make_float2(r.l, a.l.y)};
    }
    static __device__ __forceinline__ val mul_conjb(val a, val b) {
        acc c = acc_zero();
        mac_conjb(c, a, b);
        return done(c);
    }
    static __device__ __forceinline__ val minus_i(val a) {
        return {make_float2(a.h.y, -a.h.x), make_float2(a.l.y, -a.l.x)};
    }
    static __device__ __forceinline__ val conj(val a) {
        return {make_float2(a.h.x, -a.h.y), make_float2(a.l.x, -a.l.y)};
    }
    static __device__ __forceinline__ real_t re(val a) { return {a.h.x, a.l.x}; }
    static __device__ __forceinline__ real_t im(val a) { return {a.h.y, a.l.y}; }
    static __device__ __forceinline__ real_t neg_real(real_t a) { return {-a.h, -a.l}; }
    static __device__ __forceinline__ real_t real_mul(real_t a, real_t b) { return ff_mul(a, b); }
    // acc += c b, c real
    static __device__ __forceinline__ void mac_real(acc &w, real_t c, val b) {
        p_lacc_fma(w.h, w.l, p_b(c.h), p_b(c.l), b.h, b.l);
    }
    static __device__ __forceinline__ val axpy(real_t s, val w, val x) {
        val v;
        p_axpy(p_b(s.h), p_b(s.l), w.h, w.l, x.h, x.l, v.h, v.l);
        return v;
    }
    static __device__ __forceinline__ val lin2(real_t g, val x, real_t b, val w) {
        val v;
        p_lin2(p_b(g.h), p_b(g.l), x.h, x.l, p_b(b.h), p_b(b.l), w.h, w.l, v.h, v.l);
        return v;
    }
    static __device__ __forceinline__ val scale(real_t s, val a) {
        val v;
        p_mulff(p_b(s.h), p_b(s.l), a.h, a.l, v.h, v.l);
        return v;
    }
    static __device__ __forceinline__ double2 to_double2(val v) {
        return make_double2(ff_to_double(re(v)), ff_to_double(im(v)));
    }
    static __device__ __forceinline__ val from_double2(double2 v) {
        const ff r = ff_from_double(v.x), i = ff_from_double(v.y);
        return {make_float2(r.h, i.h), make_float2(r.l, i.l)};
    }
};

}  // namespace grape_num
