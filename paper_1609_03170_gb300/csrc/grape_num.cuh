// grape_num.cuh - the two complex number types the kernels are written over.
//
//  NumD   native FP64 complex (double2 storage).
//  NumF   double-float complex: every real part is an unevaluated sum hi + lo
//         of two FP32 numbers with |lo| <= ulp(hi)/2, about 48 significant
//         bits (float4 storage: re.hi, re.lo, im.hi, im.lo).  Arithmetic
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

struct NumF {
    using store_t = float4;   // re.h, re.l, im.h, im.l
    using real_t = ff;
    struct val { ff re, im; };
    struct acc { lacc re, im; };

    static __device__ __forceinline__ val load(const store_t &s) { return {{s.x, s.y}, {s.z, s.w}}; }
    // the real part alone (8-byte load of re.h, re.l)
    static __device__ __forceinline__ real_t load_re(const store_t &s) {
        const float2 v = *reinterpret_cast<const float2 *>(&s);
        return {v.x, v.y};
    }
    static __device__ __forceinline__ store_t store(val v) {
        return make_float4(v.re.h, v.re.l, v.im.h, v.im.l);
    }
    static __device__ __forceinline__ val zero() { return {{0.f, 0.f}, {0.f, 0.f}}; }
    static __device__ __forceinline__ acc acc_zero() { return {{0.f, 0.f}, {0.f, 0.f}}; }
    static __device__ __forceinline__ real_t real_const(double x) { return ff_from_double(x); }
    static __device__ __forceinline__ void mac(acc &c, val a, val b) {
        lacc_fma(c.re, a.re.h, a.re.l, b.re.h, b.re.l);
        lacc_fms(c.re, a.im.h, a.im.l, b.im.h, b.im.l);
        lacc_fma(c.im, a.re.h, a.re.l, b.im.h, b.im.l);
        lacc_fma(c.im, a.im.h, a.im.l, b.re.h, b.re.l);
    }
    static __device__ __forceinline__ void mac_conj_neg(acc &c, val a, val b) {
        // -(a.re - i a.im)(b.re + i b.im) = -(a.re b.re + a.im b.im) - i(a.re b.im - a.im b.re)
        lacc_fms(c.re, a.re.h, a.re.l, b.re.h, b.re.l);
        lacc_fms(c.re, a.im.h, a.im.l, b.im.h, b.im.l);
        lacc_fms(c.im, a.re.h, a.re.l, b.im.h, b.im.l);
        lacc_fma(c.im, a.im.h, a.im.l, b.re.h, b.re.l);
    }
    static __device__ __forceinline__ void mac_conjb(acc &c, val a, val b) {
        // a conj(b) = (a.re b.re + a.im b.im) + i(a.im b.re - a.re b.im)
        lacc_fma(c.re, a.re.h, a.re.l, b.re.h, b.re.l);
        lacc_fma(c.re, a.im.h, a.im.l, b.im.h, b.im.l);
        lacc_fma(c.im, a.im.h, a.im.l, b.re.h, b.re.l);
        lacc_fms(c.im, a.re.h, a.re.l, b.im.h, b.im.l);
    }
    static __device__ __forceinline__ val done(acc c) { return {lacc_done(c.re), lacc_done(c.im)}; }
    // the accumulator's pairs as they stand (the low parts not renormalised;
    // consumers that multiply keep every cross term, so nothing is lost)
    static __device__ __forceinline__ val raw(acc c) { return {{c.re.h, c.re.l}, {c.im.h, c.im.l}}; }
    static __device__ __forceinline__ acc acc_minus_i(acc c) { return {c.im, {-c.re.h, -c.re.l}}; }
    // a + b of two accumulators: the high parts with TwoSum, every error in
    // the low part (still unnormalised)
    static __device__ __forceinline__ acc acc_add(acc a, acc b) {
        const ff r = two_sum(a.re.h, b.re.h), i = two_sum(a.im.h, b.im.h);
        return {{r.h, __fadd_rn(r.l, __fadd_rn(a.re.l, b.re.l))}, {i.h, __fadd_rn(i.l, __fadd_rn(a.im.l, b.im.l))}};
    }
    static __device__ __forceinline__ val sub_conj(val a, val b) {
        return {ff_sum(a.re, {-b.re.h, -b.re.l}), ff_sum(a.im, b.im)};
    }
    static __device__ __forceinline__ val add(val a, val b) { return {ff_sum(a.re, b.re), ff_sum(a.im, b.im)}; }
    static __device__ __forceinline__ val add_real(val a, real_t c) { return {ff_sum(a.re, c), a.im}; }
    static __device__ __forceinline__ val mul_conjb(val a, val b) {
        acc c = acc_zero();
        mac_conjb(c, a, b);
        return done(c);
    }
    static __device__ __forceinline__ val minus_i(val a) {
        return {a.im, {-a.re.h, -a.re.l}};
    }
    static __device__ __forceinline__ real_t re(val a) { return a.re; }
    static __device__ __forceinline__ real_t neg_real(real_t a) { return {-a.h, -a.l}; }
    static __device__ __forceinline__ real_t real_mul(real_t a, real_t b) { return ff_mul(a, b); }
    static __device__ __forceinline__ void mac_real(acc &w, real_t c, val b) {
        lacc_fma(w.re, c.h, c.l, b.re.h, b.re.l);
        lacc_fma(w.im, c.h, c.l, b.im.h, b.im.l);
    }
    static __device__ __forceinline__ val axpy(real_t s, val w, val x) {
        return {ff_axpy(s, w.re, x.re), ff_axpy(s, w.im, x.im)};
    }
    static __device__ __forceinline__ val lin2(real_t g, val x, real_t b, val w) {
        return {ff_lin2(g, x.re, b, w.re), ff_lin2(g, x.im, b, w.im)};
    }
    static __device__ __forceinline__ val scale(real_t s, val a) {
        return {ff_mul(s, a.re), ff_mul(s, a.im)};
    }
    static __device__ __forceinline__ double2 to_double2(val v) {
        return make_double2(ff_to_double(v.re), ff_to_double(v.im));
    }
    static __device__ __forceinline__ val from_double2(double2 v) {
        return {ff_from_double(v.x), ff_from_double(v.y)};
    }
};

}  // namespace grape_num
