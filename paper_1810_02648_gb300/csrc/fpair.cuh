// Compensated FP32 arithmetic: a value carried as the unevaluated sum of two
// FP32 numbers h + l (|l| <= ulp(h)/2 once normalised), about 48 significant
// bits computed on the FP32 pipes.
//
// The graph stage's PCG runs its vectors, its matrix-free J^T J p and its dot
// products in this form.  CG at tens of iterations on the Jacobi-scaled normal
// equations (condition numbers of 1e6 on the body capture) is forward
// unstable: a relative perturbation of 1e-7 per matrix-vector product (one
// FP32 rounding) moves the iterate by percent, while 1e-12 leaves it at the
// FP64 iterate to ~1e-8.  The operator itself (H_i, the rotated offsets, the
// weights) stays FP32: a fixed FP32 matrix is a consistent operator, and CG
// on it follows the FP64 CG on that matrix.  FP64 arithmetic would do the
// same at a far lower rate on this GPU (about 2 FP64 FMAs per clock per SM
// against 128 FP32 FMAs).
//
// The building blocks are the two error-free transformations: Knuth's
// TwoSum (a + b = s + e exactly, six additions) and the FMA form of Dekker's
// TwoProduct (a * b = p + e exactly, one multiplication and one FMA).  Every
// operation below is an explicitly rounded intrinsic, so the compiler can
// neither contract nor reassociate them.
#pragma once

#include <cuda_runtime.h>

namespace lc {

struct fp2 {
    float h, l;
};

__device__ __forceinline__ fp2 fp2_of(float a) { return {a, 0.f}; }
__device__ __forceinline__ double fp2_to_double(fp2 a) { return (double)a.h + (double)a.l; }
__device__ __forceinline__ fp2 fp2_from_double(double d) {
    const float h = __double2float_rn(d);
    return {h, __double2float_rn(d - (double)h)};
}

// s + e = a + b exactly (any magnitudes)
__device__ __forceinline__ fp2 two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}

// s + e = a + b exactly when |a| >= |b| (or a = 0)
__device__ __forceinline__ fp2 quick_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

// p + e = a * b exactly (no underflow)
__device__ __forceinline__ fp2 two_prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    return {p, __fmaf_rn(a, b, -p)};
}

__device__ __forceinline__ fp2 fp2_neg(fp2 a) { return {-a.h, -a.l}; }

// a + b, normalised (relative error ~2^-45 of |a| + |b|)
__device__ __forceinline__ fp2 fp2_add(fp2 a, fp2 b) {
    fp2 s = two_sum(a.h, b.h);
    s.l = __fadd_rn(s.l, __fadd_rn(a.l, b.l));
    return quick_two_sum(s.h, s.l);
}

__device__ __forceinline__ fp2 fp2_sub(fp2 a, fp2 b) { return fp2_add(a, fp2_neg(b)); }

// c * a with an FP32 factor, normalised
__device__ __forceinline__ fp2 fp2_scale(float c, fp2 a) {
    fp2 p = two_prod(c, a.h);
    p.l = __fmaf_rn(c, a.l, p.l);
    return quick_two_sum(p.h, p.l);
}

// a * b, normalised (the l * l term is below the format's precision)
__device__ __forceinline__ fp2 fp2_mul(fp2 a, fp2 b) {
    fp2 p = two_prod(a.h, b.h);
    p.l = __fmaf_rn(a.h, b.l, __fmaf_rn(a.l, b.h, p.l));
    return quick_two_sum(p.h, p.l);
}

// a / b: an FP32 quotient, its remainder a - q b formed exactly enough, and a
// second FP32 quotient of the remainder (long division in two digits)
__device__ __forceinline__ fp2 fp2_div(fp2 a, fp2 b) {
    const float q1 = __fdiv_rn(a.h, b.h);
    const fp2 qb = fp2_scale(q1, b);
    const fp2 rem = fp2_sub(a, qb);
    const float q2 = __fdiv_rn(rem.h, b.h);
    return quick_two_sum(q1, q2);
}

// Running sum of many terms: the high parts through TwoSum, every rounding
// error and low part gathered in one FP32 word (cascaded summation; the error
// is ~n * 2^-48 of the sum of |terms| for n terms).  Normalise with get().
struct fp2acc {
    float h = 0.f, l = 0.f;
    __device__ __forceinline__ void add(fp2 t) {
        const fp2 s = two_sum(h, t.h);
        h = s.h;
        l = __fadd_rn(l, __fadd_rn(s.l, t.l));
    }
    __device__ __forceinline__ void add(float t) {
        const fp2 s = two_sum(h, t);
        h = s.h;
        l = __fadd_rn(l, s.l);
    }
    // += c * a, c FP32, a a pair (the product's rounding error kept)
    __device__ __forceinline__ void mac(float c, fp2 a) {
        fp2 p = two_prod(c, a.h);
        p.l = __fmaf_rn(c, a.l, p.l);
        add(p);
    }
    // += c * a, both FP32 (exact product)
    __device__ __forceinline__ void mac(float c, float a) { add(two_prod(c, a)); }
    // += a * b, both pairs
    __device__ __forceinline__ void mac(fp2 a, fp2 b) {
        fp2 p = two_prod(a.h, b.h);
        p.l = __fmaf_rn(a.h, b.l, __fmaf_rn(a.l, b.h, p.l));
        add(p);
    }
    __device__ __forceinline__ void add(const fp2acc& o) { add(fp2{o.h, o.l}); }
    __device__ __forceinline__ fp2 get() const { return quick_two_sum(h, l); }
};

// 3-vectors of pairs
struct fp2v3 {
    fp2 x, y, z;
};

// c x a with c FP32 and a pairs
__device__ __forceinline__ fp2v3 fp2_cross(float3 c, const fp2v3& a) {
    fp2acc x, y, z;
    x.mac(c.y, a.z); x.mac(-c.z, a.y);
    y.mac(c.z, a.x); y.mac(-c.x, a.z);
    z.mac(c.x, a.y); z.mac(-c.y, a.x);
    return {x.get(), y.get(), z.get()};
}

// Warp-wide sum of a pair (fixed xor-shuffle tree; every lane gets the total)
__device__ __forceinline__ fp2 fp2_warp_sum(fp2 v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        fp2 w;
        w.h = __shfl_xor_sync(0xffffffffu, v.h, o);
        w.l = __shfl_xor_sync(0xffffffffu, v.l, o);
        v = fp2_add(v, w);
    }
    return v;
}

// Block-wide sum of one pair per thread (NWARPS warps, sh holds NWARPS
// entries); the total is valid in warp 0.
template <int NWARPS>
__device__ __forceinline__ fp2 block_sum_fp2(fp2 v, float2* sh) {
    v = fp2_warp_sum(v);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) sh[w] = make_float2(v.h, v.l);
    __syncthreads();
    fp2 t = {0.f, 0.f};
    if (w == 0) {
        const float2 a = l < NWARPS ? sh[l] : make_float2(0.f, 0.f);
        t = fp2_warp_sum(fp2{a.x, a.y});
    }
    return t;
}

}  // namespace lc
