// arith.cuh -- per-precision loads, stores and SU(3) x colour-vector arithmetic.
//
// Every precision exposes the same three things to the Dslash kernel:
//   Link   : one 3x3 complex link in compute registers (rebuilt from 12 reals if needed)
//   Vec    : one colour 3-vector in compute registers
//   Acc    : an accumulating colour 3-vector
// and  hop<DAG, SUB>(acc, U, v):  acc (+|-)= U v   (DAG: U^+ v).
//
// HISQ_F64X stores every real as an unevaluated float pair (hi + lo) and accumulates with
// error-free transformations on the FP32 pipes (the FP64 unit of this GPU runs at about
// 1/60 of the FP32 rate): each product a*b of pairs is split exactly with TwoProd (FMA),
// each running sum is updated with Knuth's TwoSum, and the rounding errors are collected
// in a second float per component (a compensated dot product in the sense of Ogita, Rump
// and Oishi, "Accurate sum and dot product", SISC 2005).  Intrinsics with explicit
// rounding keep the compiler from contracting the transformations into FMAs.
#pragma once

#include <type_traits>

#include "internal.cuh"

namespace hisq {

// ---------------------------------------------------------------- raw loads
__device__ __forceinline__ uint4 ld_nc16(const void *p)
{
    uint4 r;
    asm("ld.global.nc.L1::no_allocate.v4.u32 {%0,%1,%2,%3}, [%4];"
        : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
        : "l"(p));
    return r;
}
__device__ __forceinline__ uint2 ld_nc8(const void *p)
{
    uint2 r;
    asm("ld.global.nc.L1::no_allocate.v2.u32 {%0,%1}, [%2];" : "=r"(r.x), "=r"(r.y) : "l"(p));
    return r;
}
__device__ __forceinline__ uint32_t ld_nc4(const void *p)
{
    uint32_t r;
    asm("ld.global.nc.L1::no_allocate.u32 %0, [%1];" : "=r"(r) : "l"(p));
    return r;
}

// the same loads with an L2 eviction-priority policy (createpolicy): data read once per
// application that should not push reused lines out of L2
__device__ __forceinline__ uint64_t l2_evict_first_policy()
{
    uint64_t pol;
    asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}
__device__ __forceinline__ uint4 ld_nc16(const void *p, uint64_t pol)
{
    uint4 r;
    asm("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.u32 {%0,%1,%2,%3}, [%4], %5;"
        : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
        : "l"(p), "l"(pol));
    return r;
}
__device__ __forceinline__ uint2 ld_nc8(const void *p, uint64_t pol)
{
    uint2 r;
    asm("ld.global.nc.L1::no_allocate.L2::cache_hint.v2.u32 {%0,%1}, [%2], %3;" : "=r"(r.x), "=r"(r.y) : "l"(p), "l"(pol));
    return r;
}
__device__ __forceinline__ uint32_t ld_nc4(const void *p, uint64_t pol)
{
    uint32_t r;
    asm("ld.global.nc.L1::no_allocate.L2::cache_hint.u32 %0, [%1], %2;" : "=r"(r) : "l"(p), "l"(pol));
    return r;
}

// the same loads kept in L1 (read-only path, L1 allocation): links that other warps of the
// same block read again right afterwards (right-hand-side groups sharing a block's sites)
__device__ __forceinline__ uint4 ld_l1_16(const void *p, uint64_t pol, bool hint)
{
    uint4 r;
    if (hint)
        asm("ld.global.nc.L2::cache_hint.v4.u32 {%0,%1,%2,%3}, [%4], %5;"
            : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
            : "l"(p), "l"(pol));
    else
        asm("ld.global.nc.v4.u32 {%0,%1,%2,%3}, [%4];" : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w) : "l"(p));
    return r;
}
__device__ __forceinline__ uint2 ld_l1_8(const void *p, uint64_t pol, bool hint)
{
    uint2 r;
    if (hint) asm("ld.global.nc.L2::cache_hint.v2.u32 {%0,%1}, [%2], %3;" : "=r"(r.x), "=r"(r.y) : "l"(p), "l"(pol));
    else asm("ld.global.nc.v2.u32 {%0,%1}, [%2];" : "=r"(r.x), "=r"(r.y) : "l"(p));
    return r;
}
__device__ __forceinline__ uint32_t ld_l1_4(const void *p, uint64_t pol, bool hint)
{
    uint32_t r;
    if (hint) asm("ld.global.nc.L2::cache_hint.u32 %0, [%1], %2;" : "=r"(r) : "l"(p), "l"(pol));
    else asm("ld.global.nc.u32 %0, [%1];" : "=r"(r) : "l"(p));
    return r;
}

// link words of site s in a slot; LB = link bytes.  With `hint`, the loads are marked
// evict-first in L2; with L1, they allocate in L1 (read again by other warps of the block).
template <int LB, bool L1 = false>
__device__ __forceinline__ void load_link_words(const char *slot, uint32_t s, uint32_t (&w)[LB / 4], bool hint = false)
{
    constexpr int NQ = LB / 16, TB = LB % 16;
    const uint64_t pol = hint ? l2_evict_first_policy() : 0ull;
    const char *blk = slot + (size_t)(s >> 5) * (32 * LB);
    const uint32_t lane = s & 31;
#pragma unroll
    for (int q = 0; q < NQ; q++) {
        const char *a = blk + q * 512 + lane * 16;
        uint4 v = L1 ? ld_l1_16(a, pol, hint) : hint ? ld_nc16(a, pol) : ld_nc16(a);
        w[4 * q + 0] = v.x;
        w[4 * q + 1] = v.y;
        w[4 * q + 2] = v.z;
        w[4 * q + 3] = v.w;
    }
    if constexpr (TB == 8) {
        const char *a = blk + NQ * 512 + lane * 8;
        uint2 v = L1 ? ld_l1_8(a, pol, hint) : hint ? ld_nc8(a, pol) : ld_nc8(a);
        w[4 * NQ + 0] = v.x;
        w[4 * NQ + 1] = v.y;
    } else if constexpr (TB == 4) {
        const char *a = blk + NQ * 512 + lane * 4;
        w[4 * NQ] = L1 ? ld_l1_4(a, pol, hint) : hint ? ld_nc4(a, pol) : ld_nc4(a);
    }
}

// ---------------------------------------------------------------- float-float helpers
struct DD {
    float h, l;
};
// running compensated sum: value = h + e (e collects rounding errors)
struct DAcc {
    float h, e;
};

__device__ __forceinline__ void dd_mac(DAcc &a, float xh, float xl, float yh, float yl)
{
    const float p = __fmul_rn(xh, yh);
    float pe = __fmaf_rn(xh, yh, -p);      // exact: xh*yh = p + pe
    pe = __fmaf_rn(xh, yl, pe);
    pe = __fmaf_rn(xl, yh, pe);
    const float s = __fadd_rn(a.h, p);     // TwoSum(a.h, p)
    const float z = __fsub_rn(s, a.h);
    const float t = __fadd_rn(__fsub_rn(a.h, __fsub_rn(s, z)), __fsub_rn(p, z));
    a.h = s;
    a.e = __fadd_rn(a.e, __fadd_rn(t, pe));
}

// normalised pair of a compensated sum (Fast2Sum, |h| >= |e|)
__device__ __forceinline__ DD dd_norm(DAcc a)
{
    const float hi = __fadd_rn(a.h, a.e);
    const float lo = __fsub_rn(a.e, __fsub_rn(hi, a.h));
    return {hi, lo};
}

// fold the error term back into the running sum (keeps |e| <= ulp(h) / 2)
__device__ __forceinline__ void dd_renorm(DAcc &a)
{
    const DD d = dd_norm(a);
    a.h = d.h;
    a.e = d.l;
}

// a += b for two compensated sums (TwoSum of the leading parts, then renormalise)
__device__ __forceinline__ void dd_add(DAcc &a, const DAcc &b)
{
    const float s = __fadd_rn(a.h, b.h);
    const float z = __fsub_rn(s, a.h);
    float t = __fadd_rn(__fsub_rn(a.h, __fsub_rn(s, z)), __fsub_rn(b.h, z));
    t = __fadd_rn(t, __fadd_rn(a.e, b.e));
    const float hi = __fadd_rn(s, t);
    a.h = hi;
    a.e = __fsub_rn(t, __fsub_rn(hi, s));
}

// ---------------------------------------------------------------- precision traits
template <int P> struct Prec;

// IEEE double, DFMA arithmetic
template <> struct Prec<HISQ_F64> {
    using Real = double;
    struct Link { double v[18]; };
    struct Vec { double v[6]; };
    struct Acc { double v[6]; };
    static constexpr int SB = 48;
    template <int NREAL>
    __device__ static void unpack(const uint32_t *w, Link &U)
    {
#pragma unroll
        for (int i = 0; i < NREAL; i++) U.v[i] = __hiloint2double(w[2 * i + 1], w[2 * i]);
    }
    __device__ static void zero(Acc &a)
    {
#pragma unroll
        for (int i = 0; i < 6; i++) a.v[i] = 0.0;
    }
    __device__ static void load(const void *base, uint32_t s, Vec &v)
    {
        const double2 *p = reinterpret_cast<const double2 *>(static_cast<const char *>(base) + (size_t)s * SB);
#pragma unroll
        for (int i = 0; i < 3; i++) {
            double2 d = __ldg(p + i);
            v.v[2 * i] = d.x;
            v.v[2 * i + 1] = d.y;
        }
    }
    __device__ static void store(void *base, uint32_t s, const Acc &a)
    {
        double2 *p = reinterpret_cast<double2 *>(static_cast<char *>(base) + (size_t)s * SB);
#pragma unroll
        for (int i = 0; i < 3; i++) p[i] = make_double2(a.v[2 * i], a.v[2 * i + 1]);
    }
    // components as doubles (for epilogues / reductions)
    __device__ static double comp(const Acc &a, int i) { return a.v[i]; }
    __device__ static double vcomp(const Vec &v, int i) { return v.v[i]; }
    __device__ static void set_acc(Acc &a, int i, double x) { a.v[i] = x; }
    __device__ static void negate(Vec &v)
    {
#pragma unroll
        for (int i = 0; i < 6; i++) v.v[i] = -v.v[i];
    }
    template <bool DAG, bool SUB>
    __device__ static void hop(Acc &a, const Link &U, const Vec &v)
    {
#pragma unroll
        for (int i = 0; i < 3; i++)
#pragma unroll
            for (int j = 0; j < 3; j++) {
                double ur = DAG ? U.v[2 * (3 * j + i)] : U.v[2 * (3 * i + j)];
                double ui = DAG ? -U.v[2 * (3 * j + i) + 1] : U.v[2 * (3 * i + j) + 1];
                if (SUB) { ur = -ur; ui = -ui; }
                a.v[2 * i] = fma(ur, v.v[2 * j], a.v[2 * i]);
                a.v[2 * i] = fma(-ui, v.v[2 * j + 1], a.v[2 * i]);
                a.v[2 * i + 1] = fma(ur, v.v[2 * j + 1], a.v[2 * i + 1]);
                a.v[2 * i + 1] = fma(ui, v.v[2 * j], a.v[2 * i + 1]);
            }
    }
    // third row of an SU(3) matrix from the first two: conj(row0 x row1), times sign
    __device__ static void rebuild(Link &U, bool neg)
    {
        const double s = neg ? -1.0 : 1.0;
#pragma unroll
        for (int k = 0; k < 3; k++) {
            const int a = (k + 1) % 3, b = (k + 2) % 3;
            // c = r0_a r1_b - r0_b r1_a
            double cr = U.v[2 * a] * U.v[6 + 2 * b] - U.v[2 * a + 1] * U.v[6 + 2 * b + 1];
            double ci = U.v[2 * a] * U.v[6 + 2 * b + 1] + U.v[2 * a + 1] * U.v[6 + 2 * b];
            cr -= U.v[2 * b] * U.v[6 + 2 * a] - U.v[2 * b + 1] * U.v[6 + 2 * a + 1];
            ci -= U.v[2 * b] * U.v[6 + 2 * a + 1] + U.v[2 * b + 1] * U.v[6 + 2 * a];
            U.v[12 + 2 * k] = s * cr;
            U.v[12 + 2 * k + 1] = -s * ci;
        }
    }
    __device__ static void axpy_acc(Acc &out, double a, const Acc &x)
    {
#pragma unroll
        for (int i = 0; i < 6; i++) out.v[i] = fma(a, x.v[i], out.v[i]);
    }
    // o = m4 p - o
    __device__ static void mdagm_epilogue(Acc &o, double m4, const Vec &p)
    {
#pragma unroll
        for (int i = 0; i < 6; i++) o.v[i] = fma(m4, p.v[i], -o.v[i]);
    }
    static constexpr bool kSplitDirections = false;
    __device__ static void add_acc(Acc &, const Acc &) {}
    // a += the same accumulator of lane (lane ^ off)
    __device__ static void shfl_xor_add(Acc &a, int off)
    {
#pragma unroll
        for (int i = 0; i < 6; i++) a.v[i] += __shfl_xor_sync(0xffffffffu, a.v[i], off);
    }
    // Re <p, o>
    __device__ static double dot(const Vec &p, const Acc &o)
    {
        double d = 0.0;
#pragma unroll
        for (int i = 0; i < 6; i++) d = fma(p.v[i], o.v[i], d);
        return d;
    }
};

// float storage (F32) and the float-arithmetic base shared by F16 / BF16
struct FloatArith {
    using Real = float;
    struct Link { float v[18]; };
    struct Vec { float v[6]; };
    struct Acc { float v[6]; };
    __device__ static void zero(Acc &a)
    {
#pragma unroll
        for (int i = 0; i < 6; i++) a.v[i] = 0.f;
    }
    __device__ static double comp(const Acc &a, int i) { return (double)a.v[i]; }
    __device__ static double vcomp(const Vec &v, int i) { return (double)v.v[i]; }
    __device__ static void set_acc(Acc &a, int i, double x) { a.v[i] = (float)x; }
    __device__ static void negate(Vec &v)
    {
#pragma unroll
        for (int i = 0; i < 6; i++) v.v[i] = -v.v[i];
    }
    template <bool DAG, bool SUB>
    __device__ static void hop(Acc &a, const Link &U, const Vec &v)
    {
#pragma unroll
        for (int i = 0; i < 3; i++)
#pragma unroll
            for (int j = 0; j < 3; j++) {
                float ur = DAG ? U.v[2 * (3 * j + i)] : U.v[2 * (3 * i + j)];
                float ui = DAG ? -U.v[2 * (3 * j + i) + 1] : U.v[2 * (3 * i + j) + 1];
                if (SUB) { ur = -ur; ui = -ui; }
                a.v[2 * i] = fmaf(ur, v.v[2 * j], a.v[2 * i]);
                a.v[2 * i] = fmaf(-ui, v.v[2 * j + 1], a.v[2 * i]);
                a.v[2 * i + 1] = fmaf(ur, v.v[2 * j + 1], a.v[2 * i + 1]);
                a.v[2 * i + 1] = fmaf(ui, v.v[2 * j], a.v[2 * i + 1]);
            }
    }
    __device__ static void rebuild(Link &U, bool neg)
    {
        const float s = neg ? -1.f : 1.f;
#pragma unroll
        for (int k = 0; k < 3; k++) {
            const int a = (k + 1) % 3, b = (k + 2) % 3;
            float cr = U.v[2 * a] * U.v[6 + 2 * b] - U.v[2 * a + 1] * U.v[6 + 2 * b + 1];
            float ci = U.v[2 * a] * U.v[6 + 2 * b + 1] + U.v[2 * a + 1] * U.v[6 + 2 * b];
            cr -= U.v[2 * b] * U.v[6 + 2 * a] - U.v[2 * b + 1] * U.v[6 + 2 * a + 1];
            ci -= U.v[2 * b] * U.v[6 + 2 * a + 1] + U.v[2 * b + 1] * U.v[6 + 2 * a];
            U.v[12 + 2 * k] = s * cr;
            U.v[12 + 2 * k + 1] = -s * ci;
        }
    }
    __device__ static void axpy_acc(Acc &out, float a, const Acc &x)
    {
#pragma unroll
        for (int i = 0; i < 6; i++) out.v[i] = fmaf(a, x.v[i], out.v[i]);
    }
    static constexpr bool kSplitDirections = false;
    __device__ static void add_acc(Acc &, const Acc &) {}
    // a += the same accumulator of lane (lane ^ off)
    __device__ static void shfl_xor_add(Acc &a, int off)
    {
#pragma unroll
        for (int i = 0; i < 6; i++) a.v[i] += __shfl_xor_sync(0xffffffffu, a.v[i], off);
    }
    __device__ static void mdagm_epilogue(Acc &o, float m, const Vec &p)
    {
#pragma unroll
        for (int i = 0; i < 6; i++) o.v[i] = fmaf(m, p.v[i], -o.v[i]);
    }
    __device__ static void mdagm_epilogue(Acc &o, double m4, const Vec &p) { mdagm_epilogue(o, (float)m4, p); }
    __device__ static float dotf(const Vec &p, const Acc &o)
    {
        float d = 0.f;
#pragma unroll
        for (int i = 0; i < 6; i++) d = fmaf(p.v[i], o.v[i], d);
        return d;
    }
    __device__ static double dot(const Vec &p, const Acc &o) { return (double)dotf(p, o); }
};

template <> struct Prec<HISQ_F32> : FloatArith {
    static constexpr int SB = 24;
    template <int NREAL>
    __device__ static void unpack(const uint32_t *w, Link &U)
    {
#pragma unroll
        for (int i = 0; i < NREAL; i++) U.v[i] = __uint_as_float(w[i]);
    }
    __device__ static void load(const void *base, uint32_t s, Vec &v)
    {
        const float2 *p = reinterpret_cast<const float2 *>(static_cast<const char *>(base) + (size_t)s * SB);
#pragma unroll
        for (int i = 0; i < 3; i++) {
            float2 d = __ldg(p + i);
            v.v[2 * i] = d.x;
            v.v[2 * i + 1] = d.y;
        }
    }
    __device__ static void store(void *base, uint32_t s, const Acc &a)
    {
        float2 *p = reinterpret_cast<float2 *>(static_cast<char *>(base) + (size_t)s * SB);
#pragma unroll
        for (int i = 0; i < 3; i++) p[i] = make_float2(a.v[2 * i], a.v[2 * i + 1]);
    }
    // ordinary (coherent) loads, for vectors that other blocks of the same launch write
    // between grid barriers: the read-only path of load() may serve such data stale
    __device__ static void load_coh(const void *base, uint32_t s, Vec &v)
    {
        const float2 *p = reinterpret_cast<const float2 *>(static_cast<const char *>(base) + (size_t)s * SB);
#pragma unroll
        for (int i = 0; i < 3; i++) {
            const float2 d = p[i];
            v.v[2 * i] = d.x;
            v.v[2 * i + 1] = d.y;
        }
    }
};

// 16-bit storage; spinor record = 3 x (2 x 16-bit) + float scale
template <class H2> struct Half16 : FloatArith {
    static constexpr int SB = 16;
    __device__ static float2 to2(uint32_t w)
    {
        H2 h = *reinterpret_cast<const H2 *>(&w);
        if constexpr (std::is_same<H2, __half2>::value) return __half22float2(h);
        else return __bfloat1622float2(h);
    }
    __device__ static uint32_t from2(float a, float b)
    {
        H2 h;
        if constexpr (std::is_same<H2, __half2>::value) h = __floats2half2_rn(a, b);
        else h = __floats2bfloat162_rn(a, b);
        return *reinterpret_cast<uint32_t *>(&h);
    }
    template <int NREAL>
    __device__ static void unpack(const uint32_t *w, Link &U)
    {
#pragma unroll
        for (int i = 0; i < NREAL / 2; i++) {
            float2 f = to2(w[i]);
            U.v[2 * i] = f.x;
            U.v[2 * i + 1] = f.y;
        }
    }
    __device__ static void load(const void *base, uint32_t s, Vec &v)
    {
        const uint4 d = __ldg(reinterpret_cast<const uint4 *>(static_cast<const char *>(base) + (size_t)s * SB));
        const float sc = __uint_as_float(d.w);
        float2 a = to2(d.x), b = to2(d.y), c = to2(d.z);
        v.v[0] = a.x * sc; v.v[1] = a.y * sc;
        v.v[2] = b.x * sc; v.v[3] = b.y * sc;
        v.v[4] = c.x * sc; v.v[5] = c.y * sc;
    }
    __device__ static void store(void *base, uint32_t s, const Acc &a)
    {
        float m = 0.f;
#pragma unroll
        for (int i = 0; i < 6; i++) m = fmaxf(m, fabsf(a.v[i]));
        const float inv = m > 0.f ? 1.f / m : 0.f;
        uint4 d;
        d.x = from2(a.v[0] * inv, a.v[1] * inv);
        d.y = from2(a.v[2] * inv, a.v[3] * inv);
        d.z = from2(a.v[4] * inv, a.v[5] * inv);
        d.w = __float_as_uint(m);
        *reinterpret_cast<uint4 *>(static_cast<char *>(base) + (size_t)s * SB) = d;
    }
};
template <> struct Prec<HISQ_F16> : Half16<__half2> {};
template <> struct Prec<HISQ_BF16> : Half16<__nv_bfloat162> {};

// float pairs, compensated arithmetic (18-real links only)
template <> struct Prec<HISQ_F64X> {
    using Real = double;
    struct Link { float h[18], l[18]; };
    struct Vec { float h[6], l[6]; };
    struct Acc { DAcc v[6]; };
    static constexpr int SB = 48;
    template <int NREAL>
    __device__ static void unpack(const uint32_t *w, Link &U)
    {
#pragma unroll
        for (int i = 0; i < NREAL; i++) {
            U.h[i] = __uint_as_float(w[i]);
            U.l[i] = __uint_as_float(w[NREAL + i]);
        }
    }
    __device__ static void zero(Acc &a)
    {
#pragma unroll
        for (int i = 0; i < 6; i++) a.v[i] = {0.f, 0.f};
    }
    __device__ static void load(const void *base, uint32_t s, Vec &v)
    {
        const float4 *p = reinterpret_cast<const float4 *>(static_cast<const char *>(base) + (size_t)s * SB);
        float4 a = __ldg(p), b = __ldg(p + 1), c = __ldg(p + 2);
        v.h[0] = a.x; v.h[1] = a.y; v.h[2] = a.z; v.h[3] = a.w; v.h[4] = b.x; v.h[5] = b.y;
        v.l[0] = b.z; v.l[1] = b.w; v.l[2] = c.x; v.l[3] = c.y; v.l[4] = c.z; v.l[5] = c.w;
    }
    __device__ static void store(void *base, uint32_t s, const Acc &a)
    {
        DD d[6];
#pragma unroll
        for (int i = 0; i < 6; i++) d[i] = dd_norm(a.v[i]);
        float4 *p = reinterpret_cast<float4 *>(static_cast<char *>(base) + (size_t)s * SB);
        p[0] = make_float4(d[0].h, d[1].h, d[2].h, d[3].h);
        p[1] = make_float4(d[4].h, d[5].h, d[0].l, d[1].l);
        p[2] = make_float4(d[2].l, d[3].l, d[4].l, d[5].l);
    }
    __device__ static double comp(const Acc &a, int i) { return (double)a.v[i].h + (double)a.v[i].e; }
    __device__ static double vcomp(const Vec &v, int i) { return (double)v.h[i] + (double)v.l[i]; }
    __device__ static void set_acc(Acc &a, int i, double x)
    {
        const float h = (float)x;
        a.v[i] = {h, (float)(x - (double)h)};
    }
    __device__ static void negate(Vec &v)
    {
#pragma unroll
        for (int i = 0; i < 6; i++) { v.h[i] = -v.h[i]; v.l[i] = -v.l[i]; }
    }
    template <bool DAG, bool SUB>
    __device__ static void hop(Acc &a, const Link &U, const Vec &v)
    {
#pragma unroll
        for (int i = 0; i < 3; i++)
#pragma unroll
            for (int j = 0; j < 3; j++) {
                const int e = DAG ? 3 * j + i : 3 * i + j;
                float urh = U.h[2 * e], url = U.l[2 * e];
                float uih = U.h[2 * e + 1], uil = U.l[2 * e + 1];
                if (DAG) { uih = -uih; uil = -uil; }
                if (SUB) { urh = -urh; url = -url; uih = -uih; uil = -uil; }
                // re += ur vr - ui vi ; im += ur vi + ui vr
                dd_mac(a.v[2 * i], urh, url, v.h[2 * j], v.l[2 * j]);
                dd_mac(a.v[2 * i], -uih, -uil, v.h[2 * j + 1], v.l[2 * j + 1]);
                dd_mac(a.v[2 * i + 1], urh, url, v.h[2 * j + 1], v.l[2 * j + 1]);
                dd_mac(a.v[2 * i + 1], uih, uil, v.h[2 * j], v.l[2 * j]);
            }
        // one renormalisation per hop (every six products of a component)
#pragma unroll
        for (int c = 0; c < 6; c++) dd_renorm(a.v[c]);
    }
    // directions are summed separately (24 products each) and combined pairwise: the
    // rounding error of a compensated sum grows with the number of terms it absorbs
    static constexpr bool kSplitDirections = true;
    __device__ static void add_acc(Acc &a, const Acc &b)
    {
#pragma unroll
        for (int c = 0; c < 6; c++) dd_add(a.v[c], b.v[c]);
    }
    __device__ static void shfl_xor_add(Acc &a, int off)
    {
#pragma unroll
        for (int c = 0; c < 6; c++) {
            const DAcc b = {__shfl_xor_sync(0xffffffffu, a.v[c].h, off), __shfl_xor_sync(0xffffffffu, a.v[c].e, off)};
            dd_add(a.v[c], b);
        }
    }
    __device__ static void rebuild(Link &, bool) {}
    __device__ static void axpy_acc(Acc &, double, const Acc &) {}
    __device__ static void mdagm_epilogue(Acc &o, double m4, const Vec &p)
    {
        const float mh = (float)m4, ml = (float)(m4 - (double)mh);
#pragma unroll
        for (int i = 0; i < 6; i++) {
            o.v[i].h = -o.v[i].h;
            o.v[i].e = -o.v[i].e;
            dd_mac(o.v[i], mh, ml, p.h[i], p.l[i]);
        }
    }
    __device__ static double dot(const Vec &p, const Acc &o)
    {
        DAcc d = {0.f, 0.f};
#pragma unroll
        for (int i = 0; i < 6; i++) {
            const DD x = dd_norm(o.v[i]);
            dd_mac(d, p.h[i], p.l[i], x.h, x.l);
        }
        return (double)d.h + (double)d.e;
    }
};

}  // namespace hisq
