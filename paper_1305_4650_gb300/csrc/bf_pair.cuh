// Phase factors of the mixed precision, two at a time.
//
// sm_100 and later issue FP32 add, multiply and fused multiply-add on a pair of
// registers as one instruction (add/sub/mul/fma .f32x2).  The double-float
// evaluation of Phi and the sincos polynomial are long chains of such operations,
// so two independent phases (two lanes of a float2) take about the issue slots of
// one.  Every lane performs the operations of the scalar code in bf_device.cuh; where
// a caller sums the per-coordinate parts in another order than the scalar code, the
// two agree to FP32 rounding.
// Included by bf_device.cuh after the scalar phase code it builds on.
#pragma once

namespace bfk {

__device__ __forceinline__ float2 dup2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b)
{
    float2 r;
    asm("{ .reg .b64 u, v, d; mov.b64 u, {%2, %3}; mov.b64 v, {%4, %5}; sub.rn.f32x2 d, u, v; mov.b64 {%0, %1}, d; }"
        : "=f"(r.x), "=f"(r.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return r;
}
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }

struct df2 {
    float2 hi, lo;
};

__device__ __forceinline__ df2 two_sum2(float2 a, float2 b)
{
    const float2 s = add2(a, b);
    const float2 bb = sub2(s, a);
    return {s, add2(sub2(a, sub2(s, bb)), sub2(b, bb))};
}

__device__ __forceinline__ df2 fast_two_sum2(float2 a, float2 b)
{
    const float2 s = add2(a, b);
    return {s, sub2(b, sub2(s, a))};
}

__device__ __forceinline__ df2 df_mul_u2(const df2 &x, const df2 &y)
{
    const float2 p = mul2(x.hi, y.hi);
    float2 e = fma2(x.hi, y.hi, neg2(p));
    e = fma2(x.hi, y.lo, e);
    e = fma2(x.lo, y.hi, e);
    return {p, e};
}

__device__ __forceinline__ df2 df_mul2(const df2 &x, const df2 &y)
{
    const df2 u = df_mul_u2(x, y);
    return fast_two_sum2(u.hi, u.lo);
}

__device__ __forceinline__ df2 df_add2(const df2 &x, const df2 &y)
{
    const df2 s = two_sum2(x.hi, y.hi);
    return fast_two_sum2(s.hi, add2(s.lo, add2(x.lo, y.lo)));
}

__device__ __forceinline__ float2 fround2(float2 x)
{
    const float2 M = dup2(12582912.0f);
    return sub2(add2(x, M), M);
}

__device__ __forceinline__ df2 df_sqrt_u2(const df2 &x)
{
    const float2 r = make_float2(rsqrtf(fmaxf(x.hi.x, 1e-30f)), rsqrtf(fmaxf(x.hi.y, 1e-30f)));
    const float2 s = mul2(x.hi, r);
    const float2 res = add2(fma2(neg2(s), s, x.hi), x.lo);
    return {s, mul2(res, mul2(dup2(0.5f), r))};
}

__device__ __forceinline__ float2 df_frac2(const df2 &x) { return add2(sub2(x.hi, fround2(x.hi)), x.lo); }

__device__ __forceinline__ float2 df_mul_frac2(const df2 &x, const df2 &y)
{
    const float2 M = dup2(12582912.0f);
    const float2 n = sub2(fma2(x.hi, y.hi, M), M);
    const float2 f = fma2(x.hi, y.hi, neg2(n));
    return fma2(x.hi, y.lo, fma2(x.lo, y.hi, f));
}

// the polynomial sincos of bf_device.cuh on both lanes
__device__ __forceinline__ void sincos2pi2(float2 f, float2 &s, float2 &c)
{
    const float2 M = dup2(12582912.0f);
    const float2 t = fma2(dup2(4.0f), f, M);
    const float2 r = fma2(dup2(-0.25f), sub2(t, M), f);
    const float2 u = mul2(r, r);
    float2 ps = fma2(u, dup2(SC_S3), dup2(SC_S2));
    ps = fma2(u, ps, dup2(SC_S1));
    ps = fma2(u, ps, dup2(SC_S0));
    const float2 sn = mul2(r, ps);
    float2 pc = fma2(u, dup2(SC_C3), dup2(SC_C2));
    pc = fma2(u, pc, dup2(SC_C1));
    const float2 cs = fma2(u, pc, dup2(1.0f));
    const int q0 = __float_as_int(t.x), q1 = __float_as_int(t.y);
    const float s0 = (q0 & 1) ? cs.x : sn.x, c0 = (q0 & 1) ? sn.x : cs.x;
    const float s1 = (q1 & 1) ? cs.y : sn.y, c1 = (q1 & 1) ? sn.y : cs.y;
    s.x = __int_as_float(__float_as_int(s0) ^ ((q0 & 2) << 30));
    s.y = __int_as_float(__float_as_int(s1) ^ ((q1 & 2) << 30));
    c.x = __int_as_float(__float_as_int(c0) ^ (((q0 + 1) & 2) << 30));
    c.y = __int_as_float(__float_as_int(c1) ^ (((q1 + 1) & 2) << 30));
}

// Ph<PMIXT> on two lanes: targets and sources are per lane (a shared one is duplicated)
template <class P, int D, int K> struct Ph2;

template <bool F, int D, int K>
struct Ph2<PMIXT<F>, D, K> {
    using PH = Ph<PMIXT<F>, D, K>;
    struct T { df2 x[D]; df2 A[D]; };
    struct Part { float2 f; df2 q; };

    static __device__ __forceinline__ df2 pack(const df &a, const df &b) { return {make_float2(a.hi, b.hi), make_float2(a.lo, b.lo)}; }

    static __device__ __forceinline__ T dup(const typename PH::T &a) { return pair(a, a); }
    static __device__ __forceinline__ Part dup(const typename PH::Part &p)
    {
        return Part{dup2(p.f), {dup2(p.q.hi), dup2(p.q.lo)}};
    }
    static __device__ __forceinline__ typename PH::Part lane0(const Part &p)
    {
        return typename PH::Part{p.f.x, {p.q.hi.x, p.q.lo.x}};
    }

    static __device__ __forceinline__ T pair(const typename PH::T &a, const typename PH::T &b)
    {
        T t;
#pragma unroll
        for (int k = 0; k < D; ++k) {
            t.x[k] = pack(a.x[k], b.x[k]);
            t.A[k] = pack(a.A[k], b.A[k]);
        }
        return t;
    }

    // contribution of source coordinate k: entries e0 (lane 0) and e1 (lane 1)
    static __device__ __forceinline__ Part part(const T &t, const MixSE &e0, const MixSE &e1, int k)
    {
        Part p{dup2(0.0f), {dup2(0.0f), dup2(0.0f)}};
        const df2 y = {make_float2(e0.a.x, e1.a.x), make_float2(e0.a.y, e1.a.y)};
        const df2 y2 = {make_float2(e0.a.z, e1.a.z), make_float2(e0.a.w, e1.a.w)};
        if constexpr (K == KIND_DOT) {
            p.f = df_mul_frac2(t.x[k], y);
        } else if constexpr (K == KIND_GENRADON) {
            p.f = df_mul_frac2(t.x[k], y);
            p.q = df_mul_u2(t.A[k], y2);
        } else if constexpr (K == KIND_HYPRADON) {
            p.q = (k == 0) ? y2 : df_mul_u2(t.A[1], y2);
        } else {
            p.q = df_add2(t.x[k], y);
        }
        return p;
    }
    static __device__ __forceinline__ Part add(const Part &u, const Part &v)
    {
        df2 s;
        if constexpr (K == KIND_GENRADON || K == KIND_HYPRADON)   // non-negative parts, larger first
            s = fast_two_sum2(make_float2(fmaxf(u.q.hi.x, v.q.hi.x), fmaxf(u.q.hi.y, v.q.hi.y)),
                              make_float2(fminf(u.q.hi.x, v.q.hi.x), fminf(u.q.hi.y, v.q.hi.y)));
        else
            s = two_sum2(u.q.hi, v.q.hi);
        return Part{add2(u.f, v.f), {s.hi, add2(add2(u.q.lo, v.q.lo), s.lo)}};
    }
    static __device__ __forceinline__ float2 fin(const KArgs<PMIXT<F>> &a, const T &t, const Part &p)
    {
        if constexpr (K == KIND_DOT) {
            return p.f;
        } else if constexpr (K == KIND_GENRADON) {
            return fma2(dup2(a.sc.sgn), df_frac2(df_sqrt_u2(p.q)), p.f);
        } else if constexpr (K == KIND_HYPRADON) {
            return df_mul_frac2(t.x[0], df_sqrt_u2(p.q));
        } else {
            return df_frac2(p.q);
        }
    }
};

// e^{2 pi i Phi} on two lanes from the summed parts: lane 0 -> e0, lane 1 -> e1
template <class P, int D, int K>
__device__ __forceinline__ void expphase_part2(const KArgs<P> &a, const typename Ph2<P, D, K>::T &t,
                                               const typename Ph2<P, D, K>::Part &pt, float2 &e0, float2 &e1)
{
    const float2 fr = Ph2<P, D, K>::fin(a, t, pt);
    float2 s, c;
    if constexpr (P::sfu) {
        sincos2pi_sfu(fr.x, s.x, c.x);
        sincos2pi_sfu(fr.y, s.y, c.y);
    } else {
        sincos2pi2(fr, s, c);
    }
    e0 = make_float2(c.x, s.x);
    e1 = make_float2(c.y, s.y);
}

}  // namespace bfk
