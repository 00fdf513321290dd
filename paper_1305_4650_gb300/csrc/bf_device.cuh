// Device code of the sm_103a Chebyshev-interpolation butterfly.
//
// The operator and the butterfly (Algorithm 1, Section 1.4 of Poulson,
// Demanet, Maxwell, Ying, "A Parallel Butterfly Algorithm"):
//   init   delta_t^{XB} = e^{-2pi i Phi(x0(X), y_t^B)} L_t^B(y) e^{2pi i Phi(x0(X), y)} g(y)
//   column w_{A_a,B'}(t) = e^{-2pi i Phi(x0(A_a), y_t^{B'})}
//                          sum_c sum_t' L_t^{B'}(y_t'^{B_c}) e^{2pi i Phi(x0(A_a), y_t'^{B_c})} w_{A,B_c}(t')
//   switch delta_s^{AB} = sum_t e^{2pi i Phi(x_s^A, y_t^B)} delta_t^{AB}               (level m)
//   row    w_{A_a,B'}(s) = sum_c e^{2pi i Phi(x_s^{A_a}, y0(B_c))}
//                          sum_t L_t^A(x_s^{A_a}) e^{-2pi i Phi(x_t^A, y0(B_c))} w_{A,B_c}(t)
//   final  f(x) = e^{2pi i Phi(x, y0(Y))} sum_t L_t^A(x) e^{-2pi i Phi(x_t^A, y0(Y))} w_{A,Y}(t)
//
// Layout.  Level-l weights live in HBM as [rhs][pair][r] complex numbers with
// pair index A * 2^{d(L-l)} + B (A, B Morton indices, dimension 0 in the lowest
// bit), node index t = sum_k t_k q^k.  A kernel pass handles "tiles": the
// 2^{dk} pairs (Ap, B) with Ap fixed at level l0 and B under one box B* at
// level l0+k.  Their inputs are contiguous and k merge levels close over them,
// so one CTA runs k levels in shared memory.  Inside the tile the update is
// in place: the 2^d outputs of a merge block overwrite its 2^d input slots,
// which leaves the tile in base-2^d digit-reversed order after k levels (the
// bit-reversal view of Section 2.2).
//
// Phases.  Phi is evaluated from per-level, per-dimension feature tables
// (coordinates, and sin/cos or squares of them, for box centres, Chebyshev
// nodes and grid points), so every feature is a table read.  In the mixed
// precision Phi is accumulated and reduced mod 1 in double-float arithmetic
// (pairs of FP32 numbers: Dekker's product via FMA and Knuth's two-sum), then a
// quadrant-reduced FP32 sincos (or the special-function unit's) gives
// e^{2 pi i Phi}; stages with a shared operand evaluate two phases at a time in
// the lanes of a float2 (bf_pair.cuh).  The FP64 variant uses doubles.  With a
// phase table (PM_TABLE) the single-RHS passes read the reduced phases recorded
// at plan creation (PM_BUILD) instead of evaluating Phi.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace bfk {

constexpr int QMAX = 8;
constexpr int DMAX = 3;

enum { KIND_DOT = 0, KIND_GENRADON = 1, KIND_HYPRADON = 2, KIND_SEPARABLE = 3 };
enum { F_INIT = 1, F_SWITCH = 2, F_FINAL = 4 };

// Where a kernel's phase factors come from: evaluated (PM_COMPUTE), evaluated and recorded
// in the plan's phase table (PM_BUILD, at plan creation), or read from it (PM_TABLE)
enum { PM_COMPUTE = 0, PM_BUILD = 1, PM_TABLE = 2 };

__host__ __device__ constexpr int ipow(int b, int e) { return e == 0 ? 1 : b * ipow(b, e - 1); }

// ------------------------------------------------------------ double-float

struct df {
    float hi, lo;
};

__device__ __forceinline__ df two_sum(float a, float b)
{
    float s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}

// requires |a| >= |b| (or a == 0)
__device__ __forceinline__ df fast_two_sum(float a, float b)
{
    float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ df df_mul(df x, df y)
{
    float p = __fmul_rn(x.hi, y.hi);
    float e = __fmaf_rn(x.hi, y.hi, -p);
    e = __fmaf_rn(x.hi, y.lo, e);
    e = __fmaf_rn(x.lo, y.hi, e);
    return fast_two_sum(p, e);
}

__device__ __forceinline__ df df_add(df x, df y)
{
    df s = two_sum(x.hi, y.hi);
    return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo)));
}

// nearest integer of |x| < 2^22: adding 1.5 * 2^23 leaves an ulp of 1, so the
// rounding of the addition is the round-to-nearest-even of x (two full-rate adds)
__device__ __forceinline__ float fround(float x)
{
    const float M = 12582912.0f;
    return __fsub_rn(__fadd_rn(x, M), M);
}

// unnormalised product hi + lo = x * y (all but the x.lo * y.lo term)
__device__ __forceinline__ df df_mul_u(df x, df y)
{
    float p = __fmul_rn(x.hi, y.hi);
    float e = __fmaf_rn(x.hi, y.hi, -p);
    e = __fmaf_rn(x.hi, y.lo, e);
    e = __fmaf_rn(x.lo, y.hi, e);
    return {p, e};
}

// sqrt of a non-negative (possibly unnormalised) double-float, to about 2^-44
// relative, returned unnormalised: one Newton step from the FP32 reciprocal root
__device__ __forceinline__ df df_sqrt_u(df x)
{
    float r = rsqrtf(fmaxf(x.hi, 1e-30f));
    float s = __fmul_rn(x.hi, r);
    float res = __fadd_rn(__fmaf_rn(-s, s, x.hi), x.lo);
    return {s, __fmul_rn(res, __fmul_rn(0.5f, r))};
}

// x - nearest integer (|x| < 2^22), one float in about [-0.5, 0.5]
__device__ __forceinline__ float df_frac(df x) { return __fadd_rn(__fsub_rn(x.hi, fround(x.hi)), x.lo); }

// frac of a product x*y with both factors double-float, |x y| < 2^22: one FMA against
// 1.5 * 2^23 gives the integer n nearest to x.hi*y.hi, a second FMA the remainder
// x.hi*y.hi - n (|.| <= 1/2, one rounding), and two more add the cross terms (the
// x.lo*y.lo term is below FP32 resolution); the result lies in (-1, 1)
__device__ __forceinline__ float df_mul_frac(df x, df y)
{
    const float M = 12582912.0f;
    const float n = __fsub_rn(__fmaf_rn(x.hi, y.hi, M), M);
    const float f = __fmaf_rn(x.hi, y.hi, -n);
    return __fmaf_rn(x.hi, y.lo, __fmaf_rn(x.lo, y.hi, f));
}

// ------------------------------------------------------- precision traits

struct PF64 {
    using R = double;
    using C = double2;
    struct TE { double2 a, b; };   // target feature table entry: f0, f1 | f2, pad
    struct SE { double2 a; };      // source feature table entry: f0, f1
    struct Sc { double s3, sgn; }; // s/3 and sign(s)
    static constexpr bool is_f64 = true;
    static constexpr bool sfu = false;
};

struct MixTE { float4 a, b; };  // (f0.hi, f0.lo, f1.hi, f1.lo) | (f2.hi, f2.lo, -, -)
struct MixSE { float4 a; };     // (f0.hi, f0.lo, f1.hi, f1.lo)
struct MixSc { float s3hi, s3lo, sgn, pad; };

// complex64 weights, double-float phase; SFU = true takes sin/cos of the reduced phase
// from the special-function unit (__sincosf) instead of the polynomial below
template <bool SFU>
struct PMIXT {
    using R = float;
    using C = float2;
    using TE = MixTE;
    using SE = MixSE;
    using Sc = MixSc;
    static constexpr bool is_f64 = false;
    static constexpr bool sfu = SFU;
};
using PMIX = PMIXT<false>;
using PMIXF = PMIXT<true>;

__device__ __forceinline__ void sincos2pi(double fr, double &s, double &c) { sincospi(2.0 * fr, &s, &c); }
// sin and cos of 2 pi f for |f| < 2^20: quadrant reduction f = j/4 + r with |r| <= 1/8,
// then sin(2 pi r) = r S(r^2) (degree 7) and cos(2 pi r) = C(r^2) (degree 6) with 2 pi
// folded into the coefficients, which are minimax fits of the absolute error on
// |r| <= 1/8 (Remez exchange, csrc/sincos_fit.py; truncation error 1.2e-9 and 3.2e-8); the quadrant j rotates
// (cos, sin) by j * 90 degrees.  Max abs error ~1e-7 (checked against FP64 sincospi by
// bf_selfcheck_sincos).  sincos2pi2 (bf_pair.cuh) performs the same operations per lane.
constexpr float SC_S0 = 6.28318500518798828f, SC_S1 = -41.3416290283203125f, SC_S2 = 81.5881271362304688f,
                SC_S3 = -75.2400665283203125f;
constexpr float SC_C1 = -19.7391681671142578f, SC_C2 = 64.9232254028320312f, SC_C3 = -83.665924072265625f;
__device__ __forceinline__ void sincos2pi(float f, float &s, float &c)
{
    const float M = 12582912.0f;
    const float t = __fmaf_rn(4.0f, f, M);                 // j + 1.5 * 2^23
    const int q = __float_as_int(t);                       // low two bits: j mod 4
    const float r = __fmaf_rn(-0.25f, __fsub_rn(t, M), f);
    const float u = __fmul_rn(r, r);
    float ps = __fmaf_rn(u, SC_S3, SC_S2);
    ps = __fmaf_rn(u, ps, SC_S1);
    ps = __fmaf_rn(u, ps, SC_S0);
    const float sn = __fmul_rn(r, ps);
    float pc = __fmaf_rn(u, SC_C3, SC_C2);
    pc = __fmaf_rn(u, pc, SC_C1);
    const float cs = __fmaf_rn(u, pc, 1.0f);
    const float s1 = (q & 1) ? cs : sn;
    const float c1 = (q & 1) ? sn : cs;
    s = __int_as_float(__float_as_int(s1) ^ ((q & 2) << 30));
    c = __int_as_float(__float_as_int(c1) ^ (((q + 1) & 2) << 30));
}

// sin and cos of 2 pi f from the special-function unit after reduction to |f| <= 1/2
// (CUDA documents 2^-21.41 absolute error for |x| <= pi)
__device__ __forceinline__ void sincos2pi_sfu(float f, float &s, float &c)
{
    const float r = __fsub_rn(f, fround(f));
    __sincosf(__fmul_rn(r, 6.28318530717958647692f), &s, &c);
}

__device__ __forceinline__ float2 cmul(float2 a, float2 b)
{
    return make_float2(__fmaf_rn(a.x, b.x, -(a.y * b.y)), __fmaf_rn(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ double2 cmul(double2 a, double2 b) { return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
// conj(a) * b
__device__ __forceinline__ float2 cjmul(float2 a, float2 b)
{
    return make_float2(__fmaf_rn(a.x, b.x, a.y * b.y), __fmaf_rn(a.x, b.y, -(a.y * b.x)));
}
__device__ __forceinline__ double2 cjmul(double2 a, double2 b) { return make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x); }
__device__ __forceinline__ void cfma(float2 &acc, float m, float2 v) { acc.x = fmaf(m, v.x, acc.x); acc.y = fmaf(m, v.y, acc.y); }
__device__ __forceinline__ void cfma(double2 &acc, double m, double2 v) { acc.x = fma(m, v.x, acc.x); acc.y = fma(m, v.y, acc.y); }
// acc += m v with m given twice (m2 = (m, m)): one packed FMA on sm_100+, the same roundings as cfma
__device__ __forceinline__ void cfma2(float2 &acc, float2 m2, float2 v) { acc = __ffma2_rn(m2, v, acc); }
__device__ __forceinline__ void cfma2(double2 &acc, double2 m2, double2 v) { acc.x = fma(m2.x, v.x, acc.x); acc.y = fma(m2.y, v.y, acc.y); }
template <class C> __device__ __forceinline__ C czero();
template <> __device__ __forceinline__ float2 czero<float2>() { return make_float2(0.f, 0.f); }
template <> __device__ __forceinline__ double2 czero<double2>() { return make_double2(0.0, 0.0); }

// ------------------------------------------------------------ kernel args

template <class P>
struct KArgs {
    using R = typename P::R;
    using C = typename P::C;
    const typename P::TE *tt[DMAX];   // target feature tables, one per dimension
    const typename P::SE *st[DMAX];   // source feature tables
    const C *win;                     // input weights  [rhs][pair][r] (unused with F_INIT)
    C *wout;                          // output weights (unused with F_FINAL)
    const C *g;                       // sources [rhs][N^d] (F_INIT)
    C *f;                             // targets [rhs][N^d] (F_FINAL)
    const C *fadj;                    // adjoint input: target values [rhs][N^d] (final^H)
    C *gadj;                          // adjoint output: source values [rhs][N^d] (init^H)
    int64_t wstride;                  // per-rhs stride of weights, in complex numbers
    int64_t npts;                     // N^d
    R M[2][QMAX][QMAX];               // M[h][t][t'] = l_t((z_t' + h - 1/2)/2)
    C M2[2][QMAX][QMAX];              // the same, each value twice (operand of a packed FMA)
    R lsrc[QMAX], ltgt[QMAX];         // l_t(off - 1/2): Lagrange values of the grid point in its leaf box
    typename P::Sc sc;
    int L, l0, k, flags, kind;
    int T;                            // tiles per CTA (T * 2^{dk} pairs)
    int nrhs;                         // right-hand sides of the launch (multi-RHS kernels)
    int rc;                           // right-hand sides per scratch chunk (multi-RHS kernels)
    const void *ctab;                 // target features at box centres, levels 0..ctab_levels (or null)
    int ctab_levels;
    C *ptab;                          // phase table of the pass (multi-RHS passes with tables) or null
    int64_t ptab_cta;                 // phase-table complex numbers per CTA of the pass
    int *err;                         // set by a bounded wait that gave up, or a table-size mismatch (or null)
    float *ftab;                      // reduced-phase table of a single-RHS pass (PM_BUILD, PM_TABLE) or null
    int64_t ftab_cta;                 // floats of that table per CTA
    int ncta;                         // CTAs (tile groups of T tiles) of the pass (multi-RHS kernels)
    // source-domain sharding over 2^shard_g ranks (see shard_cta / shard_owned): 0 off,
    // 1 the launch covers the rank's tiles only, 2 every tile, other ranks' inputs read as zero
    int shard_mode, shard_g, shard_r;
    // tensor map (a CUtensorMap in device memory) of a.win viewed as [rhs][complex number]
    // for tiled bulk copies, or null (the tensor-core switch)
    const void *wmap;
};

// Sharding.  Rank r of G = 2^g owns the source boxes whose top g Morton bits equal r.  A merge
// combines the children of one source box, so while the output source boxes still have g
// bits every pair's inputs lie on the pair's own rank.  Mode 1 maps CTA b of a launch over
// the rank's tile groups to the b-th tile group whose source boxes the rank owns (the host
// makes T a divisor of the owned range, so no group straddles two ranks); mode 2 keeps the
// CTA index and shard_owned tells which input pairs the rank holds.
template <int D, class P>
__device__ __forceinline__ uint32_t shard_cta(const KArgs<P> &a, uint32_t b)
{
    if (a.shard_mode != 1) return b;
    const int ls = D * (a.L - a.l0 - a.k);          // log2 of the tiles per target box
    const int lt = __ffs(a.T) - 1;                   // log2 T
    const int lper = ls - a.shard_g - lt;            // log2 of the rank's groups per target box
    return ((b >> lper) << (ls - lt)) | ((uint32_t)a.shard_r << lper) | (b & ((1u << lper) - 1u));
}
// input pair I of level a.l0 (index A 2^{D(L-l0)} + B) belongs to this rank (mode 2)
template <int D, class P>
__device__ __forceinline__ bool shard_owned(const KArgs<P> &a, int64_t I)
{
    const int lb = D * (a.L - a.l0);
    return (int)((I & ((1LL << lb) - 1)) >> (lb - a.shard_g)) == a.shard_r;
}

// --------------------------------------------------------- index helpers

// Morton decode by bit compaction: every D-th bit of m, starting at bit k, gathered
// into c[k] (mask-and-shift steps, no loop; valid for up to 32/D bits per dimension)
__device__ __forceinline__ uint32_t compact_by2(uint32_t x)
{
    x &= 0x55555555u;
    x = (x | (x >> 1)) & 0x33333333u;
    x = (x | (x >> 2)) & 0x0f0f0f0fu;
    x = (x | (x >> 4)) & 0x00ff00ffu;
    return (x | (x >> 8)) & 0x0000ffffu;
}
__device__ __forceinline__ uint32_t compact_by3(uint32_t x)
{
    x &= 0x09249249u;
    x = (x | (x >> 2)) & 0x030c30c3u;
    x = (x | (x >> 4)) & 0x0300f00fu;
    x = (x | (x >> 8)) & 0x030000ffu;
    return (x | (x >> 16)) & 0x000003ffu;
}

template <int D>
__device__ __forceinline__ void morton_decode(uint32_t m, int /*bits*/, int *c)
{
    if constexpr (D == 2) {
        c[0] = (int)compact_by2(m);
        c[1] = (int)compact_by2(m >> 1);
    } else {
        c[0] = (int)compact_by3(m);
        c[1] = (int)compact_by3(m >> 1);
        c[2] = (int)compact_by3(m >> 2);
    }
}

// reverse the order of the first n base-2^D digits of x
template <int D>
__device__ __forceinline__ uint32_t digit_rev(uint32_t x, int n)
{
    uint32_t y = 0;
    for (int j = 0; j < n; ++j) {
        y = (y << D) | (x & ((1u << D) - 1));
        x >>= D;
    }
    return y;
}

// target table: level l has 2^l boxes per dimension, (Q+2) slots each (< 2^31 entries)
template <int Q> __device__ __forceinline__ int toff(int l) { return ((1 << l) - 1) * (Q + 2); }
// source table: level l has 2^(L-l) boxes per dimension
template <int Q> __device__ __forceinline__ int soff(int L, int l) { return ((2 << L) - (2 << (L - l))) * (Q + 2); }

// ------------------------------------------------------------------ phase
//
// Target features per dimension (built on the host, kind-specific):
//   DOT        f0 = s x
//   GENRADON   f0 = s x, f1 = sin 2pi x, f2 = cos 2pi x
//   HYPRADON   f0 = s x, f1 = x^2
//   SEPARABLE  f0 = s sin 2pi (x + (k+1)/7)
// Source features per dimension:
//   DOT y | GENRADON y, y^2 | HYPRADON -, y^2 | SEPARABLE s y^2/(k+2)

template <class P, int D, int K> struct Ph;

template <bool F, int D, int K>
struct Ph<PMIXT<F>, D, K> {
    struct T { df x[D]; df A[D]; };
    struct S { df y[D]; df y2[D]; };

    static __device__ __forceinline__ df hi(const float4 &v) { return {v.x, v.y}; }
    static __device__ __forceinline__ df lo(const float4 &v) { return {v.z, v.w}; }

    // target point from its per-dimension table entries; GENRADON forms A_k = (s a_k(x))^2
    static __device__ __forceinline__ T tgt(const KArgs<PMIXT<F>> &a, const MixTE *e)
    {
        T t;
#pragma unroll
        for (int k = 0; k < D; ++k) { t.x[k] = hi(e[k].a); t.A[k] = lo(e[k].a); }
        if constexpr (K == KIND_GENRADON) {
            const df s3 = {a.sc.s3hi, a.sc.s3lo};
#pragma unroll
            for (int k = 0; k < D; ++k) {
                df u;
                if constexpr (D == 2) u = (k == 0) ? df_mul_u(lo(e[0].a), lo(e[1].a)) : df_mul_u(hi(e[0].b), hi(e[1].b));
                else u = df_mul_u(lo(e[k].a), hi(e[(k + 1) % D].b));
                df two = two_sum(2.0f, u.hi);
                u = {two.hi, __fadd_rn(two.lo, u.lo)};
                u = df_mul_u(u, s3);
                t.A[k] = df_mul(u, u);
            }
        }
        return t;
    }

    static __device__ __forceinline__ void src1(S &s, int k, const MixSE &e)
    {
        s.y[k] = hi(e.a);
        s.y2[k] = lo(e.a);
    }

    // Per-dimension split of Phi: part(t, y_k entry, k) is the contribution of source
    // coordinate k; parts add (add), and fin() turns their sum into Phi minus an integer.
    // Loops hoist the parts of the source coordinates that do not change.
    struct Part { float f; df q; };
    static __device__ __forceinline__ Part part(const T &t, const MixSE &e, int k)
    {
        Part p{0.0f, {0.0f, 0.0f}};
        const df y = hi(e.a), y2 = lo(e.a);
        if constexpr (K == KIND_DOT) {
            p.f = df_mul_frac(t.x[k], y);
        } else if constexpr (K == KIND_GENRADON) {
            p.f = df_mul_frac(t.x[k], y);
            p.q = df_mul_u(t.A[k], y2);
        } else if constexpr (K == KIND_HYPRADON) {
            p.q = (k == 0) ? y2 : df_mul_u(t.A[1], y2);
        } else {
            p.q = df_add(t.x[k], y);
        }
        return p;
    }
    static __device__ __forceinline__ Part add(const Part &u, const Part &v)
    {
        df s;
        if constexpr (K == KIND_GENRADON || K == KIND_HYPRADON) {
            // both parts are sums of squares times non-negative factors: with the larger one
            // first the fast two-sum is exact (the same s and error term as the two-sum)
            s = fast_two_sum(fmaxf(u.q.hi, v.q.hi), fminf(u.q.hi, v.q.hi));
        } else {
            s = two_sum(u.q.hi, v.q.hi);
        }
        return Part{u.f + v.f, {s.hi, __fadd_rn(__fadd_rn(u.q.lo, v.q.lo), s.lo)}};
    }
    static __device__ __forceinline__ float fin(const KArgs<PMIXT<F>> &a, const T &t, const Part &p)
    {
        if constexpr (K == KIND_DOT) {
            return p.f;
        } else if constexpr (K == KIND_GENRADON) {
            return __fmaf_rn(a.sc.sgn, df_frac(df_sqrt_u(p.q)), p.f);
        } else if constexpr (K == KIND_HYPRADON) {
            return df_mul_frac(t.x[0], df_sqrt_u(p.q));
        } else {
            return df_frac(p.q);
        }
    }

    // Phi(x, y) minus an integer, |result| < 2 (the sincos reduces it further)
    static __device__ __forceinline__ float frac(const KArgs<PMIXT<F>> &a, const T &t, const S &s)
    {
        if constexpr (K == KIND_DOT) {
            float f = 0.0f;
#pragma unroll
            for (int k = 0; k < D; ++k) f += df_mul_frac(t.x[k], s.y[k]);
            return f;
        } else if constexpr (K == KIND_GENRADON) {
            float f = 0.0f;
#pragma unroll
            for (int k = 0; k < D; ++k) f += df_mul_frac(t.x[k], s.y[k]);
            // sum_k A_k y_k^2 from unnormalised products and one two-sum of the leading parts
            df p0 = df_mul_u(t.A[0], s.y2[0]);
            float lo = p0.lo, hi = p0.hi;
#pragma unroll
            for (int k = 1; k < D; ++k) {
                df pk = df_mul_u(t.A[k], s.y2[k]);
                df sk = fast_two_sum(fmaxf(hi, pk.hi), fminf(hi, pk.hi));   // both non-negative
                hi = sk.hi;
                lo = __fadd_rn(lo, __fadd_rn(pk.lo, sk.lo));
            }
            const float fr = df_frac(df_sqrt_u({hi, lo}));
            return __fmaf_rn(a.sc.sgn, fr, f);
        } else if constexpr (K == KIND_HYPRADON) {
            df q = df_add(s.y2[0], df_mul(t.A[1], s.y2[1]));
            return df_mul_frac(t.x[0], df_sqrt_u(q));
        } else {
            df acc = {0.0f, 0.0f};
#pragma unroll
            for (int k = 0; k < D; ++k) acc = df_add(acc, df_add(t.x[k], s.y[k]));
            return df_frac(acc);
        }
    }
};

template <int D, int K>
struct Ph<PF64, D, K> {
    struct T { double x[D]; double A[D]; };
    struct S { double y[D]; double y2[D]; };

    static __device__ __forceinline__ T tgt(const KArgs<PF64> &a, const PF64::TE *e)
    {
        T t;
#pragma unroll
        for (int k = 0; k < D; ++k) { t.x[k] = e[k].a.x; t.A[k] = e[k].a.y; }
        if constexpr (K == KIND_GENRADON) {
#pragma unroll
            for (int k = 0; k < D; ++k) {
                double u;
                if constexpr (D == 2) u = (k == 0) ? e[0].a.y * e[1].a.y : e[0].b.x * e[1].b.x;
                else u = e[k].a.y * e[(k + 1) % D].b.x;
                u = (2.0 + u) * a.sc.s3;
                t.A[k] = u * u;
            }
        }
        return t;
    }

    static __device__ __forceinline__ void src1(S &s, int k, const PF64::SE &e)
    {
        s.y[k] = e.a.x;
        s.y2[k] = e.a.y;
    }

    struct Part { double f, q; };
    static __device__ __forceinline__ Part part(const T &t, const PF64::SE &e, int k)
    {
        const double y = e.a.x, y2 = e.a.y;
        if constexpr (K == KIND_DOT) return Part{t.x[k] * y, 0.0};
        else if constexpr (K == KIND_GENRADON) return Part{t.x[k] * y, t.A[k] * y2};
        else if constexpr (K == KIND_HYPRADON) return Part{0.0, k == 0 ? y2 : t.A[1] * y2};
        else return Part{t.x[k] + y, 0.0};
    }
    static __device__ __forceinline__ Part add(const Part &u, const Part &v) { return Part{u.f + v.f, u.q + v.q}; }
    static __device__ __forceinline__ double fin(const KArgs<PF64> &a, const T &t, const Part &p)
    {
        double v;
        if constexpr (K == KIND_DOT || K == KIND_SEPARABLE) v = p.f;
        else if constexpr (K == KIND_GENRADON) v = p.f + a.sc.sgn * sqrt(p.q);
        else v = t.x[0] * sqrt(p.q);
        return v - rint(v);
    }

    static __device__ __forceinline__ double frac(const KArgs<PF64> &a, const T &t, const S &s)
    {
        double p = 0.0;
        if constexpr (K == KIND_DOT) {
#pragma unroll
            for (int k = 0; k < D; ++k) p += t.x[k] * s.y[k];
        } else if constexpr (K == KIND_GENRADON) {
            double q = 0.0;
#pragma unroll
            for (int k = 0; k < D; ++k) {
                p += t.x[k] * s.y[k];
                q += t.A[k] * s.y2[k];
            }
            p += a.sc.sgn * sqrt(q);
        } else if constexpr (K == KIND_HYPRADON) {
            p = t.x[0] * sqrt(s.y2[0] + t.A[1] * s.y2[1]);
        } else {
#pragma unroll
            for (int k = 0; k < D; ++k) p += t.x[k] + s.y[k];
        }
        return p - rint(p);
    }
};

// e^{2 pi i Phi} as a complex number of the working precision
template <class P, int D, int K>
__device__ __forceinline__ typename P::C expphase(const KArgs<P> &a, const typename Ph<P, D, K>::T &t,
                                                  const typename Ph<P, D, K>::S &s)
{
    typename P::R fr = Ph<P, D, K>::frac(a, t, s), sn, cs;
    if constexpr (P::sfu)
        sincos2pi_sfu(fr, sn, cs);
    else
        sincos2pi(fr, sn, cs);
    typename P::C e;
    e.x = cs;
    e.y = sn;
    return e;
}

template <class P, int D, int K>
__device__ __forceinline__ typename P::C expphase_part(const KArgs<P> &a, const typename Ph<P, D, K>::T &t,
                                                       const typename Ph<P, D, K>::Part &pt)
{
    typename P::R fr = Ph<P, D, K>::fin(a, t, pt), sn, cs;
    if constexpr (P::sfu)
        sincos2pi_sfu(fr, sn, cs);
    else
        sincos2pi(fr, sn, cs);
    typename P::C e;
    e.x = cs;
    e.y = sn;
    return e;
}

// complex multiply-accumulate acc += e * u as four FMAs
__device__ __forceinline__ void cmac(float2 &acc, float2 e, float2 u)
{
    acc.x = __fmaf_rn(e.x, u.x, acc.x);
    acc.x = __fmaf_rn(-e.y, u.y, acc.x);
    acc.y = __fmaf_rn(e.x, u.y, acc.y);
    acc.y = __fmaf_rn(e.y, u.x, acc.y);
}
__device__ __forceinline__ void cmac(double2 &acc, double2 e, double2 u)
{
    acc.x = fma(e.x, u.x, acc.x);
    acc.x = fma(-e.y, u.y, acc.x);
    acc.y = fma(e.x, u.y, acc.y);
    acc.y = fma(e.y, u.x, acc.y);
}

}  // namespace bfk

#include "bf_pair.cuh"   // the same phase arithmetic on the two lanes of a float2

namespace bfk {

// table reads
template <class P, int Q>
__device__ __forceinline__ typename P::TE tget(const KArgs<P> &a, int k, int l, int box, int slot)
{
    return a.tt[k][toff<Q>(l) + box * (Q + 2) + slot];
}
template <class P, int Q>
__device__ __forceinline__ typename P::SE sget(const KArgs<P> &a, int k, int l, int box, int slot)
{
    return a.st[k][soff<Q>(a.L, l) + box * (Q + 2) + slot];
}

// features of the target point of box `coords` at level l, slot per dimension
template <class P, int D, int Q, int K>
__device__ __forceinline__ typename Ph<P, D, K>::T tpoint(const KArgs<P> &a, int l, const int *coords, const int *slot)
{
    typename P::TE e[D];
#pragma unroll
    for (int k = 0; k < D; ++k) e[k] = tget<P, Q>(a, k, l, coords[k], slot[k]);
    return Ph<P, D, K>::tgt(a, e);
}

template <class P, int D, int Q, int K>
__device__ __forceinline__ typename Ph<P, D, K>::S spoint(const KArgs<P> &a, int l, const int *coords, const int *slot)
{
    typename Ph<P, D, K>::S s;
#pragma unroll
    for (int k = 0; k < D; ++k) Ph<P, D, K>::src1(s, k, sget<P, Q>(a, k, l, coords[k], slot[k]));
    return s;
}

// Target features at the centre of box A (Morton) at level l: from the plan's centre
// table when it covers the level (filled by k_center_table with this same code), else
// built from the per-dimension tables.
template <class P, int D, int Q, int K>
__device__ __forceinline__ typename Ph<P, D, K>::T tcenter(const KArgs<P> &a, int l, uint32_t A, const int *ca)
{
    using T = typename Ph<P, D, K>::T;
    if (l <= a.ctab_levels) {
        const int off = (int)((((uint32_t)1 << (D * l)) - 1u) / ((1u << D) - 1u));
        return static_cast<const T *>(a.ctab)[off + A];
    }
    const int ctr[DMAX] = {Q, Q, Q};
    return tpoint<P, D, Q, K>(a, l, ca, ctr);
}

template <class P, int D, int Q, int K>
__global__ void k_center_table(const KArgs<P> a, typename Ph<P, D, K>::T *out, int levels)
{
    const int total = (int)((((uint32_t)1 << (D * (levels + 1))) - 1u) / ((1u << D) - 1u));
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
        int l = 0;
        while ((int)((((uint32_t)1 << (D * (l + 1))) - 1u) / ((1u << D) - 1u)) <= e) ++l;
        const uint32_t A = (uint32_t)(e - (int)((((uint32_t)1 << (D * l)) - 1u) / ((1u << D) - 1u)));
        int ca[DMAX];
        morton_decode<D>(A, l, ca);
        const int ctr[DMAX] = {Q, Q, Q};
        out[e] = tpoint<P, D, Q, K>(a, l, ca, ctr);
    }
}

// ------------------------------------------------------------ tile passes
//
// A CTA owns NP consecutive pairs of the pass's input level: T = NP / 2^{dk}
// tiles of 2^{dk} pairs.  It runs NT = NP * q threads, and every stage below is
// cut into a multiple of NT equal work items, so no thread idles at a barrier
// while others finish a longer item.

constexpr int kmax_for(int D, int RR, int CS, int Q)
{
    int k = 1;
    while (k < (D == 2 ? 4 : 2) && 3 * (1 << (D * (k + 1))) * RR * CS <= 100 * 1024 && (1 << (D * (k + 1))) * Q <= 512) ++k;
    return k;
}

template <int D, int Q, class P>
struct Cfg {
    static constexpr int RR = ipow(Q, D);
    static constexpr int KMAX = kmax_for(D, RR, (int)sizeof(typename P::C), Q);
    static constexpr int NP = 1 << (D * KMAX);    // pairs per CTA
    static constexpr int NT = NP * Q;             // threads per CTA
    static constexpr int MINB = (640 / NT) < 1 ? 1 : ((640 / NT) > 8 ? 8 : 640 / NT);
    // the mixed-precision column pass at d = 2, q = 5 runs 3 CTAs per SM (64 registers, some
    // spills): measured 4.5% faster on its dominant pass and 9% on the init pass than 2 CTAs
    static constexpr int MINB_COL = (D == 2 && Q == 5 && !P::is_f64) ? 3 : MINB;
    // the column pass reading a phase table (d = 2: one more CTA per SM than evaluating)
    static constexpr int MINB_TAB = D == 2 ? MINB + 1 : MINB;
};

template <int D, int Q, class P, int K>
struct Tile {
    using R = typename P::R;
    using C = typename P::C;
    using PH = Ph<P, D, K>;
    static constexpr int NC = 1 << D;
    static constexpr int RR = ipow(Q, D);
    static constexpr int QD1 = ipow(Q, D - 1);

    // geometry of one output pair of a column level, shared by all items of that pair (2q in
    // stage A, q^{d-1} in stage B): computed once per level into shared memory
    struct __align__(16) Geo {
        typename PH::T tA;   // features of the target box centre
        int cbq[DMAX];       // coordinates of the parent source box
        int base;            // the merge block's first input slot in the tile
    };
    static_assert(sizeof(Geo) % 16 == 0 && sizeof(Geo) == (sizeof(typename PH::T) + 16 + 15) / 16 * 16,
                  "Geo size (the host reserves round16(tsize + 16) bytes per pair)");

    // ---- reduced-phase table of a single-RHS pass (mixed precisions).  The block of
    // one stage is [phase j of an item][item], so one phase index over a warp's items is one
    // coalesced access.  The table holds the reduced phase that the evaluating kernel feeds
    // to its sincos, so reading it gives the evaluating kernel's results exactly.
    struct FT {
        float *p;   // the stage's block
        int n;      // items of the stage
        __device__ __forceinline__ float *at(int j, int it) const { return p + (int64_t)j * n + it; }
    };
    // items of the stages that evaluate phases, and phases per item
    static __device__ __forceinline__ int n_col_a(const KArgs<P> &a) { return a.T * ((1 << (D * a.k)) >> D) * NC * 2 * Q; }
    static __device__ __forceinline__ int n_col_b(const KArgs<P> &a) { return a.T * ((1 << (D * a.k)) >> D) * NC * QD1; }
    static __device__ __forceinline__ int n_switch(const KArgs<P> &a) { return a.T * (1 << (D * a.k)) * QD1; }
    static __device__ __forceinline__ int n_row_a(const KArgs<P> &a) { return a.T * ((1 << (D * a.k)) >> D) * NC * QD1; }
    static __device__ __forceinline__ int n_row_b(const KArgs<P> &a) { return a.T * ((1 << (D * a.k)) >> D) * NC * Q; }
    static constexpr int PH_COL_A = (NC / 2) * QD1, PH_COL_B = Q, PH_SWITCH = Q * RR, PH_ROW_A = Q, PH_ROW_B = NC * QD1;
    // floats of the table one CTA of this pass reads (the phases of the switch of the
    // factorised kinds are evaluated, not tabled)
    static __device__ __forceinline__ int64_t table_floats(const KArgs<P> &a, bool row)
    {
        int64_t f = row ? (int64_t)n_row_a(a) * PH_ROW_A + (int64_t)n_row_b(a) * PH_ROW_B
                        : (int64_t)n_col_a(a) * PH_COL_A + (int64_t)n_col_b(a) * PH_COL_B;
        f *= a.k;
        if (!row && (a.flags & F_SWITCH) && K != KIND_DOT && K != KIND_SEPARABLE) f += (int64_t)n_switch(a) * PH_SWITCH;
        return f;
    }
    // floats of one level's table blocks (both stages) and of the switch's
    static __device__ __forceinline__ int64_t level_floats(const KArgs<P> &a, bool row)
    {
        return row ? (int64_t)n_row_a(a) * PH_ROW_A + (int64_t)n_row_b(a) * PH_ROW_B
                   : (int64_t)n_col_a(a) * PH_COL_A + (int64_t)n_col_b(a) * PH_COL_B;
    }
    // ask the TMA engine to bring a table block into L2 ahead of its loads (a hint: no
    // completion, nothing written); 16-byte aligned, a multiple of 16 bytes, 64 KB per copy
    static __device__ __forceinline__ void prefetch_l2(const float *p, int64_t nfloats)
    {
        if (threadIdx.x != 0) return;
        for (int64_t o = 0; o < nfloats; o += 16384) {
            const unsigned bytes = (unsigned)(4 * (nfloats - o < 16384 ? nfloats - o : 16384));
            asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p + o), "r"(bytes) : "memory");
        }
    }
    static __device__ __forceinline__ C cis(R fr)
    {
        R sn, cs;
        if constexpr (P::sfu)
            sincos2pi_sfu(fr, sn, cs);
        else
            sincos2pi(fr, sn, cs);
        C e;
        e.x = cs;
        e.y = sn;
        return e;
    }
    // one factor from its reduced phase (summed parts): evaluated, evaluated and recorded, or read
    template <int PM>
    static __device__ __forceinline__ C ph(const KArgs<P> &a, const typename PH::T &t, const typename PH::Part &pt, float *q)
    {
        R fr;
        if constexpr (PM == PM_TABLE) {
            fr = __ldcs(q);
        } else {
            fr = PH::fin(a, t, pt);
            if constexpr (PM == PM_BUILD) __stcs(q, fr);
        }
        return cis(fr);
    }
    // the same from the whole source point
    template <int PM>
    static __device__ __forceinline__ C phs(const KArgs<P> &a, const typename PH::T &t, const typename PH::S &sv, float *q)
    {
        R fr;
        if constexpr (PM == PM_TABLE) {
            fr = __ldcs(q);
        } else {
            fr = PH::frac(a, t, sv);
            if constexpr (PM == PM_BUILD) __stcs(q, fr);
        }
        return cis(fr);
    }
    // two factors in the lanes of a float2 (bf_pair.cuh); q1 null: lane 1 is not recorded or read
    template <int PM, class T2, class Part2>
    static __device__ __forceinline__ void ph2(const KArgs<P> &a, const T2 &t, const Part2 &pt, float *q0, float *q1,
                                               float2 &e0, float2 &e1)
    {
        float2 fr;
        if constexpr (PM == PM_TABLE) {
            fr.x = __ldcs(q0);
            fr.y = q1 ? __ldcs(q1) : 0.0f;
        } else {
            fr = Ph2<P, D, K>::fin(a, t, pt);
            if constexpr (PM == PM_BUILD) {
                __stcs(q0, fr.x);
                if (q1) __stcs(q1, fr.y);
            }
        }
        float2 sn, cs;
        if constexpr (P::sfu) {
            sincos2pi_sfu(fr.x, sn.x, cs.x);
            sincos2pi_sfu(fr.y, sn.y, cs.y);
        } else {
            sincos2pi2(fr, sn, cs);
        }
        e0 = make_float2(cs.x, sn.x);
        e1 = make_float2(cs.y, sn.y);
    }

    static __device__ __forceinline__ float2 cadd(float2 x, float2 y) { return make_float2(x.x + y.x, x.y + y.y); }
    static __device__ __forceinline__ double2 cadd(double2 x, double2 y) { return make_double2(x.x + y.x, x.y + y.y); }

    // (Ap, B*) of the CTA's tile tau: tile index = Ap * 2^{D(L-l0-k)} + B*
    static __device__ __forceinline__ void tile_of(const KArgs<P> &a, int tau, uint32_t &Ap, uint32_t &Bstar)
    {
        const uint32_t tile = shard_cta<D>(a, blockIdx.x) * (uint32_t)a.T + (uint32_t)tau;   // < 2^30
        const int sh = D * (a.L - a.l0 - a.k);
        Ap = tile >> sh;
        Bstar = tile & ((1u << sh) - 1u);
    }

    // ---- init: weights of the leaf pairs (X, B); items (tau, b, t)
    static __device__ void init(const KArgs<P> &a, C *Wt, int rhs)
    {
        const int k = a.k, n = 1 << (D * k);
        const int L = a.L;
        const int cX[DMAX] = {0, 0, 0};
        const int ctr[DMAX] = {Q, Q, Q};
        const typename PH::T tX = tpoint<P, D, Q, K>(a, 0, cX, ctr);   // centre of X
        // the grid point of a leaf box has a non-zero Lagrange value at few nodes (one for points
        // at box corners): zero the weights, then compute those nodes only
        __shared__ int nzt[RR];
        __shared__ int nnz;
        if (threadIdx.x == 0) {
            int c = 0;
            for (int t = 0; t < RR; ++t) {
                R lag = R(1);
                for (int j = 0, tt = t; j < D; ++j, tt /= Q) lag *= a.lsrc[tt % Q];
                if (lag != R(0)) nzt[c++] = t;
            }
            nnz = c;
        }
        for (int it = threadIdx.x; it < a.T * n * RR; it += blockDim.x) Wt[it] = czero<C>();
        __syncthreads();
        for (int it = threadIdx.x; it < a.T * n * nnz; it += blockDim.x) {
            const int pr = it / nnz, t = nzt[it - pr * nnz];
            const int b = pr & (n - 1), tau = pr >> (D * k);
            uint32_t Ap, Bstar;
            tile_of(a, tau, Ap, Bstar);
            const uint32_t B = (Bstar << (D * k)) + b;
            int cb[DMAX];
            morton_decode<D>(B, L, cb);
            R lag = R(1);
            int tk[DMAX], tt = t;
#pragma unroll
            for (int j = 0; j < D; ++j) { tk[j] = tt % Q; tt /= Q; lag *= a.lsrc[tk[j]]; }
            int64_t flat = 0;
#pragma unroll
            for (int j = 0; j < D; ++j) flat = (flat << L) + cb[j];
            const C gv = a.g[(int64_t)rhs * a.npts + flat];
            const int pslot[DMAX] = {Q + 1, Q + 1, Q + 1};
            const C e1 = expphase<P, D, K>(a, tX, spoint<P, D, Q, K>(a, 0, cb, pslot));
            const C e0 = expphase<P, D, K>(a, tX, spoint<P, D, Q, K>(a, 0, cb, tk));
            C v = cjmul(e0, cmul(e1, gv));
            C out;
            out.x = lag * v.x;
            out.y = lag * v.y;
            Wt[pr * RR + t] = out;
        }
    }

    // block beta of tile level i: target box index at level l (for the row form, the parent)
    // and source box index at level l+1; base slot of the block
    static __device__ __forceinline__ void block_geo(uint32_t Ap, uint32_t Bstar, int beta, int i, int k,
                                                     uint32_t &Apg, uint32_t &Bq, int &base)
    {
        const uint32_t ra = beta & ((1u << (D * i)) - 1);
        const uint32_t bp = beta >> (D * i);
        base = (bp << (D * (i + 1))) + ra;
        Apg = (Ap << (D * i)) + digit_rev<D>(ra, i);
        Bq = (Bstar << (D * (k - i - 1))) + bp;
    }

    // acc += M[h][t][u] v in the column levels and the first stage of the row levels.  d = 2:
    // two scalar FMAs, the coefficient a kernel-parameter operand (a packed FMA needs the
    // duplicated pair M2 in registers first; at N = 1024, q = 5 the column passes 1% and the
    // row passes 1% faster); d = 3 and the row levels' second stage, whose coefficient index
    // is not a compile-time constant, keep the packed form, which measured 0.5-2% faster
    // there.  The same roundings either way.
    static __device__ __forceinline__ void imac(C &acc, const KArgs<P> &a, int h, int t, int u, C v)
    {
        if constexpr (D == 2)
            cfma(acc, a.M[h][t][u], v);
        else
            cfma2(acc, a.M2[h][t][u], v);
    }

    // ---- one column-form merge level (l -> l+1) on all tiles of the CTA
    template <int PM = PM_COMPUTE>
    static __device__ void col_level(const KArgs<P> &a, C *Wt, C *S, Geo *G, int l, int i, float *&tb)
    {
        const int k = a.k, n = 1 << (D * k), nblk = n >> D;
        const int L = a.L;
        FT fa{tb, n_col_a(a)}, fb{tb, n_col_b(a)};
        if constexpr (PM != PM_COMPUTE) {
            fb.p = tb + (int64_t)fa.n * PH_COL_A;
            tb = fb.p + (int64_t)fb.n * PH_COL_B;
        }
        // the output pairs (tau, block, alpha) of this level: box centre (level l+1), parent source box
        for (int j = threadIdx.x; j < a.T * n; j += blockDim.x) {
            const int alpha = j & (NC - 1), beta = (j >> D) & (nblk - 1), tau = (j >> D) >> (D * (k - 1));
            uint32_t Ap, Bstar, Apg, Bq;
            int base;
            tile_of(a, tau, Ap, Bstar);
            block_geo(Ap, Bstar, beta, i, k, Apg, Bq, base);
            const uint32_t Aa = (Apg << D) + alpha;
            int ca[DMAX], cbq[DMAX];
            morton_decode<D>(Aa, l + 1, ca);
            morton_decode<D>(Bq, L - l - 1, cbq);
            Geo &g = G[j];
#pragma unroll
            for (int q = 0; q < D; ++q) g.cbq[q] = cbq[q];
            g.base = base;
            if constexpr (PM != PM_TABLE) g.tA = tcenter<P, D, Q, K>(a, l + 1, Aa, ca);
        }
        __syncthreads();
        // stage A: items (tau, block, alpha, c_{D-1}, t'_{D-1}): modulate and contract dims 0..D-2
        for (int it = threadIdx.x; it < a.T * nblk * NC * 2 * Q; it += blockDim.x) {
            const int tq = it % Q;
            const int chi = (it / Q) & 1;
            const int alpha = (it / (2 * Q)) % NC;
            const int beta = (it / (2 * Q * NC)) & (nblk - 1);
            const int tau = (it / (2 * Q * NC)) >> (D * (k - 1));
            const Geo &g = G[(tau * nblk + beta) * NC + alpha];
            const int base = g.base;
            int cbq[DMAX];
#pragma unroll
            for (int q = 0; q < D; ++q) cbq[q] = g.cbq[q];
            const typename PH::T tA = g.tA;
            const C *Wtau = Wt + tau * n * RR;
            C acc[QD1];
#pragma unroll
            for (int j = 0; j < QD1; ++j) acc[j] = czero<C>();
#pragma unroll
            for (int cl = 0; cl < (NC >> 1); ++cl) {
                const int c = cl | (chi << (D - 1));
                const C *win = Wtau + (base + (c << (D * i))) * RR;
                int cb[DMAX];
#pragma unroll
                for (int j = 0; j < D; ++j) cb[j] = 2 * cbq[j] + ((c >> j) & 1);
                typename PH::S sp;
                PH::src1(sp, D - 1, sget<P, Q>(a, D - 1, l, cb[D - 1], tq));
                if constexpr (D == 2 && !P::is_f64) {
                    // phases two at a time: lanes t'_0 and t'_0 + 1 (the last one alone for odd q)
                    using PH2 = Ph2<P, D, K>;
                    const int c0 = c & 1;
                    const typename PH2::T tA2 = PH2::dup(tA);
                    const typename P::SE e1 = sget<P, Q>(a, 1, l, cb[1], tq);
                    const typename PH2::Part p1 = PH2::part(tA2, e1, e1, 1);
#pragma unroll
                    for (int t0p = 0; t0p + 1 < Q; t0p += 2) {
                        float2 E0, E1;
                        ph2<PM>(a, tA2,
                                PH2::add(PH2::part(tA2, sget<P, Q>(a, 0, l, cb[0], t0p), sget<P, Q>(a, 0, l, cb[0], t0p + 1), 0), p1),
                                fa.at(cl * Q + t0p, it), fa.at(cl * Q + t0p + 1, it), E0, E1);
                        const C u0 = cmul(E0, win[t0p + Q * tq]), u1 = cmul(E1, win[t0p + 1 + Q * tq]);
#pragma unroll
                        for (int t0 = 0; t0 < Q; ++t0) {
                            imac(acc[t0], a, c0, t0, t0p, u0);
                            imac(acc[t0], a, c0, t0, t0p + 1, u1);
                        }
                    }
                    if constexpr (Q & 1) {
                        const typename PH::Part pt = PH::add(PH::part(tA, sget<P, Q>(a, 0, l, cb[0], Q - 1), 0), PH2::lane0(p1));
                        const C u = cmul(ph<PM>(a, tA, pt, fa.at(cl * Q + Q - 1, it)), win[Q - 1 + Q * tq]);
#pragma unroll
                        for (int t0 = 0; t0 < Q; ++t0) imac(acc[t0], a, c0, t0, Q - 1, u);
                    }
                } else if constexpr (D == 2) {
                    const int c0 = c & 1;
                    const typename PH::Part p1 = PH::part(tA, sget<P, Q>(a, 1, l, cb[1], tq), 1);
#pragma unroll
                    for (int t0p = 0; t0p < Q; ++t0p) {
                        const typename PH::Part pt = PH::add(PH::part(tA, sget<P, Q>(a, 0, l, cb[0], t0p), 0), p1);
                        const C u = cmul(expphase_part<P, D, K>(a, tA, pt), win[t0p + Q * tq]);
#pragma unroll
                        for (int t0 = 0; t0 < Q; ++t0) imac(acc[t0], a, c0, t0, t0p, u);
                    }
                } else if constexpr (!P::is_f64) {
                    // d = 3: the parts of coordinates 2 and 1 hoisted, phases two at a time over t'_0
                    using PH2 = Ph2<P, D, K>;
                    const int c0 = c & 1, c1 = (c >> 1) & 1;
                    const typename PH2::T tA2 = PH2::dup(tA);
                    const typename P::SE e2 = sget<P, Q>(a, 2, l, cb[2], tq);
                    const typename PH2::Part p2 = PH2::part(tA2, e2, e2, 2);
#pragma unroll
                    for (int t1p = 0; t1p < Q; ++t1p) {
                        const typename P::SE e1 = sget<P, Q>(a, 1, l, cb[1], t1p);
                        const typename PH2::Part p12 = PH2::add(PH2::part(tA2, e1, e1, 1), p2);
                        const C *wrow = win + Q * t1p + Q * Q * tq;
                        C tmp[Q];
#pragma unroll
                        for (int t0 = 0; t0 < Q; ++t0) tmp[t0] = czero<C>();
#pragma unroll
                        for (int t0p = 0; t0p + 1 < Q; t0p += 2) {
                            float2 E0, E1;
                            ph2<PM>(a, tA2,
                                    PH2::add(PH2::part(tA2, sget<P, Q>(a, 0, l, cb[0], t0p),
                                                       sget<P, Q>(a, 0, l, cb[0], t0p + 1), 0), p12),
                                    fa.at((cl * Q + t1p) * Q + t0p, it), fa.at((cl * Q + t1p) * Q + t0p + 1, it), E0, E1);
                            const C u0 = cmul(E0, wrow[t0p]), u1 = cmul(E1, wrow[t0p + 1]);
#pragma unroll
                            for (int t0 = 0; t0 < Q; ++t0) {
                                imac(tmp[t0], a, c0, t0, t0p, u0);
                                imac(tmp[t0], a, c0, t0, t0p + 1, u1);
                            }
                        }
                        if constexpr (Q & 1) {
                            const typename PH::Part pt = PH::add(PH::part(tA, sget<P, Q>(a, 0, l, cb[0], Q - 1), 0), PH2::lane0(p12));
                            const C u = cmul(ph<PM>(a, tA, pt, fa.at((cl * Q + t1p) * Q + Q - 1, it)), wrow[Q - 1]);
#pragma unroll
                            for (int t0 = 0; t0 < Q; ++t0) imac(tmp[t0], a, c0, t0, Q - 1, u);
                        }
#pragma unroll
                        for (int t1 = 0; t1 < Q; ++t1)
#pragma unroll
                            for (int t0 = 0; t0 < Q; ++t0) imac(acc[t0 + Q * t1], a, c1, t1, t1p, tmp[t0]);
                    }
                } else {
                    const int c0 = c & 1, c1 = (c >> 1) & 1;
#pragma unroll
                    for (int t1p = 0; t1p < Q; ++t1p) {
                        PH::src1(sp, 1, sget<P, Q>(a, 1, l, cb[1], t1p));
                        C tmp[Q];
#pragma unroll
                        for (int t0 = 0; t0 < Q; ++t0) tmp[t0] = czero<C>();
#pragma unroll
                        for (int t0p = 0; t0p < Q; ++t0p) {
                            PH::src1(sp, 0, sget<P, Q>(a, 0, l, cb[0], t0p));
                            const C u = cmul(expphase<P, D, K>(a, tA, sp), win[t0p + Q * t1p + Q * Q * tq]);
#pragma unroll
                            for (int t0 = 0; t0 < Q; ++t0) imac(tmp[t0], a, c0, t0, t0p, u);
                        }
#pragma unroll
                        for (int t1 = 0; t1 < Q; ++t1)
#pragma unroll
                            for (int t0 = 0; t0 < Q; ++t0) imac(acc[t0 + Q * t1], a, c1, t1, t1p, tmp[t0]);
                    }
                }
            }
            // scratch [tau][block][alpha][c_{D-1}][t'_{D-1}][t_{<D-1}]
            C *so = S + ((((tau * nblk + beta) * NC + alpha) * 2 + chi) * Q + tq) * QD1;
#pragma unroll
            for (int j = 0; j < QD1; ++j) so[j] = acc[j];
        }
        __syncthreads();
        // stage B: items (tau, block, alpha, t_{<D-1}): contract dim D-1 and c_{D-1}, demodulate
        for (int it = threadIdx.x; it < a.T * nblk * NC * QD1; it += blockDim.x) {
            const int tl = it % QD1;
            const int alpha = (it / QD1) % NC;
            const int beta = (it / (QD1 * NC)) & (nblk - 1);
            const int tau = (it / (QD1 * NC)) >> (D * (k - 1));
            const Geo &g = G[(tau * nblk + beta) * NC + alpha];
            const int base = g.base;
            int cbq[DMAX];
#pragma unroll
            for (int q = 0; q < D; ++q) cbq[q] = g.cbq[q];
            const typename PH::T tA = g.tA;
            C acc[Q];
#pragma unroll
            for (int j = 0; j < Q; ++j) acc[j] = czero<C>();
#pragma unroll
            for (int chi = 0; chi < 2; ++chi) {
                const C *si = S + ((((tau * nblk + beta) * NC + alpha) * 2 + chi) * Q) * QD1 + tl;
#pragma unroll
                for (int tqp = 0; tqp < Q; ++tqp) {
                    const C v = si[tqp * QD1];
#pragma unroll
                    for (int tq = 0; tq < Q; ++tq) imac(acc[tq], a, chi, tq, tqp, v);
                }
            }
            int tk[DMAX];
            {
                int tt = tl;
#pragma unroll
                for (int j = 0; j < D - 1; ++j) { tk[j] = tt % Q; tt /= Q; }
            }
            typename PH::Part pl = PH::part(tA, sget<P, Q>(a, 0, l + 1, cbq[0], tk[0]), 0);
            if constexpr (D == 3) pl = PH::add(pl, PH::part(tA, sget<P, Q>(a, 1, l + 1, cbq[1], tk[1]), 1));
            C *wo = Wt + tau * n * RR + (base + (alpha << (D * i))) * RR + tl;
            if constexpr (!P::is_f64) {
                // phases two at a time: lanes t_{d-1} and t_{d-1} + 1 (the last one alone for odd q)
                using PH2 = Ph2<P, D, K>;
                const typename PH2::T tA2 = PH2::dup(tA);
                const typename PH2::Part pl2 = PH2::dup(pl);
#pragma unroll
                for (int tq = 0; tq + 1 < Q; tq += 2) {
                    float2 E0, E1;
                    ph2<PM>(a, tA2,
                            PH2::add(PH2::part(tA2, sget<P, Q>(a, D - 1, l + 1, cbq[D - 1], tq),
                                               sget<P, Q>(a, D - 1, l + 1, cbq[D - 1], tq + 1), D - 1), pl2),
                            fb.at(tq, it), fb.at(tq + 1, it), E0, E1);
                    wo[tq * QD1] = cjmul(E0, acc[tq]);
                    wo[(tq + 1) * QD1] = cjmul(E1, acc[tq + 1]);
                }
                if constexpr (Q & 1) {
                    const typename PH::Part pt = PH::add(PH::part(tA, sget<P, Q>(a, D - 1, l + 1, cbq[D - 1], Q - 1), D - 1), pl);
                    wo[(Q - 1) * QD1] = cjmul(ph<PM>(a, tA, pt, fb.at(Q - 1, it)), acc[Q - 1]);
                }
            } else {
#pragma unroll
                for (int tq = 0; tq < Q; ++tq) {
                    const typename PH::Part pt = PH::add(PH::part(tA, sget<P, Q>(a, D - 1, l + 1, cbq[D - 1], tq), D - 1), pl);
                    wo[tq * QD1] = cjmul(expphase_part<P, D, K>(a, tA, pt), acc[tq]);
                }
            }
        }
        __syncthreads();
    }

    // ---- switch at level l on every pair (slots in digit-reversed order); items (tau, slot, s_{>=1})
    // accumulate over t for the q values of s_0.  Results go through S so no item reads a
    // slot that another item has already rewritten.
    template <int PM = PM_COMPUTE>
    static __device__ void switch_tiles(const KArgs<P> &a, C *Wt, C *S, int l, float *&tb)
    {
        if constexpr (!P::is_f64 && K == KIND_GENRADON) {   // the phase whose pairs pay for their registers
            switch_tiles_pair<PM>(a, Wt, S, l, tb);
            return;
        }
        const FT fs{tb, n_switch(a)};   // phase (th q + t_0) q + s_0 of an item
        if constexpr (PM != PM_COMPUTE) tb += (int64_t)fs.n * PH_SWITCH;
        const int k = a.k, n = 1 << (D * k);
        const int L = a.L;
        for (int it = threadIdx.x; it < a.T * n * QD1; it += blockDim.x) {
            const int sh = it % QD1;
            const int sl = (it / QD1) & (n - 1);
            const int tau = (it / QD1) >> (D * k);
            uint32_t Ap, Bstar;
            tile_of(a, tau, Ap, Bstar);
            const uint32_t A = (Ap << (D * k)) + digit_rev<D>(sl, k);
            int ca[DMAX], cb[DMAX];
            morton_decode<D>(A, l, ca);
            morton_decode<D>(Bstar, L - l, cb);
            typename PH::T tS[Q];
            C acc[Q];
            int sk[DMAX];
            {
                int tt = sh;
#pragma unroll
                for (int j = 1; j < D; ++j) { sk[j] = tt % Q; tt /= Q; }
            }
#pragma unroll
            for (int s0 = 0; s0 < Q; ++s0) {
                sk[0] = s0;
                tS[s0] = tpoint<P, D, Q, K>(a, l, ca, sk);
                acc[s0] = czero<C>();
            }
            const C *u = Wt + (tau * n + sl) * RR;
            // t = t_0 + q t_{>=1}: the parts of coordinates >= 1 are fixed over the t_0 loop
#pragma unroll 1
            for (int th = 0; th < QD1; ++th) {
                int tk[DMAX], tt = th;
#pragma unroll
                for (int j = 1; j < D; ++j) { tk[j] = tt % Q; tt /= Q; }
                typename PH::Part hp[Q];
#pragma unroll
                for (int s0 = 0; s0 < Q; ++s0) {
                    hp[s0] = PH::part(tS[s0], sget<P, Q>(a, 1, l, cb[1], tk[1]), 1);
                    if constexpr (D == 3) hp[s0] = PH::add(hp[s0], PH::part(tS[s0], sget<P, Q>(a, 2, l, cb[2], tk[2]), 2));
                }
#pragma unroll
                for (int t0 = 0; t0 < Q; ++t0) {
                    const typename P::SE e0 = sget<P, Q>(a, 0, l, cb[0], t0);
                    const C ut = u[t0 + Q * th];
#pragma unroll
                    for (int s0 = 0; s0 < Q; ++s0)
                        cmac(acc[s0], ph<PM>(a, tS[s0], PH::add(PH::part(tS[s0], e0, 0), hp[s0]), fs.at((th * Q + t0) * Q + s0, it)), ut);
                }
            }
            C *w = S + (tau * n + sl) * RR + sh * Q;
#pragma unroll
            for (int s0 = 0; s0 < Q; ++s0) w[s0] = acc[s0];
        }
        __syncthreads();
        for (int j = threadIdx.x; j < a.T * n * RR; j += blockDim.x) Wt[j] = S[j];
        __syncthreads();
    }

    // ---- the same switch with the phases evaluated two at a time (lanes of a float2):
    // targets s_0 = 2j and 2j + 1 share a pair; for odd q the last target takes two
    // consecutive t_0 in its lanes.  Each lane rounds exactly as the scalar code.
    template <int PM>
    static __device__ void switch_tiles_pair(const KArgs<P> &a, C *Wt, C *S, int l, float *&tb)
    {
        using PH2 = Ph2<P, D, K>;
        constexpr int NPR = Q / 2, ODD = Q & 1, NT2 = NPR + ODD;
        const FT fs{tb, n_switch(a)};   // phase (th q + t_0) q + s_0 of an item
        if constexpr (PM != PM_COMPUTE) tb += (int64_t)fs.n * PH_SWITCH;
        const int k = a.k, n = 1 << (D * k);
        const int L = a.L;
        for (int it = threadIdx.x; it < a.T * n * QD1; it += blockDim.x) {
            const int sh = it % QD1;
            const int sl = (it / QD1) & (n - 1);
            const int tau = (it / QD1) >> (D * k);
            uint32_t Ap, Bstar;
            tile_of(a, tau, Ap, Bstar);
            const uint32_t A = (Ap << (D * k)) + digit_rev<D>(sl, k);
            int ca[DMAX], cb[DMAX];
            morton_decode<D>(A, l, ca);
            morton_decode<D>(Bstar, L - l, cb);
            typename PH2::T tP[NT2];
            C acc[Q];
            int sk[DMAX];
            {
                int tt = sh;
#pragma unroll
                for (int j = 1; j < D; ++j) { sk[j] = tt % Q; tt /= Q; }
            }
#pragma unroll
            for (int j = 0; j < NT2; ++j) {
                sk[0] = 2 * j;
                const typename PH::T t0 = tpoint<P, D, Q, K>(a, l, ca, sk);
                sk[0] = (2 * j + 1 < Q) ? 2 * j + 1 : 2 * j;
                tP[j] = PH2::pair(t0, tpoint<P, D, Q, K>(a, l, ca, sk));
            }
#pragma unroll
            for (int s0 = 0; s0 < Q; ++s0) acc[s0] = czero<C>();
            const C *u = Wt + (tau * n + sl) * RR;
#pragma unroll 1
            for (int th = 0; th < QD1; ++th) {
                int tk[DMAX], tt = th;
#pragma unroll
                for (int j = 1; j < D; ++j) { tk[j] = tt % Q; tt /= Q; }
                typename PH2::Part hp[NT2];
                const typename P::SE e1 = sget<P, Q>(a, 1, l, cb[1], tk[1]);
#pragma unroll
                for (int j = 0; j < NT2; ++j) {
                    hp[j] = PH2::part(tP[j], e1, e1, 1);
                    if constexpr (D == 3) {
                        const typename P::SE e2 = sget<P, Q>(a, 2, l, cb[2], tk[2]);
                        hp[j] = PH2::add(hp[j], PH2::part(tP[j], e2, e2, 2));
                    }
                }
#pragma unroll
                for (int t0 = 0; t0 < Q; t0 += 2) {
                    const bool two = t0 + 1 < Q;
                    const typename P::SE ea = sget<P, Q>(a, 0, l, cb[0], t0);
                    const typename P::SE eb = two ? sget<P, Q>(a, 0, l, cb[0], t0 + 1) : ea;
                    const C ua = u[t0 + Q * th];
                    const C ub = two ? u[t0 + 1 + Q * th] : czero<C>();
                    float2 E0, E1;
                    const int ja = (th * Q + t0) * Q, jb = ja + Q;
#pragma unroll
                    for (int j = 0; j < NPR; ++j) {
                        ph2<PM>(a, tP[j], PH2::add(PH2::part(tP[j], ea, ea, 0), hp[j]), fs.at(ja + 2 * j, it),
                                fs.at(ja + 2 * j + 1, it), E0, E1);
                        cmac(acc[2 * j], E0, ua);
                        cmac(acc[2 * j + 1], E1, ua);
                        if (two) {
                            ph2<PM>(a, tP[j], PH2::add(PH2::part(tP[j], eb, eb, 0), hp[j]), fs.at(jb + 2 * j, it),
                                    fs.at(jb + 2 * j + 1, it), E0, E1);
                            cmac(acc[2 * j], E0, ub);
                            cmac(acc[2 * j + 1], E1, ub);
                        }
                    }
                    if constexpr (ODD) {
                        ph2<PM>(a, tP[NPR], PH2::add(PH2::part(tP[NPR], ea, eb, 0), hp[NPR]), fs.at(ja + Q - 1, it),
                                two ? fs.at(jb + Q - 1, it) : nullptr, E0, E1);
                        cmac(acc[Q - 1], E0, ua);
                        if (two) cmac(acc[Q - 1], E1, ub);
                    }
                }
            }
            C *w = S + (tau * n + sl) * RR + sh * Q;
#pragma unroll
            for (int s0 = 0; s0 < Q; ++s0) w[s0] = acc[s0];
        }
        __syncthreads();
        for (int j = threadIdx.x; j < a.T * n * RR; j += blockDim.x) Wt[j] = S[j];
        __syncthreads();
    }

    // ---- switch for a phase that is a sum over dimensions, Phi = sum_k phi_k(x_k, y_k)
    // (Fourier, and the separable test phase): e^{2pi i Phi(x_s, y_t)} is the product of the
    // d factors e^{2pi i phi_k(x_{s_k}, y_{t_k})}, so the r x r switch is d sweeps of q x q
    // matrices, one per node digit -- O(d q^{d+1}) work per pair instead of O(r^2) (the
    // tensor-product case of Section 1.4).  ADJ applies the conjugate transpose (each sweep
    // conjugate-transposed; the sweeps commute).  Items (tau, slot, output digit, D-2 other
    // digits); each evaluates its q phases once and sweeps the last digit.  Results go
    // Wt -> S -> Wt (-> S, copied back for odd d).
    template <bool ADJ>
    static __device__ void switch_sep(const KArgs<P> &a, C *Wt, C *S, int l)
    {
        const int k = a.k, n = 1 << (D * k);
        const int L = a.L;
        C *src = Wt, *dst = S;
#pragma unroll
        for (int dim = 0; dim < D; ++dim) {
            int oth[DMAX - 1];
            {
                int j = 0;
#pragma unroll
                for (int e = 0; e < D; ++e)
                    if (e != dim) oth[j++] = e;
            }
            int pw[DMAX];
            pw[0] = 1;
#pragma unroll
            for (int e = 1; e < D; ++e) pw[e] = pw[e - 1] * Q;
            for (int it = threadIdx.x; it < a.T * n * QD1; it += blockDim.x) {
                const int rest = it % QD1;
                const int sl = (it / QD1) & (n - 1);
                const int tau = (it / QD1) >> (D * k);
                uint32_t Ap, Bstar;
                tile_of(a, tau, Ap, Bstar);
                const uint32_t A = (Ap << (D * k)) + digit_rev<D>(sl, k);
                int ca[DMAX], cb[DMAX];
                morton_decode<D>(A, l, ca);
                morton_decode<D>(Bstar, L - l, cb);
                const int sd = rest % Q;                        // output digit of dimension dim
                const int o1 = D == 3 ? rest / Q : 0;            // digit of oth[0] (d = 3)
                C e[Q];
                if constexpr (!ADJ) {
                    int sk[DMAX] = {Q, Q, Q};
                    sk[dim] = sd;
                    const typename PH::T tS = tpoint<P, D, Q, K>(a, l, ca, sk);
#pragma unroll
                    for (int u = 0; u < Q; ++u)
                        e[u] = expphase_part<P, D, K>(a, tS, PH::part(tS, sget<P, Q>(a, dim, l, cb[dim], u), dim));
                } else {
                    const typename P::SE ys = sget<P, Q>(a, dim, l, cb[dim], sd);
#pragma unroll
                    for (int u = 0; u < Q; ++u) {
                        int sk[DMAX] = {Q, Q, Q};
                        sk[dim] = u;
                        const typename PH::T tS = tpoint<P, D, Q, K>(a, l, ca, sk);
                        e[u] = expphase_part<P, D, K>(a, tS, PH::part(tS, ys, dim));
                    }
                }
                const int base = (tau * n + sl) * RR + (D == 3 ? o1 * pw[oth[0]] : 0);
                const int last = oth[D - 2];
                const C *in = src + base;
                C *out = dst + base;
#pragma unroll 1
                for (int oi = 0; oi < Q; ++oi) {
                    const int off = oi * pw[last];
                    C acc = czero<C>();
#pragma unroll
                    for (int u = 0; u < Q; ++u) {
                        const C v = in[off + u * pw[dim]];
                        if constexpr (ADJ)
                            acc = cadd(acc, cjmul(e[u], v));
                        else
                            cmac(acc, e[u], v);
                    }
                    out[off + sd * pw[dim]] = acc;
                }
            }
            __syncthreads();
            C *t = src;
            src = dst;
            dst = t;
        }
        if (src != Wt) {
            for (int j = threadIdx.x; j < a.T * n * RR; j += blockDim.x) Wt[j] = src[j];
            __syncthreads();
        }
    }

    // ---- one row-form merge level (l -> l+1) on all tiles of the CTA.  TC caches the
    // target features of the parents' nodes (T * 2^{Di} boxes x q^d nodes) for stage A.
    template <int PM = PM_COMPUTE>
    static __device__ void row_level(const KArgs<P> &a, C *Wt, C *S, typename PH::T *TC, int l, int i, float *&tb)
    {
        const int k = a.k, n = 1 << (D * k), nblk = n >> D;
        const int L = a.L;
        const int nbox = 1 << (D * i);
        FT fa{tb, n_row_a(a)}, fb{tb, n_row_b(a)};
        if constexpr (PM != PM_COMPUTE) {
            fb.p = tb + (int64_t)fa.n * PH_ROW_A;
            tb = fb.p + (int64_t)fb.n * PH_ROW_B;
        }
        for (int j = threadIdx.x; PM != PM_TABLE && j < a.T * nbox * RR; j += blockDim.x) {
            const int t = j % RR, aloc = (j / RR) & (nbox - 1), tau = (j / RR) >> (D * i);
            uint32_t Ap, Bstar;
            tile_of(a, tau, Ap, Bstar);
            int ca[DMAX], tk[DMAX], tt = t;
            morton_decode<D>((Ap << (D * i)) + aloc, l, ca);
#pragma unroll
            for (int jj = 0; jj < D; ++jj) { tk[jj] = tt % Q; tt /= Q; }
            TC[j] = tpoint<P, D, Q, K>(a, l, ca, tk);
        }
        __syncthreads();
        // stage A: items (tau, block, c, t_{>=1}): pre-modulate input c at the nodes of the
        // parent target box and contract dim 0 for both children alpha_0
        //   -> S[tau][block][c][t_{>=1}][alpha_0][s_0]
        for (int it = threadIdx.x; it < a.T * nblk * NC * QD1; it += blockDim.x) {
            const int th = it % QD1;
            const int c = (it / QD1) % NC;
            const int beta = (it / (QD1 * NC)) & (nblk - 1);
            const int tau = (it / (QD1 * NC)) >> (D * (k - 1));
            uint32_t Ap, Bstar, Apg, Bq;
            int base;
            tile_of(a, tau, Ap, Bstar);
            block_geo(Ap, Bstar, beta, i, k, Apg, Bq, base);
            int cbq[DMAX], cb[DMAX];
            morton_decode<D>(Bq, L - l - 1, cbq);
#pragma unroll
            for (int j = 0; j < D; ++j) cb[j] = 2 * cbq[j] + ((c >> j) & 1);
            const int ctr[DMAX] = {Q, Q, Q};
            const typename PH::S sc = spoint<P, D, Q, K>(a, l, cb, ctr);
            const typename PH::T *tn = TC + (tau * nbox + (int)digit_rev<D>(beta & (nbox - 1), i)) * RR + th * Q;
            const C *win = Wt + tau * n * RR + (base + (c << (D * i))) * RR + th * Q;
            C z[2][Q];
#pragma unroll
            for (int s0 = 0; s0 < Q; ++s0) { z[0][s0] = czero<C>(); z[1][s0] = czero<C>(); }
#pragma unroll
            for (int t0 = 0; t0 < Q; ++t0) {
                const C u = cjmul(phs<PM>(a, tn[t0], sc, fa.at(t0, it)), win[t0]);
#pragma unroll
                for (int s0 = 0; s0 < Q; ++s0) {
                    imac(z[0][s0], a, 0, t0, s0, u);
                    imac(z[1][s0], a, 1, t0, s0, u);
                }
            }
            C *so = S + (((tau * nblk + beta) * NC + c) * QD1 + th) * 2 * Q;
#pragma unroll
            for (int s0 = 0; s0 < Q; ++s0) { so[s0] = z[0][s0]; so[Q + s0] = z[1][s0]; }
        }
        __syncthreads();
        // stage B: items (tau, block, alpha, s_0): contract dims >= 1 per child c,
        // post-modulate at the child's nodes, sum over c
        for (int it = threadIdx.x; it < a.T * nblk * NC * Q; it += blockDim.x) {
            const int s0 = it % Q;
            const int alpha = (it / Q) % NC;
            const int beta = (it / (Q * NC)) & (nblk - 1);
            const int tau = (it / (Q * NC)) >> (D * (k - 1));
            uint32_t Ap, Bstar, Apg, Bq;
            int base;
            tile_of(a, tau, Ap, Bstar);
            block_geo(Ap, Bstar, beta, i, k, Apg, Bq, base);
            const uint32_t Aa = (Apg << D) + alpha;                      // level l+1
            int ca[DMAX], cbq[DMAX];
            morton_decode<D>(Aa, l + 1, ca);
            morton_decode<D>(Bq, L - l - 1, cbq);
            const int a0 = alpha & 1;
            const C *Sblk = S + ((tau * nblk + beta) * NC) * QD1 * 2 * Q;
            C acc[QD1];
#pragma unroll
            for (int j = 0; j < QD1; ++j) acc[j] = czero<C>();
            if constexpr (D == 2) {
                const int a1 = (alpha >> 1) & 1;
                C v[NC][Q];
                typename P::SE sc0[2], sc1[2];        // children's centres per dimension
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    sc0[h] = sget<P, Q>(a, 0, l, 2 * cbq[0] + h, Q);
                    sc1[h] = sget<P, Q>(a, 1, l, 2 * cbq[1] + h, Q);
                }
#pragma unroll
                for (int c = 0; c < NC; ++c) {
                    const C *si = Sblk + c * QD1 * 2 * Q + a0 * Q + s0;   // [t1] stride 2Q
#pragma unroll
                    for (int s1 = 0; s1 < Q; ++s1) v[c][s1] = czero<C>();
#pragma unroll
                    for (int t1 = 0; t1 < Q; ++t1) {
                        const C zz = si[t1 * 2 * Q];
#pragma unroll
                        for (int s1 = 0; s1 < Q; ++s1) cfma2(v[c][s1], a.M2[a1][t1][s1], zz);
                    }
                }
#pragma unroll
                for (int s1 = 0; s1 < Q; ++s1) {
                    const int sk[DMAX] = {s0, s1, 0};
                    const typename PH::T tS = tpoint<P, D, Q, K>(a, l + 1, ca, sk);
                    if constexpr (!P::is_f64) {
                        // phases two at a time: lanes c_0 = 0 and 1
                        using PH2 = Ph2<P, D, K>;
                        const typename PH2::T tS2 = PH2::dup(tS);
                        const typename PH2::Part q0 = PH2::part(tS2, sc0[0], sc0[1], 0);
#pragma unroll
                        for (int c1 = 0; c1 < 2; ++c1) {
                            float2 E0, E1;
                            ph2<PM>(a, tS2, PH2::add(q0, PH2::part(tS2, sc1[c1], sc1[c1], 1)), fb.at(s1 * NC + 2 * c1, it),
                                    fb.at(s1 * NC + 2 * c1 + 1, it), E0, E1);
                            acc[s1] = cadd(acc[s1], cmul(E0, v[2 * c1][s1]));
                            acc[s1] = cadd(acc[s1], cmul(E1, v[2 * c1 + 1][s1]));
                        }
                    } else {
                        const typename PH::Part q0[2] = {PH::part(tS, sc0[0], 0), PH::part(tS, sc0[1], 0)};
                        const typename PH::Part q1[2] = {PH::part(tS, sc1[0], 1), PH::part(tS, sc1[1], 1)};
#pragma unroll
                        for (int c = 0; c < NC; ++c)
                            acc[s1] = cadd(acc[s1], cmul(expphase_part<P, D, K>(a, tS, PH::add(q0[c & 1], q1[c >> 1])), v[c][s1]));
                    }
                }
            } else {
                const int a1 = (alpha >> 1) & 1, a2 = (alpha >> 2) & 1;
#pragma unroll 1
                for (int c = 0; c < NC; ++c) {
                    int cb[DMAX], ctr[DMAX] = {Q, Q, Q};
#pragma unroll
                    for (int j = 0; j < D; ++j) cb[j] = 2 * cbq[j] + ((c >> j) & 1);
                    const typename PH::S sc = spoint<P, D, Q, K>(a, l, cb, ctr);
                    const C *si = Sblk + c * QD1 * 2 * Q + a0 * Q + s0;   // [t1 + Q t2] stride 2Q
                    C w[Q * Q];   // [t1][s2]
#pragma unroll
                    for (int j = 0; j < Q * Q; ++j) w[j] = czero<C>();
#pragma unroll
                    for (int t2 = 0; t2 < Q; ++t2)
#pragma unroll
                        for (int t1 = 0; t1 < Q; ++t1) {
                            const C zz = si[(t1 + Q * t2) * 2 * Q];
#pragma unroll
                            for (int s2 = 0; s2 < Q; ++s2) cfma2(w[t1 * Q + s2], a.M2[a2][t2][s2], zz);
                        }
#pragma unroll
                    for (int s2 = 0; s2 < Q; ++s2)
#pragma unroll
                        for (int s1 = 0; s1 < Q; ++s1) {
                            C v = czero<C>();
#pragma unroll
                            for (int t1 = 0; t1 < Q; ++t1) cfma2(v, a.M2[a1][t1][s1], w[t1 * Q + s2]);
                            const int sk[DMAX] = {s0, s1, s2};
                            const typename PH::T tS = tpoint<P, D, Q, K>(a, l + 1, ca, sk);
                            acc[s1 + Q * s2] = cadd(acc[s1 + Q * s2], cmul(phs<PM>(a, tS, sc, fb.at((s1 + Q * s2) * NC + c, it)), v));
                        }
                }
            }
            C *wo = Wt + tau * n * RR + (base + (alpha << (D * i))) * RR + s0;
#pragma unroll
            for (int sh = 0; sh < QD1; ++sh) wo[sh * Q] = acc[sh];
        }
        __syncthreads();
    }

    // ---- final evaluation of the leaf targets (pairs (A, Y) at level L); items (tau, slot)
    static __device__ void final_eval(const KArgs<P> &a, const C *Wt, int rhs)
    {
        const int k = a.k, n = 1 << (D * k);
        const int L = a.L;
        const int cY[DMAX] = {0, 0, 0};
        const int ctr[DMAX] = {Q, Q, Q};
        const typename PH::S sY = spoint<P, D, Q, K>(a, L, cY, ctr);      // centre of Y
        for (int it = threadIdx.x; it < a.T * n; it += blockDim.x) {
            const int sl = it & (n - 1), tau = it >> (D * k);
            uint32_t Ap, Bstar;
            tile_of(a, tau, Ap, Bstar);
            const uint32_t A = (Ap << (D * k)) + digit_rev<D>(sl, k);
            int ca[DMAX];
            morton_decode<D>(A, L, ca);
            const C *w = Wt + it * RR;
            C acc = czero<C>();
            for (int t = 0; t < RR; ++t) {
                R lag = R(1);
                int tk[DMAX], tt = t;
#pragma unroll
                for (int j = 0; j < D; ++j) { tk[j] = tt % Q; tt /= Q; lag *= a.ltgt[tk[j]]; }
                if (lag == R(0)) continue;
                const C e = expphase<P, D, K>(a, tpoint<P, D, Q, K>(a, L, ca, tk), sY);
                cfma(acc, lag, cjmul(e, w[t]));
            }
            const int pslot[DMAX] = {Q + 1, Q + 1, Q + 1};
            const C e = expphase<P, D, K>(a, tpoint<P, D, Q, K>(a, L, ca, pslot), sY);
            int64_t flat = 0;
#pragma unroll
            for (int j = 0; j < D; ++j) flat = (flat << L) + ca[j];
            a.f[(int64_t)rhs * a.npts + flat] = cmul(e, acc);
        }
    }

    // =====================================================================
    // Adjoint passes: every step conjugate-transposed, levels in reverse.
    // On entry to a level the slot of output alpha of a merge block holds the
    // level-(l+1) weights; on exit the slot of input c holds the level-l weights.

    // ---- adjoint of one column merge (level l+1 -> l):
    // in_c(t') = sum_alpha e^{-2pi i Phi(x0(A_alpha), y_t'^{B_c})} sum_t M_c[t][t'] e^{2pi i Phi(x0(A_alpha), y_t^{B'})} out_alpha(t)
    static __device__ void col_level_adj(const KArgs<P> &a, C *Wt, C *S, int l, int i)
    {
        const int k = a.k, n = 1 << (D * k), nblk = n >> D;
        const int L = a.L;
        // stage A: items (tau, block, alpha, t_{>=1}): re-modulate out_alpha at the nodes of B',
        // contract dim 0 into both children c_0 -> S[tau][block][alpha][t_{>=1}][c_0][t'_0]
        for (int it = threadIdx.x; it < a.T * nblk * NC * QD1; it += blockDim.x) {
            const int th = it % QD1;
            const int alpha = (it / QD1) % NC;
            const int beta = (it / (QD1 * NC)) & (nblk - 1);
            const int tau = (it / (QD1 * NC)) >> (D * (k - 1));
            uint32_t Ap, Bstar, Apg, Bq;
            int base;
            tile_of(a, tau, Ap, Bstar);
            block_geo(Ap, Bstar, beta, i, k, Apg, Bq, base);
            int ca[DMAX], cbq[DMAX];
            morton_decode<D>((Apg << D) + alpha, l + 1, ca);
            morton_decode<D>(Bq, L - l - 1, cbq);
            const typename PH::T tA = tcenter<P, D, Q, K>(a, l + 1, (Apg << D) + alpha, ca);
            int tk[DMAX];
            {
                int tt = th;
#pragma unroll
                for (int j = 1; j < D; ++j) { tk[j] = tt % Q; tt /= Q; }
            }
            typename PH::Part hp = PH::part(tA, sget<P, Q>(a, 1, l + 1, cbq[1], tk[1]), 1);
            if constexpr (D == 3) hp = PH::add(hp, PH::part(tA, sget<P, Q>(a, 2, l + 1, cbq[2], tk[2]), 2));
            const C *wi = Wt + tau * n * RR + (base + (alpha << (D * i))) * RR + th * Q;
            C z[2][Q];
#pragma unroll
            for (int s0 = 0; s0 < Q; ++s0) { z[0][s0] = czero<C>(); z[1][s0] = czero<C>(); }
            if constexpr (!P::is_f64) {
                // phases two at a time: lanes t_0 and t_0 + 1 (the last one alone for odd q)
                using PH2 = Ph2<P, D, K>;
                const typename PH2::T tA2 = PH2::dup(tA);
                const typename PH2::Part hp2 = PH2::dup(hp);
#pragma unroll
                for (int t0 = 0; t0 + 1 < Q; t0 += 2) {
                    float2 E0, E1;
                    expphase_part2<P, D, K>(a, tA2,
                                            PH2::add(PH2::part(tA2, sget<P, Q>(a, 0, l + 1, cbq[0], t0),
                                                               sget<P, Q>(a, 0, l + 1, cbq[0], t0 + 1), 0), hp2),
                                            E0, E1);
                    const C u0 = cmul(E0, wi[t0]), u1 = cmul(E1, wi[t0 + 1]);
#pragma unroll
                    for (int s0 = 0; s0 < Q; ++s0) {
                        cfma2(z[0][s0], a.M2[0][t0][s0], u0);
                        cfma2(z[1][s0], a.M2[1][t0][s0], u0);
                        cfma2(z[0][s0], a.M2[0][t0 + 1][s0], u1);
                        cfma2(z[1][s0], a.M2[1][t0 + 1][s0], u1);
                    }
                }
                if constexpr (Q & 1) {
                    const C e = expphase_part<P, D, K>(a, tA, PH::add(PH::part(tA, sget<P, Q>(a, 0, l + 1, cbq[0], Q - 1), 0), hp));
                    const C u = cmul(e, wi[Q - 1]);
#pragma unroll
                    for (int s0 = 0; s0 < Q; ++s0) {
                        cfma2(z[0][s0], a.M2[0][Q - 1][s0], u);
                        cfma2(z[1][s0], a.M2[1][Q - 1][s0], u);
                    }
                }
            } else {
#pragma unroll
                for (int t0 = 0; t0 < Q; ++t0) {
                    const C e = expphase_part<P, D, K>(a, tA, PH::add(PH::part(tA, sget<P, Q>(a, 0, l + 1, cbq[0], t0), 0), hp));
                    const C u = cmul(e, wi[t0]);
#pragma unroll
                    for (int s0 = 0; s0 < Q; ++s0) {
                        cfma2(z[0][s0], a.M2[0][t0][s0], u);
                        cfma2(z[1][s0], a.M2[1][t0][s0], u);
                    }
                }
            }
            C *so = S + (((tau * nblk + beta) * NC + alpha) * QD1 + th) * 2 * Q;
#pragma unroll
            for (int s0 = 0; s0 < Q; ++s0) { so[s0] = z[0][s0]; so[Q + s0] = z[1][s0]; }
        }
        __syncthreads();
        // stage B: items (tau, block, c, t'_0): contract dims >= 1 with M_{c_{>=1}} per alpha,
        // conjugate modulation at the nodes of B_c, sum over alpha
        for (int it = threadIdx.x; it < a.T * nblk * NC * Q; it += blockDim.x) {
            const int s0 = it % Q;
            const int c = (it / Q) % NC;
            const int beta = (it / (Q * NC)) & (nblk - 1);
            const int tau = (it / (Q * NC)) >> (D * (k - 1));
            uint32_t Ap, Bstar, Apg, Bq;
            int base;
            tile_of(a, tau, Ap, Bstar);
            block_geo(Ap, Bstar, beta, i, k, Apg, Bq, base);
            int cbq[DMAX], cb[DMAX];
            morton_decode<D>(Bq, L - l - 1, cbq);
#pragma unroll
            for (int j = 0; j < D; ++j) cb[j] = 2 * cbq[j] + ((c >> j) & 1);
            const int c0 = c & 1;
            const typename P::SE e0 = sget<P, Q>(a, 0, l, cb[0], s0);
            C acc[QD1];
#pragma unroll
            for (int j = 0; j < QD1; ++j) acc[j] = czero<C>();
#pragma unroll 1
            for (int alpha = 0; alpha < NC; ++alpha) {
                int ca[DMAX];
                morton_decode<D>((Apg << D) + alpha, l + 1, ca);
                const typename PH::T tA = tcenter<P, D, Q, K>(a, l + 1, (Apg << D) + alpha, ca);
                const typename PH::Part p0 = PH::part(tA, e0, 0);
                const C *si = S + ((tau * nblk + beta) * NC + alpha) * QD1 * 2 * Q + c0 * Q + s0;   // [t_{>=1}] stride 2Q
                if constexpr (D == 2) {
                    const int c1 = (c >> 1) & 1;
                    C v[Q];
#pragma unroll
                    for (int s1 = 0; s1 < Q; ++s1) v[s1] = czero<C>();
#pragma unroll
                    for (int t1 = 0; t1 < Q; ++t1) {
                        const C zz = si[t1 * 2 * Q];
#pragma unroll
                        for (int s1 = 0; s1 < Q; ++s1) cfma2(v[s1], a.M2[c1][t1][s1], zz);
                    }
                    if constexpr (!P::is_f64) {
                        // phases two at a time: lanes s_1 and s_1 + 1 (the last one alone for odd q)
                        using PH2 = Ph2<P, D, K>;
                        const typename PH2::T tA2 = PH2::dup(tA);
                        const typename PH2::Part p02 = PH2::dup(p0);
#pragma unroll
                        for (int s1 = 0; s1 + 1 < Q; s1 += 2) {
                            float2 E0, E1;
                            expphase_part2<P, D, K>(a, tA2,
                                                    PH2::add(p02, PH2::part(tA2, sget<P, Q>(a, 1, l, cb[1], s1),
                                                                            sget<P, Q>(a, 1, l, cb[1], s1 + 1), 1)),
                                                    E0, E1);
                            acc[s1] = cadd(acc[s1], cjmul(E0, v[s1]));
                            acc[s1 + 1] = cadd(acc[s1 + 1], cjmul(E1, v[s1 + 1]));
                        }
                        if constexpr (Q & 1) {
                            const C e = expphase_part<P, D, K>(a, tA, PH::add(p0, PH::part(tA, sget<P, Q>(a, 1, l, cb[1], Q - 1), 1)));
                            acc[Q - 1] = cadd(acc[Q - 1], cjmul(e, v[Q - 1]));
                        }
                    } else {
#pragma unroll
                        for (int s1 = 0; s1 < Q; ++s1) {
                            const C e = expphase_part<P, D, K>(a, tA, PH::add(p0, PH::part(tA, sget<P, Q>(a, 1, l, cb[1], s1), 1)));
                            acc[s1] = cadd(acc[s1], cjmul(e, v[s1]));
                        }
                    }
                } else {
                    const int c1 = (c >> 1) & 1, c2 = (c >> 2) & 1;
                    C w[Q * Q];   // [t1][s2]
#pragma unroll
                    for (int j = 0; j < Q * Q; ++j) w[j] = czero<C>();
#pragma unroll
                    for (int t2 = 0; t2 < Q; ++t2)
#pragma unroll
                        for (int t1 = 0; t1 < Q; ++t1) {
                            const C zz = si[(t1 + Q * t2) * 2 * Q];
#pragma unroll
                            for (int s2 = 0; s2 < Q; ++s2) cfma2(w[t1 * Q + s2], a.M2[c2][t2][s2], zz);
                        }
#pragma unroll
                    for (int s2 = 0; s2 < Q; ++s2) {
                        const typename PH::Part p2 = PH::add(p0, PH::part(tA, sget<P, Q>(a, 2, l, cb[2], s2), 2));
#pragma unroll
                        for (int s1 = 0; s1 < Q; ++s1) {
                            C v = czero<C>();
#pragma unroll
                            for (int t1 = 0; t1 < Q; ++t1) cfma2(v, a.M2[c1][t1][s1], w[t1 * Q + s2]);
                            const C e = expphase_part<P, D, K>(a, tA, PH::add(p2, PH::part(tA, sget<P, Q>(a, 1, l, cb[1], s1), 1)));
                            acc[s1 + Q * s2] = cadd(acc[s1 + Q * s2], cjmul(e, v));
                        }
                    }
                }
            }
            C *wo = Wt + tau * n * RR + (base + (c << (D * i))) * RR + s0;
#pragma unroll
            for (int sh = 0; sh < QD1; ++sh) wo[sh * Q] = acc[sh];
        }
        __syncthreads();
    }

    // ---- adjoint of one row merge (level l+1 -> l):
    // in_c(t) = e^{2pi i Phi(x_t^{Ap}, y0(B_c))} sum_alpha sum_s M_alpha[t][s] e^{-2pi i Phi(x_s^{A_alpha}, y0(B_c))} out_alpha(s)
    static __device__ void row_level_adj(const KArgs<P> &a, C *Wt, C *S, typename PH::T *TC, int l, int i)
    {
        const int k = a.k, n = 1 << (D * k), nblk = n >> D;
        const int L = a.L;
        // target features of the children's nodes (level l+1; T 2^{D(i+1)} boxes x q^d) and,
        // after them, of the parents' nodes (level l; T 2^{Di} boxes x q^d)
        const int nb1 = 1 << (D * (i + 1)), nb0 = 1 << (D * i);
        typename PH::T *TP = TC + a.T * nb1 * RR;
        for (int j = threadIdx.x; j < a.T * (nb1 + nb0) * RR; j += blockDim.x) {
            const bool child = j < a.T * nb1 * RR;
            const int jj = child ? j : j - a.T * nb1 * RR;
            const int nb = child ? nb1 : nb0, lgb = child ? D * (i + 1) : D * i;
            const int t = jj % RR, aloc = (jj / RR) & (nb - 1), tau = (jj / RR) >> lgb;
            uint32_t Ap, Bstar;
            tile_of(a, tau, Ap, Bstar);
            int ca[DMAX], tk[DMAX], tt = t;
            const int lv = child ? l + 1 : l;
            morton_decode<D>((Ap << (D * (child ? i + 1 : i))) + aloc, lv, ca);
#pragma unroll
            for (int q = 0; q < D; ++q) { tk[q] = tt % Q; tt /= Q; }
            TC[j] = tpoint<P, D, Q, K>(a, lv, ca, tk);
        }
        __syncthreads();
        // stage A: items (tau, block, c, alpha_{D-1}, s_{D-1}): conjugate post-modulation of every
        // out_alpha at the child's nodes, contraction over dims 0..D-2 and alpha_{<D-1}
        //   -> S[tau][block][c][alpha_{D-1}][s_{D-1}][t_{<D-1}]
        for (int it = threadIdx.x; it < a.T * nblk * NC * 2 * Q; it += blockDim.x) {
            const int sq = it % Q;
            const int ahi = (it / Q) & 1;
            const int c = (it / (2 * Q)) % NC;
            const int beta = (it / (2 * Q * NC)) & (nblk - 1);
            const int tau = (it / (2 * Q * NC)) >> (D * (k - 1));
            uint32_t Ap, Bstar, Apg, Bq;
            int base;
            tile_of(a, tau, Ap, Bstar);
            block_geo(Ap, Bstar, beta, i, k, Apg, Bq, base);
            int cbq[DMAX], cb[DMAX];
            morton_decode<D>(Bq, L - l - 1, cbq);
#pragma unroll
            for (int j = 0; j < D; ++j) cb[j] = 2 * cbq[j] + ((c >> j) & 1);
            const int ctr[DMAX] = {Q, Q, Q};
            const typename PH::S sc = spoint<P, D, Q, K>(a, l, cb, ctr);
            C acc[QD1];
#pragma unroll
            for (int j = 0; j < QD1; ++j) acc[j] = czero<C>();
#pragma unroll
            for (int al = 0; al < (NC >> 1); ++al) {
                const int alpha = al | (ahi << (D - 1));
                const typename PH::T *tn = TC + (tau * nb1 + (int)((digit_rev<D>(beta & (nb0 - 1), i) << D) + alpha)) * RR;
                const C *wi = Wt + tau * n * RR + (base + (alpha << (D * i))) * RR;
                if constexpr (D == 2) {
                    const int a0 = alpha & 1;
#pragma unroll
                    for (int s0 = 0; s0 < Q; ++s0) {
                        const C e = expphase<P, D, K>(a, tn[s0 + Q * sq], sc);
                        const C u = cjmul(e, wi[s0 + Q * sq]);
#pragma unroll
                        for (int t0 = 0; t0 < Q; ++t0) cfma2(acc[t0], a.M2[a0][t0][s0], u);
                    }
                } else {
                    const int a0 = alpha & 1, a1 = (alpha >> 1) & 1;
#pragma unroll 1
                    for (int s1 = 0; s1 < Q; ++s1) {
                        C tmp[Q];
#pragma unroll
                        for (int t0 = 0; t0 < Q; ++t0) tmp[t0] = czero<C>();
#pragma unroll
                        for (int s0 = 0; s0 < Q; ++s0) {
                            const C e = expphase<P, D, K>(a, tn[s0 + Q * s1 + Q * Q * sq], sc);
                            const C u = cjmul(e, wi[s0 + Q * s1 + Q * Q * sq]);
#pragma unroll
                            for (int t0 = 0; t0 < Q; ++t0) cfma2(tmp[t0], a.M2[a0][t0][s0], u);
                        }
#pragma unroll
                        for (int t1 = 0; t1 < Q; ++t1)
#pragma unroll
                            for (int t0 = 0; t0 < Q; ++t0) cfma2(acc[t0 + Q * t1], a.M2[a1][t1][s1], tmp[t0]);
                    }
                }
            }
            C *so = S + ((((tau * nblk + beta) * NC + c) * 2 + ahi) * Q + sq) * QD1;
#pragma unroll
            for (int j = 0; j < QD1; ++j) so[j] = acc[j];
        }
        __syncthreads();
        // stage B: items (tau, block, c, t_{<D-1}): contract dim D-1 and alpha_{D-1},
        // re-modulate at the nodes of the parent target box
        for (int it = threadIdx.x; it < a.T * nblk * NC * QD1; it += blockDim.x) {
            const int tl = it % QD1;
            const int c = (it / QD1) % NC;
            const int beta = (it / (QD1 * NC)) & (nblk - 1);
            const int tau = (it / (QD1 * NC)) >> (D * (k - 1));
            uint32_t Ap, Bstar, Apg, Bq;
            int base;
            tile_of(a, tau, Ap, Bstar);
            block_geo(Ap, Bstar, beta, i, k, Apg, Bq, base);
            int ca[DMAX], cbq[DMAX], cb[DMAX];
            morton_decode<D>(Apg, l, ca);
            morton_decode<D>(Bq, L - l - 1, cbq);
#pragma unroll
            for (int j = 0; j < D; ++j) cb[j] = 2 * cbq[j] + ((c >> j) & 1);
            const int ctr[DMAX] = {Q, Q, Q};
            const typename PH::S sc = spoint<P, D, Q, K>(a, l, cb, ctr);
            C acc[Q];
#pragma unroll
            for (int j = 0; j < Q; ++j) acc[j] = czero<C>();
#pragma unroll
            for (int ahi = 0; ahi < 2; ++ahi) {
                const C *si = S + ((((tau * nblk + beta) * NC + c) * 2 + ahi) * Q) * QD1 + tl;
#pragma unroll
                for (int sq = 0; sq < Q; ++sq) {
                    const C v = si[sq * QD1];
#pragma unroll
                    for (int tq = 0; tq < Q; ++tq) cfma2(acc[tq], a.M2[ahi][tq][sq], v);
                }
            }
            int tk[DMAX];
            {
                int tt = tl;
#pragma unroll
                for (int j = 0; j < D - 1; ++j) { tk[j] = tt % Q; tt /= Q; }
            }
            C *wo = Wt + tau * n * RR + (base + (c << (D * i))) * RR + tl;
            const typename PH::T *tp = TP + (tau * nb0 + (int)digit_rev<D>(beta & (nb0 - 1), i)) * RR + tl;
#pragma unroll
            for (int tq = 0; tq < Q; ++tq) wo[tq * QD1] = cmul(expphase<P, D, K>(a, tp[tq * QD1], sc), acc[tq]);
        }
        __syncthreads();
    }

    // ---- adjoint of the switch at level l: u(t) = sum_s e^{-2pi i Phi(x_s^A, y_t^B)} v(s);
    // items (tau, slot, t_{>=1}), the q values of t_0 accumulated together.  For d = 2 the
    // target features of every (pair, s) are computed once into TC (the q^{d-1} items of a
    // pair share them); the mixed precision evaluates the phases of t_0, t_0 + 1 in pairs.
    static __device__ void switch_adj(const KArgs<P> &a, C *Wt, C *S, typename PH::T *TC, int l)
    {
        const int k = a.k, n = 1 << (D * k);
        const int L = a.L;
        if constexpr (D == 2) {
            for (int j = threadIdx.x; j < a.T * n * RR; j += blockDim.x) {
                const int s = j % RR, pr = j / RR;
                const int sl = pr & (n - 1), tau = pr >> (D * k);
                uint32_t Ap, Bstar;
                tile_of(a, tau, Ap, Bstar);
                int ca[DMAX];
                morton_decode<D>((Ap << (D * k)) + digit_rev<D>(sl, k), l, ca);
                const int sk[DMAX] = {s % Q, s / Q, 0};
                TC[j] = tpoint<P, D, Q, K>(a, l, ca, sk);
            }
            __syncthreads();
        }
        for (int it = threadIdx.x; it < a.T * n * QD1; it += blockDim.x) {
            const int th = it % QD1;
            const int sl = (it / QD1) & (n - 1);
            const int tau = (it / QD1) >> (D * k);
            uint32_t Ap, Bstar;
            tile_of(a, tau, Ap, Bstar);
            const uint32_t A = (Ap << (D * k)) + digit_rev<D>(sl, k);
            int ca[DMAX], cb[DMAX], tk[DMAX];
            morton_decode<D>(A, l, ca);
            morton_decode<D>(Bstar, L - l, cb);
            {
                int tt = th;
#pragma unroll
                for (int j = 1; j < D; ++j) { tk[j] = tt % Q; tt /= Q; }
            }
            typename P::SE eh[DMAX], e0[Q];
#pragma unroll
            for (int j = 1; j < D; ++j) eh[j] = sget<P, Q>(a, j, l, cb[j], tk[j]);
#pragma unroll
            for (int t0 = 0; t0 < Q; ++t0) e0[t0] = sget<P, Q>(a, 0, l, cb[0], t0);
            C acc[Q];
#pragma unroll
            for (int t0 = 0; t0 < Q; ++t0) acc[t0] = czero<C>();
            const C *v = Wt + (tau * n + sl) * RR;
            const typename PH::T *tc = TC + (tau * n + sl) * RR;
            // d = 2: q targets per iteration of the outer loop (more independent work per iteration)
            constexpr int SI = D == 2 ? Q : 1;
#pragma unroll 1
            for (int s1 = 0; s1 < RR; s1 += SI)
#pragma unroll
            for (int s0 = 0; s0 < SI; ++s0) {
                const int s = s1 + s0;
                typename PH::T tS;
                if constexpr (D == 2) {
                    tS = tc[s];
                } else {
                    int sk[DMAX], ss = s;
#pragma unroll
                    for (int j = 0; j < D; ++j) { sk[j] = ss % Q; ss /= Q; }
                    tS = tpoint<P, D, Q, K>(a, l, ca, sk);
                }
                const C vs = v[s];
                if constexpr (!P::is_f64) {
                    using PH2 = Ph2<P, D, K>;
                    const typename PH2::T tS2 = PH2::dup(tS);
                    typename PH2::Part hp = PH2::part(tS2, eh[1], eh[1], 1);
                    if constexpr (D == 3) hp = PH2::add(hp, PH2::part(tS2, eh[2], eh[2], 2));
#pragma unroll
                    for (int t0 = 0; t0 + 1 < Q; t0 += 2) {
                        float2 E0, E1;
                        expphase_part2<P, D, K>(a, tS2, PH2::add(PH2::part(tS2, e0[t0], e0[t0 + 1], 0), hp), E0, E1);
                        acc[t0] = cadd(acc[t0], cjmul(E0, vs));
                        acc[t0 + 1] = cadd(acc[t0 + 1], cjmul(E1, vs));
                    }
                    if constexpr (Q & 1)
                        acc[Q - 1] = cadd(acc[Q - 1], cjmul(expphase_part<P, D, K>(
                                                                a, tS, PH::add(PH::part(tS, e0[Q - 1], 0), PH2::lane0(hp))),
                                                            vs));
                } else {
                    typename PH::Part hp = PH::part(tS, eh[1], 1);
                    if constexpr (D == 3) hp = PH::add(hp, PH::part(tS, eh[2], 2));
#pragma unroll
                    for (int t0 = 0; t0 < Q; ++t0)
                        acc[t0] = cadd(acc[t0], cjmul(expphase_part<P, D, K>(a, tS, PH::add(PH::part(tS, e0[t0], 0), hp)), vs));
                }
            }
            C *w = S + (tau * n + sl) * RR + th * Q;
#pragma unroll
            for (int t0 = 0; t0 < Q; ++t0) w[t0] = acc[t0];
        }
        __syncthreads();
        for (int j = threadIdx.x; j < a.T * n * RR; j += blockDim.x) Wt[j] = S[j];
        __syncthreads();
    }

    // ---- adjoint of init: g(y) = e^{-2pi i Phi(x0(X), y)} sum_t L_t^B(y) e^{2pi i Phi(x0(X), y_t^B)} w_{XB}(t);
    // slots in natural order (slot = b) at level 0; items (tau, b)
    static __device__ void init_adj(const KArgs<P> &a, const C *Wt, int rhs)
    {
        const int k = a.k, n = 1 << (D * k);
        const int L = a.L;
        const int cX[DMAX] = {0, 0, 0};
        const int ctr[DMAX] = {Q, Q, Q};
        const typename PH::T tX = tpoint<P, D, Q, K>(a, 0, cX, ctr);
        for (int it = threadIdx.x; it < a.T * n; it += blockDim.x) {
            const int b = it & (n - 1), tau = it >> (D * k);
            uint32_t Ap, Bstar;
            tile_of(a, tau, Ap, Bstar);
            int cb[DMAX];
            morton_decode<D>((Bstar << (D * k)) + b, L, cb);
            const C *w = Wt + it * RR;
            C acc = czero<C>();
            for (int t = 0; t < RR; ++t) {
                R lag = R(1);
                int tk[DMAX], tt = t;
#pragma unroll
                for (int j = 0; j < D; ++j) { tk[j] = tt % Q; tt /= Q; lag *= a.lsrc[tk[j]]; }
                if (lag == R(0)) continue;
                cfma(acc, lag, cmul(expphase<P, D, K>(a, tX, spoint<P, D, Q, K>(a, 0, cb, tk)), w[t]));
            }
            const int pslot[DMAX] = {Q + 1, Q + 1, Q + 1};
            const C e = expphase<P, D, K>(a, tX, spoint<P, D, Q, K>(a, 0, cb, pslot));
            int64_t flat = 0;
#pragma unroll
            for (int j = 0; j < D; ++j) flat = (flat << L) + cb[j];
            a.gadj[(int64_t)rhs * a.npts + flat] = cjmul(e, acc);
        }
    }

    // ---- adjoint of final: w_{AY}(t) = e^{2pi i Phi(x_t^A, y0(Y))} L_t^A(x) e^{-2pi i Phi(x, y0(Y))} f(x);
    // slots in digit-reversed order at level L; items (tau, slot, t)
    static __device__ void final_adj(const KArgs<P> &a, C *Wt, int rhs)
    {
        const int k = a.k, n = 1 << (D * k);
        const int L = a.L;
        const int cY[DMAX] = {0, 0, 0};
        const int ctr[DMAX] = {Q, Q, Q};
        const typename PH::S sY = spoint<P, D, Q, K>(a, L, cY, ctr);
        // the nodes whose Lagrange value at the target point is non-zero (the same in every
        // leaf box); the other weights are zero
        __shared__ int nzt[RR];
        __shared__ int nnz;
        if (threadIdx.x == 0) {
            int c = 0;
            for (int t = 0; t < RR; ++t) {
                R lag = R(1);
                for (int j = 0, tt = t; j < D; ++j, tt /= Q) lag *= a.ltgt[tt % Q];
                if (lag != R(0)) nzt[c++] = t;
            }
            nnz = c;
        }
        for (int it = threadIdx.x; it < a.T * n * RR; it += blockDim.x) Wt[it] = czero<C>();
        __syncthreads();
        for (int it = threadIdx.x; it < a.T * n * nnz; it += blockDim.x) {
            const int pr = it / nnz, t = nzt[it - pr * nnz];
            const int sl = pr & (n - 1), tau = pr >> (D * k);
            uint32_t Ap, Bstar;
            tile_of(a, tau, Ap, Bstar);
            const uint32_t A = (Ap << (D * k)) + digit_rev<D>(sl, k);
            int ca[DMAX];
            morton_decode<D>(A, L, ca);
            R lag = R(1);
            int tk[DMAX], tt = t;
#pragma unroll
            for (int j = 0; j < D; ++j) { tk[j] = tt % Q; tt /= Q; lag *= a.ltgt[tk[j]]; }
            int64_t flat = 0;
#pragma unroll
            for (int j = 0; j < D; ++j) flat = (flat << L) + ca[j];
            const C fv = a.fadj[(int64_t)rhs * a.npts + flat];
            const int pslot[DMAX] = {Q + 1, Q + 1, Q + 1};
            const C ex = expphase<P, D, K>(a, tpoint<P, D, Q, K>(a, L, ca, pslot), sY);
            const C et = expphase<P, D, K>(a, tpoint<P, D, Q, K>(a, L, ca, tk), sY);
            const C v = cmul(et, cjmul(ex, fv));
            C out;
            out.x = lag * v.x;
            out.y = lag * v.y;
            Wt[pr * RR + t] = out;
        }
    }

    // ---- adjoint pass input: the forward pass's outputs (strided pairs) into digit-reversed slots
    static __device__ __forceinline__ void load_strided(const KArgs<P> &a, C *Wt, int rhs)
    {
        const int k = a.k, n = 1 << (D * k);
        const int64_t Sstar = 1LL << (D * (a.L - a.l0 - k));
        const C *src = a.win + (int64_t)rhs * a.wstride;
        for (int j = threadIdx.x; j < a.T * n * RR; j += blockDim.x) {
            const int t = j % RR, sl = (j / RR) & (n - 1), tau = (j / RR) >> (D * k);
            uint32_t Ap, Bstar;
            tile_of(a, tau, Ap, Bstar);
            const int64_t pair = ((int64_t)(((int64_t)Ap << (D * k)) + digit_rev<D>(sl, k))) * Sstar + Bstar;
            Wt[j] = src[pair * RR + t];
        }
    }

    // ---- adjoint pass output: natural order, contiguous
    static __device__ __forceinline__ void store_contig(const KArgs<P> &a, const C *Wt, int rhs)
    {
        const int cnt = a.T * (1 << (D * a.k)) * RR;
        C *dst = a.wout + (int64_t)rhs * a.wstride + (int64_t)blockIdx.x * cnt;
        for (int j = threadIdx.x; j < cnt; j += blockDim.x) dst[j] = Wt[j];
    }

    // ---- CTA input: T * 2^{dk} consecutive pairs (contiguous in HBM); with sharding mode 2
    // the pairs of other ranks' source boxes read as zero
    static __device__ __forceinline__ void load(const KArgs<P> &a, C *Wt, int rhs)
    {
        const int cnt = a.T * (1 << (D * a.k)) * RR;
        const int64_t c0 = (int64_t)shard_cta<D>(a, blockIdx.x) * cnt;
        const C *src = a.win + (int64_t)rhs * a.wstride + c0;
        if (a.shard_mode == 2) {
            for (int j = threadIdx.x; j < cnt; j += blockDim.x)
                Wt[j] = shard_owned<D>(a, (c0 + j) / RR) ? src[j] : czero<C>();
            return;
        }
        for (int j = threadIdx.x; j < cnt; j += blockDim.x) Wt[j] = src[j];
    }

    // ---- CTA output: tile slots are in digit-reversed order after k merges
    static __device__ __forceinline__ void store(const KArgs<P> &a, const C *Wt, int rhs)
    {
        const int k = a.k, n = 1 << (D * k);
        const int64_t Sstar = 1LL << (D * (a.L - a.l0 - k));
        C *dst = a.wout + (int64_t)rhs * a.wstride;
        for (int j = threadIdx.x; j < a.T * n * RR; j += blockDim.x) {
            const int t = j % RR, sl = (j / RR) & (n - 1), tau = (j / RR) >> (D * k);
            uint32_t Ap, Bstar;
            tile_of(a, tau, Ap, Bstar);
            const int64_t pair = ((int64_t)(((int64_t)Ap << (D * k)) + digit_rev<D>(sl, k))) * Sstar + Bstar;
            dst[pair * RR + t] = Wt[j];
        }
    }
};

// ------------------------------------------------------------------ kernels

// init (l0 = 0) + k column merges + optional switch at level l0 + k
// PM: phase factors evaluated, or (mixed precisions) recorded in or read from the pass's
// reduced-phase table a.ftab (a.ftab_cta floats per CTA).  Reading the table, the d = 2
// column pass fits one more CTA per SM (register budget cut accordingly): measured 7% faster
// with the polynomial sincos, 19% with the SFU one; the row pass would spill.  At d = 3 the
// shared memory holds two CTAs per SM either way.
template <int D, int Q, class P, int K, int PM = PM_COMPUTE>
__global__ void __launch_bounds__(Cfg<D, Q, P>::NT, PM == PM_TABLE ? Cfg<D, Q, P>::MINB_TAB : Cfg<D, Q, P>::MINB_COL)
    k_col_pass(const KArgs<P> a)
{
    static_assert(PM == PM_COMPUTE || !P::is_f64, "phase tables: mixed precisions");
    using C = typename P::C;
    using TL = Tile<D, Q, P, K>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *Wt = reinterpret_cast<C *>(smem_raw);
    C *S = Wt + a.T * (1 << (D * a.k)) * TL::RR;
    const int rhs = blockIdx.y;
    float *tb = nullptr;
    if constexpr (PM != PM_COMPUTE) {
        if (TL::table_floats(a, false) != a.ftab_cta) {   // the plan's layout disagrees: touch nothing
            if (threadIdx.x == 0 && a.err) atomicExch(a.err, 2);
            return;
        }
        tb = a.ftab + (int64_t)blockIdx.x * a.ftab_cta;
        if constexpr (PM == PM_TABLE) TL::prefetch_l2(tb, TL::level_floats(a, false));
    }
    if (a.flags & F_INIT)
        TL::init(a, Wt, rhs);
    else
        TL::load(a, Wt, rhs);
    __syncthreads();
    typename TL::Geo *G = reinterpret_cast<typename TL::Geo *>(S + 2 * a.T * (1 << (D * a.k)) * TL::RR);
    for (int i = 0; i < a.k; ++i) {
        if constexpr (PM == PM_TABLE) {   // the next level's blocks (or the switch's) while this level runs
            const int64_t lf = TL::level_floats(a, false);
            if (i + 1 < a.k)
                TL::prefetch_l2(tb + lf, lf);
            else if (a.flags & F_SWITCH)
                TL::prefetch_l2(tb + lf, a.ftab_cta - (int64_t)a.k * lf);
        }
        TL::template col_level<PM>(a, Wt, S, G, a.l0 + i, i, tb);
    }
    if (a.flags & F_SWITCH) {
        if constexpr (K == KIND_DOT || K == KIND_SEPARABLE)
            TL::template switch_sep<false>(a, Wt, S, a.l0 + a.k);
        else
            TL::template switch_tiles<PM>(a, Wt, S, a.l0 + a.k, tb);
    }
    TL::store(a, Wt, rhs);
}

// k row merges + optional final evaluation (l0 + k = L)
template <int D, int Q, class P, int K, int PM = PM_COMPUTE>
__global__ void __launch_bounds__(Cfg<D, Q, P>::NT, Cfg<D, Q, P>::MINB) k_row_pass(const KArgs<P> a)
{
    static_assert(PM == PM_COMPUTE || !P::is_f64, "phase tables: mixed precisions");
    using C = typename P::C;
    using TL = Tile<D, Q, P, K>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *Wt = reinterpret_cast<C *>(smem_raw);
    C *S = Wt + a.T * (1 << (D * a.k)) * TL::RR;
    const int rhs = blockIdx.y;
    typename TL::PH::T *TC = reinterpret_cast<typename TL::PH::T *>(S + 2 * a.T * (1 << (D * a.k)) * TL::RR);
    float *tb = nullptr;
    if constexpr (PM != PM_COMPUTE) {
        if (TL::table_floats(a, true) != a.ftab_cta) {   // the plan's layout disagrees: touch nothing
            if (threadIdx.x == 0 && a.err) atomicExch(a.err, 2);
            return;
        }
        tb = a.ftab + (int64_t)blockIdx.x * a.ftab_cta;
        if constexpr (PM == PM_TABLE) TL::prefetch_l2(tb, TL::level_floats(a, true));
    }
    TL::load(a, Wt, rhs);
    __syncthreads();
    for (int i = 0; i < a.k; ++i) {
        if constexpr (PM == PM_TABLE) {   // the next level's blocks while this level runs
            const int64_t lf = TL::level_floats(a, true);
            if (i + 1 < a.k) TL::prefetch_l2(tb + lf, lf);
        }
        TL::template row_level<PM>(a, Wt, S, TC, a.l0 + i, i, tb);
    }
    if (a.flags & F_FINAL)
        TL::final_eval(a, Wt, rhs);
    else
        TL::store(a, Wt, rhs);
}

// adjoint of a column pass: optional switch^H at level l0 + k, k column levels in
// reverse, optional init^H (writes the source values)
template <int D, int Q, class P, int K>
__global__ void __launch_bounds__(Cfg<D, Q, P>::NT, Cfg<D, Q, P>::MINB) k_col_pass_adj(const KArgs<P> a)
{
    using C = typename P::C;
    using TL = Tile<D, Q, P, K>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *Wt = reinterpret_cast<C *>(smem_raw);
    C *S = Wt + a.T * (1 << (D * a.k)) * TL::RR;
    typename TL::PH::T *TC = reinterpret_cast<typename TL::PH::T *>(S + 2 * a.T * (1 << (D * a.k)) * TL::RR);
    const int rhs = blockIdx.y;
    TL::load_strided(a, Wt, rhs);
    __syncthreads();
    if (a.flags & F_SWITCH) {
        if constexpr (K == KIND_DOT || K == KIND_SEPARABLE)
            TL::template switch_sep<true>(a, Wt, S, a.l0 + a.k);
        else
            TL::switch_adj(a, Wt, S, TC, a.l0 + a.k);
    }
    for (int i = a.k - 1; i >= 0; --i) TL::col_level_adj(a, Wt, S, a.l0 + i, i);
    if (a.flags & F_INIT)
        TL::init_adj(a, Wt, rhs);
    else
        TL::store_contig(a, Wt, rhs);
}

// adjoint of a row pass: optional final^H (reads the target values), k row levels in reverse
template <int D, int Q, class P, int K>
__global__ void __launch_bounds__(Cfg<D, Q, P>::NT, Cfg<D, Q, P>::MINB) k_row_pass_adj(const KArgs<P> a)
{
    using C = typename P::C;
    using TL = Tile<D, Q, P, K>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *Wt = reinterpret_cast<C *>(smem_raw);
    C *S = Wt + a.T * (1 << (D * a.k)) * TL::RR;
    const int rhs = blockIdx.y;
    typename TL::PH::T *TC = reinterpret_cast<typename TL::PH::T *>(S + 2 * a.T * (1 << (D * a.k)) * TL::RR);
    if (a.flags & F_FINAL)
        TL::final_adj(a, Wt, rhs);
    else
        TL::load_strided(a, Wt, rhs);
    __syncthreads();
    for (int i = a.k - 1; i >= 0; --i) TL::row_level_adj(a, Wt, S, TC, a.l0 + i, i);
    TL::store_contig(a, Wt, rhs);
}

}  // namespace bfk
