// Self-checks of the mixed-precision arithmetic on the device:
//   * the FP32 sincos2pi against CUDA's FP64 sincospi on evenly spaced arguments;
//   * the double-float Phi (mod 1) against FP64 arithmetic on the same table
//     features (each double-float feature hi + lo taken as an FP64 number),
//     for pseudo-random (target node, source node) pairs of a plan's tables.
#include <cmath>
#include <cstdint>
#include <vector>

#include "bf_device.cuh"
#include "bf_launch.h"
#include "bf_pair.cuh"
#include "bf_tc.cuh"

namespace {

__device__ __forceinline__ void atomic_max_nonneg(double *addr, double v)
{
    // non-negative doubles order like their bit patterns
    atomicMax(reinterpret_cast<unsigned long long *>(addr), (unsigned long long)__double_as_longlong(v));
}

__global__ void k_check_sincos(int n, double *out)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float f = -1.0f + 2.0f * (float)i / (float)n;
        float s, c;
        bfk::sincos2pi(f, s, c);
        double sd, cd;
        sincospi(2.0 * (double)f, &sd, &cd);
        atomic_max_nonneg(out, fmax(fabs((double)s - sd), fabs((double)c - cd)));
    }
}

__device__ __forceinline__ uint32_t hash32(uint32_t x)
{
    x ^= x >> 16;
    x *= 0x7feb352dU;
    x ^= x >> 15;
    x *= 0x846ca68bU;
    x ^= x >> 16;
    return x;
}

template <int D, int K>
__global__ void k_check_phase(bfk::KArgs<bfk::PMIX> am, bfk::KArgs<bfk::PF64> ad, int L, int q, int n, double *out)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        uint32_t h = hash32(0x9e3779b9u * (uint32_t)(i + 1));
        const int lt = (int)(h % (uint32_t)(L + 1));
        h = hash32(h);
        const int ls = (int)(h % (uint32_t)(L + 1));
        bfk::PMIX::TE te[D];
        bfk::PF64::TE ted[D];
        typename bfk::Ph<bfk::PMIX, D, K>::S sm;
        typename bfk::Ph<bfk::PF64, D, K>::S sd;
        for (int k = 0; k < D; ++k) {
            h = hash32(h);
            const int bt = (int)(h % (1u << lt)), jt = (int)((h >> 20) % (uint32_t)(q + 2));
            h = hash32(h);
            const int bs = (int)(h % (1u << (L - ls))), js = (int)((h >> 20) % (uint32_t)(q + 2));
            te[k] = am.tt[k][((1LL << lt) - 1) * (q + 2) + (int64_t)bt * (q + 2) + jt];
            const bfk::PMIX::SE se = am.st[k][((2LL << L) - (2LL << (L - ls))) * (q + 2) + (int64_t)bs * (q + 2) + js];
            ted[k].a = make_double2((double)te[k].a.x + te[k].a.y, (double)te[k].a.z + te[k].a.w);
            ted[k].b = make_double2((double)te[k].b.x + te[k].b.y, 0.0);
            bfk::Ph<bfk::PMIX, D, K>::src1(sm, k, se);
            bfk::PF64::SE sed;
            sed.a = make_double2((double)se.a.x + se.a.y, (double)se.a.z + se.a.w);
            bfk::Ph<bfk::PF64, D, K>::src1(sd, k, sed);
        }
        const float fm = bfk::Ph<bfk::PMIX, D, K>::frac(am, bfk::Ph<bfk::PMIX, D, K>::tgt(am, te), sm);
        const double fd = bfk::Ph<bfk::PF64, D, K>::frac(ad, bfk::Ph<bfk::PF64, D, K>::tgt(ad, ted), sd);
        double e = (double)fm - fd;
        e -= rint(e);
        atomic_max_nonneg(out, fabs(e));
    }
}

// dependent FMA chains, 8 (FP32) or 4 (FP64) independent per thread
__global__ void k_fma32(int iters, float *out)
{
    float a0 = threadIdx.x, a1 = a0 + 1, a2 = a0 + 2, a3 = a0 + 3, a4 = a0 + 4, a5 = a0 + 5, a6 = a0 + 6, a7 = a0 + 7;
    const float b = 0.999f, c = 0.001f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            a0 = fmaf(a0, b, c); a1 = fmaf(a1, b, c); a2 = fmaf(a2, b, c); a3 = fmaf(a3, b, c);
            a4 = fmaf(a4, b, c); a5 = fmaf(a5, b, c); a6 = fmaf(a6, b, c); a7 = fmaf(a7, b, c);
        }
    }
    out[blockIdx.x * blockDim.x + threadIdx.x] = a0 + a1 + a2 + a3 + a4 + a5 + a6 + a7;
}

// packed pairs: one instruction does two FP32 FMAs (sm_100 and later)
__global__ void k_fma32x2(int iters, float *out)
{
    const float f = threadIdx.x;
    float2 a0 = make_float2(f, f + 1), a1 = make_float2(f + 2, f + 3), a2 = make_float2(f + 4, f + 5),
           a3 = make_float2(f + 6, f + 7), a4 = make_float2(f + 8, f + 9), a5 = make_float2(f + 10, f + 11),
           a6 = make_float2(f + 12, f + 13), a7 = make_float2(f + 14, f + 15);
    const float2 b = make_float2(0.999f, 0.999f), c = make_float2(0.001f, 0.001f);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            a0 = __ffma2_rn(a0, b, c); a1 = __ffma2_rn(a1, b, c); a2 = __ffma2_rn(a2, b, c); a3 = __ffma2_rn(a3, b, c);
            a4 = __ffma2_rn(a4, b, c); a5 = __ffma2_rn(a5, b, c); a6 = __ffma2_rn(a6, b, c); a7 = __ffma2_rn(a7, b, c);
        }
    }
    out[blockIdx.x * blockDim.x + threadIdx.x] =
        a0.x + a1.x + a2.x + a3.x + a4.x + a5.x + a6.x + a7.x + a0.y + a1.y + a2.y + a3.y + a4.y + a5.y + a6.y + a7.y;
}

__global__ void k_fma64(int iters, double *out)
{
    double a0 = threadIdx.x, a1 = a0 + 1, a2 = a0 + 2, a3 = a0 + 3;
    const double b = 0.999, c = 0.001;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < 16; ++j) { a0 = fma(a0, b, c); a1 = fma(a1, b, c); a2 = fma(a2, b, c); a3 = fma(a3, b, c); }
    }
    out[blockIdx.x * blockDim.x + threadIdx.x] = a0 + a1 + a2 + a3;
}

// Phase-evaluation rate (d = 2): every thread holds two target nodes and 4 + 4
// per-dimension source entries of a plan's tables and evaluates e^{2 pi i Phi} for
// all 2 x 4 x 4 combinations per iteration, with the part of source coordinate 1
// hoisted as in the kernels; every source entry moves every iteration (16 adds per
// 32 phases) so nothing is loop invariant.  PAIRED = 1 evaluates the two targets in the lanes of a float2.
template <class P, int K, int PAIRED>
__global__ void k_phase_rate(const bfk::KArgs<P> a, int L, int q, int iters, float *out)
{
    using PH = bfk::Ph<P, 2, K>;
    using PH2 = bfk::Ph2<P, 2, K>;
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t h = hash32(tid + 1);
    const int lv = L / 2;
    typename PH::T tg[2];
    for (int j = 0; j < 2; ++j) {
        typename P::TE e[2];
        for (int k = 0; k < 2; ++k) {
            h = hash32(h);
            e[k] = a.tt[k][((1LL << lv) - 1) * (q + 2) + (int64_t)(h % (1u << lv)) * (q + 2) + (h >> 24) % q];
        }
        tg[j] = PH::tgt(a, e);
    }
    typename P::SE s0[4], s1[4];
    for (int j = 0; j < 4; ++j) {
        h = hash32(h);
        const int64_t off = ((2LL << L) - (2LL << (L - lv))) * (q + 2);
        s0[j] = a.st[0][off + (int64_t)(h % (1u << (L - lv))) * (q + 2) + (h >> 24) % q];
        h = hash32(h);
        s1[j] = a.st[1][off + (int64_t)(h % (1u << (L - lv))) * (q + 2) + (h >> 24) % q];
    }
    float2 acc = make_float2(0.f, 0.f);
    const typename PH2::T t2 = PH2::pair(tg[0], tg[1]);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            s0[j].a.x = __fadd_rn(s0[j].a.x, 1e-3f);
            s0[j].a.z = __fadd_rn(s0[j].a.z, 1e-3f);
            s1[j].a.x = __fadd_rn(s1[j].a.x, 1e-3f);
            s1[j].a.z = __fadd_rn(s1[j].a.z, 1e-3f);
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if constexpr (PAIRED) {
                const typename PH2::Part hp = PH2::part(t2, s1[j], s1[j], 1);
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    float2 e0, e1;
                    bfk::expphase_part2<P, 2, K>(a, t2, PH2::add(PH2::part(t2, s0[i], s0[i], 0), hp), e0, e1);
                    acc.x += e0.x + e1.x;
                    acc.y += e0.y + e1.y;
                }
            } else {
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    const typename PH::Part hp = PH::part(tg[u], s1[j], 1);
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const float2 e = bfk::expphase_part<P, 2, K>(a, tg[u], PH::add(PH::part(tg[u], s0[i], 0), hp));
                        acc.x += e.x;
                        acc.y += e.y;
                    }
                }
            }
        }
    }
    out[tid] = acc.x + acc.y;
}

// Self-check of the tensor-core building blocks with the operand layout above: one CTA
// computes D = A B^T (M = 128, N = 32, K = KK) from row-major FP32 inputs A [128][KK] and
// B [32][KK], either from the roundings of the inputs to the operand format (split = 0: one
// product per K step) or from their split into hi + lo (split = 1: three products), and
// writes D [128][32] row-major.  F = 0: BF16 operands (kind::f16), KK = 64; F = 1: TF32
// operands (kind::tf32), KK = 32.
template <int F>
__global__ void __launch_bounds__(128) k_umma_selfcheck(const float *A, const float *B, float *Dout, int split, int *err)
{
    constexpr int M = 128, N = 32, KK = F ? 32 : 64, EPC = F ? 4 : 8;   // EPC: elements per 16-byte piece
    constexpr uint32_t LBO = 128, SBO = (KK / EPC) * 128, AB = (M / 8) * SBO, BB = (N / 8) * SBO;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned char *Ah = smem_raw, *Al = Ah + AB, *Bh = Al + AB, *Bl = Bh + BB;
    uint64_t *bar = reinterpret_cast<uint64_t *>(Bl + BB);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bar + 1);
    int *sfail = reinterpret_cast<int *>(tslot + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // one 32-bit word per item: two BF16 values or one TF32 value
    auto put = [&](const float *X, int rows, unsigned char *hp, unsigned char *lp) {
        constexpr int VPW = F ? 1 : 2;   // values per word
        for (int j = tid; j < rows * KK / VPW; j += 128) {
            const int m = j / (KK / VPW), k = VPW * (j % (KK / VPW));
            uint32_t hi, lo;
            if constexpr (F)
                bfk::umma::split_tf32(X[m * KK + k], hi, lo);
            else
                bfk::umma::split2(X[m * KK + k], X[m * KK + k + 1], hi, lo);
            const uint32_t off = bfk::umma::kmajor_piece_off(m, k / EPC, LBO, SBO) + (uint32_t)(k % EPC) * (F ? 4u : 2u);
            *reinterpret_cast<uint32_t *>(hp + off) = hi;
            *reinterpret_cast<uint32_t *>(lp + off) = split ? lo : 0u;
        }
    };
    put(A, M, Ah, Al);
    put(B, N, Bh, Bl);
    if (warp == 0) bfk::umma::alloc(tslot, 32);
    if (tid == 0) {
        bfk::mbar_init(bar, 1);
        bfk::mbar_init_fence();
        *sfail = 0;
    }
    bfk::umma::fence_smem_to_async();
    bfk::umma::fence_before_sync();
    __syncthreads();
    bfk::umma::fence_after_sync();
    const uint32_t tmem = *tslot;
    if (tid == 0) {
        const uint32_t idesc = F ? bfk::umma::idesc_tf32_f32(M, N) : bfk::umma::idesc_bf16_f32(M, N);
        auto mma = [&](uint64_t da, uint64_t db, int acc) {
            if constexpr (F)
                bfk::umma::mma_tf32(tmem, da, db, idesc, acc);
            else
                bfk::umma::mma_bf16(tmem, da, db, idesc, acc);
        };
        for (int ks = 0; ks < KK / (2 * EPC); ++ks) {
            const uint32_t o = (uint32_t)ks * 2u * LBO;
            const uint64_t dah = bfk::umma::desc_kmajor(bfk::umma::saddr(Ah) + o, LBO, SBO);
            const uint64_t dal = bfk::umma::desc_kmajor(bfk::umma::saddr(Al) + o, LBO, SBO);
            const uint64_t dbh = bfk::umma::desc_kmajor(bfk::umma::saddr(Bh) + o, LBO, SBO);
            const uint64_t dbl = bfk::umma::desc_kmajor(bfk::umma::saddr(Bl) + o, LBO, SBO);
            mma(dah, dbh, ks > 0);
            if (split) {
                mma(dah, dbl, 1);
                mma(dal, dbh, 1);
            }
        }
        bfk::umma::commit(bar);
        if (!bfk::mbar_wait_ns(bar, 0, bfk::TC_WAIT_NS)) {
            atomicExch(err, 1);
            *sfail = 1;
            bfk::mbar_wait_ns(bar, 0, bfk::TC_WAIT_NS);
        }
    }
    __syncthreads();
    bfk::umma::fence_after_sync();
    if (!*sfail) {
        for (int c0 = 0; c0 < N; c0 += 8) {
            float v[8];
            bfk::umma::ld8(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)c0, v);
            for (int j = 0; j < 8; ++j) Dout[(32 * warp + lane) * N + c0 + j] = v[j];
        }
    }
    bfk::umma::fence_before_sync();
    __syncthreads();
    if (warp == 0) bfk::umma::dealloc(tmem, 32);
}

template <class P>
cudaError_t phase_rate_t(const void *kargs, int L, int q, int kind, int paired, double *gphases)
{
    const bfk::KArgs<P> &a = *static_cast<const bfk::KArgs<P> *>(kargs);
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int blocks = sms * 8, threads = 256, iters = 200;
    float *out = nullptr;
    cudaError_t e = cudaMalloc(&out, (size_t)blocks * threads * sizeof(float));
    if (e != cudaSuccess) return e;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    auto launch = [&](int n) {
#define BF_PR(KK)                                                                                         \
    (paired ? k_phase_rate<P, KK, 1><<<blocks, threads>>>(a, L, q, n, out)                                \
            : k_phase_rate<P, KK, 0><<<blocks, threads>>>(a, L, q, n, out))
        switch (kind) {
        case bfk::KIND_DOT: BF_PR(bfk::KIND_DOT); break;
        case bfk::KIND_GENRADON: BF_PR(bfk::KIND_GENRADON); break;
        case bfk::KIND_HYPRADON: BF_PR(bfk::KIND_HYPRADON); break;
        default: BF_PR(bfk::KIND_SEPARABLE); break;
        }
#undef BF_PR
    };
    launch(4);
    cudaEventRecord(e0);
    launch(iters);
    cudaEventRecord(e1);
    e = cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    *gphases = (double)blocks * threads * iters * 32 / (ms * 1e-3) / 1e9;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    if (e == cudaSuccess) e = cudaGetLastError();
    return e;
}

}  // namespace

namespace bfl {

cudaError_t phase_rate(const void *kargs, int sfu, int L, int q, int kind, int paired, double *gphases)
{
    return sfu ? phase_rate_t<bfk::PMIXF>(kargs, L, q, kind, paired, gphases)
               : phase_rate_t<bfk::PMIX>(kargs, L, q, kind, paired, gphases);
}


cudaError_t measure_fma(int fp64, double *tflops)
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int blocks = sms * 32, threads = 256;
    void *out = nullptr;
    cudaError_t e = cudaMalloc(&out, (size_t)blocks * threads * 8);
    if (e != cudaSuccess) return e;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int iters = fp64 == 1 ? 100 : 2000;
    for (int rep = 0; rep < 2; ++rep) {
        if (rep == 1) cudaEventRecord(e0);
        if (fp64 == 1)
            k_fma64<<<blocks, threads>>>(rep ? iters : 2, static_cast<double *>(out));
        else if (fp64 == 2)
            k_fma32x2<<<blocks, threads>>>(rep ? iters : 10, static_cast<float *>(out));
        else
            k_fma32<<<blocks, threads>>>(rep ? iters : 10, static_cast<float *>(out));
    }
    cudaEventRecord(e1);
    e = cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    const double flops = 2.0 * blocks * threads * (double)iters * 16 * (fp64 == 1 ? 4 : fp64 == 2 ? 16 : 8);
    *tflops = flops / (ms * 1e-3) / 1e12;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    if (e == cudaSuccess) e = cudaGetLastError();
    return e;
}

cudaError_t selfcheck_sincos(int n, double *max_err)
{
    double *d = nullptr;
    cudaError_t e = cudaMalloc(&d, sizeof(double));
    if (e != cudaSuccess) return e;
    cudaMemset(d, 0, sizeof(double));
    k_check_sincos<<<512, 256>>>(n, d);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpy(max_err, d, sizeof(double), cudaMemcpyDeviceToHost);
    cudaFree(d);
    return e;
}

cudaError_t selfcheck_phase(const void *kargs_mix, const void *kargs_f64, int d, int L, int q, int kind, int n,
                            double *max_err)
{
    double *dd = nullptr;
    cudaError_t e = cudaMalloc(&dd, sizeof(double));
    if (e != cudaSuccess) return e;
    cudaMemset(dd, 0, sizeof(double));
    const auto &am = *static_cast<const bfk::KArgs<bfk::PMIX> *>(kargs_mix);
    const auto &ad = *static_cast<const bfk::KArgs<bfk::PF64> *>(kargs_f64);
    switch (d * 8 + kind) {
    case 16 + bfk::KIND_DOT: k_check_phase<2, bfk::KIND_DOT><<<512, 256>>>(am, ad, L, q, n, dd); break;
    case 16 + bfk::KIND_GENRADON: k_check_phase<2, bfk::KIND_GENRADON><<<512, 256>>>(am, ad, L, q, n, dd); break;
    case 16 + bfk::KIND_HYPRADON: k_check_phase<2, bfk::KIND_HYPRADON><<<512, 256>>>(am, ad, L, q, n, dd); break;
    case 16 + bfk::KIND_SEPARABLE: k_check_phase<2, bfk::KIND_SEPARABLE><<<512, 256>>>(am, ad, L, q, n, dd); break;
    case 24 + bfk::KIND_DOT: k_check_phase<3, bfk::KIND_DOT><<<512, 256>>>(am, ad, L, q, n, dd); break;
    case 24 + bfk::KIND_GENRADON: k_check_phase<3, bfk::KIND_GENRADON><<<512, 256>>>(am, ad, L, q, n, dd); break;
    default: k_check_phase<3, bfk::KIND_SEPARABLE><<<512, 256>>>(am, ad, L, q, n, dd); break;
    }
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpy(max_err, dd, sizeof(double), cudaMemcpyDeviceToHost);
    cudaFree(dd);
    return e;
}

// The tensor-core path on fixed operands (fmt 0: BF16, 1: TF32): split = 0 uses small
// integers (every product and sum exact, so the result must equal the FP64 product),
// split = 1 uniform values in [-1, 1) through the hi + lo split.  max_rel_err: largest
// |D - D_ref| over max |D_ref|; timed_out: the completion wait gave up.
cudaError_t selfcheck_umma(int fmt, int split, double *max_rel_err, int *timed_out)
{
    constexpr int M = 128, N = 32;
    const int KK = fmt ? 32 : 64, EPC = fmt ? 4 : 8;
    std::vector<float> A((size_t)M * KK), B((size_t)N * KK);
    uint32_t h = 12345u;
    for (auto *v : {&A, &B})
        for (float &x : *v) {
            h = h * 1664525u + 1013904223u;
            x = split ? (float)((int)(h >> 8) - (1 << 23)) / (float)(1 << 23) : (float)((int)((h >> 24) % 17u) - 8);
        }
    float *dA = nullptr, *dB = nullptr, *dD = nullptr;
    int *derr = nullptr;
    cudaError_t e = cudaMalloc(&dA, A.size() * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&dB, B.size() * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&dD, (size_t)M * N * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&derr, sizeof(int));
    if (e == cudaSuccess) e = cudaMemcpy(dA, A.data(), A.size() * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dB, B.data(), B.size() * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(dD, 0, (size_t)M * N * sizeof(float));
    if (e == cudaSuccess) e = cudaMemset(derr, 0, sizeof(int));
    if (e == cudaSuccess) {
        const size_t sbo = (size_t)(KK / EPC) * 128;
        const size_t smem = 2 * (size_t)(M / 8) * sbo + 2 * (size_t)(N / 8) * sbo + 64;   // < 48 KB
        if (fmt)
            k_umma_selfcheck<1><<<1, 128, smem>>>(dA, dB, dD, split, derr);
        else
            k_umma_selfcheck<0><<<1, 128, smem>>>(dA, dB, dD, split, derr);
        e = cudaGetLastError();
    }
    std::vector<float> D((size_t)M * N);
    int terr = 0;
    if (e == cudaSuccess) e = cudaMemcpy(D.data(), dD, D.size() * sizeof(float), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(&terr, derr, sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) {
        double mx = 0.0, md = 0.0;
        for (int m = 0; m < M; ++m)
            for (int n = 0; n < N; ++n) {
                double ref = 0.0;
                for (int k = 0; k < KK; ++k) ref += (double)A[(size_t)m * KK + k] * (double)B[(size_t)n * KK + k];
                md = std::fmax(md, std::fabs(ref));
                mx = std::fmax(mx, std::fabs((double)D[(size_t)m * N + n] - ref));
            }
        *max_rel_err = md > 0.0 ? mx / md : mx;
        *timed_out = terr;
    }
    cudaFree(dA);
    cudaFree(dB);
    cudaFree(dD);
    cudaFree(derr);
    return e;
}

}  // namespace bfl
