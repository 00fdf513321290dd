// Self-checks of the mixed-precision arithmetic on the device:
//   * the FP32 sincos2pi against CUDA's FP64 sincospi on evenly spaced arguments;
//   * the double-float Phi (mod 1) against FP64 arithmetic on the same table
//     features (each double-float feature hi + lo taken as an FP64 number),
//     for pseudo-random (target node, source node) pairs of a plan's tables.
#include <cstdint>

#include "bf_device.cuh"
#include "bf_launch.h"

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

}  // namespace

namespace bfl {

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
    const int iters = fp64 ? 100 : 2000;
    for (int rep = 0; rep < 2; ++rep) {
        if (rep == 1) cudaEventRecord(e0);
        if (fp64)
            k_fma64<<<blocks, threads>>>(rep ? iters : 2, static_cast<double *>(out));
        else
            k_fma32<<<blocks, threads>>>(rep ? iters : 10, static_cast<float *>(out));
    }
    cudaEventRecord(e1);
    e = cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    const double flops = 2.0 * blocks * threads * (double)iters * 16 * (fp64 ? 4 : 8);
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

}  // namespace bfl
