// Explicit instantiation helpers: one translation unit per (d, precision).
#pragma once

#include "bf_device.cuh"
#include "bf_mr.cuh"
#include "bf_tc.cuh"
#include "bf_launch.h"

namespace bfl {

// Raise the kernel's dynamic shared-memory limit to what this launch needs,
// checked against the device's opt-in maximum.  `granted` is owned by the one
// kernel instantiation that calls this (per device).
template <class K>
inline cudaError_t prepare(K kern, size_t smem, size_t *granted)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (smem <= 48 * 1024 || smem <= granted[dev]) return cudaSuccess;
    int optin = 0;
    e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    if (smem > (size_t)optin) return cudaErrorInvalidValue;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    granted[dev] = smem;
    return cudaSuccess;
}

template <int D, int Q, class P, int K, int PM = bfk::PM_COMPUTE>
cudaError_t launch_col(const void *kargs, unsigned gx, unsigned gy, size_t smem, cudaStream_t s)
{
    static size_t granted[64] = {0};
    cudaError_t e = prepare(bfk::k_col_pass<D, Q, P, K, PM>, smem, granted);
    if (e != cudaSuccess) return e;
    bfk::k_col_pass<D, Q, P, K, PM><<<dim3(gx, gy), bfk::Cfg<D, Q, P>::NT, smem, s>>>(*static_cast<const bfk::KArgs<P> *>(kargs));
    return cudaGetLastError();
}

template <int D, int Q, class P, int K, int PM = bfk::PM_COMPUTE>
cudaError_t launch_row(const void *kargs, unsigned gx, unsigned gy, size_t smem, cudaStream_t s)
{
    static size_t granted[64] = {0};
    cudaError_t e = prepare(bfk::k_row_pass<D, Q, P, K, PM>, smem, granted);
    if (e != cudaSuccess) return e;
    bfk::k_row_pass<D, Q, P, K, PM><<<dim3(gx, gy), bfk::Cfg<D, Q, P>::NT, smem, s>>>(*static_cast<const bfk::KArgs<P> *>(kargs));
    return cudaGetLastError();
}

template <int D, int Q, class P, int K>
cudaError_t launch_col_adj(const void *kargs, unsigned gx, unsigned gy, size_t smem, cudaStream_t s)
{
    static size_t granted[64] = {0};
    cudaError_t e = prepare(bfk::k_col_pass_adj<D, Q, P, K>, smem, granted);
    if (e != cudaSuccess) return e;
    bfk::k_col_pass_adj<D, Q, P, K><<<dim3(gx, gy), bfk::Cfg<D, Q, P>::NT, smem, s>>>(*static_cast<const bfk::KArgs<P> *>(kargs));
    return cudaGetLastError();
}

template <int D, int Q, class P, int K>
cudaError_t launch_row_adj(const void *kargs, unsigned gx, unsigned gy, size_t smem, cudaStream_t s)
{
    static size_t granted[64] = {0};
    cudaError_t e = prepare(bfk::k_row_pass_adj<D, Q, P, K>, smem, granted);
    if (e != cudaSuccess) return e;
    bfk::k_row_pass_adj<D, Q, P, K><<<dim3(gx, gy), bfk::Cfg<D, Q, P>::NT, smem, s>>>(*static_cast<const bfk::KArgs<P> *>(kargs));
    return cudaGetLastError();
}

template <int Q, class P, int K, int PM>
cudaError_t launch_col_mr(const void *kargs, unsigned gx, unsigned gy, size_t smem, cudaStream_t s)
{
    static size_t granted[64] = {0};
    cudaError_t e = prepare(bfk::k_col_pass_mr<Q, P, K, PM>, smem, granted);
    if (e != cudaSuccess) return e;
    bfk::k_col_pass_mr<Q, P, K, PM><<<dim3(gx, gy), bfk::CfgMR<Q>::NT, smem, s>>>(*static_cast<const bfk::KArgs<P> *>(kargs));
    return cudaGetLastError();
}

template <int Q, class P, int K, int PM>
cudaError_t launch_row_mr(const void *kargs, unsigned gx, unsigned gy, size_t smem, cudaStream_t s)
{
    static size_t granted[64] = {0};
    cudaError_t e = prepare(bfk::k_row_pass_mr<Q, P, K, PM>, smem, granted);
    if (e != cudaSuccess) return e;
    bfk::k_row_pass_mr<Q, P, K, PM><<<dim3(gx, gy), bfk::CfgMR<Q>::NT, smem, s>>>(*static_cast<const bfk::KArgs<P> *>(kargs));
    return cudaGetLastError();
}

// CTAs per SM of the table-reading multi-RHS passes with `smem` bytes of shared memory
template <int Q, class P, int K>
int mr_table_occupancy(int row, size_t smem)
{
    static size_t granted_c[64] = {0}, granted_r[64] = {0};
    int n = 0;
    if (row) {
        if (prepare(bfk::k_row_pass_mr<Q, P, K, bfk::PM_TABLE>, smem, granted_r) != cudaSuccess) return 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, bfk::k_row_pass_mr<Q, P, K, bfk::PM_TABLE>,
                                                          bfk::CfgMR<Q>::NT, smem) != cudaSuccess)
            return 0;
    } else {
        if (prepare(bfk::k_col_pass_mr<Q, P, K, bfk::PM_TABLE>, smem, granted_c) != cudaSuccess) return 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, bfk::k_col_pass_mr<Q, P, K, bfk::PM_TABLE>,
                                                          bfk::CfgMR<Q>::NT, smem) != cudaSuccess)
            return 0;
    }
    return n;
}

template <int Q, class P, int K>
cudaError_t launch_batch(const void *bargs, unsigned grid, size_t smem, cudaStream_t s)
{
    static size_t granted[64] = {0};
    cudaError_t e = prepare(bfk::k_batch_mr<Q, P, K>, smem, granted);
    if (e != cudaSuccess) return e;
    bfk::k_batch_mr<Q, P, K><<<grid, bfk::CfgMR<Q>::NT, smem, s>>>(*static_cast<const bfk::BatchArgs<P> *>(bargs));
    return cudaGetLastError();
}

template <int Q, class P, int K>
int batch_ctas_per_sm(size_t smem)
{
    static size_t granted[64] = {0};
    if (prepare(bfk::k_batch_mr<Q, P, K>, smem, granted) != cudaSuccess) return 0;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, bfk::k_batch_mr<Q, P, K>, bfk::CfgMR<Q>::NT, smem) != cudaSuccess)
        return 0;
    return n;
}

// the switch kernel of operand format F (0 BF16, 1 TF32)
template <int Q, class P, int K, int F> struct KSW;
template <int Q, class P, int K> struct KSW<Q, P, K, 0> { static constexpr auto fn = bfk::k_switch_tc<Q, P, K>; };
template <int Q, class P, int K> struct KSW<Q, P, K, 1> { static constexpr auto fn = bfk::k_switch_tc32<Q, P, K>; };

template <int Q, class P, int K, int F>
cudaError_t launch_switch_tc(const void *kargs, unsigned gx, unsigned gy, size_t smem, cudaStream_t s)
{
    static size_t granted[64] = {0};
    cudaError_t e = prepare(KSW<Q, P, K, F>::fn, smem, granted);
    if (e != cudaSuccess) return e;
    KSW<Q, P, K, F>::fn<<<dim3(gx, gy), bfk::SwTC<Q, F>::NT, smem, s>>>(*static_cast<const bfk::KArgs<P> *>(kargs));
    return cudaGetLastError();
}

// CTAs of the tensor-core switch (operand format F) that fit on one SM by its registers, shared memory and
// threads (its grid is persistent, so a count above what the hardware keeps resident only
// queues CTAs; the occupancy query is taken when it allows more)
template <int Q, class P, int K, int F>
int switch_tc_ctas_per_sm()
{
    static size_t granted[64] = {0};
    if (prepare(KSW<Q, P, K, F>::fn, bfk::SwTC<Q, F>::SMEM, granted) != cudaSuccess) return 0;
    int dev = 0, n = 0;
    cudaFuncAttributes fa{};
    cudaDeviceProp pr{};
    if (cudaGetDevice(&dev) != cudaSuccess || cudaFuncGetAttributes(&fa, KSW<Q, P, K, F>::fn) != cudaSuccess ||
        cudaGetDeviceProperties(&pr, dev) != cudaSuccess)
        return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, KSW<Q, P, K, F>::fn, bfk::SwTC<Q, F>::NT,
                                                      bfk::SwTC<Q, F>::SMEM) != cudaSuccess)
        n = 0;
    const int warps = bfk::SwTC<Q, F>::NT / 32;
    const int regs_cta = warps * ((fa.numRegs * 32 + 255) / 256 * 256);
    const size_t smem_cta = bfk::SwTC<Q, F>::SMEM + fa.sharedSizeBytes + pr.reservedSharedMemPerBlock;
    int res = pr.maxBlocksPerMultiProcessor;
    if (regs_cta > 0 && pr.regsPerMultiprocessor / regs_cta < res) res = pr.regsPerMultiprocessor / regs_cta;
    if ((int)(pr.sharedMemPerMultiprocessor / smem_cta) < res) res = (int)(pr.sharedMemPerMultiprocessor / smem_cta);
    if (pr.maxThreadsPerMultiProcessor / bfk::SwTC<Q, F>::NT < res) res = pr.maxThreadsPerMultiProcessor / bfk::SwTC<Q, F>::NT;
    return n > res ? n : res;
}

template <int Q, class P, int K>
cudaError_t launch_col_tc(const void *kargs, unsigned gx, unsigned gy, size_t smem, cudaStream_t s)
{
    static size_t granted[64] = {0};
    cudaError_t e = prepare(bfk::k_col_tc<Q, P, K>, smem, granted);
    if (e != cudaSuccess) return e;
    bfk::k_col_tc<Q, P, K><<<dim3(gx, gy), bfk::ColTC<Q>::NT, smem, s>>>(*static_cast<const bfk::KArgs<P> *>(kargs));
    return cudaGetLastError();
}

// as switch_tc_ctas_per_sm, for the tensor-core column level
template <int Q, class P, int K>
int col_tc_ctas_per_sm()
{
    static size_t granted[64] = {0};
    if (prepare(bfk::k_col_tc<Q, P, K>, bfk::ColTC<Q>::SMEM, granted) != cudaSuccess) return 0;
    int dev = 0;
    cudaFuncAttributes fa{};
    cudaDeviceProp pr{};
    if (cudaGetDevice(&dev) != cudaSuccess || cudaFuncGetAttributes(&fa, bfk::k_col_tc<Q, P, K>) != cudaSuccess ||
        cudaGetDeviceProperties(&pr, dev) != cudaSuccess)
        return 0;
    const int regs_cta = (bfk::ColTC<Q>::NT / 32) * ((fa.numRegs * 32 + 255) / 256 * 256);
    const size_t smem_cta = bfk::ColTC<Q>::SMEM + fa.sharedSizeBytes + pr.reservedSharedMemPerBlock;
    int res = pr.maxBlocksPerMultiProcessor;
    if (regs_cta > 0 && pr.regsPerMultiprocessor / regs_cta < res) res = pr.regsPerMultiprocessor / regs_cta;
    if ((int)(pr.sharedMemPerMultiprocessor / smem_cta) < res) res = (int)(pr.sharedMemPerMultiprocessor / smem_cta);
    if (pr.maxThreadsPerMultiProcessor / bfk::ColTC<Q>::NT < res) res = pr.maxThreadsPerMultiProcessor / bfk::ColTC<Q>::NT;
    return res;
}

template <int D, int Q, class P, int K>
cudaError_t launch_ctab(const void *kargs, void *out, int levels)
{
    const int total = (int)((((uint32_t)1 << (D * (levels + 1))) - 1u) / ((1u << D) - 1u));
    const int blocks = (total + 255) / 256;
    bfk::k_center_table<P, D, Q, K><<<blocks < 4096 ? blocks : 4096, 256>>>(
        *static_cast<const bfk::KArgs<P> *>(kargs), static_cast<typename bfk::Ph<P, D, K>::T *>(out), levels);
    return cudaGetLastError();
}

template <int D, int Q, class P, int K>
const PassFns *fns_for()
{
    using CF = bfk::Cfg<D, Q, P>;
    if constexpr (D == 2 && !P::is_f64) {
        // single-RHS passes with a reduced-phase table (record, read): q <= 5
        constexpr bool TAB = Q <= 5;
        // tensor-core switch: q <= 5, polynomial sincos phases (the BF16x3 precision)
        constexpr bool TC = Q <= 5 && !P::sfu;
        constexpr int QT = TC ? Q : 2;
        static const PassFns f = {launch_col<D, Q, P, K>, launch_row<D, Q, P, K>, launch_col_adj<D, Q, P, K>,
                                  launch_row_adj<D, Q, P, K>, CF::KMAX, CF::NP, CF::NT,
                                  {launch_col_mr<Q, P, K, bfk::PM_COMPUTE>, launch_col_mr<Q, P, K, bfk::PM_BUILD>,
                                   launch_col_mr<Q, P, K, bfk::PM_TABLE>},
                                  {launch_row_mr<Q, P, K, bfk::PM_COMPUTE>, launch_row_mr<Q, P, K, bfk::PM_BUILD>,
                                   launch_row_mr<Q, P, K, bfk::PM_TABLE>},
                                  bfk::MRMAX, bfk::CfgMR<Q>::NT,
                                  launch_batch<Q, P, K>, batch_ctas_per_sm<Q, P, K>, mr_table_occupancy<Q, P, K>,
                                  launch_ctab<D, Q, P, K>, (int)sizeof(typename bfk::Ph<P, D, K>::T),
                                  {TAB ? launch_col<D, (TAB ? Q : 2), P, K, bfk::PM_BUILD> : nullptr,
                                   TAB ? launch_col<D, (TAB ? Q : 2), P, K, bfk::PM_TABLE> : nullptr},
                                  {TAB ? launch_row<D, (TAB ? Q : 2), P, K, bfk::PM_BUILD> : nullptr,
                                   TAB ? launch_row<D, (TAB ? Q : 2), P, K, bfk::PM_TABLE> : nullptr},
                                  TC ? launch_switch_tc<QT, P, K, 0> : nullptr,
                                  TC ? switch_tc_ctas_per_sm<QT, P, K, 0> : nullptr, TC ? bfk::SwTC<QT, 0>::SMEM : 0,
                                  TC ? launch_col_tc<QT, P, K> : nullptr,
                                  TC ? col_tc_ctas_per_sm<QT, P, K> : nullptr, TC ? bfk::ColTC<QT>::SMEM : 0,
                                  TC ? launch_switch_tc<QT, P, K, 1> : nullptr,
                                  TC ? switch_tc_ctas_per_sm<QT, P, K, 1> : nullptr, TC ? bfk::SwTC<QT, 1>::SMEM : 0};
        return &f;
    } else if constexpr (!P::is_f64) {
        // d = 3: single-RHS passes with a reduced-phase table; no multi-RHS kernels
        static const PassFns f = {launch_col<D, Q, P, K>, launch_row<D, Q, P, K>, launch_col_adj<D, Q, P, K>,
                                  launch_row_adj<D, Q, P, K>, CF::KMAX, CF::NP, CF::NT, {nullptr, nullptr, nullptr},
                                  {nullptr, nullptr, nullptr}, 0, 0, nullptr, nullptr, nullptr,
                                  launch_ctab<D, Q, P, K>, (int)sizeof(typename bfk::Ph<P, D, K>::T),
                                  {launch_col<D, Q, P, K, bfk::PM_BUILD>, launch_col<D, Q, P, K, bfk::PM_TABLE>},
                                  {launch_row<D, Q, P, K, bfk::PM_BUILD>, launch_row<D, Q, P, K, bfk::PM_TABLE>},
                                  nullptr, nullptr, 0, nullptr, nullptr, 0};
        return &f;
    } else {
        static const PassFns f = {launch_col<D, Q, P, K>, launch_row<D, Q, P, K>, launch_col_adj<D, Q, P, K>,
                                  launch_row_adj<D, Q, P, K>, CF::KMAX, CF::NP, CF::NT, {nullptr, nullptr, nullptr},
                                  {nullptr, nullptr, nullptr}, 0, 0, nullptr, nullptr, nullptr,
                                  launch_ctab<D, Q, P, K>, (int)sizeof(typename bfk::Ph<P, D, K>::T),
                                  {nullptr, nullptr}, {nullptr, nullptr}, nullptr, nullptr, 0, nullptr, nullptr, 0};
        return &f;
    }
}

}  // namespace bfl
