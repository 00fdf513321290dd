// The middle switch of the butterfly (Section 1.4) on the tensor cores, for several right-
// hand sides at once (d = 2, q <= 5, mixed-precision phases).
//
// At level m every pair (A, B) maps its weights through the r x r matrix
//     E[s][t] = e^{2 pi i Phi(x_s^A, y_t^B)},      delta_s <- sum_t E[s][t] delta_t,
// for every right-hand side: a complex (r x r) . (r x nrhs) product per pair, in which
// each evaluated phase factor serves all right-hand sides.  Here it is a real GEMM on
// tcgen05 tensor cores, D = A B^T with
//     A[(s, c)][(t, c')]  rows 2s (real part of the result), 2s + 1 (imaginary part),
//                         columns 2t (weight's real part), 2t + 1 (imaginary part):
//                         [Re E, -Im E] in row 2s, [Im E, Re E] in row 2s + 1;
//     B[rhs][(t, c')]     the weights of one right-hand side, as stored (re, im, re, ...),
// so D[2s][rhs] = Re(E w)_s and D[2s + 1][rhs] = Im(E w)_s.  Two pairs share one MMA of
// M = 128 rows (64 per pair, 2r of them used) and N = 32 columns (16 right-hand sides
// per pair); the off-diagonal blocks of D are computed and ignored.  Along K the source
// nodes t = t_0 + q t_1 are grouped by t_1: the 2q values of digit t_1 fill a slot of 8 or
// 16 elements (whole 16-byte pieces of a row), so each evaluating thread writes whole
// pieces; the rest of a slot stays zero.
//
// Precision (BF16x3): every FP32 operand x is split into BF16 parts hi = bf16(x) and
// lo = bf16(x - hi) (16 significant bits together), and D accumulates hi.hi + hi.lo +
// lo.hi in FP32 in tensor memory; the dropped lo.lo term and the rounding of lo are
// below 2^-17 relative per product.  TF32x3 does the same with TF32 parts (22 significant
// bits together, kind::tf32, one value per 32-bit word): ~2^-22 relative per product.
// The phase factors are those of the CUDA-core multi-RHS switch, evaluated with the same
// code.  The column merge level on the tensor cores (ColTC, below) uses BF16x3 only.
#pragma once

#include "bf_mr.cuh"
#include "bf_umma.cuh"

namespace bfk {

// wait for phase `parity` of an mbarrier; false after limit_ns nanoseconds
__device__ __forceinline__ bool mbar_wait_ns(uint64_t *bar, unsigned parity, uint64_t limit_ns)
{
    const uint64_t t0 = globaltimer_ns();
    while (!mbar_try_wait(bar, parity))
        if (globaltimer_ns() - t0 > limit_ns) return false;
    return true;
}

constexpr uint64_t TC_WAIT_NS = 2000000000ull;   // 2 s: an MMA group takes microseconds

// operand formats of the tensor-core switch.  Both split every FP32 operand x into
// hi + lo and accumulate hi.hi + hi.lo + lo.hi in FP32 (the dropped lo.lo is below the
// format's rounding): F = 0 BF16 parts (kind::f16, two values per 32-bit word, K = 16 per
// MMA; ~2^-17 relative per product), F = 1 TF32 parts (kind::tf32, one value per word,
// K = 8 per MMA; ~2^-22 relative per product, at the level of FP32 rounding).
template <int F> struct TcFmt;
template <> struct TcFmt<0> {
    static constexpr int EPC = 8;      // elements per 16-byte row piece of a core matrix
    static constexpr int KSTEP = 16;   // K of one MMA
    static constexpr int WPC = 1;      // 32-bit words of one complex value (x, y) along K
    // the hi and lo words of (x, y) as stored along K (first value low)
    static __device__ __forceinline__ void split(float x, float y, uint32_t *h, uint32_t *l) { umma::split2(x, y, h[0], l[0]); }
    // the words of (x, -y) and of (y, x) from those of (x, y)
    static __device__ __forceinline__ void neg_y(const uint32_t *w, uint32_t *o) { o[0] = w[0] ^ 0x80000000u; }
    static __device__ __forceinline__ void swap(const uint32_t *w, uint32_t *o) { o[0] = __byte_perm(w[0], 0u, 0x1032); }
    static __host__ __device__ constexpr uint32_t idesc(int M, int N) { return umma::idesc_bf16_f32(M, N); }
    static __device__ __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t id, int acc) { umma::mma_bf16(d, a, b, id, acc); }
};
template <> struct TcFmt<1> {
    static constexpr int EPC = 4;
    static constexpr int KSTEP = 8;
    static constexpr int WPC = 2;
    static __device__ __forceinline__ void split(float x, float y, uint32_t *h, uint32_t *l)
    {
        umma::split_tf32(x, h[0], l[0]);
        umma::split_tf32(y, h[1], l[1]);
    }
    static __device__ __forceinline__ void neg_y(const uint32_t *w, uint32_t *o) { o[0] = w[0]; o[1] = w[1] ^ 0x80000000u; }
    static __device__ __forceinline__ void swap(const uint32_t *w, uint32_t *o) { o[0] = w[1]; o[1] = w[0]; }
    static __host__ __device__ constexpr uint32_t idesc(int M, int N) { return umma::idesc_tf32_f32(M, N); }
    static __device__ __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t id, int acc) { umma::mma_tf32(d, a, b, id, acc); }
};

template <int Q, int F = 0>
struct SwTC {
    using FM = TcFmt<F>;
    static constexpr int RR = Q * Q;                        // r
    static constexpr int UP = 2;                            // pairs per MMA
    static constexpr int ROWS = 64;                         // MMA rows per pair
    static constexpr int NPP = 16;                          // right-hand sides (B rows) per pair
    static constexpr int M = UP * ROWS, N = UP * NPP;       // 128 x 32 accumulator
    // BF16 parts: the 2r rows of pair 1 start at row PS (the first 8-row group after pair
    // 0's), so one part of A holds A_GROUPS groups; the MMA reads M rows, and the rows past
    // the part (the start of the next parts: lo of A, then B) only reach accumulator rows
    // that nothing reads.  Where those rows would reach past B, a part keeps all M rows.
    // At q = 5 this takes the shared memory from 59 to 54 KB: four CTAs per SM instead of
    // three (switch 0.91 -> 0.88 ms at N = 512, 16 right-hand sides).  TF32 parts keep
    // 64-row blocks: two CTAs per SM either way, and the compact form measured 2% slower.
    static constexpr int PS = F == 0 ? (2 * RR + 7) / 8 * 8 : ROWS;
    static constexpr int A_USED = (PS + 2 * RR + 7) / 8;
    static constexpr int A_GROUPS = M / 8 - A_USED <= 2 * (N / 8) ? A_USED : M / 8;
    static constexpr int SLOT = 2 * Q <= 8 ? 8 : 16;        // K elements per source digit t_1
    static constexpr int PIECES = SLOT / FM::EPC;           // 16-byte pieces per slot and row
    static constexpr int NWS = Q * FM::WPC;                 // 32-bit words of a slot's 2q values
    static constexpr int KP = (SLOT * Q + FM::KSTEP - 1) / FM::KSTEP * FM::KSTEP;   // K, padded to the MMA's K step
    static constexpr int NKS = KP / FM::KSTEP;              // K steps
    static constexpr uint32_t LBO = 128;                    // core matrices along K: adjacent
    static constexpr uint32_t SBO = (KP / FM::EPC) * 128;   // 8-row groups
    static constexpr uint32_t A_BYTES = A_GROUPS * SBO;     // one part (hi or lo) of A
    static constexpr uint32_t B_BYTES = (N / 8) * SBO;      // one part of B
    static constexpr int NT = 256;                          // threads: 8 warps
    static constexpr int TMEM_COLS = 32;
    static constexpr uint32_t W_BYTES = NPP * UP * RR * 8;  // a unit's weights as stored (complex64)
    static constexpr int W_CHUNKS = W_BYTES / 16;           // 16-byte copies per unit
    static constexpr uint32_t T_BYTES = UP * RR * 32;       // target features of the unit's nodes
    static constexpr size_t SMEM = 2 * (size_t)A_BYTES + 2 * (size_t)B_BYTES + W_BYTES + T_BYTES + 64;
    static_assert(2 * RR <= ROWS, "the tensor-core switch holds r <= 32");
    static_assert(PS + 2 * RR <= M && A_GROUPS <= M / 8, "both pairs' rows lie in the M rows of the MMA");
    static_assert((M / 8 - A_GROUPS) * SBO <= 2 * B_BYTES, "the rows the MMA reads past a part lie in the next parts");
    static_assert(UP * RR * Q <= NT && UP * NPP * Q + UP * RR <= NT, "one item per thread");
    static_assert((UP * RR * 8) % 16 == 0, "a unit's weights per right-hand side are whole 16-byte pieces");
    static_assert(NWS <= 4 * PIECES, "a slot's values fit its pieces");
};

// Switch pass: reads the level-m weights a.win ([rhs][pair][r], pair = A 2^{2(L-m)} + B),
// writes the switched weights to a.wout in the same layout.  Right-hand sides
// 16 blockIdx.y .. +15; units of two consecutive pairs taken blockIdx.x, + gridDim.x, ...
// The weights of a unit (per right-hand side the two pairs' 2r complex numbers, contiguous
// and 16-byte aligned) are copied into shared memory with cp.async one unit ahead, so the
// loads overlap the previous unit's phase evaluation.
// A completion wait that gives up sets *a.err, waits once more (bounded), frees the
// tensor memory and ends the kernel (the outputs are then undefined).
template <int Q, class P, int K, int F>
__device__ __forceinline__ void switch_tc_body(const KArgs<P> &a)
{
    using ST = SwTC<Q, F>;
    using FM = typename ST::FM;
    using C = typename P::C;
    using PH = Ph<P, 2, K>;
    using PH2 = Ph2<P, 2, K>;
    using TT = typename PH::T;
    static_assert(sizeof(TT) <= 32, "target features fit their shared-memory slot");
    constexpr int RR = ST::RR, D = 2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned char *Ah = smem_raw, *Al = Ah + ST::A_BYTES, *Bh = Al + ST::A_BYTES, *Bl = Bh + ST::B_BYTES;
    unsigned char *Wst = Bl + ST::B_BYTES;                          // the unit's weights
    TT *Ts = reinterpret_cast<TT *>(Wst + ST::W_BYTES);             // target features, [pair][s]
    uint64_t *bar = reinterpret_cast<uint64_t *>(Wst + ST::W_BYTES + ST::T_BYTES);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bar + 1);
    int *sfail = reinterpret_cast<int *>(tslot + 1);
    uint64_t *wbar = reinterpret_cast<uint64_t *>(sfail + 1);       // the tiled copies of the weights
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // a unit's weights arrive by one tiled bulk copy when the plan has a tensor map of the
    // input (the staging buffer is 128-byte aligned), else by 16-byte cp.async copies
    const bool use_tma = a.wmap != nullptr && (umma::saddr(Wst) & 127u) == 0u;

    // operands start at zero: the padding rows and slots are never written again
    {
        uint4 *z = reinterpret_cast<uint4 *>(smem_raw);
        const int n16 = (int)((2 * ST::A_BYTES + 2 * ST::B_BYTES) / 16);
        for (int i = tid; i < n16; i += ST::NT) z[i] = make_uint4(0u, 0u, 0u, 0u);
    }
    if (warp == 0) umma::alloc(tslot, ST::TMEM_COLS);
    if (tid == 0) {
        mbar_init(bar, 1);
        mbar_init(wbar, 1);
        mbar_init_fence();
        *sfail = 0;
    }
    umma::fence_before_sync();
    __syncthreads();
    umma::fence_after_sync();
    const uint32_t tmem = *tslot;

    const int l = a.l0, L = a.L;
    const int shB = D * (L - l);
    const uint32_t maskB = (1u << shB) - 1u;
    // units (two consecutive pairs); sharding mode 1: the launch covers the rank's units only
    // (those whose source boxes carry its top bits), unit v of the launch is unit uid(v)
    const int64_t nunits = (a.npts / ST::UP) >> (a.shard_mode == 1 ? a.shard_g : 0);
    auto uid = [&](int64_t v) -> int64_t {
        if (a.shard_mode != 1) return v;
        const int lper = shB - 1 - a.shard_g;            // log2 of the rank's units per target box
        return ((v >> lper) << (shB - 1)) | ((int64_t)a.shard_r << lper) | (v & ((1LL << lper) - 1));
    };
    const int rhs0 = (int)blockIdx.y * ST::NPP;
    const int nr = min(ST::NPP, a.nrhs - rhs0);
    const uint32_t idesc = FM::idesc(ST::M, ST::N);
    unsigned parity = 0;

    // weights of unit v into the staging buffer: per right-hand side rb < nr, the two pairs'
    // 2r complex numbers.  Tiled: one copy of the box (2r complex numbers x 16 right-hand
    // sides) at (unit offset, first right-hand side), rows past the last right-hand side read
    // as zero; its phase of wbar completes when the bytes have landed.  Else 16-byte pieces,
    // one commit group per call.
    unsigned wpar = 0;       // phase of wbar the next wait expects
    bool inflight = false;   // a tiled copy was issued and not yet waited for
    auto fetch = [&](int64_t v) {
        if (use_tma) {
            if (v < nunits) {
                if (tid == 0) {
                    fence_proxy_async();   // the generic reads of the staging buffer come first
                    mbar_expect_tx(wbar, ST::W_BYTES);
                    bulk_tensor_2d_g2s(Wst, a.wmap, (int)(uid(v) * ST::UP * RR), rhs0, wbar);
                }
                inflight = true;
            }
            return;
        }
        constexpr int per_rhs = ST::W_CHUNKS / ST::NPP;
        if (v < nunits) {
            for (int c = tid; c < nr * per_rhs; c += ST::NT) {
                const int rb = c / per_rhs, o = c - rb * per_rhs;
                const char *src =
                    reinterpret_cast<const char *>(a.win + (int64_t)(rhs0 + rb) * a.wstride + uid(v) * ST::UP * RR) + 16 * o;
                const uint32_t dst = umma::saddr(Wst + rb * (ST::W_BYTES / ST::NPP) + 16 * o);
                asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
            }
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    // slot th of row `row` in a part: PIECES 16-byte pieces (the NWS words of 2q values,
    // then zeros)
    auto put_slot = [&](unsigned char *base, int row, int th, const uint32_t *w) {
#pragma unroll
        for (int pc = 0; pc < ST::PIECES; ++pc) {
            uint4 v;
            v.x = 4 * pc + 0 < ST::NWS ? w[4 * pc + 0] : 0u;
            v.y = 4 * pc + 1 < ST::NWS ? w[4 * pc + 1] : 0u;
            v.z = 4 * pc + 2 < ST::NWS ? w[4 * pc + 2] : 0u;
            v.w = 4 * pc + 3 < ST::NWS ? w[4 * pc + 3] : 0u;
            *reinterpret_cast<uint4 *>(base + umma::kmajor_piece_off(row, ST::SLOT / FM::EPC * th + pc, ST::LBO, ST::SBO)) = v;
        }
    };
    fetch(blockIdx.x);

    for (int64_t u = blockIdx.x; u < nunits; u += gridDim.x) {
        if (use_tma) {   // every thread waits for the unit's weights (bounded)
            if (!mbar_wait_ns(wbar, wpar, TC_WAIT_NS)) {
                if (a.err) atomicExch(a.err, 1);
                *sfail = 1;
            }
            wpar ^= 1u;
            inflight = false;
        } else {
            asm volatile("cp.async.wait_group 0;" ::: "memory");   // the unit's weights have landed
        }
        __syncthreads();
        if (*sfail) break;
        // ---- B: items (rhs, pair, t_1): q weights, split into hi and lo parts, one slot each
        {
            const int rb = tid % ST::NPP, up = (tid / ST::NPP) % ST::UP, th = tid / (ST::NPP * ST::UP);
            if (th < Q && rb < nr) {
                const C *w = reinterpret_cast<const C *>(Wst) + (rb * ST::UP + up) * RR + Q * th;
                uint32_t hi[ST::NWS], lo[ST::NWS];
#pragma unroll
                for (int t0 = 0; t0 < Q; ++t0) FM::split(w[t0].x, w[t0].y, hi + FM::WPC * t0, lo + FM::WPC * t0);
                put_slot(Bh, up * ST::NPP + rb, th, hi);
                put_slot(Bl, up * ST::NPP + rb, th, lo);
            }
        }
        // ---- target features of the unit's nodes (pair, s), once per node, by the threads
        // that have no weight item
        if (tid >= ST::UP * ST::NPP * Q && tid < ST::UP * ST::NPP * Q + ST::UP * RR) {
            const int it = tid - ST::UP * ST::NPP * Q;
            const int s = it % RR, up = it / RR;
            const uint32_t I = (uint32_t)(uid(u) * ST::UP + up);
            int ca[DMAX];
            morton_decode<D>(I >> shB, l, ca);
            const int sk[DMAX] = {s % Q, s / Q, 0};
            Ts[it] = tpoint<P, D, Q, K>(a, l, ca, sk);
        }
        __syncthreads();
        fetch(u + gridDim.x);   // the staging buffer is free again: the next unit's copies overlap this one
        // ---- A: items (pair, t_1, s), s fastest: q factors e^{2 pi i Phi(x_s^A, y_t^B)} each,
        // evaluated as in the CUDA-core multi-RHS switch, split into the rows 2s, 2s + 1 of slot t_1
        for (int it = tid; it < ST::UP * RR * Q; it += ST::NT) {
            const int s = it % RR, th = (it / RR) % Q, up = it / (RR * Q);
            const uint32_t I = (uint32_t)(uid(u) * ST::UP + up);
            int cb[DMAX];
            morton_decode<D>(I & maskB, L - l, cb);
            const TT tS = Ts[up * RR + s];
            C ev[Q];
            const typename PH2::T tS2 = PH2::dup(tS);
            const typename P::SE e1 = sget<P, Q>(a, 1, l, cb[1], th);
            const typename PH2::Part hp = PH2::part(tS2, e1, e1, 1);
#pragma unroll
            for (int t0 = 0; t0 + 1 < Q; t0 += 2)
                expphase_part2<P, D, K>(
                    a, tS2, PH2::add(PH2::part(tS2, sget<P, Q>(a, 0, l, cb[0], t0), sget<P, Q>(a, 0, l, cb[0], t0 + 1), 0), hp),
                    ev[t0], ev[t0 + 1]);
            if constexpr (Q & 1)
                ev[Q - 1] = expphase_part<P, D, K>(a, tS, PH::add(PH::part(tS, sget<P, Q>(a, 0, l, cb[0], Q - 1), 0),
                                                                 PH2::lane0(hp)));
            // row 2s takes (x, -y), row 2s + 1 takes (y, x) of every factor x + iy
            uint32_t h0[ST::NWS], l0[ST::NWS], h1[ST::NWS], l1[ST::NWS];
#pragma unroll
            for (int t0 = 0; t0 < Q; ++t0) {
                uint32_t h[FM::WPC], l[FM::WPC];
                FM::split(ev[t0].x, ev[t0].y, h, l);
                FM::neg_y(h, h0 + FM::WPC * t0);
                FM::neg_y(l, l0 + FM::WPC * t0);
                FM::swap(h, h1 + FM::WPC * t0);
                FM::swap(l, l1 + FM::WPC * t0);
            }
            const int r0 = up * ST::PS + 2 * s;
            put_slot(Ah, r0, th, h0);
            put_slot(Al, r0, th, l0);
            put_slot(Ah, r0 + 1, th, h1);
            put_slot(Al, r0 + 1, th, l1);
        }
        umma::fence_smem_to_async();
        __syncthreads();
        // ---- D = Ah Bh^T + Ah Bl^T + Al Bh^T, one thread issues; completion on the mbarrier
        if (tid == 0) {
            umma::fence_after_sync();
            const uint32_t ah = umma::saddr(Ah), al = umma::saddr(Al), bh = umma::saddr(Bh), bl = umma::saddr(Bl);
#pragma unroll
            for (int ks = 0; ks < ST::NKS; ++ks) {
                const uint32_t o = (uint32_t)ks * 2u * ST::LBO;
                const uint64_t dah = umma::desc_kmajor(ah + o, ST::LBO, ST::SBO);
                const uint64_t dal = umma::desc_kmajor(al + o, ST::LBO, ST::SBO);
                const uint64_t dbh = umma::desc_kmajor(bh + o, ST::LBO, ST::SBO);
                const uint64_t dbl = umma::desc_kmajor(bl + o, ST::LBO, ST::SBO);
                FM::mma(tmem, dah, dbh, idesc, ks > 0);
                FM::mma(tmem, dah, dbl, idesc, 1);
                FM::mma(tmem, dal, dbh, idesc, 1);
            }
            umma::commit(bar);
            if (!mbar_wait_ns(bar, parity, TC_WAIT_NS)) {
                if (a.err) atomicExch(a.err, 1);
                *sfail = 1;
                mbar_wait_ns(bar, parity, TC_WAIT_NS);
            }
        }
        parity ^= 1u;
        __syncthreads();
        if (*sfail) break;
        umma::fence_after_sync();
        // ---- epilogue: warp w reads lanes 32 (w % 4) .. + 31 (row 32 (w % 4) + lane: rows
        // 2s + c of pair 0, or of pair 1 from row PS on), columns of the lane's pair's right-
        // hand sides 8 (w / 4) .. + 7 (a quarter that holds rows of both pairs reads both
        // column blocks); lanes 2s and 2s + 1 swap halves so that each writes complete
        // complex numbers
        {
            const int quad = warp & 3, half = warp >> 2;
            const int row = 32 * quad + lane, up = row >= ST::PS ? 1 : 0, loc = row - up * ST::PS;
            const int s = loc >> 1, c = lane & 1;
            const int pa = 32 * quad >= ST::PS ? 1 : 0, pb = 32 * quad + 31 >= ST::PS ? 1 : 0;   // warp-uniform
            const uint32_t lanes = (uint32_t)(32 * quad) << 16;
            float v[8];
            umma::ld8(tmem + lanes + (uint32_t)(pa * ST::NPP + 8 * half), v);
            if (pb != pa) {
                float w[8];
                umma::ld8(tmem + lanes + (uint32_t)(pb * ST::NPP + 8 * half), w);
                if (up == pb) {
#pragma unroll
                    for (int j = 0; j < 8; ++j) v[j] = w[j];
                }
            }
            float recv[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) recv[j] = __shfl_xor_sync(0xffffffffu, c ? v[j] : v[4 + j], 1);
            if (s < RR) {
                const int64_t pair = uid(u) * ST::UP + up;
                C *wo = a.wout + pair * RR + s;
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int rb = 8 * half + 4 * c + j;
                    if (rb < nr) {
                        C z;
                        z.x = c ? recv[j] : v[j];
                        z.y = c ? v[4 + j] : recv[j];
                        __stcs(wo + (int64_t)(rhs0 + rb) * a.wstride, z);
                    }
                }
            }
        }
        // the next unit's first barrier orders these tensor-memory reads before its MMAs
        umma::fence_before_sync();
    }
    asm volatile("cp.async.wait_all;" ::: "memory");   // no copy outlives the kernel
    if (use_tma && inflight && tid == 0) mbar_wait_ns(wbar, wpar, TC_WAIT_NS);
    umma::fence_before_sync();
    __syncthreads();
    if (warp == 0) umma::dealloc(tmem, ST::TMEM_COLS);
}

// The switch kernels of the two operand formats.  BF16 keeps the compiler's default register
// target (64 registers; three CTAs fit an SM by shared memory; an explicit bound measured
// 8% slower), TF32 is compiled for two CTAs per SM, which its shared memory admits (89
// registers; with 64 its staging code spilled).
template <int Q, class P, int K>
__global__ void __launch_bounds__(SwTC<Q, 0>::NT) k_switch_tc(const KArgs<P> a)
{
    switch_tc_body<Q, P, K, 0>(a);
}
template <int Q, class P, int K>
__global__ void __launch_bounds__(SwTC<Q, 1>::NT, 2) k_switch_tc32(const KArgs<P> a)
{
    switch_tc_body<Q, P, K, 1>(a);
}

// ============================================================================
// One column-form merge level (Section 1.4) on the tensor cores, for several right-hand
// sides: per merge block (target box A at level l, parent source box B_p at level l+1; its
// inputs are the 4 consecutive pairs (A, B_c), its outputs the pairs (A_alpha, B_p))
//     w_out(alpha, t) = conj(e_d(alpha, t)) sum_{c, t'} Mk[t][(c, t')] e_m(alpha, c, t') w_c(t')
// with e_m = e^{2 pi i Phi(x0(A_alpha), y_t'^{B_c})} (modulation), e_d = e^{2 pi i Phi(x0(A_alpha),
// y_t^{B_p})} (demodulation) and Mk the constant Kronecker product M_{c_0}(t_0, t'_0)
// M_{c_1}(t_1, t'_1) of the child->parent matrices.  The sum is a real GEMM D = A Bt:
//     A[(alpha, rhs, re/im)][(c, t')]  the modulated inputs u = e_m w_c, split re / im over
//                                      rows: 4 x 16 x 2 = 128 rows (M = 128);
//     B[t][(c, t')] = Mk               N = 32 (r <= 25 used), the same for every block;
//     K = (c, t') in slots of 32 per child c: 128 (4 r used), 8 MMA steps.
// BF16x3 split of both operands, FP32 accumulation in tensor memory, as in the switch.
template <int Q>
struct ColTC {
    static constexpr int RR = Q * Q;
    static constexpr int NPP = 16;                          // right-hand sides per block
    static constexpr int KS = 32;                           // K slot per input child
    static constexpr int M = 128, N = 32, KP = 4 * KS, NKS = KP / 16;
    static constexpr uint32_t LBO = 128, SBO = (KP / 8) * 128;
    static constexpr uint32_t A_BYTES = (M / 8) * SBO;      // one BF16 part of A (32 KB)
    static constexpr uint32_t B_BYTES = (N / 8) * SBO;      // one BF16 part of B (8 KB)
    static constexpr int NT = 256;
    static constexpr int TMEM_COLS = 32;
    static constexpr uint32_t W_BYTES = NPP * 4 * RR * 8;   // a block's inputs for 16 right-hand sides
    static constexpr size_t SMEM = 2 * (size_t)A_BYTES + 2 * (size_t)B_BYTES + W_BYTES + 5 * 4 * RR * 8 + 64;
    static_assert(RR <= 32 && RR <= KS, "one slot per child holds its r nodes");
    static_assert((4 * RR * 8) % 16 == 0, "a block's inputs per right-hand side are whole 16-byte pieces");
};

// Column level l -> l+1 (a.l0 = l): reads a.win (level l), writes a.wout (level l+1), both
// [rhs][pair][r]; right-hand sides 16 blockIdx.y .. +15; blocks taken blockIdx.x, + gridDim.x.
// Sharding mode 1: the launch covers the blocks whose parent source box carries the rank's bits.
template <int Q, class P, int K>
__global__ void __launch_bounds__(ColTC<Q>::NT) k_col_tc(const KArgs<P> a)
{
    using ST = ColTC<Q>;
    using C = typename P::C;
    using PH = Ph<P, 2, K>;
    constexpr int RR = ST::RR, D = 2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned char *Ah = smem_raw, *Al = Ah + ST::A_BYTES, *Bh = Al + ST::A_BYTES, *Bl = Bh + ST::B_BYTES;
    unsigned char *Wst = Bl + ST::B_BYTES;                                   // [rhs][c][t'] inputs
    C *PM = reinterpret_cast<C *>(Wst + ST::W_BYTES);                        // [alpha][c][t'] e_m
    C *PD = PM + 4 * 4 * RR;                                                 // [alpha][t]      e_d
    uint64_t *bar = reinterpret_cast<uint64_t *>(PD + 4 * RR);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bar + 1);
    int *sfail = reinterpret_cast<int *>(tslot + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    {
        uint4 *z = reinterpret_cast<uint4 *>(smem_raw);
        const int n16 = (int)((2 * ST::A_BYTES + 2 * ST::B_BYTES) / 16);
        for (int i = tid; i < n16; i += ST::NT) z[i] = make_uint4(0u, 0u, 0u, 0u);
    }
    if (warp == 0) umma::alloc(tslot, ST::TMEM_COLS);
    if (tid == 0) {
        mbar_init(bar, 1);
        mbar_init_fence();
        *sfail = 0;
    }
    umma::fence_before_sync();
    __syncthreads();
    umma::fence_after_sync();
    const uint32_t tmem = *tslot;
    // B = Mk, once: items (t, c), rows t, slot c
    for (int it = tid; it < RR * 4; it += ST::NT) {
        const int t = it % RR, c = it / RR, t0 = t % Q, t1 = t / Q, c0 = c & 1, c1 = c >> 1;
        for (int j = 0; j < RR; j += 2) {
            const float m0 = a.M[c0][t0][j % Q] * a.M[c1][t1][j / Q];
            const float m1 = j + 1 < RR ? a.M[c0][t0][(j + 1) % Q] * a.M[c1][t1][(j + 1) / Q] : 0.0f;
            uint32_t hi, lo;
            umma::split2(m0, m1, hi, lo);
            const uint32_t off = umma::kmajor_off(t, ST::KS * c + j, ST::LBO, ST::SBO);
            *reinterpret_cast<uint32_t *>(Bh + off) = hi;
            *reinterpret_cast<uint32_t *>(Bl + off) = lo;
        }
    }

    const int l = a.l0, L = a.L;
    const int lbp = D * (L - l - 1);                      // log2 of the parent source boxes per target box
    const int64_t nunits = (a.npts / 4) >> (a.shard_mode == 1 ? a.shard_g : 0);
    auto uid = [&](int64_t v) -> int64_t {
        if (a.shard_mode != 1) return v;
        const int lper = lbp - a.shard_g;
        return ((v >> lper) << lbp) | ((int64_t)a.shard_r << lper) | (v & ((1LL << lper) - 1));
    };
    const int rhs0 = (int)blockIdx.y * ST::NPP;
    const int nr = min(ST::NPP, a.nrhs - rhs0);
    const uint32_t idesc = umma::idesc_bf16_f32(ST::M, ST::N);
    unsigned parity = 0;

    auto fetch = [&](int64_t v) {
        constexpr int per_rhs = 4 * RR * 8 / 16;
        if (v < nunits) {
            for (int c = tid; c < nr * per_rhs; c += ST::NT) {
                const int rb = c / per_rhs, o = c - rb * per_rhs;
                const char *src = reinterpret_cast<const char *>(a.win + (int64_t)(rhs0 + rb) * a.wstride + 4 * uid(v) * RR) + 16 * o;
                const uint32_t dst = umma::saddr(Wst + rb * (4 * RR * 8) + 16 * o);
                asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
            }
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    fetch(blockIdx.x);

    for (int64_t u = blockIdx.x; u < nunits; u += gridDim.x) {
        const int64_t U = uid(u);                          // block: target box A, parent source box B_p
        const uint32_t A = (uint32_t)(U >> lbp), Bp = (uint32_t)(U & ((1LL << lbp) - 1));
        int cbq[DMAX];
        morton_decode<D>(Bp, L - l - 1, cbq);
        // ---- phase factors: e_m (alpha, c, t') and e_d (alpha, t)
        for (int it = tid; it < 4 * 4 * RR + 4 * RR; it += ST::NT) {
            const bool mod = it < 16 * RR;
            const int jt = mod ? it : it - 16 * RR;
            const int alpha = jt / (mod ? 4 * RR : RR), rest = jt % (mod ? 4 * RR : RR);
            const uint32_t Aa = (A << D) + alpha;
            int ca[DMAX];
            morton_decode<D>(Aa, l + 1, ca);
            const typename PH::T tA = tcenter<P, D, Q, K>(a, l + 1, Aa, ca);
            if (mod) {
                const int c = rest / RR, tp = rest % RR;
                const typename PH::Part pt = PH::add(PH::part(tA, sget<P, Q>(a, 0, l, 2 * cbq[0] + (c & 1), tp % Q), 0),
                                                     PH::part(tA, sget<P, Q>(a, 1, l, 2 * cbq[1] + (c >> 1), tp / Q), 1));
                PM[jt] = expphase_part<P, D, K>(a, tA, pt);
            } else {
                const typename PH::Part pt = PH::add(PH::part(tA, sget<P, Q>(a, 0, l + 1, cbq[0], rest % Q), 0),
                                                     PH::part(tA, sget<P, Q>(a, 1, l + 1, cbq[1], rest / Q), 1));
                PD[jt] = expphase_part<P, D, K>(a, tA, pt);
            }
        }
        asm volatile("cp.async.wait_group 0;" ::: "memory");   // the block's inputs have landed
        __syncthreads();
        // ---- A: items (rhs, c, alpha), rhs fastest: u = e_m w_c over the slot of c, rows re / im
        {
            const int rb = tid % ST::NPP, c = (tid / ST::NPP) % 4, alpha = tid / (4 * ST::NPP);
            if (rb < nr) {
                const C *w = reinterpret_cast<const C *>(Wst) + (rb * 4 + c) * RR;
                const C *e = PM + (alpha * 4 + c) * RR;
                const int row = 32 * alpha + 2 * rb;
#pragma unroll
                for (int pc = 0; pc < ST::KS / 8; ++pc) {
                    uint32_t rh[4], rl[4], ih[4], il[4];
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const int t0 = 8 * pc + 2 * j, t1 = t0 + 1;
                        const C u0 = t0 < RR ? cmul(e[t0], w[t0]) : czero<C>();
                        const C u1 = t1 < RR ? cmul(e[t1], w[t1]) : czero<C>();
                        umma::split2(u0.x, u1.x, rh[j], rl[j]);
                        umma::split2(u0.y, u1.y, ih[j], il[j]);
                    }
                    const int k = ST::KS * c + 8 * pc;
                    *reinterpret_cast<uint4 *>(Ah + umma::kmajor_off(row, k, ST::LBO, ST::SBO)) = make_uint4(rh[0], rh[1], rh[2], rh[3]);
                    *reinterpret_cast<uint4 *>(Al + umma::kmajor_off(row, k, ST::LBO, ST::SBO)) = make_uint4(rl[0], rl[1], rl[2], rl[3]);
                    *reinterpret_cast<uint4 *>(Ah + umma::kmajor_off(row + 1, k, ST::LBO, ST::SBO)) = make_uint4(ih[0], ih[1], ih[2], ih[3]);
                    *reinterpret_cast<uint4 *>(Al + umma::kmajor_off(row + 1, k, ST::LBO, ST::SBO)) = make_uint4(il[0], il[1], il[2], il[3]);
                }
            }
        }
        umma::fence_smem_to_async();
        __syncthreads();
        fetch(u + gridDim.x);   // every A item has read the staging buffer: the next block's copies overlap the rest
        if (tid == 0) {
            umma::fence_after_sync();
            const uint32_t ah = umma::saddr(Ah), al = umma::saddr(Al), bh = umma::saddr(Bh), bl = umma::saddr(Bl);
#pragma unroll
            for (int ks = 0; ks < ST::NKS; ++ks) {
                const uint32_t o = (uint32_t)ks * 2u * ST::LBO;
                const uint64_t dah = umma::desc_kmajor(ah + o, ST::LBO, ST::SBO);
                const uint64_t dal = umma::desc_kmajor(al + o, ST::LBO, ST::SBO);
                const uint64_t dbh = umma::desc_kmajor(bh + o, ST::LBO, ST::SBO);
                const uint64_t dbl = umma::desc_kmajor(bl + o, ST::LBO, ST::SBO);
                umma::mma_bf16(tmem, dah, dbh, idesc, ks > 0);
                umma::mma_bf16(tmem, dah, dbl, idesc, 1);
                umma::mma_bf16(tmem, dal, dbh, idesc, 1);
            }
            umma::commit(bar);
            if (!mbar_wait_ns(bar, parity, TC_WAIT_NS)) {
                if (a.err) atomicExch(a.err, 1);
                *sfail = 1;
                mbar_wait_ns(bar, parity, TC_WAIT_NS);
            }
        }
        parity ^= 1u;
        __syncthreads();
        if (*sfail) break;
        umma::fence_after_sync();
        // ---- epilogue: warp w reads the rows of child alpha = w % 4 (lane = 2 rhs + re/im),
        // columns t = 16 (w / 4) .. + 15; lanes 2 rhs and 2 rhs + 1 swap halves, demodulate, store
        {
            const int alpha = warp & 3, half = warp >> 2, rb = lane >> 1, cmp = lane & 1;
            float v[16];
            umma::ld8(tmem + ((uint32_t)(32 * alpha) << 16) + (uint32_t)(16 * half), v);
            umma::ld8(tmem + ((uint32_t)(32 * alpha) << 16) + (uint32_t)(16 * half + 8), v + 8);
            float recv[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) recv[j] = __shfl_xor_sync(0xffffffffu, cmp ? v[j] : v[8 + j], 1);
            if (rb < nr) {
                const int64_t outp = ((int64_t)((A << D) + alpha) << lbp) + Bp;   // pair (A_alpha, B_p) at level l+1
                C *wo = a.wout + (int64_t)(rhs0 + rb) * a.wstride + outp * RR;
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const int t = 16 * half + 8 * cmp + j;
                    if (t < RR) {
                        C z;
                        z.x = cmp ? recv[j] : v[j];
                        z.y = cmp ? v[8 + j] : recv[j];
                        __stcs(wo + t, cjmul(PD[alpha * RR + t], z));
                    }
                }
            }
        }
        umma::fence_before_sync();
        __syncthreads();   // the next block's phase stage rewrites PD, its MMAs the tensor memory
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
    umma::fence_before_sync();
    __syncthreads();
    if (warp == 0) umma::dealloc(tmem, ST::TMEM_COLS);
}

}  // namespace bfk
