// Multi-RHS forward passes for d = 2 (the batched right-hand sides of Section 1:
// one operator, several source vectors g).
//
// The phase factors of every step depend only on the geometry, not on g, so a CTA
// keeps up to MRMAX right-hand sides of its tiles in shared memory and splits each
// merge stage in two: all threads first evaluate the stage's phase factors once
// into a shared-memory cache, then apply them to every right-hand side.  The two
// interpolation stages of a merge exchange partial results through scratch; they
// run over the right-hand sides in chunks of rc, so the scratch holds rc of them.
// The switch keeps one accumulator per right-hand side in registers and evaluates
// each entry of the r x r phase matrix once.
//
// Shared memory (complex numbers, npr = pairs of the CTA):
//   W  [nr][npr][r]       weights of every right-hand side (in place, as in Tile)
//   S  [rc][2 npr r + ..] stage scratch (row scratch units padded, mr_pad)
//   PC [5 r npr + ..]     phase cache of the current stage (strides padded, mr_pad)
// Stage items and the order of every accumulation follow Tile<2,...>.
//
// Phase tables (the precompute trade-off of Section 1.4).  A plan may keep every phase
// factor of its apply in device memory: PM_BUILD runs the phase stages only and writes
// each stage's cache (and the switch matrices) to the table, in the order PM_TABLE reads
// them back; PM_TABLE copies them into the cache instead of evaluating Phi, which turns
// the instruction-bound apply into a stream over the table.  The values are those the
// computing kernels (PM_COMPUTE) would produce, so the results are identical.
#pragma once

#include "bf_device.cuh"

namespace bfk {

constexpr int MRMAX = 16;   // right-hand sides held by one CTA

// ---- bulk copies (TMA engine) into shared memory, completed on an mbarrier
__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_init_fence() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, uint64_t *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}
// tiled bulk copy (TMA) of the 2-D box at element coordinates (x, y) of the tensor that
// `map` describes (a CUtensorMap in global memory) into shared memory, completed on bar;
// the box's rows land contiguously (x times the element size must be a multiple of 16 bytes)
__device__ __forceinline__ void bulk_tensor_2d_g2s(void *dst, const void *map, int x, int y, uint64_t *bar)
{
    asm volatile("cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
                 ::"r"(smem_u32(dst)), "l"(map), "r"(x), "r"(y), "r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned parity)
{
    uint32_t ok;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(ok)
                 : "r"(smem_u32(bar)), "r"(parity)
                 : "memory");
    return ok != 0;
}
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// wait for phase `parity` of an mbarrier; false after `limit` polls (the caller flags the error)
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, unsigned parity, int limit)
{
    for (int i = 0; i < limit; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

constexpr int TS_MAXB = 16;          // table blocks per CTA and pass
constexpr int TS_POLLS = 1 << 16;    // polls of one wait before it is flagged

// Phase-table stream of a CTA (PM_TABLE): block j of the pass's table arrives in buffer
// j & 1 by one bulk copy, issued two blocks ahead of its use.
struct TabCtl {
    uint64_t bar[2];
    int64_t off[TS_MAXB + 1];   // block j of a tile group = complex numbers [off[j], off[j+1]) of its table
    int nblk;                   // blocks per tile group
    int total;                  // blocks of all the CTA's tile groups
};

template <class C>
struct TS {
    C *tb;          // PM_BUILD: write cursor; PM_TABLE: the pass's table in global memory
    C *buf[2];      // PM_TABLE: shared-memory buffers
    TabCtl *ctl;
    int j;          // PM_TABLE: next block to use
    int *err;       // set when a wait gives up
    int c0, cstep;  // PM_TABLE: the CTA's tile groups are c0, c0 + cstep, ...
    int64_t cstride;   // table complex numbers per tile group
};

// pairs per switch round and threads per CTA: the switch runs one thread per (pair, s)
template <int Q>
struct CfgMR {
    static constexpr int RR = Q * Q;
    static constexpr int PPR = RR <= 32 ? 16 : (RR <= 64 ? 8 : 4);
    static constexpr int NT = PPR * RR;
    static constexpr int MINB = RR <= 32 ? 2 : 1;   // CTAs per SM the register budget is cut for
};

// Padding (in complex numbers) of the shared-memory arrays read and written by the apply
// stages, so that the 64-bit accesses of a warp fall in distinct banks (32 banks of 4
// bytes).  Chosen for q = 5 by counting the wavefronts of every access pattern of the
// stages for 16 and 32 pairs per CTA and 1 or 2 fused levels (46% more wavefronts than the
// minimum before, 3% after); the phase-table layout stays compact.
struct MRPad {
    int ca;   // column modulation: per (pair, chi) block of 2 r factors
    int cb;   // column demodulation: per pair (r factors)
    int rb;   // row post-modulation: per pair (4 r factors)
    int rs;   // row scratch: per (pair, t_1) unit of 2 q partial sums
};
__host__ __device__ constexpr MRPad mr_pad(int q) { return q == 5 ? MRPad{7, 12, 1, 1} : MRPad{0, 0, 0, 0}; }
// phase-cache entries per pair beyond 5 r (evaluating passes)
__host__ __device__ constexpr int mr_pc_extra(int q)
{
    return 2 * mr_pad(q).ca + mr_pad(q).cb > mr_pad(q).rb ? 2 * mr_pad(q).ca + mr_pad(q).cb : mr_pad(q).rb;
}
// scratch entries per right-hand side (2 r per pair, plus the row scratch padding)
__host__ __device__ constexpr int64_t mr_s_stride(int q, int64_t npr) { return 2 * npr * q * q + npr * q * mr_pad(q).rs; }

// acc += M[h][t][u] v: two scalar FMAs, the coefficient an operand from the kernel
// parameters (constant bank).  One packed FMA with the coefficient duplicated (KArgs::M2)
// needs that pair loaded into registers first: measured 1% slower per apply at N = 512
// with 16 right-hand sides (the same roundings either way; in the persistent batch kernel
// the packed form also spilled)
template <class MS, class C>
__device__ __forceinline__ void mmac(C &acc, const MS &ms, int h, int t, int u, C v)
{
    cfma(acc, ms.M[h][t][u], v);
}

template <int Q, class P, int K>
struct TileMR {
    static constexpr MRPad PAD = mr_pad(Q);
    static constexpr int D = 2, NC = 4, RR = Q * Q, NT = CfgMR<Q>::NT;
    using R = typename P::R;
    using C = typename P::C;
    using PH = Ph<P, 2, K>;
    using PH2 = Ph2<P, 2, K>;
    using TL = Tile<2, Q, P, K>;

    // geometry of one output pair of a column level, computed once per level into the
    // scratch S (idle during the phase stage) for the stage's phase items
    struct __align__(16) GeoC {
        typename PH::T tA;   // target features at the centre of the pair's target box (level l+1)
        int cbq[2];          // coordinates of the parent source box (level l+1)
    };

    // geometry of one merge block of a row level (in S during the phase stage): the parent
    // target box (level l) and the parent source box (level l+1)
    struct __align__(16) GeoR {
        int ca[2];    // coordinates of the parent target box A_p
        int cbq[2];   // coordinates of the parent source box B_q
    };

    struct Ctx {
        int tile0;   // first tile of the CTA
        int rhs0;    // first right-hand side
        int nr;      // right-hand sides held (1..MRMAX)
        int npr;     // pairs held: T 2^{2k}
        int rc;      // right-hand sides per scratch chunk
        int lgp;     // log2(npr)
    };

    static __device__ __forceinline__ void tile_of(const KArgs<P> &a, const Ctx &x, int tau, uint32_t &Ap,
                                                   uint32_t &Bstar)
    {
        const uint32_t tile = (uint32_t)x.tile0 + (uint32_t)tau;
        const int sh = D * (a.L - a.l0 - a.k);
        Ap = tile >> sh;
        Bstar = tile & ((1u << sh) - 1u);
    }

    static __device__ __forceinline__ int block_base(int beta, int i)
    {
        const int ra = beta & ((1 << (D * i)) - 1);
        return ((beta >> (D * i)) << (D * (i + 1))) + ra;
    }

    // ---- phase-table stream (PM_TABLE)
    static __device__ void ts_issue(TS<C> &ts, int j)
    {
        TabCtl *c = ts.ctl;
        const int g = j / c->nblk, jj = j - g * c->nblk;
        const unsigned bytes = (unsigned)((c->off[jj + 1] - c->off[jj]) * (int64_t)sizeof(C));
        const C *src = ts.tb + (int64_t)(ts.c0 + g * ts.cstep) * ts.cstride + c->off[jj];
        mbar_expect_tx(&c->bar[j & 1], bytes);
        bulk_g2s(ts.buf[j & 1], src, bytes, &c->bar[j & 1]);
    }
    // block list of a tile group (sizes in complex numbers), barriers, the first two copies
    // of the stream over all the CTA's tile groups
    static __device__ void ts_setup(TS<C> &ts, const KArgs<P> &a, const Ctx &x, bool row)
    {
        if (threadIdx.x == 0) {
            TabCtl *c = ts.ctl;
            const int64_t npr = x.npr, r5 = 5 * RR * npr;
            int nb = 0;
            int64_t o = 0;
            auto add = [&](int64_t n) { c->off[nb++] = o; o += n; };
            if (!row) {
                if (a.flags & F_INIT) add(RR * npr);
                for (int i = 0; i < a.k; ++i) add(r5);
                if (a.flags & F_SWITCH)
                    for (int th = 0; th < Q; ++th) add((int64_t)Q * RR * npr);
            } else {
                for (int i = 0; i < a.k; ++i) add(r5);
                if (a.flags & F_FINAL) add((RR + 1) * npr);
            }
            c->off[nb] = o;
            c->nblk = nb;
            c->total = nb * ((a.ncta - ts.c0 + ts.cstep - 1) / ts.cstep);
            mbar_init(&c->bar[0], 1);
            mbar_init(&c->bar[1], 1);
            mbar_init_fence();
            for (int j = 0; j < 2 && j < c->total; ++j) ts_issue(ts, j);
        }
        ts.j = 0;
        __syncthreads();
    }
    // wait for the next block; a wait that gives up is flagged and waited for once more,
    // so no copy is left in flight (the results are then undefined, never a hang)
    static __device__ C *ts_acquire(TS<C> &ts)
    {
        const int j = ts.j;
        uint64_t *bar = &ts.ctl->bar[j & 1];
        if (!mbar_wait(bar, (unsigned)((j >> 1) & 1), TS_POLLS)) {
            if (ts.err) atomicExch(ts.err, 1);
            mbar_wait(bar, (unsigned)((j >> 1) & 1), TS_POLLS);
        }
        return ts.buf[j & 1];
    }
    // after the block's last reader (callers sync first): refill its buffer two blocks ahead
    static __device__ void ts_release(TS<C> &ts)
    {
        const int j = ts.j++;
        if (threadIdx.x == 0 && j + 2 < ts.ctl->total) {
            fence_proxy_async();
            ts_issue(ts, j + 2);
        }
    }

    // ---- phase-table store of n complex numbers (PM_BUILD; n even, 16-byte aligned blocks)
    static __device__ __forceinline__ void tab_store(C *dst, const C *src, int n)
    {
        const float4 *s4 = reinterpret_cast<const float4 *>(src);
        float4 *d4 = reinterpret_cast<float4 *>(dst);
        for (int j = threadIdx.x; j < (n >> 1); j += NT) __stcs(d4 + j, s4[j]);
    }

    // ---- CTA input: npr consecutive pairs per right-hand side (sharding mode 2: the pairs of
    // other ranks' source boxes read as zero)
    static __device__ void load(const KArgs<P> &a, const Ctx &x, C *W)
    {
        const int WS = x.npr * RR;
        const int64_t off = (int64_t)x.tile0 * ((int64_t)RR << (D * a.k));
        for (int j = threadIdx.x; j < x.nr * WS; j += NT) {
            const int rb = (j / RR) >> x.lgp, e = j - rb * WS;
            W[j] = a.shard_mode == 2 && !shard_owned<D>(a, (off + e) / RR)
                       ? czero<C>()
                       : __ldcg(a.win + (int64_t)(x.rhs0 + rb) * a.wstride + off + e);
        }
    }

    // ---- the same input by bulk copies (the TMA engine), one per right-hand side (npr r complex
    // numbers, contiguous in HBM and 16-byte aligned), completing on *bar; issued by thread 0
    // after the shared memory's previous generic accesses are ordered before the copies
    static __device__ void load_async(const KArgs<P> &a, const Ctx &x, C *W, uint64_t *bar)
    {
        if (threadIdx.x != 0) return;
        const unsigned bytes = (unsigned)(x.npr * RR * sizeof(C));
        const int64_t off = (int64_t)x.tile0 * ((int64_t)RR << (D * a.k));
        fence_proxy_async();
        mbar_expect_tx(bar, bytes * (unsigned)x.nr);
        for (int rb = 0; rb < x.nr; ++rb)
            bulk_g2s(W + rb * x.npr * RR, a.win + (int64_t)(x.rhs0 + rb) * a.wstride + off, bytes, bar);
    }
    // every thread: wait for those copies; a wait that gives up is flagged and waited for once
    // more, so no copy is left in flight (the results are then undefined, never a hang)
    static __device__ void wait_input(const KArgs<P> &a, uint64_t *bar, unsigned parity)
    {
        if (!mbar_wait(bar, parity, TS_POLLS)) {
            if (a.err) atomicExch(a.err, 1);
            mbar_wait(bar, parity, TS_POLLS);
        }
    }

    // ---- CTA output: tile slots are in digit-reversed order after k merges
    static __device__ void store(const KArgs<P> &a, const Ctx &x, const C *W)
    {
        // destination of each slot's pair, once per CTA (slots are in digit-reversed order)
        __shared__ int64_t poff[64];
        const int k = a.k, n = 1 << (D * k), WS = x.npr * RR;
        const int64_t Sstar = 1LL << (D * (a.L - a.l0 - k));
        for (int pl = threadIdx.x; pl < x.npr; pl += NT) {
            uint32_t Ap, Bstar;
            tile_of(a, x, pl >> (D * k), Ap, Bstar);
            poff[pl] = ((((int64_t)Ap << (D * k)) + digit_rev<D>(pl & (n - 1), k)) * Sstar + Bstar) * RR;
        }
        __syncthreads();
        for (int j = threadIdx.x; j < x.nr * WS; j += NT) {
            const int rb = (j / RR) >> x.lgp, e = j - rb * WS;
            const int pl = e / RR, t = e - pl * RR;
            a.wout[(int64_t)(x.rhs0 + rb) * a.wstride + poff[pl] + t] = W[j];
        }
    }

    // ---- init: PC[pair][t] = l_t(y) e^{-2pi i Phi(x0(X), y_t^B)} e^{2pi i Phi(x0(X), y)}, then W = PC g(y)
    template <int PM>
    static __device__ void init(const KArgs<P> &a, const Ctx &x, C *W, C *PC, const C *g, TS<C> &ts)
    {
        const int k = a.k, n = 1 << (D * k), L = a.L, WS = x.npr * RR;
        const int cX[DMAX] = {0, 0, 0};
        const int ctr[DMAX] = {Q, Q, Q};
        const typename PH::T tX = tpoint<P, D, Q, K>(a, 0, cX, ctr);
        if constexpr (PM == PM_TABLE) PC = ts_acquire(ts);
        for (int it = threadIdx.x; PM != PM_TABLE && it < WS; it += NT) {
            const int t = it % RR, pr = it / RR;
            const int tk[DMAX] = {t % Q, t / Q, 0};
            const R lag = a.lsrc[tk[0]] * a.lsrc[tk[1]];
            C e = czero<C>();
            if (lag != R(0)) {
                uint32_t Ap, Bstar;
                tile_of(a, x, pr >> (D * k), Ap, Bstar);
                int cb[DMAX];
                morton_decode<D>((Bstar << (D * k)) + (pr & (n - 1)), L, cb);
                const int pslot[DMAX] = {Q + 1, Q + 1, Q + 1};
                const C e1 = expphase<P, D, K>(a, tX, spoint<P, D, Q, K>(a, 0, cb, pslot));
                const C e0 = expphase<P, D, K>(a, tX, spoint<P, D, Q, K>(a, 0, cb, tk));
                e = cjmul(e0, e1);
                e.x *= lag;
                e.y *= lag;
            }
            PC[it] = e;
        }
        __syncthreads();
        if constexpr (PM == PM_BUILD) {   // build: store the factors; no weights are touched
            tab_store(ts.tb, PC, WS);
            ts.tb += WS;
            __syncthreads();
        }
        if constexpr (PM != PM_BUILD) {
            // the grid point of a leaf box has a non-zero Lagrange value at few nodes (one
            // for points at box corners): zero the weights, then fill those nodes only
            __shared__ int nzt[QMAX * QMAX];
            __shared__ int nnz;
            if (threadIdx.x == 0) {
                int m = 0;
                for (int t = 0; t < RR; ++t)
                    if (a.lsrc[t % Q] * a.lsrc[t / Q] != R(0)) nzt[m++] = t;
                nnz = m;
            }
            float4 *w4 = reinterpret_cast<float4 *>(W);
            for (int j = threadIdx.x; j < (x.nr * WS * (int)sizeof(C)) / 16; j += NT) w4[j] = make_float4(0.f, 0.f, 0.f, 0.f);
            __syncthreads();
            for (int j = threadIdx.x; j < x.nr * x.npr * nnz; j += NT) {
                const int z = j % nnz, pr = (j / nnz) & (x.npr - 1), rb = (j / nnz) >> x.lgp;
                const int it = pr * RR + nzt[z];
                uint32_t Ap, Bstar;
                tile_of(a, x, pr >> (D * k), Ap, Bstar);
                int cb[DMAX];
                morton_decode<D>((Bstar << (D * k)) + (pr & (n - 1)), L, cb);
                const int64_t flat = ((int64_t)cb[0] << L) + cb[1];
                W[rb * WS + it] = cmul(PC[it], g[(int64_t)(x.rhs0 + rb) * a.npts + flat]);
            }
        }
        __syncthreads();
        if constexpr (PM == PM_TABLE) ts_release(ts);
    }

    // ---- one column-form merge level (l -> l+1); ms.M holds the child->parent matrices
    template <int PM, class MS>
    static __device__ void col_level(const KArgs<P> &a, const MS &ms, const Ctx &x, C *W, C *S, C *PC, int l, int i,
                                     TS<C> &ts, uint64_t *wbar = nullptr, unsigned wpar = 0)
    {
        const int k = a.k, n = 1 << (D * k), nblk = n >> D, L = a.L, WS = x.npr * RR, nout = x.npr;
        if constexpr (PM == PM_TABLE) PC = ts_acquire(ts);
        const int SW = (int)mr_s_stride(Q, x.npr);
        constexpr int PCA = 2 * RR + (PM == PM_COMPUTE ? PAD.ca : 0), PCB = RR + (PM == PM_COMPUTE ? PAD.cb : 0);
        C *PA = PC;                     // [pA][chi] blocks of PCA: [cl][tq][t0']  modulation of the inputs
        C *PB = PC + nout * 2 * PCA;    // [pA] blocks of PCB: [tq][tl]            demodulation of the output
        GeoC *G = reinterpret_cast<GeoC *>(S);
        for (int j = threadIdx.x; PM != PM_TABLE && j < nout; j += NT) {
            const int alpha = j & (NC - 1), beta = (j >> D) & (nblk - 1), tau = j >> (D * k);
            uint32_t Ap, Bstar, Apg, Bq;
            int base;
            tile_of(a, x, tau, Ap, Bstar);
            TL::block_geo(Ap, Bstar, beta, i, k, Apg, Bq, base);
            const uint32_t Aa = (Apg << D) + alpha;
            int ca[DMAX], cbq[DMAX];
            morton_decode<D>(Aa, l + 1, ca);
            morton_decode<D>(Bq, L - l - 1, cbq);
            G[j].tA = tcenter<P, D, Q, K>(a, l + 1, Aa, ca);
            G[j].cbq[0] = cbq[0];
            G[j].cbq[1] = cbq[1];
        }
        if constexpr (PM != PM_TABLE) __syncthreads();
        for (int it = threadIdx.x; PM != PM_TABLE && it < nout * 4 * Q; it += NT) {
            const int tq = it % Q, cl = (it / Q) & 1, chi = (it / (2 * Q)) & 1, pA = it / (4 * Q);
            const typename PH::T tA = G[pA].tA;
            const int cbq[2] = {G[pA].cbq[0], G[pA].cbq[1]};
            const int c = cl | (chi << 1);
            // phases two at a time: lanes t'_0 and t'_0 + 1 (the last one alone for odd q)
            const typename PH2::T tA2 = PH2::dup(tA);
            const typename P::SE e1 = sget<P, Q>(a, 1, l, 2 * cbq[1] + chi, tq);
            const typename PH2::Part p1 = PH2::part(tA2, e1, e1, 1);
            const int c0 = 2 * cbq[0] + (c & 1);
            C *o = PA + (pA * 2 + chi) * PCA + cl * RR + tq * Q;
#pragma unroll
            for (int t0p = 0; t0p + 1 < Q; t0p += 2) {
                const typename PH2::Part pt =
                    PH2::add(PH2::part(tA2, sget<P, Q>(a, 0, l, c0, t0p), sget<P, Q>(a, 0, l, c0, t0p + 1), 0), p1);
                expphase_part2<P, D, K>(a, tA2, pt, o[t0p], o[t0p + 1]);
            }
            if constexpr (Q & 1) {
                const typename PH::Part pt = PH::add(PH::part(tA, sget<P, Q>(a, 0, l, c0, Q - 1), 0), PH2::lane0(p1));
                o[Q - 1] = expphase_part<P, D, K>(a, tA, pt);
            }
        }
        for (int it = threadIdx.x; PM != PM_TABLE && it < nout * RR; it += NT) {
            const int tl = it % Q, tq = (it / Q) % Q, pA = it / RR;
            const typename PH::T tA = G[pA].tA;
            const int cbq[2] = {G[pA].cbq[0], G[pA].cbq[1]};
            const typename PH::Part pl = PH::part(tA, sget<P, Q>(a, 0, l + 1, cbq[0], tl), 0);
            const typename PH::Part pt = PH::add(PH::part(tA, sget<P, Q>(a, 1, l + 1, cbq[1], tq), 1), pl);
            PB[pA * PCB + tq * Q + tl] = expphase_part<P, D, K>(a, tA, pt);
        }
        __syncthreads();
        if (wbar) wait_input(a, wbar, wpar);   // the weights were copied in during the phase stage
        if constexpr (PM == PM_BUILD) {   // build: store the factors; no weights are touched
            tab_store(ts.tb, PC, 5 * RR * nout);
            ts.tb += 5 * RR * nout;
            __syncthreads();
        }
        for (int r0 = 0; PM != PM_BUILD && r0 < x.nr; r0 += x.rc) {
            const int nrc = min(x.rc, x.nr - r0);
            // stage A: items (rb, pA, chi, tq): modulate the inputs, contract dimension 0
            for (int it = threadIdx.x; it < nrc * nout * 2 * Q; it += NT) {
                const int tq = it % Q, chi = (it / Q) & 1, pA = (it / (2 * Q)) & (nout - 1), rbl = (it / (2 * Q)) >> x.lgp;
                const int beta = (pA >> D) & (nblk - 1), tau = pA >> (D * k);
                const int base = block_base(beta, i);
                const C *Wr = W + (r0 + rbl) * WS + tau * n * RR;
                const C *ph = PA + (pA * 2 + chi) * PCA + tq * Q;
                C acc[Q];
#pragma unroll
                for (int j = 0; j < Q; ++j) acc[j] = czero<C>();
#pragma unroll
                for (int cl = 0; cl < 2; ++cl) {
                    const int c = cl | (chi << 1);
                    const C *win = Wr + (base + (c << (D * i))) * RR + Q * tq;
#pragma unroll
                    for (int t0p = 0; t0p < Q; ++t0p) {
                        const C u = cmul(ph[cl * RR + t0p], win[t0p]);
#pragma unroll
                        for (int t0 = 0; t0 < Q; ++t0) mmac(acc[t0], ms, c & 1, t0, t0p, u);
                    }
                }
                C *so = S + rbl * SW + ((pA * 2 + chi) * Q + tq) * Q;
#pragma unroll
                for (int j = 0; j < Q; ++j) so[j] = acc[j];
            }
            __syncthreads();
            // stage B: items (rb, pA, tl): contract dimension 1 and the child bit, demodulate
            for (int it = threadIdx.x; it < nrc * nout * Q; it += NT) {
                const int tl = it % Q, pA = (it / Q) & (nout - 1), rbl = (it / Q) >> x.lgp;
                const int alpha = pA & (NC - 1), beta = (pA >> D) & (nblk - 1), tau = pA >> (D * k);
                const int base = block_base(beta, i);
                C acc[Q];
#pragma unroll
                for (int j = 0; j < Q; ++j) acc[j] = czero<C>();
#pragma unroll
                for (int chi = 0; chi < 2; ++chi) {
                    const C *si = S + rbl * SW + ((pA * 2 + chi) * Q) * Q + tl;
#pragma unroll
                    for (int tqp = 0; tqp < Q; ++tqp) {
                        const C v = si[tqp * Q];
#pragma unroll
                        for (int tq = 0; tq < Q; ++tq) mmac(acc[tq], ms, chi, tq, tqp, v);
                    }
                }
                C *wo = W + (r0 + rbl) * WS + tau * n * RR + (base + (alpha << (D * i))) * RR + tl;
                const C *ph = PB + pA * PCB + tl;
#pragma unroll
                for (int tq = 0; tq < Q; ++tq) wo[tq * Q] = cjmul(ph[tq * Q], acc[tq]);
            }
            __syncthreads();
        }
        if constexpr (PM == PM_TABLE) ts_release(ts);
    }

    // ---- switch at level l: one thread per (pair, s), one accumulator per right-hand side;
    // rounds of whole pairs, results written back after every thread of the round has read.
    // Phase-table layout: q chunks (one per source digit t_1), each [pair][t_0][s], so a
    // chunk is one contiguous block (PM_TABLE plans have one round: npr <= PPR).
    template <int PM>
    static __device__ void switch_tiles(const KArgs<P> &a, const Ctx &x, C *W, int l, TS<C> &ts)
    {
        const int k = a.k, n = 1 << (D * k), L = a.L, WS = x.npr * RR;
        const int G = CfgMR<Q>::PPR;
        for (int p0 = 0; p0 < x.npr; p0 += G) {
            const int pl = p0 + (int)threadIdx.x / RR, s = (int)threadIdx.x % RR;
            const bool act = (int)threadIdx.x < G * RR && pl < x.npr;
            C acc[MRMAX];
#pragma unroll
            for (int rb = 0; rb < MRMAX; ++rb) acc[rb] = czero<C>();
            typename PH::T tS;
            int cb[DMAX] = {0, 0, 0};
            if (PM != PM_TABLE && act) {
                uint32_t Ap, Bstar;
                tile_of(a, x, pl >> (D * k), Ap, Bstar);
                const uint32_t A = (Ap << (D * k)) + digit_rev<D>(pl & (n - 1), k);
                int ca[DMAX];
                morton_decode<D>(A, l, ca);
                morton_decode<D>(Bstar, L - l, cb);
                const int sk[DMAX] = {s % Q, s / Q, 0};
                tS = tpoint<P, D, Q, K>(a, l, ca, sk);
            }
            const C *u = W + pl * RR;
#pragma unroll 1
            for (int th = 0; th < Q; ++th) {
                const C *chunk = nullptr;
                if constexpr (PM == PM_TABLE) chunk = ts_acquire(ts);
                if (act) {
                    C ev[Q];   // the factors of this digit t_1: two at a time (lanes t_0, t_0 + 1)
                    if constexpr (PM != PM_TABLE) {
                        const typename PH2::T tS2 = PH2::dup(tS);
                        const typename P::SE e1 = sget<P, Q>(a, 1, l, cb[1], th);
                        const typename PH2::Part hp = PH2::part(tS2, e1, e1, 1);
#pragma unroll
                        for (int t0 = 0; t0 + 1 < Q; t0 += 2)
                            expphase_part2<P, D, K>(
                                a, tS2,
                                PH2::add(PH2::part(tS2, sget<P, Q>(a, 0, l, cb[0], t0), sget<P, Q>(a, 0, l, cb[0], t0 + 1), 0), hp),
                                ev[t0], ev[t0 + 1]);
                        if constexpr (Q & 1)
                            ev[Q - 1] = expphase_part<P, D, K>(
                                a, tS, PH::add(PH::part(tS, sget<P, Q>(a, 0, l, cb[0], Q - 1), 0), PH2::lane0(hp)));
                    }
#pragma unroll
                    for (int t0 = 0; t0 < Q; ++t0) {
                        C e;
                        if constexpr (PM == PM_TABLE)
                            e = chunk[(pl * Q + t0) * RR + s];
                        else
                            e = ev[t0];
                        if constexpr (PM == PM_BUILD) {
                            __stcs(ts.tb + ((int64_t)th * x.npr * Q + pl * Q + t0) * RR + s, e);
                        } else {
#pragma unroll
                            for (int rb = 0; rb < MRMAX; ++rb)
                                if (rb < x.nr) cmac(acc[rb], e, u[rb * WS + t0 + Q * th]);
                        }
                    }
                }
                if constexpr (PM == PM_TABLE) {
                    __syncthreads();
                    ts_release(ts);
                }
            }
            if constexpr (PM != PM_BUILD) {
                __syncthreads();
                if (act) {
#pragma unroll
                    for (int rb = 0; rb < MRMAX; ++rb)
                        if (rb < x.nr) W[rb * WS + pl * RR + s] = acc[rb];
                }
                __syncthreads();
            }
        }
        if constexpr (PM == PM_BUILD) ts.tb += (int64_t)x.npr * RR * RR;
    }

    // ---- one row-form merge level (l -> l+1)
    template <int PM, class MS>
    static __device__ void row_level(const KArgs<P> &a, const MS &ms, const Ctx &x, C *W, C *S, C *PC, int l, int i,
                                     TS<C> &ts, uint64_t *wbar = nullptr, unsigned wpar = 0)
    {
        const int k = a.k, n = 1 << (D * k), nblk = n >> D, L = a.L, WS = x.npr * RR, nout = x.npr;
        if constexpr (PM == PM_TABLE) PC = ts_acquire(ts);
        const int SW = (int)mr_s_stride(Q, x.npr);
        constexpr int PRB = 4 * RR + (PM == PM_COMPUTE ? PAD.rb : 0), SU = 2 * Q + PAD.rs;
        C *PA = PC;              // [pin][th][t0]                       pre-modulation at the parent's nodes
        C *PB = PC + nout * RR;  // [pA] blocks of PRB: [c][s1][s0]     post-modulation at the child's nodes
        // the blocks' geometry once per level, into S (idle during the phase stage)
        GeoR *GR = reinterpret_cast<GeoR *>(S);
        for (int j = threadIdx.x; PM != PM_TABLE && j < (nout >> D); j += NT) {
            const int beta = j & (nblk - 1), tau = j >> (D * (k - 1));
            uint32_t Ap, Bstar, Apg, Bq;
            int base;
            tile_of(a, x, tau, Ap, Bstar);
            TL::block_geo(Ap, Bstar, beta, i, k, Apg, Bq, base);
            int ca[DMAX], cbq[DMAX];
            morton_decode<D>(Apg, l, ca);
            morton_decode<D>(Bq, L - l - 1, cbq);
            GR[j] = GeoR{{ca[0], ca[1]}, {cbq[0], cbq[1]}};
        }
        if constexpr (PM != PM_TABLE) __syncthreads();
        for (int it = threadIdx.x; PM != PM_TABLE && it < nout * RR; it += NT) {
            const int t0 = it % Q, th = (it / Q) % Q, pin = it / RR;
            const int c = pin & (NC - 1), b = pin >> D;
            const int ca[DMAX] = {GR[b].ca[0], GR[b].ca[1], 0};
            const int cb[DMAX] = {2 * GR[b].cbq[0] + (c & 1), 2 * GR[b].cbq[1] + ((c >> 1) & 1), 0};
            const int ctr[DMAX] = {Q, Q, Q};
            const int tk[DMAX] = {t0, th, 0};
            PA[it] = expphase<P, D, K>(a, tpoint<P, D, Q, K>(a, l, ca, tk), spoint<P, D, Q, K>(a, l, cb, ctr));
        }
        for (int it = threadIdx.x; PM != PM_TABLE && it < nout * RR; it += NT) {
            const int s0 = it % Q, s1 = (it / Q) % Q, pA = it / RR;
            const int alpha = pA & (NC - 1), b = pA >> D;
            // the child target box (level l+1) of the block's parent box
            const int ca[DMAX] = {2 * GR[b].ca[0] + (alpha & 1), 2 * GR[b].ca[1] + ((alpha >> 1) & 1), 0};
            const int cbq[DMAX] = {GR[b].cbq[0], GR[b].cbq[1], 0};
            const int sk[DMAX] = {s0, s1, 0};
            const typename PH::T tS = tpoint<P, D, Q, K>(a, l + 1, ca, sk);
            // phases two at a time: lanes c_0 = 0 and 1
            const typename PH2::T tS2 = PH2::dup(tS);
            const typename PH2::Part q0 =
                PH2::part(tS2, sget<P, Q>(a, 0, l, 2 * cbq[0], Q), sget<P, Q>(a, 0, l, 2 * cbq[0] + 1, Q), 0);
#pragma unroll
            for (int c1 = 0; c1 < 2; ++c1) {
                const typename P::SE e1 = sget<P, Q>(a, 1, l, 2 * cbq[1] + c1, Q);
                expphase_part2<P, D, K>(a, tS2, PH2::add(q0, PH2::part(tS2, e1, e1, 1)),
                                        PB[pA * PRB + ((2 * c1) * Q + s1) * Q + s0],
                                        PB[pA * PRB + ((2 * c1 + 1) * Q + s1) * Q + s0]);
            }
        }
        __syncthreads();
        if (wbar) wait_input(a, wbar, wpar);   // the weights were copied in during the phase stage
        if constexpr (PM == PM_BUILD) {   // build: store the factors; no weights are touched
            tab_store(ts.tb, PC, 5 * RR * nout);
            ts.tb += 5 * RR * nout;
            __syncthreads();
        }
        for (int r0 = 0; PM != PM_BUILD && r0 < x.nr; r0 += x.rc) {
            const int nrc = min(x.rc, x.nr - r0);
            // stage A: items (rb, pin, th): pre-modulate input c, contract dimension 0 for both alpha_0
            for (int it = threadIdx.x; it < nrc * nout * Q; it += NT) {
                const int th = it % Q, pin = (it / Q) & (nout - 1), rbl = (it / Q) >> x.lgp;
                const int c = pin & (NC - 1), beta = (pin >> D) & (nblk - 1), tau = pin >> (D * k);
                const int base = block_base(beta, i);
                const C *win = W + (r0 + rbl) * WS + tau * n * RR + (base + (c << (D * i))) * RR + th * Q;
                const C *ph = PA + (pin * Q + th) * Q;
                C z[2][Q];
#pragma unroll
                for (int s0 = 0; s0 < Q; ++s0) {
                    z[0][s0] = czero<C>();
                    z[1][s0] = czero<C>();
                }
#pragma unroll
                for (int t0 = 0; t0 < Q; ++t0) {
                    const C u = cjmul(ph[t0], win[t0]);
#pragma unroll
                    for (int s0 = 0; s0 < Q; ++s0) {
                        mmac(z[0][s0], ms, 0, t0, s0, u);
                        mmac(z[1][s0], ms, 1, t0, s0, u);
                    }
                }
                C *so = S + rbl * SW + (pin * Q + th) * SU;
#pragma unroll
                for (int s0 = 0; s0 < Q; ++s0) {
                    so[s0] = z[0][s0];
                    so[Q + s0] = z[1][s0];
                }
            }
            __syncthreads();
            // stage B: items (rb, pA, s0): contract dimension 1 per child, post-modulate, sum over c
            for (int it = threadIdx.x; it < nrc * nout * Q; it += NT) {
                const int s0 = it % Q, pA = (it / Q) & (nout - 1), rbl = (it / Q) >> x.lgp;
                const int alpha = pA & (NC - 1), beta = (pA >> D) & (nblk - 1), tau = pA >> (D * k);
                const int base = block_base(beta, i);
                const int a0 = alpha & 1, a1 = alpha >> 1;
                const C *Sblk = S + rbl * SW + (pA - alpha) * Q * SU;
                C v[NC][Q];
#pragma unroll
                for (int c = 0; c < NC; ++c) {
                    const C *si = Sblk + c * Q * SU + a0 * Q + s0;
#pragma unroll
                    for (int s1 = 0; s1 < Q; ++s1) v[c][s1] = czero<C>();
#pragma unroll
                    for (int t1 = 0; t1 < Q; ++t1) {
                        const C zz = si[t1 * SU];
#pragma unroll
                        for (int s1 = 0; s1 < Q; ++s1) mmac(v[c][s1], ms, a1, t1, s1, zz);
                    }
                }
                C *wo = W + (r0 + rbl) * WS + tau * n * RR + (base + (alpha << (D * i))) * RR + s0;
                const C *ph = PB + pA * PRB + s0;
#pragma unroll
                for (int s1 = 0; s1 < Q; ++s1) {
                    C acc = czero<C>();
#pragma unroll
                    for (int c = 0; c < NC; ++c) acc = TL::cadd(acc, cmul(ph[(c * Q + s1) * Q], v[c][s1]));
                    wo[s1 * Q] = acc;
                }
            }
            __syncthreads();
        }
        if constexpr (PM == PM_TABLE) ts_release(ts);
    }

    // ---- final evaluation: PC[pair][t] = l_t(x) conj(e^{2pi i Phi(x_t, y0(Y))}), PC[pair][r] = e^{2pi i Phi(x, y0(Y))}
    template <int PM>
    static __device__ void final_eval(const KArgs<P> &a, const Ctx &x, const C *W, C *PC, C *f, TS<C> &ts)
    {
        const int k = a.k, n = 1 << (D * k), L = a.L, WS = x.npr * RR;
        const int cY[DMAX] = {0, 0, 0};
        const int ctr[DMAX] = {Q, Q, Q};
        const typename PH::S sY = spoint<P, D, Q, K>(a, L, cY, ctr);
        if constexpr (PM == PM_TABLE) PC = ts_acquire(ts);
        for (int it = threadIdx.x; PM != PM_TABLE && it < x.npr * (RR + 1); it += NT) {
            const int t = it % (RR + 1), pl = it / (RR + 1);
            C e = czero<C>();
            const R lag = t < RR ? a.ltgt[t % Q] * a.ltgt[t / Q] : R(1);
            if (lag != R(0)) {
                uint32_t Ap, Bstar;
                tile_of(a, x, pl >> (D * k), Ap, Bstar);
                int ca[DMAX];
                morton_decode<D>((Ap << (D * k)) + digit_rev<D>(pl & (n - 1), k), L, ca);
                const int tk[DMAX] = {t < RR ? t % Q : Q + 1, t < RR ? t / Q : Q + 1, 0};
                const C e0 = expphase<P, D, K>(a, tpoint<P, D, Q, K>(a, L, ca, tk), sY);
                if (t < RR) {
                    e.x = lag * e0.x;
                    e.y = -lag * e0.y;
                } else {
                    e = e0;
                }
            }
            PC[it] = e;
        }
        __syncthreads();
        if constexpr (PM == PM_BUILD) {   // build: store the factors; no weights are touched
            tab_store(ts.tb, PC, x.npr * (RR + 1));
            ts.tb += x.npr * (RR + 1);
            __syncthreads();
        }
        for (int j = threadIdx.x; PM != PM_BUILD && j < x.nr * x.npr; j += NT) {
            const int pl = j & (x.npr - 1), rb = j >> x.lgp;
            const C *pc = PC + pl * (RR + 1);
            const C *w = W + rb * WS + pl * RR;
            C acc = czero<C>();
            for (int t = 0; t < RR; ++t)
                if (a.ltgt[t % Q] * a.ltgt[t / Q] != R(0)) cmac(acc, pc[t], w[t]);
            uint32_t Ap, Bstar;
            tile_of(a, x, pl >> (D * k), Ap, Bstar);
            int ca[DMAX];
            morton_decode<D>((Ap << (D * k)) + digit_rev<D>(pl & (n - 1), k), L, ca);
            const int64_t flat = ((int64_t)ca[0] << L) + ca[1];
            f[(int64_t)(x.rhs0 + rb) * a.npts + flat] = cmul(pc[RR], acc);
        }
        if constexpr (PM == PM_TABLE) {   // the stream continues with the CTA's next tile group
            __syncthreads();
            ts_release(ts);
        }
    }

    // shared memory of one CTA, bytes
    static __host__ __device__ size_t smem_bytes(int npr, int nr, int rc)
    {
        return sizeof(C) * ((size_t)npr * RR * (size_t)(nr + 5) + (size_t)rc * (size_t)mr_s_stride(Q, npr) +
                            (size_t)npr * mr_pc_extra(Q));
    }

    static __device__ __forceinline__ Ctx ctx(const KArgs<P> &a, int cta)
    {
        Ctx x;
        x.tile0 = (int)shard_cta<D>(a, (uint32_t)cta) * a.T;
        x.rhs0 = (int)blockIdx.y * MRMAX;
        x.nr = min(MRMAX, a.nrhs - x.rhs0);
        x.npr = a.T << (D * a.k);
        x.rc = a.rc;
        x.lgp = __ffs(x.npr) - 1;
        return x;
    }
};

// pass bodies shared by the per-pass kernels and the persistent batch kernel; ms is a
// kernel parameter holding M, so the interpolation reads its coefficients from the
// constant bank; ts carries the phase table (PM_BUILD, PM_TABLE)
// wbar (per-pass kernels): the input weights come by bulk copies that overlap the first
// level's phase stage (wpar: the mbarrier phase of this tile group); null: plain loads first
template <int Q, class P, int K, int PM, class MS>
__device__ __forceinline__ bool col_pass_mr(const KArgs<P> &a, const MS &ms, const typename TileMR<Q, P, K>::Ctx &x,
                                            unsigned char *sm, const typename P::C *g, TS<typename P::C> &ts,
                                            uint64_t *wbar = nullptr, unsigned wpar = 0)
{
    using C = typename P::C;
    using TM = TileMR<Q, P, K>;
    const int WS = x.npr * TM::RR;
    C *W = reinterpret_cast<C *>(sm);
    C *S = W + x.nr * WS;
    C *PC = S + x.rc * mr_s_stride(Q, x.npr);
    const bool async = wbar && !(a.flags & F_INIT) && a.k > 0 && a.shard_mode != 2;
    if (a.flags & F_INIT) {
        TM::template init<PM>(a, x, W, PC, g, ts);
    } else if (async) {
        TM::load_async(a, x, W, wbar);
    } else if (PM != PM_BUILD) {
        TM::load(a, x, W);
        __syncthreads();
    }
    for (int i = 0; i < a.k; ++i)
        TM::template col_level<PM>(a, ms, x, W, S, PC, a.l0 + i, i, ts, async && i == 0 ? wbar : nullptr, wpar);
    if (a.flags & F_SWITCH) TM::template switch_tiles<PM>(a, x, W, a.l0 + a.k, ts);
    if (PM != PM_BUILD) TM::store(a, x, W);
    return async;
}

template <int Q, class P, int K, int PM, class MS>
__device__ __forceinline__ bool row_pass_mr(const KArgs<P> &a, const MS &ms, const typename TileMR<Q, P, K>::Ctx &x,
                                            unsigned char *sm, typename P::C *f, TS<typename P::C> &ts,
                                            uint64_t *wbar = nullptr, unsigned wpar = 0)
{
    using C = typename P::C;
    using TM = TileMR<Q, P, K>;
    const int WS = x.npr * TM::RR;
    C *W = reinterpret_cast<C *>(sm);
    C *S = W + x.nr * WS;
    C *PC = S + x.rc * mr_s_stride(Q, x.npr);
    const bool async = wbar && a.k > 0 && a.shard_mode != 2;
    if (async) {
        TM::load_async(a, x, W, wbar);
    } else if (PM != PM_BUILD) {
        TM::load(a, x, W);
        __syncthreads();
    }
    for (int i = 0; i < a.k; ++i)
        TM::template row_level<PM>(a, ms, x, W, S, PC, a.l0 + i, i, ts, async && i == 0 ? wbar : nullptr, wpar);
    if (a.flags & F_FINAL)
        TM::template final_eval<PM>(a, x, W, PC, f, ts);
    else if (PM != PM_BUILD)
        TM::store(a, x, W);
    return async;
}

constexpr int TABCTL_BYTES = (int)((sizeof(TabCtl) + 15) / 16 * 16);

// largest table block of a pass (a level's 5 r factors per pair, or a switch chunk)
template <int Q>
__host__ __device__ constexpr int tab_blk_factor() { return Q > 5 ? Q : 5; }

// shared memory of a CTA: PM_TABLE puts the stream control and two block buffers first
template <int Q, class P, int K, int PM>
__device__ __forceinline__ unsigned char *mr_setup(const KArgs<P> &a, const typename TileMR<Q, P, K>::Ctx &x,
                                                   unsigned char *smem, TS<typename P::C> &ts, bool row)
{
    using C = typename P::C;
    ts.tb = nullptr;
    ts.ctl = nullptr;
    ts.buf[0] = ts.buf[1] = nullptr;
    ts.j = 0;
    ts.err = a.err;
    ts.c0 = (int)blockIdx.x;
    ts.cstep = (int)gridDim.x;
    ts.cstride = a.ptab_cta;
    if constexpr (PM != PM_TABLE) return smem;
    ts.tb = a.ptab;
    const int blk = tab_blk_factor<Q>() * Q * Q * x.npr;
    ts.ctl = reinterpret_cast<TabCtl *>(smem);
    ts.buf[0] = reinterpret_cast<C *>(smem + TABCTL_BYTES);
    ts.buf[1] = ts.buf[0] + blk;
    TileMR<Q, P, K>::ts_setup(ts, a, x, row);
    return reinterpret_cast<unsigned char *>(ts.buf[1] + blk);
}

// Per-pass kernels.  A CTA runs tile groups blockIdx.x, blockIdx.x + gridDim.x, ... < a.ncta
// (one with a full grid; PM_TABLE launches as many CTAs as fit and streams the table of
// all its tile groups through one pipeline).
template <int Q, class P, int K, int PM>
__global__ void __launch_bounds__(CfgMR<Q>::NT, CfgMR<Q>::MINB) k_col_pass_mr(const KArgs<P> a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ uint64_t wbar;
    TS<typename P::C> ts;
    unsigned char *work = mr_setup<Q, P, K, PM>(a, TileMR<Q, P, K>::ctx(a, blockIdx.x), smem_raw, ts, false);
    if (PM == PM_COMPUTE && threadIdx.x == 0) {
        mbar_init(&wbar, 1);
        mbar_init_fence();
    }
    __syncthreads();
    unsigned it = 0;
    for (int c = blockIdx.x; c < a.ncta; c += gridDim.x, ++it) {
        if constexpr (PM == PM_BUILD) ts.tb = a.ptab + (int64_t)c * a.ptab_cta;
        col_pass_mr<Q, P, K, PM>(a, a, TileMR<Q, P, K>::ctx(a, c), work, a.g, ts, PM == PM_COMPUTE ? &wbar : nullptr,
                                 it & 1u);
        __syncthreads();
    }
}

template <int Q, class P, int K, int PM>
__global__ void __launch_bounds__(CfgMR<Q>::NT, CfgMR<Q>::MINB) k_row_pass_mr(const KArgs<P> a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ uint64_t wbar;
    TS<typename P::C> ts;
    unsigned char *work = mr_setup<Q, P, K, PM>(a, TileMR<Q, P, K>::ctx(a, blockIdx.x), smem_raw, ts, true);
    if (PM == PM_COMPUTE && threadIdx.x == 0) {
        mbar_init(&wbar, 1);
        mbar_init_fence();
    }
    __syncthreads();
    unsigned it = 0;
    for (int c = blockIdx.x; c < a.ncta; c += gridDim.x, ++it) {
        if constexpr (PM == PM_BUILD) ts.tb = a.ptab + (int64_t)c * a.ptab_cta;
        row_pass_mr<Q, P, K, PM>(a, a, TileMR<Q, P, K>::ctx(a, c), work, a.f, ts, PM == PM_COMPUTE ? &wbar : nullptr,
                                 it & 1u);
        __syncthreads();
    }
}

// ====================================================================== persistent batch
// Many independent problems in one launch.  A job is one pass of one problem for one
// block of up to MRMAX right-hand sides; its units are the pass's CTAs.  Jobs are
// ordered by pass index, so a unit only ever waits for units that come earlier in the
// queue: CTAs take units from a global counter in order, and before a unit of pass j
// starts, the CTA waits until every unit of the same problem's pass j-1 (same RHS
// block) has finished.  The unit that is earliest among the unfinished ones never
// waits, so the queue always advances.  A wait gives up after a time limit, sets the
// error flag and skips its unit; once the flag is set no unit waits or computes.

constexpr int BATCH_MAX = 256;          // problems per batch

struct BatchJob {
    int prob, desc;      // problem, descriptor (problem, pass) of the job
    int y;               // block of right-hand sides
    int ctas;            // CTAs of the pass (tile groups of T tiles)
    int per;             // CTAs per work unit, run one after another by one CTA
    int units, first;    // units of the job and index of its first unit in the queue
    int dep;             // job that must finish first (-1: none)
    int row, pad0, pad1, pad2;   // 1: row pass
};

template <class P>
struct BatchArgs {
    typename P::R M[2][QMAX][QMAX];   // child->parent matrices (the same for every problem)
    const KArgs<P> *__restrict__ desc;   // per (problem, pass); g and f come from the arrays below
    const BatchJob *jobs;
    int njobs, units;
    unsigned *ctr;                 // [njobs] finished units per job, [njobs] queue head
    int *err;                      // set when a wait times out
    unsigned long long *stats;     // [0] nanoseconds spent waiting, [1] waits
    unsigned long long wait_ns;    // time limit of one wait
    int dep_extra;                 // added to every wait's target (0; 1 only in the time-out self-test)
    const typename P::C *g[BATCH_MAX];
    typename P::C *f[BATCH_MAX];
};

__device__ __forceinline__ uint64_t globaltimer_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// wait (one thread) until *ctr >= target; 1 if given up (time limit or error flag)
__device__ __forceinline__ int wait_count(const unsigned *ctr, unsigned target, int *err, unsigned long long limit,
                                          unsigned long long *stats)
{
    const uint64_t t0 = globaltimer_ns();
    for (int n = 0;; ++n) {
        unsigned v;
        asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(ctr) : "memory");
        if (v >= target) {
            if (n > 0) {
                atomicAdd(&stats[0], (unsigned long long)(globaltimer_ns() - t0));
                atomicAdd(&stats[1], 1ull);
            }
            return 0;
        }
        if (*reinterpret_cast<volatile int *>(err)) return 1;
        if (globaltimer_ns() - t0 > limit) {
            atomicExch(err, 1);
            return 1;
        }
        __nanosleep(256);
    }
}

template <int Q, class P, int K>
__global__ void __launch_bounds__(CfgMR<Q>::NT, CfgMR<Q>::MINB) k_batch_mr(const BatchArgs<P> b)
{
    using TM = TileMR<Q, P, K>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_unit, s_job, s_skip;
    __shared__ uint64_t wbar;                                  // the units' input copies
    if (threadIdx.x == 0) {
        mbar_init(&wbar, 1);
        mbar_init_fence();
    }
    __syncthreads();
    unsigned wuse = 0;                                         // phases of wbar used so far
    for (;;) {
        if (threadIdx.x == 0) {
            const int u = (int)atomicAdd(&b.ctr[b.njobs], 1u);
            s_unit = u;
            if (u < b.units) {
                int lo = 0, hi = b.njobs - 1;
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (__ldg(&b.jobs[mid].first) <= u) lo = mid; else hi = mid - 1;
                }
                s_job = lo;
                int skip = *reinterpret_cast<volatile int *>(b.err);
                const int dep = __ldg(&b.jobs[lo].dep);
                if (!skip && dep >= 0)
                    skip = wait_count(&b.ctr[dep], (unsigned)(__ldg(&b.jobs[dep].units) + b.dep_extra), b.err, b.wait_ns,
                                      b.stats);
                s_skip = skip;
            }
        }
        __syncthreads();
        const int u = s_unit;
        if (u >= b.units) break;
        const BatchJob jb = b.jobs[s_job];
        if (!s_skip) {
            // the pass's arguments stay in global memory (read-only for the whole launch; the
            // kernel's shared memory is at the two-CTAs-per-SM limit)
            const KArgs<P> &a = b.desc[jb.desc];
            const int c0 = (u - jb.first) * jb.per;
            const int c1 = min(c0 + jb.per, jb.ctas);
            for (int c = c0; c < c1; ++c) {
                typename TM::Ctx x;
                x.tile0 = c * a.T;
                x.rhs0 = jb.y * MRMAX;
                x.nr = min(MRMAX, a.nrhs - x.rhs0);
                x.npr = a.T << (2 * a.k);
                x.rc = a.rc;
                x.lgp = __ffs(x.npr) - 1;
                TS<typename P::C> ts{};
                const bool used = jb.row ? row_pass_mr<Q, P, K, PM_COMPUTE>(a, b, x, smem_raw, b.f[jb.prob], ts, &wbar, wuse & 1u)
                                         : col_pass_mr<Q, P, K, PM_COMPUTE>(a, b, x, smem_raw, b.g[jb.prob], ts, &wbar, wuse & 1u);
                wuse += used ? 1u : 0u;
                __syncthreads();
            }
        }
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) atomicAdd(&b.ctr[s_job], 1u);
    }
}

}  // namespace bfk
