// Host side of the C ABI declared in include/bf.h: validation, plan
// construction (Chebyshev nodes, Lagrange child->parent matrices, per-level
// feature tables, fusion schedule), device workspace and kernel launches.
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include <cuda.h>   // CUtensorMap and its enums only; the encoder comes from the runtime's driver entry point

#include "../../include/bf.h"
#include "bf_device.cuh"
#include "bf_launch.h"
#include "bf_mr.cuh"
#include <algorithm>

namespace {

constexpr double kPi = 3.14159265358979323846264338327950288;

struct Pass {
    int row;     // 0: init/column/switch pass, 1: row/final pass
    int l0, k, flags;
    int T;       // tiles of 2^{dk} pairs per CTA
};

}  // namespace

struct bf_plan_s {
    int d = 0, L = 0, q = 0, r = 0, m = 0, kind = 0, prec = 0, node_kind = 0, max_nrhs = 1;
    int kc = 0, kr = 0;        // fused levels per column / row pass
    int64_t N = 0, npts = 0;   // N, N^d (= pairs per level)
    bf_params prm{};
    double z[bfk::QMAX] = {};
    double M[2][bfk::QMAX][bfk::QMAX] = {};
    double lsrc[bfk::QMAX] = {}, ltgt[bfk::QMAX] = {};
    void *tt[3] = {}, *st[3] = {};
    void *w0 = nullptr, *w1 = nullptr;
    void *ctab = nullptr;      // target features at box centres, levels 0..ctab_levels
    int ctab_levels = -1;
    void *gstage = nullptr, *fstage = nullptr;
    size_t csize = 8;          // bytes per complex number
    int64_t ws_bytes = 0;
    std::vector<Pass> passes;
    std::vector<Pass> passes_mr;   // schedule of the multi-RHS kernels (empty if not compiled)
    void *ptab = nullptr;          // phase table of the multi-RHS schedule (bf_params.phase_tables)
    int *errflag = nullptr;        // device flag of the table stream's bounded waits
    void *tmaps = nullptr;         // device: CUtensorMap of w0 and of w1 ([rhs][complex]) for the tensor-core switch
    int64_t ptab_bytes = 0;
    std::vector<int64_t> ptab_off, ptab_cta;   // per pass: offset and per-CTA size, complex numbers
    float ptab_build_ms = 0.f;
    float *ftab = nullptr;         // reduced-phase table of the single-RHS schedule (plans with max_nrhs = 1)
    std::vector<int64_t> ftab_off, ftab_cta;   // per pass: offset and per-CTA size, floats
    // arbitrary point sets (bf_plan_create_points): per-point data and the forward passes
    // without init and final, which the point kernels replace
    int points = 0;
    int64_t nsrc = 0, ntgt = 0;
    bfl::PointsData pd{};
    std::vector<void *> pts_mem;
    std::vector<Pass> passes_pts;
    int mr_rc = 1;                 // right-hand sides per scratch chunk of the multi-RHS kernels
    std::vector<Pass> passes_adj;  // schedule whose reverse is the adjoint (fits the row caches)
    const bfl::PassFns *fns = nullptr;
    int last_cuda = 0;
    cudaEvent_t busy_ev = nullptr;     // recorded after the last apply outside a stream capture
    cudaStream_t busy_stream = nullptr;   // the stream it was recorded on
};

struct bf_batch_s {
    int count = 0, njobs = 0, units = 0, prec = 0;
    size_t smem = 0;
    unsigned grid = 0;
    const bfl::PassFns *fns = nullptr;
    void *desc = nullptr;       // device: KArgs per (problem, pass)
    void *jobs = nullptr;       // device: BatchJob per job, in queue order
    void *state = nullptr;      // device: 2 x u64 wait statistics, then the counters below
    unsigned *ctr = nullptr;    // device: [njobs] counters, [njobs] queue head, [njobs + 1] error flag
    float M[2][bfk::QMAX][bfk::QMAX] = {};   // child->parent matrices shared by the problems
    int last_cuda = 0;
};

namespace bfl {
const PassFns *get_fns(int d, int q, int prec, int kind)
{
#define BFL_PICK(dd, kn) (prec == 0 ? fns_d##dd##_f64_##kn(q) : prec == 1 ? fns_d##dd##_mix_##kn(q) : fns_d##dd##_sfu_##kn(q))
    if (d == 2) {
        switch (kind) {
        case BF_PHASE_DOT: return BFL_PICK(2, dot);
        case BF_PHASE_GENRADON: return BFL_PICK(2, genradon);
        case BF_PHASE_HYPRADON: return BFL_PICK(2, hypradon);
        case BF_PHASE_SEPARABLE: return BFL_PICK(2, separable);
        }
    } else if (d == 3) {
        switch (kind) {
        case BF_PHASE_DOT: return BFL_PICK(3, dot);
        case BF_PHASE_GENRADON: return BFL_PICK(3, genradon);
        case BF_PHASE_SEPARABLE: return BFL_PICK(3, separable);
        }
    }
#undef BFL_PICK
    return nullptr;
}
}  // namespace bfl

namespace {

double lagrange1(int q, const double *z, int t, double xi)
{
    double v = 1.0;
    for (int k = 0; k < q; ++k)
        if (k != t) v *= (xi - z[k]) / (z[t] - z[k]);
    return v;
}

bf_status cuda_fail(bf_plan p, cudaError_t e);

// A plan owns one workspace, so an apply issued on another stream while the plan's last
// apply is still running would race on it: that returns BF_ERR_UNSUPPORTED.  Applies
// captured into a CUDA graph are not checked (the graph's launches are the caller's order).
bf_status stream_guard(bf_plan p, cudaStream_t s, bool *capturing)
{
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(s, &cs);
    if (e != cudaSuccess) return cuda_fail(p, e);
    *capturing = cs != cudaStreamCaptureStatusNone;
    if (*capturing || !p->busy_ev || p->busy_stream == s) return BF_OK;
    e = cudaEventQuery(p->busy_ev);
    if (e == cudaErrorNotReady) return BF_ERR_UNSUPPORTED;
    if (e != cudaSuccess) return cuda_fail(p, e);
    return BF_OK;
}

// after an apply's launches: remember its stream and completion (outside a capture)
void stream_mark(bf_plan p, cudaStream_t s, bool capturing)
{
    if (capturing) return;
    if (!p->busy_ev && cudaEventCreateWithFlags(&p->busy_ev, cudaEventDisableTiming) != cudaSuccess) {
        p->busy_ev = nullptr;
        return;
    }
    if (cudaEventRecord(p->busy_ev, s) == cudaSuccess) p->busy_stream = s;
}

bf_status cuda_fail(bf_plan p, cudaError_t e)
{
    if (p) p->last_cuda = (int)e;
    return e == cudaErrorMemoryAllocation ? BF_ERR_NOMEM : BF_ERR_CUDA;
}

// per-dimension feature values of a target (x) or source (y) coordinate, see bf_device.cuh
void tfeat(int kind, double s, int k, double x, double f[3])
{
    f[0] = f[1] = f[2] = 0.0;
    switch (kind) {
    case BF_PHASE_DOT: f[0] = s * x; break;
    case BF_PHASE_GENRADON: f[0] = s * x; f[1] = std::sin(2 * kPi * x); f[2] = std::cos(2 * kPi * x); break;
    case BF_PHASE_HYPRADON: f[0] = s * x; f[1] = x * x; break;
    default: f[0] = s * std::sin(2 * kPi * (x + (k + 1) / 7.0)); break;
    }
}

void sfeat(int kind, double s, int k, double y, double f[2])
{
    if (kind == BF_PHASE_SEPARABLE) {
        f[0] = s * y * y / (k + 2.0);
        f[1] = 0.0;
    } else {
        f[0] = y;
        f[1] = y * y;
    }
}

inline void split(double v, float &hi, float &lo)
{
    hi = (float)v;
    lo = (float)(v - (double)hi);
}

template <class T>
bf_status upload(bf_plan p, const std::vector<T> &h, void **dptr)
{
    cudaError_t e = cudaMalloc(dptr, h.size() * sizeof(T));
    if (e != cudaSuccess) return cuda_fail(p, e);
    e = cudaMemcpy(*dptr, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(p, e);
    return BF_OK;
}

// Feature tables: level l, box i, slot j (j < q: node z_j, j = q: centre, j = q+1: grid point).
bf_status build_tables(bf_plan p)
{
    const int q = p->q, L = p->L, d = p->d;
    const double s = p->prm.phase_scale;
    const int64_t nent = ((2LL << L) - 1) * (q + 2);
    for (int k = 0; k < d; ++k) {
        std::vector<double> T(nent * 3), S(nent * 2);
        for (int l = 0; l <= L; ++l) {
            const int64_t nb = 1LL << l;
            const double w = p->prm.x_w[k] / (double)nb;
            for (int64_t i = 0; i < nb; ++i) {
                const double c = p->prm.x_lo[k] + ((double)i + 0.5) * w;
                for (int j = 0; j < q + 2; ++j) {
                    double x = j < q ? c + w * p->z[j] : (j == q ? c : p->prm.x_lo[k] + ((double)i + p->prm.tgt_off) * w);
                    tfeat(p->kind, s, k, x, &T[((((1LL << l) - 1) * (q + 2)) + i * (q + 2) + j) * 3]);
                }
            }
            const int64_t ns = 1LL << (L - l);
            const double ws = p->prm.y_w[k] * (double)(1LL << l) / (double)(1LL << L);
            for (int64_t i = 0; i < ns; ++i) {
                const double c = p->prm.y_lo[k] + ((double)i + 0.5) * ws;
                for (int j = 0; j < q + 2; ++j) {
                    double y = j < q ? c + ws * p->z[j] : (j == q ? c : p->prm.y_lo[k] + ((double)i + p->prm.src_off) * ws);
                    const int64_t off = ((2LL << L) - (2LL << (L - l))) * (q + 2);
                    sfeat(p->kind, s, k, y, &S[(off + i * (q + 2) + j) * 2]);
                }
            }
        }
        bf_status st;
        if (p->prec == BF_PREC_FP64) {
            std::vector<bfk::PF64::TE> te(nent);
            std::vector<bfk::PF64::SE> se(nent);
            for (int64_t e = 0; e < nent; ++e) {
                te[e].a = make_double2(T[3 * e], T[3 * e + 1]);
                te[e].b = make_double2(T[3 * e + 2], 0.0);
                se[e].a = make_double2(S[2 * e], S[2 * e + 1]);
            }
            if ((st = upload(p, te, &p->tt[k])) != BF_OK) return st;
            if ((st = upload(p, se, &p->st[k])) != BF_OK) return st;
        } else {
            std::vector<bfk::PMIX::TE> te(nent);
            std::vector<bfk::PMIX::SE> se(nent);
            for (int64_t e = 0; e < nent; ++e) {
                float a[8] = {};
                for (int f = 0; f < 3; ++f) split(T[3 * e + f], a[2 * f], a[2 * f + 1]);
                te[e].a = make_float4(a[0], a[1], a[2], a[3]);
                te[e].b = make_float4(a[4], a[5], 0.f, 0.f);
                float b[4];
                split(S[2 * e], b[0], b[1]);
                split(S[2 * e + 1], b[2], b[3]);
                se[e].a = make_float4(b[0], b[1], b[2], b[3]);
            }
            if ((st = upload(p, te, &p->tt[k])) != BF_OK) return st;
            if ((st = upload(p, se, &p->st[k])) != BF_OK) return st;
        }
    }
    return BF_OK;
}

// shared memory of a pass: T tiles of 2^{dk} pairs, plus twice that as stage scratch
size_t pass_smem(const bf_plan_s *p, const Pass &ps)
{
    return (size_t)3 * (size_t)ps.T * ((size_t)1 << (p->d * ps.k)) * (size_t)p->r * p->csize;
}

// plus, for a row pass, the cache of the parents' node features (T 2^{d(k-1)} boxes x r nodes);
// for a column pass, the geometry of every output pair of a level (T 2^{dk} records of the
// centre features and four ints, rounded to 16 bytes)
size_t row_cache_smem(const bf_plan_s *p, const Pass &ps)
{
    if (!ps.row) return (size_t)ps.T * ((size_t)1 << (p->d * ps.k)) * (((size_t)p->fns->tsize + 16 + 15) / 16 * 16);
    if (ps.k < 1) return 0;
    return (size_t)ps.T * ((size_t)1 << (p->d * (ps.k - 1))) * (size_t)p->r * (size_t)p->fns->tsize;
}

// the adjoint row pass caches children's and parents' node features (T (2^{dk} + 2^{d(k-1)}) boxes x r);
// the adjoint column pass with the (unfactorised, d = 2) switch caches the features of every
// (pair, node) of its tiles (T 2^{dk} pairs x r)
size_t row_adj_cache_smem(const bf_plan_s *p, const Pass &ps)
{
    if (!ps.row && (ps.flags & bfk::F_SWITCH) && p->d == 2 && p->kind != BF_PHASE_DOT && p->kind != BF_PHASE_SEPARABLE)
        return (size_t)ps.T * ((size_t)1 << (p->d * ps.k)) * (size_t)p->r * (size_t)p->fns->tsize;
    if (!ps.row || ps.k < 1) return 0;
    return (size_t)ps.T * (((size_t)1 << (p->d * ps.k)) + ((size_t)1 << (p->d * (ps.k - 1)))) * (size_t)p->r *
           (size_t)p->fns->tsize;
}

// multi-RHS pass: nr right-hand sides of T 2^{dk} pairs, scratch for rc of them, a phase cache
// of 5 r factors per pair, with the bank-conflict padding of bf_mr.cuh
size_t mr_smem(const bf_plan_s *p, const Pass &ps, int nr, int rc)
{
    const size_t npr = (size_t)ps.T << (p->d * ps.k);
    return p->csize * (npr * (size_t)p->r * (size_t)(nr + 5) + (size_t)rc * (size_t)bfk::mr_s_stride(p->q, (int64_t)npr) +
                       npr * (size_t)bfk::mr_pc_extra(p->q));
}

// multi-RHS pass reading a phase table: stream control and two table-block buffers, then
// the weights and scratch (no phase cache)
size_t mr_smem_table(const bf_plan_s *p, const Pass &ps, int nr, int rc)
{
    const size_t npr = (size_t)ps.T << (p->d * ps.k);
    const size_t blk = (size_t)(p->q > 5 ? p->q : 5) * (size_t)p->r * npr;
    return (size_t)bfk::TABCTL_BYTES + 2 * blk * p->csize +
           p->csize * (npr * (size_t)p->r * (size_t)nr + (size_t)rc * (size_t)bfk::mr_s_stride(p->q, (int64_t)npr));
}

// A CTA owns np pairs (2^{d kmax} of the instantiation, fewer for tiny problems):
// T = np / 2^{dk} tiles of a k-level pass.
Pass make_pass(const bf_plan_s *p, int64_t np_cta, int row, int l0, int k, int flags)
{
    const int64_t np = p->npts < np_cta ? p->npts : np_cta;
    Pass ps{row, l0, k, flags, (int)(np >> (p->d * k))};
    if (ps.T < 1) ps.T = 1;
    return ps;
}

// column passes of <= kmax levels (init first, switch last), then row passes (final last)
// (rem_first: the short pass of each run of levels goes first instead of last)
std::vector<Pass> schedule(const bf_plan_s *p, int kmax, int64_t np_cta, bool rem_first = false)
{
    std::vector<Pass> out;
    const int m = p->m, L = p->L;
    auto chunk = [&](int left, int total) {
        const int r = total % kmax;
        if (rem_first && r && left == total) return r;
        return left < kmax ? left : kmax;
    };
    if (m == 0) {
        out.push_back(make_pass(p, np_cta, 0, 0, 0, bfk::F_INIT | bfk::F_SWITCH));
    } else {
        for (int l = 0; l < m;) {
            const int k = chunk(m - l, m);
            int fl = 0;
            if (l == 0) fl |= bfk::F_INIT;
            if (l + k == m) fl |= bfk::F_SWITCH;
            out.push_back(make_pass(p, np_cta, 0, l, k, fl));
            l += k;
        }
    }
    for (int l = m; l < L;) {
        const int k = chunk(L - l, L - m);
        out.push_back(make_pass(p, np_cta, 1, l, k, (l + k == L) ? bfk::F_FINAL : 0));
        l += k;
    }
    return out;
}

// whether a precision runs the multi-RHS switch on the tensor cores
bool tc_prec(int prec) { return prec == BF_PREC_BF16X3 || prec == BF_PREC_TF32X3; }

// BF_PREC_BF16X3 / BF_PREC_TF32X3: the multi-RHS column pass that ends at the switch level stops before
// the switch, and a tensor-core switch pass (row = 2, l0 = m) follows it.  With tc_levels
// every column merge level becomes a tensor-core pass of its own (row = 3, k = 1) and the
// init a multi-RHS pass without levels.
void tc_switch_split(const bf_plan_s *p, std::vector<Pass> &sc)
{
    if (!tc_prec(p->prec) || !(p->prec == BF_PREC_TF32X3 ? p->fns->switch_tc32 : p->fns->switch_tc)) return;
    std::vector<Pass> out;
    const bool levels = p->prec == BF_PREC_BF16X3 && p->prm.tc_levels && p->fns->col_tc;
    for (const Pass &ps : sc) {
        if (ps.row != 0) {
            out.push_back(ps);
            continue;
        }
        if (levels) {
            if (ps.flags & bfk::F_INIT)
                out.push_back(make_pass(p, p->fns->mr_nthreads / p->r, 0, 0, 0, bfk::F_INIT));
            for (int l = ps.l0; l < ps.l0 + ps.k; ++l) out.push_back(Pass{3, l, 1, 0, 1});
        } else {
            Pass c = ps;
            c.flags &= ~bfk::F_SWITCH;
            out.push_back(c);
        }
        if (ps.flags & bfk::F_SWITCH) out.push_back(Pass{2, p->m, 0, bfk::F_SWITCH, 1});
    }
    sc = out;
}

template <class P>
void fill_args(const bf_plan_s *p, bfk::KArgs<P> &a)
{
    std::memset(&a, 0, sizeof(a));
    for (int k = 0; k < p->d; ++k) {
        a.tt[k] = static_cast<const typename P::TE *>(p->tt[k]);
        a.st[k] = static_cast<const typename P::SE *>(p->st[k]);
    }
    for (int h = 0; h < 2; ++h)
        for (int t = 0; t < p->q; ++t)
            for (int u = 0; u < p->q; ++u) {
                a.M[h][t][u] = (typename P::R)p->M[h][t][u];
                a.M2[h][t][u].x = a.M2[h][t][u].y = a.M[h][t][u];
            }
    for (int t = 0; t < p->q; ++t) {
        a.lsrc[t] = (typename P::R)p->lsrc[t];
        a.ltgt[t] = (typename P::R)p->ltgt[t];
    }
    const double s = p->prm.phase_scale;
    const double sgn = s > 0 ? 1.0 : (s < 0 ? -1.0 : 0.0);
    if constexpr (P::is_f64) {
        a.sc.s3 = s / 3.0;
        a.sc.sgn = sgn;
    } else {
        float hi, lo;
        split(s / 3.0, hi, lo);
        a.sc.s3hi = hi;
        a.sc.s3lo = lo;
        a.sc.sgn = (float)sgn;
    }
    a.ctab = p->ctab;
    a.ctab_levels = p->ctab_levels;
    a.L = p->L;
    a.kind = p->kind;
    a.npts = p->npts;
    a.wstride = p->npts * p->r;
}

// Sharded apply (bf_apply_shard), rank sr of 2^sg: every pass but the last runs the rank's
// tile groups only (mode 1), T capped so that a group never straddles two ranks' source
// ranges; the last pass runs every tile with the other ranks' inputs read as zero (mode 2).
// Returns the pass to launch and sets the mode and the launch's CTAs (tile groups).
Pass shard_pass(const bf_plan_s *p, Pass ps, bool last, int sg, int *mode, int64_t *ctas)
{
    *mode = 0;
    if (sg > 0 && !last) {
        const int ls = p->d * (p->L - ps.l0 - ps.k);            // log2 of the tiles per target box
        const int64_t tmax = (int64_t)1 << (ls - sg);
        if (ps.T > tmax) ps.T = (int)tmax;
        *mode = 1;
    } else if (sg > 0) {
        *mode = 2;
    }
    *ctas = ((p->npts >> (p->d * ps.k)) / ps.T) >> (*mode == 1 ? sg : 0);
    return ps;
}

// Run passes [first, last) of the forward schedule.  Pass i reads workspace
// buffer i % 2 (or g when it initialises) and writes buffer (i + 1) % 2 (or f
// when it evaluates the targets).
// Multi-RHS forward: every CTA keeps up to mr_max right-hand sides of its tiles and
// evaluates each phase factor once for all of them.
template <class P>
bf_status run_forward_mr(bf_plan p, const void *g, void *f, int nrhs, cudaStream_t s, int first, int last, int sg = 0,
                         int sr = 0, const std::vector<Pass> *sched = nullptr)
{
    const std::vector<Pass> &sc = sched ? *sched : p->passes_mr;
    bfk::KArgs<P> a;
    fill_args<P>(p, a);
    a.g = static_cast<const typename P::C *>(g);
    a.f = static_cast<typename P::C *>(f);
    a.nrhs = nrhs;
    const int mx = p->fns->mr_max;
    const int nr = nrhs < mx ? nrhs : mx;
    a.rc = p->mr_rc < nr ? p->mr_rc : nr;
    void *buf[2] = {p->w0, p->w1};
    const int mode = p->ptab ? bfk::PM_TABLE : bfk::PM_COMPUTE;
    for (int i = first; i < last; ++i) {
        int64_t ctas = 0;
        const Pass ps = shard_pass(p, sc[i], i + 1 == (int)sc.size(), sg, &a.shard_mode, &ctas);
        a.shard_g = sg;
        a.shard_r = sr;
        a.l0 = ps.l0;
        a.k = ps.k;
        a.flags = ps.flags;
        a.T = ps.T;
        a.win = static_cast<const typename P::C *>(buf[i & 1]);
        a.wout = static_cast<typename P::C *>(buf[(i + 1) & 1]);
        a.err = p->errflag;
        a.wmap = (ps.row == 2 && p->tmaps) ? static_cast<const char *>(p->tmaps) + (size_t)(i & 1) * sizeof(CUtensorMap)
                                           : nullptr;   // the map of a.win
        if (ps.row >= 2) {   // the switch (2) or a column level (3) on the tensor cores, persistent CTAs
            int dev = 0, sms = 0;
            cudaGetDevice(&dev);
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            const bool sw = ps.row == 2, t32 = p->prec == BF_PREC_TF32X3;
            const int per_sm = sw ? (t32 ? p->fns->switch_tc32_ctas_per_sm() : p->fns->switch_tc_ctas_per_sm())
                                  : p->fns->col_tc_ctas_per_sm();
            if (per_sm < 1) return BF_ERR_UNSUPPORTED;
            int64_t grid = (p->npts / (sw ? 2 : 4)) >> (a.shard_mode == 1 ? sg : 0);
            if ((int64_t)sms * per_sm < grid) grid = (int64_t)sms * per_sm;
            const bfl::pass_fn fn = sw ? (t32 ? p->fns->switch_tc32 : p->fns->switch_tc) : p->fns->col_tc;
            const size_t smem = sw ? (t32 ? p->fns->switch_tc32_smem : p->fns->switch_tc_smem) : p->fns->col_tc_smem;
            cudaError_t e = fn(&a, (unsigned)grid, (unsigned)((nrhs + 15) / 16), smem, s);
            if (e != cudaSuccess) return cuda_fail(p, e);
            continue;
        }
        a.ptab = p->ptab ? static_cast<typename P::C *>(p->ptab) + p->ptab_off[i] : nullptr;
        a.ptab_cta = p->ptab ? p->ptab_cta[i] : 0;
        a.ncta = (int)ctas;
        const size_t smem = p->ptab ? mr_smem_table(p, ps, nr, a.rc) : mr_smem(p, ps, nr, a.rc);
        int64_t grid = ctas;
        if (p->ptab) {   // as many CTAs as fit; each streams the table of several tile groups
            int dev = 0, sms = 0;
            cudaGetDevice(&dev);
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            const int per_sm = p->fns->mr_table_occupancy(ps.row, smem);
            if (per_sm < 1) return BF_ERR_UNSUPPORTED;
            if ((int64_t)sms * per_sm < grid) grid = (int64_t)sms * per_sm;
        }
        cudaError_t e = (ps.row ? p->fns->row_mr : p->fns->col_mr)[mode](&a, (unsigned)grid,
                                                                         (unsigned)((nrhs + mx - 1) / mx), smem, s);
        if (e != cudaSuccess) return cuda_fail(p, e);
    }
    return BF_OK;
}

template <class P>
bf_status run_forward(bf_plan p, const void *g, void *f, int nrhs, cudaStream_t s, int first, int last, int sg = 0,
                      int sr = 0, const std::vector<Pass> *sched = nullptr)
{
    const std::vector<Pass> &sc = sched ? *sched : p->passes;
    bfk::KArgs<P> a;
    fill_args<P>(p, a);
    a.g = static_cast<const typename P::C *>(g);
    a.f = static_cast<typename P::C *>(f);
    void *buf[2] = {p->w0, p->w1};
    const bool tab = p->ftab && nrhs == 1;   // read the phases from the plan's table
    a.err = p->errflag;
    for (int i = first; i < last; ++i) {
        int64_t ctas = 0;
        const Pass ps = shard_pass(p, sc[i], i + 1 == (int)sc.size(), sg, &a.shard_mode, &ctas);
        a.shard_g = sg;
        a.shard_r = sr;
        a.l0 = ps.l0;
        a.k = ps.k;
        a.flags = ps.flags;
        a.T = ps.T;
        a.win = static_cast<const typename P::C *>(buf[i & 1]);
        a.wout = static_cast<typename P::C *>(buf[(i + 1) & 1]);
        a.ftab = tab ? p->ftab + p->ftab_off[i] : nullptr;
        a.ftab_cta = tab ? p->ftab_cta[i] : 0;
        const size_t smem = pass_smem(p, ps) + row_cache_smem(p, ps);
        const bfl::pass_fn fn = tab ? (ps.row ? p->fns->row_tab : p->fns->col_tab)[1] : (ps.row ? p->fns->row : p->fns->col);
        cudaError_t e = fn(&a, (unsigned)ctas, (unsigned)nrhs, smem, s);
        if (e != cudaSuccess) return cuda_fail(p, e);
    }
    return BF_OK;
}

// Adjoint: the forward schedule reversed.  The adjoint of forward pass i reads
// buffer (i + 1) % 2 (or f when it starts with final^H) and writes buffer i % 2
// (or g when it ends with init^H).
template <class P>
bf_status run_adjoint(bf_plan p, const void *f, void *g, int nrhs, cudaStream_t s)
{
    bfk::KArgs<P> a;
    fill_args<P>(p, a);
    a.fadj = static_cast<const typename P::C *>(f);
    a.gadj = static_cast<typename P::C *>(g);
    void *buf[2] = {p->w0, p->w1};
    for (int i = (int)p->passes_adj.size() - 1; i >= 0; --i) {
        const Pass &ps = p->passes_adj[i];
        a.l0 = ps.l0;
        a.k = ps.k;
        a.flags = ps.flags;
        a.T = ps.T;
        a.win = static_cast<const typename P::C *>(buf[(i + 1) & 1]);
        a.wout = static_cast<typename P::C *>(buf[i & 1]);
        const int64_t ctas = (p->npts >> (p->d * ps.k)) / ps.T;
        const size_t smem = pass_smem(p, ps) + row_adj_cache_smem(p, ps);
        cudaError_t e = (ps.row ? p->fns->row_adj : p->fns->col_adj)(&a, (unsigned)ctas, (unsigned)nrhs, smem, s);
        if (e != cudaSuccess) return cuda_fail(p, e);
    }
    return BF_OK;
}

// Upper bound of |Phi| over X x Y.  The mixed path rounds to integers by adding
// 1.5 * 2^23, which is exact only below 2^22 cycles (kept under 2^21 here).
double phase_bound(int d, int kind, const bf_params *p)
{
    double mx[3], my[3];
    for (int k = 0; k < d; ++k) {
        mx[k] = std::fmax(std::fabs(p->x_lo[k]), std::fabs(p->x_lo[k] + p->x_w[k]));
        my[k] = std::fmax(std::fabs(p->y_lo[k]), std::fabs(p->y_lo[k] + p->y_w[k]));
    }
    double b = 0.0;
    switch (kind) {
    case BF_PHASE_DOT:
        for (int k = 0; k < d; ++k) b += mx[k] * my[k];
        break;
    case BF_PHASE_GENRADON: {
        double q2 = 0.0;
        for (int k = 0; k < d; ++k) {
            b += mx[k] * my[k];
            q2 += my[k] * my[k];                      // a_k(x) <= 1
        }
        b += std::sqrt(q2);
        break;
    }
    case BF_PHASE_HYPRADON:
        b = mx[0] * std::sqrt(my[0] * my[0] + my[1] * my[1] * mx[1] * mx[1]);
        break;
    default:
        for (int k = 0; k < d; ++k) b += 1.0 + my[k] * my[k] / (k + 2.0);
    }
    return std::fabs(p->phase_scale) * b;
}

// the multi-RHS schedule serves nrhs >= 2 where it is compiled (mixed precisions, d = 2)
bool use_mr(const bf_plan_s *p, int nrhs)
{
    return (nrhs >= 2 || p->ptab) && p->prec != BF_PREC_FP64 && !p->passes_mr.empty() && !p->points;
}

// ------------------------------------------------------------ point sets

// Phi in FP64 (cycles) from coordinates, the phase kinds of bf.h
double phi_host(int kind, int d, double s, const double *x, const double *y)
{
    switch (kind) {
    case BF_PHASE_DOT: {
        double v = 0.0;
        for (int k = 0; k < d; ++k) v += x[k] * y[k];
        return s * v;
    }
    case BF_PHASE_GENRADON: {
        double xy = 0.0, q2 = 0.0;
        for (int k = 0; k < d; ++k) xy += x[k] * y[k];
        if (d == 2) {
            const double a0 = (2.0 + std::sin(2 * kPi * x[0]) * std::sin(2 * kPi * x[1])) / 3.0;
            const double a1 = (2.0 + std::cos(2 * kPi * x[0]) * std::cos(2 * kPi * x[1])) / 3.0;
            q2 = a0 * a0 * y[0] * y[0] + a1 * a1 * y[1] * y[1];
        } else {
            for (int k = 0; k < d; ++k) {
                const double a = (2.0 + std::sin(2 * kPi * x[k]) * std::cos(2 * kPi * x[(k + 1) % d])) / 3.0;
                q2 += a * a * y[k] * y[k];
            }
        }
        return s * (xy + std::sqrt(q2));
    }
    case BF_PHASE_HYPRADON:
        return s * x[0] * std::sqrt(y[0] * y[0] + y[1] * y[1] * x[1] * x[1]);
    default: {
        double v = 0.0;
        for (int k = 0; k < d; ++k) v += std::sin(2 * kPi * (x[k] + (k + 1) / 7.0)) + y[k] * y[k] / (k + 2.0);
        return s * v;
    }
    }
}

// leaf box (Morton) of a point and its Lagrange values l_t(xi_k) in that box, [d][q]
int64_t leaf_and_lagrange(const bf_plan_s *p, bool src, const double *pt, double *lag)
{
    const int d = p->d, q = p->q;
    int64_t c[3] = {0, 0, 0}, mort = 0;
    for (int k = 0; k < d; ++k) {
        const double lo = src ? p->prm.y_lo[k] : p->prm.x_lo[k];
        const double w = (src ? p->prm.y_w[k] : p->prm.x_w[k]) / (double)p->N;
        int64_t ck = (int64_t)std::floor((pt[k] - lo) / w);
        ck = ck < 0 ? 0 : (ck >= p->N ? p->N - 1 : ck);
        c[k] = ck;
        const double xi = (pt[k] - (lo + ((double)ck + 0.5) * w)) / w;
        for (int t = 0; t < q; ++t) lag[k * q + t] = lagrange1(q, p->z, t, xi);
    }
    for (int j = 0; j < p->L; ++j)
        for (int k = 0; k < d; ++k) mort |= ((c[k] >> j) & 1) << (j * d + k);
    return mort;
}

template <class T>
bf_status pts_upload(bf_plan p, const std::vector<T> &h, const void **dst)
{
    void *ptr = nullptr;
    if (h.empty()) {
        *dst = nullptr;
        return BF_OK;
    }
    bf_status st = upload(p, h, &ptr);
    if (ptr) p->pts_mem.push_back(ptr);
    *dst = ptr;
    return st;
}

template <class R, class C>
bf_status setup_points_t(bf_plan p, int64_t nsrc, const double *src, int64_t ntgt, const double *tgt)
{
    const int d = p->d, q = p->q;
    const int64_t nbox = p->npts;
    double x0[3], y0[3];
    for (int k = 0; k < d; ++k) {
        x0[k] = p->prm.x_lo[k] + 0.5 * p->prm.x_w[k];
        y0[k] = p->prm.y_lo[k] + 0.5 * p->prm.y_w[k];
    }
    auto cexp = [](double th) {
        const double f = th - std::nearbyint(th);
        C e;
        e.x = (R)std::cos(2 * kPi * f);
        e.y = (R)std::sin(2 * kPi * f);
        return e;
    };
    // sources: leaf boxes, counting sort (stable), Lagrange values and phase factors in sorted order
    std::vector<int64_t> box(nsrc), off(nbox + 1, 0), perm(nsrc);
    std::vector<double> lagd((size_t)nsrc * d * q);
    for (int64_t j = 0; j < nsrc; ++j) {
        box[j] = leaf_and_lagrange(p, true, src + j * d, &lagd[(size_t)j * d * q]);
        ++off[box[j] + 1];
    }
    for (int64_t b = 0; b < nbox; ++b) off[b + 1] += off[b];
    {
        std::vector<int64_t> fill(off.begin(), off.end() - 1);
        for (int64_t j = 0; j < nsrc; ++j) perm[fill[box[j]]++] = j;
    }
    std::vector<R> slag((size_t)nsrc * d * q);
    std::vector<C> se(nsrc);
    for (int64_t i = 0; i < nsrc; ++i) {
        const int64_t j = perm[i];
        for (int e = 0; e < d * q; ++e) slag[(size_t)i * d * q + e] = (R)lagd[(size_t)j * d * q + e];
        se[i] = cexp(phi_host(p->kind, d, p->prm.phase_scale, x0, src + j * d));
    }
    // targets in the caller's order
    std::vector<int64_t> tbox(ntgt);
    std::vector<R> tlag((size_t)ntgt * d * q);
    std::vector<C> te(ntgt);
    std::vector<double> tl(d * q);
    for (int64_t i = 0; i < ntgt; ++i) {
        tbox[i] = leaf_and_lagrange(p, false, tgt + i * d, tl.data());
        for (int e = 0; e < d * q; ++e) tlag[(size_t)i * d * q + e] = (R)tl[e];
        te[i] = cexp(phi_host(p->kind, d, p->prm.phase_scale, tgt + i * d, y0));
    }
    bfl::PointsData &pd = p->pd;
    pd.d = d;
    pd.q = q;
    pd.nbox = nbox;
    pd.nsrc = nsrc;
    pd.ntgt = ntgt;
    pd.wstride = p->npts * p->r;
    bf_status st = BF_OK;
    const void *ptr = nullptr;
    if ((st = pts_upload(p, off, &ptr)) != BF_OK) return st;
    pd.src_off = static_cast<const int64_t *>(ptr);
    if ((st = pts_upload(p, perm, &ptr)) != BF_OK) return st;
    pd.src_perm = static_cast<const int64_t *>(ptr);
    if ((st = pts_upload(p, slag, &pd.src_lag)) != BF_OK) return st;
    if ((st = pts_upload(p, se, &pd.src_e)) != BF_OK) return st;
    if ((st = pts_upload(p, tbox, &ptr)) != BF_OK) return st;
    pd.tgt_box = static_cast<const int64_t *>(ptr);
    if ((st = pts_upload(p, tlag, &pd.tgt_lag)) != BF_OK) return st;
    if ((st = pts_upload(p, te, &pd.tgt_e)) != BF_OK) return st;
    // node factors of every leaf box
    void *ni = nullptr, *nf = nullptr;
    cudaError_t e = cudaMalloc(&ni, (size_t)nbox * p->r * sizeof(C));
    if (ni) p->pts_mem.push_back(ni);
    if (e == cudaSuccess) e = cudaMalloc(&nf, (size_t)nbox * p->r * sizeof(C));
    if (nf) p->pts_mem.push_back(nf);
    if (e != cudaSuccess) return cuda_fail(p, e);
    bfl::PointsGeom geo{};
    geo.d = d;
    geo.L = p->L;
    geo.q = q;
    geo.kind = p->kind;
    geo.s = p->prm.phase_scale;
    for (int k = 0; k < 3; ++k) {
        geo.x_lo[k] = p->prm.x_lo[k];
        geo.x_w[k] = p->prm.x_w[k];
        geo.y_lo[k] = p->prm.y_lo[k];
        geo.y_w[k] = p->prm.y_w[k];
    }
    for (int t = 0; t < q; ++t) geo.z[t] = p->z[t];
    e = bfl::points_nodes(geo, sizeof(R) == 8, ni, nf);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(p, e);
    pd.node_init = ni;
    pd.node_final = nf;
    // the grid schedule without its init and final steps
    p->passes_pts = p->passes;
    p->passes_pts.front().flags &= ~bfk::F_INIT;
    p->passes_pts.back().flags &= ~bfk::F_FINAL;
    p->points = 1;
    p->nsrc = nsrc;
    p->ntgt = ntgt;
    return BF_OK;
}

template <class P>
bf_status run_points(bf_plan p, const void *g, void *f, int nrhs, cudaStream_t s)
{
    const int fp64 = P::is_f64 ? 1 : 0;
    void *buf[2] = {p->w0, p->w1};
    cudaError_t e = p->nsrc ? bfl::points_init(p->pd, fp64, p->r, g, buf[0], nrhs, s)
                            : cudaMemsetAsync(buf[0], 0, (size_t)nrhs * p->npts * p->r * p->csize, s);
    if (e != cudaSuccess) return cuda_fail(p, e);
    bfk::KArgs<P> a;
    fill_args<P>(p, a);
    const int n = (int)p->passes_pts.size();
    for (int i = 0; i < n; ++i) {
        const Pass &ps = p->passes_pts[i];
        a.l0 = ps.l0;
        a.k = ps.k;
        a.flags = ps.flags;
        a.T = ps.T;
        a.win = static_cast<const typename P::C *>(buf[i & 1]);
        a.wout = static_cast<typename P::C *>(buf[(i + 1) & 1]);
        const int64_t ctas = (p->npts >> (p->d * ps.k)) / ps.T;
        const size_t smem = pass_smem(p, ps) + row_cache_smem(p, ps);
        e = (ps.row ? p->fns->row : p->fns->col)(&a, (unsigned)ctas, (unsigned)nrhs, smem, s);
        if (e != cudaSuccess) return cuda_fail(p, e);
    }
    e = bfl::points_final(p->pd, fp64, p->r, buf[n & 1], f, nrhs, s);
    if (e != cudaSuccess) return cuda_fail(p, e);
    return BF_OK;
}

// Phase table of the multi-RHS schedule: per pass and CTA, the init factors, 5 r per pair for
// each level, the r x r switch matrices and the final factors, in the order the kernels read them.
template <class P>
bf_status build_phase_table(bf_plan p)
{
    const int64_t r = p->r;
    int64_t total = 0;
    p->ptab_off.clear();
    p->ptab_cta.clear();
    for (const Pass &ps : p->passes_mr) {
        const int64_t npr = (int64_t)ps.T << (p->d * ps.k), ctas = (p->npts >> (p->d * ps.k)) / ps.T;
        int64_t per = ps.k * 5 * r * npr;
        if (ps.flags & bfk::F_INIT) per += r * npr;
        if (ps.flags & bfk::F_SWITCH) per += r * r * npr;
        if (ps.flags & bfk::F_FINAL) per += (r + 1) * npr;
        p->ptab_off.push_back(total);
        p->ptab_cta.push_back(per);
        total += per * ctas;
    }
    p->ptab_bytes = total * (int64_t)sizeof(typename P::C);
    cudaError_t e = cudaMalloc(&p->ptab, (size_t)p->ptab_bytes);
    if (e != cudaSuccess) {
        p->ptab = nullptr;
        return cuda_fail(p, e);
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0);
    bfk::KArgs<P> a;
    fill_args<P>(p, a);
    a.nrhs = 1;
    a.rc = 1;
    for (size_t i = 0; i < p->passes_mr.size() && e == cudaSuccess; ++i) {
        const Pass &ps = p->passes_mr[i];
        a.l0 = ps.l0;
        a.k = ps.k;
        a.flags = ps.flags;
        a.T = ps.T;
        a.ptab = static_cast<typename P::C *>(p->ptab) + p->ptab_off[i];
        a.ptab_cta = p->ptab_cta[i];
        const int64_t ctas = (p->npts >> (p->d * ps.k)) / ps.T;
        a.ncta = (int)ctas;
        e = (ps.row ? p->fns->row_mr : p->fns->col_mr)[bfk::PM_BUILD](&a, (unsigned)ctas, 1u, mr_smem(p, ps, 1, 1), 0);
    }
    cudaEventRecord(e1);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    p->ptab_build_ms = ms;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return cuda_fail(p, e);
    return BF_OK;
}

// Reduced-phase table of the single-RHS schedule: the build passes run the evaluating
// kernels on zero input and record, per CTA and stage, the reduced phase of every factor
// (floats, [phase of an item][item]); the apply reads them instead of evaluating Phi.
// The switch of the factorised kinds keeps evaluating (d q^2 phases per pair).
template <class P>
bf_status build_tile_table(bf_plan p)
{
    const int64_t r = p->r;
    const bool tab_switch = p->kind != BF_PHASE_DOT && p->kind != BF_PHASE_SEPARABLE;
    int64_t total = 0;
    p->ftab_off.clear();
    p->ftab_cta.clear();
    for (const Pass &ps : p->passes) {
        const int64_t npr = (int64_t)ps.T << (p->d * ps.k), ctas = (p->npts >> (p->d * ps.k)) / ps.T;
        int64_t per = ps.k * ((1 << p->d) + 1) * r * npr;   // per pair and level: 2^d r modulations, r demodulations
        if (!ps.row && (ps.flags & bfk::F_SWITCH) && tab_switch) per += r * r * npr;
        p->ftab_off.push_back(total);
        p->ftab_cta.push_back(per);
        total += per * ctas;
    }
    p->ptab_bytes = total * (int64_t)sizeof(float);
    cudaError_t e = cudaMalloc(&p->ftab, (size_t)p->ptab_bytes);
    if (e != cudaSuccess) {
        p->ftab = nullptr;
        return cuda_fail(p, e);
    }
    void *gz = nullptr, *fz = nullptr;
    const size_t vbytes = (size_t)p->npts * p->csize;
    e = cudaMalloc(&gz, vbytes);
    if (e == cudaSuccess) e = cudaMalloc(&fz, vbytes);
    if (e == cudaSuccess) e = cudaMemset(gz, 0, vbytes);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) e = cudaEventRecord(e0);
    bfk::KArgs<P> a;
    fill_args<P>(p, a);
    a.g = static_cast<const typename P::C *>(gz);
    a.f = static_cast<typename P::C *>(fz);
    a.err = p->errflag;
    void *buf[2] = {p->w0, p->w1};
    for (size_t i = 0; i < p->passes.size() && e == cudaSuccess; ++i) {
        const Pass &ps = p->passes[i];
        a.l0 = ps.l0;
        a.k = ps.k;
        a.flags = ps.flags;
        a.T = ps.T;
        a.win = static_cast<const typename P::C *>(buf[i & 1]);
        a.wout = static_cast<typename P::C *>(buf[(i + 1) & 1]);
        a.ftab = p->ftab + p->ftab_off[i];
        a.ftab_cta = p->ftab_cta[i];
        const int64_t ctas = (p->npts >> (p->d * ps.k)) / ps.T;
        const size_t smem = pass_smem(p, ps) + row_cache_smem(p, ps);
        e = (ps.row ? p->fns->row_tab : p->fns->col_tab)[0](&a, (unsigned)ctas, 1u, smem, 0);
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
    p->ptab_build_ms = ms;
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (gz) cudaFree(gz);
    if (fz) cudaFree(fz);
    if (e != cudaSuccess) return cuda_fail(p, e);
    return BF_OK;
}

const std::vector<Pass> &schedule_for(const bf_plan_s *p, int nrhs) { return use_mr(p, nrhs) ? p->passes_mr : p->passes; }

// Tensor maps of the two weight buffers viewed as [rhs][complex number] (8-byte elements,
// max_nrhs rows of N^d r), with boxes of 2 r complex numbers x 16 right-hand sides: one
// tiled bulk copy stages a unit (two pairs) of the tensor-core switch.  The encoder comes
// from the driver through the runtime (no link to the driver library).  Left null -- the
// switch then stages with cp.async -- when the encoder is not available or refuses.
void build_weight_maps(bf_plan p)
{
    typedef CUresult (*encode_fn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
    static const encode_fn enc = []() -> encode_fn {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            return nullptr;
        return reinterpret_cast<encode_fn>(fn);
    }();
    if (!enc || p->d != 2 || 2 * p->r > 256) return;
    CUtensorMap maps[2];
    const cuuint64_t dims[2] = {(cuuint64_t)p->npts * (cuuint64_t)p->r, (cuuint64_t)p->max_nrhs};
    const cuuint64_t strides[1] = {(cuuint64_t)p->npts * (cuuint64_t)p->r * 8u};
    const cuuint32_t box[2] = {(cuuint32_t)(2 * p->r), 16u};
    const cuuint32_t estr[2] = {1u, 1u};
    void *bufs[2] = {p->w0, p->w1};
    for (int j = 0; j < 2; ++j)
        if (enc(&maps[j], CU_TENSOR_MAP_DATA_TYPE_UINT64, 2, bufs[j], dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return;
    void *d = nullptr;
    if (cudaMalloc(&d, sizeof(maps)) != cudaSuccess) return;
    if (cudaMemcpy(d, maps, sizeof(maps), cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaFree(d);
        return;
    }
    p->tmaps = d;
}

bool supported_q(int d, int q) { return bfl::get_fns(d, q, 1, 0) != nullptr && bfl::get_fns(d, q, 0, 0) != nullptr; }

}  // namespace

// ---------------------------------------------------------------- batches

namespace {

template <class P>
bf_status batch_build(bf_batch b, const bf_plan *plans, const int *nrhs, int count)
{
    std::vector<bfk::KArgs<P>> desc;
    struct J { bfk::BatchJob j; int pass; int key; };
    std::vector<J> jobs;
    std::vector<int> desc0(count);
    size_t smem = 0;
    for (int i = 0; i < count; ++i) {
        const bf_plan p = plans[i];
        const int nr = nrhs[i] < p->fns->mr_max ? nrhs[i] : p->fns->mr_max;
        const int rc = p->mr_rc < nr ? p->mr_rc : nr;
        const int ny = (nrhs[i] + p->fns->mr_max - 1) / p->fns->mr_max;
        void *buf[2] = {p->w0, p->w1};
        desc0[i] = (int)desc.size();
        for (size_t j = 0; j < p->passes_mr.size(); ++j) {
            const Pass &ps = p->passes_mr[j];
            bfk::KArgs<P> a;
            fill_args<P>(p, a);
            a.l0 = ps.l0;
            a.k = ps.k;
            a.flags = ps.flags;
            a.T = ps.T;
            a.win = static_cast<const typename P::C *>(buf[j & 1]);
            a.wout = static_cast<typename P::C *>(buf[(j + 1) & 1]);
            a.nrhs = nrhs[i];
            a.rc = rc;
            a.ncta = (int)((p->npts >> (p->d * ps.k)) / ps.T);
            desc.push_back(a);
            const size_t sm = mr_smem(p, ps, nr, rc);
            if (sm > smem) smem = sm;
            const int ctas = (int)((p->npts >> (p->d * ps.k)) / ps.T);
            for (int y = 0; y < ny; ++y) {
                J jb{};
                jb.j.prob = i;
                jb.j.desc = desc0[i] + (int)j;
                jb.j.y = y;
                jb.j.ctas = ctas;
                jb.j.row = ps.row;
                jb.pass = (int)j;
                jobs.push_back(jb);
            }
        }
    }
    // queue order: pass index first (a job's dependency is always earlier), larger jobs first
    std::stable_sort(jobs.begin(), jobs.end(), [](const J &x, const J &y) {
        if (x.pass != y.pass) return x.pass < y.pass;
        return x.j.ctas > y.j.ctas;
    });
    // a work unit runs `per` consecutive CTAs of a job: about 512 units per CTA slot over the
    // whole queue, so taking a unit (an atomic and a table search) costs a few percent at
    // most while the last units still balance
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const size_t smem_total = smem;
    if (smem_total > 227 * 1024) return BF_ERR_UNSUPPORTED;
    const int per_sm = b->fns->batch_ctas_per_sm(smem_total);
    if (per_sm < 1) return BF_ERR_UNSUPPORTED;
    int64_t all_ctas = 0;
    for (const J &x : jobs) all_ctas += x.j.ctas;
    const int64_t slots = (int64_t)sms * per_sm;
    int64_t per = all_ctas / (slots * 512);
    per = per < 1 ? 1 : (per > 16 ? 16 : per);
    std::vector<bfk::BatchJob> hj(jobs.size());
    int first = 0;
    for (size_t n = 0; n < jobs.size(); ++n) {
        hj[n] = jobs[n].j;
        hj[n].per = (int)per;
        hj[n].units = (int)((hj[n].ctas + per - 1) / per);
        hj[n].first = first;
        first += hj[n].units;
        hj[n].dep = -1;
        if (jobs[n].pass > 0)
            for (size_t m = 0; m < n; ++m)
                if (jobs[m].j.prob == jobs[n].j.prob && jobs[m].j.y == jobs[n].j.y && jobs[m].pass == jobs[n].pass - 1)
                    hj[n].dep = (int)m;
        if (jobs[n].pass > 0 && hj[n].dep < 0) return BF_ERR_INTERNAL;
    }
    b->njobs = (int)hj.size();
    b->units = first;
    b->smem = smem_total;
    cudaError_t e = cudaMalloc(&b->desc, desc.size() * sizeof(bfk::KArgs<P>));
    if (e == cudaSuccess) e = cudaMemcpy(b->desc, desc.data(), desc.size() * sizeof(bfk::KArgs<P>), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&b->jobs, hj.size() * sizeof(bfk::BatchJob));
    if (e == cudaSuccess) e = cudaMemcpy(b->jobs, hj.data(), hj.size() * sizeof(bfk::BatchJob), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&b->state, 16 + (hj.size() + 2) * sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMemset(b->state, 0, 16 + (hj.size() + 2) * sizeof(unsigned));
    b->ctr = reinterpret_cast<unsigned *>(static_cast<char *>(b->state) + 16);
    for (int h = 0; h < 2; ++h)
        for (int t = 0; t < bfk::QMAX; ++t)
            for (int u = 0; u < bfk::QMAX; ++u) b->M[h][t][u] = (float)desc[0].M[h][t][u];
    if (e != cudaSuccess) {
        b->last_cuda = (int)e;
        return e == cudaErrorMemoryAllocation ? BF_ERR_NOMEM : BF_ERR_CUDA;
    }
    const int64_t grid = slots;
    b->grid = (unsigned)(grid < b->units ? grid : b->units);
    return BF_OK;
}

template <class P>
bf_status batch_launch(bf_batch b, const void *const *g, void *const *f, cudaStream_t s, unsigned long long wait_ns,
                       int dep_extra)
{
    bfk::BatchArgs<P> a;
    std::memset(&a, 0, sizeof(a));
    a.desc = static_cast<const bfk::KArgs<P> *>(b->desc);
    a.jobs = static_cast<const bfk::BatchJob *>(b->jobs);
    a.njobs = b->njobs;
    a.units = b->units;
    a.ctr = b->ctr;
    a.err = reinterpret_cast<int *>(b->ctr + b->njobs + 1);
    a.stats = static_cast<unsigned long long *>(b->state);
    std::memcpy(a.M, b->M, sizeof(a.M));
    a.wait_ns = wait_ns;
    a.dep_extra = dep_extra;
    for (int i = 0; i < b->count; ++i) {
        a.g[i] = static_cast<const typename P::C *>(g[i]);
        a.f[i] = static_cast<typename P::C *>(f[i]);
    }
    cudaError_t e = cudaMemsetAsync(b->state, 0, 16 + (size_t)(b->njobs + 2) * sizeof(unsigned), s);
    if (e == cudaSuccess) e = b->fns->batch(&a, b->grid, b->smem, s);
    if (e != cudaSuccess) {
        b->last_cuda = (int)e;
        return BF_ERR_CUDA;
    }
    return BF_OK;
}

bf_status batch_apply(bf_batch b, const void *const *g, void *const *f, void *stream, unsigned long long wait_ns,
                      int dep_extra)
{
    if (!b || !g || !f) return BF_ERR_INVALID_ARG;
    for (int i = 0; i < b->count; ++i)
        if (!g[i] || !f[i] || ((uintptr_t)g[i] & 15) || ((uintptr_t)f[i] & 15)) return BF_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (b->prec == BF_PREC_MIXED_SFU) return batch_launch<bfk::PMIXF>(b, g, f, s, wait_ns, dep_extra);
    return batch_launch<bfk::PMIX>(b, g, f, s, wait_ns, dep_extra);
}

}  // namespace

extern "C" {

const char *bf_status_string(bf_status s)
{
    switch (s) {
    case BF_OK: return "BF_OK";
    case BF_ERR_INVALID_ARG: return "BF_ERR_INVALID_ARG";
    case BF_ERR_UNSUPPORTED: return "BF_ERR_UNSUPPORTED";
    case BF_ERR_NOMEM: return "BF_ERR_NOMEM";
    case BF_ERR_CUDA: return "BF_ERR_CUDA";
    case BF_ERR_TIMEOUT: return "BF_ERR_TIMEOUT";
    case BF_ERR_INTERNAL: return "BF_ERR_INTERNAL";
    }
    return "BF_ERR_UNKNOWN";
}

bf_status bf_params_default(int d, int64_t N, bf_params *out)
{
    if (!out || d < 1 || d > 3 || N < 1) return BF_ERR_INVALID_ARG;
    std::memset(out, 0, sizeof(*out));
    for (int k = 0; k < 3; ++k) {
        out->x_lo[k] = 0.0;
        out->x_w[k] = 1.0;
        out->y_lo[k] = -0.5 * (double)N;
        out->y_w[k] = (double)N;
    }
    out->phase_scale = 1.0;
    out->precision = BF_PREC_MIXED;
    out->switch_level = -1;
    out->max_nrhs = 1;
    return BF_OK;
}

bf_status bf_plan_create(int d, int64_t N, int q, bf_phase_kind phase, const bf_params *prm, bf_plan *out)
{
    if (!out || !prm) return BF_ERR_INVALID_ARG;
    *out = nullptr;
    if (d < 2 || d > 3) return d == 1 ? BF_ERR_UNSUPPORTED : BF_ERR_INVALID_ARG;
    if (N < 2 || (N & (N - 1))) return BF_ERR_INVALID_ARG;
    int L = 0;
    while ((1LL << L) < N) ++L;
    if ((int64_t)L * d > 30) return BF_ERR_INVALID_ARG;
    if (q < 2 || q > bfk::QMAX) return BF_ERR_INVALID_ARG;
    if ((int)phase < 0 || (int)phase > 3) return BF_ERR_INVALID_ARG;
    if (phase == BF_PHASE_HYPRADON && d != 2) return BF_ERR_INVALID_ARG;
    if (prm->precision < BF_PREC_FP64 || prm->precision > BF_PREC_TF32X3) return BF_ERR_INVALID_ARG;
    if (!supported_q(d, q)) return BF_ERR_UNSUPPORTED;
    if (prm->precision != BF_PREC_FP64 && phase_bound(d, (int)phase, prm) >= 2097152.0) return BF_ERR_UNSUPPORTED;
    for (int k = 0; k < d; ++k) {
        if (!(prm->x_w[k] > 0.0) || !(prm->y_w[k] > 0.0)) return BF_ERR_INVALID_ARG;
        if (!std::isfinite(prm->x_lo[k]) || !std::isfinite(prm->y_lo[k]) || !std::isfinite(prm->x_w[k]) ||
            !std::isfinite(prm->y_w[k]))
            return BF_ERR_INVALID_ARG;
    }
    if (!std::isfinite(prm->phase_scale)) return BF_ERR_INVALID_ARG;
    if (!(prm->tgt_off >= 0.0 && prm->tgt_off < 1.0 && prm->src_off >= 0.0 && prm->src_off < 1.0))
        return BF_ERR_INVALID_ARG;
    if (prm->switch_level < -1 || prm->switch_level >= L) return BF_ERR_INVALID_ARG;
    if (prm->node_kind != 0 && prm->node_kind != 1) return BF_ERR_INVALID_ARG;
    if (prm->max_nrhs < 1 || prm->max_nrhs > 65535) return BF_ERR_INVALID_ARG;
    if (prm->fuse_levels < 0 || prm->fuse_levels > 8) return BF_ERR_INVALID_ARG;
    for (int i = 0; i < 4; ++i)
        if (prm->reserved[i]) return BF_ERR_INVALID_ARG;
    if (prm->phase_tables != 0 && prm->phase_tables != 1) return BF_ERR_INVALID_ARG;
    if (prm->tc_levels != 0 && prm->tc_levels != 1) return BF_ERR_INVALID_ARG;
    if (prm->tc_cpasync != 0 && prm->tc_cpasync != 1) return BF_ERR_INVALID_ARG;
    if (prm->phase_tables && (prm->precision == BF_PREC_FP64 || tc_prec(prm->precision) || (d == 2 && q > 5)))
        return BF_ERR_UNSUPPORTED;

    bf_plan p = new (std::nothrow) bf_plan_s();
    if (!p) return BF_ERR_NOMEM;
    p->d = d;
    p->L = L;
    p->q = q;
    p->r = bfk::ipow(q, d);
    p->N = N;
    p->npts = 1LL << (L * d);
    p->m = prm->switch_level < 0 ? L / 2 : prm->switch_level;
    p->kind = (int)phase;
    p->prec = prm->precision;
    p->node_kind = prm->node_kind;
    p->max_nrhs = prm->max_nrhs;
    p->prm = *prm;
    p->csize = p->prec == BF_PREC_FP64 ? 16 : 8;
    // BF16X3 and TF32X3 evaluate their phases as BF_PREC_MIXED does and run the same kernels but the switch
    p->fns = bfl::get_fns(d, q, tc_prec(p->prec) ? (int)BF_PREC_MIXED : (int)p->prec, (int)phase);
    if (!p->fns) {   // this combination was not compiled into the library
        delete p;
        return BF_ERR_UNSUPPORTED;
    }

    for (int j = 0; j < q; ++j)
        p->z[j] = p->node_kind == 0 ? 0.5 * std::cos(j * kPi / (q - 1)) : 0.5 * std::cos((2 * j + 1) * kPi / (2.0 * q));
    for (int h = 0; h < 2; ++h)
        for (int t = 0; t < q; ++t)
            for (int u = 0; u < q; ++u) p->M[h][t][u] = lagrange1(q, p->z, t, (p->z[u] + h - 0.5) / 2.0);
    for (int t = 0; t < q; ++t) {
        p->lsrc[t] = lagrange1(q, p->z, t, prm->src_off - 0.5);
        p->ltgt[t] = lagrange1(q, p->z, t, prm->tgt_off - 0.5);
    }

    const int kfit = p->fns->kmax;
    const int kreq = prm->fuse_levels > 0 ? prm->fuse_levels : kfit;
    p->kc = p->kr = kreq < kfit ? kreq : kfit;
    p->passes = schedule(p, p->kc, p->fns->np, true);
    if (p->fns->col_mr[0]) {
        // 2 fused levels, as many pairs per CTA as one switch round covers (at least one tile);
        // scratch for enough right-hand sides to give every thread an item, fewer if the
        // shared memory of one CTA does not hold them
        const int kmr = kreq < 2 ? kreq : 2;
        const int nr = p->max_nrhs < p->fns->mr_max ? p->max_nrhs : p->fns->mr_max;
        const int64_t ppr = p->fns->mr_nthreads / p->r;
        p->passes_mr = schedule(p, kmr, ppr, true);
        tc_switch_split(p, p->passes_mr);
        int64_t npr = 0;
        for (const Pass &ps : p->passes_mr)
            if (((int64_t)ps.T << (d * ps.k)) > npr) npr = (int64_t)ps.T << (d * ps.k);
        int rc = (int)(p->fns->mr_nthreads / (npr * q));
        rc = rc < 1 ? 1 : (rc > nr ? nr : rc);
        bool fits = false;
        for (; rc >= 1 && !fits; --rc) {
            fits = true;
            for (const Pass &ps : p->passes_mr)
                if (ps.row < 2 && mr_smem(p, ps, nr, rc) > 227 * 1024) fits = false;
            if (fits) p->mr_rc = rc;
        }
        if (!fits) p->passes_mr.clear();
    }
    // the adjoint's row passes also hold target-feature caches: fuse fewer levels, then put
    // fewer tiles in a CTA, until every pass fits the shared memory of one CTA
    {
        bool fits = false;
        for (int ka = p->kc; ka >= 1 && !fits; --ka) {
            for (int64_t np = p->fns->np; np >= (1LL << (d * ka)) && !fits; np >>= d) {
                p->passes_adj = schedule(p, ka, np);
                fits = true;
                for (const Pass &ps : p->passes_adj)
                    if (pass_smem(p, ps) + row_adj_cache_smem(p, ps) > 227 * 1024) fits = false;
            }
        }
    }

    bf_status st = build_tables(p);
    if (st == BF_OK) {
        // target features at box centres for the column levels (<= 2^18 records)
        int lv = p->m;
        while (lv > 0 && (((1LL << (d * (lv + 1))) - 1) / ((1LL << d) - 1)) > (1LL << 18)) --lv;
        const size_t bytes = (size_t)((((1LL << (d * (lv + 1))) - 1) / ((1LL << d) - 1))) * p->fns->tsize;
        cudaError_t e = cudaMalloc(&p->ctab, bytes);
        if (e == cudaSuccess) {
            if (p->prec == BF_PREC_FP64) {
                bfk::KArgs<bfk::PF64> a;
                fill_args<bfk::PF64>(p, a);
                e = p->fns->center_table(&a, p->ctab, lv);
            } else {
                bfk::KArgs<bfk::PMIX> a;
                fill_args<bfk::PMIX>(p, a);
                e = p->fns->center_table(&a, p->ctab, lv);
            }
            if (e == cudaSuccess) e = cudaDeviceSynchronize();
        }
        if (e != cudaSuccess)
            st = cuda_fail(p, e);
        else
            p->ctab_levels = lv;
    }
    // phase tables: the single-RHS schedule's reduced phases for plans of one right-hand side,
    // the multi-RHS schedule's factors otherwise
    const bool tile_table = prm->phase_tables && p->max_nrhs == 1 && p->fns->col_tab[0];
    if (st == BF_OK && prm->phase_tables) {
        cudaError_t e = cudaMalloc(&p->errflag, sizeof(int));
        if (e == cudaSuccess) e = cudaMemset(p->errflag, 0, sizeof(int));
        if (e != cudaSuccess)
            st = cuda_fail(p, e);
        else if (tile_table)
            ;   // built below, once the weight buffers exist
        else if (p->passes_mr.empty())
            st = BF_ERR_UNSUPPORTED;
        else
            st = p->prec == BF_PREC_MIXED_SFU ? build_phase_table<bfk::PMIXF>(p) : build_phase_table<bfk::PMIX>(p);
    }
    if (st == BF_OK && !p->errflag && tc_prec(p->prec)) {   // the tensor-core switch's bounded waits
        cudaError_t e = cudaMalloc(&p->errflag, sizeof(int));
        if (e == cudaSuccess) e = cudaMemset(p->errflag, 0, sizeof(int));
        if (e != cudaSuccess) st = cuda_fail(p, e);
    }
    if (st == BF_OK) {
        const size_t wbytes = (size_t)p->max_nrhs * (size_t)p->npts * (size_t)p->r * p->csize;
        cudaError_t e = cudaMalloc(&p->w0, wbytes);
        if (e == cudaSuccess) e = cudaMalloc(&p->w1, wbytes);
        if (e != cudaSuccess) st = cuda_fail(p, e);
        if (st == BF_OK && tile_table)
            st = p->prec == BF_PREC_MIXED_SFU ? build_tile_table<bfk::PMIXF>(p) : build_tile_table<bfk::PMIX>(p);
        // tiled copies for the tensor-core switch (measured faster than cp.async in both formats)
        if (st == BF_OK && tc_prec(p->prec) && !prm->tc_cpasync && p->max_nrhs >= 2 && p->fns->switch_tc)
            build_weight_maps(p);
        p->ws_bytes = (int64_t)(2 * wbytes) + p->ptab_bytes;
    }
    if (st != BF_OK) {
        bf_destroy(p);
        return st;
    }
    *out = p;
    return BF_OK;
}

bf_status bf_plan_create_points(int d, int64_t N, int q, bf_phase_kind phase, const bf_params *prm, int64_t nsrc,
                                const double *src, int64_t ntgt, const double *tgt, bf_plan *out)
{
    if (!out) return BF_ERR_INVALID_ARG;
    *out = nullptr;
    if (!prm || nsrc < 0 || ntgt < 0 || (nsrc > 0 && !src) || (ntgt > 0 && !tgt)) return BF_ERR_INVALID_ARG;
    if (nsrc > ((int64_t)1 << 40) || ntgt > ((int64_t)1 << 40)) return BF_ERR_INVALID_ARG;
    if (prm->phase_tables) return BF_ERR_UNSUPPORTED;
    for (int64_t i = 0; i < nsrc * (int64_t)(d > 0 ? d : 0); ++i)
        if (!std::isfinite(src[i])) return BF_ERR_INVALID_ARG;
    for (int64_t i = 0; i < ntgt * (int64_t)(d > 0 ? d : 0); ++i)
        if (!std::isfinite(tgt[i])) return BF_ERR_INVALID_ARG;
    bf_plan p = nullptr;
    bf_status st = bf_plan_create(d, N, q, phase, prm, &p);
    if (st != BF_OK) return st;
    st = p->prec == BF_PREC_FP64 ? setup_points_t<double, double2>(p, nsrc, src, ntgt, tgt)
                                 : setup_points_t<float, float2>(p, nsrc, src, ntgt, tgt);
    if (st != BF_OK) {
        bf_destroy(p);
        return st;
    }
    *out = p;
    return BF_OK;
}

bf_status bf_plan_points_info(bf_plan p, int *is_points, int64_t *nsrc, int64_t *ntgt)
{
    if (!p) return BF_ERR_INVALID_ARG;
    if (is_points) *is_points = p->points;
    if (nsrc) *nsrc = p->points ? p->nsrc : p->npts;
    if (ntgt) *ntgt = p->points ? p->ntgt : p->npts;
    return BF_OK;
}

bf_status bf_apply(bf_plan p, const void *g, void *f, int nrhs, void *stream)
{
    if (!p) return BF_ERR_INVALID_ARG;
    if (nrhs < 0 || nrhs > p->max_nrhs) return BF_ERR_INVALID_ARG;
    if (nrhs == 0) return BF_OK;
    // (an empty point set needs no buffer)
    if ((!g && !(p->points && p->nsrc == 0)) || (!f && !(p->points && p->ntgt == 0))) return BF_ERR_INVALID_ARG;
    if (((uintptr_t)g & 15) || ((uintptr_t)f & 15)) return BF_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    bool capturing = false;
    bf_status st = stream_guard(p, s, &capturing);
    if (st != BF_OK) return st;
    if (p->points) {
        if (p->prec == BF_PREC_FP64) st = run_points<bfk::PF64>(p, g, f, nrhs, s);
        else if (p->prec == BF_PREC_MIXED_SFU) st = run_points<bfk::PMIXF>(p, g, f, nrhs, s);
        else st = run_points<bfk::PMIX>(p, g, f, nrhs, s);
    } else {
        const int n = (int)schedule_for(p, nrhs).size();
        if (p->prec == BF_PREC_FP64) st = run_forward<bfk::PF64>(p, g, f, nrhs, s, 0, n);
        else if (use_mr(p, nrhs))
            st = p->prec == BF_PREC_MIXED_SFU ? run_forward_mr<bfk::PMIXF>(p, g, f, nrhs, s, 0, n)
                                              : run_forward_mr<bfk::PMIX>(p, g, f, nrhs, s, 0, n);
        else
            st = p->prec == BF_PREC_MIXED_SFU ? run_forward<bfk::PMIXF>(p, g, f, nrhs, s, 0, n)
                                              : run_forward<bfk::PMIX>(p, g, f, nrhs, s, 0, n);
    }
    stream_mark(p, s, capturing);
    return st;
}

bf_status bf_apply_shard(bf_plan p, const void *g, void *f, int nrhs, int shard_g, int shard_r, void *stream)
{
    if (!p) return BF_ERR_INVALID_ARG;
    if (nrhs < 0 || nrhs > p->max_nrhs) return BF_ERR_INVALID_ARG;
    if (shard_g < 0 || shard_g > p->d || shard_r < 0 || shard_r >= (1 << shard_g)) return BF_ERR_INVALID_ARG;
    if (p->points || p->ptab || p->ftab) return BF_ERR_UNSUPPORTED;
    if (nrhs == 0) return BF_OK;
    if (!g || !f || ((uintptr_t)g & 15) || ((uintptr_t)f & 15)) return BF_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    bool capturing = false;
    bf_status st = stream_guard(p, s, &capturing);
    if (st != BF_OK) return st;
    // the last pass runs on every pair: keep it to one level (its other levels become a pass
    // of their own, with the same pairs per CTA, that runs on the rank's pairs)
    std::vector<Pass> sc = schedule_for(p, nrhs);
    if (shard_g > 0 && sc.back().k > 1) {
        const Pass last = sc.back();
        const int64_t npr = (int64_t)last.T << (p->d * last.k);
        sc.back() = Pass{last.row, last.l0, last.k - 1, last.flags & ~bfk::F_FINAL, (int)(npr >> (p->d * (last.k - 1)))};
        sc.push_back(Pass{last.row, last.l0 + last.k - 1, 1, last.flags, (int)(npr >> p->d)});
    }
    const int n = (int)sc.size();
    if (p->prec == BF_PREC_FP64) st = run_forward<bfk::PF64>(p, g, f, nrhs, s, 0, n, shard_g, shard_r, &sc);
    else if (use_mr(p, nrhs))
        st = p->prec == BF_PREC_MIXED_SFU ? run_forward_mr<bfk::PMIXF>(p, g, f, nrhs, s, 0, n, shard_g, shard_r, &sc)
                                          : run_forward_mr<bfk::PMIX>(p, g, f, nrhs, s, 0, n, shard_g, shard_r, &sc);
    else
        st = p->prec == BF_PREC_MIXED_SFU ? run_forward<bfk::PMIXF>(p, g, f, nrhs, s, 0, n, shard_g, shard_r, &sc)
                                          : run_forward<bfk::PMIX>(p, g, f, nrhs, s, 0, n, shard_g, shard_r, &sc);
    stream_mark(p, s, capturing);
    return st;
}

bf_status bf_plan_autotune(bf_plan p, int nrhs, int reps, void *stream, double *best_ms)
{
    if (!p || nrhs < 1 || nrhs > p->max_nrhs || reps < 1 || reps > 1000) return BF_ERR_INVALID_ARG;
    if (p->points) return BF_ERR_UNSUPPORTED;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t bytes = (size_t)nrhs * (size_t)p->npts * p->csize;
    void *g = nullptr, *f = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaMalloc(&g, bytes);
    if (e == cudaSuccess) e = cudaMalloc(&f, bytes);
    if (e == cudaSuccess) e = cudaMemsetAsync(g, 0, bytes, s);   // the run time does not depend on the values
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    bf_status st = e == cudaSuccess ? BF_OK : cuda_fail(p, e);
    // one candidate: warm-up apply, then reps applies between events
    auto time_it = [&](double &ms) -> bf_status {
        bf_status r = bf_apply(p, g, f, nrhs, stream);
        if (r != BF_OK) return r;
        cudaEventRecord(e0, s);
        for (int i = 0; i < reps && r == BF_OK; ++i) r = bf_apply(p, g, f, nrhs, stream);
        cudaEventRecord(e1, s);
        if (r != BF_OK) return r;
        cudaError_t ce = cudaEventSynchronize(e1);
        if (ce != cudaSuccess) return cuda_fail(p, ce);
        float t = 0.f;
        cudaEventElapsedTime(&t, e0, e1);
        ms = (double)t / reps;
        return BF_OK;
    };
    double best = 1e300;
    if (st == BF_OK && (p->ptab || p->ftab)) {
        st = time_it(best);          // the phase table fixes the schedule
    } else if (st == BF_OK && use_mr(p, nrhs)) {
        // multi-RHS tiles: fused levels, pairs per CTA, right-hand sides per scratch chunk
        const int nr = nrhs < p->fns->mr_max ? nrhs : p->fns->mr_max;
        const int64_t ppr = p->fns->mr_nthreads / p->r;
        std::vector<Pass> keep = p->passes_mr;
        int keep_rc = p->mr_rc;
        if (!keep.empty()) st = time_it(best);   // the incumbent: replaced only by a candidate 1% faster
        const int rcs[6] = {1, 2, 4, 5, 8, 16};
        for (int k = 1; k <= 2 && st == BF_OK; ++k)
            for (int64_t np = ppr; np <= 2 * ppr && st == BF_OK; np *= 2)
                for (int rem = 0; rem < 2 && st == BF_OK; ++rem)
                    for (int ri = 0; ri < 6 && st == BF_OK; ++ri) {
                        const int rc = rcs[ri];
                        if (rc > nr) continue;
                        std::vector<Pass> cand = schedule(p, k, np, rem != 0);
                        tc_switch_split(p, cand);
                        bool fits = true;
                        for (const Pass &ps : cand)
                            if (ps.row < 2 && mr_smem(p, ps, nr, rc) > 227 * 1024) fits = false;
                        if (!fits) continue;
                        p->passes_mr = cand;
                        p->mr_rc = rc;
                        double ms = 0.0;
                        st = time_it(ms);
                        if (st == BF_OK && ms < 0.99 * best) {
                            best = ms;
                            keep = cand;
                            keep_rc = rc;
                        }
                    }
        p->passes_mr = keep;
        p->mr_rc = keep_rc;
    } else if (st == BF_OK) {
        // single-RHS tiles: fused levels per pass and where the short pass goes; the current
        // schedule is kept unless a candidate is 1% faster (no flipping between equal schedules)
        std::vector<Pass> keep = p->passes;
        int keep_k = p->kc;
        st = time_it(best);
        for (int k = 1; k <= p->fns->kmax && st == BF_OK; ++k)
            for (int rem = 0; rem < 2 && st == BF_OK; ++rem) {
                std::vector<Pass> cand = schedule(p, k, p->fns->np, rem != 0);
                bool fits = true;
                for (const Pass &ps : cand)
                    if (pass_smem(p, ps) + row_cache_smem(p, ps) > 227 * 1024) fits = false;
                if (!fits) continue;
                p->passes = cand;
                double ms = 0.0;
                st = time_it(ms);
                if (st == BF_OK && ms < 0.99 * best) {
                    best = ms;
                    keep = cand;
                    keep_k = k;
                }
            }
        p->passes = keep;
        p->kc = p->kr = keep_k;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (g) cudaFree(g);
    if (f) cudaFree(f);
    if (st == BF_OK && best_ms) *best_ms = best;
    return st;
}

bf_status bf_pass_count(bf_plan p, int nrhs, int *count)
{
    if (!p || !count || nrhs < 1 || nrhs > p->max_nrhs) return BF_ERR_INVALID_ARG;
    *count = p->points ? (int)p->passes_pts.size() + 2 : (int)schedule_for(p, nrhs).size();
    return BF_OK;
}

bf_status bf_apply_pass(bf_plan p, int i, const void *g, void *f, int nrhs, void *stream)
{
    if (!p) return BF_ERR_INVALID_ARG;
    if (nrhs < 0 || nrhs > p->max_nrhs) return BF_ERR_INVALID_ARG;
    if (nrhs == 0) return BF_OK;
    if (p->points) return BF_ERR_UNSUPPORTED;
    if (i < 0 || i >= (int)schedule_for(p, nrhs).size()) return BF_ERR_INVALID_ARG;
    if (!g || !f) return BF_ERR_INVALID_ARG;
    if (((uintptr_t)g & 15) || ((uintptr_t)f & 15)) return BF_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    bool capturing = false;
    bf_status st = stream_guard(p, s, &capturing);
    if (st != BF_OK) return st;
    if (p->prec == BF_PREC_FP64) st = run_forward<bfk::PF64>(p, g, f, nrhs, s, i, i + 1);
    else if (use_mr(p, nrhs))
        st = p->prec == BF_PREC_MIXED_SFU ? run_forward_mr<bfk::PMIXF>(p, g, f, nrhs, s, i, i + 1)
                                          : run_forward_mr<bfk::PMIX>(p, g, f, nrhs, s, i, i + 1);
    else
        st = p->prec == BF_PREC_MIXED_SFU ? run_forward<bfk::PMIXF>(p, g, f, nrhs, s, i, i + 1)
                                          : run_forward<bfk::PMIX>(p, g, f, nrhs, s, i, i + 1);
    stream_mark(p, s, capturing);
    return st;
}

bf_status bf_pass_info(bf_plan p, int nrhs, int i, int *kind, int *l0, int *k, int *flags)
{
    if (!p || nrhs < 1 || nrhs > p->max_nrhs) return BF_ERR_INVALID_ARG;
    if (p->points) return BF_ERR_UNSUPPORTED;
    const std::vector<Pass> &sc = schedule_for(p, nrhs);
    if (i < 0 || i >= (int)sc.size()) return BF_ERR_INVALID_ARG;
    const Pass &ps = sc[i];
    if (kind) *kind = ps.row;
    if (l0) *l0 = ps.l0;
    if (k) *k = ps.k;
    if (flags) *flags = ps.flags;
    return BF_OK;
}

bf_status bf_apply_adjoint(bf_plan p, const void *f, void *g, int nrhs, void *stream)
{
    if (!p) return BF_ERR_INVALID_ARG;
    if (p->points) return BF_ERR_UNSUPPORTED;
    if (nrhs < 0 || nrhs > p->max_nrhs) return BF_ERR_INVALID_ARG;
    if (nrhs == 0) return BF_OK;
    if (!g || !f) return BF_ERR_INVALID_ARG;
    if (((uintptr_t)g & 15) || ((uintptr_t)f & 15)) return BF_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    bool capturing = false;
    bf_status st = stream_guard(p, s, &capturing);
    if (st != BF_OK) return st;
    if (p->prec == BF_PREC_FP64) st = run_adjoint<bfk::PF64>(p, f, g, nrhs, s);
    else if (p->prec == BF_PREC_MIXED_SFU) st = run_adjoint<bfk::PMIXF>(p, f, g, nrhs, s);
    else st = run_adjoint<bfk::PMIX>(p, f, g, nrhs, s);
    stream_mark(p, s, capturing);
    return st;
}

bf_status bf_apply_host(bf_plan p, const void *g_host, void *f_host, int nrhs, void *stream)
{
    if (!p) return BF_ERR_INVALID_ARG;
    if (nrhs < 0 || nrhs > p->max_nrhs) return BF_ERR_INVALID_ARG;
    if (nrhs == 0) return BF_OK;
    if (!g_host || !f_host) return BF_ERR_INVALID_ARG;
    const int64_t ng = p->points ? p->nsrc : p->npts, nf = p->points ? p->ntgt : p->npts;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    bool capturing = false;
    bf_status st = stream_guard(p, s, &capturing);   // before the staging copy into the workspace
    if (st != BF_OK) return st;
    cudaError_t e;
    if (!p->gstage) {   // 16 bytes at least, so that empty point sets still get valid pointers
        if ((e = cudaMalloc(&p->gstage, (size_t)p->max_nrhs * ng * p->csize + 16)) != cudaSuccess) return cuda_fail(p, e);
        if ((e = cudaMalloc(&p->fstage, (size_t)p->max_nrhs * nf * p->csize + 16)) != cudaSuccess) return cuda_fail(p, e);
    }
    const size_t bg = (size_t)nrhs * ng * p->csize, bfo = (size_t)nrhs * nf * p->csize;
    if (bg && (e = cudaMemcpyAsync(p->gstage, g_host, bg, cudaMemcpyHostToDevice, s)) != cudaSuccess) return cuda_fail(p, e);
    st = bf_apply(p, p->gstage, p->fstage, nrhs, stream);
    if (st != BF_OK) return st;
    if (bfo && (e = cudaMemcpyAsync(f_host, p->fstage, bfo, cudaMemcpyDeviceToHost, s)) != cudaSuccess) return cuda_fail(p, e);
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(p, e);
    return BF_OK;
}

bf_status bf_apply_batched(const bf_plan *plans, const void *const *g, void *const *f, const int *nrhs, int count,
                           void *stream)
{
    if (count < 0) return BF_ERR_INVALID_ARG;
    if (count == 0) return BF_OK;
    if (!plans || !g || !f || !nrhs) return BF_ERR_INVALID_ARG;
    for (int i = 0; i < count; ++i)
        if (!plans[i] || nrhs[i] < 0 || nrhs[i] > plans[i]->max_nrhs) return BF_ERR_INVALID_ARG;
    for (int i = 0; i < count; ++i) {
        bf_status st = bf_apply(plans[i], g[i], f[i], nrhs[i], stream);
        if (st != BF_OK) return st;
    }
    return BF_OK;
}

bf_status bf_batch_create(const bf_plan *plans, const int *nrhs, int count, bf_batch *out)
{
    if (!out) return BF_ERR_INVALID_ARG;
    *out = nullptr;
    if (!plans || !nrhs || count < 1 || count > bfk::BATCH_MAX) return BF_ERR_INVALID_ARG;
    for (int i = 0; i < count; ++i)
        if (!plans[i] || nrhs[i] < 1 || nrhs[i] > plans[i]->max_nrhs) return BF_ERR_INVALID_ARG;
    const bf_plan p0 = plans[0];
    for (int i = 0; i < count; ++i) {
        const bf_plan p = plans[i];
        if (p->d != 2 || p->prec == BF_PREC_FP64 || tc_prec(p->prec) || p->passes_mr.empty() ||
            !p->fns->batch || p->points)
            return BF_ERR_UNSUPPORTED;
        if (p->q != p0->q || p->kind != p0->kind || p->prec != p0->prec || p->node_kind != p0->node_kind)
            return BF_ERR_UNSUPPORTED;
        for (int j = 0; j < i; ++j)
            if (plans[j] == p) return BF_ERR_INVALID_ARG;   // one workspace per problem
    }
    bf_batch b = new (std::nothrow) bf_batch_s();
    if (!b) return BF_ERR_NOMEM;
    b->count = count;
    b->prec = p0->prec;
    b->fns = p0->fns;
    bf_status st = b->prec == BF_PREC_MIXED_SFU ? batch_build<bfk::PMIXF>(b, plans, nrhs, count)
                                                : batch_build<bfk::PMIX>(b, plans, nrhs, count);
    if (st != BF_OK) {
        bf_batch_destroy(b);
        return st;
    }
    *out = b;
    return BF_OK;
}

bf_status bf_batch_apply(bf_batch b, const void *const *g_dev, void *const *f_dev, void *stream)
{
    return batch_apply(b, g_dev, f_dev, stream, 4000000000ull, 0);
}

bf_status bf_batch_status(bf_batch b, int *timed_out)
{
    if (!b || !timed_out) return BF_ERR_INVALID_ARG;
    int v = 0;
    cudaError_t e = cudaMemcpy(&v, b->ctr + b->njobs + 1, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
        b->last_cuda = (int)e;
        return BF_ERR_CUDA;
    }
    *timed_out = v != 0;
    return BF_OK;
}

bf_status bf_batch_selftest_timeout(bf_batch b, const void *const *g_dev, void *const *f_dev, void *stream,
                                    int *timed_out)
{
    if (!timed_out) return BF_ERR_INVALID_ARG;
    bf_status st = batch_apply(b, g_dev, f_dev, stream, 20000000ull, 1);
    if (st != BF_OK) return st;
    cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) {
        b->last_cuda = (int)e;
        return BF_ERR_CUDA;
    }
    return bf_batch_status(b, timed_out);
}

bf_status bf_batch_info(bf_batch b, int *jobs, int *units, int *grid, int64_t *smem_bytes)
{
    if (!b) return BF_ERR_INVALID_ARG;
    if (jobs) *jobs = b->njobs;
    if (units) *units = b->units;
    if (grid) *grid = (int)b->grid;
    if (smem_bytes) *smem_bytes = (int64_t)b->smem;
    return BF_OK;
}

bf_status bf_batch_wait_stats(bf_batch b, double *wait_ms_total, int64_t *waits)
{
    if (!b) return BF_ERR_INVALID_ARG;
    unsigned long long v[2] = {0, 0};
    cudaError_t e = cudaMemcpy(v, b->state, sizeof(v), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
        b->last_cuda = (int)e;
        return BF_ERR_CUDA;
    }
    if (wait_ms_total) *wait_ms_total = (double)v[0] * 1e-6;
    if (waits) *waits = (int64_t)v[1];
    return BF_OK;
}

bf_status bf_batch_destroy(bf_batch b)
{
    if (!b) return BF_OK;
    if (b->desc) cudaFree(b->desc);
    if (b->jobs) cudaFree(b->jobs);
    if (b->state) cudaFree(b->state);
    delete b;
    return BF_OK;
}

bf_status bf_destroy(bf_plan p)
{
    if (!p) return BF_OK;
    for (int k = 0; k < 3; ++k) {
        if (p->tt[k]) cudaFree(p->tt[k]);
        if (p->st[k]) cudaFree(p->st[k]);
    }
    if (p->w0) cudaFree(p->w0);
    if (p->w1) cudaFree(p->w1);
    if (p->ctab) cudaFree(p->ctab);
    if (p->ptab) cudaFree(p->ptab);
    if (p->ftab) cudaFree(p->ftab);
    if (p->errflag) cudaFree(p->errflag);
    if (p->tmaps) cudaFree(p->tmaps);
    if (p->busy_ev) cudaEventDestroy(p->busy_ev);
    for (void *m : p->pts_mem) cudaFree(m);
    if (p->gstage) cudaFree(p->gstage);
    if (p->fstage) cudaFree(p->fstage);
    delete p;
    return BF_OK;
}

bf_status bf_selfcheck_sincos(int n, double *max_abs_err)
{
    if (n < 1 || !max_abs_err) return BF_ERR_INVALID_ARG;
    cudaError_t e = bfl::selfcheck_sincos(n, max_abs_err);
    return e == cudaSuccess ? BF_OK : BF_ERR_CUDA;
}

bf_status bf_selfcheck_umma(int split, double *max_rel_err, int *timed_out)
{
    if ((split != 0 && split != 1) || !max_rel_err || !timed_out) return BF_ERR_INVALID_ARG;
    return bfl::selfcheck_umma(0, split, max_rel_err, timed_out) == cudaSuccess ? BF_OK : BF_ERR_CUDA;
}

bf_status bf_selfcheck_umma_tf32(int split, double *max_rel_err, int *timed_out)
{
    if ((split != 0 && split != 1) || !max_rel_err || !timed_out) return BF_ERR_INVALID_ARG;
    return bfl::selfcheck_umma(1, split, max_rel_err, timed_out) == cudaSuccess ? BF_OK : BF_ERR_CUDA;
}

bf_status bf_measure_fma_rate(int fp64, double *tflops)
{
    if (!tflops || fp64 < 0 || fp64 > 2) return BF_ERR_INVALID_ARG;
    return bfl::measure_fma(fp64, tflops) == cudaSuccess ? BF_OK : BF_ERR_CUDA;
}

bf_status bf_selfcheck_phase(bf_plan p, int n, double *max_err_cycles)
{
    if (!p || n < 1 || !max_err_cycles || p->prec == BF_PREC_FP64) return BF_ERR_INVALID_ARG;
    bfk::KArgs<bfk::PMIX> am;
    bfk::KArgs<bfk::PF64> ad;
    fill_args<bfk::PMIX>(p, am);
    fill_args<bfk::PF64>(p, ad);
    cudaError_t e = bfl::selfcheck_phase(&am, &ad, p->d, p->L, p->q, p->kind, n, max_err_cycles);
    if (e != cudaSuccess) return cuda_fail(p, e);
    return BF_OK;
}

bf_status bf_measure_phase_rate(bf_plan p, int paired, double *gphases_per_s)
{
    if (!p || !gphases_per_s || p->prec == BF_PREC_FP64 || p->d != 2 || (paired != 0 && paired != 1))
        return BF_ERR_INVALID_ARG;
    bfk::KArgs<bfk::PMIX> am;
    fill_args<bfk::PMIX>(p, am);
    cudaError_t e = bfl::phase_rate(&am, p->prec == BF_PREC_MIXED_SFU, p->L, p->q, p->kind, paired, gphases_per_s);
    if (e != cudaSuccess) return cuda_fail(p, e);
    return BF_OK;
}

bf_status bf_plan_tc_info(bf_plan p, int *tiled_copies)
{
    if (!p || !tiled_copies) return BF_ERR_INVALID_ARG;
    *tiled_copies = p->tmaps ? 1 : 0;
    return BF_OK;
}

bf_status bf_plan_table_info(bf_plan p, int64_t *bytes, double *build_ms, int *timed_out)
{
    if (!p) return BF_ERR_INVALID_ARG;
    if (bytes) *bytes = p->ptab_bytes;
    if (build_ms) *build_ms = p->ptab_build_ms;
    if (timed_out) {
        int v = 0;
        if (p->errflag) {
            cudaError_t e = cudaMemcpy(&v, p->errflag, sizeof(int), cudaMemcpyDeviceToHost);
            if (e != cudaSuccess) return cuda_fail(p, e);
        }
        *timed_out = v != 0;
    }
    return BF_OK;
}

bf_status bf_last_cuda_error(bf_plan p, int *cuda_err)
{
    if (!p || !cuda_err) return BF_ERR_INVALID_ARG;
    *cuda_err = p->last_cuda;
    return BF_OK;
}

bf_status bf_plan_info(bf_plan p, int *d, int64_t *N, int *q, int *m, int *fuse_levels, int *launches,
                       int64_t *ws_bytes)
{
    if (!p) return BF_ERR_INVALID_ARG;
    if (d) *d = p->d;
    if (N) *N = p->N;
    if (q) *q = p->q;
    if (m) *m = p->m;
    if (fuse_levels) *fuse_levels = p->kc;
    if (launches) *launches = (int)p->passes.size();
    if (ws_bytes) *ws_bytes = p->ws_bytes;
    return BF_OK;
}

}  // extern "C"
