// bf_apply_noalloc: the forward apply with its geometry tables and weight
// buffers in one static device array instead of memory from cudaMalloc.
//
// For callers that cannot allocate device memory (a host application that
// owns all GPU memory through a fixed pool, or code that must not allocate
// once it is running).  The tables are built on the device by k_noalloc_tables
// from the same formulas the plan builds on the host; the butterfly passes are
// the same kernels bf_apply launches.  No cudaMalloc, cudaFree or other
// allocating routine is called, on the device or the host.
#include <cmath>
#include <cstring>
#include <mutex>

#include "../../include/bf.h"
#include "bf_device.cuh"
#include "bf_launch.h"

// Every GPU that loads the library holds this array until the process exits.
static __device__ __align__(256) unsigned char g_bf_noalloc_scratch[BF_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr double kPi = 3.14159265358979323846264338327950288;
constexpr int kMaxDevices = 64;
constexpr int kMaxPasses = 64;

std::mutex g_setup_mu;
unsigned char *g_scratch_dev[kMaxDevices] = {};

// Device address of the static array on the current device (looked up once per device).
bf_status scratch_address(unsigned char **out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return BF_ERR_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return BF_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lk(g_setup_mu);
    if (!g_scratch_dev[dev]) {
        void *ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_bf_noalloc_scratch) != cudaSuccess || !ptr) return BF_ERR_CUDA;
        g_scratch_dev[dev] = static_cast<unsigned char *>(ptr);
    }
    *out = g_scratch_dev[dev];
    return BF_OK;
}

struct NaPass {
    int row, l0, k, flags, T;
};

struct NaGeom {
    double x_lo, x_w, y_lo, y_w, s, tgt_off, src_off;
    double z[bfk::QMAX];
};

// One thread per (level, box, slot) entry of dimension k's target and source tables,
// with the layout and feature definitions of the plan's host-built tables.
template <class P>
__global__ void k_noalloc_tables(NaGeom g, int kdim, int L, int q, int kind, typename P::TE *tt, typename P::SE *st)
{
    const int64_t nent = ((2LL << L) - 1) * (q + 2);
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nent; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t box_slot = e;
        // target table: level l holds 2^l boxes of (q+2) slots, starting at (2^l - 1)(q+2)
        int l = 0;
        while (((2LL << l) - 1) * (q + 2) <= box_slot) ++l;
        int64_t r0 = box_slot - ((1LL << l) - 1) * (q + 2);
        int64_t i = r0 / (q + 2);
        int j = (int)(r0 % (q + 2));
        double w = g.x_w / (double)(1LL << l);
        double c = g.x_lo + ((double)i + 0.5) * w;
        double x = j < q ? c + w * g.z[j] : (j == q ? c : g.x_lo + ((double)i + g.tgt_off) * w);
        double f0 = 0.0, f1 = 0.0, f2 = 0.0;
        switch (kind) {
        case BF_PHASE_DOT: f0 = g.s * x; break;
        case BF_PHASE_GENRADON: f0 = g.s * x; f1 = sin(2 * kPi * x); f2 = cos(2 * kPi * x); break;
        case BF_PHASE_HYPRADON: f0 = g.s * x; f1 = x * x; break;
        default: f0 = g.s * sin(2 * kPi * (x + (kdim + 1) / 7.0)); break;
        }
        // source table: level l holds 2^(L-l) boxes, starting at (2^(L+1) - 2^(L-l+1))(q+2)
        int ls = 0;
        while (ls < L && ((2LL << L) - (2LL << (L - ls - 1))) * (q + 2) <= box_slot) ++ls;
        int64_t r1 = box_slot - ((2LL << L) - (2LL << (L - ls))) * (q + 2);
        int64_t is = r1 / (q + 2);
        int js = (int)(r1 % (q + 2));
        double ws = g.y_w * (double)(1LL << ls) / (double)(1LL << L);
        double cs = g.y_lo + ((double)is + 0.5) * ws;
        double y = js < q ? cs + ws * g.z[js] : (js == q ? cs : g.y_lo + ((double)is + g.src_off) * ws);
        double s0, s1;
        if (kind == BF_PHASE_SEPARABLE) {
            s0 = g.s * y * y / (kdim + 2.0);
            s1 = 0.0;
        } else {
            s0 = y;
            s1 = y * y;
        }
        if constexpr (P::is_f64) {
            tt[e].a = make_double2(f0, f1);
            tt[e].b = make_double2(f2, 0.0);
            st[e].a = make_double2(s0, s1);
        } else {
            auto sp = [](double v, float &h, float &lo) { h = (float)v; lo = (float)(v - (double)h); };
            float a[6], b[4];
            sp(f0, a[0], a[1]);
            sp(f1, a[2], a[3]);
            sp(f2, a[4], a[5]);
            sp(s0, b[0], b[1]);
            sp(s1, b[2], b[3]);
            tt[e].a = make_float4(a[0], a[1], a[2], a[3]);
            tt[e].b = make_float4(a[4], a[5], 0.f, 0.f);
            st[e].a = make_float4(b[0], b[1], b[2], b[3]);
        }
    }
}

double lagrange1(int q, const double *z, int t, double xi)
{
    double v = 1.0;
    for (int k = 0; k < q; ++k)
        if (k != t) v *= (xi - z[k]) / (z[t] - z[k]);
    return v;
}

template <class P>
bf_status run(int d, int L, int q, int kind, const bf_params *prm, const void *g, void *f, int nrhs,
              cudaStream_t s, unsigned char *base, const bfl::PassFns *fns)
{
    const int r = bfk::ipow(q, d);
    const int64_t npts = 1LL << (L * d);
    const int64_t nent = ((2LL << L) - 1) * (q + 2);
    auto align = [](size_t v) { return (v + 255) & ~(size_t)255; };
    bfk::KArgs<P> a;
    std::memset(&a, 0, sizeof(a));
    size_t off = 0;
    NaGeom geo;
    double z[bfk::QMAX];
    for (int j = 0; j < q; ++j)
        z[j] = prm->node_kind == 0 ? 0.5 * std::cos(j * kPi / (q - 1)) : 0.5 * std::cos((2 * j + 1) * kPi / (2.0 * q));
    for (int k = 0; k < d; ++k) {
        typename P::TE *tt = reinterpret_cast<typename P::TE *>(base + off);
        off = align(off + nent * sizeof(typename P::TE));
        typename P::SE *st = reinterpret_cast<typename P::SE *>(base + off);
        off = align(off + nent * sizeof(typename P::SE));
        geo = NaGeom{prm->x_lo[k], prm->x_w[k], prm->y_lo[k], prm->y_w[k], prm->phase_scale, prm->tgt_off,
                     prm->src_off, {}};
        for (int j = 0; j < q; ++j) geo.z[j] = z[j];
        const int nb = (int)((nent + 255) / 256);
        k_noalloc_tables<P><<<nb < 1024 ? nb : 1024, 256, 0, s>>>(geo, k, L, q, kind, tt, st);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? BF_ERR_NOMEM : BF_ERR_CUDA;
        a.tt[k] = tt;
        a.st[k] = st;
    }
    const size_t wbytes = (size_t)nrhs * (size_t)npts * (size_t)r * sizeof(typename P::C);
    void *w0 = base + off;
    off = align(off + wbytes);
    void *w1 = base + off;
    for (int h = 0; h < 2; ++h)
        for (int t = 0; t < q; ++t)
            for (int u = 0; u < q; ++u) {
                a.M[h][t][u] = (typename P::R)lagrange1(q, z, t, (z[u] + h - 0.5) / 2.0);
                a.M2[h][t][u].x = a.M2[h][t][u].y = a.M[h][t][u];
            }
    for (int t = 0; t < q; ++t) {
        a.lsrc[t] = (typename P::R)lagrange1(q, z, t, prm->src_off - 0.5);
        a.ltgt[t] = (typename P::R)lagrange1(q, z, t, prm->tgt_off - 0.5);
    }
    const double sc = prm->phase_scale;
    const double sgn = sc > 0 ? 1.0 : (sc < 0 ? -1.0 : 0.0);
    if constexpr (P::is_f64) {
        a.sc.s3 = sc / 3.0;
        a.sc.sgn = sgn;
    } else {
        a.sc.s3hi = (float)(sc / 3.0);
        a.sc.s3lo = (float)(sc / 3.0 - (double)a.sc.s3hi);
        a.sc.sgn = (float)sgn;
    }
    a.ctab = nullptr;
    a.ctab_levels = -1;
    a.L = L;
    a.kind = kind;
    a.npts = npts;
    a.wstride = npts * r;
    a.g = static_cast<const typename P::C *>(g);
    a.f = static_cast<typename P::C *>(f);

    // the default schedule of bf_plan_create: column passes of <= kmax levels (init first,
    // switch last), then row passes (final last); in each run of levels the short pass
    // (levels mod kmax) comes first
    const int m = prm->switch_level < 0 ? L / 2 : prm->switch_level;
    const int kmax = prm->fuse_levels > 0 && prm->fuse_levels < fns->kmax ? prm->fuse_levels : fns->kmax;
    NaPass ps[kMaxPasses];
    int np = 0;
    auto add = [&](int row, int l0, int k, int fl) {
        const int64_t cta_pairs = npts < fns->np ? npts : fns->np;
        int T = (int)(cta_pairs >> (d * k));
        ps[np++] = NaPass{row, l0, k, fl, T < 1 ? 1 : T};
    };
    auto chunk = [&](int left, int total) {
        const int rem = total % kmax;
        if (rem && left == total) return rem;
        return left < kmax ? left : kmax;
    };
    if (m == 0) {
        add(0, 0, 0, bfk::F_INIT | bfk::F_SWITCH);
    } else {
        for (int l = 0; l < m;) {
            const int k = chunk(m - l, m);
            add(0, l, k, (l == 0 ? bfk::F_INIT : 0) | (l + k == m ? bfk::F_SWITCH : 0));
            l += k;
        }
    }
    for (int l = m; l < L;) {
        const int k = chunk(L - l, L - m);
        add(1, l, k, l + k == L ? bfk::F_FINAL : 0);
        l += k;
    }
    void *buf[2] = {w0, w1};
    for (int i = 0; i < np; ++i) {
        a.l0 = ps[i].l0;
        a.k = ps[i].k;
        a.flags = ps[i].flags;
        a.T = ps[i].T;
        a.win = static_cast<const typename P::C *>(buf[i & 1]);
        a.wout = static_cast<typename P::C *>(buf[(i + 1) & 1]);
        const int64_t ctas = (npts >> (d * ps[i].k)) / ps[i].T;
        size_t smem = (size_t)3 * ps[i].T * ((size_t)1 << (d * ps[i].k)) * r * sizeof(typename P::C);
        if (ps[i].row && ps[i].k >= 1)   // cache of the parents' node features in the row kernels
            smem += (size_t)ps[i].T * ((size_t)1 << (d * (ps[i].k - 1))) * r * (size_t)fns->tsize;
        if (!ps[i].row)                  // geometry of a level's output pairs in the column kernels
            smem += (size_t)ps[i].T * ((size_t)1 << (d * ps[i].k)) * (((size_t)fns->tsize + 16 + 15) / 16 * 16);
        cudaError_t e = (ps[i].row ? fns->row : fns->col)(&a, (unsigned)ctas, (unsigned)nrhs, smem, s);
        if (e != cudaSuccess) return BF_ERR_CUDA;
    }
    return BF_OK;
}

}  // namespace

extern "C" bf_status bf_apply_noalloc(int d, int64_t N, int q, bf_phase_kind phase, const bf_params *prm,
                                      const void *g, void *f, int nrhs, void *stream)
{
    if (!prm) return BF_ERR_INVALID_ARG;
    if (d < 2 || d > 3) return d == 1 ? BF_ERR_UNSUPPORTED : BF_ERR_INVALID_ARG;
    if (N < 2 || (N & (N - 1))) return BF_ERR_INVALID_ARG;
    int L = 0;
    while ((1LL << L) < N) ++L;
    if ((int64_t)L * d > 30) return BF_ERR_INVALID_ARG;
    if (q < 2 || q > bfk::QMAX) return BF_ERR_INVALID_ARG;
    if ((int)phase < 0 || (int)phase > 3) return BF_ERR_INVALID_ARG;
    if (phase == BF_PHASE_HYPRADON && d != 2) return BF_ERR_INVALID_ARG;
    if (prm->precision < BF_PREC_FP64 || prm->precision > BF_PREC_MIXED_SFU) return BF_ERR_INVALID_ARG;
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
    if (prm->fuse_levels < 0 || prm->fuse_levels > 8) return BF_ERR_INVALID_ARG;
    for (int i = 0; i < 4; ++i)
        if (prm->reserved[i]) return BF_ERR_INVALID_ARG;
    if (prm->tc_levels || prm->tc_cpasync) return BF_ERR_INVALID_ARG;   // BF_PREC_BF16X3 options
    if (prm->phase_tables) return BF_ERR_INVALID_ARG;   // a table would need device memory
    if (nrhs < 0 || nrhs > 65535) return BF_ERR_INVALID_ARG;
    const int prec = prm->precision;
    if (prec != BF_PREC_FP64) {   // |Phi| < 2^21 cycles for the mixed path's integer rounding
        double b = 0.0, mx[3], my[3];
        for (int k = 0; k < d; ++k) {
            mx[k] = std::fmax(std::fabs(prm->x_lo[k]), std::fabs(prm->x_lo[k] + prm->x_w[k]));
            my[k] = std::fmax(std::fabs(prm->y_lo[k]), std::fabs(prm->y_lo[k] + prm->y_w[k]));
        }
        if (phase == BF_PHASE_DOT || phase == BF_PHASE_GENRADON) {
            double q2 = 0.0;
            for (int k = 0; k < d; ++k) { b += mx[k] * my[k]; q2 += my[k] * my[k]; }
            if (phase == BF_PHASE_GENRADON) b += std::sqrt(q2);
        } else if (phase == BF_PHASE_HYPRADON) {
            b = mx[0] * std::sqrt(my[0] * my[0] + my[1] * my[1] * mx[1] * mx[1]);
        } else {
            for (int k = 0; k < d; ++k) b += 1.0 + my[k] * my[k] / (k + 2.0);
        }
        if (std::fabs(prm->phase_scale) * b >= 2097152.0) return BF_ERR_UNSUPPORTED;
    }
    const bfl::PassFns *fns = bfl::get_fns(d, q, prec, (int)phase);
    if (!fns) return BF_ERR_UNSUPPORTED;

    // scratch needed: 2d tables of nent entries (32 B target, 16 B source) + 2 weight buffers
    const int64_t npts = 1LL << (L * d);
    const int64_t nent = ((2LL << L) - 1) * (q + 2);
    const size_t c = prec == 0 ? 16 : 8;
    const size_t need = (size_t)d * (((size_t)nent * 32 + 255) / 256 * 256 + ((size_t)nent * 16 + 255) / 256 * 256) +
                        2 * (((size_t)nrhs * (size_t)npts * (size_t)bfk::ipow(q, d) * c + 255) / 256 * 256);
    if (need > BF_NOALLOC_SCRATCH_BYTES) return BF_ERR_INVALID_ARG;
    if (nrhs == 0) return BF_OK;
    if (!g || !f || ((uintptr_t)g & 15) || ((uintptr_t)f & 15)) return BF_ERR_INVALID_ARG;

    unsigned char *base = nullptr;
    bf_status st = scratch_address(&base);
    if (st != BF_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (prec == 0) return run<bfk::PF64>(d, L, q, (int)phase, prm, g, f, nrhs, s, base, fns);
    if (prec == 2) return run<bfk::PMIXF>(d, L, q, (int)phase, prm, g, f, nrhs, s, base, fns);
    return run<bfk::PMIX>(d, L, q, (int)phase, prm, g, f, nrhs, s, base, fns);
}
