// Arbitrary source and target point sets (Section 1.4: the field of a pair is an
// interpolant that can be evaluated anywhere in the target box; only the first and
// the last step of Algorithm 1 see the points).
//
//   init   delta_t^{XB} = conj(e^{2pi i Phi(x0(X), y_t^B)}) sum_{y in B} L_t^B(y) e^{2pi i Phi(x0(X), y)} g(y)
//   final  f(x) = e^{2pi i Phi(x, y0(Y))} sum_t L_t^A(x) conj(e^{2pi i Phi(x_t^A, y0(Y))}) w_{A,Y}(t)
//
// The per-point factors (Lagrange values of the point in its leaf box, one phase
// factor) are computed on the host in FP64 when the plan is made; the node factors of
// every leaf box by k_points_nodes below (FP64, once per plan).  The merges in between
// are the tile kernels of the uniform-grid path.
#include <cuda_runtime.h>
#include <stdint.h>

#include "bf_launch.h"

namespace {

// Phi in FP64 (cycles) for the phase kinds of bf.h, from coordinates
__device__ double phi64(int kind, int d, double s, const double *x, const double *y)
{
    const double twopi = 6.283185307179586476925286766559;
    switch (kind) {
    case 0: {   // Fourier
        double v = 0.0;
        for (int k = 0; k < d; ++k) v += x[k] * y[k];
        return s * v;
    }
    case 1: {   // generalized Radon analogue
        double xy = 0.0, q2 = 0.0;
        for (int k = 0; k < d; ++k) xy += x[k] * y[k];
        if (d == 2) {
            const double a0 = (2.0 + sin(twopi * x[0]) * sin(twopi * x[1])) / 3.0;
            const double a1 = (2.0 + cos(twopi * x[0]) * cos(twopi * x[1])) / 3.0;
            q2 = a0 * a0 * y[0] * y[0] + a1 * a1 * y[1] * y[1];
        } else {
            for (int k = 0; k < d; ++k) {
                const double a = (2.0 + sin(twopi * x[k]) * cos(twopi * x[(k + 1) % d])) / 3.0;
                q2 += a * a * y[k] * y[k];
            }
        }
        return s * (xy + sqrt(q2));
    }
    case 2:     // hyperbolic Radon
        return s * x[0] * sqrt(y[0] * y[0] + y[1] * y[1] * x[1] * x[1]);
    default: {  // separable test phase
        double v = 0.0;
        for (int k = 0; k < d; ++k) v += sin(twopi * (x[k] + (k + 1) / 7.0)) + y[k] * y[k] / (k + 2.0);
        return s * v;
    }
    }
}

template <class C> __device__ __forceinline__ C mkc(double re, double im);
template <> __device__ __forceinline__ float2 mkc<float2>(double re, double im) { return make_float2((float)re, (float)im); }
template <> __device__ __forceinline__ double2 mkc<double2>(double re, double im) { return make_double2(re, im); }

// conj(e^{2 pi i Phi}) of every (leaf box, node): init nodes y_t^B against x0(X) (src = 1),
// final nodes x_t^A against y0(Y) (src = 0).  Boxes in Morton order, node t = sum t_k q^k.
template <class C>
__global__ void k_points_nodes(bfl::PointsGeom geo, int src, C *out)
{
    const int d = geo.d, q = geo.q;
    int r = 1;
    for (int k = 0; k < d; ++k) r *= q;
    const int64_t N = 1LL << geo.L, total = ((int64_t)1 << (d * geo.L)) * r;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t box = e / r;
        int t = (int)(e % r);
        double node[3], other[3];
        for (int k = 0; k < d; ++k) {
            int64_t c = 0;
            for (int j = 0; j < geo.L; ++j) c |= ((box >> (j * d + k)) & 1) << j;
            const int tk = t % q;
            t /= q;
            const double lo = src ? geo.y_lo[k] : geo.x_lo[k], w = (src ? geo.y_w[k] : geo.x_w[k]) / (double)N;
            node[k] = lo + (c + 0.5) * w + w * geo.z[tk];
            other[k] = src ? geo.x_lo[k] + 0.5 * geo.x_w[k] : geo.y_lo[k] + 0.5 * geo.y_w[k];
        }
        const double th = src ? phi64(geo.kind, d, geo.s, other, node) : phi64(geo.kind, d, geo.s, node, other);
        const double f = th - rint(th);
        double sn, cs;
        sincospi(2.0 * f, &sn, &cs);
        out[e] = mkc<C>(cs, -sn);
    }
}

template <class C> __device__ __forceinline__ C cmul_(C a, C b);
template <> __device__ __forceinline__ float2 cmul_(float2 a, float2 b)
{
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <> __device__ __forceinline__ double2 cmul_(double2 a, double2 b)
{
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// level-0 weights: one thread per (leaf box, node), blockIdx.y = right-hand side
template <class C, class R>
__global__ void k_points_init(bfl::PointsData pd, int r, const C *g, C *w0)
{
    const int q = pd.q, d = pd.d;
    const int64_t total = pd.nbox * r, rhs = blockIdx.y;
    const C *node = static_cast<const C *>(pd.node_init);
    const C *pe = static_cast<const C *>(pd.src_e);
    const R *lag = static_cast<const R *>(pd.src_lag);
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t B = e / r;
        const int t = (int)(e % r);
        int tk[3] = {0, 0, 0};
        for (int k = 0, tt = t; k < d; ++k, tt /= q) tk[k] = tt % q;
        C acc;
        acc.x = 0;
        acc.y = 0;
        for (int64_t j = pd.src_off[B]; j < pd.src_off[B + 1]; ++j) {
            R l = lag[(j * d) * q + tk[0]];
            for (int k = 1; k < d; ++k) l *= lag[(j * d + k) * q + tk[k]];
            const C v = cmul_(pe[j], g[rhs * pd.nsrc + pd.src_perm[j]]);
            acc.x += l * v.x;
            acc.y += l * v.y;
        }
        w0[rhs * pd.wstride + e] = cmul_(node[e], acc);
    }
}

// targets: one thread per target, blockIdx.y = right-hand side; wl = level-L weights [A][t]
template <class C, class R>
__global__ void k_points_final(bfl::PointsData pd, int r, const C *wl, C *f)
{
    const int q = pd.q, d = pd.d;
    const int64_t rhs = blockIdx.y;
    const C *node = static_cast<const C *>(pd.node_final);
    const C *pe = static_cast<const C *>(pd.tgt_e);
    const R *lag = static_cast<const R *>(pd.tgt_lag);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < pd.ntgt; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t A = pd.tgt_box[i];
        const C *w = wl + rhs * pd.wstride + A * r;
        const C *nd = node + A * r;
        C acc;
        acc.x = 0;
        acc.y = 0;
        for (int t = 0; t < r; ++t) {
            R l = 1;
            for (int k = 0, tt = t; k < d; ++k, tt /= q) l *= lag[(i * d + k) * q + tt % q];
            const C v = cmul_(nd[t], w[t]);
            acc.x += l * v.x;
            acc.y += l * v.y;
        }
        f[rhs * pd.ntgt + i] = cmul_(pe[i], acc);
    }
}

int grid_for(int64_t n)
{
    const int64_t b = (n + 255) / 256;
    return (int)(b < 65536 ? (b > 0 ? b : 1) : 65536);
}

}  // namespace

namespace bfl {

cudaError_t points_nodes(const PointsGeom &geo, int fp64, void *node_init, void *node_final)
{
    const int64_t total = ((int64_t)1 << (geo.d * geo.L)) * [&] { int r = 1; for (int k = 0; k < geo.d; ++k) r *= geo.q; return r; }();
    if (fp64) {
        k_points_nodes<double2><<<grid_for(total), 256>>>(geo, 1, static_cast<double2 *>(node_init));
        k_points_nodes<double2><<<grid_for(total), 256>>>(geo, 0, static_cast<double2 *>(node_final));
    } else {
        k_points_nodes<float2><<<grid_for(total), 256>>>(geo, 1, static_cast<float2 *>(node_init));
        k_points_nodes<float2><<<grid_for(total), 256>>>(geo, 0, static_cast<float2 *>(node_final));
    }
    return cudaGetLastError();
}

cudaError_t points_init(const PointsData &pd, int fp64, int r, const void *g, void *w0, int nrhs, cudaStream_t s)
{
    const dim3 grid(grid_for(pd.nbox * r), nrhs);
    if (fp64)
        k_points_init<double2, double><<<grid, 256, 0, s>>>(pd, r, static_cast<const double2 *>(g), static_cast<double2 *>(w0));
    else
        k_points_init<float2, float><<<grid, 256, 0, s>>>(pd, r, static_cast<const float2 *>(g), static_cast<float2 *>(w0));
    return cudaGetLastError();
}

cudaError_t points_final(const PointsData &pd, int fp64, int r, const void *wl, void *f, int nrhs, cudaStream_t s)
{
    if (pd.ntgt == 0) return cudaSuccess;
    const dim3 grid(grid_for(pd.ntgt), nrhs);
    if (fp64)
        k_points_final<double2, double><<<grid, 256, 0, s>>>(pd, r, static_cast<const double2 *>(wl), static_cast<double2 *>(f));
    else
        k_points_final<float2, float><<<grid, 256, 0, s>>>(pd, r, static_cast<const float2 *>(wl), static_cast<float2 *>(f));
    return cudaGetLastError();
}

}  // namespace bfl
