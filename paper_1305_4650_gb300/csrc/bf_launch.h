// Launch table shared between the host plan code and the kernel instantiation units.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

namespace bfl {

// kargs points to a bfk::KArgs<P> of the table's precision
typedef cudaError_t (*pass_fn)(const void *kargs, unsigned grid_x, unsigned grid_y, size_t smem, cudaStream_t s);

struct PassFns {
    pass_fn col, row;            // forward: init/column/switch pass, row/final pass
    pass_fn col_adj, row_adj;    // adjoint passes: transposes of col and row, levels reversed
    int kmax;                    // most levels one pass fuses
    int np;                      // pairs per CTA (2^{d kmax})
    int nthreads;                // threads per CTA
    // multi-RHS forward passes with a phase cache (null if absent), per phase mode:
    // [0] evaluate, [1] build the plan's phase table, [2] read the phase table
    pass_fn col_mr[3], row_mr[3];
    int mr_max;                  // right-hand sides one multi-RHS CTA holds
    int mr_nthreads;             // threads per multi-RHS CTA
    // persistent batch kernel (bf_mr.cuh): bargs points to a bfk::BatchArgs<P>
    cudaError_t (*batch)(const void *bargs, unsigned grid, size_t smem, cudaStream_t s);
    int (*batch_ctas_per_sm)(size_t smem);
    int (*mr_table_occupancy)(int row, size_t smem);   // CTAs per SM of the table-reading passes
    cudaError_t (*center_table)(const void *kargs, void *out, int levels);   // target features at box centres
    int tsize;                   // bytes of one target-feature record
    // single-RHS passes with a reduced-phase table (mixed; d = 2 with q <= 5, d = 3; null if absent):
    // [0] record the table (plan creation), [1] read it
    pass_fn col_tab[2], row_tab[2];
    // multi-RHS switch on the tensor cores (bf_tc.cuh; d = 2, q <= 5, BF16x3 products;
    // null if absent): grid_x CTAs take units of two pairs, grid_y blocks of 16 right-hand sides
    pass_fn switch_tc;
    int (*switch_tc_ctas_per_sm)();   // CTAs of switch_tc that fit on one SM
    size_t switch_tc_smem;            // its dynamic shared memory per CTA
    // one column merge level on the tensor cores (bf_tc.cuh, same conditions; null if absent):
    // grid_x CTAs take merge blocks, grid_y blocks of 16 right-hand sides
    pass_fn col_tc;
    int (*col_tc_ctas_per_sm)();
    size_t col_tc_smem;
    // the multi-RHS switch on the tensor cores with TF32x3 products (BF_PREC_TF32X3; same
    // conditions and grid as switch_tc)
    pass_fn switch_tc32 = nullptr;
    int (*switch_tc32_ctas_per_sm)() = nullptr;
    size_t switch_tc32_smem = 0;
};

// (d, q, precision, phase kind) -> kernels, or null if that combination is not compiled.
// precision: 0 FP64, 1 mixed, 2 mixed with SFU sincos; kind: bf_phase_kind
const PassFns *get_fns(int d, int q, int prec, int kind);

// one function per instantiation unit: bf_inst_d{d}_{f64|mix}_{kind}.cu
#define BFL_DECLARE(d, pr, kn) const PassFns *fns_d##d##_##pr##_##kn(int q);
BFL_DECLARE(2, f64, dot) BFL_DECLARE(2, f64, genradon) BFL_DECLARE(2, f64, hypradon) BFL_DECLARE(2, f64, separable)
BFL_DECLARE(2, mix, dot) BFL_DECLARE(2, mix, genradon) BFL_DECLARE(2, mix, hypradon) BFL_DECLARE(2, mix, separable)
BFL_DECLARE(3, f64, dot) BFL_DECLARE(3, f64, genradon) BFL_DECLARE(3, f64, separable)
BFL_DECLARE(3, mix, dot) BFL_DECLARE(3, mix, genradon) BFL_DECLARE(3, mix, separable)
BFL_DECLARE(2, sfu, dot) BFL_DECLARE(2, sfu, genradon) BFL_DECLARE(2, sfu, hypradon) BFL_DECLARE(2, sfu, separable)
BFL_DECLARE(3, sfu, dot) BFL_DECLARE(3, sfu, genradon) BFL_DECLARE(3, sfu, separable)
#undef BFL_DECLARE


// arbitrary point sets (bf_points.cu)
struct PointsGeom {
    int d, L, q, kind;
    double s;
    double x_lo[3], x_w[3], y_lo[3], y_w[3];
    double z[8];                  // Chebyshev nodes on [-1/2, 1/2]
};
struct PointsData {
    int d, q;
    int64_t nbox, nsrc, ntgt, wstride;
    const int64_t *src_off;       // [nbox + 1] sources of leaf box B: sorted positions src_off[B] .. src_off[B+1]-1
    const int64_t *src_perm;      // [nsrc] caller's index of each sorted source
    const void *src_lag;          // [nsrc][d][q] Lagrange values in the leaf box (R)
    const void *src_e;            // [nsrc] e^{2 pi i Phi(x0(X), y)} (C)
    const int64_t *tgt_box;       // [ntgt] leaf box of each target (caller's order)
    const void *tgt_lag;          // [ntgt][d][q] (R)
    const void *tgt_e;            // [ntgt] e^{2 pi i Phi(x, y0(Y))} (C)
    const void *node_init;        // [nbox][r] conj(e^{2 pi i Phi(x0(X), y_t^B)}) (C)
    const void *node_final;       // [nbox][r] conj(e^{2 pi i Phi(x_t^A, y0(Y))}) (C)
};
cudaError_t points_nodes(const PointsGeom &geo, int fp64, void *node_init, void *node_final);
cudaError_t points_init(const PointsData &pd, int fp64, int r, const void *g, void *w0, int nrhs, cudaStream_t s);
cudaError_t points_final(const PointsData &pd, int fp64, int r, const void *wl, void *f, int nrhs, cudaStream_t s);

// device self-checks and the FMA rate probe (bf_selfcheck.cu)
cudaError_t measure_fma(int fp64, double *tflops);
cudaError_t selfcheck_sincos(int n, double *max_err);
cudaError_t phase_rate(const void *kargs_mix, int sfu, int L, int q, int kind, int paired, double *gphases);
cudaError_t selfcheck_phase(const void *kargs_mix, const void *kargs_f64, int d, int L, int q, int kind, int n,
                            double *max_err);
cudaError_t selfcheck_umma(int fmt, int split, double *max_rel_err, int *timed_out);   // fmt 0 BF16, 1 TF32

}  // namespace bfl
