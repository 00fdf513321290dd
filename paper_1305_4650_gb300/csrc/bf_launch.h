// Launch table shared between the host plan code and the kernel instantiation units.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

namespace bfl {

// kargs points to a bfk::KArgs<P> of the table's precision
typedef cudaError_t (*pass_fn)(const void *kargs, unsigned grid_x, unsigned grid_y, size_t smem, cudaStream_t s);

struct PassFns {
    pass_fn col, row;            // forward: init/column/switch pass, row/final pass
    pass_fn col_adj, row_adj;    // adjoint passes (null until compiled)
    int kmax;                    // most levels one pass fuses
    int np;                      // pairs per CTA (2^{d kmax})
    int nthreads;                // threads per CTA
};

// (d, q, precision) -> kernels, or null if that combination is not compiled.
// precision: 0 FP64, 1 mixed
const PassFns *get_fns(int d, int q, int prec);

const PassFns *fns_d2_f64(int q);
const PassFns *fns_d2_mix(int q);
const PassFns *fns_d3_f64(int q);
const PassFns *fns_d3_mix(int q);


}  // namespace bfl
