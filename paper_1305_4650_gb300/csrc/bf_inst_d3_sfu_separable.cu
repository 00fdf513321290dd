// Kernels for d = 3, precision PMIXF (mixed, SFU sincos), phase kind separable (q in {2,3,4}).
#include "bf_inst.cuh"

namespace bfl {

const PassFns *fns_d3_sfu_separable(int q)
{
    switch (q) {
    case 2: return fns_for<3, 2, bfk::PMIXF, bfk::KIND_SEPARABLE>();
    case 3: return fns_for<3, 3, bfk::PMIXF, bfk::KIND_SEPARABLE>();
    case 4: return fns_for<3, 4, bfk::PMIXF, bfk::KIND_SEPARABLE>();
    default: return nullptr;
    }
}

}  // namespace bfl
