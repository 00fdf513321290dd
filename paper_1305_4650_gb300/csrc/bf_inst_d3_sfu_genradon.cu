// Kernels for d = 3, precision PMIXF (mixed, SFU sincos), phase kind genradon (q in {2,3,4}).
#include "bf_inst.cuh"

namespace bfl {

const PassFns *fns_d3_sfu_genradon(int q)
{
    switch (q) {
    case 2: return fns_for<3, 2, bfk::PMIXF, bfk::KIND_GENRADON>();
    case 3: return fns_for<3, 3, bfk::PMIXF, bfk::KIND_GENRADON>();
    case 4: return fns_for<3, 4, bfk::PMIXF, bfk::KIND_GENRADON>();
    default: return nullptr;
    }
}

}  // namespace bfl
