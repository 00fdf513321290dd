// Kernels for d = 2, precision PMIXF (mixed, SFU sincos), phase kind genradon (q in {2,3,4,5,6,8}).
#include "bf_inst.cuh"

namespace bfl {

const PassFns *fns_d2_sfu_genradon(int q)
{
    switch (q) {
    case 2: return fns_for<2, 2, bfk::PMIXF, bfk::KIND_GENRADON>();
    case 3: return fns_for<2, 3, bfk::PMIXF, bfk::KIND_GENRADON>();
    case 4: return fns_for<2, 4, bfk::PMIXF, bfk::KIND_GENRADON>();
    case 5: return fns_for<2, 5, bfk::PMIXF, bfk::KIND_GENRADON>();
    case 6: return fns_for<2, 6, bfk::PMIXF, bfk::KIND_GENRADON>();
    case 8: return fns_for<2, 8, bfk::PMIXF, bfk::KIND_GENRADON>();
    default: return nullptr;
    }
}

}  // namespace bfl
