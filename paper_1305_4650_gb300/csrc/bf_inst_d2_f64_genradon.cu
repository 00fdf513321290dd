// Kernels for d = 2, precision PF64, phase kind genradon (q in {2,3,4,5,6,8}).
#include "bf_inst.cuh"

namespace bfl {

const PassFns *fns_d2_f64_genradon(int q)
{
    switch (q) {
    case 2: return fns_for<2, 2, bfk::PF64, bfk::KIND_GENRADON>();
    case 3: return fns_for<2, 3, bfk::PF64, bfk::KIND_GENRADON>();
    case 4: return fns_for<2, 4, bfk::PF64, bfk::KIND_GENRADON>();
    case 5: return fns_for<2, 5, bfk::PF64, bfk::KIND_GENRADON>();
    case 6: return fns_for<2, 6, bfk::PF64, bfk::KIND_GENRADON>();
    case 8: return fns_for<2, 8, bfk::PF64, bfk::KIND_GENRADON>();
    default: return nullptr;
    }
}

}  // namespace bfl
