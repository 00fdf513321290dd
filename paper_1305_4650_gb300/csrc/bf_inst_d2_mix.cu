// Kernels for d = 2, precision PMIX (q in {2,3,4,5,6,8}).
#include "bf_inst.cuh"

namespace bfl {

const PassFns *fns_d2_mix(int q)
{
    switch (q) {
    case 2: return fns_for<2, 2, bfk::PMIX>();
    case 3: return fns_for<2, 3, bfk::PMIX>();
    case 4: return fns_for<2, 4, bfk::PMIX>();
    case 5: return fns_for<2, 5, bfk::PMIX>();
    case 6: return fns_for<2, 6, bfk::PMIX>();
    case 8: return fns_for<2, 8, bfk::PMIX>();
    default: return nullptr;
    }
}

}  // namespace bfl
