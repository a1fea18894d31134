// Element-kernel instantiations: dim 3, double arithmetic, (n = order+1, q) pairs.
#include "tmop_element.cuh"

namespace tmop {

#define TMOP_ENTRY(N, Q, OP) \
    {3, N, Q, 0, OP, launch_elem<3, N, Q, double, OP>, prepare_elem<3, N, Q, double, OP>, \
     ElemCfg<3, N, Q, double, OP>::WARPS}
#define TMOP_ENTRIES(N, Q)                                                                      \
  TMOP_ENTRY(N, Q, OP_ENERGY), TMOP_ENTRY(N, Q, OP_GRADIENT), TMOP_ENTRY(N, Q, OP_HESS),         \
      TMOP_ENTRY(N, Q, OP_LINEARIZE), TMOP_ENTRY(N, Q, OP_HESS_PA), TMOP_ENTRY(N, Q, OP_ENERGY_GRAD)

extern const ElemEntry kElem_3d_f64[] = {
    TMOP_ENTRIES(2,2),
    TMOP_ENTRIES(2,3),
    TMOP_ENTRIES(3,3),
    TMOP_ENTRIES(3,4),
    TMOP_ENTRIES(4,4),
    TMOP_ENTRIES(4,5),
    TMOP_ENTRIES(5,5),
    TMOP_ENTRIES(5,6),
};
extern const int kElem_3d_f64_len = sizeof(kElem_3d_f64) / sizeof(ElemEntry);

}  // namespace tmop
