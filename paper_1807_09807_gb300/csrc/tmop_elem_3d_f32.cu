// Element-kernel instantiations: dim 3, float arithmetic, (n = order+1, q)
// pairs, including the compact partially assembled pair (its product is the
// software-pipelined kernel of tmop_pa_compact.cu).
#include "tmop_element.cuh"
#include "tmop_pa_compact.h"

namespace tmop {

#define TMOP_ENTRY(N, Q, OP) \
    {3, N, Q, 1, OP, launch_elem<3, N, Q, float, OP>, prepare_elem<3, N, Q, float, OP>, \
     ElemCfg<3, N, Q, float, OP>::WARPS}
#define TMOP_ENTRIES(N, Q)                                                                      \
  TMOP_ENTRY(N, Q, OP_ENERGY), TMOP_ENTRY(N, Q, OP_GRADIENT), TMOP_ENTRY(N, Q, OP_HESS),         \
      TMOP_ENTRY(N, Q, OP_LINEARIZE), TMOP_ENTRY(N, Q, OP_HESS_PA), TMOP_ENTRY(N, Q, OP_LINEARIZE_C), \
      {3, N, Q, 1, OP_HESS_PA_C, launch_pac<N, Q>, prepare_pac<N, Q>, kPacWarps}, \
      {3, N, Q, 1, OP_HESS_C, launch_pacr<N, Q>, prepare_pacr<N, Q>, kPacrWarps}

extern const ElemEntry kElem_3d_f32[] = {
    TMOP_ENTRIES(2,2),
    TMOP_ENTRIES(2,3),
    TMOP_ENTRIES(3,3),
    TMOP_ENTRIES(3,4),
    TMOP_ENTRIES(4,4),
    TMOP_ENTRIES(4,5),
    TMOP_ENTRIES(5,5),
    TMOP_ENTRIES(5,6),
};
extern const int kElem_3d_f32_len = sizeof(kElem_3d_f32) / sizeof(ElemEntry);

}  // namespace tmop
