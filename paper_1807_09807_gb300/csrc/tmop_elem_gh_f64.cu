// Element-kernel instantiations of the fused gradient + Hessian action
// (OP_GRAD_HESS), FP64, dims 2 and 3, the (n = order+1, q) pairs of the other
// FP64 tables.
#include "tmop_element.cuh"

namespace tmop {

#define TMOP_GH(D, N, Q)                                                                          \
  {D, N, Q, 0, OP_GRAD_HESS, launch_elem<D, N, Q, double, OP_GRAD_HESS>,                          \
   prepare_elem<D, N, Q, double, OP_GRAD_HESS>, ElemCfg<D, N, Q, double, OP_GRAD_HESS>::WARPS}

extern const ElemEntry kElem_gh_f64[] = {
    TMOP_GH(2, 2, 2), TMOP_GH(2, 2, 3), TMOP_GH(2, 3, 3), TMOP_GH(2, 3, 4), TMOP_GH(2, 3, 5),
    TMOP_GH(2, 4, 4), TMOP_GH(2, 4, 5), TMOP_GH(2, 4, 6), TMOP_GH(2, 5, 5), TMOP_GH(2, 5, 6),
    TMOP_GH(3, 2, 2), TMOP_GH(3, 2, 3), TMOP_GH(3, 3, 3), TMOP_GH(3, 3, 4), TMOP_GH(3, 4, 4),
    TMOP_GH(3, 4, 5), TMOP_GH(3, 5, 5), TMOP_GH(3, 5, 6),
};
extern const int kElem_gh_f64_len = sizeof(kElem_gh_f64) / sizeof(ElemEntry);

}  // namespace tmop
