// Restricted-movement term (eq. (4.2)): value-contraction kernels.
#pragma once
#include <stdint.h>

#include "tmop_kparams.h"

namespace tmop {

struct MassParams {
  int dim, nelem, nnode, sx, sy, sz;
  const int32_t* elem_nodes;  // [nelem][n^d] (unstructured) or null
  const uint8_t* fixed;       // [d][nnode] or null
  const double* x;            // positions (energy, gradient)
  const double* x0;           // x_init of the term
  const double* v;            // direction (Hessian action)
  double* y;                  // accumulated output (gradient, Hessian action)
  double* part;               // [grid] energy partials
  double B[kMaxQ * kMaxN];    // B[q][i] = phi_i(xi_q)
  double w1[kMaxQ];
  double delta;
  double detW;                // constant det W
  const double* detW_qp;      // [nelem][Q] per-point det W, or null
  const int32_t* elist;       // one colour's elements (one add per node and launch), or null: all
  int ecount;
};

typedef int (*mass_launch_fn)(const MassParams& p, int grid, void* stream);

// mode 0: energy partials, 1: gradient (from x), 2: Hessian action (from v)
mass_launch_fn find_mass(int dim, int n, int q, int mode);
int mass_grid(int nelem);

}  // namespace tmop
