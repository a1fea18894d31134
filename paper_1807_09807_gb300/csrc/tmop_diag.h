// Diagonal of the partially assembled Hessian (Jacobi preconditioner).
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "tmop_kparams.h"

namespace tmop {

struct DiagParams {
  int dim, nelem, nnode, sx, sy, sz;
  const int32_t* elem_nodes;  // [nelem][n^d] (unstructured) or null
  const void* pa;             // packed Hessians [nelem][pa_stride] (float or double)
  int pa_stride;
  double* diag;               // [d][nnode], accumulated (zero it first)
  double B[kMaxQ * kMaxN], G[kMaxQ * kMaxN], w1[kMaxQ];
  double delta, detW;         // restricted-movement term (delta = 0: none)
  const double* detW_qp;
  int compact;                // pa holds 3D compact records (T, scaled partials of mu)
  int identity;               // W = I (else the constant Winv)
  double Winv[9];
  const int32_t* elist;       // one colour's elements (one add per node and launch), or null: all
  int ecount;
};

typedef int (*diag_launch_fn)(const DiagParams& p, int grid, void* stream);

diag_launch_fn find_diag(int dim, int n, int q, int fp32);
int diag_grid(int nelem);
// fixed dofs -> 1
int diag_finish(double* diag, const uint8_t* fixed, size_t n, cudaStream_t s);
// minv = 1 / max(|diag|, floor_abs)
int diag_inverse(const double* diag, double* minv, size_t n, double floor_abs, cudaStream_t s);

}  // namespace tmop
