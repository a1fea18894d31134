// Jacobians at the quadrature points and targets built from them (setup-time
// work, FP64).
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "tmop_kparams.h"

namespace tmop {

struct JacParams {
  int dim, nelem, nnode, n, q1, sx, sy, sz;
  const int32_t* elem_nodes;  // [nelem][n^d] (unstructured) or null
  const double* x;            // [d][nnode]
  double* J;                  // [nelem][Q][d][d] out
  double B[kMaxQ * kMaxN], G[kMaxQ * kMaxN], w1[kMaxQ];
};

// J = A(x) at every point.
int jacobians(const JacParams& p, cudaStream_t s);

// From J ([cnt][d][d]) at every point: W = J (kind 0) or W = det(J)^{1/d} I
// (kind 1); writes W^-1 and det W, and counts points with det J <= 0 into
// *bad (device int, zeroed by the caller).
int targets_from_jacobians(int dim, int kind, const double* J, size_t cnt, double* Winv, double* detW, int* bad,
                           cudaStream_t s);

// *out (device) = sum_E sum_q w_q det J (the measure of the mesh),
// deterministic; w1 HOST 1D weights.
int mesh_measure(int dim, int q1, const double* J, size_t nelem, const double* w1, double* out, cudaStream_t s);

}  // namespace tmop
