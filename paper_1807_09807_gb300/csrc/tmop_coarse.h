// Two-level preconditioner for the Krylov solves of Section 5 on structured
// order-k grids: the Jacobi part (the inverse diagonal of the stored
// Hessians) plus a coarse correction on the element-vertex lattice,
//   M^-1 r = D^-1 r + P (alpha K_c)^-1 P^t r,
// with P the interpolation of the trilinear (bilinear) vertex field at the
// element's Gauss-Lobatto nodes, K_c the reference-space Laplacian of that
// vertex field (per component; interior vertices, the boundary fixed), and
// alpha a Rayleigh quotient of the Hessian on the smoothest coarse mode, so
// that alpha K_c matches P^t H P at the low end of the spectrum. K_c is a
// Kronecker sum of 1D stiffness and mass matrices, which the sine transform
// diagonalises, so (alpha K_c)^-1 is applied exactly by three 1D transforms,
// one diagonal scaling and three more transforms. Both parts are symmetric
// positive definite, so M is, as MINRES needs.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>

namespace tmop {

struct CoarseSpace;

// Build the transfer and transform tables for a dim-dimensional structured
// grid of n[0] x n[1] (x n[2]) order-k elements (n >= 2 per axis; in 2D,
// n[2] > 1 is a stack of that many equal grids, each with its own coarse
// grid), Gauss-Lobatto nodes z[0..k] on [0,1]. fp32: the transforms run in
// FP32 (the FP32 forms); else FP64. Returns nullptr on a CUDA error or bad
// sizes.
CoarseSpace* coarse_create(int dim, int k, const int n[3], const double* z, bool fp32);
void coarse_destroy(CoarseSpace* cs);

// Coarse vector sizes: values per component, and the full [dim][..] count.
size_t coarse_size(const CoarseSpace* cs);

// y_fine = P w_coarse (FP64, [dim][nfine], overwritten)
int coarse_prolong(CoarseSpace* cs, const double* w, double* y, cudaStream_t s);
// The smoothest coarse mode (the first sine of every axis, unit norm per
// component and grid) in every component: w [dim][ncoarse]; *lambda0 =
// w_c^t K_c w_c for one component w_c (its K_c eigenvalue times the number
// of grids of a 2D stack).
int coarse_mode0(CoarseSpace* cs, double* w, double* lambda0, cudaStream_t s);
void coarse_set_alpha(CoarseSpace* cs, double alpha);

// y += P (alpha K_c)^-1 P^t r (r, y FP64 [dim][nfine]); if part is given,
// per-block partials (at most 256) of r . P (alpha K_c)^-1 P^t r, summed on
// the coarse grid in the sine basis, into part. Returns the number of
// partials, or -1.
int coarse_apply_add(void* cs, const double* r, double* y, double* part, cudaStream_t s);
// the same for FP32 fine vectors r, y (the FP32 forms' Krylov vectors)
int coarse_apply_add32(void* cs, const float* r, float* y, double* part, cudaStream_t s);

}  // namespace tmop
