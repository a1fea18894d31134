// Launch parameters of the TMOP element kernels, passed by value (they live
// in the kernel-parameter constant bank). The 1D tables are always FP64 here;
// FP32 kernels round them once into shared memory.
#pragma once
#include <stddef.h>
#include <stdint.h>

namespace tmop {

constexpr int kMaxQ = 8;   // 1D quadrature points
constexpr int kMaxN = 5;   // 1D nodes (order <= 4)

// OP_LINEARIZE stores the A-space Hessian of w det W mu at every point (once
// per Newton step); OP_HESS_PA applies it (partial assembly). The compact
// pair (3D FP32 only) stores instead what the second derivative of an
// (|T|^2, det T) metric is made of: T and the five scaled partials
// w det W (mu_1, mu_t, mu_11, mu_1t, mu_tt), 14 values per point instead of
// 45, and OP_HESS_PA_C rebuilds dP from them. OP_ENERGY_GRAD is the
// gradient with the energy partials of OP_ENERGY taken from the same points
// (one pass where the line search of the Newton step needs both).
// OP_GRAD_HESS (FP64) is the gradient (into g) and the Hessian action (into y)
// at the same x in one pass: A(x) and the point's metric terms serve both.
enum {
  OP_ENERGY = 0, OP_GRADIENT = 1, OP_HESS = 2, OP_LINEARIZE = 3, OP_HESS_PA = 4,
  OP_LINEARIZE_C = 5, OP_HESS_PA_C = 6, OP_ENERGY_GRAD = 7, OP_HESS_C = 8, OP_GRAD_HESS = 9, OP_COUNT = 10
};
constexpr int kCompactRec = 14;  // values per point of the compact record (3D)
enum { WK_IDENTITY = 0, WK_CONST = 1, WK_PER_QP = 2 };

struct KParams {
  int dim, nelem, nnode, metric, wkind;
  int sx, sy, sz;                 // structured grid (sx > 0) or elem_nodes
  const int32_t* elem_nodes;      // [nelem][n^d]
  const uint8_t* fixed;           // [d][nnode] or null
  const double* x;                // [d][nnode]
  const double* v;                // [d][nnode] (Hessian action)
  double* y;                      // [d][nnode] accumulated output
  double* g;                      // [d][nnode] accumulated gradient of OP_GRAD_HESS
  // FP32 direction and output of the stored-Hessian products (the FP32
  // forms' Krylov vectors), used instead of v and y when set
  const float* v32;
  float* y32;
  const double* Winv_qp;          // [nelem][Q][d][d] (per-point targets)
  const double* detW_qp;          // [nelem][Q]
  double* part_F;                 // [grid] energy partials
  double* part_min;               // [grid] min det A partials
  double* elem_min;               // [nelem] per-element min det A, or null
  void* pa;                       // [nelem][pa_stride] packed Hessians [DD(DD+1)/2][Q] (float or double)
  double* vdot;                   // product from compact records: per-warp partials of v . (H v), or null
  // Deterministic sums: when elist is set, the launch runs only the ecount
  // elements listed there, which share no node (one colour of the mesh), so
  // every node receives at most one (atomic) add per launch; the host
  // launches the colours one after another in a fixed order, which fixes the
  // order of every node's sum.
  const int32_t* elist;
  int ecount;
  int pa_stride;                  // elements per element block, padded to 16 bytes
  double B[kMaxQ * kMaxN];              // B[q][i] = phi_i(xi_q)
  double G[kMaxQ * kMaxN];              // G[q][i] = phi_i'(xi_q)
  double w1[kMaxQ];                // 1D quadrature weights
  double Winv[9];                 // constant W^-1 (row-major)
  double detW;                    // constant det W
  // optional second term of a composite metric (eq. (4.1)): + eta_q mu2(A W2^-1)
  int metric2;                    // 0 = no second term
  double Winv2[9];                // constant W2^-1
  double detW2;                   // det W2
  const double* eta2;             // [nelem][Q] weights of the second term, or null (= 1)
};

// Metrics of Table 3.1 (and mu98 of Section 4.3.2, mu302) available in
// dimension d.
inline bool metric_supported(int d, int id) {
  return id == 1 || id == 14 || id == 98 || (d == 2 && (id == 2 || id == 7 || id == 9 || id == 77)) ||
         (d == 3 && (id == 302 || id == 303));
}

// Per-element block of packed Hessians (or compact records), in elements of
// `elt` bytes, padded so that every block starts on a 16-byte boundary.
inline int pa_stride_for(int dim, int Q, int elt, bool compact = false) {
  const int dd = dim * dim, ns = compact ? kCompactRec : dd * (dd + 1) / 2;
  const int bytes = ((ns * Q * elt + 15) / 16) * 16;
  return bytes / elt;
}

// Metrics whose second derivative MetricLin writes in (|T|^2, det T).
inline bool metric_is_lin(int id) { return id != 302 && id != 98; }

typedef int (*elem_launch_fn)(const KParams& p, int grid, void* stream);
typedef int (*elem_prepare_fn)(int nelem, int* grid);

struct ElemEntry {
  int dim, n, q, fp32, op;
  elem_launch_fn launch;
  elem_prepare_fn prepare;
  int warps;  // warps (elements in flight) per block of this instantiation
};

// Defined in the per-dimension/precision instantiation units.
const ElemEntry* find_elem(int dim, int n, int q, int fp32, int op);

// Host-side 1D tables and target inversion (tmop_capi.cu).
bool rule_gl(int q, double* x, double* w);
bool rule_gll(int q, double* x, double* w);
void lagrange_bary(int n, const double* z, double s, double* phi, double* dphi);
bool inv_h(int d, const double* W, double* Wi, double* detW);

}  // namespace tmop
