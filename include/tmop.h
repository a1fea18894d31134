/*
 * tmop.h -- C ABI of the GB300 (sm_103a) high-order TMOP library.
 *
 * The library evaluates the variational TMOP objective of Dobrev, Knupp,
 * Kolev, Mittal and Tomov, "The Target-Matrix Optimization Paradigm for
 * High-Order Meshes" (SIAM J. Sci. Comput., 2019), on quadrilateral and
 * hexahedral meshes with continuous Q_k node positions, together with its
 * gradient and its matrix-free Hessian action, and minimises it with the
 * damped Newton method and det(A) > 0 line search of Section 3.4.
 *
 * Conventions for every call:
 *   - d = dim (2 or 3), k = order, n = k + 1, q = quadrature points per
 *     direction, Q = q^d points per element.
 *   - Position-like vectors (x, g, v, y) are caller-owned DEVICE pointers to
 *     FP64 arrays in SoA layout [d][nnode]: component a of node i is at
 *     index a * nnode + i. They must not overlap each other.
 *   - The reference element is [0,1]^d; the nodal basis is the Lagrange basis
 *     on the Gauss-Lobatto points of the element (x fastest, then y, then z).
 *   - Fixed degrees of freedom (the "fixed boundary nodes" of Section 4.1)
 *     read as zero in every direction vector and are written as zero in
 *     every output vector.
 *   - stream is a cudaStream_t passed as void* (NULL = the legacy default
 *     stream). Every call is asynchronous on that stream unless it returns
 *     host scalars, in which case it synchronises that stream before returning.
 *   - Every call returns a status code (tmop_status). No call blocks without a
 *     bound: there are no device-side spin waits anywhere in the library.
 *   - A context is not thread-safe: calls on one context must not overlap.
 */
#ifndef TMOP_H
#define TMOP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  TMOP_OK = 0,
  TMOP_ERR_ARG = 1,           /* invalid argument (sizes, ids, null pointers) */
  TMOP_ERR_CUDA = 2,          /* a CUDA runtime call failed */
  TMOP_ERR_INVERTED = 3,      /* some quadrature point has det A <= 0 (Section 3.2, ideal barrier) */
  TMOP_ERR_LINESEARCH = 4,    /* no admissible step length (Section 3.4) */
  TMOP_ERR_NOT_CONVERGED = 5, /* an iteration cap was reached */
  TMOP_ERR_CAPACITY = 6       /* the problem needs more scratch than a fixed-size buffer holds */
} tmop_status;

enum { TMOP_GL = 0, TMOP_GLL = 1 };                                     /* quadrature kind */
enum { TMOP_W_IDENTITY = 0, TMOP_W_CONST = 1, TMOP_W_SCALED = 2, TMOP_W_PER_QP = 3 }; /* target kind */
enum { TMOP_FP64 = 0, TMOP_FP32_MIXED = 1, TMOP_FP32_BULK = 2 };        /* precision form */
enum { TMOP_KRYLOV_MINRES = 0, TMOP_KRYLOV_CG = 1 };                     /* inner solver */
enum { TMOP_WT_EQUAL_SIZE = 0, TMOP_WT_LOCAL_SIZE = 1, TMOP_WT_INITIAL = 2 }; /* targets from positions */

typedef struct tmop_ctx tmop_ctx; /* opaque; owns device tables and workspace */

/* Mesh topology (Section 2.1, eq. (2.1)): nelem elements, each with
 * (order+1)^dim nodes in local lexicographic order (x fastest), continuous
 * across elements through the global node ids in elem_nodes. */
typedef struct {
  int dim;                    /* 2 or 3 */
  int nelem;                  /* number of elements, >= 1 */
  int nnode;                  /* number of global nodes, >= 1 */
  const int32_t* elem_nodes;  /* HOST [nelem][(order+1)^dim] global node ids, copied at setup;
                                 may be NULL when structured[] is set */
  const uint8_t* fixed;       /* HOST [dim][nnode], 1 = fixed dof; NULL = nothing fixed; copied */
  int structured[3];          /* nx, ny, (nz) of a lexicographic order-k grid whose node lattice is
                                 (k*nx+1) x (k*ny+1) (x (k*nz+1)), x fastest, elements x fastest;
                                 all 0 = unstructured. When set, node ids are computed, not read. */
} tmop_mesh;

/* Quadrature (Section 3.3): tensor Gauss-Legendre or Gauss-Lobatto rule with
 * npts1d points per direction on [0,1] (weights sum to 1). */
typedef struct {
  int kind;    /* TMOP_GL or TMOP_GLL */
  int npts1d;  /* 2..8; Section 3.3 asks for at least order+1 */
} tmop_quad;

/* Target matrices W (Section 3.1), fixed during the optimisation, det W > 0:
 *   TMOP_W_IDENTITY  W = I                       (the paper's W1)
 *   TMOP_W_SCALED    W = scale * I, scale > 0    (e.g. W2 = sqrt(alpha_bar) I, eq. (3.1))
 *   TMOP_W_CONST     W = the HOST [dim][dim] row-major matrix at W
 *   TMOP_W_PER_QP    W = HOST [nelem][Q][dim][dim] array, one matrix per
 *                    quadrature point (e.g. W3 = sqrt(det A(x0)) I). */
typedef struct {
  int kind;
  double scale;
  const double* W;
} tmop_targets;

/* Create a context: validates the mesh, builds the 1D quadrature and the
 * Lagrange value/derivative tables at the quadrature points, inverts the
 * targets, uploads everything and allocates the workspace (reduction
 * partials, Krylov vectors).
 *   order     1..4 (k of Q_k)
 *   metric_id 2D: 1, 2, 7, 9, 14, 77, 98; 3D: 1, 14, 98, 302, 303
 *             (Table 3.1; mu98 = |T - I|^2 / det T is the replication
 *             metric of Section 4.3.2; mu302 = |T|^2 |T^-1|^2 / 9 - 1 is not
 *             in the paper)
 *   precision TMOP_FP64: every kernel in FP64.
 *             TMOP_FP32_MIXED: the Hessian action (the Krylov operator) in
 *             FP32; objective, det A, gradient, dot products, line search
 *             and convergence tests in FP64, so Newton converges to the FP64
 *             solution with FP32 inner solves.
 *             TMOP_FP32_BULK: every element kernel (Jacobian contractions, mu
 *             and its derivatives, Hessian action) in FP32, with F, min det A,
 *             dot products and norms reduced in FP64.
 * Errors: TMOP_ERR_ARG (bad sizes or ids, node ids out of range, det W <= 0,
 * structured[] inconsistent with elem_nodes), TMOP_ERR_CUDA. On error *out is NULL. */
int tmop_setup(const tmop_mesh* mesh, int order, const tmop_quad* quad, int metric_id,
               const tmop_targets* targets, int precision, tmop_ctx** out);

/* Objective F_V(x) = sum_E sum_q w_q det W(x_q) mu(T(x_q)), T = A W^-1 with
 * A = sum_i x_i grad w_i (eq. (2.2), eq. (2.4)), and min over all points of
 * det A. F and min_detA are HOST pointers written after the stream is
 * synchronised. If some det A <= 0, *F = +inf for barrier metrics (the
 * large objective Section 3.4 asks for at inverted points) and TMOP_ERR_INVERTED is returned with
 * *min_detA set. */
int tmop_energy(tmop_ctx* ctx, const double* x, double* F, double* min_detA, void* stream);

/* Same objective and minimum as tmop_energy, written asynchronously to the
 * DEVICE scalars F and min_detA (one FP64 each) on the stream, without a
 * host synchronisation (for autograd and stream-ordered callers). Points with
 * det A <= 0 make *F = +inf under a barrier metric; the caller reads
 * *min_detA to detect inversion. */
int tmop_energy_device(tmop_ctx* ctx, const double* x, double* F, double* min_detA, void* stream);

/* Gradient g = dF_V/dx (Section 3.4): g_{i,a} = sum_E sum_q w_q det W
 * [ (dmu/dT)(T) W^-t grad w_i ]_a, zero at fixed dofs. g: DEVICE [d][nnode],
 * overwritten. Asynchronous. Points with det A <= 0 contribute nothing under a
 * barrier metric; check tmop_energy first. */
int tmop_gradient(tmop_ctx* ctx, const double* x, double* g, void* stream);

/* The gradient (as tmop_gradient, g: DEVICE [d][nnode], overwritten) and F
 * and min det A (as tmop_energy_device: DEVICE pointers, one double each) of
 * the same x in one element pass where the context allows it (not with
 * tmop_set_deterministic or the restricted-movement term, and FP64 element
 * kernels: TMOP_FP64 or TMOP_FP32_MIXED), else the two passes one after the
 * other; the results agree with the separate calls up to the order of the
 * sums. The Newton line search uses it at every trial. Asynchronous. */
int tmop_energy_gradient(tmop_ctx* ctx, const double* x, double* g, double* F, double* min_detA, void* stream);

/* Hessian action y = (d^2 F_V / dx^2)(x) v (Section 3.4: second derivatives
 * of mu with respect to T): y_{i,a} = sum_E sum_q w_q det W
 * [ (d^2mu/dT^2 : dT) W^-t grad w_i ]_a with dT = (sum_j v_j grad w_j) W^-1,
 * v masked at fixed dofs, y zero there. Matrix-free (recomputes A from x).
 * y: DEVICE [d][nnode], overwritten. Asynchronous. */
int tmop_hess_apply(tmop_ctx* ctx, const double* x, const double* v, double* y, void* stream);

/* The gradient g = dF/dx (as tmop_gradient) and the Hessian action
 * y = H(x) v (as tmop_hess_apply) at the same x (Section 3.4: both are
 * built from the same T = A W^-1, its P = dmu/dT and d^2mu/dT^2), in one
 * element pass: x is gathered and A(x) contracted once, the metric's terms
 * at each point serve both outputs, and two adjoint contractions scatter g
 * and y. The pass covers FP64 contexts with atomic sums, no composite term
 * and no restricted movement; any other context runs tmop_gradient and then
 * tmop_hess_apply. Results equal the two calls' up to rounding.
 * g, y: DEVICE [d][nnode], distinct from each other and from x and v,
 * overwritten (zero at fixed dofs). TMOP_ERR_ARG for a null pointer or an
 * output aliasing another argument. Asynchronous. */
int tmop_gradient_hess_apply(tmop_ctx* ctx, const double* x, const double* v, double* g, double* y, void* stream);

/* Partial assembly of the Hessian (Section 3.4: the Hessian from d^2mu/dT^2):
 * stores, at every quadrature point of x, the symmetric A-space matrix
 *   H_q = w_q det W (d^2mu/dT^2 composed with W^-1 on both sides)
 * (dim^2 (dim^2 + 1) / 2 values per point, FP64 under TMOP_FP64 and FP32
 * under the FP32 forms) in the context (allocated on first use:
 * nelem * Q * 45 * 8 bytes for order-k hexes in FP64). A 3D FP32 context
 * whose metric is written in |T|^2 and det T (1, 14, 303), with a constant
 * target and no second term, stores instead 14 values per point from which
 * the product rebuilds H_q (see tmop_pa_layout). Asynchronous. */
int tmop_linearize(tmop_ctx* ctx, const double* x, void* stream);

/* y = H(x) v with the Hessians stored by the last tmop_linearize(x): same
 * result as tmop_hess_apply(ctx, x, v, y) up to rounding, without reading x.
 * TMOP_ERR_ARG if the context holds no linearisation. Asynchronous. */
int tmop_hess_apply_pa(tmop_ctx* ctx, const double* v, double* y, void* stream);

/* y += H(x) v at the free dofs (y unchanged at the fixed ones), with the
 * Hessians stored by the last tmop_linearize(x): tmop_hess_apply_pa without
 * zeroing y first. The Krylov solves use this form on a buffer that their
 * previous vector pass left zero. TMOP_ERR_ARG if the context holds no
 * linearisation. Asynchronous. */
int tmop_hess_apply_pa_add(tmop_ctx* ctx, const double* v, double* y, void* stream);

/* The same accumulating product on FP32 vectors (DEVICE [dim][nnode]
 * float): y += H(x) v at the free dofs with FP32 atomics, the form the FP32
 * contexts' MINRES runs (tmop_newton_opts.krylov_fp64 = 0). TMOP_ERR_ARG for
 * a TMOP_FP64 context, with the restricted-movement term, or without a
 * linearisation. Asynchronous. */
int tmop_hess_apply_pa_add_f32(tmop_ctx* ctx, const float* v, float* y, void* stream);

/* Layout of the stored linearisation: values per quadrature point (the
 * packed upper triangle of the d^2 x d^2 A-space Hessian, 10 in 2D and 45 in
 * 3D; or, for a 3D FP32 context with an (|T|^2, det T) metric, a constant
 * target and no second term, the 14-value record T, w det W (mu_1, mu_t,
 * mu_11, mu_1t, mu_tt) the product rebuilds the Hessian from), the element
 * stride in values (each element's block [value][point], padded to 16 bytes)
 * and the bytes per value (8 FP64, 4 FP32). Any pointer may be NULL.
 * Errors: TMOP_ERR_ARG if nothing is stored. */
int tmop_pa_layout(const tmop_ctx* ctx, int* values_per_point, int* stride, int* elt_bytes);

/* Diagonal of the Hessian stored by the last tmop_linearize (including the
 * restricted-movement term), 1 at fixed dofs: out DEVICE [dim][nnode] FP64.
 * TMOP_ERR_ARG if the context holds no linearisation. Asynchronous. */
int tmop_hessian_diagonal(tmop_ctx* ctx, double* out, void* stream);

/* Newton options (Section 3.4 and Section 5). Zero-initialised fields take
 * the defaults in brackets. */
typedef struct {
  int max_newton;        /* [10] Newton iterations for tmop_newton_solve */
  double rtol;           /* [1e-12] stop when |g| <= rtol |g(x0)| (Section 5) */
  int krylov;            /* [TMOP_KRYLOV_MINRES] (Section 5 uses MINRES) */
  double krylov_rtol;    /* [1e-10 FP64, 1e-6 FP32 forms] relative residual of the inner solve */
  int krylov_maxit;      /* [2000] */
  double alpha_shrink;   /* [0.5] step reduction factor */
  int max_halvings;      /* [30] */
  double f_factor;       /* [1.2] accept only if F(x_new) < f_factor F(x) */
  double g_factor;       /* [1.2] accept only if |g(x_new)| < g_factor |g(x)| */
  double atol;           /* [0 = off] also stop when |g| <= atol (an absolute target, e.g. to
                            compare runs that start from different iterates) */
  int matrix_free;       /* [0] 0: the Krylov operator is partially assembled once per Newton
                            step (tmop_linearize), 1: recomputed from x at every product */
  int precond;           /* [0] 0: none (the paper's standard MINRES), 1: Jacobi, the diagonal of the
                            partially assembled Hessian (MINRES only; needs matrix_free = 0),
                            2: two-level, Jacobi plus an exact coarse correction on the element
                            vertices (structured grids whose fixed dofs are exactly the
                            boundary; else TMOP_ERR_ARG): see tmop_precond_apply */
  int krylov_fp64;       /* [0] the FP32 forms run MINRES on FP32 vectors (the Hessian action
                            is FP32 there; scalars, reductions and the Newton step stay FP64)
                            whenever the operator is partially assembled and no
                            restricted-movement term is set; 1: FP64 vectors. TMOP_FP64: always
                            FP64. */
} tmop_newton_opts;

typedef struct {
  int status;            /* tmop_status of the step or solve */
  int iterations;        /* Newton steps taken (solve) or 1 (step) */
  int krylov_iterations; /* inner iterations of the last step (sum for a solve) */
  double alpha;          /* accepted step length of the last step (0 if none) */
  double F;              /* objective at the returned x */
  double grad_norm;      /* |g| (free dofs) at the returned x */
  double grad_norm0;     /* |g| at the starting x */
  double min_detA;       /* min det A at the returned x */
} tmop_newton_report;

/* One damped Newton step (Section 3.4): p = H(x)^-1 g(x) by MINRES or CG on
 * the free dofs, then alpha = 1, alpha_shrink, ... until x - alpha p has
 * det A > 0 at every point, F < f_factor F(x) and |g| < g_factor |g(x)|.
 * x: DEVICE [d][nnode], updated in place only when a step is accepted.
 * report: HOST, may be NULL. Returns TMOP_ERR_LINESEARCH when no step
 * length is admissible (x unchanged), TMOP_ERR_INVERTED when x itself is
 * inverted. Synchronises the stream (the line-search decisions are taken on
 * the host from FP64 device reductions). */
int tmop_newton_step(tmop_ctx* ctx, double* x, const tmop_newton_opts* opts, tmop_newton_report* report,
                     void* stream);

/* Newton iterations from x until |g| <= rtol |g(x0)| or |g| <= atol (TMOP_OK), no admissible
 * step (TMOP_ERR_LINESEARCH, the termination rule of Section 3.4) or
 * max_newton steps (TMOP_ERR_NOT_CONVERGED). x: DEVICE, in/out. */
int tmop_newton_solve(tmop_ctx* ctx, double* x, const tmop_newton_opts* opts, tmop_newton_report* report,
                      void* stream);

/* The preconditioner of the Krylov solves (Section 5 runs MINRES; the paper
 * does not state its preconditioner): z = M^-1 r for the linearisation at x
 * (stored as by tmop_linearize). precond 1: M^-1 = D^-1, the floored
 * inverse diagonal of the stored Hessian (fixed dofs 1). precond 2:
 *   M^-1 r = D^-1 r + P (alpha K_c)^-1 P^t r,
 * with P the interpolation of a bilinear (2D) / trilinear (3D) field on the
 * element vertices at the Gauss-Lobatto nodes of each element, K_c the
 * reference-space Laplacian of the vertex field (per component, interior
 * vertices; the Kronecker sum of the 1D element stiffness and mass
 * matrices, applied inversely by sine transforms, in FP64 for TMOP_FP64
 * and FP32 otherwise) and alpha = (P w)^t H (P w) / (w^t K_c w) for the
 * smoothest coarse mode w in every component (*alpha, 0 if H is not
 * positive on it: then the coarse part is left out). Needs a structured
 * grid whose fixed dofs are exactly the boundary (TMOP_ERR_ARG otherwise).
 * r, z DEVICE [d][nnode]; alpha HOST or NULL. Synchronises the stream. */
int tmop_precond_apply(tmop_ctx* ctx, const double* x, int precond, const double* r, double* z, double* alpha,
                       void* stream);

/* Inner Krylov solve H(x) p = b alone (MINRES or CG, zero initial guess),
 * for tests: b, p DEVICE [d][nnode]. Returns iterations through *iters
 * (negative if krylov_maxit was reached). */
int tmop_krylov_solve(tmop_ctx* ctx, const double* x, const double* b, double* p, const tmop_newton_opts* opts,
                      int* iters, void* stream);

/* Per-element minimum of det A over its quadrature points: out DEVICE
 * [nelem] FP64 (the validity test behind the barrier of Section 3.2). */
int tmop_element_min_detA(tmop_ctx* ctx, const double* x, double* out, void* stream);

/* Objective and minimum det A WITHOUT ANY DEVICE ALLOCATION. The paper has
 * no counterpart: this is a convenience for callers that may not call
 * cudaMalloc where they evaluate mesh quality -- e.g. an application whose
 * own allocator or memory pool owns the GPU, or code running inside another
 * program's time step where cudaMalloc's implicit synchronisation is not
 * acceptable -- and that therefore cannot create a tmop_setup context.
 *
 * Same F and min det A as tmop_energy (eq. (2.4)), FP64, on a structured
 * order-k grid only (node ids are computed from structured[] = nx, ny, nz,
 * laid out as for tmop_mesh.structured): dim 2 or 3, order 1..4, quad as for
 * tmop_setup, metric_id as for tmop_setup, targets of kind IDENTITY, SCALED
 * or CONST (TMOP_W_PER_QP is rejected with TMOP_ERR_ARG). x: DEVICE
 * [dim][nnode] FP64. F, min_detA: DEVICE FP64 scalars, written
 * asynchronously on stream (no host synchronisation). F = +inf under a barrier
 * metric when some det A <= 0.
 *
 * Scratch: the per-block partial sums live in one file-scope device array of
 * 2 x 32768 doubles (512 KiB) that every GPU loading this library keeps until
 * the process exits. The launch uses one block per group of elements in
 * flight (4 to 8 per block, set by the kernel's shared memory), so the limit
 * is 32768 x that many elements (131 072 to 262 144); larger grids return
 * TMOP_ERR_CAPACITY before anything is launched. The array is shared by every
 * call in the process and keeps the last call's contents (each call overwrites
 * the partials it reads, so nothing has to start at zero); calls that overlap
 * on the GPU -- on different streams, or from different host threads --
 * race on it and must be serialised by the caller.
 *
 * The first call on each device looks up the device address of that array
 * (cudaGetSymbolAddress, with the device current) and may load the kernels
 * it launches; make that first call before any stream capture. */
int tmop_energy_noalloc(int dim, int order, const int structured[3], const tmop_quad* quad, int metric_id,
                        const tmop_targets* targets, const double* x, double* F, double* min_detA, void* stream);

/* Composite metric (Section 4.2, eq. (4.1)): adds a second term so that the
 * objective becomes sum_E sum_q w_q [ det W mu(A W^-1) + eta_q det W2 mu2(A W2^-1) ]
 * in every call (energy, gradient, Hessian actions, linearisation, Newton).
 * metric2 as for tmop_setup (0 removes the term); W2: HOST [dim][dim]
 * constant target, det W2 > 0; eta2: HOST [nelem][Q] per-point weights
 * (copied; held fixed during the optimisation), or NULL for 1 everywhere.
 * Invalidates a stored linearisation. Errors: TMOP_ERR_ARG, TMOP_ERR_CUDA. */
int tmop_set_composite(tmop_ctx* ctx, int metric2, const double* W2, const double* eta2);

/* Deterministic sums (on = 1) or atomics (on = 0, the default). The nodal
 * outputs -- gradient (Section 3.4, summed over the elements that contain
 * node i), Hessian actions, the stored-Hessian product, the Jacobi
 * diagonal, the restricted-movement terms -- are sums of element
 * contributions. By default every element adds with FP64 atomics, whose
 * order (and so the last bits) varies from run to run. With on = 1 the
 * elements are split into colours whose elements share no node (the 2^dim
 * parity classes of a structured grid; a greedy colouring otherwise, at most
 * 64 colours) and launched one colour after another in a fixed order: each
 * node then receives at most one add per launch, so the order of every
 * node's sum is fixed, and every output -- and every Newton and Krylov
 * iterate -- is the same bit for bit on every run with the same launch
 * shapes. Costs one launch per colour per operator application. Errors:
 * TMOP_ERR_ARG (more than 64 colours), TMOP_ERR_CUDA. */
int tmop_set_deterministic(tmop_ctx* ctx, int on);

/* Restricted node movement (Section 4.3.1, eq. (4.2)): every call then
 * evaluates F + sum_E int_{E_t} delta |x - x_init|^2 dx_t (weights w_q det W),
 * with the matching gradient and Hessian-action terms (FP64, whatever the
 * precision form). delta >= 0 (0 removes the term); x_init: DEVICE
 * [dim][nnode] FP64, copied on the stream. Errors: TMOP_ERR_ARG,
 * TMOP_ERR_CUDA. */
int tmop_set_restricted_movement(tmop_ctx* ctx, double delta, const double* x_init, void* stream);

/* Jacobians A(x_q) = sum_i x_i grad phi_i(xi_q) (eq. (2.2)) at every
 * quadrature point: x DEVICE [dim][nnode], J DEVICE [nelem][Q][dim][dim]
 * row-major (J[e][q][a][b] = d x_a / d xi_b), points ordered as the
 * quadrature (first direction fastest). Asynchronous on the stream. Errors:
 * TMOP_ERR_ARG, TMOP_ERR_CUDA. */
int tmop_jacobians(tmop_ctx* ctx, const double* x, double* J, void* stream);

/* Replace the context's targets by a set built from the positions x0
 * (DEVICE [dim][nnode]):
 *   TMOP_WT_EQUAL_SIZE  W2 = alpha^{1/d} I, alpha = (1/N_E) sum_E sum_q w_q
 *                       det A(x0), the quadrature of eq. (3.1) (constant)
 *   TMOP_WT_LOCAL_SIZE  W3 = det(A(x0))^{1/d} I at every point (Section 3.1)
 *   TMOP_WT_INITIAL     W0 = A(x0) at every point: the target of the
 *                       replication metric mu98 in the second restricted
 *                       node movement algorithm (Section 4.3.2), where
 *                       (1 - gamma) mu98(A W0^-1) + gamma mu(A W^-1) is a
 *                       context with metric 98 and these targets plus
 *                       tmop_set_composite(mu, W, eta2 = gamma / (1 - gamma))
 *                       (the same objective times 1 / (1 - gamma)).
 * Allocates temporaries, synchronises the stream, invalidates a stored
 * linearisation. Errors: TMOP_ERR_INVERTED if det A(x0) <= 0 at some point
 * (per-point kinds) or the measure is not positive (targets unchanged),
 * TMOP_ERR_ARG, TMOP_ERR_CUDA. */
int tmop_set_targets_from_positions(tmop_ctx* ctx, int kind, const double* x0, void* stream);

/* Diagnostic: the FP64 -> FP32 -> FP64 conversions the FP32 kernels apply
 * to gathered values and to their contributions (integer-pipe
 * implementations: round to nearest even, results below 2^-126 in magnitude
 * become a signed zero, FP32 -> FP64 exact). in DEVICE [n] FP64; f32 DEVICE
 * [n] receives the converted values, back DEVICE [n] FP64 their exact
 * widening. Asynchronous. Errors: TMOP_ERR_ARG, TMOP_ERR_CUDA. */
int tmop_selftest_convert(const double* in, float* f32, double* back, size_t n, void* stream);

/* Diagnostic: tau^{-1/3} as the FP64 kernels evaluate it (mu303 and its
 * derivatives): Newton's method from an FP32 estimate on [2^-120, 2^120],
 * the library cube root elsewhere. in, out DEVICE [n] FP64. Asynchronous.
 * Errors: TMOP_ERR_ARG, TMOP_ERR_CUDA. */
int tmop_selftest_rcbrt(const double* in, double* out, size_t n, void* stream);

/* Measured FMA throughput of the current GPU (not part of the method: the
 * denominator of the rooflines of the FP64 and FP32 element kernels, which
 * are bound by their arithmetic pipes, not by HBM). kind TMOP_PEAK_FP64
 * (DFMA), TMOP_PEAK_FP32 (FFMA) or TMOP_PEAK_FP32X2 (the paired FP32
 * instruction, two multiply-adds each). Every thread of a grid of 1024
 * threads per SM runs 8 independent multiply-add chains for a fixed count
 * (a few ms per launch); one untimed launch, then the best of 3 timed with
 * CUDA events on the stream, which this call synchronises. scratch: DEVICE,
 * at least SMs * 1024 * 8 bytes (each thread's sum, so that no work is dead
 * code). *gflops = 2 * multiply-adds / best time (GFLOP/s); *ms = that time
 * (may be NULL). Errors: TMOP_ERR_ARG, TMOP_ERR_CAPACITY (scratch too
 * small), TMOP_ERR_CUDA. */
enum { TMOP_PEAK_FP64 = 0, TMOP_PEAK_FP32 = 1, TMOP_PEAK_FP32X2 = 2 };
int tmop_fma_peak(int kind, void* scratch, size_t scratch_bytes, double* gflops, double* ms, void* stream);

/* Vector helpers for callers that split a mesh over GPUs (slab sharding:
 * a halo sum of the node planes two slabs share, and dot products that count
 * each shared plane once). Not part of the paper's method.
 * tmop_vec_add: y += b, DEVICE [n] FP64. Asynchronous.
 * tmop_vec_dot_segments: *out (DEVICE scalar) = sum over c < ncomp, i < count
 * of a[c stride + first + i] b[c stride + first + i] (FP64, a fixed-order
 * two-pass reduction); scratch DEVICE, at least 2048 doubles (the block
 * partials; TMOP_ERR_CAPACITY if scratch_len is smaller than the grid).
 * Asynchronous. Errors: TMOP_ERR_ARG, TMOP_ERR_CAPACITY, TMOP_ERR_CUDA.
 * tmop_vec_axpby: y = a x + b y, DEVICE [n] FP64 (b = 0: y = a x, y's old
 * contents not read), the vector updates of a Newton-MINRES driver over
 * such slabs. x may be y. Asynchronous. */
int tmop_vec_add(double* y, const double* b, size_t n, void* stream);
int tmop_vec_axpby(double* y, double a, const double* x, double b, size_t n, void* stream);
int tmop_vec_dot_segments(const double* a, const double* b, int ncomp, size_t stride, size_t first, size_t count,
                          double* scratch, size_t scratch_len, double* out, void* stream);

/* Sizes of a context: Q (points per element), ndof = dim * nnode. */
int tmop_sizes(const tmop_ctx* ctx, int* dim, int* nelem, int* nnode, int* Q);

/* Release every device allocation of the context. NULL is ignored. */
void tmop_destroy(tmop_ctx* ctx);

/* Static text for a status code. */
const char* tmop_status_string(int status);

#ifdef __cplusplus
}
#endif
#endif /* TMOP_H */
