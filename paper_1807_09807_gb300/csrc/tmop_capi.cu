// C ABI of the GB300 TMOP library (declared in include/tmop.h).
//
// Host responsibilities: validate inputs, build the 1D quadrature and
// Lagrange tables, invert the targets, own the device workspace, sequence the
// kernels, and take the Newton line-search decisions (Section 3.4) from FP64
// device reductions. All arithmetic on mesh-sized data runs in the CUDA
// kernels of this library; there is no host fallback.
#include <type_traits>
#include <cuda_runtime.h>
#include <utility>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <vector>

#include "../../include/tmop.h"
#include "tmop_coarse.h"
#include "tmop_diag.h"
#include "tmop_targets.h"
#include "tmop_kparams.h"
#include "tmop_mass.h"
#include "tmop_vec.h"

namespace tmop {

extern const ElemEntry kElem_2d_f64[];
extern const int kElem_2d_f64_len;
extern const ElemEntry kElem_2d_f32[];
extern const int kElem_2d_f32_len;
extern const ElemEntry kElem_3d_f64[];
extern const int kElem_3d_f64_len;
extern const ElemEntry kElem_3d_f32[];
extern const int kElem_3d_f32_len;
extern const ElemEntry kElem_gh_f64[];
extern const int kElem_gh_f64_len;

const ElemEntry* find_elem(int dim, int n, int q, int fp32, int op) {
  const ElemEntry* t;
  int len;
  if (op == OP_GRAD_HESS) {  // FP64 only, both dimensions in one table
    if (fp32) return nullptr;
    for (int i = 0; i < kElem_gh_f64_len; ++i)
      if (kElem_gh_f64[i].dim == dim && kElem_gh_f64[i].n == n && kElem_gh_f64[i].q == q) return &kElem_gh_f64[i];
    return nullptr;
  }
  if (dim == 2) { t = fp32 ? kElem_2d_f32 : kElem_2d_f64; len = fp32 ? kElem_2d_f32_len : kElem_2d_f64_len; }
  else { t = fp32 ? kElem_3d_f32 : kElem_3d_f64; len = fp32 ? kElem_3d_f32_len : kElem_3d_f64_len; }
  for (int i = 0; i < len; ++i)
    if (t[i].n == n && t[i].q == q && t[i].op == op) return &t[i];
  return nullptr;
}

// ---------------------------------------------------------------- 1D tables
// Legendre P_m and P_m' by the Bonnet recurrence, with P_m' from the
// identity (1 - t^2) P_m' = m (P_{m-1} - t P_m).
static void legendre_pd(int m, double t, double* p, double* dp) {
  double a = 1.0, b = t;
  if (m == 0) { *p = 1.0; *dp = 0.0; return; }
  for (int k = 1; k < m; ++k) {
    double c = ((2 * k + 1) * t * b - k * a) / (k + 1);
    a = b;
    b = c;
  }
  *p = b;
  *dp = m * (a - t * b) / (1.0 - t * t);
}

// Gauss-Legendre: roots of P_q by Newton from Chebyshev-like guesses;
// weights 2 / ((1 - t^2) P_q'(t)^2) on [-1,1], mapped to [0,1].
bool rule_gl(int q, double* x, double* w) {
  for (int i = 0; i < q; ++i) {
    double t = -cos(M_PI * (4 * i + 3) / (4.0 * q + 2.0)), p, dp;
    for (int it = 0; it < 64; ++it) {
      legendre_pd(q, t, &p, &dp);
      const double dt = p / dp;
      t -= dt;
      if (fabs(dt) <= 1e-16) break;
    }
    legendre_pd(q, t, &p, &dp);
    x[i] = 0.5 + 0.5 * t;
    w[i] = 1.0 / ((1.0 - t * t) * dp * dp);
  }
  return true;
}

// Gauss-Lobatto: endpoints plus the roots of P_{q-1}', found by Newton on
// P_{q-1}' with P_{q-1}'' from the Legendre equation; weights
// 2 / (q (q-1) P_{q-1}(t)^2) on [-1,1], mapped to [0,1].
bool rule_gll(int q, double* x, double* w) {
  if (q < 2) return false;
  const int m = q - 1;
  for (int i = 0; i < q; ++i) {
    double t = -cos(M_PI * i / m);
    if (i > 0 && i < m) {
      for (int it = 0; it < 64; ++it) {
        double p, dp;
        legendre_pd(m, t, &p, &dp);
        const double d2p = (2.0 * t * dp - m * (m + 1.0) * p) / (1.0 - t * t);
        const double dt = dp / d2p;
        t -= dt;
        if (fabs(dt) <= 1e-16) break;
      }
    }
    double p;
    if (i == 0) p = (m % 2) ? -1.0 : 1.0;
    else if (i == m) p = 1.0;
    else { double dp; legendre_pd(m, t, &p, &dp); }
    x[i] = (i == 0) ? 0.0 : (i == m ? 1.0 : 0.5 + 0.5 * t);
    w[i] = 1.0 / (m * (m + 1.0) * p * p);
  }
  return true;
}

// Lagrange basis on nodes z (barycentric form): values and derivatives at s.
void lagrange_bary(int n, const double* z, double s, double* phi, double* dphi) {
  double bw[kMaxN];
  for (int i = 0; i < n; ++i) {
    double prod = 1.0;
    for (int j = 0; j < n; ++j)
      if (j != i) prod *= (z[i] - z[j]);
    bw[i] = 1.0 / prod;
  }
  int hit = -1;
  for (int i = 0; i < n; ++i)
    if (s == z[i]) hit = i;
  if (hit >= 0) {
    // at a node: phi = delta, phi' from the differentiation matrix
    for (int i = 0; i < n; ++i) phi[i] = (i == hit) ? 1.0 : 0.0;
    double diag = 0.0;
    for (int i = 0; i < n; ++i) {
      if (i == hit) continue;
      dphi[i] = (bw[i] / bw[hit]) / (z[hit] - z[i]);
      diag += 1.0 / (z[hit] - z[i]);
    }
    dphi[hit] = diag;
    return;
  }
  double ell = 1.0;
  for (int j = 0; j < n; ++j) ell *= (s - z[j]);
  for (int i = 0; i < n; ++i) {
    phi[i] = ell * bw[i] / (s - z[i]);
    double sum = 0.0;
    for (int j = 0; j < n; ++j)
      if (j != i) sum += 1.0 / (s - z[j]);
    dphi[i] = phi[i] * sum;
  }
}

static double det_h(int d, const double* M) {
  if (d == 2) return M[0] * M[3] - M[1] * M[2];
  return M[0] * (M[4] * M[8] - M[5] * M[7]) - M[1] * (M[3] * M[8] - M[5] * M[6]) +
         M[2] * (M[3] * M[7] - M[4] * M[6]);
}

// W^-1 by the adjugate; false when det W <= 0 (Section 3.1 requires det W > 0).
bool inv_h(int d, const double* W, double* Wi, double* detW) {
  const double dt = det_h(d, W);
  *detW = dt;
  if (!(dt > 0.0) || !isfinite(dt)) return false;
  if (d == 2) {
    Wi[0] = W[3] / dt; Wi[1] = -W[1] / dt; Wi[2] = -W[2] / dt; Wi[3] = W[0] / dt;
    return true;
  }
  Wi[0] = (W[4] * W[8] - W[5] * W[7]) / dt;
  Wi[1] = (W[2] * W[7] - W[1] * W[8]) / dt;
  Wi[2] = (W[1] * W[5] - W[2] * W[4]) / dt;
  Wi[3] = (W[5] * W[6] - W[3] * W[8]) / dt;
  Wi[4] = (W[0] * W[8] - W[2] * W[6]) / dt;
  Wi[5] = (W[2] * W[3] - W[0] * W[5]) / dt;
  Wi[6] = (W[3] * W[7] - W[4] * W[6]) / dt;
  Wi[7] = (W[1] * W[6] - W[0] * W[7]) / dt;
  Wi[8] = (W[0] * W[4] - W[1] * W[3]) / dt;
  return true;
}

}  // namespace tmop

using namespace tmop;

struct tmop_ctx {
  int dim, order, n, nq, Q, nelem, nnode, metric, precision;
  size_t ndof;
  KParams base;
  const ElemEntry* ent[OP_COUNT];
  int grid[OP_COUNT];
  int32_t* d_elem_nodes = nullptr;
  uint8_t* d_fixed = nullptr;
  double* d_Winv_qp = nullptr;
  double* d_detW_qp = nullptr;
  double* d_part = nullptr;   // 2 * kMaxRedBlocks (energy partials, reduction partials)
  double* d_res = nullptr;    // [0] F, [1] min det A, [2] dot result, [3..] Krylov state
  double* h_res = nullptr;    // pinned mirror
  double* d_vec = nullptr;    // Krylov / Newton vectors, allocated on first use
  int nvec = 0;
  void* d_pa = nullptr;       // packed per-point Hessians (partial assembly), allocated on first use
  bool pa_valid = false;      // d_pa holds the linearisation of some x
  bool pa_compact = false;    // ... as compact records (OP_LINEARIZE_C / OP_HESS_PA_C)
  double* d_eta2 = nullptr;   // per-point weights of the composite second term
  double delta = 0.0;         // restricted-movement weight (0: term off)
  double* d_x_init = nullptr; // its reference positions [d][nnode]
  mass_launch_fn mass[3] = {nullptr, nullptr, nullptr};
  int mass_grid = 1;
  double* d_diag = nullptr;   // Hessian diagonal [d][nnode] and its floored inverse [d][nnode]
  double* d_vdot = nullptr;   // per-warp partials of v . (H v) from the compact-record product
  float* d_kvec32 = nullptr;  // FP32 Krylov vectors of the FP32 forms (8 x ndof: 6 work, solution, Jacobi inverse)
  // two-level preconditioner (structured grids whose fixed dofs are exactly the boundary)
  bool boundary_fixed = false;
  int grid_n[3] = {0, 0, 0};
  CoarseSpace* coarse = nullptr;
  double* d_coarse_w = nullptr;  // [dim][coarse vertices], the smoothest coarse mode
  double coarse_alpha = 0.0;     // Rayleigh quotient of the last linearisation (0: coarse part off)
  // deterministic scatter: element colours (no two elements of a colour share
  // a node), launched one after another in colour order
  bool det = false;
  int ncolour = 0;
  int32_t* d_colour = nullptr;   // the elements of every colour, concatenated
  std::vector<int> colour_off, colour_cnt;
  cudaStream_t cap = nullptr; // internal stream for capturing Krylov iterations into a graph
  cudaEvent_t ev = nullptr;   // orders the internal stream after / before the caller's stream
};

namespace {

constexpr int kResKrylov = 8;
constexpr int kNumVec = 10;

#define CUDA_TRY(call)                              \
  do {                                              \
    cudaError_t e_ = (call);                        \
    if (e_ != cudaSuccess) return TMOP_ERR_CUDA;    \
  } while (0)

MassParams mass_params(const tmop_ctx* c) {
  MassParams mp;
  memset(&mp, 0, sizeof(mp));
  const KParams& b = c->base;
  mp.dim = b.dim; mp.nelem = b.nelem; mp.nnode = b.nnode;
  mp.sx = b.sx; mp.sy = b.sy; mp.sz = b.sz;
  mp.elem_nodes = b.elem_nodes;
  mp.fixed = b.fixed;
  mp.x0 = c->d_x_init;
  memcpy(mp.B, b.B, sizeof(mp.B));
  memcpy(mp.w1, b.w1, sizeof(mp.w1));
  mp.delta = c->delta;
  mp.detW = b.detW;
  mp.detW_qp = b.wkind == WK_PER_QP ? b.detW_qp : nullptr;
  mp.part = c->d_part + 2 * kMaxRedBlocks;
  return mp;
}

JacParams jac_params(const tmop_ctx* c, const double* x, double* J) {
  JacParams jp;
  memset(&jp, 0, sizeof(jp));
  const KParams& b = c->base;
  jp.dim = b.dim; jp.nelem = b.nelem; jp.nnode = b.nnode; jp.n = c->n; jp.q1 = c->nq;
  jp.sx = b.sx; jp.sy = b.sy; jp.sz = b.sz;
  jp.elem_nodes = b.elem_nodes;
  jp.x = x;
  jp.J = J;
  memcpy(jp.B, b.B, sizeof(jp.B));
  memcpy(jp.G, b.G, sizeof(jp.G));
  memcpy(jp.w1, b.w1, sizeof(jp.w1));
  return jp;
}

// The 3D FP32 recomputed Hessian action runs through compact records built in
// shared memory (OP_HESS_C) for the metrics and targets of the compact pair.
bool hess_c_ok(const tmop_ctx* c) {
  return c->ent[OP_HESS_C] && metric_is_lin(c->base.metric) && c->base.metric2 == 0 && c->base.wkind != WK_PER_QP;
}

// accumulate: y += the scatter op's result (y not zeroed first); v32, y32:
// FP32 direction and output of the stored-Hessian products instead of v, y
int launch_op(tmop_ctx* c, int op, const double* x, const double* v, double* y, double* elem_min,
              cudaStream_t s, double* vdot = nullptr, bool accumulate = false, const float* v32 = nullptr,
              float* y32 = nullptr) {
  if ((v32 || y32) && !(v32 && y32 && (op == OP_HESS_PA || (op == OP_HESS && hess_c_ok(c))) && c->delta == 0.0))
    return TMOP_ERR_ARG;
  KParams p = c->base;
  p.x = x;
  p.v = v;
  p.y = y;
  p.v32 = v32;
  p.y32 = y32;
  p.elem_min = elem_min;
  p.part_F = c->d_part;
  p.part_min = c->d_part + kMaxRedBlocks;
  p.pa = c->d_pa;
  if ((op == OP_GRADIENT || op == OP_HESS || op == OP_HESS_PA || op == OP_ENERGY_GRAD) && !accumulate) {
    if (y32) CUDA_TRY(cudaMemsetAsync(y32, 0, sizeof(float) * c->ndof, s));
    else CUDA_TRY(cudaMemsetAsync(y, 0, sizeof(double) * c->ndof, s));
  }
  int kop = op;  // the stored linearisation decides which form of the pair runs
  if (c->pa_compact && op == OP_LINEARIZE) kop = OP_LINEARIZE_C;
  if (c->pa_compact && op == OP_HESS_PA) kop = OP_HESS_PA_C;
  // the recomputed FP32 product through compact records built on the fly
  if (op == OP_HESS && hess_c_ok(c)) kop = OP_HESS_C;
  p.vdot = kop == OP_HESS_PA_C ? vdot : nullptr;
  const bool scatter = op == OP_GRADIENT || op == OP_HESS || op == OP_HESS_PA || op == OP_ENERGY_GRAD;
  // deterministic scatter: one launch per colour, in colour order
  const int passes = (c->det && scatter) ? c->ncolour : 1;
  for (int k = 0; k < passes; ++k) {
    if (c->det && scatter) {
      p.elist = c->d_colour + c->colour_off[k];
      p.ecount = c->colour_cnt[k];
    }
    if (c->ent[kop]->launch(p, c->grid[kop], s) != 0) return TMOP_ERR_CUDA;
  }
  if (c->delta != 0.0 && op != OP_ENERGY && op != OP_LINEARIZE) {
    // restricted movement (eq. (4.2)): its gradient (from x) or Hessian action (from v)
    MassParams mp = mass_params(c);
    mp.x = x;
    mp.v = v;
    mp.y = y;
    for (int k = 0; k < passes; ++k) {
      if (c->det) {
        mp.elist = c->d_colour + c->colour_off[k];
        mp.ecount = c->colour_cnt[k];
      }
      if (c->mass[op == OP_GRADIENT ? 1 : 2](mp, c->mass_grid, s) != 0) return TMOP_ERR_CUDA;
    }
  }
  return TMOP_OK;
}

// F and min det A into device memory (d_res[0..1] by default), asynchronously.
int energy_async(tmop_ctx* c, const double* x, cudaStream_t s, double* outF = nullptr, double* outMin = nullptr) {
  int rc = launch_op(c, OP_ENERGY, x, nullptr, nullptr, nullptr, s);
  if (rc) return rc;
  const double* extra = nullptr;
  if (c->delta != 0.0) {  // restricted movement: its own block partials of F
    MassParams mp = mass_params(c);
    mp.x = x;
    if (c->mass[0](mp, c->mass_grid, s) != 0) return TMOP_ERR_CUDA;
    extra = mp.part;
  }
  if (energy_final(c->d_part, c->d_part + kMaxRedBlocks, c->grid[OP_ENERGY], extra, c->mass_grid,
                   outF ? outF : c->d_res, outMin ? outMin : c->d_res + 1, s))
    return TMOP_ERR_CUDA;
  return TMOP_OK;
}

// The fused energy + gradient pass (one element pass instead of two): not in
// the deterministic mode (whose per-colour launches would each overwrite the
// energy partials) nor with the restricted-movement term (its own kernels).
bool fused_energy_grad(const tmop_ctx* c) { return c->ent[OP_ENERGY_GRAD] && !c->det && c->delta == 0.0; }

// g = dF/dx and (F, min det A) into device memory (d_res[0..1] by default),
// asynchronously: one fused pass, or the two separate ones.
int energy_grad_async(tmop_ctx* c, const double* x, double* g, cudaStream_t s, double* outF = nullptr,
                      double* outMin = nullptr) {
  if (!fused_energy_grad(c)) {
    int rc = energy_async(c, x, s, outF, outMin);
    if (rc) return rc;
    return launch_op(c, OP_GRADIENT, x, nullptr, g, nullptr, s);
  }
  int rc = launch_op(c, OP_ENERGY_GRAD, x, nullptr, g, nullptr, s);
  if (rc) return rc;
  if (energy_final(c->d_part, c->d_part + kMaxRedBlocks, c->grid[OP_ENERGY_GRAD], nullptr, 0,
                   outF ? outF : c->d_res, outMin ? outMin : c->d_res + 1, s))
    return TMOP_ERR_CUDA;
  return TMOP_OK;
}

int read_res(tmop_ctx* c, int first, int count, cudaStream_t s) {
  CUDA_TRY(cudaMemcpyAsync(c->h_res + first, c->d_res + first, sizeof(double) * count, cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  return TMOP_OK;
}

int energy_host(tmop_ctx* c, const double* x, double* F, double* mdet, cudaStream_t s) {
  int rc = energy_async(c, x, s);
  if (rc) return rc;
  rc = read_res(c, 0, 2, s);
  if (rc) return rc;
  *F = c->h_res[0];
  *mdet = c->h_res[1];
  return TMOP_OK;
}

int norm_host(tmop_ctx* c, const double* a, double* out, cudaStream_t s) {
  if (dot(a, a, c->ndof, c->d_part, c->d_res + 2, s)) return TMOP_ERR_CUDA;
  int rc = read_res(c, 2, 1, s);
  if (rc) return rc;
  *out = sqrt(c->h_res[2]);
  return TMOP_OK;
}

int ensure_vectors(tmop_ctx* c) {
  if (c->d_vec) return TMOP_OK;
  CUDA_TRY(cudaMalloc(&c->d_vec, sizeof(double) * c->ndof * kNumVec));
  c->nvec = kNumVec;
  return TMOP_OK;
}

double* vec(tmop_ctx* c, int i) { return c->d_vec + (size_t)i * c->ndof; }

// Store the per-point A-space Hessians of x (partial assembly): the 45 (3D)
// or 10 (2D) packed entries, or, for a 3D FP32 context with an (|T|^2, det T)
// metric, one constant target and no second term, the 14-value compact
// record the product rebuilds them from.
int linearize(tmop_ctx* c, const double* x, cudaStream_t s) {
  const int elt = c->precision == TMOP_FP64 ? (int)sizeof(double) : (int)sizeof(float);
  if (!c->d_pa) {  // sized for the packed form, which is never smaller than the compact one
    const size_t stride = (size_t)pa_stride_for(c->dim, c->Q, elt);
    CUDA_TRY(cudaMalloc(&c->d_pa, (size_t)elt * stride * (size_t)c->nelem));
  }
  c->pa_compact = c->ent[OP_LINEARIZE_C] && c->ent[OP_HESS_PA_C] && metric_is_lin(c->base.metric) &&
                  c->base.metric2 == 0 && c->base.wkind != WK_PER_QP;
  c->base.pa_stride = pa_stride_for(c->dim, c->Q, elt, c->pa_compact);
  c->pa_valid = false;
  int rc = launch_op(c, OP_LINEARIZE, x, nullptr, nullptr, nullptr, s);
  if (rc) return rc;
  c->pa_valid = true;
  return TMOP_OK;
}

// Vector slots
enum { V_G = 0, V_P, V_XT, V_GT, V_K0, V_K1, V_K2, V_K3, V_K4, V_K5 };

tmop_newton_opts defaults(const tmop_ctx* c, const tmop_newton_opts* in) {
  tmop_newton_opts o;
  memset(&o, 0, sizeof(o));
  if (in) o = *in;
  if (o.max_newton <= 0) o.max_newton = 10;
  if (!(o.rtol > 0.0)) o.rtol = 1e-12;
  if (o.krylov != TMOP_KRYLOV_CG) o.krylov = TMOP_KRYLOV_MINRES;
  if (!(o.krylov_rtol > 0.0)) o.krylov_rtol = (c->precision == TMOP_FP64) ? 1e-10 : 1e-6;
  if (o.krylov_maxit <= 0) o.krylov_maxit = 2000;
  if (!(o.alpha_shrink > 0.0 && o.alpha_shrink < 1.0)) o.alpha_shrink = 0.5;
  if (o.max_halvings <= 0) o.max_halvings = 30;
  if (!(o.f_factor > 0.0)) o.f_factor = 1.2;
  if (!(o.g_factor > 0.0)) o.g_factor = 1.2;
  if (!(o.atol > 0.0)) o.atol = 0.0;
  return o;
}

// Diagonal of the stored linearisation (+ the restricted-movement mass term),
// fixed dofs 1, into d_diag[0..ndof); with `inverse`, also the Jacobi
// inverse 1 / max(|diag|, 1e-8 rms|diag|) into d_diag[ndof..2 ndof).
int hessian_diagonal(tmop_ctx* c, bool inverse, cudaStream_t s) {
  if (!c->pa_valid) return TMOP_ERR_ARG;
  const int fp32 = c->precision != TMOP_FP64;
  diag_launch_fn f = find_diag(c->dim, c->n, c->nq, fp32);
  if (!f) return TMOP_ERR_ARG;
  if (!c->d_diag) CUDA_TRY(cudaMalloc(&c->d_diag, sizeof(double) * 2 * c->ndof));
  CUDA_TRY(cudaMemsetAsync(c->d_diag, 0, sizeof(double) * c->ndof, s));
  DiagParams dp;
  memset(&dp, 0, sizeof(dp));
  const KParams& b = c->base;
  dp.dim = b.dim; dp.nelem = b.nelem; dp.nnode = b.nnode; dp.sx = b.sx; dp.sy = b.sy; dp.sz = b.sz;
  dp.elem_nodes = b.elem_nodes;
  dp.pa = c->d_pa;
  dp.pa_stride = b.pa_stride;
  dp.diag = c->d_diag;
  memcpy(dp.B, b.B, sizeof(dp.B));
  memcpy(dp.G, b.G, sizeof(dp.G));
  memcpy(dp.w1, b.w1, sizeof(dp.w1));
  dp.delta = c->delta;
  dp.detW = b.detW;
  dp.detW_qp = b.wkind == WK_PER_QP ? b.detW_qp : nullptr;
  dp.compact = c->pa_compact ? 1 : 0;
  dp.identity = b.wkind == WK_IDENTITY ? 1 : 0;
  memcpy(dp.Winv, b.Winv, sizeof(dp.Winv));
  for (int k = 0; k < (c->det ? c->ncolour : 1); ++k) {
    if (c->det) {
      dp.elist = c->d_colour + c->colour_off[k];
      dp.ecount = c->colour_cnt[k];
    }
    if (f(dp, diag_grid(c->nelem), s) != 0) return TMOP_ERR_CUDA;
  }
  if (diag_finish(c->d_diag, b.fixed, c->ndof, s) != 0) return TMOP_ERR_CUDA;
  if (inverse) {
    double rms2;
    if (dot(c->d_diag, c->d_diag, c->ndof, c->d_part, c->d_res + 2, s)) return TMOP_ERR_CUDA;
    int rc = read_res(c, 2, 1, s);
    if (rc) return rc;
    rms2 = c->h_res[2] / (double)c->ndof;
    const double floor_abs = 1e-8 * sqrt(rms2) + 1e-300;
    if (diag_inverse(c->d_diag, c->d_diag + c->ndof, c->ndof, floor_abs, s) != 0) return TMOP_ERR_CUDA;
  }
  return TMOP_OK;
}

// The coarse part of the two-level preconditioner for the linearisation at
// x: the transfer and transform tables (once per context) and alpha, the
// Rayleigh quotient (P w)^t H (P w) / (w^t K_c w) of the smoothest coarse
// mode w in every component (one product with the Krylov operator). A
// Hessian that is not positive on that mode leaves the coarse part off
// (alpha = 0) for this solve.
int coarse_setup(tmop_ctx* c, const double* x, int hop, cudaStream_t s) {
  if (!c->coarse) {
    double z[kMaxN], zw[kMaxN];
    rule_gll(c->n, z, zw);
    c->coarse = coarse_create(c->dim, c->order, c->grid_n, z, c->precision != TMOP_FP64);
    if (!c->coarse) return TMOP_ERR_CUDA;
    CUDA_TRY(cudaMalloc(&c->d_coarse_w, sizeof(double) * c->dim * coarse_size(c->coarse)));
  }
  double lam0 = 0.0;
  double *w = vec(c, V_K0), *hw = vec(c, V_K1);
  if (coarse_mode0(c->coarse, c->d_coarse_w, &lam0, s) != 0) return TMOP_ERR_CUDA;
  if (coarse_prolong(c->coarse, c->d_coarse_w, w, s) != 0) return TMOP_ERR_CUDA;
  int rc = launch_op(c, hop, x, w, hw, nullptr, s);
  if (rc) return rc;
  if (dot(w, hw, c->ndof, c->d_part, c->d_res + 2, s)) return TMOP_ERR_CUDA;
  rc = read_res(c, 2, 1, s);
  if (rc) return rc;
  const double q = c->h_res[2] / (c->dim * lam0);
  c->coarse_alpha = (q > 0.0 && isfinite(q)) ? q : 0.0;
  coarse_set_alpha(c->coarse, c->coarse_alpha);
  return TMOP_OK;
}

// Krylov solve H(x) p = b; returns iterations (negative if the cap was hit).
// The Krylov solve of H p = b on T vectors (FP64, or FP32 for the FP32
// forms), after the linearisation and the preconditioner set-up.
template <class T>
int krylov_run(tmop_ctx* c, const double* x, const double* b, double* p, const tmop_newton_opts& o, int* iters,
               cudaStream_t s, int hop, const double* minv, const PrecondAdd* pc) {
  double* st = c->d_res + kResKrylov;
  double* part = c->d_part;
  const size_t n = c->ndof;
  // The device records convergence (KS_DONE, KS_CONV_IT) and freezes the
  // iterate from then on (also at the iteration cap), so the host reads the
  // state only every kCheck iterations: the result is the same as stopping at
  // the converged iteration. The kCheck iterations are captured once into a
  // CUDA graph on an internal stream and replayed (direct launches if capture
  // is not possible).
  // (6: plain MINRES renames its vectors with period 3 and 2, preconditioned
  // MINRES with period 2, so a batch of 6 iterations starts and ends with the
  // same assignment)
  constexpr int kCheck = 6;
  const bool cg = o.krylov == TMOP_KRYLOV_CG;
  if (cg && !std::is_same<T, double>::value) return TMOP_ERR_ARG;
  int rc = TMOP_OK;
  T *k0, *k1, *k2, *k3, *k4, *k5, *sol;
  const T* minvT = nullptr;
  if constexpr (std::is_same<T, double>::value) {
    k0 = vec(c, V_K0), k1 = vec(c, V_K1), k2 = vec(c, V_K2), k3 = vec(c, V_K3), k4 = vec(c, V_K4), k5 = vec(c, V_K5);
    sol = p;
    minvT = minv;
  } else {   // FP32 Krylov vectors: six work vectors, the solution, the FP32 Jacobi inverse
    if (!c->d_kvec32) CUDA_TRY(cudaMalloc(&c->d_kvec32, sizeof(float) * n * 8));
    float* b32 = c->d_kvec32;
    k0 = b32, k1 = b32 + n, k2 = b32 + 2 * n, k3 = b32 + 3 * n, k4 = b32 + 4 * n, k5 = b32 + 5 * n;
    sol = b32 + 6 * n;
    if (minv) {
      if (narrow(minv, b32 + 7 * n, n, s)) return TMOP_ERR_CUDA;
      minvT = b32 + 7 * n;
    }
  }
  // the product of the stored Hessians on T vectors, accumulating into a zeroed buffer
  auto product = [&](T* v, T* y, cudaStream_t q, double* vd) -> int {
    if constexpr (std::is_same<T, double>::value) return launch_op(c, hop, x, v, y, nullptr, q, vd, true);
    else return launch_op(c, hop, x, nullptr, nullptr, nullptr, q, vd, true, v, y);
  };
  if (cg) {
    if constexpr (std::is_same<T, double>::value)
      if (cg_init(b, k0, k1, p, st, part, n, o.krylov_rtol, o.krylov_maxit, s)) return TMOP_ERR_CUDA;
  } else if (minv) {  // r1 = k0, r2 = k1, u = k2 (product into q = k3), w = k4, wprev = k5
    if (pminres_init<T>(b, minvT, k0, k1, k2, k3, k4, k5, sol, st, part, n, o.krylov_rtol, o.krylov_maxit, s, pc))
      return TMOP_ERR_CUDA;
  } else {
    if (minres_init<T>(b, k0, k1, k2, k3, k4, sol, st, part, n, o.krylov_rtol, o.krylov_maxit, s))
      return TMOP_ERR_CUDA;
  }
  // the compact-record product also returns v . (H v) (not with the restricted-movement term, whose
  // contribution it does not see)
  double* vdot = nullptr;
  int vdot_np = 0;
  if (!cg && !minv && hop == OP_HESS_PA && c->pa_compact && c->delta == 0.0 && !c->det) {
    vdot_np = c->grid[OP_HESS_PA_C] * c->ent[OP_HESS_PA_C]->warps;
    if (!c->d_vdot) CUDA_TRY(cudaMalloc(&c->d_vdot, sizeof(double) * vdot_np));
    vdot = c->d_vdot;
  }
  auto enqueue_batch = [&](cudaStream_t q) -> int {
    for (int j = 0; j < kCheck; ++j) {
      int r;
      if (minv) {   // the pairs (r1, r2), (u, q), (w, wprev) swap roles every iteration
        const bool ev = j % 2 == 0;
        T *r1 = ev ? k0 : k1, *r2 = ev ? k1 : k0, *u = ev ? k2 : k3, *hu = ev ? k3 : k2;
        T *w = ev ? k4 : k5, *wp = ev ? k5 : k4;
        r = product(u, hu, q, nullptr);   // hu was left zero
        if (r) return r;
        if (pminres_after_hv<T>(minvT, r1, r2, u, hu, w, wp, sol, st, part, n, q, pc)) return TMOP_ERR_CUDA;
        continue;
      }
      if (cg) {  // r = k0, d = k1, Hd = k2
        if constexpr (std::is_same<T, double>::value) {
          r = launch_op(c, hop, x, k1, k2, nullptr, q);
          if (r) return r;
          if (cg_after_hv(p, k0, k1, k2, st, part, n, q)) return TMOP_ERR_CUDA;
        }
      } else {   // Lanczos vectors rotate over k0, k1, k2 (period 3), search directions over k3, k4
        T* V[3] = {k0, k1, k2};
        T* W[2] = {k3, k4};
        const int iv = (3 - j % 3) % 3;
        T *v = V[iv], *vprev = V[(iv + 1) % 3], *Av = V[(iv + 2) % 3];
        T *w = W[j % 2], *wp = W[(j + 1) % 2];
        r = product(v, Av, q, vdot);   // Av was left zero
        if (r) return r;
        if (minres_after_hv_rot<T>(v, vprev, Av, w, wp, sol, st, part, n, q, vdot, vdot_np)) return TMOP_ERR_CUDA;
      }
    }
    return TMOP_OK;
  };
  // try to capture one batch on the internal stream
  cudaGraphExec_t exec = nullptr;
  if (!c->cap) {
    if (cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking) != cudaSuccess) c->cap = nullptr;
    if (cudaEventCreateWithFlags(&c->ev, cudaEventDisableTiming) != cudaSuccess) c->ev = nullptr;
  }
  cudaStream_t q = s;
  if (c->cap && c->ev && cudaEventRecord(c->ev, s) == cudaSuccess && cudaStreamWaitEvent(c->cap, c->ev, 0) == cudaSuccess) {
    cudaGraph_t graph = nullptr;
    if (cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
      const int r = enqueue_batch(c->cap);
      const cudaError_t ec = cudaStreamEndCapture(c->cap, &graph);
      if (r == TMOP_OK && ec == cudaSuccess && graph &&
          cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess)
        exec = nullptr;
      if (graph) cudaGraphDestroy(graph);
    }
    cudaGetLastError();  // a failed capture leaves no sticky error; fall back below
    q = c->cap;
  }
  const double* h = c->h_res + kResKrylov;
  rc = read_res(c, kResKrylov, KS_COUNT, q);
  if (rc) { if (exec) cudaGraphExecDestroy(exec); return rc; }
  int enqueued = 0;
  while (h[KS_DONE] == 0.0 && enqueued < o.krylov_maxit) {
    if (exec) {
      if (cudaGraphLaunch(exec, q) != cudaSuccess) { cudaGraphExecDestroy(exec); return TMOP_ERR_CUDA; }
    } else {
      rc = enqueue_batch(q);
      if (rc) return rc;
    }
    enqueued += kCheck;
    rc = read_res(c, kResKrylov, KS_COUNT, q);
    if (rc) { if (exec) cudaGraphExecDestroy(exec); return rc; }
  }
  if (exec) cudaGraphExecDestroy(exec);
  if (q != s) {  // the caller's stream continues after the internal one
    if (cudaEventRecord(c->ev, q) != cudaSuccess || cudaStreamWaitEvent(s, c->ev, 0) != cudaSuccess)
      return TMOP_ERR_CUDA;
  }
  if constexpr (!std::is_same<T, double>::value)
    if (widen(sol, p, n, s)) return TMOP_ERR_CUDA;   // the Newton step in FP64
  const int it = h[KS_DONE] != 0.0 ? (int)h[KS_CONV_IT] : (int)h[KS_ITER];
  const bool converged = h[KS_DONE] != 0.0 && h[KS_BREAKDOWN] == 0.0 && h[KS_HITMAX] == 0.0;
  *iters = converged ? it : -it;
  return TMOP_OK;
}

int krylov(tmop_ctx* c, const double* x, const double* b, double* p, const tmop_newton_opts& o, int* iters,
           cudaStream_t s) {
  int rc = ensure_vectors(c);
  if (rc) return rc;
  // the Krylov operator: partially assembled at x (default) or recomputed from x
  const int hop = o.matrix_free ? OP_HESS : OP_HESS_PA;
  if (o.precond < 0 || o.precond > 2) return TMOP_ERR_ARG;
  if (o.precond && (hop != OP_HESS_PA || o.krylov == TMOP_KRYLOV_CG)) return TMOP_ERR_ARG;
  if (o.precond == 2 && !c->boundary_fixed) return TMOP_ERR_ARG;
  if (hop == OP_HESS_PA) {
    rc = linearize(c, x, s);
    if (rc) return rc;
  }
  const double* minv = nullptr;
  if (o.precond) {  // Jacobi: the diagonal of the linearisation just stored
    rc = hessian_diagonal(c, true, s);
    if (rc) return rc;
    minv = c->d_diag + c->ndof;
  }
  PrecondAdd pc_add{coarse_apply_add, coarse_apply_add32, nullptr};
  const PrecondAdd* pc = nullptr;
  if (o.precond == 2) {  // two-level: plus the coarse correction on the element vertices
    rc = coarse_setup(c, x, hop, s);
    if (rc) return rc;
    if (c->coarse_alpha > 0.0) {
      pc_add.obj = c->coarse;
      pc = &pc_add;
    }
  }
  // FP32 forms: MINRES on FP32 vectors (the operator is FP32 there), unless asked otherwise
  const bool cg = o.krylov == TMOP_KRYLOV_CG;
  const bool use32 = c->precision != TMOP_FP64 && !o.krylov_fp64 && (hop == OP_HESS_PA || hess_c_ok(c)) && !cg &&
                     c->delta == 0.0;
  if (use32) return krylov_run<float>(c, x, b, p, o, iters, s, hop, minv, pc);
  return krylov_run<double>(c, x, b, p, o, iters, s, hop, minv, pc);
}

struct NewtonState {
  double F, mdet, gnorm;
  // the current iterate and its gradient, and the buffers the line search
  // writes its trial into: an accepted trial swaps roles with the current
  // pair instead of being copied over it (x starts as the caller's array)
  double *x, *xt, *g, *gt;
};

// One Section 3.4 step from ns->x with cached F, det, g (ns->g) and |g|.
int newton_iter(tmop_ctx* c, const tmop_newton_opts& o, NewtonState* ns, tmop_newton_report* rep, cudaStream_t s) {
  double* p = vec(c, V_P);
  int kit = 0;
  int rc = krylov(c, ns->x, ns->g, p, o, &kit, s);
  if (rc) return rc;
  rep->krylov_iterations += kit < 0 ? -kit : kit;
  double alpha = 1.0;
  for (int h = 0; h <= o.max_halvings; ++h, alpha *= o.alpha_shrink) {
    if (step(ns->x, p, alpha, ns->xt, c->ndof, s)) return TMOP_ERR_CUDA;
    double Ft, mdt;
    // the trial's energy, and with the fused pass its gradient too (wasted
    // only when the trial is rejected)
    const bool fused = fused_energy_grad(c);
    rc = fused ? energy_grad_async(c, ns->xt, ns->gt, s) : energy_async(c, ns->xt, s);
    if (rc) return rc;
    rc = read_res(c, 0, 2, s);
    if (rc) return rc;
    Ft = c->h_res[0];
    mdt = c->h_res[1];
    // the new configuration must be valid (det A > 0 everywhere) and F may
    // grow by at most the f_factor
    if (!(mdt > 0.0) || !(Ft < o.f_factor * ns->F)) continue;
    if (!fused) {
      rc = launch_op(c, OP_GRADIENT, ns->xt, nullptr, ns->gt, nullptr, s);
      if (rc) return rc;
    }
    double gn;
    rc = norm_host(c, ns->gt, &gn, s);
    if (rc) return rc;
    if (!(gn < o.g_factor * ns->gnorm)) continue;
    std::swap(ns->x, ns->xt);
    std::swap(ns->g, ns->gt);
    ns->F = Ft;
    ns->mdet = mdt;
    ns->gnorm = gn;
    rep->alpha = alpha;
    return TMOP_OK;
  }
  rep->alpha = 0.0;
  return TMOP_ERR_LINESEARCH;
}

int newton_start(tmop_ctx* c, double* x, NewtonState* ns, cudaStream_t s) {
  int rc = ensure_vectors(c);
  if (rc) return rc;
  ns->x = x;
  ns->xt = vec(c, V_XT);
  ns->g = vec(c, V_G);
  ns->gt = vec(c, V_GT);
  rc = energy_grad_async(c, x, ns->g, s);
  if (rc) return rc;
  rc = read_res(c, 0, 2, s);
  if (rc) return rc;
  ns->F = c->h_res[0];
  ns->mdet = c->h_res[1];
  if (!(ns->mdet > 0.0)) return TMOP_ERR_INVERTED;
  return norm_host(c, ns->g, &ns->gnorm, s);
}

// The last accepted iterate into the caller's array (one copy, only when it
// sits in the context's buffer).
int newton_finish(tmop_ctx* c, double* x, const NewtonState& ns, cudaStream_t s) {
  if (ns.x && ns.x != x) CUDA_TRY(cudaMemcpyAsync(x, ns.x, sizeof(double) * c->ndof, cudaMemcpyDeviceToDevice, s));
  return TMOP_OK;
}

}  // namespace

extern "C" {

const char* tmop_status_string(int status) {
  switch (status) {
    case TMOP_OK: return "ok";
    case TMOP_ERR_ARG: return "invalid argument";
    case TMOP_ERR_CUDA: return "CUDA error";
    case TMOP_ERR_INVERTED: return "inverted element: det A <= 0 at some quadrature point";
    case TMOP_ERR_LINESEARCH: return "line search found no admissible step";
    case TMOP_ERR_NOT_CONVERGED: return "iteration limit reached";
    case TMOP_ERR_CAPACITY: return "problem too large for the fixed scratch buffer of the no-allocation entry point";
    default: return "unknown status";
  }
}

void tmop_destroy(tmop_ctx* c) {
  if (!c) return;
  cudaFree(c->d_elem_nodes);
  cudaFree(c->d_fixed);
  cudaFree(c->d_Winv_qp);
  cudaFree(c->d_detW_qp);
  cudaFree(c->d_part);
  cudaFree(c->d_res);
  cudaFree(c->d_vec);
  cudaFree(c->d_pa);
  cudaFree(c->d_eta2);
  cudaFree(c->d_x_init);
  cudaFree(c->d_diag);
  cudaFree(c->d_vdot);
  cudaFree(c->d_kvec32);
  cudaFree(c->d_colour);
  coarse_destroy(c->coarse);
  cudaFree(c->d_coarse_w);
  cudaFreeHost(c->h_res);
  if (c->cap) cudaStreamDestroy(c->cap);
  if (c->ev) cudaEventDestroy(c->ev);
  delete c;
}

int tmop_setup(const tmop_mesh* mesh, int order, const tmop_quad* quad, int metric_id, const tmop_targets* targets,
               int precision, tmop_ctx** out) {
  if (!out) return TMOP_ERR_ARG;
  *out = nullptr;
  if (!mesh || !quad || !targets) return TMOP_ERR_ARG;
  const int d = mesh->dim;
  if (d != 2 && d != 3) return TMOP_ERR_ARG;
  if (order < 1 || order > 4 || mesh->nelem < 1 || mesh->nnode < 1) return TMOP_ERR_ARG;
  if (quad->kind != TMOP_GL && quad->kind != TMOP_GLL) return TMOP_ERR_ARG;
  if (quad->npts1d < 2 || quad->npts1d > kMaxQ) return TMOP_ERR_ARG;
  if (precision != TMOP_FP64 && precision != TMOP_FP32_MIXED && precision != TMOP_FP32_BULK) return TMOP_ERR_ARG;
  const bool ok_metric = metric_supported(d, metric_id);
  if (!ok_metric) return TMOP_ERR_ARG;
  const int n = order + 1, nq = quad->npts1d;
  const int ndof_e = d == 2 ? n * n : n * n * n;
  const int Q = d == 2 ? nq * nq : nq * nq * nq;
  const ElemEntry* ent[OP_COUNT];
  for (int op = 0; op < OP_COUNT; ++op) {
    // FP32_MIXED: FP32 only for the Hessian action (and its partial assembly);
    // FP32_BULK: every element kernel
    const bool hess = op == OP_HESS || op == OP_LINEARIZE || op == OP_HESS_PA || op == OP_LINEARIZE_C ||
                      op == OP_HESS_PA_C || op == OP_HESS_C || op == OP_GRAD_HESS;
    const int fp32 = precision == TMOP_FP32_BULK || (precision == TMOP_FP32_MIXED && hess);
    ent[op] = find_elem(d, n, nq, fp32, op);
    // unsupported (order, points) pair; the compact pair exists for 3D FP32 only
    if (!ent[op] && op < OP_LINEARIZE_C) return TMOP_ERR_ARG;
  }
  // structured grid: sizes must match, and elem_nodes (if given) must agree
  const int* sd = mesh->structured;
  const bool structured = sd[0] > 0;
  // 2D: structured[2] > 1 stacks that many equal grids (nodes grid after grid)
  const int stack = (d == 2 && structured && sd[2] > 1) ? sd[2] : 1;
  if (structured) {
    long long ne = (long long)sd[0] * sd[1] * (d == 3 ? sd[2] : stack);
    long long nn = (long long)(order * sd[0] + 1) * (order * sd[1] + 1) * (d == 3 ? (order * sd[2] + 1) : stack);
    if (sd[1] < 1 || (d == 3 && sd[2] < 1) || ne != mesh->nelem || nn != mesh->nnode) return TMOP_ERR_ARG;
  } else if (!mesh->elem_nodes) {
    return TMOP_ERR_ARG;
  }
  if (mesh->elem_nodes) {
    const size_t cnt = (size_t)mesh->nelem * ndof_e;
    for (size_t i = 0; i < cnt; ++i)
      if (mesh->elem_nodes[i] < 0 || mesh->elem_nodes[i] >= mesh->nnode) return TMOP_ERR_ARG;
    if (structured) {
      const int Nx = order * sd[0] + 1, Ny = order * sd[1] + 1;
      for (int e = 0; e < mesh->nelem; ++e) {
        const int ex = e % sd[0], ey = (e / sd[0]) % sd[1], ez = e / (sd[0] * sd[1]);
        for (int t = 0; t < ndof_e; ++t) {
          const int i = t % n, j = (t / n) % n, l = d == 3 ? t / (n * n) : 0;
          const int g = (d == 3 ? ((ez * order + l) * Ny + ey * order + j) : (ez * Ny + ey * order + j)) * Nx +
                        ex * order + i;
          if (mesh->elem_nodes[(size_t)e * ndof_e + t] != g) return TMOP_ERR_ARG;
        }
      }
    }
  }

  tmop_ctx* c = new tmop_ctx();
  c->dim = d; c->order = order; c->n = n; c->nq = nq; c->Q = Q;
  c->nelem = mesh->nelem; c->nnode = mesh->nnode; c->metric = metric_id; c->precision = precision;
  c->ndof = (size_t)d * mesh->nnode;
  for (int op = 0; op < OP_COUNT; ++op) c->ent[op] = ent[op];
  KParams& p = c->base;
  memset(&p, 0, sizeof(p));
  p.dim = d; p.nelem = mesh->nelem; p.nnode = mesh->nnode; p.metric = metric_id;
  p.sx = structured ? sd[0] : 0; p.sy = structured ? sd[1] : 0;
  p.sz = structured ? (d == 3 ? sd[2] : (stack > 1 ? stack : 0)) : 0;

  // tables
  double qx[kMaxQ], qw[kMaxQ], z[kMaxN], zw[kMaxN];
  if (quad->kind == TMOP_GL) rule_gl(nq, qx, qw);
  else rule_gll(nq, qx, qw);
  rule_gll(n, z, zw);
  for (int a = 0; a < nq; ++a) {
    double phi[kMaxN], dphi[kMaxN];
    lagrange_bary(n, z, qx[a], phi, dphi);
    for (int i = 0; i < n; ++i) {
      p.B[a * n + i] = phi[i];
      p.G[a * n + i] = dphi[i];
    }
    p.w1[a] = qw[a];
  }

  // targets
  const int dd = d * d;
  int rc = TMOP_OK;
  double Wc[9] = {0};
  switch (targets->kind) {
    case TMOP_W_IDENTITY:
      for (int i = 0; i < d; ++i) Wc[i * d + i] = 1.0;
      p.wkind = WK_IDENTITY;
      break;
    case TMOP_W_SCALED:
      if (!(targets->scale > 0.0) || !isfinite(targets->scale)) rc = TMOP_ERR_ARG;
      for (int i = 0; i < d; ++i) Wc[i * d + i] = targets->scale;
      p.wkind = WK_CONST;
      break;
    case TMOP_W_CONST:
      if (!targets->W) rc = TMOP_ERR_ARG;
      else memcpy(Wc, targets->W, sizeof(double) * dd);
      p.wkind = WK_CONST;
      break;
    case TMOP_W_PER_QP:
      if (!targets->W) rc = TMOP_ERR_ARG;
      p.wkind = WK_PER_QP;
      for (int i = 0; i < d; ++i) Wc[i * d + i] = 1.0;
      break;
    default:
      rc = TMOP_ERR_ARG;
  }
  if (rc == TMOP_OK && !inv_h(d, Wc, p.Winv, &p.detW)) rc = TMOP_ERR_ARG;
  if (rc == TMOP_OK && p.wkind == WK_PER_QP) {
    const size_t cnt = (size_t)mesh->nelem * Q;
    std::vector<double> Wi(cnt * dd), dW(cnt);
    for (size_t k = 0; k < cnt && rc == TMOP_OK; ++k)
      if (!inv_h(d, targets->W + k * dd, &Wi[k * dd], &dW[k])) rc = TMOP_ERR_ARG;
    if (rc == TMOP_OK) {
      if (cudaMalloc(&c->d_Winv_qp, sizeof(double) * cnt * dd) != cudaSuccess ||
          cudaMalloc(&c->d_detW_qp, sizeof(double) * cnt) != cudaSuccess ||
          cudaMemcpy(c->d_Winv_qp, Wi.data(), sizeof(double) * cnt * dd, cudaMemcpyHostToDevice) != cudaSuccess ||
          cudaMemcpy(c->d_detW_qp, dW.data(), sizeof(double) * cnt, cudaMemcpyHostToDevice) != cudaSuccess)
        rc = TMOP_ERR_CUDA;
      p.Winv_qp = c->d_Winv_qp;
      p.detW_qp = c->d_detW_qp;
    }
  }
  // mesh arrays
  if (rc == TMOP_OK && !structured) {
    const size_t bytes = sizeof(int32_t) * (size_t)mesh->nelem * ndof_e;
    if (cudaMalloc(&c->d_elem_nodes, bytes) != cudaSuccess ||
        cudaMemcpy(c->d_elem_nodes, mesh->elem_nodes, bytes, cudaMemcpyHostToDevice) != cudaSuccess)
      rc = TMOP_ERR_CUDA;
    p.elem_nodes = c->d_elem_nodes;
  }
  if (rc == TMOP_OK && mesh->fixed) {
    if (cudaMalloc(&c->d_fixed, c->ndof) != cudaSuccess ||
        cudaMemcpy(c->d_fixed, mesh->fixed, c->ndof, cudaMemcpyHostToDevice) != cudaSuccess)
      rc = TMOP_ERR_CUDA;
    p.fixed = c->d_fixed;
  }
  // the two-level preconditioner's coarse space has the boundary fixed: record
  // whether the fixed dofs are exactly the boundary of a structured grid
  if (rc == TMOP_OK && structured && mesh->fixed) {
    const int Nx = order * sd[0] + 1, Ny = order * sd[1] + 1, Nz = d == 3 ? order * sd[2] + 1 : 1;
    bool ok = true;
    for (int comp = 0; comp < d && ok; ++comp)
      for (int node = 0; node < mesh->nnode && ok; ++node) {
        const int gx = node % Nx, gy = (node / Nx) % Ny, gz = node / (Nx * Ny);
        const bool bnd = gx == 0 || gx == Nx - 1 || gy == 0 || gy == Ny - 1 || (d == 3 && (gz == 0 || gz == Nz - 1));
        if ((mesh->fixed[(size_t)comp * mesh->nnode + node] != 0) != bnd) ok = false;
      }
    c->boundary_fixed = ok;
    for (int a = 0; a < d; ++a) c->grid_n[a] = sd[a];
    if (d == 2) c->grid_n[2] = stack;   // the coarse space of a 2D stack: one vertex grid per grid
  }
  // launch shapes and workspace
  for (int op = 0; op < OP_COUNT && rc == TMOP_OK; ++op) {
    if (!ent[op]) continue;
    if (ent[op]->prepare(mesh->nelem, &c->grid[op]) != 0) rc = TMOP_ERR_CUDA;
    else if (c->grid[op] > kMaxRedBlocks) c->grid[op] = kMaxRedBlocks;
  }
  if (rc == TMOP_OK) {
    if (cudaMalloc(&c->d_part, sizeof(double) * 3 * kMaxRedBlocks) != cudaSuccess ||
        cudaMalloc(&c->d_res, sizeof(double) * (kResKrylov + KS_COUNT)) != cudaSuccess ||
        cudaMemset(c->d_res, 0, sizeof(double) * (kResKrylov + KS_COUNT)) != cudaSuccess ||
        cudaMallocHost(&c->h_res, sizeof(double) * (kResKrylov + KS_COUNT)) != cudaSuccess)
      rc = TMOP_ERR_CUDA;
  }
  if (rc != TMOP_OK) {
    tmop_destroy(c);
    return rc;
  }
  *out = c;
  return TMOP_OK;
}

int tmop_set_composite(tmop_ctx* c, int metric2, const double* W2, const double* eta2) {
  if (!c) return TMOP_ERR_ARG;
  const int d = c->dim;
  if (metric2 == 0) {
    c->base.metric2 = 0;
    c->base.eta2 = nullptr;
    c->pa_valid = false;
    return TMOP_OK;
  }
  const bool ok_metric = metric_supported(d, metric2);
  if (!ok_metric || !W2) return TMOP_ERR_ARG;
  double Wi[9], det;
  if (!inv_h(d, W2, Wi, &det)) return TMOP_ERR_ARG;
  if (eta2) {
    const size_t cnt = (size_t)c->nelem * c->Q;
    for (size_t i = 0; i < cnt; ++i)
      if (!isfinite(eta2[i])) return TMOP_ERR_ARG;
    if (!c->d_eta2 && cudaMalloc(&c->d_eta2, sizeof(double) * cnt) != cudaSuccess) return TMOP_ERR_CUDA;
    if (cudaMemcpy(c->d_eta2, eta2, sizeof(double) * cnt, cudaMemcpyHostToDevice) != cudaSuccess)
      return TMOP_ERR_CUDA;
  }
  c->base.metric2 = metric2;
  memcpy(c->base.Winv2, Wi, sizeof(Wi));
  c->base.detW2 = det;
  c->base.eta2 = eta2 ? c->d_eta2 : nullptr;
  c->pa_valid = false;
  return TMOP_OK;
}

int tmop_set_deterministic(tmop_ctx* c, int on) {
  if (!c) return TMOP_ERR_ARG;
  if (!on) {
    c->det = false;
    return TMOP_OK;
  }
  if (c->d_colour) {
    c->det = true;
    return TMOP_OK;
  }
  const int ne = c->nelem, d = c->dim;
  std::vector<int> colour(ne, 0);
  int ncol = 0;
  if (c->base.sx > 0) {
    // structured grid: the parity of the element index along every axis;
    // elements of equal parities are at least one element apart
    const int sx = c->base.sx, sy = c->base.sy;
    for (int e = 0; e < ne; ++e) {
      const int ex = e % sx, ey = (e / sx) % sy, ez = e / (sx * sy);
      colour[e] = (ex & 1) | ((ey & 1) << 1) | (d == 3 ? ((ez & 1) << 2) : 0);
    }
    ncol = 1 << d;
  } else {
    // greedy: each element, in order, takes the smallest colour no element
    // sharing one of its nodes has taken
    const int nd = d == 2 ? c->n * c->n : c->n * c->n * c->n;
    std::vector<int32_t> en((size_t)ne * nd);
    if (cudaMemcpy(en.data(), c->d_elem_nodes, sizeof(int32_t) * en.size(), cudaMemcpyDeviceToHost) != cudaSuccess)
      return TMOP_ERR_CUDA;
    std::vector<int> start(c->nnode + 1, 0), list((size_t)ne * nd);
    for (size_t i = 0; i < en.size(); ++i) start[en[i] + 1]++;
    for (int i = 0; i < c->nnode; ++i) start[i + 1] += start[i];
    std::vector<int> fill(start.begin(), start.end() - 1);
    for (int e = 0; e < ne; ++e)
      for (int t = 0; t < nd; ++t) list[fill[en[(size_t)e * nd + t]]++] = e;
    std::vector<int> seen(64, -1);
    for (int e = 0; e < ne; ++e) {
      for (int t = 0; t < nd; ++t) {
        const int g = en[(size_t)e * nd + t];
        for (int j = start[g]; j < start[g + 1]; ++j)
          if (list[j] < e) seen[colour[list[j]]] = e;
      }
      int k = 0;
      while (k < 64 && seen[k] == e) ++k;
      if (k == 64) return TMOP_ERR_ARG;  // more than 64 colours: not a mesh this library targets
      colour[e] = k;
      if (k + 1 > ncol) ncol = k + 1;
    }
  }
  std::vector<int32_t> order;
  order.reserve(ne);
  c->colour_off.assign(ncol, 0);
  c->colour_cnt.assign(ncol, 0);
  for (int k = 0; k < ncol; ++k) {
    c->colour_off[k] = (int)order.size();
    for (int e = 0; e < ne; ++e)
      if (colour[e] == k) order.push_back(e);
    c->colour_cnt[k] = (int)order.size() - c->colour_off[k];
  }
  CUDA_TRY(cudaMalloc(&c->d_colour, sizeof(int32_t) * order.size()));
  CUDA_TRY(cudaMemcpy(c->d_colour, order.data(), sizeof(int32_t) * order.size(), cudaMemcpyHostToDevice));
  c->ncolour = ncol;
  c->det = true;
  return TMOP_OK;
}

int tmop_set_restricted_movement(tmop_ctx* c, double delta, const double* x_init, void* stream) {
  if (!c || !(delta >= 0.0) || !isfinite(delta) || (delta > 0.0 && !x_init)) return TMOP_ERR_ARG;
  if (delta == 0.0) {
    c->delta = 0.0;
    return TMOP_OK;
  }
  for (int mode = 0; mode < 3; ++mode) {
    c->mass[mode] = find_mass(c->dim, c->n, c->nq, mode);
    if (!c->mass[mode]) return TMOP_ERR_ARG;
  }
  if (!c->d_x_init) CUDA_TRY(cudaMalloc(&c->d_x_init, sizeof(double) * c->ndof));
  CUDA_TRY(cudaMemcpyAsync(c->d_x_init, x_init, sizeof(double) * c->ndof, cudaMemcpyDeviceToDevice,
                           (cudaStream_t)stream));
  c->mass_grid = mass_grid(c->nelem);
  if (c->mass_grid > kMaxRedBlocks) c->mass_grid = kMaxRedBlocks;
  c->delta = delta;
  return TMOP_OK;
}

int tmop_jacobians(tmop_ctx* c, const double* x, double* J, void* stream) {
  if (!c || !x || !J) return TMOP_ERR_ARG;
  JacParams jp = jac_params(c, x, J);
  return jacobians(jp, (cudaStream_t)stream) == 0 ? TMOP_OK : TMOP_ERR_CUDA;
}

int tmop_set_targets_from_positions(tmop_ctx* c, int kind, const double* x0, void* stream) {
  if (!c || !x0) return TMOP_ERR_ARG;
  if (kind != TMOP_WT_EQUAL_SIZE && kind != TMOP_WT_LOCAL_SIZE && kind != TMOP_WT_INITIAL) return TMOP_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const int d = c->dim, dd = d * d;
  const size_t cnt = (size_t)c->nelem * c->Q;
  double *J = nullptr, *Wi = nullptr, *dW = nullptr;
  int* bad = nullptr;
  int rc = TMOP_OK;
  if (cudaMalloc(&J, sizeof(double) * cnt * dd) != cudaSuccess) return TMOP_ERR_CUDA;
  JacParams jp = jac_params(c, x0, J);
  if (jacobians(jp, s) != 0) rc = TMOP_ERR_CUDA;
  if (rc == TMOP_OK && kind == TMOP_WT_EQUAL_SIZE) {
    // W2 = alpha^{1/d} I, alpha = (mesh measure) / N_E (eq. (3.1))
    if (mesh_measure(d, c->nq, J, (size_t)c->nelem, c->base.w1, c->d_res + 2, s) != 0) rc = TMOP_ERR_CUDA;
    if (rc == TMOP_OK) rc = read_res(c, 2, 1, s);
    const double alpha = rc == TMOP_OK ? c->h_res[2] / c->nelem : 0.0;
    if (rc == TMOP_OK && !(alpha > 0.0 && isfinite(alpha))) rc = TMOP_ERR_INVERTED;
    if (rc == TMOP_OK) {
      const double scale = d == 2 ? sqrt(alpha) : cbrt(alpha);
      for (int k = 0; k < 9; ++k) c->base.Winv[k] = 0.0;
      for (int a = 0; a < d; ++a) c->base.Winv[a * d + a] = 1.0 / scale;
      c->base.detW = alpha;
      c->base.wkind = WK_CONST;
      c->base.Winv_qp = nullptr;
      c->base.detW_qp = nullptr;
      cudaFree(c->d_Winv_qp);
      cudaFree(c->d_detW_qp);
      c->d_Winv_qp = c->d_detW_qp = nullptr;
    }
  } else if (rc == TMOP_OK) {
    // per point: W0 = A(x0) (Section 4.3.2) or W3 = det(A(x0))^{1/d} I (Section 3.1)
    if (cudaMalloc(&Wi, sizeof(double) * cnt * dd) != cudaSuccess || cudaMalloc(&dW, sizeof(double) * cnt) != cudaSuccess ||
        cudaMalloc(&bad, sizeof(int)) != cudaSuccess || cudaMemsetAsync(bad, 0, sizeof(int), s) != cudaSuccess)
      rc = TMOP_ERR_CUDA;
    if (rc == TMOP_OK &&
        targets_from_jacobians(d, kind == TMOP_WT_INITIAL ? 0 : 1, J, cnt, Wi, dW, bad, s) != 0)
      rc = TMOP_ERR_CUDA;
    int h_bad = 0;
    if (rc == TMOP_OK && (cudaMemcpyAsync(&h_bad, bad, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                          cudaStreamSynchronize(s) != cudaSuccess))
      rc = TMOP_ERR_CUDA;
    if (rc == TMOP_OK && h_bad > 0) rc = TMOP_ERR_INVERTED;
    if (rc == TMOP_OK) {
      cudaFree(c->d_Winv_qp);
      cudaFree(c->d_detW_qp);
      c->d_Winv_qp = Wi;
      c->d_detW_qp = dW;
      Wi = dW = nullptr;
      for (int k = 0; k < 9; ++k) c->base.Winv[k] = 0.0;
      for (int a = 0; a < d; ++a) c->base.Winv[a * d + a] = 1.0;
      c->base.detW = 1.0;
      c->base.wkind = WK_PER_QP;
      c->base.Winv_qp = c->d_Winv_qp;
      c->base.detW_qp = c->d_detW_qp;
    }
  }
  cudaStreamSynchronize(s);  // the temporaries are in use until here
  cudaFree(J);
  cudaFree(Wi);
  cudaFree(dW);
  cudaFree(bad);
  if (rc == TMOP_OK) c->pa_valid = false;
  return rc;
}

int tmop_sizes(const tmop_ctx* c, int* dim, int* nelem, int* nnode, int* Q) {
  if (!c) return TMOP_ERR_ARG;
  if (dim) *dim = c->dim;
  if (nelem) *nelem = c->nelem;
  if (nnode) *nnode = c->nnode;
  if (Q) *Q = c->Q;
  return TMOP_OK;
}

int tmop_energy(tmop_ctx* c, const double* x, double* F, double* min_detA, void* stream) {
  if (!c || !x || !F || !min_detA) return TMOP_ERR_ARG;
  double f, m;
  int rc = energy_host(c, x, &f, &m, (cudaStream_t)stream);
  if (rc) return rc;
  *F = f;
  *min_detA = m;
  return (m > 0.0) ? TMOP_OK : TMOP_ERR_INVERTED;
}

int tmop_energy_device(tmop_ctx* c, const double* x, double* F, double* min_detA, void* stream) {
  if (!c || !x || !F || !min_detA) return TMOP_ERR_ARG;
  return energy_async(c, x, (cudaStream_t)stream, F, min_detA);
}

int tmop_energy_gradient(tmop_ctx* c, const double* x, double* g, double* F, double* min_detA, void* stream) {
  if (!c || !x || !g || !F || !min_detA) return TMOP_ERR_ARG;
  return energy_grad_async(c, x, g, (cudaStream_t)stream, F, min_detA);
}

int tmop_gradient(tmop_ctx* c, const double* x, double* g, void* stream) {
  if (!c || !x || !g) return TMOP_ERR_ARG;
  return launch_op(c, OP_GRADIENT, x, nullptr, g, nullptr, (cudaStream_t)stream);
}

int tmop_hess_apply(tmop_ctx* c, const double* x, const double* v, double* y, void* stream) {
  if (!c || !x || !v || !y) return TMOP_ERR_ARG;
  return launch_op(c, OP_HESS, x, v, y, nullptr, (cudaStream_t)stream);
}

int tmop_gradient_hess_apply(tmop_ctx* c, const double* x, const double* v, double* g, double* y, void* stream) {
  // g and y are zeroed before x and v are read: no output may alias an input
  if (!c || !x || !v || !g || !y || g == y || g == x || g == v || y == x || y == v) return TMOP_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  // one element pass where the fused kernel covers the context (FP64, no
  // composite term, no restricted movement, atomic sums); else the two kernels
  if (!c->ent[OP_GRAD_HESS] || c->base.metric2 || c->delta != 0.0 || c->det) {
    const int rc = launch_op(c, OP_GRADIENT, x, nullptr, g, nullptr, s);
    return rc != TMOP_OK ? rc : launch_op(c, OP_HESS, x, v, y, nullptr, s);
  }
  KParams p = c->base;
  p.x = x;
  p.v = v;
  p.y = y;
  p.g = g;
  CUDA_TRY(cudaMemsetAsync(g, 0, sizeof(double) * c->ndof, s));
  CUDA_TRY(cudaMemsetAsync(y, 0, sizeof(double) * c->ndof, s));
  if (c->ent[OP_GRAD_HESS]->launch(p, c->grid[OP_GRAD_HESS], s) != 0) return TMOP_ERR_CUDA;
  return TMOP_OK;
}

int tmop_linearize(tmop_ctx* c, const double* x, void* stream) {
  if (!c || !x) return TMOP_ERR_ARG;
  return linearize(c, x, (cudaStream_t)stream);
}

int tmop_hess_apply_pa(tmop_ctx* c, const double* v, double* y, void* stream) {
  if (!c || !v || !y) return TMOP_ERR_ARG;
  if (!c->pa_valid) return TMOP_ERR_ARG;
  return launch_op(c, OP_HESS_PA, nullptr, v, y, nullptr, (cudaStream_t)stream);
}

int tmop_hess_apply_pa_add(tmop_ctx* c, const double* v, double* y, void* stream) {
  if (!c || !v || !y) return TMOP_ERR_ARG;
  if (!c->pa_valid) return TMOP_ERR_ARG;
  return launch_op(c, OP_HESS_PA, nullptr, v, y, nullptr, (cudaStream_t)stream, nullptr, true);
}

int tmop_hess_apply_pa_add_f32(tmop_ctx* c, const float* v, float* y, void* stream) {
  if (!c || !v || !y) return TMOP_ERR_ARG;
  if (!c->pa_valid || c->precision == TMOP_FP64 || c->delta != 0.0) return TMOP_ERR_ARG;
  return launch_op(c, OP_HESS_PA, nullptr, nullptr, nullptr, nullptr, (cudaStream_t)stream, nullptr, true, v, y);
}

int tmop_pa_layout(const tmop_ctx* c, int* values_per_point, int* stride, int* elt_bytes) {
  if (!c || !c->pa_valid) return TMOP_ERR_ARG;
  const int dd = c->dim * c->dim;
  if (values_per_point) *values_per_point = c->pa_compact ? kCompactRec : dd * (dd + 1) / 2;
  if (stride) *stride = c->base.pa_stride;
  if (elt_bytes) *elt_bytes = c->precision == TMOP_FP64 ? 8 : 4;
  return TMOP_OK;
}

int tmop_hessian_diagonal(tmop_ctx* c, double* out, void* stream) {
  if (!c || !out) return TMOP_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  int rc = hessian_diagonal(c, false, s);
  if (rc) return rc;
  CUDA_TRY(cudaMemcpyAsync(out, c->d_diag, sizeof(double) * c->ndof, cudaMemcpyDeviceToDevice, s));
  return TMOP_OK;
}

int tmop_element_min_detA(tmop_ctx* c, const double* x, double* out, void* stream) {
  if (!c || !x || !out) return TMOP_ERR_ARG;
  return launch_op(c, OP_ENERGY, x, nullptr, nullptr, out, (cudaStream_t)stream);
}

int tmop_precond_apply(tmop_ctx* c, const double* x, int precond, const double* r, double* z, double* alpha,
                       void* stream) {
  if (!c || !x || !r || !z || precond < 1 || precond > 2) return TMOP_ERR_ARG;
  if (precond == 2 && !c->boundary_fixed) return TMOP_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  int rc = ensure_vectors(c);
  if (!rc) rc = linearize(c, x, s);
  if (!rc) rc = hessian_diagonal(c, true, s);
  if (rc) return rc;
  double a = 0.0;
  if (precond == 2) {
    rc = coarse_setup(c, x, OP_HESS_PA, s);
    if (rc) return rc;
    a = c->coarse_alpha;
  }
  if (vec_mul(c->d_diag + c->ndof, r, z, c->ndof, s)) return TMOP_ERR_CUDA;
  if (a > 0.0 && coarse_apply_add(c->coarse, r, z, nullptr, s) < 0) return TMOP_ERR_CUDA;
  if (alpha) *alpha = a;
  CUDA_TRY(cudaStreamSynchronize(s));
  return TMOP_OK;
}

int tmop_krylov_solve(tmop_ctx* c, const double* x, const double* b, double* p, const tmop_newton_opts* opts,
                      int* iters, void* stream) {
  if (!c || !x || !b || !p || !iters) return TMOP_ERR_ARG;
  tmop_newton_opts o = defaults(c, opts);
  return krylov(c, x, b, p, o, iters, (cudaStream_t)stream);
}

int tmop_newton_step(tmop_ctx* c, double* x, const tmop_newton_opts* opts, tmop_newton_report* report,
                     void* stream) {
  if (!c || !x) return TMOP_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  tmop_newton_opts o = defaults(c, opts);
  tmop_newton_report rep;
  memset(&rep, 0, sizeof(rep));
  NewtonState ns = {0.0, 0.0, 0.0, nullptr, nullptr, nullptr, nullptr};
  int rc = newton_start(c, x, &ns, s);
  rep.grad_norm0 = (rc == TMOP_OK) ? ns.gnorm : 0.0;
  if (rc == TMOP_OK) {
    rc = newton_iter(c, o, &ns, &rep, s);
    rep.iterations = 1;
  }
  const int rf = newton_finish(c, x, ns, s);
  if (rc == TMOP_OK) rc = rf;
  rep.status = rc;
  rep.F = ns.F;
  rep.grad_norm = ns.gnorm;
  rep.min_detA = ns.mdet;
  if (report) *report = rep;
  return rc;
}

int tmop_newton_solve(tmop_ctx* c, double* x, const tmop_newton_opts* opts, tmop_newton_report* report,
                      void* stream) {
  if (!c || !x) return TMOP_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  tmop_newton_opts o = defaults(c, opts);
  tmop_newton_report rep;
  memset(&rep, 0, sizeof(rep));
  NewtonState ns = {0.0, 0.0, 0.0, nullptr, nullptr, nullptr, nullptr};
  int rc = newton_start(c, x, &ns, s);
  if (rc == TMOP_OK) {
    rep.grad_norm0 = ns.gnorm;
    rc = TMOP_ERR_NOT_CONVERGED;
    for (int it = 0; it < o.max_newton; ++it) {
      if (ns.gnorm <= o.rtol * rep.grad_norm0 || ns.gnorm <= o.atol) { rc = TMOP_OK; break; }
      int r = newton_iter(c, o, &ns, &rep, s);
      rep.iterations = it + 1;
      if (r != TMOP_OK) { rc = r; break; }
    }
    if (rc == TMOP_ERR_NOT_CONVERGED && (ns.gnorm <= o.rtol * rep.grad_norm0 || ns.gnorm <= o.atol)) rc = TMOP_OK;
  }
  const int rf = newton_finish(c, x, ns, s);
  if (rc == TMOP_OK) rc = rf;
  rep.status = rc;
  rep.F = ns.F;
  rep.grad_norm = ns.gnorm;
  rep.min_detA = ns.mdet;
  if (report) *report = rep;
  return rc;
}

}  // extern "C"
