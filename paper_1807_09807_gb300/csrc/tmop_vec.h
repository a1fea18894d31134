// Vector kernels (reductions, MINRES/CG steps, line-search updates). The
// MINRES vectors are FP64, or FP32 (T = float) for the Krylov solves of the
// FP32 forms; scalars and reductions are FP64 either way.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>

namespace tmop {

constexpr int kMaxRedBlocks = 2048;  // capacity of the per-block partial buffers

// Device scalar slots of the Krylov state (an array of doubles).
enum {
  KS_ALPHA = 0, KS_BETA, KS_BETA_NEXT2, KS_BETA_NEXT, KS_BETA1, KS_ETA, KS_C_OLD, KS_S_OLD, KS_C, KS_S,
  KS_R1, KS_R2, KS_INV_RHO, KS_PHI, KS_INV_BETA_NEXT, KS_RESID,
  KS_RR, KS_A, KS_B, KS_BREAKDOWN,
  KS_TOL,      // absolute residual target (rtol * |b|)
  KS_ITER,     // iterations executed on the device
  KS_DONE,     // 1 once the target is met (or a breakdown): later iterations change nothing
  KS_CONV_IT,  // the iteration at which KS_DONE was set
  KS_MAXIT,    // iteration cap: reaching it freezes the iterate (not converged)
  KS_HITMAX,   // 1 when KS_DONE was set by the cap
  // MINRES keeps its Lanczos vectors unnormalised: v = st[KS_SV] * (the v
  // array), vprev = st[KS_SVP] * (the vprev array), and the direction update
  // reads v at st[KS_SW] (the scale before the rotation)
  KS_SV, KS_SVP, KS_SW,
  // preconditioned MINRES
  KS_OLDB, KS_DBAR, KS_EPSLN, KS_OLDEPS, KS_PHIBAR, KS_CS, KS_SN, KS_DELTA, KS_INV_GAMMA, KS_INV_BETA,
  KS_INV_BETA_OLD, KS_WU, KS_WP, KS_WW,   // direction update coefficients of v (u), w_{k-2}, w_{k-1}
  KS_COUNT
};

int red_grid(size_t n);
int dot(const double* a, const double* b, size_t n, double* part, double* out, cudaStream_t s);
int energy_final(const double* pf, const double* pm, int np, const double* pf2, int np2, double* outF,
                 double* outMin, cudaStream_t s);
int step(const double* x, const double* p, double alpha, double* y, size_t n, cudaStream_t s);
// out = a * b elementwise
int vec_mul(const double* a, const double* b, double* out, size_t n, cudaStream_t s);
// (Av: the first product's output buffer, zeroed here; every later product
// accumulates into the buffer the Lanczos step of the previous iteration
// zeroed)
template <class T>
int minres_init(const double* b, T* v, T* vprev, T* Av, T* w, T* wprev, T* sol, double* st, double* part, size_t n,
                double rtol, int maxit, cudaStream_t s);
// one MINRES step after Av = H v, on rotating buffers: afterwards (v, vprev, Av) -> (Av, v, vprev),
// (w, wp) -> (wp, w);
// Av is the product of the stored v array (not of the scaled vector); vdot (vdot_np partials of
// v array . Av from the product kernel) replaces the dot-product pass when given. The new Lanczos
// vector is left in Av unnormalised, its scale in st[KS_SV]; vprev is zeroed (the next product
// accumulates into it).
template <class T>
int minres_after_hv_rot(const T* v, T* vprev, T* Av, const T* w, T* wp, T* sol, double* st, double* part, size_t n,
                        cudaStream_t s, const double* vdot = nullptr, int vdot_np = 0);
// Preconditioned MINRES (M^-1 = minv, a diagonal): r1, r2, y, v, w, wprev, sol
// An additive part of the preconditioner beside the diagonal minv: y += C r,
// with the per-block partials of r . (C r) written to part (at most
// kMaxRedBlocks of them; they are summed with the diagonal part's partials
// of r . (minv r)); apply returns the number of partials, or -1 on a launch
// error.
struct PrecondAdd {
  int (*apply)(void* obj, const double* r, double* y, double* part, cudaStream_t s);
  int (*apply32)(void* obj, const float* r, float* y, double* part, cudaStream_t s);   // FP32 vectors (or null)
  void* obj;
  int apply_t(void* o, const double* r, double* y, double* part, cudaStream_t s) const {
    return apply(o, r, y, part, s);
  }
  int apply_t(void* o, const float* r, float* y, double* part, cudaStream_t s) const {
    return apply32 ? apply32(o, r, y, part, s) : -1;
  }
};
// Preconditioned MINRES on rotating buffers. The Lanczos vector is kept
// unnormalised: u = beta v, and the product runs on u (q = H u). Per
// iteration: pminres_after_hv writes the new residual-direction vector into
// r1's buffer, the new u = M^-1 r into q's buffer and the new direction into
// wprev's buffer, so the caller then swaps (r1, r2), (u, q) and (w, wprev).
// Initially r1 = r2 = b, u = M^-1 b, q = w = wprev = sol = 0. The product
// accumulates into q: the direction pass zeroes u once it has read it, so
// the next iteration's q starts at zero.
template <class T>
int pminres_init(const double* b, const T* minv, T* r1, T* r2, T* u, T* q, T* w, T* wprev, T* sol, double* st,
                 double* part, size_t n, double rtol, int maxit, cudaStream_t s, const PrecondAdd* pc = nullptr);
// after the product q = H u
template <class T>
int pminres_after_hv(const T* minv, T* r1, const T* r2, T* u, T* q, const T* w, T* wprev, T* sol, double* st,
                     double* part, size_t n, cudaStream_t s, const PrecondAdd* pc = nullptr);
// FP32 <-> FP64 copies of a vector
int widen(const float* a, double* out, size_t n, cudaStream_t s);
int narrow(const double* a, float* out, size_t n, cudaStream_t s);
int cg_init(const double* b, double* r, double* d, double* sol, double* st, double* part, size_t n, double rtol,
            int maxit, cudaStream_t s);
int cg_after_hv(double* sol, double* r, double* d, const double* Hd, double* st, double* part, size_t n,
                cudaStream_t s);

}  // namespace tmop
