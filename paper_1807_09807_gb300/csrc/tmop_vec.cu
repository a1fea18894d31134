// FP64 vector kernels for the Krylov solvers and the Newton line search.
//
// Reductions are two-pass and deterministic: a fixed grid writes one
// partial per block (fixed per-block order), then one block sums the
// partials in index order. No atomics, no inter-block waiting.
//
// MINRES (Section 5 uses MINRES for the Newton systems): Lanczos on the
// symmetric Hessian with the residual minimised through Givens rotations;
// the scalar recurrences run on the device in a one-thread kernel, so a
// step needs no host round trip. CG is the SPD alternative.
#include <cuda_runtime.h>
#include <math.h>
#include <stddef.h>

#include "../../include/tmop.h"
#include "tmop_device.cuh"
#include "tmop_vec.h"

namespace tmop {

constexpr int kThreads = 256;

static int g_sms = 0;

int red_grid(size_t n) {
  if (g_sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_sms, cudaDevAttrMultiProcessorCount, dev);
    if (g_sms <= 0) g_sms = 1;
  }
  // up to 8 blocks of 256 threads per SM (full occupancy): the update kernels
  // stream 4 to 8 vectors, and more loads in flight keep HBM busier. A grid
  // of at least one block per SM is a whole number of blocks per SM, so every
  // SM streams the same share.
  size_t want = (n + kThreads * 4 - 1) / (kThreads * 4);
  size_t cap = (size_t)g_sms * 8;
  if (cap > (size_t)kMaxRedBlocks) cap = kMaxRedBlocks;
  if (want > cap) want = cap;
  if (want >= (size_t)g_sms) want -= want % (size_t)g_sms;
  if (want < 1) want = 1;
  return (int)want;
}

__device__ __forceinline__ double block_sum(double v) {
  __shared__ double red[kThreads / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < kThreads / 32; ++i) s += red[i];
  __syncthreads();
  return s;  // valid in thread 0
}

__global__ void k_dot_part(const double* __restrict__ a, const double* __restrict__ b, size_t n,
                           double* __restrict__ part) {
  double s = 0.0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    s = fma(a[i], b[i], s);
  s = block_sum(s);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// a . b over T vectors: each thread sums its elements in T (FP32 vectors:
// ~30 elements per thread at full occupancy), the blocks in FP64
template <class T>
__global__ void k_dot_part_t(const T* __restrict__ a, const T* __restrict__ b, size_t n, double* __restrict__ part) {
  T s = T(0);
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    s = fma(a[i], b[i], s);
  const double t = block_sum((double)s);
  if (threadIdx.x == 0) part[blockIdx.x] = t;
}

__global__ void k_sum_final(const double* __restrict__ part, int np, double* __restrict__ out) {
  double s = 0.0;
  for (int i = threadIdx.x; i < np; i += blockDim.x) s += part[i];
  s = block_sum(s);
  if (threadIdx.x == 0) *out = s;
}

__global__ void k_energy_final(const double* __restrict__ pf, const double* __restrict__ pm, int np,
                               const double* __restrict__ pf2, int np2, double* __restrict__ outF,
                               double* __restrict__ outMin) {
  __shared__ double mins[kThreads];
  double s = 0.0, m = INFINITY;
  for (int i = threadIdx.x; i < np; i += blockDim.x) {
    s += pf[i];
    m = fmin(m, pm[i]);
  }
  for (int i = threadIdx.x; i < np2; i += blockDim.x) s += pf2[i];  // extra terms of F (eq. (4.2))
  mins[threadIdx.x] = m;
  s = block_sum(s);
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int i = 1; i < kThreads; ++i) m = fmin(m, mins[i]);
    *outF = s;
    *outMin = m;
  }
}

__global__ void k_mul(const double* __restrict__ a, const double* __restrict__ b, double* __restrict__ out, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    out[i] = a[i] * b[i];
}

int vec_mul(const double* a, const double* b, double* out, size_t n, cudaStream_t s) {
  k_mul<<<red_grid(n), kThreads, 0, s>>>(a, b, out, n);
  return (int)cudaGetLastError();
}

int dot(const double* a, const double* b, size_t n, double* part, double* out, cudaStream_t s) {
  const int g = red_grid(n);
  k_dot_part<<<g, kThreads, 0, s>>>(a, b, n, part);
  k_sum_final<<<1, kThreads, 0, s>>>(part, g, out);
  return (int)cudaGetLastError();
}

int energy_final(const double* pf, const double* pm, int np, const double* pf2, int np2, double* outF,
                 double* outMin, cudaStream_t s) {
  k_energy_final<<<1, kThreads, 0, s>>>(pf, pm, np, pf2, pf2 ? np2 : 0, outF, outMin);
  return (int)cudaGetLastError();
}

// y = x - alpha * p (alpha on the host)
__global__ void k_step(const double* __restrict__ x, const double* __restrict__ p, double alpha,
                       double* __restrict__ y, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    y[i] = fma(-alpha, p[i], x[i]);
}

int step(const double* x, const double* p, double alpha, double* y, size_t n, cudaStream_t s) {
  k_step<<<red_grid(n), kThreads, 0, s>>>(x, p, alpha, y, n);
  return (int)cudaGetLastError();
}

// ---------------------------------------------------------------- MINRES
// v = b / beta1, vprev = w = wprev = sol = 0 and the rotation state. (The
// vectors are T: FP64, or FP32 for the FP32 forms' Krylov solves; b is the
// FP64 gradient.)
template <class T>
__global__ void k_minres_init(const double* __restrict__ b, T* v, T* vprev, T* Av, T* w, T* wprev, T* sol,
                              double* st, size_t n, double rtol, int maxit) {
  const double beta1 = sqrt(st[KS_BETA_NEXT2]);
  const double inv = beta1 > 0.0 ? 1.0 / beta1 : 0.0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    v[i] = (T)(b[i] * inv);
    vprev[i] = T(0);
    Av[i] = T(0);
    w[i] = T(0);
    wprev[i] = T(0);
    sol[i] = T(0);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    st[KS_BETA1] = beta1;
    st[KS_BETA] = beta1;
    st[KS_ETA] = beta1;
    st[KS_RESID] = beta1;
    st[KS_C_OLD] = 1.0; st[KS_S_OLD] = 0.0; st[KS_C] = 1.0; st[KS_S] = 0.0;
    st[KS_TOL] = rtol * beta1;
    st[KS_ITER] = 0.0;
    st[KS_DONE] = beta1 > 0.0 ? 0.0 : 1.0;
    st[KS_CONV_IT] = 0.0;
    st[KS_MAXIT] = (double)maxit;
    st[KS_HITMAX] = 0.0;
    st[KS_SV] = 1.0; st[KS_SVP] = 1.0; st[KS_SW] = 1.0;
  }
}

// The next Lanczos vector, unnormalised, over Av, with per-block partials of
// its squared norm. The arrays hold v / sv, vprev / svp and H (v / sv), so
// H v - alpha v - beta vprev = sv Av - (alpha sv) v - (beta svp) vprev, and
// alpha = v . H v = sv^2 (v array . Av) from the sum in st[KS_ALPHA]. vprev
// is read here for the last time and zeroed: it is the next product's output.
template <class T>
__global__ void k_lanczos(T* __restrict__ Av, const T* __restrict__ v, T* __restrict__ vprev,
                          const double* __restrict__ st, size_t n, double* __restrict__ part) {
  const double svd = st[KS_SV];
  const T sv = (T)svd, av = (T)(st[KS_ALPHA] * svd * svd * svd), bv = (T)(st[KS_BETA] * st[KS_SVP]);
  T s = T(0);
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const T r = fma(sv, Av[i], -av * v[i]) - bv * vprev[i];
    Av[i] = r;
    vprev[i] = T(0);
    s = fma(r, r, s);
  }
  const double t = block_sum((double)s);
  if (threadIdx.x == 0) part[blockIdx.x] = t;
}

// Apply the two previous rotations to the new tridiagonal column
// (beta_k, alpha_k, beta_{k+1}), form the new rotation, update eta.
__device__ void minres_scalar_step(double* st) {
  if (st[KS_DONE] == 0.0 && st[KS_ITER] >= st[KS_MAXIT]) {  // the cap: freeze, not converged
    st[KS_DONE] = 1.0;
    st[KS_HITMAX] = 1.0;
    st[KS_CONV_IT] = st[KS_ITER];
  }
  if (st[KS_DONE] != 0.0) {  // converged earlier: this iteration leaves the solution unchanged
    st[KS_PHI] = 0.0;
    st[KS_R1] = 0.0;
    st[KS_R2] = 0.0;
    st[KS_INV_RHO] = 0.0;
    st[KS_INV_BETA_NEXT] = 0.0;
    return;
  }
  st[KS_ITER] += 1.0;
  const double beta = st[KS_BETA], alpha = st[KS_ALPHA] * st[KS_SV] * st[KS_SV];
  const double beta_next = sqrt(fmax(st[KS_BETA_NEXT2], 0.0));
  const double c_old = st[KS_C_OLD], s_old = st[KS_S_OLD], c = st[KS_C], s = st[KS_S];
  const double r1 = s_old * beta;
  const double tmp = c_old * beta;
  const double r2 = c * tmp + s * alpha;
  const double r3 = -s * tmp + c * alpha;
  const double rho = hypot(r3, beta_next);
  const double c_new = rho > 0.0 ? r3 / rho : 1.0, s_new = rho > 0.0 ? beta_next / rho : 0.0;
  const double eta = st[KS_ETA];
  st[KS_R1] = r1;
  st[KS_R2] = r2;
  st[KS_INV_RHO] = rho > 0.0 ? 1.0 / rho : 0.0;
  st[KS_PHI] = c_new * eta;
  st[KS_ETA] = -s_new * eta;
  st[KS_RESID] = fabs(s_new * eta);
  st[KS_INV_BETA_NEXT] = beta_next > 0.0 ? 1.0 / beta_next : 0.0;
  st[KS_BETA_NEXT] = beta_next;
  st[KS_C_OLD] = c; st[KS_S_OLD] = s; st[KS_C] = c_new; st[KS_S] = s_new;
  st[KS_BETA] = beta_next;
  if (fabs(s_new * eta) <= st[KS_TOL] || beta_next == 0.0) {
    st[KS_DONE] = 1.0;
    st[KS_CONV_IT] = st[KS_ITER];
  }
}

// one block: |next Lanczos vector|^2 from the Lanczos step's per-block
// partials (the same sum as k_sum_final), then the scalar step in thread 0
__global__ void k_minres_scalar(const double* __restrict__ part, int np, double* st) {
  double sum = 0.0;
  for (int i = threadIdx.x; i < np; i += blockDim.x) sum += part[i];
  sum = block_sum(sum);
  if (threadIdx.x != 0) return;
  st[KS_BETA_NEXT2] = sum;
  minres_scalar_step(st);
  // scales of the unnormalised Lanczos vectors: the direction update takes v
  // at its present scale, then the arrays rotate and the next v is the new
  // Lanczos array times 1 / beta_next (0 once done)
  st[KS_SW] = st[KS_SV];
  st[KS_SVP] = st[KS_SV];
  st[KS_SV] = st[KS_INV_BETA_NEXT];
  // the direction update's coefficients of v, w_{k-2}, w_{k-1}, divided by rho
  // here once (all 0 once done: INV_RHO = 0)
  const double ir = st[KS_INV_RHO];
  st[KS_WU] = st[KS_SW] * ir;
  st[KS_WP] = st[KS_R1] * ir;
  st[KS_WW] = st[KS_R2] * ir;
}

// The direction/solution update and the next Lanczos vector follow in
// k_minres_vec_rot. (Once KS_DONE is set, phi = 0 keeps sol fixed and the
// next Lanczos vector is 0, so every later product is zero.)

template <class T>
int minres_init(const double* b, T* v, T* vprev, T* Av, T* w, T* wprev, T* sol, double* st, double* part, size_t n,
                double rtol, int maxit, cudaStream_t s) {
  int g = red_grid(n);
  k_dot_part<<<g, kThreads, 0, s>>>(b, b, n, part);
  k_sum_final<<<1, kThreads, 0, s>>>(part, g, st + KS_BETA_NEXT2);
  k_minres_init<T><<<g, kThreads, 0, s>>>(b, v, vprev, Av, w, wprev, sol, st, n, rtol, maxit);
  return (int)cudaGetLastError();
}
template int minres_init<double>(const double*, double*, double*, double*, double*, double*, double*, double*,
                                 double*, size_t, double, int, cudaStream_t);
template int minres_init<float>(const double*, float*, float*, float*, float*, float*, float*, double*, double*,
                                size_t, double, int, cudaStream_t);


// Rotating-buffer form of the update: the new search direction overwrites
// w_{k-2} (wp) and the Lanczos vectors stay unnormalised (their scales are
// device scalars), so nothing is copied or rescaled: 6 vector passes; the
// caller then renames (v, vprev, Av) -> (Av, v, vprev) and (w, wp) -> (wp, w).
template <class T>
__global__ void k_minres_vec_rot(const T* __restrict__ v, const T* __restrict__ w, T* __restrict__ wp,
                                 T* __restrict__ sol, const double* __restrict__ st, size_t n) {
  const T cu = (T)st[KS_WU], cp = (T)st[KS_WP], cw = (T)st[KS_WW], phi = (T)st[KS_PHI];
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const T wn = fma(-cw, w[i], fma(-cp, wp[i], v[i] * cu));   // (sw v - r1 w_{k-2} - r2 w_{k-1}) / rho
    wp[i] = wn;
    sol[i] = fma(phi, wn, sol[i]);
  }
}

template <class T>
int minres_after_hv_rot(const T* v, T* vprev, T* Av, const T* w, T* wp, T* sol, double* st, double* part, size_t n,
                        cudaStream_t s, const double* vdot, int vdot_np) {
  int g = red_grid(n);
  if (vdot) {  // alpha = v . (H v) from the product kernel's own partials
    k_sum_final<<<1, kThreads, 0, s>>>(vdot, vdot_np, st + KS_ALPHA);
  } else {
    k_dot_part_t<T><<<g, kThreads, 0, s>>>(v, Av, n, part);
    k_sum_final<<<1, kThreads, 0, s>>>(part, g, st + KS_ALPHA);
  }
  k_lanczos<T><<<g, kThreads, 0, s>>>(Av, v, vprev, st, n, part);
  k_minres_scalar<<<1, kThreads, 0, s>>>(part, g, st);
  k_minres_vec_rot<T><<<g, kThreads, 0, s>>>(v, w, wp, sol, st, n);
  return (int)cudaGetLastError();
}
template int minres_after_hv_rot<double>(const double*, double*, double*, const double*, double*, double*, double*,
                                         double*, size_t, cudaStream_t, const double*, int);
template int minres_after_hv_rot<float>(const float*, float*, float*, const float*, float*, float*, double*, double*,
                                        size_t, cudaStream_t, const double*, int);

// ---------------------------------------------------------------- preconditioned MINRES
// Lanczos in the M^-1 inner product with the residual minimised through
// Givens rotations (Paige and Saunders), M = diag(1 / minv). The residual
// estimate phibar is the M^-1-norm of the residual; the solve stops when it
// falls to rtol times its initial value.
template <class T>
__global__ void k_pm_init(const double* __restrict__ b, const T* __restrict__ minv, T* r1, T* r2, T* y, T* q, T* w,
                          T* wprev, T* sol, size_t n, double* __restrict__ part) {
  T s = T(0);
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const T bi = (T)b[i], yi = minv[i] * bi;
    r1[i] = bi;
    r2[i] = bi;
    y[i] = yi;
    q[i] = T(0);
    w[i] = T(0);
    wprev[i] = T(0);
    sol[i] = T(0);
    s = fma(bi, yi, s);
  }
  const double t = block_sum((double)s);
  if (threadIdx.x == 0) part[blockIdx.x] = t;
}

__global__ void k_pm_init_scalar(double* st, double rtol, int maxit) {
  const double beta1 = sqrt(fmax(st[KS_BETA_NEXT2], 0.0));
  st[KS_BETA1] = beta1;
  st[KS_BETA] = beta1;
  st[KS_OLDB] = 0.0;
  st[KS_DBAR] = 0.0;
  st[KS_EPSLN] = 0.0;
  st[KS_OLDEPS] = 0.0;
  st[KS_PHIBAR] = beta1;
  st[KS_RESID] = beta1;
  st[KS_CS] = -1.0;
  st[KS_SN] = 0.0;
  st[KS_DELTA] = 0.0;
  st[KS_INV_GAMMA] = 0.0;
  st[KS_PHI] = 0.0;
  st[KS_INV_BETA] = beta1 > 0.0 ? 1.0 / beta1 : 0.0;
  st[KS_TOL] = rtol * beta1;
  st[KS_ITER] = 0.0;
  st[KS_DONE] = beta1 > 0.0 ? 0.0 : 1.0;
  st[KS_CONV_IT] = 0.0;
  st[KS_MAXIT] = (double)maxit;
  st[KS_HITMAX] = 0.0;
  st[KS_BREAKDOWN] = 0.0;
}

// q <- q / beta - (beta / oldb) r1 (the r1 term from the second iteration
// on), partials of u . q (alpha = their sum / beta)
template <class T>
__global__ void k_pm_a(T* __restrict__ q, const T* __restrict__ r1, const T* __restrict__ u,
                       const double* __restrict__ st, size_t n, double* __restrict__ part) {
  const double oldb = st[KS_OLDB];
  const T ib = (T)st[KS_INV_BETA];
  const T c = (T)(oldb > 0.0 ? st[KS_BETA] / oldb : 0.0);
  T s = T(0);
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const T qi = fma(-c, r1[i], q[i] * ib);
    q[i] = qi;
    s = fma(u[i], qi, s);
  }
  const double t = block_sum((double)s);
  if (threadIdx.x == 0) part[blockIdx.x] = t;
}

// out = (sum of the partials) * *scale
__global__ void k_sum_scaled(const double* __restrict__ part, int np, const double* __restrict__ scale,
                             double* __restrict__ out) {
  double s = 0.0;
  for (int i = threadIdx.x; i < np; i += blockDim.x) s += part[i];
  s = block_sum(s);
  if (threadIdx.x == 0) *out = s * *scale;
}

// t = q - (alpha / beta) r2 into r1's buffer (the old r1 is dead), then
// q <- M^-1 t (diagonal part); partials of t . q
template <class T>
__global__ void k_pm_b(const T* __restrict__ minv, T* __restrict__ r1, const T* __restrict__ r2, T* __restrict__ q,
                       const double* __restrict__ st, size_t n, double* __restrict__ part) {
  const double beta = st[KS_BETA];
  const T c = (T)(beta > 0.0 ? st[KS_ALPHA] / beta : 0.0);
  T s = T(0);
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const T t = fma(-c, r2[i], q[i]);
    r1[i] = t;
    const T yi = minv[i] * t;
    q[i] = yi;
    s = fma(t, yi, s);
  }
  const double tt = block_sum((double)s);
  if (threadIdx.x == 0) part[blockIdx.x] = tt;
}

__global__ void k_pm_scalar(double* st) {
  if (st[KS_DONE] == 0.0 && st[KS_ITER] >= st[KS_MAXIT]) {
    st[KS_DONE] = 1.0;
    st[KS_HITMAX] = 1.0;
    st[KS_CONV_IT] = st[KS_ITER];
  }
  if (st[KS_DONE] != 0.0) {  // frozen: later iterations leave the solution unchanged
    st[KS_PHI] = 0.0;
    st[KS_INV_GAMMA] = 0.0;
    st[KS_OLDEPS] = 0.0;
    st[KS_DELTA] = 0.0;
    st[KS_INV_BETA] = 0.0;
    return;
  }
  st[KS_INV_BETA_OLD] = st[KS_INV_BETA];   // the direction update reads this iteration's v = u / beta
  st[KS_ITER] += 1.0;
  const double alpha = st[KS_ALPHA];
  const double beta = sqrt(fmax(st[KS_BETA_NEXT2], 0.0));
  st[KS_OLDB] = st[KS_BETA];
  st[KS_BETA] = beta;
  const double cs = st[KS_CS], sn = st[KS_SN], dbar = st[KS_DBAR];
  st[KS_OLDEPS] = st[KS_EPSLN];
  st[KS_DELTA] = cs * dbar + sn * alpha;
  const double gbar = sn * dbar - cs * alpha;
  st[KS_EPSLN] = sn * beta;
  st[KS_DBAR] = -cs * beta;
  double gamma = hypot(gbar, beta);
  if (!(gamma > 0.0)) gamma = 1e-300;
  const double cs_new = gbar / gamma, sn_new = beta / gamma;
  st[KS_CS] = cs_new;
  st[KS_SN] = sn_new;
  const double phibar = st[KS_PHIBAR];
  st[KS_PHI] = cs_new * phibar;
  st[KS_PHIBAR] = sn_new * phibar;
  st[KS_RESID] = fabs(sn_new * phibar);
  st[KS_INV_GAMMA] = 1.0 / gamma;
  st[KS_WU] = st[KS_INV_BETA_OLD] / gamma;
  st[KS_WP] = st[KS_OLDEPS] / gamma;
  st[KS_WW] = st[KS_DELTA] / gamma;
  st[KS_INV_BETA] = beta > 0.0 ? 1.0 / beta : 0.0;
  if (fabs(sn_new * phibar) <= st[KS_TOL] || beta == 0.0) {
    st[KS_DONE] = 1.0;
    st[KS_CONV_IT] = st[KS_ITER];
  }
}

// w_k = (v - oldeps w_{k-2} - delta w_{k-1}) / gamma with v = u / beta
// (the three coefficients divided by gamma beforehand), written over
// w_{k-2}; x += phi w_k. u is read here for the last time and zeroed: it is
// the next product's output (also once frozen, so that the frozen
// iterations' products stay bounded).
template <class T>
__global__ void k_pm_w(T* __restrict__ u, const T* __restrict__ w, T* __restrict__ wprev, T* __restrict__ sol,
                       const double* __restrict__ st, size_t n) {
  const double igd = st[KS_INV_GAMMA], phid = st[KS_PHI];
  const T phi = (T)phid, cu = (T)st[KS_WU], cp = (T)st[KS_WP], cw = (T)st[KS_WW];
  const bool frozen = phid == 0.0 && igd == 0.0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    if (!frozen) {
      const T wn = fma(-cw, w[i], fma(-cp, wprev[i], u[i] * cu));
      wprev[i] = wn;
      sol[i] = fma(phi, wn, sol[i]);
    }
    u[i] = T(0);
  }
}

template <class T>
int pminres_init(const double* b, const T* minv, T* r1, T* r2, T* u, T* q, T* w, T* wprev, T* sol, double* st,
                 double* part, size_t n, double rtol, int maxit, cudaStream_t s, const PrecondAdd* pc) {
  int g = red_grid(n);
  k_pm_init<T><<<g, kThreads, 0, s>>>(b, minv, r1, r2, u, q, w, wprev, sol, n, part);
  if (pc) {   // u += C b, and the partials of b . C b after the diagonal part's
    // (the FP32 form passes its FP32 copy of b, r1 after the initialisation)
    const int np = pc->apply_t(pc->obj, r1, u, part + g, s);
    if (np < 0) return (int)cudaErrorLaunchFailure;
    g += np;
  }
  k_sum_final<<<1, kThreads, 0, s>>>(part, g, st + KS_BETA_NEXT2);
  k_pm_init_scalar<<<1, 1, 0, s>>>(st, rtol, maxit);
  return (int)cudaGetLastError();
}

template <class T>
int pminres_after_hv(const T* minv, T* r1, const T* r2, T* u, T* q, const T* w, T* wprev, T* sol, double* st,
                     double* part, size_t n, cudaStream_t s, const PrecondAdd* pc) {
  const int g = red_grid(n);
  k_pm_a<T><<<g, kThreads, 0, s>>>(q, r1, u, st, n, part);
  k_sum_scaled<<<1, kThreads, 0, s>>>(part, g, st + KS_INV_BETA, st + KS_ALPHA);
  int g2 = g;
  k_pm_b<T><<<g, kThreads, 0, s>>>(minv, r1, r2, q, st, n, part);
  if (pc) {   // q += C t (t now in r1's buffer), and the partials of t . C t after the diagonal part's
    const int np = pc->apply_t(pc->obj, r1, q, part + g, s);
    if (np < 0) return (int)cudaErrorLaunchFailure;
    g2 += np;
  }
  k_sum_final<<<1, kThreads, 0, s>>>(part, g2, st + KS_BETA_NEXT2);
  k_pm_scalar<<<1, 1, 0, s>>>(st);
  k_pm_w<T><<<g, kThreads, 0, s>>>(u, w, wprev, sol, st, n);
  return (int)cudaGetLastError();
}

#define TMOP_PMINRES(T)                                                                                        \
  template int pminres_init<T>(const double*, const T*, T*, T*, T*, T*, T*, T*, T*, double*, double*, size_t, \
                               double, int, cudaStream_t, const PrecondAdd*);                                 \
  template int pminres_after_hv<T>(const T*, T*, const T*, T*, T*, const T*, T*, T*, double*, double*, size_t, \
                                   cudaStream_t, const PrecondAdd*);
TMOP_PMINRES(double)
TMOP_PMINRES(float)
#undef TMOP_PMINRES

// sol (FP32) -> p (FP64)
__global__ void k_widen(const float* __restrict__ a, double* __restrict__ out, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    out[i] = (double)a[i];
}
// out = FP32 copy of a
__global__ void k_narrow(const double* __restrict__ a, float* __restrict__ out, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    out[i] = (float)a[i];
}
int widen(const float* a, double* out, size_t n, cudaStream_t s) {
  k_widen<<<red_grid(n), kThreads, 0, s>>>(a, out, n);
  return (int)cudaGetLastError();
}
int narrow(const double* a, float* out, size_t n, cudaStream_t s) {
  k_narrow<<<red_grid(n), kThreads, 0, s>>>(a, out, n);
  return (int)cudaGetLastError();
}

// ---------------------------------------------------------------- CG
__global__ void k_cg_init(const double* __restrict__ b, double* r, double* d, double* sol, double* st, size_t n,
                          double rtol, int maxit) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    r[i] = b[i];
    d[i] = b[i];
    sol[i] = 0.0;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    st[KS_RR] = st[KS_BETA_NEXT2];
    st[KS_BETA1] = sqrt(st[KS_BETA_NEXT2]);
    st[KS_RESID] = st[KS_BETA1];
    st[KS_BREAKDOWN] = 0.0;
    st[KS_TOL] = rtol * st[KS_BETA1];
    st[KS_ITER] = 0.0;
    st[KS_DONE] = st[KS_BETA1] > 0.0 ? 0.0 : 1.0;
    st[KS_CONV_IT] = 0.0;
    st[KS_MAXIT] = (double)maxit;
    st[KS_HITMAX] = 0.0;
  }
}

__global__ void k_cg_a(double* st) {
  const double dHd = st[KS_ALPHA];
  if (st[KS_DONE] == 0.0 && st[KS_ITER] >= st[KS_MAXIT]) {  // the cap: freeze, not converged
    st[KS_DONE] = 1.0;
    st[KS_HITMAX] = 1.0;
    st[KS_CONV_IT] = st[KS_ITER];
  }
  if (st[KS_DONE] != 0.0) {  // converged or broken down earlier: no further update
    st[KS_A] = 0.0;
    return;
  }
  st[KS_ITER] += 1.0;
  if (!(dHd > 0.0)) {
    st[KS_DONE] = 1.0;
    st[KS_CONV_IT] = st[KS_ITER];
    st[KS_BREAKDOWN] = 1.0;
    st[KS_A] = 0.0;
  } else {
    st[KS_A] = st[KS_RR] / dHd;
  }
}

__global__ void k_cg_update(double* __restrict__ sol, double* __restrict__ r, const double* __restrict__ d,
                            const double* __restrict__ Hd, const double* __restrict__ st, size_t n,
                            double* __restrict__ part) {
  const double a = st[KS_A];
  double s = 0.0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    sol[i] = fma(a, d[i], sol[i]);
    const double ri = fma(-a, Hd[i], r[i]);
    r[i] = ri;
    s = fma(ri, ri, s);
  }
  s = block_sum(s);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__global__ void k_cg_b(double* st) {
  if (st[KS_DONE] != 0.0) {
    st[KS_B] = 0.0;
    return;
  }
  const double rr_new = st[KS_BETA_NEXT2];
  st[KS_B] = st[KS_RR] > 0.0 ? rr_new / st[KS_RR] : 0.0;
  st[KS_RR] = rr_new;
  st[KS_RESID] = sqrt(fmax(rr_new, 0.0));
  if (st[KS_RESID] <= st[KS_TOL]) {
    st[KS_DONE] = 1.0;
    st[KS_CONV_IT] = st[KS_ITER];
  }
}

__global__ void k_cg_dir(double* __restrict__ d, const double* __restrict__ r, const double* __restrict__ st,
                         size_t n) {
  const double b = st[KS_B];
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    d[i] = fma(b, d[i], r[i]);
}

int cg_init(const double* b, double* r, double* d, double* sol, double* st, double* part, size_t n, double rtol,
            int maxit, cudaStream_t s) {
  int g = red_grid(n);
  k_dot_part<<<g, kThreads, 0, s>>>(b, b, n, part);
  k_sum_final<<<1, kThreads, 0, s>>>(part, g, st + KS_BETA_NEXT2);
  k_cg_init<<<g, kThreads, 0, s>>>(b, r, d, sol, st, n, rtol, maxit);
  return (int)cudaGetLastError();
}

int cg_after_hv(double* sol, double* r, double* d, const double* Hd, double* st, double* part, size_t n,
                cudaStream_t s) {
  int g = red_grid(n);
  k_dot_part<<<g, kThreads, 0, s>>>(d, Hd, n, part);
  k_sum_final<<<1, kThreads, 0, s>>>(part, g, st + KS_ALPHA);
  k_cg_a<<<1, 1, 0, s>>>(st);
  k_cg_update<<<g, kThreads, 0, s>>>(sol, r, d, Hd, st, n, part);
  k_sum_final<<<1, kThreads, 0, s>>>(part, g, st + KS_BETA_NEXT2);
  k_cg_b<<<1, 1, 0, s>>>(st);
  k_cg_dir<<<g, kThreads, 0, s>>>(d, r, st, n);
  return (int)cudaGetLastError();
}

}  // namespace tmop

namespace {
__global__ void k_selftest_convert(const double* __restrict__ in, float* __restrict__ f32, double* __restrict__ back,
                                   size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const float f = tmop::f64_to_f32(in[i]);
    f32[i] = f;
    back[i] = tmop::f32_to_f64(f);
  }
}
}  // namespace

namespace {
__global__ void k_selftest_rcbrt(const double* __restrict__ in, double* __restrict__ out, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    out[i] = tmop::rcbrt_(in[i]);
}
}  // namespace

namespace tmop {
__global__ void k_add(double* __restrict__ y, const double* __restrict__ b, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    y[i] += b[i];
}

__global__ void k_axpby(double* __restrict__ y, double a, const double* __restrict__ x, double b, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    y[i] = b == 0.0 ? a * x[i] : fma(a, x[i], b * y[i]);
}

// partials of sum_c sum_{i < count} a[c stride + first + i] b[...]
__global__ void k_dot_seg(const double* __restrict__ a, const double* __restrict__ b, int ncomp, size_t stride,
                          size_t first, size_t count, double* __restrict__ part) {
  double s = 0.0;
  const size_t n = (size_t)ncomp * count;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
    const size_t i = (t / count) * stride + first + t % count;
    s = fma(a[i], b[i], s);
  }
  s = block_sum(s);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

}  // namespace tmop

extern "C" int tmop_vec_add(double* y, const double* b, size_t n, void* stream) {
  using namespace tmop;
  if (n == 0) return TMOP_OK;
  if (!y || !b) return TMOP_ERR_ARG;
  k_add<<<red_grid(n), kThreads, 0, (cudaStream_t)stream>>>(y, b, n);
  return cudaGetLastError() == cudaSuccess ? TMOP_OK : TMOP_ERR_CUDA;
}

extern "C" int tmop_vec_axpby(double* y, double a, const double* x, double b, size_t n, void* stream) {
  using namespace tmop;
  if (n == 0) return TMOP_OK;
  if (!y || !x) return TMOP_ERR_ARG;
  k_axpby<<<red_grid(n), kThreads, 0, (cudaStream_t)stream>>>(y, a, x, b, n);
  return cudaGetLastError() == cudaSuccess ? TMOP_OK : TMOP_ERR_CUDA;
}

extern "C" int tmop_vec_dot_segments(const double* a, const double* b, int ncomp, size_t stride, size_t first,
                                     size_t count, double* scratch, size_t scratch_len, double* out, void* stream) {
  using namespace tmop;
  if (!a || !b || !scratch || !out || ncomp < 1 || first + count > stride) return TMOP_ERR_ARG;
  const size_t n = (size_t)ncomp * count;
  const int g = red_grid(n > 0 ? n : 1);
  if (scratch_len < (size_t)g) return TMOP_ERR_CAPACITY;
  cudaStream_t s = (cudaStream_t)stream;
  k_dot_seg<<<g, kThreads, 0, s>>>(a, b, ncomp, stride, first, count, scratch);
  k_sum_final<<<1, kThreads, 0, s>>>(scratch, g, out);
  return cudaGetLastError() == cudaSuccess ? TMOP_OK : TMOP_ERR_CUDA;
}

extern "C" int tmop_selftest_rcbrt(const double* in, double* out, size_t n, void* stream) {
  if (n == 0) return TMOP_OK;
  if (!in || !out) return TMOP_ERR_ARG;
  k_selftest_rcbrt<<<256, 256, 0, (cudaStream_t)stream>>>(in, out, n);
  return cudaGetLastError() == cudaSuccess ? TMOP_OK : TMOP_ERR_CUDA;
}

extern "C" int tmop_selftest_convert(const double* in, float* f32, double* back, size_t n, void* stream) {
  if (n == 0) return TMOP_OK;
  if (!in || !f32 || !back) return TMOP_ERR_ARG;
  k_selftest_convert<<<256, 256, 0, (cudaStream_t)stream>>>(in, f32, back, n);
  return cudaGetLastError() == cudaSuccess ? TMOP_OK : TMOP_ERR_CUDA;
}
