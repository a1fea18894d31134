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
  size_t want = (n + kThreads * 4 - 1) / (kThreads * 4);
  size_t cap = (size_t)g_sms * 4;
  if (want > cap) want = cap;
  if (want > (size_t)kMaxRedBlocks) want = kMaxRedBlocks;
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

__global__ void k_sum_final(const double* __restrict__ part, int np, double* __restrict__ out) {
  double s = 0.0;
  for (int i = threadIdx.x; i < np; i += blockDim.x) s += part[i];
  s = block_sum(s);
  if (threadIdx.x == 0) *out = s;
}

__global__ void k_energy_final(const double* __restrict__ pf, const double* __restrict__ pm, int np,
                               double* __restrict__ outF, double* __restrict__ outMin) {
  __shared__ double mins[kThreads];
  double s = 0.0, m = INFINITY;
  for (int i = threadIdx.x; i < np; i += blockDim.x) {
    s += pf[i];
    m = fmin(m, pm[i]);
  }
  mins[threadIdx.x] = m;
  s = block_sum(s);
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int i = 1; i < kThreads; ++i) m = fmin(m, mins[i]);
    *outF = s;
    *outMin = m;
  }
}

int dot(const double* a, const double* b, size_t n, double* part, double* out, cudaStream_t s) {
  const int g = red_grid(n);
  k_dot_part<<<g, kThreads, 0, s>>>(a, b, n, part);
  k_sum_final<<<1, kThreads, 0, s>>>(part, g, out);
  return (int)cudaGetLastError();
}

int energy_final(const double* pf, const double* pm, int np, double* outF, double* outMin, cudaStream_t s) {
  k_energy_final<<<1, kThreads, 0, s>>>(pf, pm, np, outF, outMin);
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
// v = b / beta1, vprev = w = wprev = sol = 0 and the rotation state.
__global__ void k_minres_init(const double* __restrict__ b, double* v, double* vprev, double* w, double* wprev,
                              double* sol, double* st, size_t n) {
  const double beta1 = sqrt(st[KS_BETA_NEXT2]);
  const double inv = beta1 > 0.0 ? 1.0 / beta1 : 0.0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    v[i] = b[i] * inv;
    vprev[i] = 0.0;
    w[i] = 0.0;
    wprev[i] = 0.0;
    sol[i] = 0.0;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    st[KS_BETA1] = beta1;
    st[KS_BETA] = beta1;
    st[KS_ETA] = beta1;
    st[KS_RESID] = beta1;
    st[KS_C_OLD] = 1.0; st[KS_S_OLD] = 0.0; st[KS_C] = 1.0; st[KS_S] = 0.0;
  }
}

// Av <- Av - alpha v - beta vprev, with per-block partials of |Av|^2
__global__ void k_lanczos(double* __restrict__ Av, const double* __restrict__ v, const double* __restrict__ vprev,
                          const double* __restrict__ st, size_t n, double* __restrict__ part) {
  const double alpha = st[KS_ALPHA], beta = st[KS_BETA];
  double s = 0.0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const double r = Av[i] - alpha * v[i] - beta * vprev[i];
    Av[i] = r;
    s = fma(r, r, s);
  }
  s = block_sum(s);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// Apply the two previous rotations to the new tridiagonal column
// (beta_k, alpha_k, beta_{k+1}), form the new rotation, update eta.
__global__ void k_minres_scalar(double* st) {
  const double beta = st[KS_BETA], alpha = st[KS_ALPHA];
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
}

// New search direction w_k = (v_k - r1 w_{k-2} - r2 w_{k-1}) / rho, solution
// update, and the next Lanczos vector.
__global__ void k_minres_vec(double* __restrict__ v, double* __restrict__ vprev, const double* __restrict__ Av,
                             double* __restrict__ w, double* __restrict__ wprev, double* __restrict__ sol,
                             const double* __restrict__ st, size_t n) {
  const double r1 = st[KS_R1], r2 = st[KS_R2], ir = st[KS_INV_RHO], phi = st[KS_PHI], ib = st[KS_INV_BETA_NEXT];
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const double vi = v[i];
    const double wn = (vi - r1 * wprev[i] - r2 * w[i]) * ir;
    wprev[i] = w[i];
    w[i] = wn;
    sol[i] = fma(phi, wn, sol[i]);
    vprev[i] = vi;
    v[i] = Av[i] * ib;
  }
}

int minres_init(const double* b, double* v, double* vprev, double* w, double* wprev, double* sol, double* st,
                double* part, size_t n, cudaStream_t s) {
  int g = red_grid(n);
  k_dot_part<<<g, kThreads, 0, s>>>(b, b, n, part);
  k_sum_final<<<1, kThreads, 0, s>>>(part, g, st + KS_BETA_NEXT2);
  k_minres_init<<<g, kThreads, 0, s>>>(b, v, vprev, w, wprev, sol, st, n);
  return (int)cudaGetLastError();
}

int minres_after_hv(double* v, double* vprev, double* Av, double* w, double* wprev, double* sol, double* st,
                    double* part, size_t n, cudaStream_t s) {
  int g = red_grid(n);
  k_dot_part<<<g, kThreads, 0, s>>>(v, Av, n, part);
  k_sum_final<<<1, kThreads, 0, s>>>(part, g, st + KS_ALPHA);
  k_lanczos<<<g, kThreads, 0, s>>>(Av, v, vprev, st, n, part);
  k_sum_final<<<1, kThreads, 0, s>>>(part, g, st + KS_BETA_NEXT2);
  k_minres_scalar<<<1, 1, 0, s>>>(st);
  k_minres_vec<<<g, kThreads, 0, s>>>(v, vprev, Av, w, wprev, sol, st, n);
  return (int)cudaGetLastError();
}

// ---------------------------------------------------------------- CG
__global__ void k_cg_init(const double* __restrict__ b, double* r, double* d, double* sol, double* st, size_t n) {
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
  }
}

__global__ void k_cg_a(double* st) {
  const double dHd = st[KS_ALPHA];
  if (!(dHd > 0.0)) {
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
  const double rr_new = st[KS_BETA_NEXT2];
  st[KS_B] = st[KS_RR] > 0.0 ? rr_new / st[KS_RR] : 0.0;
  st[KS_RR] = rr_new;
  st[KS_RESID] = sqrt(fmax(rr_new, 0.0));
}

__global__ void k_cg_dir(double* __restrict__ d, const double* __restrict__ r, const double* __restrict__ st,
                         size_t n) {
  const double b = st[KS_B];
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    d[i] = fma(b, d[i], r[i]);
}

int cg_init(const double* b, double* r, double* d, double* sol, double* st, double* part, size_t n,
            cudaStream_t s) {
  int g = red_grid(n);
  k_dot_part<<<g, kThreads, 0, s>>>(b, b, n, part);
  k_sum_final<<<1, kThreads, 0, s>>>(part, g, st + KS_BETA_NEXT2);
  k_cg_init<<<g, kThreads, 0, s>>>(b, r, d, sol, st, n);
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
