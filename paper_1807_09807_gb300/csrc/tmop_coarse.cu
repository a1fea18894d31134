// Coarse correction of the two-level Krylov preconditioner (see
// tmop_coarse.h): restriction P^t and prolongation P between the order-k
// node lattice and the interior element vertices, and the exact solve with
// alpha K_c by sine transforms, all as separable passes along one axis at a
// time over arrays laid out [dim][z][y][x] (x fastest).
//
// 1D transfer: lattice node g = k e + i of element e (i = 0..k, GLL node
// z_i) takes (1 - z_i) of vertex e and z_i of vertex e + 1, so P^t gives
// interior vertex v = I + 1 the sum over t = -(k-1)..k-1 of
// w(t) r[k v + t] with w(t) = 1 - z_|t| (z_{k-t} = 1 - z_t on GLL nodes).
//
// 1D coarse matrices on the n - 1 interior vertices of n unit reference
// elements: stiffness K1 = tridiag(-1, 2, -1), mass M1 = tridiag(1/6, 2/3,
// 1/6); both are diagonalised by the orthonormal sine basis
// S[j][m] = sqrt(2/n) sin((j+1)(m+1) pi / n) with eigenvalues
// lambda_j = 2 - 2 cos((j+1) pi / n), mu_j = (2 + cos((j+1) pi / n)) / 3.
// K_c = sum over axes a of K1 on a and M1 on the others, so
// K_c = S (sum_a lambda_a prod_{b != a} mu_b) S with S the product of the
// per-axis transforms (S is symmetric and its own inverse).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "tmop_coarse.h"
#include "tmop_vec.h"

namespace tmop {

struct CoarseSpace {
  int dim = 0, k = 0;
  int n[3] = {1, 1, 1}, Lf[3] = {1, 1, 1}, Lc[3] = {1, 1, 1};
  size_t nfine = 0, ncoarse = 0;   // per component
  bool fp32 = false;
  double z[8] = {0};               // GLL nodes
  double alpha = 1.0;
  void* tab = nullptr;             // per axis: S [Lc][Lc], lambda [Lc], mu [Lc] (float or double)
  size_t tab_off[3] = {0, 0, 0};
  void* buf[2] = {nullptr, nullptr};  // pass buffers (float or double)
  size_t buf_elems = 0;
};

namespace {

constexpr int kThr = 256;

__device__ __forceinline__ float fmaR(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fmaR(double a, double b, double c) { return fma(a, b, c); }

int grid_for(size_t work) {
  size_t g = (work + kThr - 1) / kThr;
  if (g > 152 * 16) g = 152 * 16;
  return g < 1 ? 1 : (int)g;
}

struct Wts {
  double w[8];  // w[t] = 1 - z_t, t = 0..k (w[0] = 1)
};

// out[o][I][j] = sum_{|t| < k} w(|t|) in[o][k (I + 1) + t][j]
template <class Rin, class Rout>
__global__ void k_restrict(const Rin* __restrict__ in, Rout* __restrict__ out, size_t outer, int Lf, int Lc,
                           size_t inner, int k, Wts w) {
  // (32-bit index arithmetic: every array here has fewer than 2^31 values,
  // and 64-bit divisions by run-time sizes cost ~5x more)
  const uint32_t total = (uint32_t)(outer * (size_t)Lc * inner), in32 = (uint32_t)inner, lc = (uint32_t)Lc;
  for (uint32_t idx = blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += gridDim.x * blockDim.x) {
    const uint32_t j = idx % in32, oI = idx / in32;
    const uint32_t I = oI % lc, o = oI / lc;
    const Rin* base = in + ((size_t)o * Lf + (size_t)k * (I + 1)) * inner + j;
    Rout acc = (Rout)base[0];   // arithmetic in the transform precision
    for (int t = 1; t < k; ++t)
      acc = fmaR((Rout)w.w[t], (Rout)base[(size_t)t * inner] + (Rout)base[-(ptrdiff_t)(t * inner)], acc);
    out[idx] = acc;
  }
}

// out[o][g][j] = (1 - z_i) in[o][e - 1][j] + z_i in[o][e][j], g = k e + i
// (interior vertex e - 1 is vertex e; vertices 0 and n are fixed: zero)
template <class R>
__device__ __forceinline__ R prolong_at(const R* __restrict__ in, size_t o, int g, size_t j, int Lc, size_t inner,
                                        int k, int n, const Wts& w) {
  int e = g / k;
  if (e > n - 1) e = n - 1;
  const int i = g - k * e;
  R v = R(0);
  if (e >= 1) v = fmaR((R)w.w[i], in[(o * Lc + (e - 1)) * inner + j], v);
  if (e <= n - 2) v = fmaR((R)(1.0 - w.w[i]), in[(o * Lc + e) * inner + j], v);
  return v;
}

template <class R>
__global__ void k_prolong(const R* __restrict__ in, R* __restrict__ out, size_t outer, int Lc, int Lf, size_t inner,
                          int k, int n, Wts w) {
  const uint32_t total = (uint32_t)(outer * (size_t)Lf * inner), in32 = (uint32_t)inner, lf = (uint32_t)Lf;
  for (uint32_t idx = blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += gridDim.x * blockDim.x) {
    const uint32_t j = idx % in32, og = idx / in32;
    out[idx] = prolong_at(in, og / lf, (int)(og % lf), j, Lc, inner, k, n, w);
  }
}

__device__ __forceinline__ double block_sum_c(double v) {
  __shared__ double red[kThr / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < kThr / 32; ++i) s += red[i];  // fixed order
  return s;
}

// the last prolongation pass (along x, into the FP64 fine array): y += P w,
// per-block partials of r . y
template <class R>
__global__ void k_prolong_add(const R* __restrict__ in, double* __restrict__ y, const double* __restrict__ r,
                              size_t outer, int Lc, int Lf, int k, int n, Wts w, double* __restrict__ part) {
  const uint32_t total = (uint32_t)(outer * (size_t)Lf), lf = (uint32_t)Lf;
  double s = 0.0;
  for (uint32_t idx = blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += gridDim.x * blockDim.x) {
    const double yi = y[idx] + (double)prolong_at(in, idx / lf, (int)(idx % lf), 0, Lc, 1, k, n, w);
    y[idx] = yi;
    if (part) s = fma(r[idx], yi, s);
  }
  if (part) {
    s = block_sum_c(s);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
  }
}

// out[o][a][j] = sum_m S[a][m] in[o][m][j] along an axis of length L
template <class R>
__global__ void k_dst(const R* __restrict__ in, R* __restrict__ out, const R* __restrict__ S, size_t outer, int L,
                      size_t inner) {
  const uint32_t total = (uint32_t)(outer * (size_t)L * inner), in32 = (uint32_t)inner, l32 = (uint32_t)L;
  for (uint32_t idx = blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += gridDim.x * blockDim.x) {
    const uint32_t j = idx % in32, oa = idx / in32;
    const uint32_t a = oa % l32, o = oa / l32;
    const R* src = in + (size_t)o * L * inner + j;
    const R* Sa = S + (size_t)a * L;
    R acc = R(0);
    for (int m = 0; m < L; ++m) acc = fmaR(__ldg(Sa + m), src[(size_t)m * inner], acc);
    out[idx] = acc;
  }
}

// divide by alpha times the eigenvalue of K_c at every coarse point
template <class R>
__global__ void k_eig_scale(R* __restrict__ v, const R* __restrict__ lx, const R* __restrict__ mx,
                            const R* __restrict__ ly, const R* __restrict__ my, const R* __restrict__ lz,
                            const R* __restrict__ mz, int dim, int L0, int L1, int L2, double inv_alpha) {
  const uint32_t per = (uint32_t)L0 * L1 * L2, total = per * dim, l0 = L0, l1 = L1;
  for (uint32_t idx = blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += gridDim.x * blockDim.x) {
    const uint32_t p = idx % per;
    const uint32_t I = p % l0, J = (p / l0) % l1, K = p / (l0 * l1);
    double lam;
    if (dim == 2) lam = (double)lx[I] * (double)my[J] + (double)mx[I] * (double)ly[J];
    else
      lam = (double)lx[I] * (double)my[J] * (double)mz[K] + (double)mx[I] * (double)ly[J] * (double)mz[K] +
            (double)mx[I] * (double)my[J] * (double)lz[K];
    v[idx] = (R)((double)v[idx] * inv_alpha / lam);
  }
}

template <class R>
__global__ void k_mode0(double* __restrict__ w, const R* __restrict__ Sx, const R* __restrict__ Sy,
                        const R* __restrict__ Sz, int dim, int L0, int L1, int L2) {
  const uint32_t per = (uint32_t)L0 * L1 * L2, total = per * dim, l0 = L0, l1 = L1;
  for (uint32_t idx = blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += gridDim.x * blockDim.x) {
    const uint32_t p = idx % per;
    const uint32_t I = p % l0, J = (p / l0) % l1, K = p / (l0 * l1);
    double v = (double)Sx[I] * (double)Sy[J];
    if (dim == 3) v *= (double)Sz[K];
    w[idx] = v;
  }
}

__global__ void k_to_float(const double* __restrict__ in, float* __restrict__ out, size_t count) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x)
    out[i] = (float)in[i];
}

Wts weights(const CoarseSpace* cs) {
  Wts w;
  for (int t = 0; t < 8; ++t) w.w[t] = t <= cs->k ? 1.0 - cs->z[t] : 0.0;
  return w;
}

// [outer][L_a][inner] view of a [dim][L2][L1][L0] array whose axes below a
// have lengths len[0..a-1] and above a len[a+1..]
void view(const CoarseSpace* cs, const int len[3], int a, size_t* outer, size_t* inner) {
  size_t in = 1, out = (size_t)cs->dim;
  for (int b = 0; b < a; ++b) in *= (size_t)len[b];
  for (int b = a + 1; b < 3; ++b) out *= (size_t)len[b];   // (a 2D stack's grids count as outer)
  *outer = out;
  *inner = in;
}

template <class R>
const R* tab_S(const CoarseSpace* cs, int a) {
  return static_cast<const R*>(cs->tab) + cs->tab_off[a];
}
template <class R>
const R* tab_lam(const CoarseSpace* cs, int a) {
  return tab_S<R>(cs, a) + (size_t)cs->Lc[a] * cs->Lc[a];
}
template <class R>
const R* tab_mu(const CoarseSpace* cs, int a) {
  return tab_lam<R>(cs, a) + cs->Lc[a];
}

// w_c = P^t r (FP64 fine -> R coarse in buf[0] or buf[1]); returns the buffer
template <class R>
R* restrict_all(CoarseSpace* cs, const double* r, cudaStream_t s) {
  const Wts w = weights(cs);
  int len[3] = {cs->Lf[0], cs->Lf[1], cs->Lf[2]};
  R* b[2] = {static_cast<R*>(cs->buf[0]), static_cast<R*>(cs->buf[1])};
  for (int a = 0; a < cs->dim; ++a) {
    size_t outer, inner;
    view(cs, len, a, &outer, &inner);
    R* dst = b[a % 2];
    const size_t work = outer * (size_t)cs->Lc[a] * inner;
    if (a == 0)
      k_restrict<double, R><<<grid_for(work), kThr, 0, s>>>(r, dst, outer, len[a], cs->Lc[a], inner, cs->k, w);
    else
      k_restrict<R, R><<<grid_for(work), kThr, 0, s>>>(b[(a - 1) % 2], dst, outer, len[a], cs->Lc[a], inner, cs->k, w);
    len[a] = cs->Lc[a];
  }
  return b[(cs->dim - 1) % 2];
}

// v <- (alpha K_c)^-1 v on the coarse array held in buf[src]; returns the buffer with the result
template <class R>
R* solve_coarse(CoarseSpace* cs, R* v, cudaStream_t s) {
  R* b[2] = {static_cast<R*>(cs->buf[0]), static_cast<R*>(cs->buf[1])};
  R* cur = v;
  auto other = [&](R* p) { return p == b[0] ? b[1] : b[0]; };
  for (int pass = 0; pass < 2; ++pass) {
    for (int a = 0; a < cs->dim; ++a) {
      size_t outer, inner;
      view(cs, cs->Lc, a, &outer, &inner);
      R* dst = other(cur);
      k_dst<R><<<grid_for(cs->ncoarse * cs->dim), kThr, 0, s>>>(cur, dst, tab_S<R>(cs, a), outer, cs->Lc[a], inner);
      cur = dst;
    }
    if (pass == 0) {
      const int a2 = cs->dim == 3 ? 2 : 1;
      k_eig_scale<R><<<grid_for(cs->ncoarse * cs->dim), kThr, 0, s>>>(
          cur, tab_lam<R>(cs, 0), tab_mu<R>(cs, 0), tab_lam<R>(cs, 1), tab_mu<R>(cs, 1), tab_lam<R>(cs, a2),
          tab_mu<R>(cs, a2), cs->dim, cs->Lc[0], cs->Lc[1], cs->Lc[2], 1.0 / cs->alpha);
    }
  }
  return cur;
}

// prolongation of the coarse array in `cur` along every axis but x (into the
// pass buffers); returns the array whose last pass (along x) is still to do
template <class R>
R* prolong_upper(CoarseSpace* cs, R* cur, int len[3], cudaStream_t s) {
  const Wts w = weights(cs);
  R* b[2] = {static_cast<R*>(cs->buf[0]), static_cast<R*>(cs->buf[1])};
  auto other = [&](R* p) { return p == b[0] ? b[1] : b[0]; };
  for (int a = 0; a < 3; ++a) len[a] = cs->Lc[a];
  for (int a = cs->dim - 1; a >= 1; --a) {
    size_t outer, inner;
    view(cs, len, a, &outer, &inner);
    R* dst = other(cur);
    const size_t work = outer * (size_t)cs->Lf[a] * inner;
    k_prolong<R><<<grid_for(work), kThr, 0, s>>>(cur, dst, outer, cs->Lc[a], cs->Lf[a], inner, cs->k, cs->n[a], w);
    len[a] = cs->Lf[a];
    cur = dst;
  }
  return cur;
}

template <class R>
int apply_add_t(CoarseSpace* cs, const double* r, double* y, double* part, cudaStream_t s) {
  R* c = restrict_all<R>(cs, r, s);
  c = solve_coarse<R>(cs, c, s);
  int len[3];
  c = prolong_upper<R>(cs, c, len, s);
  size_t outer, inner;
  view(cs, len, 0, &outer, &inner);
  const int g = red_grid(outer * (size_t)cs->Lf[0]);
  k_prolong_add<R><<<g, kThr, 0, s>>>(c, y, r, outer, cs->Lc[0], cs->Lf[0], cs->k, cs->n[0], weights(cs), part);
  return cudaGetLastError() == cudaSuccess ? g : -1;
}

}  // namespace

CoarseSpace* coarse_create(int dim, int k, const int n[3], const double* z, bool fp32) {
  if ((dim != 2 && dim != 3) || k < 1 || k > 7 || !n || !z) return nullptr;
  CoarseSpace* cs = new CoarseSpace();
  cs->dim = dim;
  cs->k = k;
  cs->fp32 = fp32;
  for (int i = 0; i <= k; ++i) cs->z[i] = z[i];
  cs->nfine = 1;
  cs->ncoarse = 1;
  for (int a = 0; a < 3; ++a) {
    // 2D: n[2] > 1 is a stack of that many grids, with no transfer between them
    const int stack = (dim == 2 && a == 2 && n[2] > 1) ? n[2] : 1;
    cs->n[a] = a < dim ? n[a] : stack;
    if (a < dim && cs->n[a] < 2) { delete cs; return nullptr; }
    cs->Lf[a] = a < dim ? k * cs->n[a] + 1 : stack;
    cs->Lc[a] = a < dim ? cs->n[a] - 1 : stack;
    cs->nfine *= (size_t)cs->Lf[a];
    cs->ncoarse *= (size_t)cs->Lc[a];
  }
  if (cs->nfine * dim >= ((size_t)1 << 31)) { delete cs; return nullptr; }   // 32-bit indices in the passes
  // tables
  const size_t elt = fp32 ? sizeof(float) : sizeof(double);
  size_t tot = 0;
  for (int a = 0; a < dim; ++a) {
    cs->tab_off[a] = tot;
    tot += (size_t)cs->Lc[a] * cs->Lc[a] + 2 * (size_t)cs->Lc[a];
  }
  if (dim == 2) cs->tab_off[2] = cs->tab_off[1];
  double* h = new double[tot];
  for (int a = 0; a < dim; ++a) {
    const int L = cs->Lc[a], na = cs->n[a];
    double* S = h + cs->tab_off[a];
    const double sc = sqrt(2.0 / na);
    for (int j = 0; j < L; ++j)
      for (int m = 0; m < L; ++m) S[(size_t)j * L + m] = sc * sin((double)(j + 1) * (m + 1) * M_PI / na);
    for (int j = 0; j < L; ++j) {
      const double c = cos((double)(j + 1) * M_PI / na);
      S[(size_t)L * L + j] = 2.0 - 2.0 * c;
      S[(size_t)L * L + L + j] = (2.0 + c) / 3.0;
    }
  }
  bool ok = cudaMalloc(&cs->tab, tot * elt) == cudaSuccess;
  if (ok) {
    if (fp32) {
      float* f = new float[tot];
      for (size_t i = 0; i < tot; ++i) f[i] = (float)h[i];
      ok = cudaMemcpy(cs->tab, f, tot * elt, cudaMemcpyHostToDevice) == cudaSuccess;
      delete[] f;
    } else {
      ok = cudaMemcpy(cs->tab, h, tot * elt, cudaMemcpyHostToDevice) == cudaSuccess;
    }
  }
  delete[] h;
  // pass buffers: the largest intermediate array of either direction
  size_t big = 0;
  {
    int len[3] = {cs->Lf[0], cs->Lf[1], cs->Lf[2]};
    for (int a = 0; a < dim; ++a) {  // restriction: x, y, z
      len[a] = cs->Lc[a];
      size_t p = dim;
      for (int b = 0; b < 3; ++b) p *= (size_t)len[b];
      if (p > big) big = p;
    }
  }
  cs->buf_elems = big;
  if (ok) ok = cudaMalloc(&cs->buf[0], big * elt) == cudaSuccess && cudaMalloc(&cs->buf[1], big * elt) == cudaSuccess;
  if (!ok) {
    coarse_destroy(cs);
    return nullptr;
  }
  return cs;
}

void coarse_destroy(CoarseSpace* cs) {
  if (!cs) return;
  cudaFree(cs->tab);
  cudaFree(cs->buf[0]);
  cudaFree(cs->buf[1]);
  delete cs;
}

size_t coarse_size(const CoarseSpace* cs) { return cs ? cs->ncoarse : 0; }

void coarse_set_alpha(CoarseSpace* cs, double alpha) {
  if (cs && alpha > 0.0 && isfinite(alpha)) cs->alpha = alpha;
}

int coarse_mode0(CoarseSpace* cs, double* w, double* lambda0, cudaStream_t s) {
  if (!cs || !w) return (int)cudaErrorInvalidValue;
  const int L0 = cs->Lc[0], L1 = cs->Lc[1], L2 = cs->Lc[2];
  const size_t work = cs->ncoarse * cs->dim;
  if (cs->fp32)
    k_mode0<float><<<grid_for(work), kThr, 0, s>>>(w, tab_S<float>(cs, 0), tab_S<float>(cs, 1),
                                                   tab_S<float>(cs, cs->dim == 3 ? 2 : 1), cs->dim, L0, L1, L2);
  else
    k_mode0<double><<<grid_for(work), kThr, 0, s>>>(w, tab_S<double>(cs, 0), tab_S<double>(cs, 1),
                                                    tab_S<double>(cs, cs->dim == 3 ? 2 : 1), cs->dim, L0, L1, L2);
  if (lambda0) {
    double lam = 0.0;
    for (int a = 0; a < cs->dim; ++a) {
      double t = 1.0;
      for (int b = 0; b < cs->dim; ++b) {
        const double c = cos(M_PI / cs->n[b]);
        t *= b == a ? 2.0 - 2.0 * c : (2.0 + c) / 3.0;
      }
      lam += t;
    }
    // w^t K_c w per component: every grid of a 2D stack holds a unit mode
    *lambda0 = lam * (cs->dim == 2 ? cs->Lc[2] : 1);
  }
  return (int)cudaGetLastError();
}

int coarse_prolong(CoarseSpace* cs, const double* w, double* y, cudaStream_t s) {
  if (!cs || !w || !y) return (int)cudaErrorInvalidValue;
  if (cudaMemsetAsync(y, 0, sizeof(double) * cs->nfine * cs->dim, s) != cudaSuccess) return (int)cudaErrorUnknown;
  // the FP64 coarse field goes through the pass buffers in the transform precision
  int len[3];
  int rc;
  if (cs->fp32) {
    float* c = static_cast<float*>(cs->buf[0]);
    k_to_float<<<grid_for(cs->ncoarse * cs->dim), kThr, 0, s>>>(w, c, cs->ncoarse * cs->dim);
    c = prolong_upper<float>(cs, c, len, s);
    size_t outer, inner;
    view(cs, len, 0, &outer, &inner);
    k_prolong_add<float><<<red_grid(outer * (size_t)cs->Lf[0]), kThr, 0, s>>>(c, y, nullptr, outer, cs->Lc[0], cs->Lf[0],
                                                                            cs->k, cs->n[0], weights(cs), nullptr);
  } else {
    double* c = static_cast<double*>(cs->buf[0]);
    cudaMemcpyAsync(c, w, sizeof(double) * cs->ncoarse * cs->dim, cudaMemcpyDeviceToDevice, s);
    c = prolong_upper<double>(cs, c, len, s);
    size_t outer, inner;
    view(cs, len, 0, &outer, &inner);
    k_prolong_add<double><<<red_grid(outer * (size_t)cs->Lf[0]), kThr, 0, s>>>(
        c, y, nullptr, outer, cs->Lc[0], cs->Lf[0], cs->k, cs->n[0], weights(cs), nullptr);
  }
  rc = (int)cudaGetLastError();
  return rc;
}

int coarse_apply_add(void* obj, const double* r, double* y, double* part, cudaStream_t s) {
  CoarseSpace* cs = static_cast<CoarseSpace*>(obj);
  if (!cs || !r || !y) return -1;
  return cs->fp32 ? apply_add_t<float>(cs, r, y, part, s) : apply_add_t<double>(cs, r, y, part, s);
}

}  // namespace tmop
