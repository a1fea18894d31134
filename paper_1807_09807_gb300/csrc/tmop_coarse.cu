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

#include <type_traits>

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
constexpr int kMaxCoarseParts = 256;   // per-block partials of the coarse dot product

__device__ __forceinline__ float fmaR(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fmaR(double a, double b, double c) { return fma(a, b, c); }

int grid_for(size_t work) {
  size_t g = (work + kThr - 1) / kThr;
  if (g > 152 * 16) g = 152 * 16;
  return g < 1 ? 1 : (int)g;
}

// transfer weights in the pass precision: w[t] = 1 - z_t, z[t] = z_t, t = 0..k
template <class R>
struct Wts {
  R w[8], z[8];
};

// Division by a run-time divisor d < 2^31 of dividends n < 2^31 as a
// multiply-high and a shift (Granlund and Montgomery, "Division by invariant
// integers using multiplication", 1994): with s = ceil(log2 d) and
// m = floor(2^32 (2^s - d) / d) + 1, n / d = (mulhi(n, m) + n) >> s.
struct FastDiv {
  uint32_t d = 1, m = 0, s = 0;
  FastDiv() = default;
  explicit FastDiv(uint32_t d_) : d(d_) {
    if (d > 1) {
      s = 32u - (uint32_t)__builtin_clz(d - 1);
      m = (uint32_t)(((((uint64_t)1) << 32) * ((((uint64_t)1) << s) - d)) / d + 1);
    }
  }
  __device__ __forceinline__ uint32_t div(uint32_t n) const { return (__umulhi(n, m) + n) >> s; }
};

// One pass along an axis of an array viewed as [outer][L][inner] (L = Lin in,
// Lout out), one output value per thread iteration, the flat output index
// split into (o, position, j) by two multiply-high divisions and the position
// along the axis into (element, node) by the compile-time order K.
struct Pass {
  uint32_t outer, Lin, Lout, inner, total;
  FastDiv by_inner, by_Lout;
};

// out[o][I][j] = sum_{|t| < K} w(|t|) in[o][K (I + 1) + t][j]
template <class Rin, class Rout, int K>
__global__ void k_restrict(const Rin* __restrict__ in, Rout* __restrict__ out, Pass p, Wts<Rout> w) {
  for (uint32_t idx = blockIdx.x * blockDim.x + threadIdx.x; idx < p.total; idx += gridDim.x * blockDim.x) {
    const uint32_t rest = p.by_inner.div(idx), j = idx - rest * p.inner;
    const uint32_t o = p.by_Lout.div(rest), I = rest - o * p.Lout;
    const Rin* base = in + ((size_t)o * p.Lin + (size_t)K * (I + 1)) * p.inner + j;
    Rout acc = (Rout)base[0];   // arithmetic in the transform precision
#pragma unroll
    for (int d = 1; d < K; ++d)
      acc = fmaR(w.w[d], (Rout)base[(size_t)d * p.inner] + (Rout)base[-(ptrdiff_t)((size_t)d * p.inner)], acc);
    out[idx] = acc;
  }
}

// (1 - z_i) in[o][e - 1][j] + z_i in[o][e][j] at g = K e + i: interior vertex
// e - 1 is vertex e; vertices 0 and n are fixed (zero)
template <class R, int K>
__device__ __forceinline__ R prolong_at(const R* __restrict__ in, size_t o, uint32_t g, size_t j, uint32_t Lc,
                                        size_t inner, uint32_t n, const Wts<R>& w) {
  uint32_t e = g / K;
  if (e > n - 1) e = n - 1;
  const uint32_t i = g - K * e;
  R wi = w.w[0], zi = w.z[0];   // by selects: no dynamic indexing into the parameter block
#pragma unroll
  for (int t = 1; t <= K; ++t)
    if (i == (uint32_t)t) wi = w.w[t], zi = w.z[t];
  R v = R(0);
  if (e >= 1) v = fmaR(wi, in[(o * Lc + (e - 1)) * inner + j], v);
  if (e + 2 <= n) v = fmaR(zi, in[(o * Lc + e) * inner + j], v);
  return v;
}

template <class R, int K>
__global__ void k_prolong(const R* __restrict__ in, R* __restrict__ out, Pass p, uint32_t n, Wts<R> w) {
  for (uint32_t idx = blockIdx.x * blockDim.x + threadIdx.x; idx < p.total; idx += gridDim.x * blockDim.x) {
    const uint32_t rest = p.by_inner.div(idx), j = idx - rest * p.inner;
    const uint32_t o = p.by_Lout.div(rest), g = rest - o * p.Lout;
    out[idx] = prolong_at<R, K>(in, o, g, j, p.Lin, p.inner, n, w);
  }
}

// the last prolongation pass (along x, inner = 1) into the fine array (FP64,
// or FP32 for FP32 Krylov vectors): y += P w
template <class R, class Ry, int K>
__global__ void k_prolong_add(const R* __restrict__ in, Ry* __restrict__ y, Pass p, uint32_t n, Wts<R> w) {
  for (uint32_t idx = blockIdx.x * blockDim.x + threadIdx.x; idx < p.total; idx += gridDim.x * blockDim.x) {
    const uint32_t o = p.by_Lout.div(idx), g = idx - o * p.Lout;
    y[idx] += (Ry)prolong_at<R, K>(in, o, g, 0, p.Lin, 1, n, w);
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
    for (int i = 0; i < (int)(blockDim.x / 32); ++i) s += red[i];  // fixed order
  return s;
}

// The sine transform along one axis as a batched product C_b = A_b B_b
// (M x N = (M x Kd)(Kd x N)), with A(i, k) = A[b sAb + i lda + k],
// B(k, j) = B[b sBb + k ldb + j], C(i, j) = C[b sCb + i ldc + j]: along x
// (inner = 1) In [rows][L] times S (symmetric), along y or z S times every
// [L][inner] slab. 64 x 64 output tiles over 16-deep chunks staged in shared
// memory, 4 x 4 outputs per thread (rows ty + 16 r, columns tx + 16 c).
constexpr int kTM = 64, kTN = 64, kTK = 16;

template <class R>
__global__ void __launch_bounds__(256, 2) k_dst(const R* __restrict__ A, const R* __restrict__ B, R* __restrict__ C,
                                             int M, int N, int Kd, int batch, size_t sAb, int lda, size_t sBb,
                                             int ldb, size_t sCb, int ldc) {
  __shared__ R As[kTK][kTM + 1];
  __shared__ R Bs[kTK][kTN];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int tiles_n = (N + kTN - 1) / kTN, tiles_m = (M + kTM - 1) / kTM;
  for (int b = blockIdx.z; b < batch; b += gridDim.z)
    for (int tm = blockIdx.y; tm < tiles_m; tm += gridDim.y)
      for (int tn = blockIdx.x; tn < tiles_n; tn += gridDim.x) {
        const R* Ab = A + b * sAb;
        const R* Bb = B + b * sBb;
        const int i0 = tm * kTM, j0 = tn * kTN;
        R acc[4][4];
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
          for (int c = 0; c < 4; ++c) acc[r][c] = R(0);
        for (int k0 = 0; k0 < Kd; k0 += kTK) {
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const int i = (tid >> 4) + 16 * q, k = tid & 15;   // A tile: 16 consecutive k per row
            As[k][i] = (i0 + i < M && k0 + k < Kd) ? Ab[(size_t)(i0 + i) * lda + k0 + k] : R(0);
            const int kb = (tid >> 6) + 4 * q, j = tid & 63;   // B tile: 64 consecutive j per row
            Bs[kb][j] = (k0 + kb < Kd && j0 + j < N) ? Bb[(size_t)(k0 + kb) * ldb + j0 + j] : R(0);
          }
          __syncthreads();
#pragma unroll
          for (int k = 0; k < kTK; ++k) {
            R a[4], bb[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) a[r] = As[k][ty + 16 * r];
#pragma unroll
            for (int c = 0; c < 4; ++c) bb[c] = Bs[k][tx + 16 * c];
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
              for (int c = 0; c < 4; ++c) acc[r][c] = fmaR(a[r], bb[c], acc[r][c]);
          }
          __syncthreads();
        }
        R* Cb = C + b * sCb;
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            const int i = i0 + ty + 16 * r, j = j0 + tx + 16 * c;
            if (i < M && j < N) Cb[(size_t)i * ldc + j] = acc[r][c];
          }
      }
}

// divide by alpha times the eigenvalue of K_c at every coarse point, in the
// sine basis; per-block partials of v_old . v_new into part (if given): with
// S orthogonal and symmetric that is c . (alpha K_c)^-1 c for the restricted
// residual c, the coarse share of r . M^-1 r
template <class R>
__global__ void k_eig_scale(R* __restrict__ v, const R* __restrict__ lx, const R* __restrict__ mx,
                            const R* __restrict__ ly, const R* __restrict__ my, const R* __restrict__ lz,
                            const R* __restrict__ mz, int dim, uint32_t L0, uint32_t L1, uint32_t L2, uint32_t total,
                            FastDiv by0, FastDiv by1, FastDiv by2, R inv_alpha, double* __restrict__ part) {
  double s = 0.0;
  for (uint32_t idx = blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += gridDim.x * blockDim.x) {
    const uint32_t row = by0.div(idx), I = idx - row * L0;
    const uint32_t rr = by1.div(row), J = row - rr * L1;
    const uint32_t K = rr - by2.div(rr) * L2;
    R lam;
    if (dim == 2) lam = fmaR(lx[I], my[J], mx[I] * ly[J]);
    else lam = fmaR(fmaR(lx[I], my[J], mx[I] * ly[J]), mz[K], mx[I] * my[J] * lz[K]);
    const R c = v[idx], w = c * (inv_alpha / lam);
    v[idx] = w;
    s = fma((double)c, (double)w, s);
  }
  if (part) {
    s = block_sum_c(s);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
  }
}

template <class R>
__global__ void k_mode0(double* __restrict__ w, const R* __restrict__ Sx, const R* __restrict__ Sy,
                        const R* __restrict__ Sz, int dim, uint32_t L0, uint32_t L1, uint32_t L2) {
  const uint32_t total = (uint32_t)dim * L0 * L1 * L2;
  for (uint32_t idx = blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += gridDim.x * blockDim.x) {
    const uint32_t I = idx % L0, J = (idx / L0) % L1, K = (idx / (L0 * L1)) % L2;
    double v = (double)Sx[I] * (double)Sy[J];
    if (dim == 3) v *= (double)Sz[K];
    w[idx] = v;
  }
}

__global__ void k_to_float(const double* __restrict__ in, float* __restrict__ out, size_t count) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x)
    out[i] = (float)in[i];
}

template <class R>
Wts<R> weights(const CoarseSpace* cs) {
  Wts<R> w;
  for (int t = 0; t < 8; ++t) {
    w.w[t] = (R)(t <= cs->k ? 1.0 - cs->z[t] : 0.0);
    w.z[t] = (R)(t <= cs->k ? cs->z[t] : 0.0);
  }
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

// calls f(std::integral_constant<int, K>{}) for the order K = k (1..7)
template <class F>
int with_order(int k, F&& f) {
  switch (k) {
    case 1: f(std::integral_constant<int, 1>{}); break;
    case 2: f(std::integral_constant<int, 2>{}); break;
    case 3: f(std::integral_constant<int, 3>{}); break;
    case 4: f(std::integral_constant<int, 4>{}); break;
    case 5: f(std::integral_constant<int, 5>{}); break;
    case 6: f(std::integral_constant<int, 6>{}); break;
    case 7: f(std::integral_constant<int, 7>{}); break;
    default: return -1;
  }
  return 0;
}

Pass make_pass(const CoarseSpace* cs, const int len[3], int a, int Lout) {
  size_t outer, inner;
  view(cs, len, a, &outer, &inner);
  Pass p;
  p.outer = (uint32_t)outer;
  p.Lin = (uint32_t)len[a];
  p.Lout = (uint32_t)Lout;
  p.inner = (uint32_t)inner;
  p.total = (uint32_t)(outer * (size_t)Lout * inner);
  p.by_inner = FastDiv(p.inner);
  p.by_Lout = FastDiv(p.Lout);
  return p;
}

// w_c = P^t r (fine, FP64 or FP32 -> R coarse in buf[0] or buf[1]); returns the buffer
template <class R, class Rf>
R* restrict_all(CoarseSpace* cs, const Rf* r, cudaStream_t s) {
  const Wts<R> w = weights<R>(cs);
  int len[3] = {cs->Lf[0], cs->Lf[1], cs->Lf[2]};
  R* b[2] = {static_cast<R*>(cs->buf[0]), static_cast<R*>(cs->buf[1])};
  for (int a = 0; a < cs->dim; ++a) {
    const Pass p = make_pass(cs, len, a, cs->Lc[a]);
    R* dst = b[a % 2];
    const R* src = a == 0 ? nullptr : b[(a - 1) % 2];
    const int g = grid_for(p.total);
    with_order(cs->k, [&](auto K) {
      if (a == 0) k_restrict<Rf, R, K.value><<<g, kThr, 0, s>>>(r, dst, p, w);
      else k_restrict<R, R, K.value><<<g, kThr, 0, s>>>(src, dst, p, w);
    });
    len[a] = cs->Lc[a];
  }
  return b[(cs->dim - 1) % 2];
}

// one sine transform along axis a of the coarse array: src -> dst
template <class R>
void dst_pass(CoarseSpace* cs, int a, const R* src, R* dst, cudaStream_t s) {
  size_t outer, inner;
  view(cs, cs->Lc, a, &outer, &inner);
  const int L = cs->Lc[a];
  const R* S = tab_S<R>(cs, a);
  if (inner == 1) {   // [rows][L] S
    const int M = (int)outer;
    const int tm = (M + kTM - 1) / kTM, tn = (L + kTN - 1) / kTN;
    const dim3 g(tn, tm < 65535 ? tm : 65535, 1);
    k_dst<R><<<g, 256, 0, s>>>(src, S, dst, M, L, L, 1, 0, L, 0, L, 0, L);
  } else {            // S [L][inner] for every outer slab
    const int N = (int)inner, batch = (int)outer;
    const int tm = (L + kTM - 1) / kTM, tn = (N + kTN - 1) / kTN;
    const dim3 g(tn < 65535 ? tn : 65535, tm < 65535 ? tm : 65535, batch < 65535 ? batch : 65535);
    const size_t slab = (size_t)L * inner;
    k_dst<R><<<g, 256, 0, s>>>(S, src, dst, L, N, L, batch, 0, L, slab, N, slab, N);
  }
}

// v <- (alpha K_c)^-1 v on the coarse array in v (one of the pass buffers);
// returns the buffer with the result. part (if given): per-block partials of
// c . (alpha K_c)^-1 c; *np their number.
template <class R>
R* solve_coarse(CoarseSpace* cs, R* v, double* part, int* np, cudaStream_t s) {
  R* b[2] = {static_cast<R*>(cs->buf[0]), static_cast<R*>(cs->buf[1])};
  R* cur = v;
  auto other = [&](R* p) { return p == b[0] ? b[1] : b[0]; };
  for (int pass = 0; pass < 2; ++pass) {
    for (int a = 0; a < cs->dim; ++a) {
      R* dst = other(cur);
      dst_pass<R>(cs, a, cur, dst, s);
      cur = dst;
    }
    if (pass == 0) {
      const int a2 = cs->dim == 3 ? 2 : 1;
      const uint32_t L0 = cs->Lc[0], L1 = cs->Lc[1], L2 = cs->Lc[2];
      const uint32_t total = (uint32_t)(cs->ncoarse * cs->dim);
      int g = grid_for(total);
      if (g > kMaxCoarseParts) g = kMaxCoarseParts;
      k_eig_scale<R><<<g, kThr, 0, s>>>(cur, tab_lam<R>(cs, 0), tab_mu<R>(cs, 0), tab_lam<R>(cs, 1), tab_mu<R>(cs, 1),
                                        tab_lam<R>(cs, a2), tab_mu<R>(cs, a2), cs->dim, L0, L1, L2, total,
                                        FastDiv(L0), FastDiv(L1), FastDiv(L2), (R)(1.0 / cs->alpha), part);
      *np = g;
    }
  }
  return cur;
}

// prolongation of the coarse array in `cur` along every axis but x (into the
// pass buffers); returns the array whose last pass (along x) is still to do
template <class R>
R* prolong_upper(CoarseSpace* cs, R* cur, int len[3], cudaStream_t s) {
  const Wts<R> w = weights<R>(cs);
  R* b[2] = {static_cast<R*>(cs->buf[0]), static_cast<R*>(cs->buf[1])};
  auto other = [&](R* p) { return p == b[0] ? b[1] : b[0]; };
  for (int a = 0; a < 3; ++a) len[a] = cs->Lc[a];
  for (int a = cs->dim - 1; a >= 1; --a) {
    const Pass p = make_pass(cs, len, a, cs->Lf[a]);
    R* dst = other(cur);
    with_order(cs->k, [&](auto K) {
      k_prolong<R, K.value><<<grid_for(p.total), kThr, 0, s>>>(cur, dst, p, (uint32_t)cs->n[a], w);
    });
    len[a] = cs->Lf[a];
    cur = dst;
  }
  return cur;
}

// the last pass (along x) into y
template <class R, class Ry>
void prolong_last(CoarseSpace* cs, const R* c, const int len[3], Ry* y, cudaStream_t s) {
  const Pass p = make_pass(cs, len, 0, cs->Lf[0]);
  const Wts<R> w = weights<R>(cs);
  with_order(cs->k, [&](auto K) {
    k_prolong_add<R, Ry, K.value><<<grid_for(p.total), kThr, 0, s>>>(c, y, p, (uint32_t)cs->n[0], w);
  });
}

template <class R, class Rf>
int apply_add_t(CoarseSpace* cs, const Rf* r, Rf* y, double* part, cudaStream_t s) {
  R* c = restrict_all<R, Rf>(cs, r, s);
  int np = 0;
  c = solve_coarse<R>(cs, c, part, &np, s);
  int len[3];
  c = prolong_upper<R>(cs, c, len, s);
  prolong_last<R, Rf>(cs, c, len, y, s);
  return cudaGetLastError() == cudaSuccess ? np : -1;
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
  const uint32_t L0 = cs->Lc[0], L1 = cs->Lc[1], L2 = cs->Lc[2];
  const int g = grid_for(cs->ncoarse * cs->dim);
  if (cs->fp32)
    k_mode0<float><<<g, kThr, 0, s>>>(w, tab_S<float>(cs, 0), tab_S<float>(cs, 1),
                                      tab_S<float>(cs, cs->dim == 3 ? 2 : 1), cs->dim, L0, L1, L2);
  else
    k_mode0<double><<<g, kThr, 0, s>>>(w, tab_S<double>(cs, 0), tab_S<double>(cs, 1),
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
  if (cs->fp32) {
    float* c = static_cast<float*>(cs->buf[0]);
    k_to_float<<<grid_for(cs->ncoarse * cs->dim), kThr, 0, s>>>(w, c, cs->ncoarse * cs->dim);
    c = prolong_upper<float>(cs, c, len, s);
    prolong_last<float, double>(cs, c, len, y, s);
  } else {
    double* c = static_cast<double*>(cs->buf[0]);
    cudaMemcpyAsync(c, w, sizeof(double) * cs->ncoarse * cs->dim, cudaMemcpyDeviceToDevice, s);
    c = prolong_upper<double>(cs, c, len, s);
    prolong_last<double, double>(cs, c, len, y, s);
  }
  return (int)cudaGetLastError();
}

int coarse_apply_add(void* obj, const double* r, double* y, double* part, cudaStream_t s) {
  CoarseSpace* cs = static_cast<CoarseSpace*>(obj);
  if (!cs || !r || !y) return -1;
  return cs->fp32 ? apply_add_t<float, double>(cs, r, y, part, s) : apply_add_t<double, double>(cs, r, y, part, s);
}

int coarse_apply_add32(void* obj, const float* r, float* y, double* part, cudaStream_t s) {
  CoarseSpace* cs = static_cast<CoarseSpace*>(obj);
  if (!cs || !r || !y) return -1;
  return cs->fp32 ? apply_add_t<float, float>(cs, r, y, part, s) : apply_add_t<double, float>(cs, r, y, part, s);
}

}  // namespace tmop
