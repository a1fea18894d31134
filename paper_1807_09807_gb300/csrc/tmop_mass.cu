// Restricted node movement (Section 4.3.1, eq. (4.2)): the term
//   sum_E int_{E_t} delta |x - x_init|^2 dx_t = sum_E sum_q w_q det W delta |u(x_q)|^2,
// u = x - x_init interpolated with the nodal basis, its gradient
// 2 delta sum_q w_q det W u(x_q) phi_i(x_q) and its Hessian action (the same
// with v: a weighted mass matrix). FP64, one warp per element, sum-factorised
// VALUE contractions (B in every direction), added to the metric kernels'
// results by the C-ABI calls when delta != 0.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "tmop_device.cuh"
#include "tmop_kparams.h"
#include "tmop_mass.h"

namespace tmop {

namespace {

// forward value contraction: X[D][N^d] -> V[D][Q^d] (tensor product of B);
// in place between two buffers, result in the returned one
template <int DIM, int N, int Q1, int NC>
__device__ double* fwd_val(const double* B, double* P0, double* P1, int lane) {
  if constexpr (DIM == 2) {
    for (int t = lane; t < NC * N * Q1; t += 32) {  // (c, j, q0)
      const int q0 = t % Q1, j = (t / Q1) % N, c = t / (Q1 * N);
      double s = 0.0;
#pragma unroll
      for (int i = 0; i < N; ++i) s = fma(P0[(c * N + j) * N + i], B[q0 * N + i], s);
      P1[(c * N + j) * Q1 + q0] = s;
    }
    __syncwarp();
    for (int t = lane; t < NC * Q1 * Q1; t += 32) {  // (c, q1, q0)
      const int q0 = t % Q1, q1 = (t / Q1) % Q1, c = t / (Q1 * Q1);
      double s = 0.0;
#pragma unroll
      for (int j = 0; j < N; ++j) s = fma(P1[(c * N + j) * Q1 + q0], B[q1 * N + j], s);
      P0[(c * Q1 + q1) * Q1 + q0] = s;
    }
    __syncwarp();
    return P0;
  } else {
    for (int t = lane; t < NC * N * N * Q1; t += 32) {  // (c, l, j, q0)
      const int q0 = t % Q1, lj = (t / Q1) % (N * N), c = t / (Q1 * N * N);
      double s = 0.0;
#pragma unroll
      for (int i = 0; i < N; ++i) s = fma(P0[(c * N * N + lj) * N + i], B[q0 * N + i], s);
      P1[(c * N * N + lj) * Q1 + q0] = s;
    }
    __syncwarp();
    for (int t = lane; t < NC * N * Q1 * Q1; t += 32) {  // (c, l, q1, q0)
      const int q0 = t % Q1, q1 = (t / Q1) % Q1, l = (t / (Q1 * Q1)) % N, c = t / (Q1 * Q1 * N);
      double s = 0.0;
#pragma unroll
      for (int j = 0; j < N; ++j) s = fma(P1[((c * N + l) * N + j) * Q1 + q0], B[q1 * N + j], s);
      P0[((c * N + l) * Q1 + q1) * Q1 + q0] = s;
    }
    __syncwarp();
    for (int t = lane; t < NC * Q1 * Q1 * Q1; t += 32) {  // (c, q2, q1, q0)
      const int q01 = t % (Q1 * Q1), q2 = (t / (Q1 * Q1)) % Q1, c = t / (Q1 * Q1 * Q1);
      double s = 0.0;
#pragma unroll
      for (int l = 0; l < N; ++l) s = fma(P0[(c * N + l) * Q1 * Q1 + q01], B[q2 * N + l], s);
      P1[(c * Q1 + q2) * Q1 * Q1 + q01] = s;
    }
    __syncwarp();
    return P1;
  }
}

// adjoint value contraction: R[D][Q^d] (in `Rb`) -> Y[D][N^d], returned buffer
template <int DIM, int N, int Q1, int NC>
__device__ double* adj_val(const double* B, double* Rb, double* Ob, int lane) {
  if constexpr (DIM == 2) {
    for (int t = lane; t < NC * N * Q1; t += 32) {  // (c, j, q0)
      const int q0 = t % Q1, j = (t / Q1) % N, c = t / (Q1 * N);
      double s = 0.0;
#pragma unroll
      for (int q1 = 0; q1 < Q1; ++q1) s = fma(Rb[(c * Q1 + q1) * Q1 + q0], B[q1 * N + j], s);
      Ob[(c * N + j) * Q1 + q0] = s;
    }
    __syncwarp();
    for (int t = lane; t < NC * N * N; t += 32) {  // (c, j, i)
      const int i = t % N, j = (t / N) % N, c = t / (N * N);
      double s = 0.0;
#pragma unroll
      for (int q0 = 0; q0 < Q1; ++q0) s = fma(Ob[(c * N + j) * Q1 + q0], B[q0 * N + i], s);
      Rb[(c * N + j) * N + i] = s;
    }
    __syncwarp();
    return Rb;
  } else {
    for (int t = lane; t < NC * N * Q1 * Q1; t += 32) {  // (c, l, q1, q0)
      const int q01 = t % (Q1 * Q1), l = (t / (Q1 * Q1)) % N, c = t / (Q1 * Q1 * N);
      double s = 0.0;
#pragma unroll
      for (int q2 = 0; q2 < Q1; ++q2) s = fma(Rb[(c * Q1 + q2) * Q1 * Q1 + q01], B[q2 * N + l], s);
      Ob[(c * N + l) * Q1 * Q1 + q01] = s;
    }
    __syncwarp();
    for (int t = lane; t < NC * N * N * Q1; t += 32) {  // (c, l, j, q0)
      const int q0 = t % Q1, j = (t / Q1) % N, l = (t / (Q1 * N)) % N, c = t / (Q1 * N * N);
      double s = 0.0;
#pragma unroll
      for (int q1 = 0; q1 < Q1; ++q1) s = fma(Ob[((c * N + l) * Q1 + q1) * Q1 + q0], B[q1 * N + j], s);
      Rb[((c * N + l) * N + j) * Q1 + q0] = s;
    }
    __syncwarp();
    for (int t = lane; t < NC * N * N * N; t += 32) {  // (c, l, j, i)
      const int i = t % N, lj = (t / N) % (N * N), c = t / (N * N * N);
      double s = 0.0;
#pragma unroll
      for (int q0 = 0; q0 < Q1; ++q0) s = fma(Rb[(c * N * N + lj) * Q1 + q0], B[q0 * N + i], s);
      Ob[(c * N * N + lj) * N + i] = s;
    }
    __syncwarp();
    return Ob;
  }
}

constexpr int kMassWarps = 4;  // static shared memory stays under 48 KB for every (n, q)

template <int DIM, int N, int Q1>
struct MassShape {
  static constexpr int NDOF = DIM == 2 ? N * N : N * N * N;
  static constexpr int QP = DIM == 2 ? Q1 * Q1 : Q1 * Q1 * Q1;
  static constexpr int T0 = DIM * (DIM == 2 ? (N * N > Q1 * Q1 ? N * N : Q1 * Q1)
                                           : (N * N * N > N * Q1 * Q1 ? N * N * N : N * Q1 * Q1));
  static constexpr int T1 = DIM * (DIM == 2 ? N * Q1 : (N * N * Q1 > Q1 * Q1 * Q1 ? N * N * Q1 : Q1 * Q1 * Q1));
  static constexpr int BUF = (DIM == 2) ? (T0 > T1 ? T0 : T1) : (T0 > T1 ? T0 : T1);
};

template <int DIM, int N, int Q1, int MODE>
__global__ void __launch_bounds__(kMassWarps * 32) mass_kernel(const MassParams p) {
  using S = MassShape<DIM, N, Q1>;
  constexpr int NDOF = S::NDOF, QP = S::QP;
  __shared__ double sB[kMaxQ * kMaxN], sw[kMaxQ];
  __shared__ double buf[kMassWarps][2][S::BUF];
  __shared__ double red[kMassWarps];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int t = threadIdx.x; t < Q1 * N; t += blockDim.x) sB[t] = p.B[t];
  for (int t = threadIdx.x; t < Q1; t += blockDim.x) sw[t] = p.w1[t];
  __syncthreads();
  double* P0 = buf[warp][0];
  double* P1 = buf[warp][1];
  double acc = 0.0;
  NodeMap<N> nodes(p.elem_nodes, p.sx, p.sy, DIM == 3 ? N - 1 : 1);
  const int ecount = p.elist ? p.ecount : p.nelem;
  for (int ei = blockIdx.x * kMassWarps + warp; ei < ecount; ei += gridDim.x * kMassWarps) {
    const int e = p.elist ? __ldg(p.elist + ei) : ei;
    nodes.element(e, NDOF);
    for (int t = lane; t < NDOF; t += 32) {
      const int g = nodes(t);
#pragma unroll
      for (int c = 0; c < DIM; ++c) {
        const size_t dof = (size_t)c * p.nnode + g;
        double u;
        if (MODE == 2) u = (p.fixed && __ldg(p.fixed + dof)) ? 0.0 : __ldg(p.v + dof);
        else u = __ldg(p.x + dof) - __ldg(p.x0 + dof);
        P0[c * NDOF + t] = u;
      }
    }
    __syncwarp();
    double* V = fwd_val<DIM, N, Q1, DIM>(sB, P0, P1, lane);
    double* O = V == P0 ? P1 : P0;
    for (int q = lane; q < QP; q += 32) {
      const int q0 = q % Q1, q1 = (q / Q1) % Q1;
      double wq = sw[q0] * sw[q1];
      if (DIM == 3) wq *= sw[q / (Q1 * Q1)];
      const double dw = p.detW_qp ? __ldg(p.detW_qp + (size_t)e * QP + q) : p.detW;
      const double s = wq * dw * p.delta;
      if (MODE == 0) {
        double u2 = 0.0;
#pragma unroll
        for (int c = 0; c < DIM; ++c) u2 = fma(V[c * QP + q], V[c * QP + q], u2);
        acc = fma(s, u2, acc);
      } else {
#pragma unroll
        for (int c = 0; c < DIM; ++c) V[c * QP + q] *= 2.0 * s;
      }
    }
    __syncwarp();
    if (MODE != 0) {
      double* Y = adj_val<DIM, N, Q1, DIM>(sB, V, O, lane);
      for (int t = lane; t < NDOF; t += 32) {
        const int g = nodes(t);
#pragma unroll
        for (int c = 0; c < DIM; ++c) {
          const size_t dof = (size_t)c * p.nnode + g;
          if (p.fixed && __ldg(p.fixed + dof)) continue;
          atomicAdd(p.y + dof, Y[c * NDOF + t]);
        }
      }
      __syncwarp();
    }
  }
  if (MODE == 0) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) red[warp] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
      double sacc = 0.0;
      for (int w = 0; w < kMassWarps; ++w) sacc += red[w];
      p.part[blockIdx.x] = sacc;
    }
  }
}

template <int DIM, int N, int Q1, int MODE>
int launch_mass(const MassParams& p, int grid, void* stream) {
  mass_kernel<DIM, N, Q1, MODE><<<grid, kMassWarps * 32, 0, (cudaStream_t)stream>>>(p);
  return (int)cudaGetLastError();
}

#define TMOP_MASS(DIM, N, Q)                                                                         \
  {DIM, N, Q, {launch_mass<DIM, N, Q, 0>, launch_mass<DIM, N, Q, 1>, launch_mass<DIM, N, Q, 2>}}

struct MassEntry {
  int dim, n, q;
  mass_launch_fn fn[3];
};

const MassEntry kMass[] = {
    TMOP_MASS(2, 2, 2), TMOP_MASS(2, 2, 3), TMOP_MASS(2, 3, 3), TMOP_MASS(2, 3, 4), TMOP_MASS(2, 3, 5),
    TMOP_MASS(2, 4, 4), TMOP_MASS(2, 4, 5), TMOP_MASS(2, 4, 6), TMOP_MASS(2, 5, 5), TMOP_MASS(2, 5, 6),
    TMOP_MASS(3, 2, 2), TMOP_MASS(3, 2, 3), TMOP_MASS(3, 3, 3), TMOP_MASS(3, 3, 4), TMOP_MASS(3, 4, 4),
    TMOP_MASS(3, 4, 5), TMOP_MASS(3, 5, 5), TMOP_MASS(3, 5, 6),
};

}  // namespace

mass_launch_fn find_mass(int dim, int n, int q, int mode) {
  for (const MassEntry& m : kMass)
    if (m.dim == dim && m.n == n && m.q == q) return m.fn[mode];
  return nullptr;
}

int mass_grid(int nelem) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int need = (nelem + kMassWarps - 1) / kMassWarps;
  const int full = 2 * (sms > 0 ? sms : 1);
  int g = need < full ? need : full;
  return g < 1 ? 1 : g;
}

}  // namespace tmop
