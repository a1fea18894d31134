// Jacobians A(x_q) = sum_i x_i grad phi_i(xi_q) at every quadrature point
// (eq. (2.2)) and the target sets built from the positions of a mesh
// (Section 3.1: W2 from the mesh measure of eq. (3.1), W3 = det(A(x0))^{1/d} I;
// Section 4.3.2: W0 = A(x_init)). These run once per setup, so the Jacobian
// kernel is the plain form: one thread per (element, point), a direct sum
// over the element's nodes with the tensor-product basis gradient.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "tmop_device.cuh"
#include "tmop_targets.h"

namespace tmop {

namespace {

__global__ void k_jacobians(const JacParams p) {
  const int Q1 = p.q1, N = p.n, D = p.dim;
  const int Q = D == 2 ? Q1 * Q1 : Q1 * Q1 * Q1, NDOF = D == 2 ? N * N : N * N * N;
  const size_t cnt = (size_t)p.nelem * Q;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < cnt; idx += (size_t)gridDim.x * blockDim.x) {
    const int e = (int)(idx / Q), qp = (int)(idx % Q);
    const int qa = qp % Q1, qb = (qp / Q1) % Q1, qc = qp / (Q1 * Q1);
    double A[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int t = 0; t < NDOF; ++t) {
      const int i = t % N, j = (t / N) % N, l = t / (N * N);
      int g;
      if (p.sx > 0) {
        const int k = N - 1, Nx = k * p.sx + 1, Ny = k * p.sy + 1;
        const int ex = e % p.sx, ey = (e / p.sx) % p.sy, ez = e / (p.sx * p.sy);
        // 3D: element layers of k lattice planes; 2D: ez is the grid of a stack
        g = (D == 3 ? ((ez * k + l) * Ny + ey * k + j) : (ez * Ny + ey * k + j)) * Nx + ex * k + i;
      } else {
        g = p.elem_nodes[(size_t)e * NDOF + t];
      }
      double dphi[3];
      if (D == 2) {
        dphi[0] = p.G[qa * N + i] * p.B[qb * N + j];
        dphi[1] = p.B[qa * N + i] * p.G[qb * N + j];
      } else {
        const double bi = p.B[qa * N + i], bj = p.B[qb * N + j], bl = p.B[qc * N + l];
        dphi[0] = p.G[qa * N + i] * bj * bl;
        dphi[1] = bi * p.G[qb * N + j] * bl;
        dphi[2] = bi * bj * p.G[qc * N + l];
      }
      for (int a = 0; a < D; ++a) {
        const double xa = p.x[(size_t)a * p.nnode + g];
        for (int b = 0; b < D; ++b) A[a * D + b] = fma(xa, dphi[b], A[a * D + b]);
      }
    }
    double* out = p.J + idx * D * D;
    for (int k = 0; k < D * D; ++k) out[k] = A[k];
  }
}

template <int D>
__global__ void k_targets(int kind, const double* J, size_t cnt, double* Winv, double* detW, int* bad) {
  constexpr int DD = D * D;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < cnt; idx += (size_t)gridDim.x * blockDim.x) {
    double M[DD], C[DD];
    for (int k = 0; k < DD; ++k) M[k] = J[idx * DD + k];
    const double dt = det_m<D>(M);
    if (!(dt > 0.0)) {
      atomicAdd(bad, 1);
      continue;
    }
    double* Wi = Winv + idx * DD;
    if (kind == 0) {  // W = A: W^-1 = cof(A)^t / det A
      cof_m<D>(M, C);
      for (int a = 0; a < D; ++a)
        for (int b = 0; b < D; ++b) Wi[a * D + b] = C[b * D + a] / dt;
      detW[idx] = dt;
    } else {          // W = s I, s = det(A)^{1/d}; det W = det A
      const double s = D == 2 ? sqrt(dt) : cbrt(dt);
      for (int k = 0; k < DD; ++k) Wi[k] = k % (D + 1) == 0 ? 1.0 / s : 0.0;
      detW[idx] = dt;
    }
  }
}

struct Weights1D {
  double w[kMaxQ];
};

// one block: sum over elements (in order, strided by thread) of sum_q w_q det J
template <int D>
__global__ void k_measure(int q1, const double* J, size_t nelem, const Weights1D wt, double* out) {
  constexpr int DD = D * D;
  __shared__ double red[1024];
  const double* w1 = wt.w;
  const int Q = D == 2 ? q1 * q1 : q1 * q1 * q1;
  double s = 0.0;
  for (size_t e = threadIdx.x; e < nelem; e += blockDim.x)
    for (int qp = 0; qp < Q; ++qp) {
      double w = w1[qp % q1] * w1[(qp / q1) % q1];
      if (D == 3) w *= w1[qp / (q1 * q1)];
      s = fma(w, det_m<D>(J + (e * Q + qp) * DD), s);
    }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0];
}

}  // namespace

int jacobians(const JacParams& p, cudaStream_t s) {
  const int Q = p.dim == 2 ? p.q1 * p.q1 : p.q1 * p.q1 * p.q1;
  const size_t cnt = (size_t)p.nelem * Q;
  const size_t blocks = (cnt + 255) / 256;
  k_jacobians<<<(unsigned)(blocks < 65536 ? blocks : 65536), 256, 0, s>>>(p);
  return (int)cudaGetLastError();
}

int targets_from_jacobians(int dim, int kind, const double* J, size_t cnt, double* Winv, double* detW, int* bad,
                           cudaStream_t s) {
  const size_t blocks = (cnt + 255) / 256;
  const unsigned g = (unsigned)(blocks < 65536 ? (blocks > 0 ? blocks : 1) : 65536);
  if (dim == 2) k_targets<2><<<g, 256, 0, s>>>(kind, J, cnt, Winv, detW, bad);
  else k_targets<3><<<g, 256, 0, s>>>(kind, J, cnt, Winv, detW, bad);
  return (int)cudaGetLastError();
}

int mesh_measure(int dim, int q1, const double* J, size_t nelem, const double* w1, double* out, cudaStream_t s) {
  Weights1D wt;
  for (int i = 0; i < kMaxQ; ++i) wt.w[i] = i < q1 ? w1[i] : 0.0;
  if (dim == 2) k_measure<2><<<1, 1024, 0, s>>>(q1, J, nelem, wt, out);
  else k_measure<3><<<1, 1024, 0, s>>>(q1, J, nelem, wt, out);
  return (int)cudaGetLastError();
}

}  // namespace tmop
