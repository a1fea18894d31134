// Diagonal of the partially assembled Hessian (for Jacobi preconditioning of
// the Newton systems of Section 3.4), from the packed per-point Hessians or,
// in 3D, from the compact records the entries are rebuilt from:
//   diag_{i,a} = sum_E sum_q sum_{b,c} H_q[(a,b),(a,c)] d_b phi_i(x_q) d_c phi_i(x_q)
// (+ 2 delta w_q det W phi_i(x_q)^2 for the restricted-movement term). The
// product d_b phi_i d_c phi_i is separable: in direction d it is the 1D
// product of (G if d == b else B) and (G if d == c else B), so every (a, b, c)
// term is one sum-factorised contraction of a per-point scalar with three
// per-direction tables. One warp per element; the contractions run in the
// precision of the stored values (FP32 for the FP32 forms: the diagonal only
// preconditions, and GB300's FP64 pipe is 64x narrower), the accumulation
// into diag in FP64.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "tmop_device.cuh"
#include "tmop_diag.h"
#include "tmop_kparams.h"

namespace tmop {

namespace {

constexpr int kDiagWarps = 4;

__device__ __forceinline__ float fmaA(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fmaA(double a, double b, double c) { return fma(a, b, c); }

// Y[n^DIM] += sum_q R[q] prod_d T_d[q_d][i_d]; R in `r` (QP values), tables T0,
// T1, T2 ([Q1][N]), scratch U, V.
template <int DIM, int N, int Q1, class A>
__device__ void contract_add(const A* r, const A* T0, const A* T1, const A* T2, A* U, A* V, A* Y, int lane) {
  if constexpr (DIM == 2) {
    for (int t = lane; t < N * Q1; t += 32) {  // U[j][q0] = sum_q1 R[q1][q0] T1[q1][j]
      const int q0 = t % Q1, j = t / Q1;
      A s = A(0);
#pragma unroll
      for (int q1 = 0; q1 < Q1; ++q1) s = fmaA(r[q1 * Q1 + q0], T1[q1 * N + j], s);
      U[j * Q1 + q0] = s;
    }
    __syncwarp();
    for (int t = lane; t < N * N; t += 32) {  // Y[j][i] += sum_q0 U[j][q0] T0[q0][i]
      const int i = t % N, j = t / N;
      A s = A(0);
#pragma unroll
      for (int q0 = 0; q0 < Q1; ++q0) s = fmaA(U[j * Q1 + q0], T0[q0 * N + i], s);
      Y[t] += s;
    }
    __syncwarp();
  } else {
    constexpr int QQ = Q1 * Q1;
    for (int t = lane; t < N * QQ; t += 32) {  // U[l][q1][q0] = sum_q2 R[q2][q1][q0] T2[q2][l]
      const int q01 = t % QQ, l = t / QQ;
      A s = A(0);
#pragma unroll
      for (int q2 = 0; q2 < Q1; ++q2) s = fmaA(r[q2 * QQ + q01], T2[q2 * N + l], s);
      U[l * QQ + q01] = s;
    }
    __syncwarp();
    for (int t = lane; t < N * N * Q1; t += 32) {  // V[l][j][q0] = sum_q1 U[l][q1][q0] T1[q1][j]
      const int q0 = t % Q1, j = (t / Q1) % N, l = t / (Q1 * N);
      A s = A(0);
#pragma unroll
      for (int q1 = 0; q1 < Q1; ++q1) s = fmaA(U[l * QQ + q1 * Q1 + q0], T1[q1 * N + j], s);
      V[(l * N + j) * Q1 + q0] = s;
    }
    __syncwarp();
    for (int t = lane; t < N * N * N; t += 32) {  // Y[l][j][i] += sum_q0 V[l][j][q0] T0[q0][i]
      const int i = t % N, lj = t / N;
      A s = A(0);
#pragma unroll
      for (int q0 = 0; q0 < Q1; ++q0) s = fmaA(V[lj * Q1 + q0], T0[q0 * N + i], s);
      Y[t] += s;
    }
    __syncwarp();
  }
}

// Row a of the response to dA = E_ac at point q from a 3D compact record
// (T, then w det W times mu_1, mu_t, mu_11, mu_1t, mu_tt), in FP32 like the
// record: out[b] = H[(a,b),(a,c)] = [w det W (d^2mu/dT^2 : E_ac W^-1) W^-t]_ab.
template <class R>
__device__ void compact_row(const DiagParams& p, const R* He, int QP, int q, int a, int c, float out[3]) {
  MetricLin<3, float> L;
#pragma unroll
  for (int i = 0; i < 9; ++i) L.T[i] = (float)He[(size_t)i * QP + q];
  cof_m<3>(L.T, L.C);
  L.m1 = (float)He[(size_t)9 * QP + q];
  L.mt = (float)He[(size_t)10 * QP + q];
  L.m11 = (float)He[(size_t)11 * QP + q];
  L.m1t = (float)He[(size_t)12 * QP + q];
  L.mtt = (float)He[(size_t)13 * QP + q];
  // (a, c) are run-time values: every index below is a compile-time one
  // with a select, so the small arrays stay in registers
  float w[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) w[k] = p.identity ? (k == c ? 1.0f : 0.0f) : (float)p.Winv[c * 3 + k];
  float dT[9], S[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) dT[i] = (i / 3 == a) ? w[i % 3] : 0.0f;
  L.dP(dT, S);
  float Sa[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) Sa[k] = a == 0 ? S[k] : (a == 1 ? S[3 + k] : S[6 + k]);
#pragma unroll
  for (int b = 0; b < 3; ++b) {
    float v = 0.0f;
    if (p.identity) {
      v = Sa[b];
    } else {
#pragma unroll
      for (int k = 0; k < 3; ++k) v = fmaf(Sa[k], (float)p.Winv[b * 3 + k], v);
    }
    out[b] = v;
  }
}

template <int DIM, int N, int Q1, class R>
__global__ void __launch_bounds__(kDiagWarps * 32) diag_kernel(const DiagParams p) {
  constexpr int NDOF = DIM == 2 ? N * N : N * N * N, QP = DIM == 2 ? Q1 * Q1 : Q1 * Q1 * Q1;
  constexpr int DD = DIM * DIM, NS = DD * (DD + 1) / 2;
  constexpr int UQ = DIM == 2 ? N * Q1 : N * Q1 * Q1, VQ = DIM == 2 ? 1 : N * N * Q1;
  // tables: B, G and the three products BB, BG, GG ([Q1][N] each)
  using A = R;   // arithmetic of the contractions
  __shared__ A tab[5][kMaxQ * kMaxN];
  __shared__ A sw[kMaxQ];
  __shared__ A wr[kDiagWarps][QP], wu[kDiagWarps][UQ], wv[kDiagWarps][VQ], wy[kDiagWarps][NDOF];
  // compact records (3D): entries b = 0..2 of row a of the response to E_ac
  __shared__ float whh[kDiagWarps][DIM == 3 ? 3 * QP : 1];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int t = threadIdx.x; t < Q1 * N; t += blockDim.x) {
    const double b = p.B[t], g = p.G[t];
    tab[0][t] = A(b * b);
    tab[1][t] = A(b * g);
    tab[2][t] = A(g * g);
  }
  for (int t = threadIdx.x; t < Q1; t += blockDim.x) sw[t] = A(p.w1[t]);
  __syncthreads();
  A *r = wr[warp], *U = wu[warp], *V = wv[warp], *Y = wy[warp];
  const R* H = static_cast<const R*>(p.pa);
  NodeMap<N> nodes(p.elem_nodes, p.sx, p.sy, DIM == 3 ? N - 1 : 1);
  const int ecount = p.elist ? p.ecount : p.nelem;
  for (int ei = blockIdx.x * kDiagWarps + warp; ei < ecount; ei += gridDim.x * kDiagWarps) {
    const int e = p.elist ? __ldg(p.elist + ei) : ei;
    nodes.element(e, NDOF);
    const R* He = H + (size_t)e * p.pa_stride;
    for (int a = 0; a < DIM; ++a) {
      for (int t = lane; t < NDOF; t += 32) Y[t] = A(0);
      __syncwarp();
      // terms (b <= c): H[(a,b),(a,c)] (twice for b != c) against the 1D
      // table products; direction d uses tab[(d == b) + (d == c)]: BB, BG or GG
      for (int c = 0; c < DIM; ++c) {
        float* hh = whh[warp];
        if (DIM == 3 && p.compact) {  // the whole row of the response to E_ac at once
          for (int q = lane; q < QP; q += 32) {
            float row[3];
            compact_row(p, He, QP, q, a, c, row);
#pragma unroll
            for (int b = 0; b < 3; ++b) hh[b * QP + q] = row[b];
          }
          __syncwarp();
        }
        for (int b = 0; b <= c; ++b) {
          const A m = b == c ? A(1) : A(2);
          if (DIM == 3 && p.compact) {
            for (int q = lane; q < QP; q += 32) r[q] = m * (A)hh[b * QP + q];
          } else {
            // packed index of (row a*DIM+b, column a*DIM+c), row <= column
            const int rr = a * DIM + b, cc = a * DIM + c;
            const int s = rr * DD - rr * (rr - 1) / 2 + (cc - rr);
            for (int q = lane; q < QP; q += 32) r[q] = m * (A)He[(size_t)s * QP + q];
          }
          __syncwarp();
          const A* T0 = tab[(b == 0) + (c == 0)];
          const A* T1 = tab[(b == 1) + (c == 1)];
          const A* T2 = tab[(b == 2) + (c == 2)];
          contract_add<DIM, N, Q1, A>(r, T0, T1, T2, U, V, Y, lane);
        }
      }
      if (p.delta != 0.0) {  // restricted movement: 2 delta w det W phi_i^2 (B^2 in every direction)
        for (int q = lane; q < QP; q += 32) {
          const int q0 = q % Q1, q1 = (q / Q1) % Q1;
          double wq = (double)sw[q0] * (double)sw[q1];
          if (DIM == 3) wq *= (double)sw[q / (Q1 * Q1)];
          const double dw = p.detW_qp ? __ldg(p.detW_qp + (size_t)e * QP + q) : p.detW;
          r[q] = A(2.0 * p.delta * wq * dw);
        }
        __syncwarp();
        contract_add<DIM, N, Q1, A>(r, tab[0], tab[0], tab[0], U, V, Y, lane);
      }
      for (int t = lane; t < NDOF; t += 32) {
        const int g = nodes(t);
        atomicAdd(p.diag + (size_t)a * p.nnode + g, (double)Y[t]);
      }
      __syncwarp();
    }
  }
}

template <int DIM, int N, int Q1, class R>
int launch_diag(const DiagParams& p, int grid, void* stream) {
  diag_kernel<DIM, N, Q1, R><<<grid, kDiagWarps * 32, 0, (cudaStream_t)stream>>>(p);
  return (int)cudaGetLastError();
}

struct DiagEntry {
  int dim, n, q;
  diag_launch_fn f64, f32;
};

#define TMOP_DIAG(DIM, N, Q) {DIM, N, Q, launch_diag<DIM, N, Q, double>, launch_diag<DIM, N, Q, float>}

const DiagEntry kDiag[] = {
    TMOP_DIAG(2, 2, 2), TMOP_DIAG(2, 2, 3), TMOP_DIAG(2, 3, 3), TMOP_DIAG(2, 3, 4), TMOP_DIAG(2, 3, 5),
    TMOP_DIAG(2, 4, 4), TMOP_DIAG(2, 4, 5), TMOP_DIAG(2, 4, 6), TMOP_DIAG(2, 5, 5), TMOP_DIAG(2, 5, 6),
    TMOP_DIAG(3, 2, 2), TMOP_DIAG(3, 2, 3), TMOP_DIAG(3, 3, 3), TMOP_DIAG(3, 3, 4), TMOP_DIAG(3, 4, 4),
    TMOP_DIAG(3, 4, 5), TMOP_DIAG(3, 5, 5), TMOP_DIAG(3, 5, 6),
};

// fixed dofs: diagonal 1 (the operator is the identity there in the masked system)
__global__ void k_diag_fix(double* diag, const uint8_t* fixed, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    if (fixed && fixed[i]) diag[i] = 1.0;
}

// Jacobi inverse with a floor: minv = 1 / max(|diag|, floor * mean |diag|)
__global__ void k_diag_inverse(const double* diag, double* minv, size_t n, double floor_abs) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    minv[i] = 1.0 / fmax(fabs(diag[i]), floor_abs);
}

}  // namespace

diag_launch_fn find_diag(int dim, int n, int q, int fp32) {
  for (const DiagEntry& d : kDiag)
    if (d.dim == dim && d.n == n && d.q == q) return fp32 ? d.f32 : d.f64;
  return nullptr;
}

int diag_grid(int nelem) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int need = (nelem + kDiagWarps - 1) / kDiagWarps;
  const int full = 4 * (sms > 0 ? sms : 1);
  const int g = need < full ? need : full;
  return g < 1 ? 1 : g;
}

int diag_finish(double* diag, const uint8_t* fixed, size_t n, cudaStream_t s) {
  k_diag_fix<<<256, 256, 0, s>>>(diag, fixed, n);
  return (int)cudaGetLastError();
}

int diag_inverse(const double* diag, double* minv, size_t n, double floor_abs, cudaStream_t s) {
  k_diag_inverse<<<256, 256, 0, s>>>(diag, minv, n, floor_abs);
  return (int)cudaGetLastError();
}

}  // namespace tmop
