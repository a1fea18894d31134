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

// ---------------------------------------------------------------- 3D compact records
// With dA = E_ac the direction dT = e_a w^T (w = row c of W^-1) touches row a
// of T only, and row a of cof T does not depend on row a of T, so the
// cofactor-derivative term of dP drops out of the row a of the response:
//   H[(a,b),(a,c)] = 2 mu_1 G_bc + tt_b P_c + cc_b Q_c,
//   P_c = 4 mu_11 tt_c + 2 mu_1t cc_c,   Q_c = 2 mu_1t tt_c + mu_tt cc_c,
// with tt = W^-1 T_a, cc = W^-1 (cof T)_a (rows a; W^-1 applied as a matrix
// to a vector) and G = W^-1 W^-t (G = I, tt = T_a, cc = (cof T)_a for W = I);
// the record's partials carry w det W. So one pass over the points gives all
// 3 x 6 fields (a, b <= c; twice the value for b != c), a few operations
// each, where the generic kernel rebuilds dP for every (a, c).
// The 18 contractions share their tables by direction: pair (b, c) uses
// BB, BG or GG in direction d as d is in neither, one or both of b and c. The
// z and y stages run per pair; after them, pairs with the same x table are
// added (x tables: GG for (0,0); BG for (0,1), (0,2); BB for (1,1), (1,2),
// (2,2)), so the x stage runs three times per component instead of six.
constexpr int kDiagCWarps = 8;

template <int N, int Q1>
struct DiagCCfg {
  static constexpr int QP = Q1 * Q1 * Q1, QQ = Q1 * Q1, NDOF = N * N * N;
  static constexpr int FS = 6 * QP;          // fields of one component: [pair][q]
  static constexpr int US = 6 * N * QQ;      // z-stage outputs: [pair][l][q1][q0]
  static constexpr int PER_WARP = 3 * FS + US;
  static_assert(3 * N * N * Q1 <= FS, "merged y-stage outputs must fit in one component's fields");
  static constexpr size_t smem_bytes() { return sizeof(float) * kDiagCWarps * PER_WARP; }
};

// pair k = 0..5 -> (b, c): (0,0) (0,1) (1,1) (0,2) (1,2) (2,2)
__host__ __device__ constexpr int pair_b(int k) { return k == 0 ? 0 : k == 1 ? 0 : k == 2 ? 1 : k == 3 ? 0 : k == 4 ? 1 : 2; }
__host__ __device__ constexpr int pair_c(int k) { return k < 1 ? 0 : k < 3 ? 1 : 2; }
// table of pair k in direction d: 0 BB, 1 BG, 2 GG
__host__ __device__ constexpr int pair_tab(int k, int d) { return (pair_b(k) == d) + (pair_c(k) == d); }

template <int N, int Q1>
__global__ void __launch_bounds__(kDiagCWarps * 32, 2) diag_compact_kernel(const DiagParams p) {
  using Cfg = DiagCCfg<N, Q1>;
  constexpr int QP = Cfg::QP, QQ = Cfg::QQ, NDOF = Cfg::NDOF;
  constexpr int NPL = (QP + 31) / 32;
  extern __shared__ __align__(16) float dsm[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float* F = dsm + warp * Cfg::PER_WARP;   // [a][pair][q]
  float* U = F + 3 * Cfg::FS;              // [pair][l][q1][q0]
  // the 1D table products BB, BG, GG ([q][i]) in FP32 registers
  float tb[3][Q1 * N];
#pragma unroll
  for (int t = 0; t < Q1 * N; ++t) {
    const double b = p.B[t], g = p.G[t];
    tb[0][t] = (float)(b * b);
    tb[1][t] = (float)(b * g);
    tb[2][t] = (float)(g * g);
  }
  float Wi[9], Gm[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) Wi[i] = p.identity ? (i % 4 == 0 ? 1.f : 0.f) : (float)p.Winv[i];
#pragma unroll
  for (int b = 0; b < 3; ++b)
#pragma unroll
    for (int c = 0; c < 3; ++c)
      Gm[b * 3 + c] = fmaf(Wi[b * 3], Wi[c * 3], fmaf(Wi[b * 3 + 1], Wi[c * 3 + 1], Wi[b * 3 + 2] * Wi[c * 3 + 2]));
  const float* H = static_cast<const float*>(p.pa);
  NodeMap<N> nodes(p.elem_nodes, p.sx, p.sy, N - 1);
  const int ecount = p.elist ? p.ecount : p.nelem;
  for (int ei = blockIdx.x * kDiagCWarps + warp; ei < ecount; ei += gridDim.x * kDiagCWarps) {
    const int e = p.elist ? __ldg(p.elist + ei) : ei;
    nodes.element(e, NDOF);
    const float* He = H + (size_t)e * p.pa_stride;
    // ---- the 18 fields at every point
#pragma unroll
    for (int k = 0; k < NPL; ++k) {
      const int q = lane + 32 * k;
      if (q < QP) {
        float T[9], C[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) T[i] = __ldg(He + (size_t)i * QP + q);
        const float m1 = __ldg(He + (size_t)9 * QP + q), m11 = __ldg(He + (size_t)11 * QP + q);
        const float m1t = __ldg(He + (size_t)12 * QP + q), mtt = __ldg(He + (size_t)13 * QP + q);
        cof_m<3>(T, C);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          float tt[3], cc[3], P[3], Q[3];
#pragma unroll
          for (int b = 0; b < 3; ++b) {
            tt[b] = fmaf(Wi[b * 3], T[a * 3], fmaf(Wi[b * 3 + 1], T[a * 3 + 1], Wi[b * 3 + 2] * T[a * 3 + 2]));
            cc[b] = fmaf(Wi[b * 3], C[a * 3], fmaf(Wi[b * 3 + 1], C[a * 3 + 1], Wi[b * 3 + 2] * C[a * 3 + 2]));
          }
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            P[c] = fmaf(4.f * m11, tt[c], 2.f * m1t * cc[c]);
            Q[c] = fmaf(2.f * m1t, tt[c], mtt * cc[c]);
          }
          float* Fa = F + a * Cfg::FS + q;
#pragma unroll
          for (int k2 = 0; k2 < 6; ++k2) {
            const int b = pair_b(k2), c = pair_c(k2);
            const float h = fmaf(2.f * m1, Gm[b * 3 + c], fmaf(tt[b], P[c], cc[b] * Q[c]));
            Fa[k2 * QP] = b == c ? h : 2.f * h;
          }
        }
      }
    }
    __syncwarp();
#pragma unroll 1
    for (int a = 0; a < 3; ++a) {
      float* Fa = F + a * Cfg::FS;
      // ---- z stage, per pair: U[pair][l][q01] = sum_q2 F[pair][q2][q01] Tz[q2][l]
#pragma unroll
      for (int k2 = 0; k2 < 6; ++k2) {
        const float* Tz = tb[pair_tab(k2, 2)];
#pragma unroll
        for (int r = 0; r < (QQ + 31) / 32; ++r) {
          const int q01 = lane + 32 * r;
          if (q01 < QQ) {
            float f[Q1];
#pragma unroll
            for (int q2 = 0; q2 < Q1; ++q2) f[q2] = Fa[k2 * QP + q2 * QQ + q01];
#pragma unroll
            for (int l = 0; l < N; ++l) {
              float s = 0.f;
#pragma unroll
              for (int q2 = 0; q2 < Q1; ++q2) s = fmaf(f[q2], Tz[q2 * N + l], s);
              U[(k2 * N + l) * QQ + q01] = s;
            }
          }
        }
      }
      __syncwarp();
      // ---- y stage, per pair, summed by x table into W[g][l][j][q0] (in Fa)
#pragma unroll
      for (int r = 0; r < (N * Q1 + 31) / 32; ++r) {
        const int it = lane + 32 * r;     // (l, q0)
        float w3[3][N];
#pragma unroll
        for (int g = 0; g < 3; ++g)
#pragma unroll
          for (int j = 0; j < N; ++j) w3[g][j] = 0.f;
        if (it < N * Q1) {
          const int l = it / Q1, q0 = it % Q1;
#pragma unroll
          for (int k2 = 0; k2 < 6; ++k2) {
            const float* Ty = tb[pair_tab(k2, 1)];
            float u[Q1];
#pragma unroll
            for (int q1 = 0; q1 < Q1; ++q1) u[q1] = U[(k2 * N + l) * QQ + q1 * Q1 + q0];
            const int g = pair_tab(k2, 0);
#pragma unroll
            for (int j = 0; j < N; ++j) {
              float s = w3[g][j];
#pragma unroll
              for (int q1 = 0; q1 < Q1; ++q1) s = fmaf(u[q1], Ty[q1 * N + j], s);
              w3[g][j] = s;
            }
          }
        }
        __syncwarp();
        if (it < N * Q1) {
          const int l = it / Q1, q0 = it % Q1;
#pragma unroll
          for (int g = 0; g < 3; ++g)
#pragma unroll
            for (int j = 0; j < N; ++j) Fa[((g * N + l) * N + j) * Q1 + q0] = w3[g][j];
        }
      }
      __syncwarp();
      // ---- x stage per group: Y[l][j][i] = sum_g sum_q0 W[g][l][j][q0] Tx_g[q0][i], then the scatter
#pragma unroll
      for (int r = 0; r < (N * N + 31) / 32; ++r) {
        const int lj = lane + 32 * r;
        if (lj < N * N) {
          float y[N];
#pragma unroll
          for (int i = 0; i < N; ++i) y[i] = 0.f;
#pragma unroll
          for (int g = 0; g < 3; ++g) {
            float w[Q1];
#pragma unroll
            for (int q0 = 0; q0 < Q1; ++q0) w[q0] = Fa[(g * N * N + lj) * Q1 + q0];
#pragma unroll
            for (int i = 0; i < N; ++i)
#pragma unroll
              for (int q0 = 0; q0 < Q1; ++q0) y[i] = fmaf(w[q0], tb[g][q0 * N + i], y[i]);
          }
#pragma unroll
          for (int i = 0; i < N; ++i) atomicAdd(p.diag + (size_t)a * p.nnode + nodes(lj * N + i), (double)y[i]);
        }
      }
      __syncwarp();
    }
  }
}

template <int N, int Q1>
int launch_diag_compact(const DiagParams& p, void* stream) {
  static int grid = 0;   // (per instantiation: the resident blocks on every SM)
  const size_t smem = DiagCCfg<N, Q1>::smem_bytes();
  if (grid == 0) {
    if (cudaFuncSetAttribute(diag_compact_kernel<N, Q1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
      return (int)cudaErrorInvalidConfiguration;
    int per_sm = 0, dev = 0, sms = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, diag_compact_kernel<N, Q1>, kDiagCWarps * 32, smem) !=
            cudaSuccess || per_sm < 1)
      return (int)cudaErrorInvalidConfiguration;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    grid = per_sm * (sms > 0 ? sms : 1);
  }
  const int need = (p.nelem + kDiagCWarps - 1) / kDiagCWarps;
  diag_compact_kernel<N, Q1><<<need < grid ? need : grid, kDiagCWarps * 32, smem, (cudaStream_t)stream>>>(p);
  return (int)cudaGetLastError();
}

template <int DIM, int N, int Q1, class R>
int launch_diag(const DiagParams& p, int grid, void* stream) {
  if constexpr (DIM == 3 && sizeof(R) == 4)
    if (p.compact && p.delta == 0.0) return launch_diag_compact<N, Q1>(p, stream);
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

// streaming passes: 8 blocks of 256 threads per SM
int stream_grid() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return 8 * (sms > 0 ? sms : 1);
}

int diag_finish(double* diag, const uint8_t* fixed, size_t n, cudaStream_t s) {
  k_diag_fix<<<stream_grid(), 256, 0, s>>>(diag, fixed, n);
  return (int)cudaGetLastError();
}

int diag_inverse(const double* diag, double* minv, size_t n, double floor_abs, cudaStream_t s) {
  k_diag_inverse<<<stream_grid(), 256, 0, s>>>(diag, minv, n, floor_abs);
  return (int)cudaGetLastError();
}

}  // namespace tmop
