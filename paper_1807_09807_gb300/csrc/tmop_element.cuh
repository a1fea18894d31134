// Fused TMOP element kernel: one warp per element.
//
//   gather  x (and v) of the element's n^d nodes into shared memory
//   forward A(q) = sum_i x_i grad phi_i(q)            (eq. (2.2), sum factorised)
//   point   T = A W^-1, mu / P / dP                   (Table 3.1, Section 3.4)
//   adjoint y_i += sum_q w_q det W [S W^-t grad phi_i] (gradient formula of Section 3.4)
//   scatter FP64 atomics into the nodal output, fixed dofs skipped
//
// OP_ENERGY instead accumulates w_q det W mu and min det A in FP64 and writes
// one partial per block (reduced in a second, fixed-order pass);
// OP_ENERGY_GRAD does both: the gradient, and the energy partials from the
// mu it evaluates anyway.
#pragma once
#include "tmop_device.cuh"
#include "tmop_kparams.h"

namespace tmop {

template <int D, int N, int Q1>
struct Shape {
  static constexpr int NDOF = (D == 2) ? N * N : N * N * N;
  static constexpr int QP = (D == 2) ? Q1 * Q1 : Q1 * Q1 * Q1;
};

template <int a, int b> struct cmax { static constexpr int value = a > b ? a : b; };

// Shared-memory words (of type R) per warp for NC gathered components.
template <int D, int N, int Q1, int NC>
struct Buf {
  static constexpr int B0 = (D == 2) ? cmax<NC * N * N, 2 * NC * Q1 * Q1>::value
                                     : cmax<NC * N * N * N, 3 * NC * N * Q1 * Q1>::value;
  static constexpr int B1 = (D == 2) ? 2 * NC * N * Q1
                                     : cmax<2 * NC * N * N * Q1, 3 * NC * Q1 * Q1 * Q1>::value;
};

// Words of type R rounded up to a whole number of 16-byte units, so every
// per-warp buffer starts on a 16-byte boundary (bulk-copy destinations).
template <class R>
constexpr int round16(int words) {
  return ((words * (int)sizeof(R) + 15) / 16) * 16 / (int)sizeof(R);
}

template <int D, int N, int Q1, class R, int OP>
struct ElemCfg {
  // 3D Hessian action: x and v are contracted one after the other and only
  // A(x) is kept (buffer B2) while v runs through the stage buffers, so the
  // stage buffers hold D components; 2D contracts both at once (2D
  // components, no B2).
  static constexpr bool HV = OP == OP_HESS || OP == OP_GRAD_HESS;  // contracts x and v
  static constexpr bool SPLIT = HV && D == 3;
  static constexpr int NC = (HV && !SPLIT) ? 2 * D : D;
  static constexpr int B0 = round16<R>(Buf<D, N, Q1, NC>::B0);
  static constexpr int B1 = round16<R>(Buf<D, N, Q1, NC>::B1);
  static constexpr int B2 = SPLIT ? round16<R>(D * D * Shape<D, N, Q1>::QP) : 0;
  static constexpr int PER_WARP = (int)sizeof(R) * (B0 + B1 + B2);
  // up to 8 warps (elements in flight) per block within ~200 KB of shared
  // memory; the FP64 3D energy, gradient and stored-Hessian product (16 KB
  // per warp for order 3) run as 6-warp blocks, two per SM: 12 warps in
  // flight instead of 8 on the FP64 pipe (gradient -2 %, stored-Hessian
  // product -8 % on 48^3 order-3 hexes)
  static constexpr bool TWO = D == 3 && sizeof(R) == 8 && OP != OP_LINEARIZE && !HV &&
                              12 * PER_WARP <= 200 * 1024;
  static constexpr int WARPS = TWO ? 6
                                   : ((200 * 1024 / PER_WARP) >= 8 ? 8
                                                                   : ((200 * 1024 / PER_WARP) < 1 ? 1 : 200 * 1024 / PER_WARP));
  // FP64 3D with an even node count: contractions in the mirror basis, whose
  // normalised forward stages need the pivot tables and their products
  static constexpr bool EO = D == 3 && sizeof(R) == 8 && N % 2 == 0;
  static constexpr int EO_FWD = 4 * kMaxQ + 3 * Q1 * Q1 * Q1;                           // pivots, ratios, scales
  static constexpr int EO_ADJ = 2 * kMaxN * kMaxQ + 2 * kMaxN + 3 * N * Q1 * N + kMaxN;  // ratios, pivots, C, ysc
  // after the 1D tables: the product weight w_q0 w_q1 (w_q2) of every point
  static constexpr int WQ_OFF = 2 * kMaxQ * kMaxN + kMaxQ + (EO ? EO_FWD + EO_ADJ : 0);
  static constexpr int TABLE = round16<R>(WQ_OFF + Shape<D, N, Q1>::QP);
  static constexpr size_t smem_bytes() { return sizeof(R) * (TABLE + WARPS * (B0 + B1 + B2)); }
};

// Second term of a composite metric at one point: T2 = A W2^-1 and, for a
// direction dA, dT2 = dA W2^-1 (Section 4.2, eq. (4.1)).
template <int D, class R>
__device__ __forceinline__ void times_w2(const KParams& p, const R* M, R* out) {
#pragma unroll
  for (int a = 0; a < D; ++a)
#pragma unroll
    for (int b = 0; b < D; ++b) {
      R s = R(0);
#pragma unroll
      for (int c = 0; c < D; ++c) s = fma(M[a * D + c], R(p.Winv2[c * D + b]), s);
      out[a * D + b] = s;
    }
}

// Metrics not written in I1 = |T|^2 and tau = det T alone (mu302 also needs
// |cof T|^2, mu98 needs T - I): their second derivative comes from
// forward-mode dual numbers instead of MetricLin.
__device__ __forceinline__ bool metric_dual(int id) { return id == 302 || id == 98; }

// dP of metric `id` at T in direction dT (closed form, or dual numbers)
template <int D, class R>
__device__ __forceinline__ bool metric_dP(int id, const R* T, const R* dT, R* S) {
  constexpr int DD = D * D;
  if (metric_dual(id)) {
    Dual<R> Td[DD], Pd[DD], mud;
#pragma unroll
    for (int i = 0; i < DD; ++i) Td[i] = Dual<R>{T[i], dT[i]};
    const bool ok = metric_P<D>(id, Td, mud, Pd);
#pragma unroll
    for (int i = 0; i < DD; ++i) S[i] = Pd[i].d;
    return ok;
  }
  MetricLin<D, R> L;
  const bool ok = L.init(id, T);
  if (ok) L.dP(dT, S);
  return ok;
}

template <int D, int N, int Q1, class R, int OP>
__global__ void __launch_bounds__(ElemCfg<D, N, Q1, R, OP>::WARPS * 32, ElemCfg<D, N, Q1, R, OP>::TWO ? 2 : 0)
    elem_kernel(const KParams p) {
  using Cfg = ElemCfg<D, N, Q1, R, OP>;
  constexpr int NDOF = Shape<D, N, Q1>::NDOF, QP = Shape<D, N, Q1>::QP, DD = D * D;
  constexpr int WARPS = Cfg::WARPS;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  R* sB = reinterpret_cast<R*>(smem_raw);
  R* sG = sB + kMaxQ * kMaxN;
  R* sw = sG + kMaxQ * kMaxN;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  R* P0 = sB + Cfg::TABLE + warp * (Cfg::B0 + Cfg::B1 + Cfg::B2);
  R* P1 = P0 + Cfg::B0;
  R* P2 = P1 + Cfg::B1;  // A(x) of the split 3D Hessian action

  // FP64 3D kernels with an even node count contract in the mirror basis
  // (fwd3_eon / adj3_eon): sB, sG then hold the folded tables, followed by
  // the normalised maps' pivots, ratios, scale products and stage-2 tables
  constexpr bool EO = Cfg::EO;
  R* s_piv = sw + kMaxQ;
  R* s_rt = s_piv + 2 * kMaxQ;
  R* s_Sc = s_rt + 2 * kMaxQ;
  R* s_arat = s_Sc + 3 * Q1 * Q1 * Q1;
  R* s_apiv = s_arat + 2 * kMaxN * kMaxQ;
  R* s_C = s_apiv + 2 * kMaxN;
  R* s_ysc = s_C + 3 * N * Q1 * N;
  __shared__ int s_kf[2 * kMaxQ];
  __shared__ int s_aperm[2 * kMaxN * kMaxQ];
  if constexpr (EO) {
    folded_tables<N, Q1, R>(p.B, p.G, sB, sG, threadIdx.x, blockDim.x);
    __syncthreads();
    normalised_tables<N, Q1, R>(sB, sG, s_kf, s_rt, s_piv, s_Sc, threadIdx.x, blockDim.x);
    adjoint_tables<N, Q1, R>(sB, sG, s_aperm, s_arat, s_apiv, s_C, s_ysc, threadIdx.x, blockDim.x);
  } else {
    for (int t = threadIdx.x; t < Q1 * N; t += blockDim.x) {
      sB[t] = R(p.B[t]);
      sG[t] = R(p.G[t]);
    }
  }
  for (int t = threadIdx.x; t < Q1; t += blockDim.x) sw[t] = R(p.w1[t]);
  // point weights, rounded as (w_q0 w_q1) w_q2 in R: two multiplies per point
  // fewer on GB300's narrow FP64 pipe
  R* sWq = sB + Cfg::WQ_OFF;
  for (int t = threadIdx.x; t < QP; t += blockDim.x) {
    R w = R(p.w1[t % Q1]) * R(p.w1[(t / Q1) % Q1]);
    if constexpr (D == 3) w *= R(p.w1[t / (Q1 * Q1)]);
    sWq[t] = w;
  }
  R Wi[DD];
#pragma unroll
  for (int i = 0; i < DD; ++i) Wi[i] = R(p.Winv[i]);
  // FP32 3D kernels: the 1D tables in registers for the register-blocked stages
  constexpr bool RB = (D == 3) && sizeof(R) == 4;
  R tB[Q1 * N], tG[Q1 * N];
  if constexpr (RB) {
#pragma unroll
    for (int t = 0; t < Q1 * N; ++t) {
      tB[t] = R(p.B[t]);
      tG[t] = R(p.G[t]);
    }
  }
  __syncthreads();

  double accF = 0.0, accMin = INFINITY;
  const int nwarps_total = gridDim.x * WARPS;
  // (the product from compact records, OP_HESS_PA_C, is pac_kernel in tmop_pa_compact.cu)
  constexpr bool PA_APPLY = OP == OP_HESS_PA;
  constexpr bool EG = OP == OP_ENERGY_GRAD;                // gradient + energy partials
  constexpr bool GRADLIKE = OP == OP_GRADIENT || EG;
  constexpr int NSH = PA_APPLY ? D * D * (D * D + 1) / 2 : 1;
  static_assert(OP != OP_HESS_PA_C, "OP_HESS_PA_C runs in pac_kernel");
  static_assert(OP != OP_GRAD_HESS || sizeof(R) == 8, "the fused gradient + Hessian action is FP64");
  // its second 3D adjoint runs its stage 2 in the A(x) buffer
  static_assert(!(OP == OP_GRAD_HESS && D == 3) || 2 * D * N * N * Q1 <= Cfg::B2, "B2 too small");
  static_assert(OP != OP_LINEARIZE_C || D == 3, "compact records are 3D");
  NodeMap<N> nodes(p.elem_nodes, p.sx, p.sy, D == 3 ? N - 1 : 1);
  const int ecount = p.elist ? p.ecount : p.nelem;
  for (int ei = blockIdx.x * WARPS + warp; ei < ecount; ei += nwarps_total) {
    const int e = p.elist ? __ldg(p.elist + ei) : ei;
    nodes.element(e, NDOF);
    // Partially assembled product: the stored values of this lane's first
    // point are loaded now, so their latency overlaps the gather and the
    // v-contraction.
    R hpre[NSH];
    if constexpr (PA_APPLY) {
      if (lane < Shape<D, N, Q1>::QP) {
        const R* H0 = static_cast<const R*>(p.pa) + (size_t)e * p.pa_stride + lane;
#pragma unroll
        for (int t = 0; t < NSH; ++t) hpre[t] = __ldg(H0 + (size_t)t * Shape<D, N, Q1>::QP);
      }
    }
    // ---- gather. In FP32 the coordinates are taken relative to the element's
    // first node (in FP64) before rounding: A is translation invariant
    // (sum_i grad phi_i = 0), and this keeps the FP32 relative error of A at
    // the level of eps32 instead of eps32 |x| / h.
    double xref[D];
    if constexpr (sizeof(R) == 4 && !PA_APPLY) {
      const int g0 = nodes(0);
#pragma unroll
      for (int c = 0; c < D; ++c) xref[c] = __ldg(p.x + (size_t)c * p.nnode + g0);
    }
    for (int t = lane; t < NDOF; t += 32) {
      const int g = nodes(t);
      if constexpr (PA_APPLY) {
        // the partially assembled product needs only the direction v
#pragma unroll
        for (int c = 0; c < D; ++c) {
          const size_t dof = (size_t)c * p.nnode + g;
          const bool fx = p.fixed && __ldg(p.fixed + dof);
          P0[c * NDOF + t] = fx ? R(0) : (p.v32 ? R(__ldg(p.v32 + dof)) : from_f64<R>(__ldg(p.v + dof)));
        }
        continue;
      }
#pragma unroll
      for (int c = 0; c < D; ++c) {
        const double xv = __ldg(p.x + (size_t)c * p.nnode + g);
        if constexpr (sizeof(R) == 4) P0[c * NDOF + t] = from_f64<R>(xv - xref[c]);
        else P0[c * NDOF + t] = R(xv);
      }
      if constexpr (Cfg::HV && !Cfg::SPLIT) {
#pragma unroll
        for (int c = 0; c < D; ++c) {
          const size_t dof = (size_t)c * p.nnode + g;
          const bool fx = p.fixed && __ldg(p.fixed + dof);
          P0[(D + c) * NDOF + t] = fx ? R(0) : from_f64<R>(__ldg(p.v + dof));
        }
      }
    }
    __syncwarp();
    // ---- forward contraction: A (and dA) at every point
    if constexpr (Cfg::SPLIT) {
      // A(x) into P2 (P2 also serves as the first stage buffer), then v
      if constexpr (EO) {
        mirror3_all<D, N, R>(P0, lane);
        fwd3_eon<N, Q1, D, R>(s_kf, s_rt, P0, P2, lane);
        unfold_points<D * D, Q1, R>(P2, s_Sc, lane);
      } else if constexpr (RB) {
        fwd3_rb<N, Q1, D, R>(tB, tG, P0, P2, lane);
      } else {
        fwd3<N, Q1, D, R>(sB, sG, P0, P2, lane);
      }
      for (int t = lane; t < NDOF; t += 32) {
        const int g = nodes(t);
#pragma unroll
        for (int c = 0; c < D; ++c) {
          const size_t dof = (size_t)c * p.nnode + g;
          const bool fx = p.fixed && __ldg(p.fixed + dof);
          P0[c * NDOF + t] = fx ? R(0) : from_f64<R>(__ldg(p.v + dof));
        }
      }
      __syncwarp();
      if constexpr (EO) {
        mirror3_all<D, N, R>(P0, lane);
        fwd3_eon<N, Q1, D, R>(s_kf, s_rt, P0, P1, lane);
        unfold_points<D * D, Q1, R>(P1, s_Sc, lane);
      } else if constexpr (RB) {
        fwd3_rb<N, Q1, D, R>(tB, tG, P0, P1, lane);
      } else {
        fwd3<N, Q1, D, R>(sB, sG, P0, P1, lane);
      }
    } else if constexpr (D == 2) {
      fwd2<N, Q1, Cfg::NC, R>(sB, sG, P0, P1, lane);
    } else if constexpr (EO) {
      mirror3_all<Cfg::NC, N, R>(P0, lane);
      fwd3_eon<N, Q1, Cfg::NC, R>(s_kf, s_rt, P0, P1, lane);
      unfold_points<Cfg::NC * D, Q1, R>(P1, s_Sc, lane);
    } else if constexpr (RB) {
      fwd3_rb<N, Q1, Cfg::NC, R>(tB, tG, P0, P1, lane);
    } else {
      fwd3<N, Q1, Cfg::NC, R>(sB, sG, P0, P1, lane);
    }
    R* Abuf = Cfg::SPLIT ? P2 : ((D == 2) ? P0 : P1);     // A: [D][D][QP]
    R* dAbuf = Cfg::SPLIT ? P1 : Abuf + DD * QP;         // dA (Hessian action)
    R* Rbuf = Cfg::SPLIT ? P1 : Abuf;                    // per-point output of the adjoint
    // ---- pointwise
    double emin = INFINITY;
    constexpr int NS = DD * (DD + 1) / 2;
    for (int q = lane; q < QP; q += 32) {
      if constexpr (OP == OP_HESS_PA) {
        // y = H dA with the stored symmetric A-space Hessian (already scaled by w det W)
        const R* H = static_cast<const R*>(p.pa) + (size_t)e * p.pa_stride + q;
        // all NS loads are issued before the first use, so their latencies overlap
        R h[NS];
        if (q == lane) {
#pragma unroll
          for (int t = 0; t < NS; ++t) h[t] = hpre[t];
        } else {
#pragma unroll
          for (int t = 0; t < NS; ++t) h[t] = __ldg(H + (size_t)t * QP);
        }
        R dA[DD], y[DD];
#pragma unroll
        for (int i = 0; i < DD; ++i) {
          dA[i] = Abuf[i * QP + q];
          y[i] = R(0);
        }
        int s = 0;
#pragma unroll
        for (int r = 0; r < DD; ++r)
#pragma unroll
          for (int c = r; c < DD; ++c, ++s) {
            y[r] = fma(h[s], dA[c], y[r]);
            if (c != r) y[c] = fma(h[s], dA[r], y[c]);
          }
#pragma unroll
        for (int i = 0; i < DD; ++i) Abuf[i * QP + q] = y[i];
        continue;
      }
      R A[DD];
#pragma unroll
      for (int a = 0; a < D; ++a)
#pragma unroll
        for (int b = 0; b < D; ++b) A[a * D + b] = Abuf[(a * D + b) * QP + q];
      const R wq = sWq[q];
      R detW = R(p.detW);
      if (p.wkind == WK_PER_QP) {
        const double* Wq = p.Winv_qp + ((size_t)e * QP + q) * DD;
#pragma unroll
        for (int i = 0; i < DD; ++i) Wi[i] = R(__ldg(Wq + i));
        detW = R(__ldg(p.detW_qp + (size_t)e * QP + q));
      }
      R T[DD];
      if (p.wkind == WK_IDENTITY) {
#pragma unroll
        for (int i = 0; i < DD; ++i) T[i] = A[i];
      } else {
#pragma unroll
        for (int a = 0; a < D; ++a)
#pragma unroll
          for (int b = 0; b < D; ++b) {
            R s = R(0);
#pragma unroll
            for (int c = 0; c < D; ++c) s = fma(A[a * D + c], Wi[c * D + b], s);
            T[a * D + b] = s;
          }
      }
      if constexpr (OP == OP_GRAD_HESS) {
        // s P and s dP[dT] at the same point (s = w det W): one evaluation of
        // the metric's terms for both. For an (|T|^2, det T) metric
        // P = 2 mu_1 T + mu_t C, i.e. s P = cA T + ct C with MetricAct's scaled
        // coefficients (mu14 = |T - I|^2 is the exception: its P from metric_P);
        // the other metrics take P and dP from one dual-number evaluation.
        const R s = wq * detW;
        R dA[DD], dT[DD], Sg[DD], Sh[DD];
#pragma unroll
        for (int i = 0; i < DD; ++i) dA[i] = dAbuf[i * QP + q];
        if (p.wkind == WK_IDENTITY) {
#pragma unroll
          for (int i = 0; i < DD; ++i) dT[i] = dA[i];
        } else {
#pragma unroll
          for (int a = 0; a < D; ++a)
#pragma unroll
            for (int b = 0; b < D; ++b) {
              R acc = R(0);
#pragma unroll
              for (int c = 0; c < D; ++c) acc = fma(dA[a * D + c], Wi[c * D + b], acc);
              dT[a * D + b] = acc;
            }
        }
        bool ok;
        if (metric_dual(p.metric)) {
          Dual<R> Td[DD], Pd[DD], mud;
#pragma unroll
          for (int i = 0; i < DD; ++i) Td[i] = Dual<R>{T[i], dT[i]};
          ok = metric_P<D>(p.metric, Td, mud, Pd);
#pragma unroll
          for (int i = 0; i < DD; ++i) {
            Sg[i] = s * Pd[i].v;
            Sh[i] = s * Pd[i].d;
          }
        } else {
          MetricAct<D, R> L;
          ok = L.init(p.metric, T, s);
          if (ok) {
            L.dP(dT, Sh);
            if (p.metric == 14) {
              R mu;
              metric_P<D>(p.metric, T, mu, Sg, s);
            } else {
#pragma unroll
              for (int i = 0; i < DD; ++i) Sg[i] = fma(L.cA, L.T[i], L.ct * L.C[i]);
            }
          }
        }
        // R = S W^-t for both: the Hessian action's in place of dA, the
        // gradient's in place of A
#pragma unroll
        for (int a = 0; a < D; ++a)
#pragma unroll
          for (int b = 0; b < D; ++b) {
            R rg = R(0), rh = R(0);
            if (p.wkind == WK_IDENTITY) {
              rg = Sg[a * D + b];
              rh = Sh[a * D + b];
            } else {
#pragma unroll
              for (int c = 0; c < D; ++c) {
                rg = fma(Sg[a * D + c], Wi[b * D + c], rg);
                rh = fma(Sh[a * D + c], Wi[b * D + c], rh);
              }
            }
            Abuf[(a * D + b) * QP + q] = ok ? rg : R(0);
            dAbuf[(a * D + b) * QP + q] = ok ? rh : R(0);
          }
        continue;
      }
      if constexpr (OP == OP_LINEARIZE_C) {
        // compact record: T and w det W times the partials of mu in (|T|^2, det T)
        R* H = static_cast<R*>(p.pa) + (size_t)e * p.pa_stride + q;
        const R s = wq * detW;
        MetricLin<D, R> L;
        const bool ok = L.init(p.metric, T);
#pragma unroll
        for (int i = 0; i < DD; ++i) H[(size_t)i * QP] = T[i];
        H[(size_t)(DD + 0) * QP] = ok ? s * L.m1 : R(0);
        H[(size_t)(DD + 1) * QP] = ok ? s * L.mt : R(0);
        H[(size_t)(DD + 2) * QP] = ok ? s * L.m11 : R(0);
        H[(size_t)(DD + 3) * QP] = ok ? s * L.m1t : R(0);
        H[(size_t)(DD + 4) * QP] = ok ? s * L.mtt : R(0);
        continue;
      }
      if constexpr (OP == OP_LINEARIZE) {
        // column kl of the A-space Hessian: direction dA = E_kl, dT = E_kl W^-1,
        // R = w det W (d^2mu/dT^2 : dT) W^-t; the upper triangle is stored
        R* H = static_cast<R*>(p.pa) + (size_t)e * p.pa_stride + q;
        const R s = wq * detW;
        MetricLin<D, R> L;
        const bool lin = !metric_dual(p.metric);
        bool ok = lin ? L.init(p.metric, T) : true;
        if constexpr (D == 3) {
          if (lin && p.wkind == WK_IDENTITY && !p.metric2) {
            // W = I, an (|T|^2, det T) metric: the 45 entries in closed form,
            //   H[(a,b),(c,d)] = 2 mu_1 d_ac d_bd + (4 mu_11 T_cd + 2 mu_1t C_cd) T_ab
            //                    + (2 mu_1t T_cd + mu_tt C_cd) C_ab + mu_t dC_ab/dT_cd,
            // with dC_ab/dT_cd = +-T_ef (e, f the indices other than a, c and
            // b, d; zero if a = c or b = d): ~4 operations per entry where the
            // directional derivative costs ~100 per column
            const R m1 = s * L.m1, mt = s * L.mt, m11 = s * L.m11, m1t = s * L.m1t, mtt = s * L.mtt;
            int off3 = 0;
#pragma unroll
            for (int kl = 0; kl < 9; ++kl) {
              const int c = kl / 3, d = kl % 3;
              const R Pc = fma(R(4) * m11, T[kl], R(2) * m1t * L.C[kl]);
              const R Qc = fma(R(2) * m1t, T[kl], mtt * L.C[kl]);
#pragma unroll
              for (int mn = kl; mn < 9; ++mn) {
                const int a = mn / 3, b = mn % 3;
                R v = fma(Pc, T[mn], Qc * L.C[mn]);
                if (mn == kl) v += R(2) * m1;
                if (a != c && b != d) {
                  const int ee = 3 - a - c, ff = 3 - b - d;
                  const bool plus = (c == (a + 1) % 3) == (d == (b + 1) % 3);
                  v = fma(plus ? mt : -mt, T[ee * 3 + ff], v);
                }
                H[(size_t)(off3 + mn - kl) * QP] = ok ? v : R(0);
              }
              off3 += 9 - kl;
            }
            continue;
          }
        }
        int off = 0;
#pragma unroll 1
        for (int kl = 0; kl < DD; ++kl) {
          const int k = kl / D, l = kl % D;
          R dT[DD], S[DD];
#pragma unroll
          for (int a = 0; a < D; ++a)
#pragma unroll
            for (int b = 0; b < D; ++b)
              dT[a * D + b] = a == k ? (p.wkind == WK_IDENTITY ? R(l == b) : Wi[l * D + b]) : R(0);
          if (lin) {
            if (ok) L.dP(dT, S);
          } else {
            Dual<R> Td[DD], Pd[DD], mud;
#pragma unroll
            for (int i = 0; i < DD; ++i) Td[i] = Dual<R>{T[i], dT[i]};
            ok = metric_P<D>(p.metric, Td, mud, Pd);
#pragma unroll
            for (int i = 0; i < DD; ++i) S[i] = Pd[i].d;
          }
          // second term: dT2 = E_kl W2^-1
          R S2[DD];
          bool ok2 = false;
          R s2 = R(0);
          if (p.metric2) {
            R T2[DD], dT2[DD];
            times_w2<D>(p, A, T2);
#pragma unroll
            for (int a = 0; a < D; ++a)
#pragma unroll
              for (int b = 0; b < D; ++b) dT2[a * D + b] = a == k ? R(p.Winv2[l * D + b]) : R(0);
            ok2 = metric_dP<D>(p.metric2, T2, dT2, S2);
            s2 = wq * R(p.detW2) * (p.eta2 ? R(__ldg(p.eta2 + (size_t)e * QP + q)) : R(1));
          }
#pragma unroll
          for (int mn = 0; mn < DD; ++mn) {
            if (mn < kl) continue;
            const int m = mn / D, nn = mn % D;
            R r = R(0);
            if (p.wkind == WK_IDENTITY) {
              r = S[mn];
            } else {
#pragma unroll
              for (int c = 0; c < D; ++c) r = fma(S[m * D + c], Wi[nn * D + c], r);
            }
            R val = ok ? s * r : R(0);
            if (ok2) {
              R r2 = R(0);
#pragma unroll
              for (int c = 0; c < D; ++c) r2 = fma(S2[m * D + c], R(p.Winv2[nn * D + c]), r2);
              val = fma(s2, r2, val);
            }
            H[(size_t)(off + mn - kl) * QP] = val;
          }
          off += DD - kl;
        }
        continue;
      }
      if constexpr (OP == OP_ENERGY) {
        double Ad[DD];
#pragma unroll
        for (int i = 0; i < DD; ++i) Ad[i] = double(A[i]);
        const double dA = det_m<D>(Ad);
        emin = fmin(emin, dA);
        R mu;
        R Pd[DD];
        if (metric_P<D>(p.metric, T, mu, Pd)) accF += double(wq * detW) * double(mu);
        else accF = INFINITY;
        if (p.metric2) {
          R T2[DD], mu2;
          times_w2<D>(p, A, T2);
          const double eta = p.eta2 ? __ldg(p.eta2 + (size_t)e * QP + q) : 1.0;
          if (metric_P<D>(p.metric2, T2, mu2, Pd)) accF += double(wq) * p.detW2 * eta * double(mu2);
          else accF = INFINITY;
        }
      } else {
        // S below is already scaled by s = w det W (folded into the metric's
        // coefficients)
        const R s = wq * detW;
        R S[DD], dA[DD];
        bool ok;
        if constexpr (GRADLIKE) {
          R mu;
          ok = metric_P<D>(p.metric, T, mu, S, s);
          if constexpr (EG) {   // the energy of OP_ENERGY from the same point
            double Ad[DD];
#pragma unroll
            for (int i = 0; i < DD; ++i) Ad[i] = double(A[i]);
            emin = fmin(emin, det_m<D>(Ad));
            if (ok) accF += double(wq * detW) * double(mu);
            else accF = INFINITY;
          }
        } else {
          R dT[DD];
#pragma unroll
          for (int i = 0; i < DD; ++i) dA[i] = dAbuf[i * QP + q];
          if (p.wkind == WK_IDENTITY) {
#pragma unroll
            for (int i = 0; i < DD; ++i) dT[i] = dA[i];
          } else {
#pragma unroll
            for (int a = 0; a < D; ++a)
#pragma unroll
              for (int b = 0; b < D; ++b) {
                R acc = R(0);
#pragma unroll
                for (int c = 0; c < D; ++c) acc = fma(dA[a * D + c], Wi[c * D + b], acc);
                dT[a * D + b] = acc;
              }
          }
          if (metric_dual(p.metric)) {
            // not an (I1, tau) metric: forward-mode dual numbers
            Dual<R> Td[DD], Pd[DD], mud;
#pragma unroll
            for (int i = 0; i < DD; ++i) Td[i] = Dual<R>{T[i], dT[i]};
            ok = metric_P<D>(p.metric, Td, mud, Pd);
#pragma unroll
            for (int i = 0; i < DD; ++i) S[i] = s * Pd[i].d;
          } else {
            MetricAct<D, R> L;
            ok = L.init(p.metric, T, s);
            if (ok) L.dP(dT, S);
          }
        }
        // R = s S W^-t (S already carries s), stored in place of A at this point
#pragma unroll
        for (int a = 0; a < D; ++a)
#pragma unroll
          for (int b = 0; b < D; ++b) {
            R r = R(0);
            if (p.wkind == WK_IDENTITY) {
              r = S[a * D + b];
            } else {
#pragma unroll
              for (int c = 0; c < D; ++c) r = fma(S[a * D + c], Wi[b * D + c], r);
            }
            Rbuf[(a * D + b) * QP + q] = ok ? r : R(0);
          }
        if (p.metric2) {
          // + eta w det W2 S2 W2^-t (S2 = P2 or dP2 at T2 = A W2^-1)
          R T2[DD], S2[DD];
          times_w2<D>(p, A, T2);
          bool ok2;
          if constexpr (GRADLIKE) {
            R mu2;
            ok2 = metric_P<D>(p.metric2, T2, mu2, S2);
            if constexpr (EG) {
              const double eta = p.eta2 ? __ldg(p.eta2 + (size_t)e * QP + q) : 1.0;
              if (ok2) accF += double(wq) * p.detW2 * eta * double(mu2);
              else accF = INFINITY;
            }
          } else {
            R dT2[DD];
            times_w2<D>(p, dA, dT2);
            ok2 = metric_dP<D>(p.metric2, T2, dT2, S2);
          }
          if (ok2) {
            const R s2 = wq * R(p.detW2) * (p.eta2 ? R(__ldg(p.eta2 + (size_t)e * QP + q)) : R(1));
#pragma unroll
            for (int a = 0; a < D; ++a)
#pragma unroll
              for (int b = 0; b < D; ++b) {
                R r2 = R(0);
#pragma unroll
                for (int c = 0; c < D; ++c) r2 = fma(S2[a * D + c], R(p.Winv2[b * D + c]), r2);
                Rbuf[(a * D + b) * QP + q] = fma(s2, r2, Rbuf[(a * D + b) * QP + q]);
              }
          }
        }
      }
    }
    if constexpr (OP == OP_LINEARIZE || OP == OP_LINEARIZE_C) {
      __syncwarp();
    } else if constexpr (OP == OP_ENERGY) {
      accMin = fmin(accMin, emin);
      if (p.elem_min) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) emin = fmin(emin, __shfl_xor_sync(0xffffffffu, emin, o));
        if (lane == 0) p.elem_min[e] = emin;
      }
    } else if constexpr (OP == OP_GRAD_HESS) {
      __syncwarp();
      // ---- two adjoint contractions: 3D, the Hessian action's fields (P1)
      // into y, then the gradient's (P2) into g, each through P0 and its own
      // buffer; 2D, both at once (components 0..D-1 the gradient's fields,
      // D..2D-1 the Hessian action's)
      if constexpr (D == 2) {
        adj2<N, Q1, 2 * D, R>(sB, sG, P0, P1, lane);
        for (int t = lane; t < NDOF; t += 32) {
          const int gn = nodes(t);
#pragma unroll
          for (int c = 0; c < D; ++c) {
            const size_t dof = (size_t)c * p.nnode + gn;
            if (p.fixed && __ldg(p.fixed + dof)) continue;
            atomicAdd(p.g + dof, to_f64(P0[c * NDOF + t]));
            atomicAdd(p.y + dof, to_f64(P0[(D + c) * NDOF + t]));
          }
        }
      } else {
#pragma unroll 1
        for (int pass = 0; pass < 2; ++pass) {
          R* Rin = pass == 0 ? P1 : P2;
          double* out = pass == 0 ? p.y : p.g;
          if constexpr (EO) {
            mirror3_all<D * D, Q1, R>(Rin, lane);
            adj3_eon<N, Q1, D, R>(sB, sG, s_aperm, s_arat, s_C, P0, Rin, lane);
            unfold_nodes<D, N, R>(P0, s_ysc, lane);
          } else {
            adj3<N, Q1, D, R>(sB, sG, P0, Rin, lane);
          }
          for (int t = lane; t < NDOF; t += 32) {
            const int gn = nodes(t);
#pragma unroll
            for (int c = 0; c < D; ++c) {
              const size_t dof = (size_t)c * p.nnode + gn;
              if (p.fixed && __ldg(p.fixed + dof)) continue;
              atomicAdd(out + dof, to_f64(P0[c * NDOF + t]));
            }
          }
          __syncwarp();
        }
      }
    } else {
      if constexpr (EG) accMin = fmin(accMin, emin);
      __syncwarp();
      // ---- adjoint contraction and scatter
      if constexpr (D == 2) {
        adj2<N, Q1, D, R>(sB, sG, P0, P1, lane);
      } else if constexpr (EO) {
        mirror3_all<D * D, Q1, R>(P1, lane);
        adj3_eon<N, Q1, D, R>(sB, sG, s_aperm, s_arat, s_C, P0, P1, lane);
        unfold_nodes<D, N, R>(P0, s_ysc, lane);
      } else if constexpr (RB) {
        adj3_rb<N, Q1, D, R>(tB, tG, P0, P1, lane);
      } else {
        adj3<N, Q1, D, R>(sB, sG, P0, P1, lane);
      }
      for (int t = lane; t < NDOF; t += 32) {
        const int g = nodes(t);
#pragma unroll
        for (int c = 0; c < D; ++c) {
          const size_t dof = (size_t)c * p.nnode + g;
          if (p.fixed && __ldg(p.fixed + dof)) continue;
          // (one colour per launch in the deterministic mode: no other
          // element of the launch adds to this node, so each node gets one
          // add per launch, in colour order)
          if (PA_APPLY && p.y32) atomicAdd(p.y32 + dof, float(P0[c * NDOF + t]));   // FP32 Krylov vectors
          else atomicAdd(p.y + dof, to_f64(P0[c * NDOF + t]));
        }
      }
    }
    __syncwarp();
  }

  if constexpr (OP == OP_ENERGY || EG) {
    __shared__ double redF[WARPS], redM[WARPS];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      accF += __shfl_xor_sync(0xffffffffu, accF, o);
      accMin = fmin(accMin, __shfl_xor_sync(0xffffffffu, accMin, o));
    }
    if (lane == 0) { redF[warp] = accF; redM[warp] = accMin; }
    __syncthreads();
    if (threadIdx.x == 0) {
      double f = 0.0, m = INFINITY;
      for (int w = 0; w < WARPS; ++w) { f += redF[w]; m = fmin(m, redM[w]); }
      p.part_F[blockIdx.x] = f;
      p.part_min[blockIdx.x] = m;
    }
  }
}

// Host-side launcher for one instantiation.
template <int D, int N, int Q1, class R, int OP>
int launch_elem(const KParams& p, int grid, void* stream) {
  using Cfg = ElemCfg<D, N, Q1, R, OP>;
  elem_kernel<D, N, Q1, R, OP><<<grid, Cfg::WARPS * 32, Cfg::smem_bytes(), (cudaStream_t)stream>>>(p);
  return (int)cudaGetLastError();
}

// Occupancy-derived grid size, and the opt-in for > 48 KB of shared memory.
template <int D, int N, int Q1, class R, int OP>
int prepare_elem_impl(int nelem, int* grid) {
  using Cfg = ElemCfg<D, N, Q1, R, OP>;
  const size_t smem = Cfg::smem_bytes();
  cudaError_t err = cudaFuncSetAttribute((const void*)elem_kernel<D, N, Q1, R, OP>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return (int)err;
  int per_sm = 0, dev = 0, sms = 0;
  err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void*)elem_kernel<D, N, Q1, R, OP>,
                                                      Cfg::WARPS * 32, smem);
  if (err != cudaSuccess) return (int)err;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (per_sm < 1) return (int)cudaErrorInvalidConfiguration;
  const int need = (nelem + Cfg::WARPS - 1) / Cfg::WARPS;
  const int full = per_sm * sms;
  *grid = need < full ? need : full;
  return 0;
}

template <int D, int N, int Q1, class R, int OP>
int prepare_elem(int nelem, int* grid) {
  return (int)prepare_elem_impl<D, N, Q1, R, OP>(nelem, grid);
}

}  // namespace tmop
