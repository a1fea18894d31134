// Hessian action from the compact partially assembled records (3D, FP32):
// per point the record holds T and w det W (mu_1, mu_t, mu_11, mu_1t, mu_tt)
// of an (|T|^2, det T) metric, and the product is rebuilt as
//   R = w det W (d^2mu/dT^2 : dA W^-1) W^-t      (Section 3.4)
// with d^2mu/dT^2 : dT = 2 mu_1 dT + 2 (mu_11 dI1 + mu_1t dtau) T
//                        + (mu_1t dI1 + mu_tt dtau) C + mu_t dC.
//
// One warp per element, as in the generic element kernel, but software
// pipelined for the memory system: while a warp finishes element e (adjoint
// contraction and scatter) the loads of element e + stride are already in
// flight (its v and fixed flags, the record of each lane's first point), and
// inside the pointwise stage the record of a lane's next point is loaded
// before the current point is computed. Everything is warp-synchronous: no
// block barriers after the prologue. With p.vdot set, each warp also sums
// v_E . (H_E v_E) over its elements, which is v . (H v) summed element by
// element (v is read as zero at fixed dofs, where H v is zero): MINRES then
// needs no separate dot-product pass over v and H v.
#include <cuda_runtime.h>
#include <stdint.h>

#include "tmop_device.cuh"
#include "tmop_kparams.h"
#include "tmop_pa_compact.h"

namespace tmop {

namespace {

constexpr int round4(int v) { return (v + 3) / 4 * 4; }
constexpr int imax(int a, int b) { return a > b ? a : b; }

template <int N, int Q1>
struct PacCfg {
  static constexpr int NDOF = N * N * N, QP = Q1 * Q1 * Q1;
  static constexpr int NT = (NDOF + 31) / 32, NPL = (QP + 31) / 32;  // nodes and points per lane
  // stage buffers of the register-blocked contractions (fwd3_rb / adj3_rb maps)
  static constexpr int B0 = round4(imax(3 * NDOF, 9 * N * Q1 * Q1));
  static constexpr int B1 = round4(imax(9 * QP, 6 * N * N * Q1));
  static constexpr size_t smem_bytes() { return sizeof(float) * kPacWarps * (B0 + B1); }
};

// v and the fixed flags at the nodes this lane gathers
template <int N, int NT>
__device__ __forceinline__ void fetch_v(const KParams& p, const NodeMap<N>& m, int lane, double (&v)[NT][3],
                                        unsigned& fmask) {
  constexpr int NDOF = N * N * N;
  fmask = 0u;
#pragma unroll
  for (int s = 0; s < NT; ++s) {
    const int t = lane + 32 * s;
    if (t < NDOF) {
      const int g = m(t);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const size_t dof = (size_t)c * p.nnode + g;
        v[s][c] = __ldg(p.v + dof);
        if (p.fixed && __ldg(p.fixed + dof)) fmask |= 1u << (s * 3 + c);
      }
    }
  }
}

template <int QP>
__device__ __forceinline__ void fetch_rec(const float* rec, int pa_stride, int e, int q, float (&h)[kCompactRec]) {
  if (q < QP) {
    const float* r = rec + (size_t)e * pa_stride + q;
#pragma unroll
    for (int k = 0; k < kCompactRec; ++k) h[k] = __ldg(r + (size_t)k * QP);
  }
}

// dA at point q (buffer [9][QP]) -> R = w det W (d^2mu/dT^2 : dA W^-1) W^-t, in place
template <int QP>
__device__ __forceinline__ void pac_point(const float (&h)[kCompactRec], bool ident, const float (&Wi)[9], float* buf,
                                          int q) {
  MetricLin<3, float> L;
#pragma unroll
  for (int i = 0; i < 9; ++i) L.T[i] = h[i];
  cof_m<3>(L.T, L.C);
  L.m1 = h[9]; L.mt = h[10]; L.m11 = h[11]; L.m1t = h[12]; L.mtt = h[13];
  float dA[9], dT[9], S[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) dA[i] = buf[i * QP + q];
  if (ident) {
#pragma unroll
    for (int i = 0; i < 9; ++i) dT[i] = dA[i];
  } else {
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b)
        dT[a * 3 + b] = fmaf(dA[a * 3 + 0], Wi[0 * 3 + b], fmaf(dA[a * 3 + 1], Wi[1 * 3 + b], dA[a * 3 + 2] * Wi[2 * 3 + b]));
  }
  L.dP(dT, S);
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      const float r = ident ? S[a * 3 + b]
                            : fmaf(S[a * 3 + 0], Wi[b * 3 + 0], fmaf(S[a * 3 + 1], Wi[b * 3 + 1], S[a * 3 + 2] * Wi[b * 3 + 2]));
      buf[(a * 3 + b) * QP + q] = r;
    }
}

template <int N, int Q1>
__global__ void __launch_bounds__(kPacWarps * 32) pac_kernel(const KParams p) {
  using Cfg = PacCfg<N, Q1>;
  constexpr int NDOF = Cfg::NDOF, QP = Cfg::QP, NT = Cfg::NT, NPL = Cfg::NPL;
  extern __shared__ __align__(16) float pac_smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float* P0 = pac_smem + warp * (Cfg::B0 + Cfg::B1);
  float* P1 = P0 + Cfg::B0;
  float tB[Q1 * N], tG[Q1 * N], Wi[9];
#pragma unroll
  for (int t = 0; t < Q1 * N; ++t) {
    tB[t] = f64_to_f32(p.B[t]);
    tG[t] = f64_to_f32(p.G[t]);
  }
#pragma unroll
  for (int i = 0; i < 9; ++i) Wi[i] = f64_to_f32(p.Winv[i]);
  const bool ident = p.wkind == WK_IDENTITY;
  const float* rec = static_cast<const float*>(p.pa);
  const int stride = gridDim.x * kPacWarps;
  int e = blockIdx.x * kPacWarps + warp;
  const int gw = blockIdx.x * kPacWarps + warp;  // this warp's slot of the v . (H v) partials
  if (e >= p.nelem) {  // whole warps only; nothing below waits on other warps
    if (p.vdot && lane == 0) p.vdot[gw] = 0.0;
    return;
  }

  NodeMap<N> cur(p.elem_nodes, p.sx, p.sy), nxt(p.elem_nodes, p.sx, p.sy);
  cur.element(e, NDOF);
  double v[NT][3], vc[NT][3];
  unsigned fnext;
  float hq[kCompactRec];
  double vdot = 0.0;  // sum over this warp's elements of v_E . (H_E v_E), FP64
  fetch_v<N, NT>(p, cur, lane, v, fnext);
  fetch_rec<QP>(rec, p.pa_stride, e, lane, hq);
  for (;;) {
    // ---- v of this element into the stage buffer (fixed dofs read as 0)
    const unsigned fcur = fnext;
#pragma unroll
    for (int s = 0; s < NT; ++s) {
      const int t = lane + 32 * s;
      if (t < NDOF) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          vc[s][c] = (fcur >> (s * 3 + c)) & 1u ? 0.0 : v[s][c];
          P0[c * NDOF + t] = f64_to_f32(vc[s][c]);
        }
      }
    }
    __syncwarp();
    // ---- dA at every point: P1 [3][3][QP]
    fwd3_rb<N, Q1, 3, float>(tB, tG, P0, P1, lane);
    // ---- pointwise; the next point's record is requested before this point is computed
#pragma unroll
    for (int k = 0; k < NPL; ++k) {
      const int q = lane + 32 * k;
      float hn[kCompactRec];
      if (k + 1 < NPL) fetch_rec<QP>(rec, p.pa_stride, e, q + 32, hn);
      if (q < QP) pac_point<QP>(hq, ident, Wi, P1, q);
      if (k + 1 < NPL) {
#pragma unroll
        for (int i = 0; i < kCompactRec; ++i) hq[i] = hn[i];
      }
    }
    // ---- the next element's loads go out before this element's adjoint and scatter
    const int en = e + stride;
    const bool more = en < p.nelem;
    if (more) {
      nxt.element(en, NDOF);
      fetch_v<N, NT>(p, nxt, lane, v, fnext);
      fetch_rec<QP>(rec, p.pa_stride, en, lane, hq);
    }
    __syncwarp();
    // ---- adjoint contraction into P0 [3][NDOF], scatter
    adj3_rb<N, Q1, 3, float>(tB, tG, P0, P1, lane);
#pragma unroll
    for (int s = 0; s < NT; ++s) {
      const int t = lane + 32 * s;
      if (t < NDOF) {
        const int g = cur(t);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const double yc = f32_to_f64(P0[c * NDOF + t]);
          vdot = fma(vc[s][c], yc, vdot);  // 0 at fixed dofs (vc = 0 there)
          if (!((fcur >> (s * 3 + c)) & 1u)) atomicAdd(p.y + (size_t)c * p.nnode + g, yc);
        }
      }
    }
    __syncwarp();
    if (!more) break;
    e = en;
    cur = nxt;
  }
  if (p.vdot) {  // fixed-order warp reduction; one partial per warp
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) vdot += __shfl_xor_sync(0xffffffffu, vdot, o);
    if (lane == 0) p.vdot[gw] = vdot;
  }
}

}  // namespace

template <int N, int Q1>
int launch_pac(const KParams& p, int grid, void* stream) {
  pac_kernel<N, Q1><<<grid, kPacWarps * 32, PacCfg<N, Q1>::smem_bytes(), (cudaStream_t)stream>>>(p);
  return (int)cudaGetLastError();
}

template <int N, int Q1>
int prepare_pac(int nelem, int* grid) {
  const size_t smem = PacCfg<N, Q1>::smem_bytes();
  cudaError_t err =
      cudaFuncSetAttribute((const void*)pac_kernel<N, Q1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return (int)err;
  int per_sm = 0, dev = 0, sms = 0;
  err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void*)pac_kernel<N, Q1>, kPacWarps * 32, smem);
  if (err != cudaSuccess) return (int)err;
  if (per_sm < 1) return (int)cudaErrorInvalidConfiguration;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int need = (nelem + kPacWarps - 1) / kPacWarps, full = per_sm * sms;
  *grid = need < full ? need : full;
  return 0;
}

#define TMOP_PAC(N, Q) template int launch_pac<N, Q>(const KParams&, int, void*); \
  template int prepare_pac<N, Q>(int, int*);
TMOP_PAC(2, 2)
TMOP_PAC(2, 3)
TMOP_PAC(3, 3)
TMOP_PAC(3, 4)
TMOP_PAC(4, 4)
TMOP_PAC(4, 5)
TMOP_PAC(5, 5)
TMOP_PAC(5, 6)
#undef TMOP_PAC

}  // namespace tmop
