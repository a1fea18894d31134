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
// before the current point is computed; when a warp starts an element, the
// record block of its next element is prefetched into L2 in one bulk
// request. Everything is warp-synchronous: no
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

// ---------------------------------------------------------------- packed-pair contractions
// The forward map v -> dA at the points and its adjoint R -> y, the same
// sum-factorised maps as the generic element kernel, written for the FP32
// pair instructions of sm_100+: __ffma2_rn rounds each half as one fmaf, so a
// pair does two independent multiply-adds in one issue slot. The 1D tables
// are held as pairs tBG[q][i] = (B[q][i], G[q][i]) (B = phi_i(xi_q),
// G = phi_i'(xi_q)), and every stage arranges its inputs so that one operand
// pair meets (B, G): stage 1 of the forward map broadcasts x and gets
// (x B, x G); the later stages read pairs stored in the order the next stage
// multiplies them, with the one product that needs B alone kept scalar.
//
// Stage buffers (words; pairs on even words):
//   x, y      [c][l*N+j][i]                    c*XC + (l*N+j)*XR + i
//   A pairs   [c][l][j][q0]                    c*AC + l*AL + j*AR + 2*q0
//   B pairs   [c][l][q1][q0]                   c*BC + l*BL + q1*BQ + 2*q0
//   B scalars [c][l][q1][q0]                   BS + c*SC + l*SL + q1*SQ + q0
//   Z pairs   [c][q] (components 1, 2)         c*ZC + 2*q
//   Z scalars [c][q] (component 0)             ZS + c*ZT + q
// x, y and B share the first buffer of a warp, A and Z the second; each
// stage reads one and writes the other.
__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 bcast2(float x) { return make_float2(x, x); }

// Strides per (N, Q1), chosen by counting, for each shared-memory access of
// the stages, the distinct words one warp instruction puts on one bank (half
// warps for 8-byte accesses) and taking the strides with the lowest total
// (ties: the smallest buffers). pac_layout_search.py, beside this file,
// regenerates the table.
template <int N, int Q1>
struct PacLayout;
#define TMOP_PAC_LAYOUT(N_, Q_, XR_, XC_, AR_, AL_, AC_, BQ_, BL_, BC_, SQ_, SL_, SC_, ZC_, ZT_) \
  template <>                                                                                  \
  struct PacLayout<N_, Q_> {                                                                   \
    static constexpr int XR = XR_, XC = XC_, AR = AR_, AL = AL_, AC = AC_;                     \
    static constexpr int BQ = BQ_, BL = BL_, BC = BC_, SQ = SQ_, SL = SL_, SC = SC_;           \
    static constexpr int ZC = ZC_, ZT = ZT_;                                                   \
    static constexpr int BS = 3 * BC, ZS = 3 * ZC;                                             \
  };
TMOP_PAC_LAYOUT(2, 2, 2, 8, 6, 12, 24, 4, 12, 24, 2, 4, 8, 20, 8)
TMOP_PAC_LAYOUT(2, 3, 2, 8, 10, 38, 76, 12, 50, 102, 3, 15, 42, 82, 41)
TMOP_PAC_LAYOUT(3, 3, 3, 27, 6, 18, 54, 6, 38, 114, 3, 14, 43, 82, 41)
TMOP_PAC_LAYOUT(3, 4, 3, 27, 10, 40, 120, 8, 40, 120, 4, 20, 60, 128, 80)
TMOP_PAC_LAYOUT(4, 4, 5, 80, 10, 40, 160, 8, 40, 160, 4, 20, 80, 128, 80)
TMOP_PAC_LAYOUT(4, 5, 5, 80, 24, 106, 424, 10, 74, 296, 6, 37, 148, 274, 153)
TMOP_PAC_LAYOUT(5, 5, 5, 125, 12, 74, 370, 10, 74, 370, 5, 25, 153, 274, 153)
TMOP_PAC_LAYOUT(5, 6, 5, 125, 14, 70, 350, 12, 76, 380, 6, 38, 190, 456, 228)
#undef TMOP_PAC_LAYOUT

template <int N, int Q1>
struct PacCfg {
  using L = PacLayout<N, Q1>;
  static constexpr int NDOF = N * N * N, QP = Q1 * Q1 * Q1;
  static constexpr int NT = (NDOF + 31) / 32, NPL = (QP + 31) / 32;  // nodes and points per lane
  // words each stage buffer spans
  static constexpr int XN = 2 * L::XC + (N * N - 1) * L::XR + N;
  static constexpr int BN = L::BS + 2 * L::SC + (N - 1) * L::SL + (Q1 - 1) * L::SQ + Q1;
  static constexpr int AN = 2 * L::AC + (N - 1) * L::AL + (N - 1) * L::AR + 2 * Q1;
  static constexpr int ZN = L::ZS + 2 * L::ZT + QP;
  static constexpr int B0 = round4(imax(XN, BN));
  static constexpr int B1 = round4(imax(AN, ZN));
  static_assert(L::XR >= N && L::XC >= N * N * L::XR, "x rows overlap");
  static_assert(L::AR >= 2 * Q1 && L::AL >= N * L::AR && L::AC >= N * L::AL, "A overlaps");
  static_assert(L::BQ >= 2 * Q1 && L::BL >= Q1 * L::BQ && L::BC >= N * L::BL, "B pairs overlap");
  static_assert(L::SQ >= Q1 && L::SL >= Q1 * L::SQ && L::SC >= N * L::SL, "B scalars overlap");
  static_assert(L::ZC >= 2 * QP && L::ZT >= QP, "points overlap");
  static_assert(L::AR % 2 == 0 && L::AL % 2 == 0 && L::AC % 2 == 0 && L::BQ % 2 == 0 && L::BL % 2 == 0 &&
                    L::BC % 2 == 0 && L::ZC % 2 == 0,
                "pairs must sit on even words");
  static constexpr size_t smem_bytes() { return sizeof(float) * kPacWarps * (B0 + B1); }
};

// x (buffer 0) -> dA at every point (Z, buffer 1)
template <int N, int Q1, class L>
__device__ __forceinline__ void pac_fwd(const float2 (&tBG)[Q1 * N], float* P0, float* P1, int lane) {
  constexpr int NC = 3, QQ = Q1 * Q1;
#pragma unroll
  for (int k = 0; k < (NC * N * N + 31) / 32; ++k) {           // rows (c, l, j) of x -> A = (x B, x G) over q0
    const int t = lane + 32 * k;
    if (t >= NC * N * N) break;
    const int c = t / (N * N), lj = t % (N * N), l = lj / N, j = lj % N;
    float2 xv[N];
#pragma unroll
    for (int i = 0; i < N; ++i) xv[i] = bcast2(P0[c * L::XC + lj * L::XR + i]);
    float2* o = reinterpret_cast<float2*>(P1 + c * L::AC + l * L::AL + j * L::AR);
#pragma unroll
    for (int q0 = 0; q0 < Q1; ++q0) {
      float2 s = make_float2(0.f, 0.f);
#pragma unroll
      for (int i = 0; i < N; ++i) s = ffma2(xv[i], tBG[q0 * N + i], s);
      o[q0] = s;
    }
  }
  __syncwarp();
#pragma unroll
  for (int k = 0; k < (NC * N * Q1 + 31) / 32; ++k) {          // rows (c, l, q0): A over j -> B
    const int t = lane + 32 * k;
    if (t >= NC * N * Q1) break;
    const int q0 = t % Q1, l = (t / Q1) % N, c = t / (Q1 * N);
    const float* in = P1 + c * L::AC + l * L::AL + 2 * q0;
    float2 xb[N];
    float xg[N];
#pragma unroll
    for (int j = 0; j < N; ++j) {
      const float2 a = *reinterpret_cast<const float2*>(in + j * L::AR);
      xb[j] = bcast2(a.x);
      xg[j] = a.y;
    }
    float* op = P0 + c * L::BC + l * L::BL + 2 * q0;
    float* os = P0 + L::BS + c * L::SC + l * L::SL + q0;
#pragma unroll
    for (int q1 = 0; q1 < Q1; ++q1) {
      float2 s = make_float2(0.f, 0.f);  // (bb, bg)
      float gb = 0.f;
#pragma unroll
      for (int j = 0; j < N; ++j) {
        s = ffma2(xb[j], tBG[q1 * N + j], s);
        gb = fmaf(xg[j], tBG[q1 * N + j].x, gb);
      }
      op[q1 * L::BQ] = s.y;      // the pair stage 3 multiplies by (B, G): (bg, bb)
      op[q1 * L::BQ + 1] = s.x;
      os[q1 * L::SQ] = gb;
    }
  }
  __syncwarp();
#pragma unroll
  for (int k = 0; k < (NC * QQ + 31) / 32; ++k) {              // columns (c, q1, q0): B over l -> dA
    const int t = lane + 32 * k;
    if (t >= NC * QQ) break;
    const int c = t / QQ, q01 = t % QQ, q1 = q01 / Q1, q0 = q01 % Q1;
    const float* ip = P0 + c * L::BC + q1 * L::BQ + 2 * q0;
    const float* is = P0 + L::BS + c * L::SC + q1 * L::SQ + q0;
    float2 pb[N];
    float gb[N];
#pragma unroll
    for (int l = 0; l < N; ++l) {
      pb[l] = *reinterpret_cast<const float2*>(ip + l * L::BL);
      gb[l] = is[l * L::SL];
    }
    float2* zp = reinterpret_cast<float2*>(P1 + c * L::ZC) + q01;
    float* zs = P1 + L::ZS + c * L::ZT + q01;
#pragma unroll
    for (int q2 = 0; q2 < Q1; ++q2) {
      float2 a12 = make_float2(0.f, 0.f);  // dA components (c, 1), (c, 2)
      float a0 = 0.f;                      // dA component (c, 0)
#pragma unroll
      for (int l = 0; l < N; ++l) {
        a12 = ffma2(pb[l], tBG[q2 * N + l], a12);
        a0 = fmaf(gb[l], tBG[q2 * N + l].x, a0);
      }
      zp[q2 * QQ] = a12;
      zs[q2 * QQ] = a0;
    }
  }
  __syncwarp();
}

// R at every point (Z, buffer 1) -> y (buffer 0)
template <int N, int Q1, class L>
__device__ __forceinline__ void pac_adj(const float2 (&tBG)[Q1 * N], float* P0, float* P1, int lane) {
  constexpr int NC = 3, QQ = Q1 * Q1;
#pragma unroll
  for (int k = 0; k < (NC * QQ + 31) / 32; ++k) {              // columns (c, q1, q0): Z over q2 -> B
    const int t = lane + 32 * k;
    if (t >= NC * QQ) break;
    const int c = t / QQ, q01 = t % QQ, q1 = q01 / Q1, q0 = q01 % Q1;
    const float2* zp = reinterpret_cast<const float2*>(P1 + c * L::ZC) + q01;
    const float* zs = P1 + L::ZS + c * L::ZT + q01;
    float2 r12[Q1];
    float r0[Q1];
#pragma unroll
    for (int q2 = 0; q2 < Q1; ++q2) {
      r12[q2] = zp[q2 * QQ];
      r0[q2] = zs[q2 * QQ];
    }
    float* op = P0 + c * L::BC + q1 * L::BQ + 2 * q0;
    float* os = P0 + L::BS + c * L::SC + q1 * L::SQ + q0;
#pragma unroll
    for (int l = 0; l < N; ++l) {
      float2 u12 = make_float2(0.f, 0.f);
      float u0 = 0.f;
#pragma unroll
      for (int q2 = 0; q2 < Q1; ++q2) {
        u12 = ffma2(r12[q2], tBG[q2 * N + l], u12);
        u0 = fmaf(r0[q2], tBG[q2 * N + l].x, u0);
      }
      op[l * L::BL] = u0;        // the pair stage 2 multiplies by (B, G): (u0, u1)
      op[l * L::BL + 1] = u12.x;
      os[l * L::SL] = u12.y;
    }
  }
  __syncwarp();
#pragma unroll
  for (int k = 0; k < (NC * N * Q1 + 31) / 32; ++k) {          // rows (c, l, q0): B over q1 -> A
    const int t = lane + 32 * k;
    if (t >= NC * N * Q1) break;
    const int q0 = t % Q1, l = (t / Q1) % N, c = t / (Q1 * N);
    const float* ip = P0 + c * L::BC + l * L::BL + 2 * q0;
    const float* is = P0 + L::BS + c * L::SC + l * L::SL + q0;
    float2 u01[Q1];
    float u2[Q1];
#pragma unroll
    for (int q1 = 0; q1 < Q1; ++q1) {
      u01[q1] = *reinterpret_cast<const float2*>(ip + q1 * L::BQ);
      u2[q1] = is[q1 * L::SQ];
    }
    float* o = P1 + c * L::AC + l * L::AL + 2 * q0;
#pragma unroll
    for (int j = 0; j < N; ++j) {
      float2 s = make_float2(0.f, 0.f);  // (u0 B, u1 G)
      float pb = 0.f;                    // u2 B
#pragma unroll
      for (int q1 = 0; q1 < Q1; ++q1) {
        s = ffma2(u01[q1], tBG[q1 * N + j], s);
        pb = fmaf(u2[q1], tBG[q1 * N + j].x, pb);
      }
      o[j * L::AR] = s.y + pb;   // the pair stage 3 multiplies by (B, G): (vb, vg)
      o[j * L::AR + 1] = s.x;
    }
  }
  __syncwarp();
#pragma unroll
  for (int k = 0; k < (NC * N * N + 31) / 32; ++k) {           // rows (c, l, j): A over q0 -> y
    const int t = lane + 32 * k;
    if (t >= NC * N * N) break;
    const int c = t / (N * N), lj = t % (N * N), l = lj / N, j = lj % N;
    const float2* in = reinterpret_cast<const float2*>(P1 + c * L::AC + l * L::AL + j * L::AR);
    float2 w[Q1];
#pragma unroll
    for (int q0 = 0; q0 < Q1; ++q0) w[q0] = in[q0];
#pragma unroll
    for (int i = 0; i < N; ++i) {
      float2 s = make_float2(0.f, 0.f);
#pragma unroll
      for (int q0 = 0; q0 < Q1; ++q0) s = ffma2(w[q0], tBG[q0 * N + i], s);
      P0[c * L::XC + lj * L::XR + i] = s.x + s.y;
    }
  }
  __syncwarp();
}

// v (rounded to FP32 as it arrives: the product's input, and half the
// registers of the prefetched copy) and the fixed flags at the nodes this
// lane gathers. Hardware conversions: this kernel is bound by instruction
// issue and leaves the FP64 pipe mostly idle, so one F2F beats the ~20
// integer instructions of f64_to_f32.
template <int N, int NT, bool IO32>
__device__ __forceinline__ void fetch_v(const KParams& p, const NodeMap<N>& m, int lane, float (&v)[NT][3],
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
        if constexpr (IO32) v[s][c] = __ldg(p.v32 + dof);
        else v[s][c] = __double2float_rn(__ldg(p.v + dof));
        if (p.fixed && __ldg(p.fixed + dof)) fmask |= 1u << (s * 3 + c);
      }
    }
  }
}

__device__ __forceinline__ void l2_prefetch(const void* p, unsigned bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

template <int QP>
__device__ __forceinline__ void fetch_rec(const float* rec, int pa_stride, int e, int q, float (&h)[kCompactRec]) {
  if (q < QP) {
    const float* r = rec + (size_t)e * pa_stride + q;
#pragma unroll
    for (int k = 0; k < kCompactRec; ++k) h[k] = __ldg(r + (size_t)k * QP);
  }
}

// dA at point q (Z) -> R = w det W (d^2mu/dT^2 : dA W^-1) W^-t, in place
// (IDENT: W = I, so dT = dA and R = S, and W^-1 is never read)
template <class L, bool IDENT>
__device__ __forceinline__ void pac_point(const float (&h)[kCompactRec], const float (&Wi)[9], float* buf, int q) {
  MetricLin<3, float> M;
#pragma unroll
  for (int i = 0; i < 9; ++i) M.T[i] = h[i];
  cof_m<3>(M.T, M.C);
  M.m1 = h[9]; M.mt = h[10]; M.m11 = h[11]; M.m1t = h[12]; M.mtt = h[13];
  float2* zp = reinterpret_cast<float2*>(buf) + q;
  float* zs = buf + L::ZS + q;
  float dA[9], dT[9], S[9];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const float2 a = zp[c * (L::ZC / 2)];
    dA[c * 3 + 0] = zs[c * L::ZT];
    dA[c * 3 + 1] = a.x;
    dA[c * 3 + 2] = a.y;
  }
  if constexpr (IDENT) {
#pragma unroll
    for (int i = 0; i < 9; ++i) dT[i] = dA[i];
  } else {
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b)
        dT[a * 3 + b] = fmaf(dA[a * 3 + 0], Wi[0 * 3 + b], fmaf(dA[a * 3 + 1], Wi[1 * 3 + b], dA[a * 3 + 2] * Wi[2 * 3 + b]));
  }
  M.dP(dT, S);
  float r[9];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b)
      if constexpr (IDENT) r[a * 3 + b] = S[a * 3 + b];
      else r[a * 3 + b] = fmaf(S[a * 3 + 0], Wi[b * 3 + 0], fmaf(S[a * 3 + 1], Wi[b * 3 + 1], S[a * 3 + 2] * Wi[b * 3 + 2]));
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    zs[c * L::ZT] = r[c * 3 + 0];
    zp[c * (L::ZC / 2)] = make_float2(r[c * 3 + 1], r[c * 3 + 2]);
  }
}

// IDENT: the target is W = I (p.wkind == WK_IDENTITY); otherwise one constant W^-1.
// IO32: v and y are the FP32 vectors p.v32, p.y32 (FP32 atomics into y).
// For n = 4 the kernel is held to 128 registers, two blocks per SM (0: no bound).
template <int N, int Q1, bool IDENT, bool IO32>
__global__ void __launch_bounds__(kPacWarps * 32, N == 4 ? 2 : 0) pac_kernel(const KParams p) {
  using Cfg = PacCfg<N, Q1>;
  using L = typename Cfg::L;
  constexpr int NDOF = Cfg::NDOF, QP = Cfg::QP, NT = Cfg::NT, NPL = Cfg::NPL;
  extern __shared__ __align__(16) float pac_smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float* P0 = pac_smem + warp * (Cfg::B0 + Cfg::B1);
  float* P1 = P0 + Cfg::B0;
  float2 tBG[Q1 * N];
  float Wi[9];
#pragma unroll
  for (int t = 0; t < Q1 * N; ++t) tBG[t] = make_float2(f64_to_f32(p.B[t]), f64_to_f32(p.G[t]));
#pragma unroll
  for (int i = 0; i < 9; ++i) Wi[i] = IDENT ? 0.f : f64_to_f32(p.Winv[i]);
  const float* rec = static_cast<const float*>(p.pa);
  const int stride = gridDim.x * kPacWarps;
  // elements ei = warp slot + k stride: all elements, or one colour's list
  // (deterministic sums: one add per node and launch, see KParams)
  const int ecount = p.elist ? p.ecount : p.nelem;
  auto elem = [&](int i) { return p.elist ? __ldg(p.elist + i) : i; };
  int ei = blockIdx.x * kPacWarps + warp;
  const int gw = blockIdx.x * kPacWarps + warp;  // this warp's slot of the v . (H v) partials
  if (ei >= ecount) {  // whole warps only; nothing below waits on other warps
    if (p.vdot && lane == 0) p.vdot[gw] = 0.0;
    return;
  }
  int e = elem(ei);

  NodeMap<N> cur(p.elem_nodes, p.sx, p.sy), nxt(p.elem_nodes, p.sx, p.sy);
  cur.element(e, NDOF);
  float v[NT][3], vc[NT][3];
  unsigned fnext;
  float hq[kCompactRec];
  // sum over this warp's elements of v_E . (H_E v_E): each lane's share of
  // an element in FP32 (v_E as the product reads it, FP32), the elements in FP64
  double vdot = 0.0;
  fetch_v<N, NT, IO32>(p, cur, lane, v, fnext);
  fetch_rec<QP>(rec, p.pa_stride, e, lane, hq);
  for (;;) {
    // ---- the record block of the next element goes to L2 ahead of its loads
    // (one bulk prefetch: the block is contiguous, 16-byte aligned and padded
    // to a multiple of 16 bytes)
    if (lane == 0 && ei + stride < ecount)
      l2_prefetch(rec + (size_t)elem(ei + stride) * p.pa_stride, (unsigned)(p.pa_stride * sizeof(float)));
    // ---- v of this element into the stage buffer (fixed dofs read as 0)
    const unsigned fcur = fnext;
#pragma unroll
    for (int s = 0; s < NT; ++s) {
      const int t = lane + 32 * s;
      if (t < NDOF) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          vc[s][c] = (fcur >> (s * 3 + c)) & 1u ? 0.f : v[s][c];
          P0[c * L::XC + (t / N) * L::XR + t % N] = vc[s][c];
        }
      }
    }
    __syncwarp();
    // ---- dA at every point (Z)
    pac_fwd<N, Q1, L>(tBG, P0, P1, lane);
    // ---- pointwise; the next point's record is requested before this point is computed
#pragma unroll
    for (int k = 0; k < NPL; ++k) {
      const int q = lane + 32 * k;
      float hn[kCompactRec];
      if (k + 1 < NPL) fetch_rec<QP>(rec, p.pa_stride, e, q + 32, hn);
      if (q < QP) pac_point<L, IDENT>(hq, Wi, P1, q);
      if (k + 1 < NPL) {
#pragma unroll
        for (int i = 0; i < kCompactRec; ++i) hq[i] = hn[i];
      }
    }
    // ---- the next element's loads go out before this element's adjoint and scatter
    const int eni = ei + stride;
    const bool more = eni < ecount;
    const int en = more ? elem(eni) : 0;
    if (more) {
      nxt.element(en, NDOF);
      fetch_v<N, NT, IO32>(p, nxt, lane, v, fnext);
      fetch_rec<QP>(rec, p.pa_stride, en, lane, hq);
    }
    __syncwarp();
    // ---- adjoint contraction into y (buffer 0), scatter
    pac_adj<N, Q1, L>(tBG, P0, P1, lane);
    float vdot_e = 0.f;
#pragma unroll
    for (int s = 0; s < NT; ++s) {
      const int t = lane + 32 * s;
      if (t < NDOF) {
        const int g = cur(t);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const float yf = P0[c * L::XC + (t / N) * L::XR + t % N];
          vdot_e = fmaf(vc[s][c], yf, vdot_e);  // 0 at fixed dofs (vc = 0 there)
          if (!((fcur >> (s * 3 + c)) & 1u)) {
            if constexpr (IO32) atomicAdd(p.y32 + (size_t)c * p.nnode + g, yf);
            else atomicAdd(p.y + (size_t)c * p.nnode + g, (double)yf);
          }
        }
      }
    }
    vdot += (double)vdot_e;
    __syncwarp();
    if (!more) break;
    ei = eni;
    e = en;
    cur = nxt;
  }
  if (p.vdot) {  // fixed-order warp reduction; one partial per warp
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) vdot += __shfl_xor_sync(0xffffffffu, vdot, o);
    if (lane == 0) p.vdot[gw] = vdot;
  }
}

// ---------------------------------------------------------------- recomputed (matrix-free) product
// The FP32 Hessian action recomputed from x (OP_HESS_C, the matrix-free
// Krylov operator of the FP32 forms for (|T|^2, det T) metrics with a
// constant target): per element, A(x) by the same forward contraction as
// dA, the compact record of the point (T and w det W times the five partials
// of mu) into shared memory, then the product exactly as from stored
// records. x is taken relative to the element's first node in FP64 before
// rounding (A is translation invariant), so A keeps FP32 relative accuracy.
template <int N, int Q1>
struct PacrCfg {
  using P = PacCfg<N, Q1>;
  static constexpr int QP = P::QP;
  static constexpr int REC = round4(kCompactRec * QP);    // the element's records [value][q]
  static constexpr int PER_WARP = P::B0 + P::B1 + REC;
  static constexpr size_t smem_bytes() { return sizeof(float) * (kPacrWarps * PER_WARP + round4(QP)); }
};

// x at the nodes this lane gathers, relative to the element's first node
template <int N, int NT>
__device__ __forceinline__ void fetch_x(const KParams& p, const NodeMap<N>& m, int lane, float (&xr)[NT][3]) {
  constexpr int NDOF = N * N * N;
  const int g0 = m(0);
  double x0[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) x0[c] = __ldg(p.x + (size_t)c * p.nnode + g0);
#pragma unroll
  for (int s = 0; s < NT; ++s) {
    const int t = lane + 32 * s;
    if (t < NDOF) {
      const int g = m(t);
#pragma unroll
      for (int c = 0; c < 3; ++c) xr[s][c] = __double2float_rn(__ldg(p.x + (size_t)c * p.nnode + g) - x0[c]);
    }
  }
}

// A at point q (Z buffer) -> the point's compact record, in shared memory
template <class L, bool IDENT>
__device__ __forceinline__ void pacr_record(int metric, const float (&Wi)[9], const float* buf, float* rec, int q,
                                            int QP, float s) {
  const float2* zp = reinterpret_cast<const float2*>(buf) + q;
  const float* zs = buf + L::ZS + q;
  float A[9], T[9];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const float2 a = zp[c * (L::ZC / 2)];
    A[c * 3 + 0] = zs[c * L::ZT];
    A[c * 3 + 1] = a.x;
    A[c * 3 + 2] = a.y;
  }
  if constexpr (IDENT) {
#pragma unroll
    for (int i = 0; i < 9; ++i) T[i] = A[i];
  } else {
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b)
        T[a * 3 + b] = fmaf(A[a * 3 + 0], Wi[0 * 3 + b], fmaf(A[a * 3 + 1], Wi[1 * 3 + b], A[a * 3 + 2] * Wi[2 * 3 + b]));
  }
  MetricLin<3, float> M;
  const bool ok = M.init(metric, T);
#pragma unroll
  for (int i = 0; i < 9; ++i) rec[i * QP + q] = T[i];
  rec[9 * QP + q] = ok ? s * M.m1 : 0.f;
  rec[10 * QP + q] = ok ? s * M.mt : 0.f;
  rec[11 * QP + q] = ok ? s * M.m11 : 0.f;
  rec[12 * QP + q] = ok ? s * M.m1t : 0.f;
  rec[13 * QP + q] = ok ? s * M.mtt : 0.f;
}

template <int N, int Q1, bool IDENT, bool IO32>
__global__ void __launch_bounds__(kPacrWarps * 32, N == 4 ? 2 : 1) pacr_kernel(const KParams p) {
  using Cfg = PacCfg<N, Q1>;
  using RC = PacrCfg<N, Q1>;
  using L = typename Cfg::L;
  constexpr int NDOF = Cfg::NDOF, QP = Cfg::QP, NT = Cfg::NT, NPL = Cfg::NPL;
  extern __shared__ __align__(16) float pac_smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float* P0 = pac_smem + warp * RC::PER_WARP;
  float* P1 = P0 + Cfg::B0;
  float* REC = P1 + Cfg::B1;
  float* sWq = pac_smem + kPacrWarps * RC::PER_WARP;   // w_q det W at every point
  for (int q = threadIdx.x; q < QP; q += blockDim.x) {
    const int q0 = q % Q1, q1 = (q / Q1) % Q1, q2 = q / (Q1 * Q1);
    sWq[q] = (float)(p.w1[q0] * p.w1[q1] * p.w1[q2] * p.detW);
  }
  float2 tBG[Q1 * N];
  float Wi[9];
#pragma unroll
  for (int t = 0; t < Q1 * N; ++t) tBG[t] = make_float2(f64_to_f32(p.B[t]), f64_to_f32(p.G[t]));
#pragma unroll
  for (int i = 0; i < 9; ++i) Wi[i] = IDENT ? 0.f : f64_to_f32(p.Winv[i]);
  __syncthreads();
  const int stride = gridDim.x * kPacrWarps;
  const int ecount = p.elist ? p.ecount : p.nelem;
  auto elem = [&](int i) { return p.elist ? __ldg(p.elist + i) : i; };
  int ei = blockIdx.x * kPacrWarps + warp;
  if (ei >= ecount) return;   // whole warps only; nothing below waits on other warps
  int e = elem(ei);
  NodeMap<N> cur(p.elem_nodes, p.sx, p.sy), nxt(p.elem_nodes, p.sx, p.sy);
  cur.element(e, NDOF);
  float v[NT][3], vc[NT][3], xr[NT][3];
  unsigned fnext;
  fetch_x<N, NT>(p, cur, lane, xr);
  fetch_v<N, NT, IO32>(p, cur, lane, v, fnext);
  for (;;) {
    // ---- x relative to the element's first node -> A at every point (Z)
#pragma unroll
    for (int s = 0; s < NT; ++s) {
      const int t = lane + 32 * s;
      if (t < NDOF) {
#pragma unroll
        for (int c = 0; c < 3; ++c) P0[c * L::XC + (t / N) * L::XR + t % N] = xr[s][c];
      }
    }
    __syncwarp();
    pac_fwd<N, Q1, L>(tBG, P0, P1, lane);
    // ---- the compact record of every point
#pragma unroll
    for (int k = 0; k < NPL; ++k) {
      const int q = lane + 32 * k;
      if (q < QP) pacr_record<L, IDENT>(p.metric, Wi, P1, REC, q, QP, sWq[q]);
    }
    __syncwarp();
    // ---- v of this element (fixed dofs read as 0) -> dA at every point
    const unsigned fcur = fnext;
#pragma unroll
    for (int s = 0; s < NT; ++s) {
      const int t = lane + 32 * s;
      if (t < NDOF) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          vc[s][c] = (fcur >> (s * 3 + c)) & 1u ? 0.f : v[s][c];
          P0[c * L::XC + (t / N) * L::XR + t % N] = vc[s][c];
        }
      }
    }
    __syncwarp();
    pac_fwd<N, Q1, L>(tBG, P0, P1, lane);
    // ---- pointwise from the records in shared memory
#pragma unroll
    for (int k = 0; k < NPL; ++k) {
      const int q = lane + 32 * k;
      if (q < QP) {
        float h[kCompactRec];
#pragma unroll
        for (int i = 0; i < kCompactRec; ++i) h[i] = REC[i * QP + q];
        pac_point<L, IDENT>(h, Wi, P1, q);
      }
    }
    // ---- the next element's loads go out before this element's adjoint and scatter
    const int eni = ei + stride;
    const bool more = eni < ecount;
    const int en = more ? elem(eni) : 0;
    if (more) {
      nxt.element(en, NDOF);
      fetch_x<N, NT>(p, nxt, lane, xr);
      fetch_v<N, NT, IO32>(p, nxt, lane, v, fnext);
    }
    __syncwarp();
    pac_adj<N, Q1, L>(tBG, P0, P1, lane);
#pragma unroll
    for (int s = 0; s < NT; ++s) {
      const int t = lane + 32 * s;
      if (t < NDOF) {
        const int g = cur(t);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const float yf = P0[c * L::XC + (t / N) * L::XR + t % N];
          if (!((fcur >> (s * 3 + c)) & 1u)) {
            if constexpr (IO32) atomicAdd(p.y32 + (size_t)c * p.nnode + g, yf);
            else atomicAdd(p.y + (size_t)c * p.nnode + g, (double)yf);
          }
        }
      }
    }
    __syncwarp();
    if (!more) break;
    ei = eni;
    e = en;
    cur = nxt;
  }
}

}  // namespace

template <int N, int Q1>
int launch_pac(const KParams& p, int grid, void* stream) {
  const size_t smem = PacCfg<N, Q1>::smem_bytes();
  const bool id = p.wkind == WK_IDENTITY, io32 = p.v32 != nullptr;
  cudaStream_t s = (cudaStream_t)stream;
  if (io32 != (p.y32 != nullptr)) return (int)cudaErrorInvalidValue;
  if (id && io32) pac_kernel<N, Q1, true, true><<<grid, kPacWarps * 32, smem, s>>>(p);
  else if (id) pac_kernel<N, Q1, true, false><<<grid, kPacWarps * 32, smem, s>>>(p);
  else if (io32) pac_kernel<N, Q1, false, true><<<grid, kPacWarps * 32, smem, s>>>(p);
  else pac_kernel<N, Q1, false, false><<<grid, kPacWarps * 32, smem, s>>>(p);
  return (int)cudaGetLastError();
}

// grid: the blocks both forms keep resident on every SM
template <int N, int Q1>
int prepare_pac(int nelem, int* grid) {
  const size_t smem = PacCfg<N, Q1>::smem_bytes();
  const void* fn[4] = {(const void*)pac_kernel<N, Q1, true, false>, (const void*)pac_kernel<N, Q1, false, false>,
                       (const void*)pac_kernel<N, Q1, true, true>, (const void*)pac_kernel<N, Q1, false, true>};
  int per_sm = 1 << 30, dev = 0, sms = 0;
  for (const void* f : fn) {
    cudaError_t err = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return (int)err;
    int b = 0;
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, f, kPacWarps * 32, smem);
    if (err != cudaSuccess) return (int)err;
    per_sm = b < per_sm ? b : per_sm;
  }
  if (per_sm < 1) return (int)cudaErrorInvalidConfiguration;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int need = (nelem + kPacWarps - 1) / kPacWarps, full = per_sm * sms;
  *grid = need < full ? need : full;
  return 0;
}

template <int N, int Q1>
int launch_pacr(const KParams& p, int grid, void* stream) {
  const size_t smem = PacrCfg<N, Q1>::smem_bytes();
  const bool id = p.wkind == WK_IDENTITY, io32 = p.v32 != nullptr;
  cudaStream_t s = (cudaStream_t)stream;
  if (io32 != (p.y32 != nullptr) || !p.x) return (int)cudaErrorInvalidValue;
  if (id && io32) pacr_kernel<N, Q1, true, true><<<grid, kPacrWarps * 32, smem, s>>>(p);
  else if (id) pacr_kernel<N, Q1, true, false><<<grid, kPacrWarps * 32, smem, s>>>(p);
  else if (io32) pacr_kernel<N, Q1, false, true><<<grid, kPacrWarps * 32, smem, s>>>(p);
  else pacr_kernel<N, Q1, false, false><<<grid, kPacrWarps * 32, smem, s>>>(p);
  return (int)cudaGetLastError();
}

template <int N, int Q1>
int prepare_pacr(int nelem, int* grid) {
  const size_t smem = PacrCfg<N, Q1>::smem_bytes();
  const void* fn[4] = {(const void*)pacr_kernel<N, Q1, true, false>, (const void*)pacr_kernel<N, Q1, false, false>,
                       (const void*)pacr_kernel<N, Q1, true, true>, (const void*)pacr_kernel<N, Q1, false, true>};
  int per_sm = 1 << 30, dev = 0, sms = 0;
  for (const void* f : fn) {
    cudaError_t err = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return (int)err;
    int b = 0;
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, f, kPacrWarps * 32, smem);
    if (err != cudaSuccess) return (int)err;
    per_sm = b < per_sm ? b : per_sm;
  }
  if (per_sm < 1) return (int)cudaErrorInvalidConfiguration;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int need = (nelem + kPacrWarps - 1) / kPacrWarps, full = per_sm * sms;
  *grid = need < full ? need : full;
  return 0;
}

#define TMOP_PAC(N, Q) template int launch_pac<N, Q>(const KParams&, int, void*); \
  template int prepare_pac<N, Q>(int, int*); \
  template int launch_pacr<N, Q>(const KParams&, int, void*); \
  template int prepare_pacr<N, Q>(int, int*);
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
