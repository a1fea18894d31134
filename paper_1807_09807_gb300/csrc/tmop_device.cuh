// Device-side building blocks of the TMOP element kernels (sm_103a).
//
//  * Dual<R>: forward-mode dual numbers. The Hessian action needs
//    d^2mu/dT^2 : dT (Section 3.4); evaluating the first derivative P(T) on
//    T + eps dT in dual arithmetic yields exactly that directional derivative,
//    so every metric is written once, generically in its scalar type.
//  * metric_P: mu and P = dmu/dT for the Table 3.1 / Section 3.2 metrics in
//    the invariants I1 = |T|^2, tau = det T, C = cof T.
//  * fwd2/fwd3, adj2/adj3: sum-factorised tensor-product contractions of one
//    element, executed by one warp in shared memory. Forward: nodal values
//    X[c][l][j][i] -> A[c][b](q) = sum_i X_i d phi_i / d xi_b (eq. (2.2)).
//    Adjoint: per-point matrices R[c][b](q) -> Y[c][i] = sum_q R[c][b](q)
//    d phi_i / d xi_b (the transposed contraction of the gradient formula).
#pragma once
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "tmop_kparams.h"

namespace tmop {



// ---------------------------------------------------------------- scalars
template <class R>
struct Dual {
  R v, d;
};

template <class R> __device__ __forceinline__ Dual<R> operator+(Dual<R> a, Dual<R> b) { return {a.v + b.v, a.d + b.d}; }
template <class R> __device__ __forceinline__ Dual<R> operator-(Dual<R> a, Dual<R> b) { return {a.v - b.v, a.d - b.d}; }
template <class R> __device__ __forceinline__ Dual<R> operator-(Dual<R> a) { return {-a.v, -a.d}; }
template <class R> __device__ __forceinline__ Dual<R> operator*(Dual<R> a, Dual<R> b) {
  return {a.v * b.v, fma(a.v, b.d, a.d * b.v)};
}
template <class R> __device__ __forceinline__ Dual<R> operator*(R s, Dual<R> a) { return {s * a.v, s * a.d}; }
template <class R> __device__ __forceinline__ Dual<R> operator*(Dual<R> a, R s) { return {s * a.v, s * a.d}; }
template <class R> __device__ __forceinline__ Dual<R> operator+(Dual<R> a, R s) { return {a.v + s, a.d}; }
template <class R> __device__ __forceinline__ Dual<R> operator-(Dual<R> a, R s) { return {a.v - s, a.d}; }

__device__ __forceinline__ double value(double a) { return a; }
__device__ __forceinline__ float value(float a) { return a; }
template <class R> __device__ __forceinline__ R value(Dual<R> a) { return a.v; }

__device__ __forceinline__ double recip(double a) { return 1.0 / a; }
__device__ __forceinline__ float recip(float a) { return 1.0f / a; }
template <class R> __device__ __forceinline__ Dual<R> recip(Dual<R> a) {
  R r = R(1) / a.v;
  return {r, -a.d * r * r};
}
// tau^{-1/3}. In FP64 from the FP32 estimate y by one third-order step
// (the cube of the start's ~1e-7 relative error is below FP64 rounding: a
// few ulp) with 6 FP64 operations, on GB300's narrow FP64 pipe the cheaper
// route. Outside
// [2^-120, 2^120] (where the FP32 start would over- or underflow) and for
// non-finite input it defers to rcbrt.
__device__ __forceinline__ double rcbrt_nr(double a);
__device__ __forceinline__ double rcbrt_(double a) { return rcbrt_nr(a); }
__device__ __forceinline__ float rcbrt_(float a) { return rcbrtf(a); }
template <class R> __device__ __forceinline__ Dual<R> rcbrt_(Dual<R> a) {
  R r = rcbrt_(a.v);
  // d(tau^{-1/3}) = -(1/3) tau^{-4/3} dtau
  return {r, R(-1) / R(3) * r / a.v * a.d};
}

// Constants enter the metric formulas as plain reals, so that a dual number
// times a constant costs two multiplications, not a full dual product.
template <class S> struct base_of { using type = S; };
template <class R> struct base_of<Dual<R>> { using type = R; };
template <class S> __device__ __forceinline__ typename base_of<S>::type sc(double c) {
  return typename base_of<S>::type(c);
}

// ---------------------------------------------------------------- node numbering
// Global node ids of the nodes of an element. A structured order-(N-1) grid
// of sx x sy (x sz) elements is numbered lexicographically, x fastest, on a
// (k sx + 1) x (k sy + 1) (x (k sz + 1)) node lattice: the first node of
// element e is found once per element (the divisions by the run-time grid
// sizes are the costly part; GB300 runs their conversions on its narrow FP64
// pipe), and local node t = i + N j + N^2 l adds compile-time digits times
// the lattice strides. Unstructured meshes read the connectivity table.
// zplanes: lattice planes per element layer along the last index, N - 1 in
// 3D; in 2D, 1: a 2D "stack" of sz grids (elements e = ex + sx (ey + sy b),
// grid b's nodes after those of grids 0..b-1), so that many equal meshes
// form one structured problem.
template <int N>
struct NodeMap {
  const int32_t* conn;
  int sx, sy, Nx, NxNy, zplanes, base;
  const int32_t* row;
  __device__ __forceinline__ NodeMap(const int32_t* elem_nodes, int sx_, int sy_, int zplanes_ = N - 1)
      : conn(elem_nodes), sx(sx_), sy(sy_), Nx((N - 1) * sx_ + 1), NxNy(((N - 1) * sx_ + 1) * ((N - 1) * sy_ + 1)),
        zplanes(zplanes_), base(0), row(nullptr) {}
  __device__ __forceinline__ void element(int e, int ndof) {
    if (sx > 0) {
      const int exy = sx * sy, ez = e / exy, r = e - ez * exy, ey = r / sx, ex = r - ey * sx;
      base = ez * zplanes * NxNy + (N - 1) * (ey * Nx + ex);
    } else {
      row = conn + (size_t)e * ndof;
    }
  }
  __device__ __forceinline__ int operator()(int t) const {
    if (sx > 0) {
      const int i = t % N, j = (t / N) % N, l = t / (N * N);
      return base + l * NxNy + j * Nx + i;
    }
    return __ldg(row + t);
  }
};

// ---------------------------------------------------------------- precision conversions
// IEEE binary64 <-> binary32 with integer operations. The FP32 kernels
// convert every gathered FP64 value of v (and x) and every FP32 contribution
// they add into an FP64 output; done with F2F instructions these run on
// GB300's narrow FP64 pipe, here on the integer pipes. f64_to_f32 rounds to
// nearest even, as a cast does, except that results below the smallest
// normal float (|d| < 2^-126) become a signed zero; f32_to_f64 is exact, with
// subnormal inputs read as zero. Infinities and NaNs are kept.
__device__ __forceinline__ float f64_to_f32(double d) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(d);
  const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
  const unsigned sign = hi & 0x80000000u;
  const int e = (int)((hi >> 20) & 0x7FFu);
  if (e == 0x7FF) return __uint_as_float(sign | 0x7F800000u | (((hi & 0xFFFFFu) | lo) ? 0x400000u : 0u));
  const int fe = e - 1023 + 127;
  if (fe <= 0) return __uint_as_float(sign);
  unsigned m = ((hi & 0xFFFFFu) << 3) | (lo >> 29);   // the top 23 of the 52 mantissa bits
  const unsigned rem = lo & 0x1FFFFFFFu, half = 0x10000000u;
  m += (rem > half || (rem == half && (m & 1u))) ? 1u : 0u;
  unsigned r = ((unsigned)fe << 23) + m;              // a carry out of m steps the exponent
  if (fe >= 255 || r >= 0x7F800000u) r = 0x7F800000u;
  return __uint_as_float(sign | r);
}

__device__ __forceinline__ double f32_to_f64(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned sign = u & 0x80000000u, e = (u >> 23) & 0xFFu, m = u & 0x7FFFFFu;
  if (e == 0) return __longlong_as_double((long long)((unsigned long long)sign << 32));
  const unsigned hi = sign | (e == 0xFFu ? 0x7FF00000u : ((e + (1023u - 127u)) << 20)) | (m >> 3);
  const unsigned lo = m << 29;
  return __longlong_as_double((long long)(((unsigned long long)hi << 32) | lo));
}

__device__ __forceinline__ double rcbrt_nr(double a) {
  if (!(a >= 0x1p-120 && a <= 0x1p120)) return rcbrt(a);
  // one step of the series y (1 + e)^(-1/3) = y (1 - e/3 + 2 e^2 / 9 - ...)
  // with e = a y^3 - 1: the FP32 start has |e| < ~1e-6, so the dropped
  // O(e^3) term is far below FP64 rounding
  const double y = f32_to_f64(rcbrtf(f64_to_f32(a)));
  const double e = fma(a, y * y * y, -1.0);
  return fma(y, e * fma(e, 2.0 / 9.0, -1.0 / 3.0), y);
}

// FP64 value -> the kernel's arithmetic type, and back
template <class R> __device__ __forceinline__ R from_f64(double d) { return R(d); }
template <> __device__ __forceinline__ float from_f64<float>(double d) { return f64_to_f32(d); }
__device__ __forceinline__ double to_f64(double v) { return v; }
__device__ __forceinline__ double to_f64(float v) { return f32_to_f64(v); }

// ---------------------------------------------------------------- matrices
template <int D, class S>
__device__ __forceinline__ S det_m(const S* M) {
  if constexpr (D == 2) {
    return M[0] * M[3] - M[1] * M[2];
  } else {
    return M[0] * (M[4] * M[8] - M[5] * M[7]) - M[1] * (M[3] * M[8] - M[5] * M[6]) +
           M[2] * (M[3] * M[7] - M[4] * M[6]);
  }
}

// cof(M) = det(M) M^{-T}: the derivative of det M with respect to M
template <int D, class S>
__device__ __forceinline__ void cof_m(const S* M, S* C) {
  if constexpr (D == 2) {
    C[0] = M[3]; C[1] = -M[2]; C[2] = -M[1]; C[3] = M[0];
  } else {
    C[0] = M[4] * M[8] - M[5] * M[7];
    C[1] = M[5] * M[6] - M[3] * M[8];
    C[2] = M[3] * M[7] - M[4] * M[6];
    C[3] = M[2] * M[7] - M[1] * M[8];
    C[4] = M[0] * M[8] - M[2] * M[6];
    C[5] = M[1] * M[6] - M[0] * M[7];
    C[6] = M[1] * M[5] - M[2] * M[4];
    C[7] = M[2] * M[3] - M[0] * M[5];
    C[8] = M[0] * M[4] - M[1] * M[3];
  }
}

// ---------------------------------------------------------------- metrics
// mu(T) and P = dmu/dT. Returns false when a barrier metric meets
// tau <= 0 (mu is +inf there, P is left unset).
//
// metric_P(id, T, mu, P, s) returns s P instead (mu unscaled): the factor
// joins the one or two scalars P is built from, so the caller's weight
// w det W costs no multiply per entry of P.
template <int D, class S>
__device__ __forceinline__ bool metric_P(int id, const S* T, S& mu, S* P, typename base_of<S>::type s) {
  using B = typename base_of<S>::type;
  constexpr int DD = D * D;
  S I1 = T[0] * T[0];
#pragma unroll
  for (int i = 1; i < DD; ++i) I1 = I1 + T[i] * T[i];
  if (id == 1) {  // |T|^2
    mu = I1;
    const B c = sc<S>(2.0) * s;
#pragma unroll
    for (int i = 0; i < DD; ++i) P[i] = c * T[i];
    return true;
  }
  if (id == 14) {  // |T - I|^2
    const B c = sc<S>(2.0) * s;
    S e0 = T[0] - sc<S>(1.0);
    S acc = e0 * e0;
    P[0] = c * e0;
#pragma unroll
    for (int i = 1; i < DD; ++i) {
      S e = (i % (D + 1) == 0) ? T[i] - sc<S>(1.0) : T[i];
      acc = acc + e * e;
      P[i] = c * e;
    }
    mu = acc;
    return true;
  }
  // det T by expansion along the first row, from the cofactors P needs anyway
  S C[DD];
  cof_m<D>(T, C);
  S tau = T[0] * C[0];
#pragma unroll
  for (int j = 1; j < D; ++j) tau = tau + T[j] * C[j];
  if (!(value(tau) > 0)) return false;
  if (id == 98) {  // |T - I|^2 / tau (Section 4.3.2); P = (2 (T - I) - mu C) / tau
    S it = recip(tau);
    S E[DD];
#pragma unroll
    for (int i = 0; i < DD; ++i) E[i] = (i % (D + 1) == 0) ? T[i] - sc<S>(1.0) : T[i];
    S acc = E[0] * E[0];
#pragma unroll
    for (int i = 1; i < DD; ++i) acc = acc + E[i] * E[i];
    mu = acc * it;
    const S its = it * s;
#pragma unroll
    for (int i = 0; i < DD; ++i) P[i] = its * (sc<S>(2.0) * E[i] - mu * C[i]);
    return true;
  }
  if constexpr (D == 2) {
    S it = recip(tau);
    if (id == 2) {  // |T|^2 / (2 tau) - 1
      mu = sc<S>(0.5) * I1 * it - sc<S>(1.0);
      S a = it * s, b = (sc<S>(0.5) * s) * I1 * it * it;
#pragma unroll
      for (int i = 0; i < 4; ++i) P[i] = a * T[i] - b * C[i];
      return true;
    }
    S it2 = it * it;
    if (id == 7) {  // |T - T^-t|^2 = I1 (1 + tau^-2) - 4
      mu = I1 * (it2 + sc<S>(1.0)) - sc<S>(4.0);
      S a = (sc<S>(2.0) * s) * (it2 + sc<S>(1.0)), b = (sc<S>(2.0) * s) * I1 * it2 * it;
#pragma unroll
      for (int i = 0; i < 4; ++i) P[i] = a * T[i] - b * C[i];
      return true;
    }
    if (id == 9) {  // tau |T - T^-t|^2 = tau I1 + I1 / tau - 4 tau
      mu = tau * I1 + I1 * it - sc<S>(4.0) * tau;
      S a = (sc<S>(2.0) * s) * (tau + it), b = (I1 - I1 * it2 - sc<S>(4.0)) * s;
#pragma unroll
      for (int i = 0; i < 4; ++i) P[i] = a * T[i] + b * C[i];
      return true;
    }
    if (id == 77) {  // (tau - 1/tau)^2 / 2
      S d = tau - it;
      mu = sc<S>(0.5) * d * d;
      S a = d * (it2 + sc<S>(1.0)) * s;
#pragma unroll
      for (int i = 0; i < 4; ++i) P[i] = a * C[i];
      return true;
    }
  } else {
    if (id == 303) {  // |T|^2 / (3 tau^{2/3}) - 1; 1 / tau = (tau^{-1/3})^3, no division
      S r = rcbrt_(tau);
      S r2 = r * r;
      S it = r2 * r;
      mu = sc<S>(1.0 / 3.0) * I1 * r2 - sc<S>(1.0);
      S a = (sc<S>(2.0 / 3.0) * s) * r2, b = a * ((sc<S>(1.0 / 3.0) * I1) * it);   // b = 2/9 s I1 r^5
#pragma unroll
      for (int i = 0; i < 9; ++i) P[i] = a * T[i] - b * C[i];
      return true;
    }
    if (id == 302) {  // |T|^2 |T^-1|^2 / 9 - 1 = I1 K / (9 tau^2) - 1, K = |cof T|^2
      S it = recip(tau);
      S K = C[0] * C[0];
#pragma unroll
      for (int i = 1; i < 9; ++i) K = K + C[i] * C[i];
      // dK/dT = 2 (I1 T - T T^t T)
      S TtT[9];
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) TtT[i * 3 + j] = T[i] * T[j] + T[3 + i] * T[3 + j] + T[6 + i] * T[6 + j];
      S a = sc<S>(1.0 / 9.0) * it * it;
      mu = a * I1 * K - sc<S>(1.0);
      S c = sc<S>(2.0) * a * I1 * K * it;
      S as = a * s, cs = c * s;
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          S M = T[i * 3 + 0] * TtT[0 * 3 + j] + T[i * 3 + 1] * TtT[1 * 3 + j] + T[i * 3 + 2] * TtT[2 * 3 + j];
          S Kp = sc<S>(2.0) * (I1 * T[i * 3 + j] - M);
          P[i * 3 + j] = as * (I1 * Kp + sc<S>(2.0) * K * T[i * 3 + j]) - cs * C[i * 3 + j];
        }
      return true;
    }
  }
  return false;
}

template <int D, class S>
__device__ __forceinline__ bool metric_P(int id, const S* T, S& mu, S* P) {
  return metric_P<D, S>(id, T, mu, P, typename base_of<S>::type(1));
}

// ---------------------------------------------------------------- linearised metric
// For metrics written in I1 = |T|^2 and tau = det T (all but mu302), the
// first derivative is P = 2 mu_1 T + mu_t C and, with dI1 = 2 T:dT and
// dtau = C:dT (C = cof T, the derivative of det),
//   dP = 2 mu_1 dT + 2 (mu_11 dI1 + mu_1t dtau) T + (mu_1t dI1 + mu_tt dtau) C + mu_t dC,
// where dC is the directional derivative of the cofactor matrix (product rule
// on its 2x2 minors in 3D; linear in 2D). MetricLin holds everything that
// depends on T only, so one point can be differentiated in many directions.
template <int D, class R>
struct MetricLin {
  static constexpr int DD = D * D;
  R T[DD], C[DD];
  R m1, mt, m11, m1t, mtt;
  bool ok;

  __device__ __forceinline__ bool init(int id, const R* Tin) {
#pragma unroll
    for (int i = 0; i < DD; ++i) T[i] = Tin[i];
    R I1 = R(0);
#pragma unroll
    for (int i = 0; i < DD; ++i) I1 = fma(T[i], T[i], I1);
    cof_m<D>(T, C);
    R tau = R(0);
#pragma unroll
    for (int j = 0; j < D; ++j) tau = fma(T[j], C[j], tau);   // expansion along the first row
    m1 = R(0); mt = R(0); m11 = R(0); m1t = R(0); mtt = R(0);
    if (id == 1 || id == 14) { m1 = R(1); ok = true; return true; }
    ok = tau > R(0);
    if (!ok) return false;
    if (id == 303) {          // I1 tau^{-2/3} / 3 - 1 (3D); 1 / tau = (tau^{-1/3})^3, no division
      const R r = rcbrt_(tau), r2 = r * r, it = r2 * r, t53 = r2 * it;
      m1 = r2 * R(1.0 / 3.0); mt = R(-2.0 / 9.0) * I1 * t53; m1t = R(-2.0 / 9.0) * t53;
      mtt = R(10.0 / 27.0) * I1 * t53 * it;
      return ok;
    }
    const R it = R(1) / tau, it2 = it * it;
    if (id == 2) {            // I1 / (2 tau) - 1
      m1 = R(0.5) * it; mt = R(-0.5) * I1 * it2; m1t = R(-0.5) * it2; mtt = I1 * it2 * it;
    } else if (id == 7) {     // I1 (1 + tau^-2) - 4 (2D)
      m1 = R(1) + it2; mt = R(-2) * I1 * it2 * it; m1t = R(-2) * it2 * it; mtt = R(6) * I1 * it2 * it2;
    } else if (id == 9) {     // tau I1 + I1 / tau - 4 tau (2D)
      m1 = tau + it; mt = I1 - I1 * it2 - R(4); m1t = R(1) - it2; mtt = R(2) * I1 * it2 * it;
    } else if (id == 77) {    // (tau - 1/tau)^2 / 2
      const R sdiff = tau - it, ds = R(1) + it2;
      mt = sdiff * ds; mtt = ds * ds - R(2) * sdiff * it2 * it;
    } else {
      ok = false;
    }
    return ok;
  }

  // dP for one direction dT
  __device__ __forceinline__ void dP(const R* dT, R* out) const {
    R dI1 = R(0), dtau = R(0);
#pragma unroll
    for (int i = 0; i < DD; ++i) {
      dI1 = fma(T[i], dT[i], dI1);
      dtau = fma(C[i], dT[i], dtau);
    }
    dI1 *= R(2);
    const R a = R(2) * m1;
    const R bT = R(2) * (m11 * dI1 + m1t * dtau);
    const R bC = m1t * dI1 + mtt * dtau;
    R mdC[DD];  // mu_t dC
    if constexpr (D == 2) {
      mdC[0] = mt * dT[3]; mdC[1] = -mt * dT[2]; mdC[2] = -mt * dT[1]; mdC[3] = mt * dT[0];
    } else {
      // each entry of dC is the derivative of a 2x2 minor, dT_a T_b + T_a dT_b
      // - dT_c T_e - T_c dT_e; with U = mu_t T the factor mu_t costs no
      // multiply per entry
      R U[DD];
#pragma unroll
      for (int i = 0; i < DD; ++i) U[i] = mt * T[i];
#define TMOP_DMINOR(a_, b_, c_, e_) fma(dT[a_], U[b_], fma(U[a_], dT[b_], -fma(dT[c_], U[e_], U[c_] * dT[e_])))
      mdC[0] = TMOP_DMINOR(4, 8, 5, 7);
      mdC[1] = TMOP_DMINOR(5, 6, 3, 8);
      mdC[2] = TMOP_DMINOR(3, 7, 4, 6);
      mdC[3] = TMOP_DMINOR(2, 7, 1, 8);
      mdC[4] = TMOP_DMINOR(0, 8, 2, 6);
      mdC[5] = TMOP_DMINOR(1, 6, 0, 7);
      mdC[6] = TMOP_DMINOR(1, 5, 2, 4);
      mdC[7] = TMOP_DMINOR(2, 3, 0, 5);
      mdC[8] = TMOP_DMINOR(0, 4, 1, 3);
#undef TMOP_DMINOR
    }
#pragma unroll
    for (int i = 0; i < DD; ++i) out[i] = fma(a, dT[i], fma(bT, T[i], fma(bC, C[i], mdC[i])));
  }
};

// The same second derivative for a matrix-free Hessian action, with the
// point's weight s = w det W and the constant factors folded into five
// coefficients when T is set, so that dP costs ~10 multiplies fewer per
// point (GB300 issues only two FP64 operations per SM and clock):
//   s dP = cA dT + (c11 t + c1t d) T + (c1t t + ctt d) C + s mu_t dC,
// with t = T:dT, d = C:dT, cA = 2 s mu_1, c11 = 4 s mu_11, c1t = 2 s mu_1t,
// ctt = s mu_tt.
template <int D, class R>
struct MetricAct {
  static constexpr int DD = D * D;
  R T[DD], C[DD];
  R cA, c11, c1t, ctt, ct;

  __device__ __forceinline__ bool init(int id, const R* Tin, R s) {
    if constexpr (D == 3) {
      if (id == 303) {  // I1 tau^{-2/3} / 3 - 1: mu_11 = 0
#pragma unroll
        for (int i = 0; i < DD; ++i) T[i] = Tin[i];
        R I1 = R(0);
#pragma unroll
        for (int i = 0; i < DD; ++i) I1 = fma(T[i], T[i], I1);
        cof_m<D>(T, C);
        R tau = R(0);
#pragma unroll
        for (int j = 0; j < D; ++j) tau = fma(T[j], C[j], tau);
        if (!(tau > R(0))) return false;
        // mu_1 = r^2 / 3, mu_1t = -2/9 r^5 = -2/3 mu_1 r^3, mu_t = I1 mu_1t,
        // mu_tt = -5/3 mu_t r^3 (r = tau^{-1/3})
        const R r = rcbrt_(tau), r2 = r * r, it = r2 * r;
        cA = (R(2.0 / 3.0) * s) * r2;
        c11 = R(0);
        c1t = cA * (R(-2.0 / 3.0) * it);
        ct = c1t * (R(0.5) * I1);
        ctt = (ct * it) * R(-5.0 / 3.0);
        return true;
      }
    }
    MetricLin<D, R> L;
    if (!L.init(id, Tin)) return false;
#pragma unroll
    for (int i = 0; i < DD; ++i) {
      T[i] = L.T[i];
      C[i] = L.C[i];
    }
    const R s2 = R(2) * s;
    cA = s2 * L.m1;
    c11 = (R(2) * s2) * L.m11;
    c1t = s2 * L.m1t;
    ctt = s * L.mtt;
    ct = s * L.mt;
    return true;
  }

  __device__ __forceinline__ void dP(const R* dT, R* out) const {
    R t = R(0), d = R(0);
#pragma unroll
    for (int i = 0; i < DD; ++i) {
      t = fma(T[i], dT[i], t);
      d = fma(C[i], dT[i], d);
    }
    const R bT = fma(c11, t, c1t * d);
    const R bC = fma(c1t, t, ctt * d);
    R mdC[DD];  // s mu_t dC
    if constexpr (D == 2) {
      mdC[0] = ct * dT[3]; mdC[1] = -ct * dT[2]; mdC[2] = -ct * dT[1]; mdC[3] = ct * dT[0];
    } else {
      R U[DD];
#pragma unroll
      for (int i = 0; i < DD; ++i) U[i] = ct * T[i];
#define TMOP_DMINOR(a_, b_, c_, e_) fma(dT[a_], U[b_], fma(U[a_], dT[b_], -fma(dT[c_], U[e_], U[c_] * dT[e_])))
      mdC[0] = TMOP_DMINOR(4, 8, 5, 7);
      mdC[1] = TMOP_DMINOR(5, 6, 3, 8);
      mdC[2] = TMOP_DMINOR(3, 7, 4, 6);
      mdC[3] = TMOP_DMINOR(2, 7, 1, 8);
      mdC[4] = TMOP_DMINOR(0, 8, 2, 6);
      mdC[5] = TMOP_DMINOR(1, 6, 0, 7);
      mdC[6] = TMOP_DMINOR(1, 5, 2, 4);
      mdC[7] = TMOP_DMINOR(2, 3, 0, 5);
      mdC[8] = TMOP_DMINOR(0, 4, 1, 3);
#undef TMOP_DMINOR
    }
#pragma unroll
    for (int i = 0; i < DD; ++i) out[i] = fma(cA, dT[i], fma(bT, T[i], fma(bC, C[i], mdC[i])));
  }
};

// ---------------------------------------------------------------- contractions
// Tables in shared memory: B[q][i] = phi_i(xi_q), G[q][i] = phi_i'(xi_q).

// 2D forward. P0: X[NC][N][N] -> (P1: S[NC][2][N][Q]) -> P0: A[NC][2][Q][Q]
template <int N, int Q1, int NC, class R>
__device__ __forceinline__ void fwd2(const R* __restrict__ B, const R* __restrict__ G, R* P0, R* P1, int lane) {
  for (int t = lane; t < NC * N * Q1; t += 32) {
    const int q0 = t % Q1, j = (t / Q1) % N, c = t / (Q1 * N);
    const R* xr = P0 + (c * N + j) * N;
    R sb = R(0), sg = R(0);
#pragma unroll
    for (int i = 0; i < N; ++i) {
      const R xv = xr[i];
      sb = fma(xv, B[q0 * N + i], sb);
      sg = fma(xv, G[q0 * N + i], sg);
    }
    P1[((c * 2 + 0) * N + j) * Q1 + q0] = sb;
    P1[((c * 2 + 1) * N + j) * Q1 + q0] = sg;
  }
  __syncwarp();
  for (int t = lane; t < NC * Q1 * Q1; t += 32) {
    const int q0 = t % Q1, q1 = (t / Q1) % Q1, c = t / (Q1 * Q1);
    const R* sB = P1 + (c * 2 + 0) * N * Q1 + q0;
    const R* sG = P1 + (c * 2 + 1) * N * Q1 + q0;
    R a0 = R(0), a1 = R(0);
#pragma unroll
    for (int j = 0; j < N; ++j) {
      a0 = fma(sG[j * Q1], B[q1 * N + j], a0);  // d/dxi_0: G in x, B in y
      a1 = fma(sB[j * Q1], G[q1 * N + j], a1);  // d/dxi_1: B in x, G in y
    }
    P0[(c * 2 + 0) * Q1 * Q1 + q1 * Q1 + q0] = a0;
    P0[(c * 2 + 1) * Q1 * Q1 + q1 * Q1 + q0] = a1;
  }
  __syncwarp();
}

// 2D adjoint. P0: R[NC][2][Q][Q] -> (P1: U[NC][2][N][Q]) -> P0: Y[NC][N][N]
template <int N, int Q1, int NC, class R>
__device__ __forceinline__ void adj2(const R* __restrict__ B, const R* __restrict__ G, R* P0, R* P1, int lane) {
  for (int t = lane; t < NC * N * Q1; t += 32) {
    const int q0 = t % Q1, j = (t / Q1) % N, c = t / (Q1 * N);
    const R* r0 = P0 + (c * 2 + 0) * Q1 * Q1 + q0;
    const R* r1 = P0 + (c * 2 + 1) * Q1 * Q1 + q0;
    R u0 = R(0), u1 = R(0);
#pragma unroll
    for (int q1 = 0; q1 < Q1; ++q1) {
      u0 = fma(r0[q1 * Q1], B[q1 * N + j], u0);
      u1 = fma(r1[q1 * Q1], G[q1 * N + j], u1);
    }
    P1[((c * 2 + 0) * N + j) * Q1 + q0] = u0;  // pairs with G in x
    P1[((c * 2 + 1) * N + j) * Q1 + q0] = u1;  // pairs with B in x
  }
  __syncwarp();
  for (int t = lane; t < NC * N * N; t += 32) {
    const int i = t % N, j = (t / N) % N, c = t / (N * N);
    const R* u0 = P1 + ((c * 2 + 0) * N + j) * Q1;
    const R* u1 = P1 + ((c * 2 + 1) * N + j) * Q1;
    R y = R(0);
#pragma unroll
    for (int q0 = 0; q0 < Q1; ++q0) y = fma(u0[q0], G[q0 * N + i], fma(u1[q0], B[q0 * N + i], y));
    P0[(c * N + j) * N + i] = y;
  }
  __syncwarp();
}

// 3D forward. P0: X[NC][N][N][N] -> P1: S1[NC][2][N][N][Q] -> P0: S2[NC][3][N][Q][Q]
// -> P1: A[NC][3][Q][Q][Q]
template <int N, int Q1, int NC, class R>
__device__ __forceinline__ void fwd3(const R* __restrict__ B, const R* __restrict__ G, R* P0, R* P1, int lane) {
  constexpr int NNQ = N * N * Q1, NQQ = N * Q1 * Q1, QQ = Q1 * Q1, QQQ = Q1 * Q1 * Q1;
  for (int t = lane; t < NC * N * N * Q1; t += 32) {
    const int q0 = t % Q1, lj = (t / Q1) % (N * N), c = t / (Q1 * N * N);
    const R* xr = P0 + (c * N * N + lj) * N;
    R sb = R(0), sg = R(0);
#pragma unroll
    for (int i = 0; i < N; ++i) {
      const R xv = xr[i];
      sb = fma(xv, B[q0 * N + i], sb);
      sg = fma(xv, G[q0 * N + i], sg);
    }
    P1[(c * 2 + 0) * NNQ + lj * Q1 + q0] = sb;
    P1[(c * 2 + 1) * NNQ + lj * Q1 + q0] = sg;
  }
  __syncwarp();
  for (int t = lane; t < NC * N * QQ; t += 32) {
    const int q0 = t % Q1, q1 = (t / Q1) % Q1, l = (t / QQ) % N, c = t / (QQ * N);
    const R* xb = P1 + (c * 2 + 0) * NNQ + l * N * Q1 + q0;
    const R* xg = P1 + (c * 2 + 1) * NNQ + l * N * Q1 + q0;
    R bb = R(0), bg = R(0), gb = R(0);
#pragma unroll
    for (int j = 0; j < N; ++j) {
      const R b = xb[j * Q1], g = xg[j * Q1];
      bb = fma(b, B[q1 * N + j], bb);
      bg = fma(b, G[q1 * N + j], bg);
      gb = fma(g, B[q1 * N + j], gb);
    }
    const int o = l * QQ + q1 * Q1 + q0;
    P0[(c * 3 + 0) * NQQ + o] = bb;
    P0[(c * 3 + 1) * NQQ + o] = bg;
    P0[(c * 3 + 2) * NQQ + o] = gb;
  }
  __syncwarp();
  for (int t = lane; t < NC * QQQ; t += 32) {
    const int q01 = t % QQ, q2 = (t / QQ) % Q1, c = t / QQQ;
    const R* sbb = P0 + (c * 3 + 0) * NQQ + q01;
    const R* sbg = P0 + (c * 3 + 1) * NQQ + q01;
    const R* sgb = P0 + (c * 3 + 2) * NQQ + q01;
    R a0 = R(0), a1 = R(0), a2 = R(0);
#pragma unroll
    for (int l = 0; l < N; ++l) {
      const R bl = B[q2 * N + l], gl = G[q2 * N + l];
      a0 = fma(sgb[l * QQ], bl, a0);
      a1 = fma(sbg[l * QQ], bl, a1);
      a2 = fma(sbb[l * QQ], gl, a2);
    }
    const int o = q2 * QQ + q01;
    P1[(c * 3 + 0) * QQQ + o] = a0;
    P1[(c * 3 + 1) * QQQ + o] = a1;
    P1[(c * 3 + 2) * QQQ + o] = a2;
  }
  __syncwarp();
}

// 3D adjoint. P1: R[NC][3][Q][Q][Q] -> P0: U[NC][3][N][Q][Q] -> P1: V[NC][2][N][N][Q]
// -> P0: Y[NC][N][N][N]
template <int N, int Q1, int NC, class R>
__device__ __forceinline__ void adj3(const R* __restrict__ B, const R* __restrict__ G, R* P0, R* P1, int lane) {
  constexpr int NNQ = N * N * Q1, NQQ = N * Q1 * Q1, QQ = Q1 * Q1, QQQ = Q1 * Q1 * Q1;
  for (int t = lane; t < NC * N * QQ; t += 32) {
    const int q01 = t % QQ, l = (t / QQ) % N, c = t / (QQ * N);
    const R* r0 = P1 + (c * 3 + 0) * QQQ + q01;
    const R* r1 = P1 + (c * 3 + 1) * QQQ + q01;
    const R* r2 = P1 + (c * 3 + 2) * QQQ + q01;
    R u0 = R(0), u1 = R(0), u2 = R(0);
#pragma unroll
    for (int q2 = 0; q2 < Q1; ++q2) {
      const R bl = B[q2 * N + l], gl = G[q2 * N + l];
      u0 = fma(r0[q2 * QQ], bl, u0);
      u1 = fma(r1[q2 * QQ], bl, u1);
      u2 = fma(r2[q2 * QQ], gl, u2);
    }
    const int o = l * QQ + q01;
    P0[(c * 3 + 0) * NQQ + o] = u0;
    P0[(c * 3 + 1) * NQQ + o] = u1;
    P0[(c * 3 + 2) * NQQ + o] = u2;
  }
  __syncwarp();
  for (int t = lane; t < NC * N * N * Q1; t += 32) {
    const int q0 = t % Q1, j = (t / Q1) % N, l = (t / (Q1 * N)) % N, c = t / (Q1 * N * N);
    const R* u0 = P0 + (c * 3 + 0) * NQQ + l * QQ + q0;
    const R* u1 = P0 + (c * 3 + 1) * NQQ + l * QQ + q0;
    const R* u2 = P0 + (c * 3 + 2) * NQQ + l * QQ + q0;
    R vg = R(0), vb = R(0);
#pragma unroll
    for (int q1 = 0; q1 < Q1; ++q1) {
      const R bj = B[q1 * N + j], gj = G[q1 * N + j];
      vg = fma(u0[q1 * Q1], bj, vg);
      vb = fma(u1[q1 * Q1], gj, fma(u2[q1 * Q1], bj, vb));
    }
    const int o = (l * N + j) * Q1 + q0;
    P1[(c * 2 + 0) * NNQ + o] = vg;  // pairs with G in x
    P1[(c * 2 + 1) * NNQ + o] = vb;  // pairs with B in x
  }
  __syncwarp();
  for (int t = lane; t < NC * N * N * N; t += 32) {
    const int i = t % N, lj = (t / N) % (N * N), c = t / (N * N * N);
    const R* vg = P1 + (c * 2 + 0) * NNQ + lj * Q1;
    const R* vb = P1 + (c * 2 + 1) * NNQ + lj * Q1;
    R y = R(0);
#pragma unroll
    for (int q0 = 0; q0 < Q1; ++q0) y = fma(vg[q0], G[q0 * N + i], fma(vb[q0], B[q0 * N + i], y));
    P0[(c * N * N + lj) * N + i] = y;
  }
  __syncwarp();
}

// ---------------------------------------------------------------- folded (even-odd) 3D contractions
// The Gauss points and the Gauss-Lobatto nodes are symmetric about the
// element centre, so B[Q-1-q][N-1-i] = B[q][i] and G[Q-1-q][N-1-i] =
// -G[q][i]. In the mirror basis of each direction -- the butterfly F,
// (v_i, v_{L-1-i}) -> (v_i + v_{L-1-i}, v_i - v_{L-1-i}) stored in place at
// (i, L-1-i), the middle entry of an odd length kept -- symmetric vectors
// live on the "even" positions p < ceil(L/2) and antisymmetric ones on the
// "odd" positions, and B maps each class to itself while G swaps them. The
// folded tables Bf = S_Q^-1 F_Q B F_N S_N^-1 and Gf alike (S = F F: 2 on
// pair positions, 1 in the middle) are therefore block-sparse: an output
// position needs only the inputs of one parity, half the multiply-adds of
// the plain 1D contraction. Since F S^-1 F = I and F, S are symmetric, the
// 3D maps become
//   forward  A = F_Q^3 (Bf/Gf contractions) F_N^3 x
//   adjoint  y = F_N^3 (Bf^T/Gf^T contractions) F_Q^3 R
// with butterfly passes in place around the stage loops. For order-3 hexes
// (N = 4, Q = 5) a forward or adjoint map takes 5 010 multiply-adds and
// 3 276 butterfly operations per element where the plain one takes 10 020
// multiply-adds. Written for an even N (every output then reads N/2 inputs
// of its parity, and the adjoint stages pair the outputs (l, N-1-l)).

// Entry (p, q) of the mirror butterfly of length L (symmetric).
__device__ __forceinline__ double mirror_entry(int L, int p, int q) {
  const int m = L - 1 - p;
  if (p == m) return q == p ? 1.0 : 0.0;
  if (q == p) return p < m ? 1.0 : -1.0;
  return q == m ? 1.0 : 0.0;
}

// Bf and Gf [Q1][N] from the physical tables B, G [Q1][N] (row-major),
// computed by threads tid, tid + nth, ... of the block.
template <int N, int Q1, class R>
__device__ void folded_tables(const double* B, const double* G, R* Bf, R* Gf, int tid, int nth) {
  for (int t = tid; t < Q1 * N; t += nth) {
    const int p = t / N, r = t % N;
    double b = 0.0, g = 0.0;
    for (int q = 0; q < Q1; ++q) {
      const double fq = mirror_entry(Q1, p, q);
      if (fq == 0.0) continue;
      for (int i = 0; i < N; ++i) {
        const double fi = mirror_entry(N, i, r);
        if (fi == 0.0) continue;
        b = fma(fq * fi, B[q * N + i], b);
        g = fma(fq * fi, G[q * N + i], g);
      }
    }
    const double sp = (2 * p == Q1 - 1) ? 1.0 : 0.5, sr = (2 * r == N - 1) ? 1.0 : 0.5;
    Bf[t] = R(b * sp * sr);
    Gf[t] = R(g * sp * sr);
  }
}

// In-place butterfly along axis AX (0 fastest) of NF consecutive fields,
// each an [L2][L1][L0] array.
template <int NF, int L0, int L1, int L2, int AX, class R>
__device__ __forceinline__ void mirror3(R* buf, int lane) {
  constexpr int L = AX == 0 ? L0 : (AX == 1 ? L1 : L2);
  constexpr int H = L / 2, FS = L0 * L1 * L2, LINES = FS / L;
  constexpr int ST = AX == 0 ? 1 : (AX == 1 ? L0 : L0 * L1);
#pragma unroll 1
  for (int t = lane; t < NF * LINES * H; t += 32) {
    const int i = t % H, line = (t / H) % LINES, f = t / (H * LINES);
    int base;
    if constexpr (AX == 0) base = line * L0;
    else if constexpr (AX == 1) base = (line / L0) * (L0 * L1) + line % L0;
    else base = line;
    R* v = buf + f * FS + base;
    const R a = v[i * ST], b = v[(L - 1 - i) * ST];
    v[i * ST] = a + b;
    v[(L - 1 - i) * ST] = a - b;
  }
  __syncwarp();
}

// The butterfly along all three axes.
template <int NF, int L, class R>
__device__ __forceinline__ void mirror3_all(R* buf, int lane) {
  mirror3<NF, L, L, L, 0, R>(buf, lane);
  mirror3<NF, L, L, L, 1, R>(buf, lane);
  mirror3<NF, L, L, L, 2, R>(buf, lane);
}

// Normalised forward: every folded dot of the forward map has N/2 terms of
// one parity; scaling it by its larger coefficient (the pivot) leaves
// x[k] + r x[k^1] (N = 4: one multiply-add instead of a multiply and a
// multiply-add) or the plain copy x[k] (N = 2). For table t (0 = B, 1 = G)
// and output position p, entry t * Q1 + p of kf is the pivot's input
// position and of rt the other coefficient over the pivot (0 for a zero
// pivot, whose outputs the scale then zeroes). The stage outputs are the
// true ones divided by the pivots along the axes done so far, so the point
// fields come out divided by Sc[d][q2][q1][q0], the product of the pivots
// of direction d's tables (G along axis d, B along the others), which the
// first unfold pass multiplies back (mirror3_scaled).
template <int N, int Q1, class R>
__device__ void normalised_tables(const R* Bf, const R* Gf, int* kf, R* rt, R* piv, R* Sc, int tid, int nth) {
  static_assert(N == 2 || N == 4, "normalised folded dots are written for N / 2 = 1 or 2 terms");
  constexpr int H = N / 2, QE = (Q1 + 1) / 2, QQQ = Q1 * Q1 * Q1;
  for (int t = tid; t < 2 * Q1; t += nth) {
    const int tb = t / Q1, p = t % Q1;
    const R* T = (tb ? Gf : Bf) + p * N;
    const int base = ((p >= QE) != (tb == 1)) ? H : 0;   // B keeps the parity, G swaps it
    int k = base;
    R b = T[base];
    if (H == 2 && fabs(T[base + 1]) > fabs(b)) {
      k = base + 1;
      b = T[base + 1];
    }
    kf[t] = k;
    rt[t] = (H == 2 && b != R(0)) ? T[k ^ 1] / b : R(0);
    piv[t] = b;
  }
  __syncthreads();
  for (int t = tid; t < 3 * QQQ; t += nth) {
    const int q0 = t % Q1, q1 = (t / Q1) % Q1, q2 = (t / (Q1 * Q1)) % Q1, d = t / QQQ;
    Sc[t] = piv[(d == 0) * Q1 + q0] * piv[(d == 1) * Q1 + q1] * piv[(d == 2) * Q1 + q2];
  }
}

// The folded dot of table entry t over inputs x[0], x[stride], ...
template <int H, class R>
__device__ __forceinline__ R norm_dot(const R* x, int stride, const int* __restrict__ kf, const R* __restrict__ rt,
                                      int t) {
  const int k = kf[t];
  if constexpr (H == 2) return fma(x[(k ^ 1) * stride], rt[t], x[k * stride]);
  else return x[k * stride];
}

// Forward stages of fwd3_eo with normalised dots; P1 holds the folded A
// divided by Sc on exit.
template <int N, int Q1, int NC, class R>
__device__ __forceinline__ void fwd3_eon(const int* __restrict__ kf, const R* __restrict__ rt, R* P0, R* P1,
                                         int lane) {
  constexpr int H = N / 2;
  constexpr int NNQ = N * N * Q1, NQQ = N * Q1 * Q1, QQ = Q1 * Q1, QQQ = Q1 * Q1 * Q1;
  for (int t = lane; t < NC * N * N * Q1; t += 32) {            // rows (c, l, j) along i -> q0
    const int q0 = t % Q1, lj = (t / Q1) % (N * N), c = t / (Q1 * N * N);
    const R* xr = P0 + (c * N * N + lj) * N;
    P1[(c * 2 + 0) * NNQ + lj * Q1 + q0] = norm_dot<H>(xr, 1, kf, rt, q0);
    P1[(c * 2 + 1) * NNQ + lj * Q1 + q0] = norm_dot<H>(xr, 1, kf, rt, Q1 + q0);
  }
  __syncwarp();
  for (int t = lane; t < NC * N * QQ; t += 32) {                // (c, l, q1, q0) along j -> q1
    const int q0 = t % Q1, q1 = (t / Q1) % Q1, l = (t / QQ) % N, c = t / (QQ * N);
    const R* xb = P1 + (c * 2 + 0) * NNQ + l * N * Q1 + q0;
    const R* xg = P1 + (c * 2 + 1) * NNQ + l * N * Q1 + q0;
    const int o = l * QQ + q1 * Q1 + q0;
    P0[(c * 3 + 0) * NQQ + o] = norm_dot<H>(xb, Q1, kf, rt, q1);
    P0[(c * 3 + 1) * NQQ + o] = norm_dot<H>(xb, Q1, kf, rt, Q1 + q1);
    P0[(c * 3 + 2) * NQQ + o] = norm_dot<H>(xg, Q1, kf, rt, q1);
  }
  __syncwarp();
  for (int t = lane; t < NC * QQQ; t += 32) {                   // (c, q2, q1, q0) along l -> q2
    const int q01 = t % QQ, q2 = (t / QQ) % Q1, c = t / QQQ;
    const int o = q2 * QQ + q01;
    P1[(c * 3 + 0) * QQQ + o] = norm_dot<H>(P0 + (c * 3 + 2) * NQQ + q01, QQ, kf, rt, q2);
    P1[(c * 3 + 1) * QQQ + o] = norm_dot<H>(P0 + (c * 3 + 1) * NQQ + q01, QQ, kf, rt, q2);
    P1[(c * 3 + 2) * QQQ + o] = norm_dot<H>(P0 + (c * 3 + 0) * NQQ + q01, QQ, kf, rt, Q1 + q2);
  }
  __syncwarp();
}

// The axis-0 butterfly of fwd3_eon's point fields with Sc multiplied back
// (field f has direction f % 3; the middle entry of an odd length is scaled
// by the unit of pair 0).
template <int NF, int L, class R>
__device__ __forceinline__ void mirror3_scaled(R* buf, const R* __restrict__ Sc, int lane) {
  constexpr int H = L / 2, FS = L * L * L, LINES = L * L;
#pragma unroll 1
  for (int t = lane; t < NF * LINES * H; t += 32) {
    const int i = t % H, line = (t / H) % LINES, f = t / (H * LINES);
    R* v = buf + f * FS + line * L;
    const R* sc = Sc + (f % 3) * FS + line * L;
    const R bs = v[L - 1 - i] * sc[L - 1 - i];
    const R a = v[i], sa = sc[i];
    v[i] = fma(a, sa, bs);
    v[L - 1 - i] = fma(a, sa, -bs);
    if (L % 2 == 1 && i == 0) v[H] *= sc[H];
  }
  __syncwarp();
}

// F_Q^3 of fwd3_eon's output, Sc multiplied back on the way: A at the points.
template <int NF, int L, class R>
__device__ __forceinline__ void unfold_points(R* buf, const R* __restrict__ Sc, int lane) {
  mirror3_scaled<NF, L, R>(buf, Sc, lane);
  mirror3<NF, L, L, L, 1, R>(buf, lane);
  mirror3<NF, L, L, L, 2, R>(buf, lane);
}


// Forward stages in the folded basis; same buffer layouts as fwd3. P0 holds
// F_N^3 x on entry; P1 holds the folded A (F_Q^3 of it is A) on exit.
template <int N, int Q1, int NC, class R>
__device__ __forceinline__ void fwd3_eo(const R* __restrict__ Bf, const R* __restrict__ Gf, R* P0, R* P1, int lane) {
  static_assert(N % 2 == 0, "folded contractions need an even node count");
  constexpr int H = N / 2, QE = (Q1 + 1) / 2;
  constexpr int NNQ = N * N * Q1, NQQ = N * Q1 * Q1, QQ = Q1 * Q1, QQQ = Q1 * Q1 * Q1;
  for (int t = lane; t < NC * N * N * Q1; t += 32) {            // rows (c, l, j) along i -> q0
    const int q0 = t % Q1, lj = (t / Q1) % (N * N), c = t / (Q1 * N * N);
    const int ob = q0 < QE ? 0 : H, og = H - ob;                 // inputs of the output's parity (B), the other (G)
    const R* xr = P0 + (c * N * N + lj) * N;
    const R* tb = Bf + q0 * N;
    const R* tg = Gf + q0 * N;
    R sb = R(0), sg = R(0);
#pragma unroll
    for (int k = 0; k < H; ++k) {
      sb = fma(xr[ob + k], tb[ob + k], sb);
      sg = fma(xr[og + k], tg[og + k], sg);
    }
    P1[(c * 2 + 0) * NNQ + lj * Q1 + q0] = sb;
    P1[(c * 2 + 1) * NNQ + lj * Q1 + q0] = sg;
  }
  __syncwarp();
  for (int t = lane; t < NC * N * QQ; t += 32) {                // (c, l, q1, q0) along j -> q1
    const int q0 = t % Q1, q1 = (t / Q1) % Q1, l = (t / QQ) % N, c = t / (QQ * N);
    const int ob = q1 < QE ? 0 : H, og = H - ob;
    const R* xb = P1 + (c * 2 + 0) * NNQ + l * N * Q1 + q0;
    const R* xg = P1 + (c * 2 + 1) * NNQ + l * N * Q1 + q0;
    const R* tb = Bf + q1 * N;
    const R* tg = Gf + q1 * N;
    R bb = R(0), bg = R(0), gb = R(0);
#pragma unroll
    for (int k = 0; k < H; ++k) {
      bb = fma(xb[(ob + k) * Q1], tb[ob + k], bb);
      bg = fma(xb[(og + k) * Q1], tg[og + k], bg);
      gb = fma(xg[(ob + k) * Q1], tb[ob + k], gb);
    }
    const int o = l * QQ + q1 * Q1 + q0;
    P0[(c * 3 + 0) * NQQ + o] = bb;
    P0[(c * 3 + 1) * NQQ + o] = bg;
    P0[(c * 3 + 2) * NQQ + o] = gb;
  }
  __syncwarp();
  for (int t = lane; t < NC * QQQ; t += 32) {                   // (c, q2, q1, q0) along l -> q2
    const int q01 = t % QQ, q2 = (t / QQ) % Q1, c = t / QQQ;
    const int ob = q2 < QE ? 0 : H, og = H - ob;
    const R* sbb = P0 + (c * 3 + 0) * NQQ + q01;
    const R* sbg = P0 + (c * 3 + 1) * NQQ + q01;
    const R* sgb = P0 + (c * 3 + 2) * NQQ + q01;
    const R* tb = Bf + q2 * N;
    const R* tg = Gf + q2 * N;
    R a0 = R(0), a1 = R(0), a2 = R(0);
#pragma unroll
    for (int k = 0; k < H; ++k) {
      a0 = fma(sgb[(ob + k) * QQ], tb[ob + k], a0);
      a1 = fma(sbg[(ob + k) * QQ], tb[ob + k], a1);
      a2 = fma(sbb[(og + k) * QQ], tg[og + k], a2);
    }
    const int o = q2 * QQ + q01;
    P1[(c * 3 + 0) * QQQ + o] = a0;
    P1[(c * 3 + 1) * QQQ + o] = a1;
    P1[(c * 3 + 2) * QQQ + o] = a2;
  }
  __syncwarp();
}

// Normalised adjoint, first stage: the folded dots along q2 read Q1/2 or
// (Q1+1)/2 inputs of one parity; each is scaled by its largest coefficient
// (the pivot), taken first, so it costs one multiply-add fewer. For table
// tb (0 = B, 1 = G) and node position r, row tb * N + r of aperm lists the
// inputs in that order and of arat their coefficients over the pivot;
// apiv holds the pivot. The stage-1 outputs of node position l are then
// u0, u1 over the B pivot and u2 over the G pivot; the second stage takes
// them through C[w][l][q][j] = (pivot / s(l)) x (Bf for w = 0, 2; Gf for
// w = 1), s(l) the larger of the two pivots (1 if both are zero, whose
// outputs C then zeroes), so that its outputs, and the nodal y, carry the
// one factor s(l): the last unfold pass multiplies it back (ysc).
template <int N, int Q1, class R>
__device__ void adjoint_tables(const R* Bf, const R* Gf, int* aperm, R* arat, R* apiv, R* C, R* ysc, int tid,
                               int nth) {
  constexpr int H = N / 2, QE = (Q1 + 1) / 2;
  for (int t = tid; t < 2 * N; t += nth) {
    const int tb = t / N, r = t % N;
    const R* T = tb ? Gf : Bf;
    const bool in_odd = (r >= H) != (tb == 1);   // B keeps the parity, G swaps it
    const int q0 = in_odd ? QE : 0, M = in_odd ? Q1 - QE : QE;
    int best = q0;
    R b = T[q0 * N + r];
    for (int k = 1; k < M; ++k) {
      const R c = T[(q0 + k) * N + r];
      if (fabs(c) > fabs(b)) {
        best = q0 + k;
        b = c;
      }
    }
    int* pm = aperm + t * QE;
    R* rt = arat + t * QE;
    pm[0] = best;
    rt[0] = R(1);
    int m = 1;
    for (int k = 0; k < M; ++k) {
      const int q = q0 + k;
      if (q == best) continue;
      pm[m] = q;
      rt[m] = b != R(0) ? T[q * N + r] / b : R(0);
      ++m;
    }
    apiv[t] = b;
  }
  __syncthreads();
  for (int t = tid; t < 3 * N * Q1 * N; t += nth) {
    const int j = t % N, q = (t / N) % Q1, l = (t / (N * Q1)) % N, w = t / (N * Q1 * N);
    const R sB = apiv[l], sG = apiv[N + l];
    const R sl = fabs(sB) >= fabs(sG) ? sB : sG;
    const R f = sl != R(0) ? (w == 2 ? sG : sB) / sl : R(0);
    C[t] = f * (w == 1 ? Gf : Bf)[q * N + j];
  }
  for (int t = tid; t < N; t += nth) {
    const R sB = apiv[t], sG = apiv[N + t];
    const R sl = fabs(sB) >= fabs(sG) ? sB : sG;
    ysc[t] = sl != R(0) ? sl : R(1);
  }
}

// adj3_eo with the normalised first stage and the stage-2 tables C; P0
// holds the folded y divided by ysc[l] on exit.
template <int N, int Q1, int NC, class R>
__device__ __forceinline__ void adj3_eon(const R* __restrict__ Bf, const R* __restrict__ Gf,
                                         const int* __restrict__ aperm, const R* __restrict__ arat,
                                         const R* __restrict__ C, R* P0, R* P1, int lane) {
  static_assert(N % 2 == 0, "folded contractions need an even node count");
  constexpr int H = N / 2, QE = (Q1 + 1) / 2, QO = Q1 / 2;
  constexpr int NNQ = N * N * Q1, NQQ = N * Q1 * Q1, QQ = Q1 * Q1, QQQ = Q1 * Q1 * Q1;
  for (int t = lane; t < NC * H * QQ; t += 32) {                // (c, l pair, q1, q0) along q2 -> l
    const int q01 = t % QQ, lp = (t / QQ) % H, c = t / (QQ * H);
    const int le = lp, lo = N - 1 - lp;
    const R* r0 = P1 + (c * 3 + 0) * QQQ + q01;
    const R* r1 = P1 + (c * 3 + 1) * QQQ + q01;
    const R* r2 = P1 + (c * 3 + 2) * QQQ + q01;
    const int* pBe = aperm + le * QE;        // B column le: the even inputs
    const int* pBo = aperm + lo * QE;        // B column lo: the odd inputs
    const int* pGe = aperm + (N + le) * QE;  // G column le: the odd inputs
    const int* pGo = aperm + (N + lo) * QE;  // G column lo: the even inputs
    const R* wBe = arat + le * QE;
    const R* wBo = arat + lo * QE;
    const R* wGe = arat + (N + le) * QE;
    const R* wGo = arat + (N + lo) * QE;
    R u0e = r0[pBe[0] * QQ], u1e = r1[pBe[0] * QQ];
#pragma unroll
    for (int k = 1; k < QE; ++k) {
      const int q = pBe[k] * QQ;
      u0e = fma(r0[q], wBe[k], u0e);
      u1e = fma(r1[q], wBe[k], u1e);
    }
    R u0o = r0[pBo[0] * QQ], u1o = r1[pBo[0] * QQ];
#pragma unroll
    for (int k = 1; k < QO; ++k) {
      const int q = pBo[k] * QQ;
      u0o = fma(r0[q], wBo[k], u0o);
      u1o = fma(r1[q], wBo[k], u1o);
    }
    R u2e = r2[pGe[0] * QQ];
#pragma unroll
    for (int k = 1; k < QO; ++k) u2e = fma(r2[pGe[k] * QQ], wGe[k], u2e);
    R u2o = r2[pGo[0] * QQ];
#pragma unroll
    for (int k = 1; k < QE; ++k) u2o = fma(r2[pGo[k] * QQ], wGo[k], u2o);
    R* u = P0 + c * 3 * NQQ + q01;
    u[0 * NQQ + le * QQ] = u0e; u[0 * NQQ + lo * QQ] = u0o;
    u[1 * NQQ + le * QQ] = u1e; u[1 * NQQ + lo * QQ] = u1o;
    u[2 * NQQ + le * QQ] = u2e; u[2 * NQQ + lo * QQ] = u2o;
  }
  __syncwarp();
  for (int t = lane; t < NC * N * H * Q1; t += 32) {            // (c, l, j pair, q0) along q1 -> j
    const int q0 = t % Q1, jp = (t / Q1) % H, l = (t / (Q1 * H)) % N, c = t / (Q1 * H * N);
    const int je = jp, jo = N - 1 - jp;
    const R* u0 = P0 + (c * 3 + 0) * NQQ + l * QQ + q0;
    const R* u1 = P0 + (c * 3 + 1) * NQQ + l * QQ + q0;
    const R* u2 = P0 + (c * 3 + 2) * NQQ + l * QQ + q0;
    const R* C0 = C + (0 * N + l) * Q1 * N;
    const R* C1 = C + (1 * N + l) * Q1 * N;
    const R* C2 = C + (2 * N + l) * Q1 * N;
    R vge = R(0), vgo = R(0), vbe = R(0), vbo = R(0);
#pragma unroll
    for (int q = 0; q < QE; ++q) {
      vge = fma(u0[q * Q1], C0[q * N + je], vge);
      vbe = fma(u2[q * Q1], C2[q * N + je], vbe);
      vbo = fma(u1[q * Q1], C1[q * N + jo], vbo);
    }
#pragma unroll
    for (int q = QE; q < Q1; ++q) {
      vgo = fma(u0[q * Q1], C0[q * N + jo], vgo);
      vbo = fma(u2[q * Q1], C2[q * N + jo], vbo);
      vbe = fma(u1[q * Q1], C1[q * N + je], vbe);
    }
    R* vg = P1 + (c * 2 + 0) * NNQ + l * N * Q1 + q0;
    R* vb = P1 + (c * 2 + 1) * NNQ + l * N * Q1 + q0;
    vg[je * Q1] = vge; vg[jo * Q1] = vgo;
    vb[je * Q1] = vbe; vb[jo * Q1] = vbo;
  }
  __syncwarp();
  for (int t = lane; t < NC * N * N * H; t += 32) {             // (c, l, j, i pair) along q0 -> i
    const int ip = t % H, lj = (t / H) % (N * N), c = t / (H * N * N);
    const int ie = ip, io = N - 1 - ip;
    const R* vg = P1 + (c * 2 + 0) * NNQ + lj * Q1;
    const R* vb = P1 + (c * 2 + 1) * NNQ + lj * Q1;
    R ye = R(0), yo = R(0);
#pragma unroll
    for (int q = 0; q < QE; ++q) {
      ye = fma(vb[q], Bf[q * N + ie], ye);
      yo = fma(vg[q], Gf[q * N + io], yo);
    }
#pragma unroll
    for (int q = QE; q < Q1; ++q) {
      yo = fma(vb[q], Bf[q * N + io], yo);
      ye = fma(vg[q], Gf[q * N + ie], ye);
    }
    R* y = P0 + (c * N * N + lj) * N;
    y[ie] = ye;
    y[io] = yo;
  }
  __syncwarp();
}

// F_N^3 of adj3_eon's output, ysc multiplied back in the axis-2 pass: y at the nodes.
template <int NF, int L, class R>
__device__ __forceinline__ void unfold_nodes(R* buf, const R* __restrict__ ysc, int lane) {
  static_assert(L % 2 == 0, "even node count");
  mirror3<NF, L, L, L, 0, R>(buf, lane);
  mirror3<NF, L, L, L, 1, R>(buf, lane);
  constexpr int H = L / 2, FS = L * L * L, LINES = L * L, ST = L * L;
#pragma unroll 1
  for (int t = lane; t < NF * LINES * H; t += 32) {
    const int i = t % H, line = (t / H) % LINES, f = t / (H * LINES);
    R* v = buf + f * FS + line;
    const R bs = v[(L - 1 - i) * ST] * ysc[L - 1 - i];
    const R a = v[i * ST], sa = ysc[i];
    v[i * ST] = fma(a, sa, bs);
    v[(L - 1 - i) * ST] = fma(a, sa, -bs);
  }
  __syncwarp();
}

// Adjoint stages in the folded basis; same buffer layouts as adj3. P1 holds
// F_Q^3 R on entry; P0 holds the folded y (F_N^3 of it is y) on exit. Each
// unit computes a mirror pair of outputs: the even position l, which reads
// the even inputs through Bf and the odd ones through Gf, and the odd
// position N-1-l, the other way round.
template <int N, int Q1, int NC, class R>
__device__ __forceinline__ void adj3_eo(const R* __restrict__ Bf, const R* __restrict__ Gf, R* P0, R* P1, int lane) {
  static_assert(N % 2 == 0, "folded contractions need an even node count");
  constexpr int H = N / 2, QE = (Q1 + 1) / 2;
  constexpr int NNQ = N * N * Q1, NQQ = N * Q1 * Q1, QQ = Q1 * Q1, QQQ = Q1 * Q1 * Q1;
  for (int t = lane; t < NC * H * QQ; t += 32) {                // (c, l pair, q1, q0) along q2 -> l
    const int q01 = t % QQ, lp = (t / QQ) % H, c = t / (QQ * H);
    const int le = lp, lo = N - 1 - lp;
    const R* r0 = P1 + (c * 3 + 0) * QQQ + q01;
    const R* r1 = P1 + (c * 3 + 1) * QQQ + q01;
    const R* r2 = P1 + (c * 3 + 2) * QQQ + q01;
    R u0e = R(0), u1e = R(0), u2e = R(0), u0o = R(0), u1o = R(0), u2o = R(0);
#pragma unroll
    for (int q = 0; q < QE; ++q) {                              // even inputs
      const R be = Bf[q * N + le], go = Gf[q * N + lo];
      u0e = fma(r0[q * QQ], be, u0e);
      u1e = fma(r1[q * QQ], be, u1e);
      u2o = fma(r2[q * QQ], go, u2o);
    }
#pragma unroll
    for (int q = QE; q < Q1; ++q) {                             // odd inputs
      const R bo = Bf[q * N + lo], ge = Gf[q * N + le];
      u0o = fma(r0[q * QQ], bo, u0o);
      u1o = fma(r1[q * QQ], bo, u1o);
      u2e = fma(r2[q * QQ], ge, u2e);
    }
    R* u = P0 + c * 3 * NQQ + q01;
    u[0 * NQQ + le * QQ] = u0e; u[0 * NQQ + lo * QQ] = u0o;
    u[1 * NQQ + le * QQ] = u1e; u[1 * NQQ + lo * QQ] = u1o;
    u[2 * NQQ + le * QQ] = u2e; u[2 * NQQ + lo * QQ] = u2o;
  }
  __syncwarp();
  for (int t = lane; t < NC * N * H * Q1; t += 32) {            // (c, l, j pair, q0) along q1 -> j
    const int q0 = t % Q1, jp = (t / Q1) % H, l = (t / (Q1 * H)) % N, c = t / (Q1 * H * N);
    const int je = jp, jo = N - 1 - jp;
    const R* u0 = P0 + (c * 3 + 0) * NQQ + l * QQ + q0;
    const R* u1 = P0 + (c * 3 + 1) * NQQ + l * QQ + q0;
    const R* u2 = P0 + (c * 3 + 2) * NQQ + l * QQ + q0;
    R vge = R(0), vgo = R(0), vbe = R(0), vbo = R(0);
#pragma unroll
    for (int q = 0; q < QE; ++q) {
      const R be = Bf[q * N + je], go = Gf[q * N + jo];
      vge = fma(u0[q * Q1], be, vge);
      vbe = fma(u2[q * Q1], be, vbe);
      vbo = fma(u1[q * Q1], go, vbo);
    }
#pragma unroll
    for (int q = QE; q < Q1; ++q) {
      const R bo = Bf[q * N + jo], ge = Gf[q * N + je];
      vgo = fma(u0[q * Q1], bo, vgo);
      vbo = fma(u2[q * Q1], bo, vbo);
      vbe = fma(u1[q * Q1], ge, vbe);
    }
    R* vg = P1 + (c * 2 + 0) * NNQ + l * N * Q1 + q0;
    R* vb = P1 + (c * 2 + 1) * NNQ + l * N * Q1 + q0;
    vg[je * Q1] = vge; vg[jo * Q1] = vgo;
    vb[je * Q1] = vbe; vb[jo * Q1] = vbo;
  }
  __syncwarp();
  for (int t = lane; t < NC * N * N * H; t += 32) {             // (c, l, j, i pair) along q0 -> i
    const int ip = t % H, lj = (t / H) % (N * N), c = t / (H * N * N);
    const int ie = ip, io = N - 1 - ip;
    const R* vg = P1 + (c * 2 + 0) * NNQ + lj * Q1;
    const R* vb = P1 + (c * 2 + 1) * NNQ + lj * Q1;
    R ye = R(0), yo = R(0);
#pragma unroll
    for (int q = 0; q < QE; ++q) {
      ye = fma(vb[q], Bf[q * N + ie], ye);
      yo = fma(vg[q], Gf[q * N + io], yo);
    }
#pragma unroll
    for (int q = QE; q < Q1; ++q) {
      yo = fma(vb[q], Bf[q * N + io], yo);
      ye = fma(vg[q], Gf[q * N + ie], ye);
    }
    R* y = P0 + (c * N * N + lj) * N;
    y[ie] = ye;
    y[io] = yo;
  }
  __syncwarp();
}

// ---------------------------------------------------------------- register-blocked 3D contractions
// Same maps as fwd3/adj3 with the same buffer layouts, but each lane owns a
// whole row of outputs: it loads the row's inputs once into registers and
// takes the 1D tables from registers (tB/tG: [Q1][N], compile-time indexed),
// so a stage issues ~4x fewer shared-memory instructions. Used by the FP32
// kernels, whose throughput the shared-memory pipe otherwise bounds. Each
// loop over lanes runs its compile-time number of passes, so the index
// arithmetic folds into straight-line code.
template <int N, int Q1, int NC, class R>
__device__ __forceinline__ void fwd3_rb(const R (&tB)[Q1 * N], const R (&tG)[Q1 * N], R* P0, R* P1, int lane) {
  constexpr int NNQ = N * N * Q1, NQQ = N * Q1 * Q1, QQ = Q1 * Q1, QQQ = Q1 * Q1 * Q1;
  #pragma unroll
  for (int k = 0; k < (NC * N * N + 31) / 32; ++k) {           // (c, l, j) rows of x
    const int t = lane + 32 * k;
    if (t >= NC * N * N) break;
    const int c = t / (N * N), lj = t % (N * N);
    R xv[N];
#pragma unroll
    for (int i = 0; i < N; ++i) xv[i] = P0[t * N + i];
#pragma unroll
    for (int q0 = 0; q0 < Q1; ++q0) {
      R sb = R(0), sg = R(0);
#pragma unroll
      for (int i = 0; i < N; ++i) {
        sb = fma(xv[i], tB[q0 * N + i], sb);
        sg = fma(xv[i], tG[q0 * N + i], sg);
      }
      P1[(c * 2 + 0) * NNQ + lj * Q1 + q0] = sb;
      P1[(c * 2 + 1) * NNQ + lj * Q1 + q0] = sg;
    }
  }
  __syncwarp();
  #pragma unroll
  for (int k = 0; k < (NC * N * Q1 + 31) / 32; ++k) {          // (c, l, q0)
    const int t = lane + 32 * k;
    if (t >= NC * N * Q1) break;
    const int q0 = t % Q1, l = (t / Q1) % N, c = t / (Q1 * N);
    R xb[N], xg[N];
#pragma unroll
    for (int j = 0; j < N; ++j) {
      xb[j] = P1[(c * 2 + 0) * NNQ + (l * N + j) * Q1 + q0];
      xg[j] = P1[(c * 2 + 1) * NNQ + (l * N + j) * Q1 + q0];
    }
#pragma unroll
    for (int q1 = 0; q1 < Q1; ++q1) {
      R bb = R(0), bg = R(0), gb = R(0);
#pragma unroll
      for (int j = 0; j < N; ++j) {
        bb = fma(xb[j], tB[q1 * N + j], bb);
        bg = fma(xb[j], tG[q1 * N + j], bg);
        gb = fma(xg[j], tB[q1 * N + j], gb);
      }
      const int o = l * QQ + q1 * Q1 + q0;
      P0[(c * 3 + 0) * NQQ + o] = bb;
      P0[(c * 3 + 1) * NQQ + o] = bg;
      P0[(c * 3 + 2) * NQQ + o] = gb;
    }
  }
  __syncwarp();
  #pragma unroll
  for (int k = 0; k < (NC * QQ + 31) / 32; ++k) {              // (c, q1, q0) columns
    const int t = lane + 32 * k;
    if (t >= NC * QQ) break;
    const int c = t / QQ, q01 = t % QQ;
    R sbb[N], sbg[N], sgb[N];
#pragma unroll
    for (int l = 0; l < N; ++l) {
      sbb[l] = P0[(c * 3 + 0) * NQQ + l * QQ + q01];
      sbg[l] = P0[(c * 3 + 1) * NQQ + l * QQ + q01];
      sgb[l] = P0[(c * 3 + 2) * NQQ + l * QQ + q01];
    }
#pragma unroll
    for (int q2 = 0; q2 < Q1; ++q2) {
      R a0 = R(0), a1 = R(0), a2 = R(0);
#pragma unroll
      for (int l = 0; l < N; ++l) {
        a0 = fma(sgb[l], tB[q2 * N + l], a0);
        a1 = fma(sbg[l], tB[q2 * N + l], a1);
        a2 = fma(sbb[l], tG[q2 * N + l], a2);
      }
      const int o = q2 * QQ + q01;
      P1[(c * 3 + 0) * QQQ + o] = a0;
      P1[(c * 3 + 1) * QQQ + o] = a1;
      P1[(c * 3 + 2) * QQQ + o] = a2;
    }
  }
  __syncwarp();
}

template <int N, int Q1, int NC, class R>
__device__ __forceinline__ void adj3_rb(const R (&tB)[Q1 * N], const R (&tG)[Q1 * N], R* P0, R* P1, int lane) {
  constexpr int NNQ = N * N * Q1, NQQ = N * Q1 * Q1, QQ = Q1 * Q1, QQQ = Q1 * Q1 * Q1;
  #pragma unroll
  for (int k = 0; k < (NC * QQ + 31) / 32; ++k) {              // (c, q1, q0) columns of R
    const int t = lane + 32 * k;
    if (t >= NC * QQ) break;
    const int c = t / QQ, q01 = t % QQ;
    R r0[Q1], r1[Q1], r2[Q1];
#pragma unroll
    for (int q2 = 0; q2 < Q1; ++q2) {
      r0[q2] = P1[(c * 3 + 0) * QQQ + q2 * QQ + q01];
      r1[q2] = P1[(c * 3 + 1) * QQQ + q2 * QQ + q01];
      r2[q2] = P1[(c * 3 + 2) * QQQ + q2 * QQ + q01];
    }
#pragma unroll
    for (int l = 0; l < N; ++l) {
      R u0 = R(0), u1 = R(0), u2 = R(0);
#pragma unroll
      for (int q2 = 0; q2 < Q1; ++q2) {
        u0 = fma(r0[q2], tB[q2 * N + l], u0);
        u1 = fma(r1[q2], tB[q2 * N + l], u1);
        u2 = fma(r2[q2], tG[q2 * N + l], u2);
      }
      const int o = l * QQ + q01;
      P0[(c * 3 + 0) * NQQ + o] = u0;
      P0[(c * 3 + 1) * NQQ + o] = u1;
      P0[(c * 3 + 2) * NQQ + o] = u2;
    }
  }
  __syncwarp();
  #pragma unroll
  for (int k = 0; k < (NC * N * Q1 + 31) / 32; ++k) {          // (c, l, q0)
    const int t = lane + 32 * k;
    if (t >= NC * N * Q1) break;
    const int q0 = t % Q1, l = (t / Q1) % N, c = t / (Q1 * N);
    R u0[Q1], u1[Q1], u2[Q1];
#pragma unroll
    for (int q1 = 0; q1 < Q1; ++q1) {
      u0[q1] = P0[(c * 3 + 0) * NQQ + l * QQ + q1 * Q1 + q0];
      u1[q1] = P0[(c * 3 + 1) * NQQ + l * QQ + q1 * Q1 + q0];
      u2[q1] = P0[(c * 3 + 2) * NQQ + l * QQ + q1 * Q1 + q0];
    }
#pragma unroll
    for (int j = 0; j < N; ++j) {
      R vg = R(0), vb = R(0);
#pragma unroll
      for (int q1 = 0; q1 < Q1; ++q1) {
        vg = fma(u0[q1], tB[q1 * N + j], vg);
        vb = fma(u1[q1], tG[q1 * N + j], fma(u2[q1], tB[q1 * N + j], vb));
      }
      const int o = (l * N + j) * Q1 + q0;
      P1[(c * 2 + 0) * NNQ + o] = vg;
      P1[(c * 2 + 1) * NNQ + o] = vb;
    }
  }
  __syncwarp();
  #pragma unroll
  for (int k = 0; k < (NC * N * N + 31) / 32; ++k) {           // (c, l, j) rows of y
    const int t = lane + 32 * k;
    if (t >= NC * N * N) break;
    const int c = t / (N * N), lj = t % (N * N);
    R vg[Q1], vb[Q1];
#pragma unroll
    for (int q0 = 0; q0 < Q1; ++q0) {
      vg[q0] = P1[(c * 2 + 0) * NNQ + lj * Q1 + q0];
      vb[q0] = P1[(c * 2 + 1) * NNQ + lj * Q1 + q0];
    }
#pragma unroll
    for (int i = 0; i < N; ++i) {
      R y = R(0);
#pragma unroll
      for (int q0 = 0; q0 < Q1; ++q0) y = fma(vg[q0], tG[q0 * N + i], fma(vb[q0], tB[q0 * N + i], y));
      P0[t * N + i] = y;
    }
  }
  __syncwarp();
}

}  // namespace tmop
