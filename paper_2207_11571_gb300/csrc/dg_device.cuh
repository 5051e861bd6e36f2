// Device-side physics of the compressible Navier-Stokes operator (Appendix A) and
// the interface fluxes of Sec. 3.1 (Roe advective, BR1 viscous), templated on the
// arithmetic type T (float: FP32 operator, double: FP64 parity operator).
//
// States are reference-shifted: s = (r, m1, m2, m3, e) with r = rho - rho_ref and
// e = rho e - E_ref (Phys); with zero references these are the conserved variables.
#pragma once

#include <cuda_runtime.h>

#include "dg_common.h"

namespace dgnn {

// Square root and reciprocal of positive arguments.  FP64: IEEE.  FP32 operator: the
// approximate hardware intrinsics (a few ulp), far below the FP32 operator's own
// rounding of the fluxes; they replace the multi-instruction IEEE sequences in the
// Roe flux and the primitive variables.
template <typename T>
__device__ __forceinline__ T dsqrt(T x);
template <>
__device__ __forceinline__ float dsqrt<float>(float x) { return x * rsqrtf(x); }
template <>
__device__ __forceinline__ double dsqrt<double>(double x) { return sqrt(x); }

template <typename T>
__device__ __forceinline__ T drcp(T x);
template <>
__device__ __forceinline__ float drcp<float>(float x) { return __fdividef(1.0f, x); }
template <>
__device__ __forceinline__ double drcp<double>(double x) { return 1.0 / x; }

// ---------------------------------------------------------------- conversions
// FP64 <-> FP32 by IEEE 754 bit manipulation on the integer pipe.  On GB300 the FP64
// pipe (which also executes F2F conversions) has a small fraction of the FP32 rate,
// so the operator converts its inputs and increments here instead.

// Round-to-nearest-even FP64 -> FP32 for finite values; magnitudes below the FP32
// normal range flush to signed zero, non-finite inputs map to NaN / Inf.
__device__ __forceinline__ float d2f_rn(double x) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const unsigned int sign = (unsigned int)(u >> 32) & 0x80000000u;
  unsigned long long a = u & 0x7FFFFFFFFFFFFFFFull;
  if (a < 0x3810000000000000ull) return __uint_as_float(sign);            // |x| < 2^-126
  if (a >= 0x47EFFFFFF0000000ull) {                                        // rounds beyond FLT_MAX, Inf, NaN
    const bool nan = a > 0x7FF0000000000000ull;
    return __uint_as_float(sign | (nan ? 0x7FC00000u : 0x7F800000u));
  }
  a += 0x0FFFFFFFull + ((a >> 29) & 1ull);   // round the 29 dropped mantissa bits, ties to even
  return __uint_as_float(sign | ((unsigned int)(a >> 29) - (896u << 23)));  // exponent bias 1023 -> 127
}

// Exact FP32 -> FP64 widening; FP32 subnormals flush to signed zero.
__device__ __forceinline__ double f2d(float x) {
  const unsigned int u = __float_as_uint(x);
  const unsigned long long sign = (unsigned long long)(u & 0x80000000u) << 32;
  const unsigned int e = (u >> 23) & 0xFFu;
  if (e == 0) return __longlong_as_double((long long)sign);
  const unsigned long long ed = (e == 0xFFu) ? 2047ull : (unsigned long long)(e + 896u);
  const unsigned long long m = (unsigned long long)(u & 0x7FFFFFu) << 29;
  return __longlong_as_double((long long)(sign | (ed << 52) | m));
}

template <typename T>
__device__ __forceinline__ T from_double(double x);
template <>
__device__ __forceinline__ float from_double<float>(double x) { return d2f_rn(x); }
template <>
__device__ __forceinline__ double from_double<double>(double x) { return x; }

// ---------------------------------------------------------------- node quantities

// Index of tau_ab in the packed 6-vector (xx, yy, zz, xy, xz, yz).
__device__ __forceinline__ int sym_index(int a, int b) {
  if (a == b) return a;
  return 2 + a + b;  // xy -> 3, xz -> 4, yz -> 5
}

// Derived quantities of a reference-shifted state.
template <typename T>
struct Prim {
  T rho, ir, v[3], pp;  // density, 1/rho, velocity, p' = p - p_ref
};

template <typename T>
__device__ __forceinline__ Prim<T> primitives(const T s[5], T rho_ref, T gm1) {
  Prim<T> w;
  w.rho = s[0] + rho_ref;
  w.ir = drcp(w.rho);
  w.v[0] = s[1] * w.ir;
  w.v[1] = s[2] * w.ir;
  w.v[2] = s[3] * w.ir;
  w.pp = gm1 * (s[4] - T(0.5) * (s[1] * w.v[0] + s[2] * w.v[1] + s[3] * w.v[2]));
  return w;
}

// Gradient variables of BR1: (v1, v2, v3, theta') with theta' = (p' - theta_ref r) / rho
// = p / rho - p_ref / rho_ref.
template <typename T>
__device__ __forceinline__ void gradient_vars(const T s[5], const Prim<T>& w, T theta_ref, T U[4]) {
  U[0] = w.v[0];
  U[1] = w.v[1];
  U[2] = w.v[2];
  U[3] = (w.pp - theta_ref * s[0]) * w.ir;
}

// Column d of the Euler flux f^a (Appendix A, Eq. A.2) without its constant part:
// (rho v_d, rho v v_d + p' e_d, v_d (rho e + p)), rho e + p = e + p' + Hc.
template <typename T>
__device__ __forceinline__ void euler_flux(const T s[5], const Prim<T>& w, T Hc, int d, T f[5]) {
  const T vd = w.v[d];
  f[0] = s[1 + d];
  f[1] = s[1] * vd;
  f[2] = s[2] * vd;
  f[3] = s[3] * vd;
  f[1 + d] += w.pp;
  f[4] = vd * (s[4] + w.pp + Hc);
}

// Column d of the viscous flux f^nu (Appendix A, Eq. A.3) from the stored viscous
// quantities vis = (tau_xx, tau_yy, tau_zz, tau_xy, tau_xz, tau_yz, k th_x, k th_y, k th_z)
// (tau already multiplied by the effective viscosity, k th by the heat coefficient):
// (0, tau_0d, tau_1d, tau_2d, sum_i v_i tau_id + k dtheta/dx_d).
template <typename T>
__device__ __forceinline__ void viscous_flux(const T vis[9], const T v[3], int d, T f[5]) {
  const T t0 = vis[sym_index(0, d)], t1 = vis[sym_index(1, d)], t2 = vis[sym_index(2, d)];
  f[0] = T(0);
  f[1] = t0;
  f[2] = t1;
  f[3] = t2;
  f[4] = v[0] * t0 + v[1] * t1 + v[2] * t2 + vis[6 + d];
}

// Roe dissipation |A~| (qR - qL) in direction +e_d between the left state sL and the
// right state sR, with Roe-averaged velocity, enthalpy and sound speed; acoustic waves
// (Vn -/+ c), entropy wave and shear waves (Vn).  The Roe flux is
// F* = (f(qL) + f(qR))/2 - diss/2.
template <typename T>
__device__ __forceinline__ void roe_dissipation(const T sL[5], const Prim<T>& wL, const T sR[5], const Prim<T>& wR,
                                                int d, T gm1, T Hc, T diss[5]) {
  const T HL = (sL[4] + wL.pp + Hc) * wL.ir, HR = (sR[4] + wR.pp + Hc) * wR.ir;
  const T sqL = dsqrt(wL.rho), sqR = dsqrt(wR.rho);
  const T wden = drcp(sqL + sqR);
  const T ut[3] = {(sqL * wL.v[0] + sqR * wR.v[0]) * wden, (sqL * wL.v[1] + sqR * wR.v[1]) * wden,
                   (sqL * wL.v[2] + sqR * wR.v[2]) * wden};
  const T Ht = (sqL * HL + sqR * HR) * wden;
  const T ke = T(0.5) * (ut[0] * ut[0] + ut[1] * ut[1] + ut[2] * ut[2]);
  const T c2 = gm1 * (Ht - ke);
  const T c = dsqrt(c2);
  const T rt = sqL * sqR;
  const T Vn = ut[d];
  const T dr = sR[0] - sL[0], dp = wR.pp - wL.pp;
  const T du[3] = {wR.v[0] - wL.v[0], wR.v[1] - wL.v[1], wR.v[2] - wL.v[2]};
  const T dVn = du[d];
  const T inv2c2 = T(0.5) * drcp(c2);
  const T a1 = (dp - rt * c * dVn) * inv2c2;
  const T a2 = dr - dp * (T(2) * inv2c2);
  const T a5 = (dp + rt * c * dVn) * inv2c2;
  const T l1 = fabs(Vn - c) * a1, l2 = fabs(Vn), l5 = fabs(Vn + c) * a5;
  diss[0] = l1 + l2 * a2 + l5;
  T shear_dot = T(0);
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const T sh = (i == d) ? T(0) : rt * du[i];  // shear wave strength (normal part removed)
    shear_dot += ut[i] * sh;
    diss[1 + i] = (l1 + l5) * ut[i] + l2 * (a2 * ut[i] + sh);
  }
  diss[1 + d] += (l5 - l1) * c;
  diss[4] = l1 * (Ht - c * Vn) + l2 * (a2 * ke + shear_dot) + l5 * (Ht + c * Vn);
}

// Roe flux F* = (f(qL) + f(qR))/2 - |A~|(qR - qL)/2 in direction +e_d.
template <typename T>
__device__ __forceinline__ void roe_flux(const T sL[5], const Prim<T>& wL, const T sR[5], const Prim<T>& wR, int d,
                                         T gm1, T Hc, T F[5]) {
  T fL[5], fR[5], diss[5];
  euler_flux(sL, wL, Hc, d, fL);
  euler_flux(sR, wR, Hc, d, fR);
  roe_dissipation(sL, wL, sR, wR, d, gm1, Hc, diss);
#pragma unroll
  for (int v = 0; v < 5; ++v) F[v] = T(0.5) * (fL[v] + fR[v] - diss[v]);
}

}  // namespace dgnn
