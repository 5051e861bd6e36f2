// Device-side physics of the compressible Navier-Stokes operator (Appendix A) and
// the interface fluxes of Sec. 3.1 (Roe advective, BR1 viscous), templated on the
// arithmetic type T (float: FP32 operator, double: FP64 parity operator).
#pragma once

#include <cuda_runtime.h>

#include "dg_common.h"

namespace dgnn {

template <typename T>
__device__ __forceinline__ T dsqrt(T x);
template <>
__device__ __forceinline__ float dsqrt<float>(float x) { return sqrtf(x); }
template <>
__device__ __forceinline__ double dsqrt<double>(double x) { return sqrt(x); }

// Index of the symmetric stress component tau_ab in the packed 6-vector
// (xx, yy, zz, xy, xz, yz).
__device__ __forceinline__ int sym_index(int a, int b) {
  if (a == b) return a;
  int s = a + b;  // 1: xy, 2: xz, 3: yz
  return 2 + s;
}

template <typename T>
__device__ __forceinline__ T pressure(const T q[5], T gm1) {
  return gm1 * (q[4] - T(0.5) * (q[1] * q[1] + q[2] * q[2] + q[3] * q[3]) / q[0]);
}

// Column d of the Euler flux f^a (Appendix A, Eq. A.2): (rho v_d, rho v v_d + p e_d, v_d (rho e + p)).
template <typename T>
__device__ __forceinline__ void euler_flux(const T q[5], T p, int d, T f[5]) {
  const T vd = q[1 + d] / q[0];
  f[0] = q[1 + d];
  f[1] = q[1] * vd;
  f[2] = q[2] * vd;
  f[3] = q[3] * vd;
  f[1 + d] += p;
  f[4] = vd * (q[4] + p);
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

// Roe flux in direction +e_d between the left state qL and the right state qR:
// F* = (f(qL) + f(qR))/2 - |A~|(qR - qL)/2 with Roe-averaged velocity, enthalpy and
// sound speed; acoustic waves (Vn -/+ c), entropy wave and shear waves (Vn).
template <typename T>
__device__ __forceinline__ void roe_flux(const T qL[5], const T qR[5], int d, T gm1, T F[5]) {
  const T rL = qL[0], rR = qR[0];
  const T iL = T(1) / rL, iR = T(1) / rR;
  const T uL[3] = {qL[1] * iL, qL[2] * iL, qL[3] * iL};
  const T uR[3] = {qR[1] * iR, qR[2] * iR, qR[3] * iR};
  const T pL = gm1 * (qL[4] - T(0.5) * rL * (uL[0] * uL[0] + uL[1] * uL[1] + uL[2] * uL[2]));
  const T pR = gm1 * (qR[4] - T(0.5) * rR * (uR[0] * uR[0] + uR[1] * uR[1] + uR[2] * uR[2]));
  const T HL = (qL[4] + pL) * iL, HR = (qR[4] + pR) * iR;
  const T sL = dsqrt(rL), sR = dsqrt(rR);
  const T wden = T(1) / (sL + sR);
  const T ut[3] = {(sL * uL[0] + sR * uR[0]) * wden, (sL * uL[1] + sR * uR[1]) * wden,
                   (sL * uL[2] + sR * uR[2]) * wden};
  const T Ht = (sL * HL + sR * HR) * wden;
  const T ke = T(0.5) * (ut[0] * ut[0] + ut[1] * ut[1] + ut[2] * ut[2]);
  const T c2 = gm1 * (Ht - ke);
  const T c = dsqrt(c2);
  const T rt = sL * sR;
  const T Vn = ut[d];
  const T dr = rR - rL, dp = pR - pL;
  const T du[3] = {uR[0] - uL[0], uR[1] - uL[1], uR[2] - uL[2]};
  const T dVn = du[d];
  const T inv2c2 = T(0.5) / c2;
  const T a1 = (dp - rt * c * dVn) * inv2c2;
  const T a2 = dr - dp * (T(2) * inv2c2);
  const T a5 = (dp + rt * c * dVn) * inv2c2;
  const T l1 = fabs(Vn - c) * a1, l2 = fabs(Vn), l5 = fabs(Vn + c) * a5;
  T fL[5], fR[5];
  euler_flux(qL, pL, d, fL);
  euler_flux(qR, pR, d, fR);
  // |A~| dq
  T diss[5];
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
#pragma unroll
  for (int v = 0; v < 5; ++v) F[v] = T(0.5) * (fL[v] + fR[v] - diss[v]);
}

// Effective viscosity and heat coefficient at a node from the velocity gradient
// G[d][a] = d u_a / d x_d (a < 3).  Smagorinsky: mu_t = rho (Cs delta)^2 sqrt(2 S:S).
template <typename T>
__device__ __forceinline__ void transport(const Phys& ph, T rho, const T G[3][4], T* mu, T* lam) {
  T m = T(ph.mu), l = T(ph.lam);
  if (ph.les) {
    T ss = T(0);
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        const T s = T(0.5) * (G[b][a] + G[a][b]);
        ss += s * s;
      }
    const T mut = rho * T(ph.csd2) * dsqrt(T(2) * ss);
    m += mut;
    l += mut * T(ph.lam_t);
  }
  *mu = m;
  *lam = l;
}

}  // namespace dgnn
