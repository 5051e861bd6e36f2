// The two phases of one evaluation of the DGSEM operator p(q) (Sec. 2, Eq. 3):
//
//  phase A (k_gradient): BR1 lifted gradient of (v1, v2, v3, theta)
//     G_d = (2/h) [ D_d U + (U^ - U)|right / w_P - (U^ - U)|left / w_0 ],  U^ central,
//     then the viscous stresses and heat flux of Appendix A (Eq. A.3), optionally with
//     the Smagorinsky viscosity.  Writes them (9 values per node) and the stage state s
//     (reference-shifted, operator precision) that phase B and the neighbours read.
//  phase B (k_flux): volume term -(2/h) sum_d D_d (f^a_d - f^nu_d), Roe + central-BR1
//     interface fluxes and their lifting (strong form), optional forcing s (Eq. 4), then
//     writes dq/dt or applies one stage of the low-storage RK3.
//
// RK3 in the FP32 operator: the state q stays FP64 and is read and written once per
// step.  Within a step the stage state is qn32 + dlt (FP32 image of q at the step start
// plus the FP32 increment accumulated by the stages); stage 3 adds the increment to q
// in FP64.  The Williamson register of stage 1 is recovered as g1 = dlt1 / B1, so only
// stage 2 stores it.  In the FP64 operator every stage updates q in FP64 (the plain
// 2N scheme).
//
// Each CUDA block owns E consecutive elements, one thread per node; element tiles (the
// derivative matrix, per-node fields) are staged in shared memory, where the 1D
// derivative contractions read them.  Neighbour interface values are gathered from
// global memory (L2-resident: neighbours are processed by nearby blocks).
#pragma once

#include "dg_device.cuh"

namespace dgnn {

// Maximum threads per block for order P (one node per thread, E elements per block).
__host__ __device__ constexpr int max_threads_for(int P) {
  return P == 1 ? 256 : P <= 4 ? 512 : P == 5 ? 448 : P == 6 ? 352 : P == 7 ? 512 : 736;
}

__device__ __forceinline__ int neighbour_elem(int e, int K, int d, int shift) {
  int c[3] = {e % K, (e / K) % K, e / (K * K)};
  c[d] = (c[d] + shift + K) % K;
  return c[0] + K * (c[1] + K * c[2]);
}

// Stage state of node gi.  SRC 0: from the FP64 state q; SRC 1: qn32 + dlt (FP32).
template <typename T, int SRC>
__device__ __forceinline__ void stage_state(const double* __restrict__ q, const float* __restrict__ qn32,
                                            const float* __restrict__ dlt, long long N, long long gi, const Phys& ph,
                                            T s[5]) {
  if (SRC == 0) {
    double qd[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) qd[v] = q[v * N + gi];
    shift_state<T>(qd, ph, s);
  } else {
#pragma unroll
    for (int v = 0; v < 5; ++v) s[v] = T(qn32[v * N + gi] + dlt[v * N + gi]);
  }
}

template <int P, typename T, int SRC>
__global__ void __launch_bounds__(max_threads_for(P))
k_gradient(const double* __restrict__ q, const float* __restrict__ qn32_in, const float* __restrict__ dlt,
           T* __restrict__ qf, float* __restrict__ qn32_out, T* __restrict__ vis, Geom geom, Phys ph) {
  constexpr int n = P + 1, n2 = n * n, np = n2 * n;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sD = reinterpret_cast<T*>(smem_raw);
  T* sU = sD + n2;
  const int E = geom.E;
  const int tileN = E * np;
  for (int t = threadIdx.x; t < n2; t += blockDim.x) sD[t] = T(geom.D[t]);

  const int le = threadIdx.x / np;
  const int node = threadIdx.x - le * np;
  const int e = blockIdx.x * E + le;
  const bool active = (le < E) && (e < geom.nel);
  const long long N = geom.N;
  const long long gi = (long long)e * np + node;
  const T gm1 = T(ph.gamma - 1.0), rho_ref = T(ph.rho_ref), th_ref = T(ph.theta_ref);

  T s[5], U[4];
  Prim<T> w;
  if (active) {
    stage_state<T, SRC>(q, qn32_in, dlt, N, gi, ph, s);
#pragma unroll
    for (int v = 0; v < 5; ++v) qf[v * N + gi] = s[v];
    if (SRC == 0 && qn32_out != nullptr) {
#pragma unroll
      for (int v = 0; v < 5; ++v) qn32_out[v * N + gi] = float(s[v]);
    }
    w = primitives(s, rho_ref, gm1);
    gradient_vars(s, w, th_ref, U);
#pragma unroll
    for (int a = 0; a < 4; ++a) sU[a * tileN + le * np + node] = U[a];
  }
  __syncthreads();
  if (!active) return;

  const int idx[3] = {node % n, (node / n) % n, node / n2};
  const int stride[3] = {1, n, n2};
  const T s2h = T(geom.two_over_h);
  const T lift = s2h * T(geom.winv) * T(0.5);
  T G[3][4];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const T* Drow = sD + idx[d] * n;
    const int base = le * np + node - idx[d] * stride[d];
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      T acc = T(0);
#pragma unroll
      for (int m = 0; m < n; ++m) acc += Drow[m] * sU[a * tileN + base + m * stride[d]];
      G[d][a] = s2h * acc;
    }
    // interface lifting with the central U^ = (U + U_nb) / 2
    const bool right = (idx[d] == P), left = (idx[d] == 0);
    if (right || left) {
      const int enb = neighbour_elem(e, geom.K, d, right ? 1 : -1);
      const long long gnb = (long long)enb * np + node + (right ? -P : P) * stride[d];
      T sn[5], Un[4];
      stage_state<T, SRC>(q, qn32_in, dlt, N, gnb, ph, sn);
      const Prim<T> wn = primitives(sn, rho_ref, gm1);
      gradient_vars(sn, wn, th_ref, Un);
      const T sgn = right ? lift : -lift;
#pragma unroll
      for (int a = 0; a < 4; ++a) G[d][a] += sgn * (Un[a] - U[a]);
    }
  }

  T mu, lam;
  transport(ph, w.rho, G, &mu, &lam);
  const T div = G[0][0] + G[1][1] + G[2][2];
  const T t23 = T(2.0 / 3.0) * mu * div;
  // G[d][a] = d u_a / d x_d, tau_ab = mu (du_a/dx_b + du_b/dx_a) - 2/3 mu div delta_ab
  T out[9];
  out[0] = T(2) * mu * G[0][0] - t23;
  out[1] = T(2) * mu * G[1][1] - t23;
  out[2] = T(2) * mu * G[2][2] - t23;
  out[3] = mu * (G[1][0] + G[0][1]);
  out[4] = mu * (G[2][0] + G[0][2]);
  out[5] = mu * (G[2][1] + G[1][2]);
  out[6] = lam * G[0][3];
  out[7] = lam * G[1][3];
  out[8] = lam * G[2][3];
#pragma unroll
  for (int c = 0; c < 9; ++c) vis[c * N + gi] = out[c];
}

// Per-launch RK data of phase B.
struct RkArgs {
  double A, B, dt;   // Williamson coefficients of the stage and the step size
  double invB1;      // 1 / B of stage 1 (the FP32 increment scheme recovers g1 = dlt1 / B1)
};

// MODE 0: dqdt = R.  MODE 1: FP64 RK stage (g = A g + dt R; q += B g, register GT).
// MODES 2, 3, 4: FP32 increment scheme, stages 1, 2, 3.
template <int P, typename T, int MODE, typename GT>
__global__ void __launch_bounds__(max_threads_for(P))
k_flux(double* __restrict__ q, const T* __restrict__ qf, const T* __restrict__ vis, double* __restrict__ dqdt,
       GT* __restrict__ greg, float* __restrict__ dlt, Forcing fc, Geom geom, Phys ph, RkArgs rk) {
  constexpr int n = P + 1, n2 = n * n, np = n2 * n;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sD = reinterpret_cast<T*>(smem_raw);
  T* sF = sD + n2;
  const int E = geom.E;
  const int tileN = E * np;
  for (int t = threadIdx.x; t < n2; t += blockDim.x) sD[t] = T(geom.D[t]);

  const int le = threadIdx.x / np;
  const int node = threadIdx.x - le * np;
  const int e = blockIdx.x * E + le;
  const bool active = (le < E) && (e < geom.nel);
  const long long N = geom.N;
  const long long gi = (long long)e * np + node;
  const T gm1 = T(ph.gamma - 1.0), rho_ref = T(ph.rho_ref), Hc = T(ph.Hc);

  T s[5], vs[9];
  Prim<T> w;
  if (active) {
#pragma unroll
    for (int v = 0; v < 5; ++v) s[v] = qf[v * N + gi];
#pragma unroll
    for (int c = 0; c < 9; ++c) vs[c] = vis[c * N + gi];
    w = primitives(s, rho_ref, gm1);
  }
  const int idx[3] = {node % n, (node / n) % n, node / n2};
  const int stride[3] = {1, n, n2};
  const T s2h = T(geom.two_over_h);
  T R[5] = {T(0), T(0), T(0), T(0), T(0)};

  // volume term, one direction at a time through shared memory
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    if (active) {
      T F[5], fv[5];
      euler_flux(s, w, Hc, d, F);
      viscous_flux(vs, w.v, d, fv);
#pragma unroll
      for (int c = 0; c < 5; ++c) sF[c * tileN + le * np + node] = F[c] - fv[c];
    }
    __syncthreads();
    if (active) {
      const T* Drow = sD + idx[d] * n;
      const int base = le * np + node - idx[d] * stride[d];
#pragma unroll
      for (int c = 0; c < 5; ++c) {
        T acc = T(0);
#pragma unroll
        for (int m = 0; m < n; ++m) acc += Drow[m] * sF[c * tileN + base + m * stride[d]];
        R[c] -= s2h * acc;
      }
    }
    __syncthreads();
  }
  if (!active) return;

  // interface fluxes and strong-form lifting
  const T lift = s2h * T(geom.winv);
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const bool right = (idx[d] == P), left = (idx[d] == 0);
    if (!(right || left)) continue;
    const int enb = neighbour_elem(e, geom.K, d, right ? 1 : -1);
    const long long gnb = (long long)enb * np + node + (right ? -P : P) * stride[d];
    T sn[5], vn[9];
#pragma unroll
    for (int v = 0; v < 5; ++v) sn[v] = qf[v * N + gnb];
#pragma unroll
    for (int c = 0; c < 9; ++c) vn[c] = vis[c * N + gnb];
    const Prim<T> wn = primitives(sn, rho_ref, gm1);
    T Fs[5], fvo[5], fvn[5], Fo[5];
    if (right) roe_flux(s, w, sn, wn, d, gm1, Hc, Fs);
    else roe_flux(sn, wn, s, w, d, gm1, Hc, Fs);
    viscous_flux(vs, w.v, d, fvo);
    viscous_flux(vn, wn.v, d, fvn);
    euler_flux(s, w, Hc, d, Fo);
    const T sgn = right ? -lift : lift;
#pragma unroll
    for (int c = 0; c < 5; ++c) {
      const T fstar = Fs[c] - T(0.5) * (fvo[c] + fvn[c]);
      R[c] += sgn * (fstar - (Fo[c] - fvo[c]));
    }
  }

  if (fc.s != nullptr) {
    const long long base = (long long)e * fc.stride + node;
#pragma unroll
    for (int c = 0; c < 5; ++c) {
      const int slot = c - fc.first_var;
      if (slot >= 0 && slot < fc.n_vars) R[c] += T(fc.s[base + (long long)slot * np]);
    }
  }

  if (MODE == 0) {
#pragma unroll
    for (int c = 0; c < 5; ++c) dqdt[c * N + gi] = double(R[c]);
  } else if (MODE == 1) {
#pragma unroll
    for (int c = 0; c < 5; ++c) {
      double gnew = rk.dt * double(R[c]);
      if (rk.A != 0.0) gnew = fma(rk.A, double(greg[c * N + gi]), gnew);
      const GT gst = GT(gnew);
      greg[c * N + gi] = gst;
      q[c * N + gi] = fma(rk.B, double(gst), q[c * N + gi]);
    }
  } else {
    // FP32 increment scheme
    const float dt = float(rk.dt), A = float(rk.A), B = float(rk.B);
#pragma unroll
    for (int c = 0; c < 5; ++c) {
      const long long o = c * N + gi;
      const float r = float(R[c]);
      if (MODE == 2) {
        dlt[o] = B * (dt * r);                       // g1 = dt R1; dlt1 = B1 g1
      } else if (MODE == 3) {
        const float d1 = dlt[o];
        const float g2 = A * (d1 * float(rk.invB1)) + dt * r;
        greg[o] = GT(g2);
        dlt[o] = d1 + B * g2;
      } else {
        const float g3 = A * float(greg[o]) + dt * r;
        const float d3 = dlt[o] + B * g3;
        q[o] = q[o] + f2d(d3);                     // once per step, in FP64
      }
    }
  }
}

}  // namespace dgnn
