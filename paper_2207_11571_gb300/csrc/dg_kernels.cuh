// The two phases of one evaluation of the DGSEM operator p(q) (Sec. 2, Eq. 3):
//
//  phase A (k_gradient): BR1 lifted gradient of (v1, v2, v3, theta = p/rho)
//     G_d = (2/h) [ D_d U + (U^ - U)|right / w_P - (U^ - U)|left / w_0 ],  U^ central,
//     then the viscous stresses and heat flux of Appendix A (Eq. A.3), optionally with
//     the Smagorinsky viscosity; writes them (9 values per node) and an operator-precision
//     copy of q that phase B reads for the neighbours' interface states.
//  phase B (k_flux): volume term -(2/h) sum_d D_d (f^a_d - f^nu_d), Roe + central-BR1
//     interface fluxes and their lifting (strong form), optional forcing s (Eq. 4), then
//     either writes dq/dt or applies one low-storage RK3 stage in FP64.
//
// Layout: each CUDA block owns E consecutive elements, one thread per node; element
// tiles (derivative matrix, per-node fields) are staged in shared memory and the 1D
// derivative contractions read them there.  Neighbour interface values are gathered
// straight from global memory (they are L2-resident: the neighbours are processed by
// nearby blocks at the same time).
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

template <typename T>
__device__ __forceinline__ void gradient_vars(const T q[5], T gm1, T U[4]) {
  const T ir = T(1) / q[0];
  U[0] = q[1] * ir;
  U[1] = q[2] * ir;
  U[2] = q[3] * ir;
  U[3] = pressure(q, gm1) * ir;
}

template <int P, typename T>
__global__ void __launch_bounds__(max_threads_for(P))
k_gradient(const double* __restrict__ q, T* __restrict__ qf, T* __restrict__ vis, Geom geom, Phys ph) {
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
  const T gm1 = T(ph.gamma - 1.0);

  T qv[5], U[4];
  if (active) {
#pragma unroll
    for (int v = 0; v < 5; ++v) qv[v] = T(q[v * N + gi]);
#pragma unroll
    for (int v = 0; v < 5; ++v) qf[v * N + gi] = qv[v];
    gradient_vars(qv, gm1, U);
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
      const int shift = right ? 1 : -1;
      const int enb = neighbour_elem(e, geom.K, d, shift);
      const long long gnb = (long long)enb * np + node + (right ? -P : P) * stride[d];
      T qn[5], Un[4];
#pragma unroll
      for (int v = 0; v < 5; ++v) qn[v] = T(q[v * N + gnb]);
      gradient_vars(qn, gm1, Un);
      const T sgn = right ? lift : -lift;
#pragma unroll
      for (int a = 0; a < 4; ++a) G[d][a] += sgn * (Un[a] - U[a]);
    }
  }

  T mu, lam;
  transport(ph, qv[0], G, &mu, &lam);
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

// MODE 0: dqdt = R.  MODE 1: RK stage g = A g + dt R, q += B g (FP64 state, register GT).
template <int P, typename T, int MODE, typename GT>
__global__ void __launch_bounds__(max_threads_for(P))
k_flux(double* __restrict__ q, const T* __restrict__ qf, const T* __restrict__ vis,
       double* __restrict__ dqdt, GT* __restrict__ greg, Forcing fc, Geom geom, Phys ph,
       double rkA, double rkB, double dt) {
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
  const T gm1 = T(ph.gamma - 1.0);

  double qd[5];
  T qv[5], vs[9], vel[3], p = T(0);
  if (active) {
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      qd[v] = q[v * N + gi];
      qv[v] = T(qd[v]);
    }
#pragma unroll
    for (int c = 0; c < 9; ++c) vs[c] = vis[c * N + gi];
    const T ir = T(1) / qv[0];
    vel[0] = qv[1] * ir;
    vel[1] = qv[2] * ir;
    vel[2] = qv[3] * ir;
    p = pressure(qv, gm1);
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
      euler_flux(qv, p, d, F);
      viscous_flux(vs, vel, d, fv);
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
    T qn[5], vn[9], veln[3];
#pragma unroll
    for (int v = 0; v < 5; ++v) qn[v] = qf[v * N + gnb];
#pragma unroll
    for (int c = 0; c < 9; ++c) vn[c] = vis[c * N + gnb];
    const T irn = T(1) / qn[0];
    veln[0] = qn[1] * irn;
    veln[1] = qn[2] * irn;
    veln[2] = qn[3] * irn;
    T Fs[5], fvo[5], fvn[5], Fo[5];
    if (right) roe_flux(qv, qn, d, gm1, Fs);
    else roe_flux(qn, qv, d, gm1, Fs);
    viscous_flux(vs, vel, d, fvo);
    viscous_flux(vn, veln, d, fvn);
    euler_flux(qv, p, d, Fo);
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
  } else {
#pragma unroll
    for (int c = 0; c < 5; ++c) {
      double gnew = dt * double(R[c]);
      if (rkA != 0.0) gnew = fma(rkA, double(greg[c * N + gi]), gnew);
      const GT gst = GT(gnew);
      greg[c * N + gi] = gst;
      q[c * N + gi] = fma(rkB, double(gst), qd[c]);
    }
  }
}

}  // namespace dgnn
