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
// Each CUDA block owns E consecutive elements (or, at P <= 3 on even K, a 2 x 2 x 2 cube
// of elements whose twelve internal faces need no halo and whose internal interface
// fluxes are computed once for both sides), one thread per node for the nodal work.
// At kernel start the block issues all its global loads: its own nodes into registers
// and a halo (the neighbours' face nodes of all six faces of its elements) into shared
// memory.  Interface fluxes are dense work items, one per (element, face, face node),
// so that every lane does useful Roe work; items are ordered (face node, side,
// direction, element) so that a warp shares one face direction and every index divisor
// is a compile-time constant.  Node threads add the lifted results in a fixed order.
// The 1D derivative contractions read element tiles in shared memory.  All constants
// arrive in the operator precision (OpConst): no FP64 arithmetic or conversion runs per
// node except where the FP64 state is read or written.
#pragma once

#include <cuda_bf16.h>

#include <type_traits>

#include "dg_device.cuh"

namespace dgnn {

// Programmatic dependent launch between the operator's launches: a kernel waits until its
// predecessor in the stream has completed and its writes are visible, then lets its
// successor be launched (which happens once every block of this grid has got here, i.e.
// in its last wave), so the next launch overlaps this one's tail.  Kernels launched
// without the attribute pass the wait at once.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_release() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Maximum threads per block for order P (one node per thread, E elements per block).
__host__ __device__ constexpr int max_threads_for(int P) {
  return P == 1 ? 256 : P <= 4 ? 512 : P == 5 ? 448 : P == 6 ? 352 : P == 7 ? 512 : 736;
}

// Mesh, basis and physics constants in the operator precision T.
// Elements processed: [e_begin, nel) of a local mesh of K x K x Kz elements (a whole
// periodic mesh: e_begin = 0, nel = K^3, Kz = K; a slab of element layers with one ghost
// layer on each side: e_begin = K^2, nel = K^2 (Kz - 1), and the ghost layers hold the
// neighbouring slabs' face data).
template <typename T>
struct OpConst {
  int K, E, nel;
  int Kz, e_begin;
  long long N;
  T gm1, rho_ref, theta_ref, Hc;  // reference-shifted state (zero references in FP64)
  T s2h;                          // 2 / h
  T winv;                         // 1 / w_0 = 1 / w_P
  T mu, lam, csd2, lam_t;         // transport
  int les;
  double drho_ref, dE_ref;        // references for shifting the FP64 state
  FeatureOut feat;                // network features written by phase A (feat.out may be NULL)
  T D[kMaxN1 * kMaxN1];
};

// Element coordinates of the first element of the block (one set of divisions per thread).
struct BlockCoords {
  int x, y, z;
};

__device__ __forceinline__ BlockCoords block_coords(int e0, int K) {
  BlockCoords b;
  b.x = e0 % K;
  const int r = e0 / K;
  b.y = r % K;
  b.z = r / K;
  return b;
}

// Periodic +/-1 step of a coordinate in [0, K).
__device__ __forceinline__ int wrap_step(int x, int shift, int K) {
  x += shift;
  return x < 0 ? x + K : (x >= K ? x - K : x);
}

// Element index of block element hl shifted by +/-1 along d (periodic; Kz layers along z),
// without division.
__device__ __forceinline__ int neighbour_of(const BlockCoords& b, int hl, int K, int Kz, int d, int shift) {
  int x = b.x + hl, y = b.y, z = b.z;
  while (x >= K) {
    x -= K;
    if (++y >= K) {
      y = 0;
      ++z;
    }
  }
  if (d == 0) x = wrap_step(x, shift, K);
  else if (d == 1) y = wrap_step(y, shift, K);
  else z = wrap_step(z, shift, Kz);
  return x + K * (y + K * z);
}


// 2 x 2 x 2 element blocks ("cubes", even K): block b covers the elements 2 c + l,
// l in {0, 1}^3, of the (K/2)^3 grid of cubes; local element hl = lx + 2 ly + 4 lz.
// Each local element has one external face per direction (on side (hl >> d) & 1) and
// shares the other with local element hl ^ (1 << d).
constexpr int kCubeElems = 8;
__host__ __device__ constexpr bool cube_ok(int P) { return P <= 3; }

__device__ __forceinline__ BlockCoords cube_coords(int b, int K) {
  const int h = K >> 1;
  BlockCoords c;
  c.x = 2 * (b % h);
  const int r = b / h;
  c.y = 2 * (r % h);
  c.z = 2 * (r / h);
  return c;
}

__device__ __forceinline__ int cube_element(const BlockCoords& c, int hl, int K) {
  return (c.x + (hl & 1)) + K * ((c.y + ((hl >> 1) & 1)) + K * (c.z + (hl >> 2)));
}

// Element index of local element hl shifted by +/-1 along d (periodic).
__device__ __forceinline__ int cube_neighbour(const BlockCoords& c, int hl, int K, int d, int shift) {
  int x = c.x + (hl & 1), y = c.y + ((hl >> 1) & 1), z = c.z + (hl >> 2);
  if (d == 0) x = wrap_step(x, shift, K);
  else if (d == 1) y = wrap_step(y, shift, K);
  else z = wrap_step(z, shift, K);
  return x + K * (y + K * z);
}

// Node of the face normal to d at normal index m with tangential index ab.
template <int P>
__device__ __forceinline__ int face_node(int d, int m, int ab) {
  constexpr int n = P + 1;
  const int a = ab % n, b = ab / n;
  return d == 0 ? m + n * (a + n * b) : d == 1 ? a + n * (m + n * b) : a + n * (b + n * m);
}

// Tangential index of node (i, j, k) on a face normal to d.
template <int P>
__device__ __forceinline__ int face_ab(int d, const int idx[3]) {
  constexpr int n = P + 1;
  return d == 0 ? idx[1] + n * idx[2] : d == 1 ? idx[0] + n * idx[2] : idx[0] + n * idx[1];
}

// Derivative matrices of every order in FP32, in constant memory (one copy per
// translation unit, filled by upload_const_D on the host before the first streamed
// launch).  Read with compile-time indices, so each entry is an FFMA operand straight
// from the constant bank.
__constant__ float c_D32[kMaxP + 1][kMaxN1 * kMaxN1];

// Derivative of component f along direction D for one line of nodes (tangential index
// ab): out[node(i)] = sum_m D[i][m] f[node(m)], i = 0..P.  Each operand is read from
// shared memory once for the whole line (instead of once per output node).
template <int P, int D>
__device__ __forceinline__ void line_derivative(const float* __restrict__ f, float* __restrict__ out, int ab) {
  constexpr int n = P + 1;
  float v[n];
#pragma unroll
  for (int m = 0; m < n; ++m) v[m] = f[face_node<P>(D, m, ab)];
#pragma unroll
  for (int i = 0; i < n; ++i) {
    float acc = 0.f;
#pragma unroll
    for (int m = 0; m < n; ++m) acc += c_D32[P][i * n + m] * v[m];
    out[face_node<P>(D, i, ab)] = acc;
  }
}

// line_derivative in place: the line's values are all read before any is written, and
// no other task touches the line, so the derivative may overwrite its operand.
template <int P, int D>
__device__ __forceinline__ void line_derivative_inplace(float* f, int ab) {
  constexpr int n = P + 1;
  float v[n];
#pragma unroll
  for (int m = 0; m < n; ++m) v[m] = f[face_node<P>(D, m, ab)];
#pragma unroll
  for (int i = 0; i < n; ++i) {
    float acc = 0.f;
#pragma unroll
    for (int m = 0; m < n; ++m) acc += c_D32[P][i * n + m] * v[m];
    f[face_node<P>(D, i, ab)] = acc;
  }
}

// Halo / interface item t <-> (ab, side, d, hl), ab fastest, element slowest.
template <int P>
struct Item {
  int ab, side, d, hl;
};

template <int P>
__device__ __forceinline__ Item<P> item_of(int t) {
  constexpr int n2 = (P + 1) * (P + 1);
  Item<P> it;
  it.ab = t % n2;
  int r = t / n2;
  it.side = r & 1;
  r >>= 1;
  it.d = r % 3;
  it.hl = r / 3;
  return it;
}

template <int P>
__device__ __forceinline__ int item_index(int ab, int side, int d, int hl) {
  constexpr int n2 = (P + 1) * (P + 1);
  return ab + n2 * (side + 2 * (d + 3 * hl));
}

// External face items of a cube, t <-> (ab, hl, d), ab fastest, direction slowest (a warp
// shares d); the face lies on side (hl >> d) & 1 of local element hl.
template <int P>
__device__ __forceinline__ Item<P> cube_item_of(int t) {
  constexpr int n2 = (P + 1) * (P + 1);
  Item<P> it;
  it.ab = t % n2;
  const int r = t / n2;
  it.hl = r % kCubeElems;
  it.d = r / kCubeElems;
  it.side = (it.hl >> it.d) & 1;
  return it;
}

template <int P>
__device__ __forceinline__ int cube_item_index(int ab, int d, int hl) {
  constexpr int n2 = (P + 1) * (P + 1);
  return ab + n2 * (hl + kCubeElems * d);
}

// Internal faces of a cube, u <-> (ab, p, d): face p (0..3) normal to d joins the local
// elements hlL (bit d clear) and hlL | 1 << d.
__device__ __forceinline__ int cube_left_of_pair(int p, int d) {
  return ((p >> d) << (d + 1)) | (p & ((1 << d) - 1));
}

template <typename T>
__device__ __forceinline__ Prim<T> prim_c(const T s[5], const OpConst<T>& C) {
  return primitives(s, C.rho_ref, C.gm1);
}

// Stage state of node gi.  SRC 0: from the FP64 state q; SRC 1: qn32 + dlt (FP32).
template <typename T, int SRC>
__device__ __forceinline__ void stage_state(const double* __restrict__ q, const float* __restrict__ qn32,
                                            const float* __restrict__ dlt, long long N, long long gi,
                                            const OpConst<T>& C, T s[5]) {
  if (SRC == 0) {
    double qd[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) qd[v] = q[v * N + gi];
    s[0] = from_double<T>(qd[0] - C.drho_ref);
    s[1] = from_double<T>(qd[1]);
    s[2] = from_double<T>(qd[2]);
    s[3] = from_double<T>(qd[3]);
    s[4] = from_double<T>(qd[4] - C.dE_ref);
  } else {
#pragma unroll
    for (int v = 0; v < 5; ++v) s[v] = T(qn32[v * N + gi] + dlt[v * N + gi]);
  }
}

// Effective viscosity and heat coefficient (Smagorinsky when les != 0).
template <typename T>
__device__ __forceinline__ void transport_c(const OpConst<T>& C, T rho, const T G[3][4], T* mu, T* lam) {
  T m = C.mu, l = C.lam;
  if (C.les) {
    T ss = T(0);
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        const T s = T(0.5) * (G[b][a] + G[a][b]);
        ss += s * s;
      }
    const T mut = rho * C.csd2 * sqrt(T(2) * ss);  // IEEE square root: the argument may be zero
    m += mut;
    l += mut * C.lam_t;
  }
  *mu = m;
  *lam = l;
}

// Phase A of block `blk` of one mesh (the body of k_gradient and k_gradient_batch).
// CUBE: the block is a 2 x 2 x 2 cube of elements; the halo holds only the external
// faces, internal faces take the neighbour's values from the own tile.  SLAB: a slab of
// element layers (owned range from C.e_begin, C.Kz local layers); a whole mesh compiles
// without it.  FEAT: also write the forcing network's input features (C.feat).
template <int P, typename T, int SRC, bool CUBE = false, bool SLAB = false, bool FEAT = false>
__device__ __forceinline__ void gradient_block(int blk, const double* __restrict__ q,
                                               const float* __restrict__ qn32_in, const float* __restrict__ dlt,
                                               T* __restrict__ qf, float* __restrict__ qn32_out,
                                               T* __restrict__ vis, const OpConst<T>& C) {
  constexpr int n = P + 1, n2 = n * n, np = n2 * n;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int E = CUBE ? kCubeElems : C.E;
  const int tileN = E * np;
  const int haloN = CUBE ? 3 * kCubeElems * n2 : E * 6 * n2;
  T* sD = reinterpret_cast<T*>(smem_raw);
  T* sU = sD + n2;            // [4][E np]
  T* sH = sU + 4 * tileN;     // [4][haloN]: neighbours' gradient variables on the (external) faces
  const int e0 = (SLAB ? C.e_begin : 0) + blk * E;
  const BlockCoords bc = CUBE ? cube_coords(blk, C.K) : block_coords(e0, C.K);
  for (int t = threadIdx.x; t < n2; t += blockDim.x) sD[t] = C.D[t];

  const int le = threadIdx.x / np;
  const int node = threadIdx.x - le * np;
  const int e = CUBE ? cube_element(bc, le, C.K) : e0 + le;
  const bool active = CUBE ? (le < kCubeElems) : (le < E) && (e < C.nel);
  const long long N = C.N;
  const long long gi = (long long)e * np + node;

  T s[5], U[4];
  Prim<T> w;
  if (active) {
    stage_state<T, SRC>(q, qn32_in, dlt, N, gi, C, s);
#pragma unroll
    for (int v = 0; v < 5; ++v) qf[v * N + gi] = s[v];
    if (SRC == 0 && qn32_out != nullptr) {
#pragma unroll
      for (int v = 0; v < 5; ++v) qn32_out[v * N + gi] = float(s[v]);
    }
    if (FEAT) {
      // the forcing network's input features of this node, from the stage state just
      // formed: the same arithmetic as the separate feature kernels of the network
      __nv_bfloat16* fo = static_cast<__nv_bfloat16*>(C.feat.out) + (long long)e * C.feat.ld + node;
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        const int slot = v - C.feat.first_var;
        if (slot < 0 || slot >= C.feat.n_vars) continue;
        const int f = slot * np + node;
        float x;
        if constexpr (sizeof(T) == 4) x = (float(s[v]) - C.feat.shift32[f]) / C.feat.sd[f];
        else x = d2f_rn(double(s[v]) - C.feat.mean64[f]) / C.feat.sd[f];
        fo[slot * np] = __float2bfloat16_rn(x);
      }
    }
    w = prim_c(s, C);
    gradient_vars(s, w, C.theta_ref, U);
#pragma unroll
    for (int a = 0; a < 4; ++a) sU[a * tileN + le * np + node] = U[a];
  }
  // halo: gradient variables of the neighbours' face nodes
  for (int t = threadIdx.x; t < haloN; t += blockDim.x) {
    const Item<P> it = CUBE ? cube_item_of<P>(t) : item_of<P>(t);
    if (!CUBE && e0 + it.hl >= C.nel) continue;
    const int enb = CUBE ? cube_neighbour(bc, it.hl, C.K, it.d, it.side ? 1 : -1)
                         : neighbour_of(bc, it.hl, C.K, SLAB ? C.Kz : C.K, it.d, it.side ? 1 : -1);
    const long long gnb = (long long)enb * np + face_node<P>(it.d, it.side ? 0 : P, it.ab);
    T sn[5], Un[4];
    stage_state<T, SRC>(q, qn32_in, dlt, N, gnb, C, sn);
    const Prim<T> wn = prim_c(sn, C);
    gradient_vars(sn, wn, C.theta_ref, Un);
#pragma unroll
    for (int a = 0; a < 4; ++a) sH[a * haloN + t] = Un[a];
  }
  __syncthreads();
  // FP32 at P >= 7 (one element per block): line-wise contraction, one task per
  // (direction, variable, line) computing the derivative at every node of the line into
  // sG [3][4][np]; each operand is read from shared memory once per line (measured: -5 %
  // at P = 8, +5 % at P = 6, where the extra barrier and buffer cost more than they save)
  constexpr bool kLines = std::is_same<T, float>::value && P >= 7;
  T* sG = sH + 4 * haloN;
  if constexpr (kLines) {
    if (E == 1) {
      for (int task = threadIdx.x; task < 12 * n2; task += blockDim.x) {
        const int da = task / n2, ab = task - da * n2;
        const float* f = reinterpret_cast<const float*>(sU) + (da % 4) * np;
        float* o = reinterpret_cast<float*>(sG) + da * np;
        if (da < 4) line_derivative<P, 0>(f, o, ab);
        else if (da < 8) line_derivative<P, 1>(f, o, ab);
        else line_derivative<P, 2>(f, o, ab);
      }
      __syncthreads();
    }
  }
  if (!active) return;

  const int idx[3] = {node % n, (node / n) % n, node / n2};
  const int stride[3] = {1, n, n2};
  const T lift = C.s2h * C.winv * T(0.5);
  T G[3][4];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const T* Drow = sD + idx[d] * n;
    const int base = le * np + node - idx[d] * stride[d];
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      T acc = T(0);
      if (kLines && E == 1) {
        acc = sG[(4 * d + a) * np + node];
      } else if (P == 3 && !CUBE && std::is_same<T, float>::value && d < 2) {
        // P3 rows: an element's 64 nodes are two whole warps (node i + 4 j + 16 k), so its
        // x- and y-lines lie within one warp: the line's values come by warp shuffles of
        // the threads' own U (same products, same order: the same bits as from shared
        // memory; measured -1 % per 32^3 RK3 step); z-lines span the two warps
        const int l0 = (threadIdx.x & 31) - idx[d] * stride[d];
#pragma unroll
        for (int m = 0; m < n; ++m) acc += Drow[m] * __shfl_sync(0xffffffffu, U[a], l0 + m * stride[d]);
      } else {
#pragma unroll
        for (int m = 0; m < n; ++m) acc += Drow[m] * sU[a * tileN + base + m * stride[d]];
      }
      G[d][a] = C.s2h * acc;
    }
    // interface lifting with the central U^ = (U + U_nb) / 2
    const bool right = (idx[d] == P), left = (idx[d] == 0);
    if (right || left) {
      const int ab = face_ab<P>(d, idx);
      const T sgn = right ? lift : -lift;
      const T* nb;  // the neighbour's four values, stride st
      int st;
      if (CUBE && (right ? 1 : 0) != ((le >> d) & 1)) {
        nb = sU + (le ^ (1 << d)) * np + face_node<P>(d, right ? 0 : P, ab);   // internal face
        st = tileN;
      } else {
        nb = sH + (CUBE ? cube_item_index<P>(ab, d, le) : item_index<P>(ab, right ? 1 : 0, d, le));
        st = haloN;
      }
#pragma unroll
      for (int a = 0; a < 4; ++a) G[d][a] += sgn * (nb[a * st] - U[a]);
    }
  }

  T mu, lam;
  transport_c(C, w.rho, G, &mu, &lam);
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

template <int P, typename T, int SRC, bool CUBE = false, bool SLAB = false, bool FEAT = false>
__global__ void __launch_bounds__(max_threads_for(P))
k_gradient(const double* __restrict__ q, const float* __restrict__ qn32_in, const float* __restrict__ dlt,
           T* __restrict__ qf, float* __restrict__ qn32_out, T* __restrict__ vis, const OpConst<T> C) {
  pdl_wait();
  pdl_release();
  gradient_block<P, T, SRC, CUBE, SLAB, FEAT>(blockIdx.x, q, qn32_in, dlt, qf, qn32_out, vis, C);
}

// Per-launch RK data of phase B in the arithmetic of the update.
template <typename R>
struct RkArgs {
  R A, B, dt;   // Williamson coefficients of the stage and the step size
  R invB1;      // 1 / B of stage 1 (the FP32 increment scheme recovers g1 = dlt1 / B1)
};

// Halo and own-node components of an interface item: stage state (5) and the viscous
// quantities entering the flux normal to the face (tau_0d, tau_1d, tau_2d, k theta_d).
constexpr int kFaceComponents = 9;
// Components of the own-element tile: stage state (5) and all viscous quantities (9);
// the tile is reused for the three directions' volume fluxes (15).
constexpr int kTileComponents = 15;

// Column D of the viscous flux from the face-normal viscous quantities t4 = (tau_0D,
// tau_1D, tau_2D, k theta_D): (0, tau_0D, tau_1D, tau_2D, v . tau_D + k theta_D).
template <typename T>
__device__ __forceinline__ void viscous_flux4(const T t4[4], const T v[3], T f[5]) {
  f[0] = T(0);
  f[1] = t4[0];
  f[2] = t4[1];
  f[3] = t4[2];
  f[4] = v[0] * t4[0] + v[1] * t4[1] + v[2] * t4[2] + t4[3];
}

// One interface work item normal to D (compile-time, so flux arrays stay in registers):
//   F* - F = (f_nb - f_own - diss)/2 + (f^nu_own - f^nu_nb)/2, lifted with -/+ (2/h)/w on
// the right / left face; diss = |A~|(q_R - q_L) in the face's left/right order.
template <int D, typename T>
__device__ __forceinline__ void interface_item(const T so[5], const T to[4], const T sn[5], const T tn[4], T* out,
                                               int ostride, int side, const OpConst<T>& C) {
  const Prim<T> wo = primitives(so, C.rho_ref, C.gm1), wn = primitives(sn, C.rho_ref, C.gm1);
  T fo[5], fnb[5], fvo[5], fvn[5], diss[5];
  euler_flux(so, wo, C.Hc, D, fo);
  euler_flux(sn, wn, C.Hc, D, fnb);
  {
    // the face's left and right states by selection, not by branching: the two sides of
    // a face sit in one warp, and a branch would run the Roe solver twice
    T sL[5], sR[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      sL[v] = side ? so[v] : sn[v];
      sR[v] = side ? sn[v] : so[v];
    }
    Prim<T> wL, wR;
    wL.rho = side ? wo.rho : wn.rho;
    wR.rho = side ? wn.rho : wo.rho;
    wL.ir = side ? wo.ir : wn.ir;
    wR.ir = side ? wn.ir : wo.ir;
    wL.pp = side ? wo.pp : wn.pp;
    wR.pp = side ? wn.pp : wo.pp;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      wL.v[i] = side ? wo.v[i] : wn.v[i];
      wR.v[i] = side ? wn.v[i] : wo.v[i];
    }
    roe_dissipation(sL, wL, sR, wR, D, C.gm1, C.Hc, diss);
  }
  viscous_flux4(to, wo.v, fvo);
  viscous_flux4(tn, wn.v, fvn);
  const T lift = C.s2h * C.winv;
  const T sgn = side ? -lift : lift;
  if (sizeof(T) == 8) {
    // FP64 parity path: the plain form, F* assembled first and F subtracted after
#pragma unroll
    for (int c = 0; c < 5; ++c) {
      const T fstar = T(0.5) * (fo[c] + fnb[c] - diss[c]) - T(0.5) * (fvo[c] + fvn[c]);
      out[c * ostride] = sgn * (fstar - (fo[c] - fvo[c]));
    }
  } else {
#pragma unroll
    for (int c = 0; c < 5; ++c)
      out[c * ostride] = sgn * (T(0.5) * (fnb[c] - fo[c] - diss[c]) + T(0.5) * (fvo[c] - fvn[c]));
  }
}

// Both sides of an internal face of a cube at once: the Roe dissipation, fluxes and
// primitives are formed once; each side's lifted term is the expression interface_item
// evaluates for it (own = left element on its side 1, own = right element on its side 0).
template <int D, typename T>
__device__ __forceinline__ void interface_pair(const T sl[5], const T tl[4], const T sr[5], const T tr[4], T* outL,
                                               T* outR, int ostride, const OpConst<T>& C) {
  const Prim<T> wl = primitives(sl, C.rho_ref, C.gm1), wr = primitives(sr, C.rho_ref, C.gm1);
  T fl[5], fr[5], fvl[5], fvr[5], diss[5];
  euler_flux(sl, wl, C.Hc, D, fl);
  euler_flux(sr, wr, C.Hc, D, fr);
  roe_dissipation(sl, wl, sr, wr, D, C.gm1, C.Hc, diss);
  viscous_flux4(tl, wl.v, fvl);
  viscous_flux4(tr, wr.v, fvr);
  const T lift = C.s2h * C.winv;
  if (sizeof(T) == 8) {
#pragma unroll
    for (int c = 0; c < 5; ++c) {
      const T fstar = T(0.5) * (fl[c] + fr[c] - diss[c]) - T(0.5) * (fvl[c] + fvr[c]);
      outL[c * ostride] = -lift * (fstar - (fl[c] - fvl[c]));
      outR[c * ostride] = lift * (fstar - (fr[c] - fvr[c]));
    }
  } else {
#pragma unroll
    for (int c = 0; c < 5; ++c) {
      outL[c * ostride] = -lift * (T(0.5) * (fr[c] - fl[c] - diss[c]) + T(0.5) * (fvl[c] - fvr[c]));
      outR[c * ostride] = lift * (T(0.5) * (fl[c] - fr[c] - diss[c]) + T(0.5) * (fvr[c] - fvl[c]));
    }
  }
}

// Index of viscous component i of the face-normal set of direction d in the 9-vector.
__device__ __forceinline__ int face_vis_index(int d, int i) { return i < 3 ? sym_index(i, d) : 6 + d; }

// Halo entry t of a phase-B block: the neighbour's stage state (5) and its viscous
// quantities normal to the face (4), for a face normal to D (compile-time, so the
// component offsets are constants).
template <int D, typename T>
__device__ __forceinline__ void load_face_data(const T* __restrict__ qf, const T* __restrict__ vis, long long N,
                                               long long g, T* dst, int stride) {
  const T* s = qf + g;
  const T* w = vis + g;
#pragma unroll
  for (int v = 0; v < 5; ++v) dst[v * stride] = s[v * N];
#pragma unroll
  for (int i = 0; i < 4; ++i) dst[(5 + i) * stride] = w[face_vis_index(D, i) * N];
}

// Nodes per thread of the flux kernel.  At P >= 6 one element has 343 to 729 nodes; two
// nodes per thread halve the block so that more blocks fit an SM's registers and one
// block's barriers overlap the others' work.
__host__ __device__ constexpr int flux_npt(int P) { return P >= 6 ? 2 : 1; }

// Maximum threads per flux block.
__host__ __device__ constexpr int flux_max_threads(int P) {
  return flux_npt(P) == 1 ? max_threads_for(P) : ((max_threads_for(P) / 2 + 31) / 32) * 32;
}

// Blocks per SM the flux kernel is compiled for (register budget, about 80 registers per
// thread in FP32): several, so that one block's barriers overlap another's work; one in
// FP64 (the parity path), whose doubled register footprint would otherwise spill.
__host__ __device__ constexpr int min_blocks_for(int P, int tsize) {
  return tsize == 8 ? 1 : P == 6 ? 4 : P == 7 ? 3 : 2;
}

// Split form: a node's primitives for the two-point flux, (rho, v1, v2, v3, p', H) with
// H = (rho e + p) / rho (the reference pressure cancels in the split pressure term, so p'
// enters it; H needs the full enthalpy).
template <typename T>
__device__ __forceinline__ void store_split_prims(const T s[5], const Prim<T>& w, const OpConst<T>& C, T* out,
                                                  int stride) {
  out[0] = w.rho;
  out[stride] = w.v[0];
  out[2 * stride] = w.v[1];
  out[3 * stride] = w.v[2];
  out[4 * stride] = w.pp;
  out[5 * stride] = (s[4] + w.pp + C.Hc) * w.ir;
}

// Pirozzoli's kinetic-energy-preserving two-point flux in direction d from two nodes'
// primitives: m = {rho}{v_d}; (m, m {v_j} + {p'} delta_jd, m {H}).
template <typename T>
__device__ __forceinline__ void kep_flux_prims(const T a[6], const T b[6], int d, T F[5]) {
  const T m = T(0.25) * (a[0] + b[0]) * (a[1 + d] + b[1 + d]);
  F[0] = m;
#pragma unroll
  for (int k = 0; k < 3; ++k) F[1 + k] = m * (T(0.5) * (a[1 + k] + b[1 + k]));
  F[1 + d] += T(0.5) * (a[4] + b[4]);
  F[4] = m * (T(0.5) * (a[5] + b[5]));
}

// Phase B forms the volume fluxes before the interface phase, in a tile of their own
// (FP32 at P = 4, 5, one node per thread): one barrier less for a larger shared
// footprint.  Measured per RK3 step, 24^3/P4 408 vs 415 us, 20^3/P5 431 vs 439 us, but
// 32^3/P3 465 vs 458 us, so P <= 3 and FP64 keep the smaller footprint.
__host__ __device__ constexpr bool flux_early(int P, int tsize) { return tsize == 4 && (P == 4 || P == 5); }

// MODE 0: dqdt = R.  MODE 1: FP64 RK stage (g = A g + dt R; q += B g).
// MODES 2, 3, 4: FP32 increment scheme, stages 1, 2, 3.
// Phase B of block `blk` of one mesh (the body of k_flux and k_flux_batch).
//
// Thread j-th node: tile index tix = threadIdx.x + j blockDim.x, j < NPT.  With one node
// per thread the own state and viscous values stay in registers across the interface
// phase and the RK operands are loaded first; with two, they are read back from the
// tile and the RK operands are loaded after the interface phase (register budget).
// CUBE: the block is a 2 x 2 x 2 cube of elements; the halo holds only the external
// faces, and each internal face is one work item that writes both sides' lifted terms.
// SPLIT: the Euler part of the volume term in the kinetic-energy-preserving split form,
// 2 sum_m D_im F#(q_i, q_m) along each line with Pirozzoli's two-point flux F# (mass flux
// {rho}{v_d}; momentum m {v_j} + {p'} delta_jd; energy m {H}), from a tile of primitives;
// the viscous part and the surface terms keep the standard form.
template <int P, typename T, int MODE, bool CUBE = false, bool SPLIT = false, bool SLAB = false>
__device__ __forceinline__ void flux_block(int blk, double* __restrict__ q, const T* __restrict__ qf,
                                           const T* __restrict__ vis, double* __restrict__ dqdt,
                                           T* __restrict__ greg, float* __restrict__ dlt, const Forcing& fc,
                                           const OpConst<T>& C, const RkArgs<T>& rk) {
  constexpr int n = P + 1, n2 = n * n, np = n2 * n;
  constexpr int FC = kFaceComponents;
  constexpr int NPT = flux_npt(P);
  constexpr bool kHold = (NPT == 1);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int E = CUBE ? kCubeElems : C.E;
  const int tileN = E * np;
  const int faceN = E * 6 * n2;                          // lifted terms: every face of every element
  const int haloN = CUBE ? 3 * kCubeElems * n2 : faceN;  // neighbours' face data: external faces
  // flux_early: the volume fluxes are formed right after the own loads, into their own
  // tile, so that the interface phase and the contraction need one barrier less.
  // Otherwise they overwrite the own tile after the interface phase (register and
  // shared-memory budget).
  constexpr bool kEarlyF = flux_early(P, sizeof(T));
  T* sD = reinterpret_cast<T*>(smem_raw);
  T* sX = sD + n2;                        // own data [14][E np] (late fluxes: [15], then the fluxes)
  T* sF = kEarlyF ? sX + 14 * tileN : sX; // [15][E np]: volume fluxes
  T* sH = kEarlyF ? sF + kTileComponents * tileN : sX + kTileComponents * tileN;  // [9][E 6 n2]
  T* sS = sH + FC * haloN;                // [5][E 6 n2]: lifted interface terms
  T* sW = sS + 5 * faceN;                 // SPLIT: primitives [6][E np] (rho, v, p', H)
  const int e0 = (SLAB ? C.e_begin : 0) + blk * E;
  const BlockCoords bc = CUBE ? cube_coords(blk, C.K) : block_coords(e0, C.K);
  for (int t = threadIdx.x; t < n2; t += blockDim.x) sD[t] = C.D[t];
  const long long N = C.N;

  int le[NPT], node[NPT], tix[NPT];
  long long gi[NPT];
  bool active[NPT];
#pragma unroll
  for (int j = 0; j < NPT; ++j) {
    tix[j] = threadIdx.x + j * blockDim.x;
    le[j] = tix[j] / np;
    node[j] = tix[j] - le[j] * np;
    active[j] = CUBE ? (le[j] < kCubeElems) : (le[j] < E) && (e0 + le[j] < C.nel);
    gi[j] = (long long)(CUBE ? cube_element(bc, le[j], C.K) : e0 + le[j]) * np + node[j];
  }

  // RK operands of the update (loaded first with one node per thread, late with two)
  T gold[NPT][5], dold[NPT][5];
  // P3 rows in FP32: the x- and y-direction volume fluxes stay in registers and the
  // contraction takes a line's values by warp shuffles (an element is two whole warps, its
  // x- and y-lines lie within one); the z-fluxes go through shared memory
  constexpr bool kShfl = (P == 3) && !CUBE && !SPLIT && std::is_same<T, float>::value && !flux_early(P, sizeof(T));
  T Fr[NPT][2][5];
  auto load_rk = [&](int j) {
    if (MODE == 3 || MODE == 4) {
#pragma unroll
      for (int v = 0; v < 5; ++v) dold[j][v] = T(dlt[v * N + gi[j]]);
    }
    if (MODE == 4 || MODE == 1) {
#pragma unroll
      for (int v = 0; v < 5; ++v) gold[j][v] = (MODE == 1 && rk.A == T(0)) ? T(0) : greg[v * N + gi[j]];
      // the FP64 state is read only by the final update: start its lines towards L1 now, so
      // that read does not wait on DRAM at the end of the block (no registers held)
#pragma unroll
      for (int v = 0; v < 5; ++v) asm volatile("prefetch.global.L1 [%0];" ::"l"(q + v * N + gi[j]));
    }
    if (fc.s != nullptr) {   // likewise the forcing, added to R at the end
      const float* fs = fc.s + (gi[j] / np) * fc.stride + node[j];
      for (int slot = 0; slot < fc.n_vars; ++slot) asm volatile("prefetch.global.L1 [%0];" ::"l"(fs + slot * np));
    }
  };

  // own loads first (all independent)
  T s[NPT][5], vs[NPT][9];
  auto own_loads = [&](int j) {
#pragma unroll
    for (int v = 0; v < 5; ++v) s[j][v] = qf[v * N + gi[j]];
#pragma unroll
    for (int c = 0; c < 9; ++c) vs[j][c] = vis[c * N + gi[j]];
    if (kHold) load_rk(j);
  };
  auto own_stores = [&](int j) {
#pragma unroll
    for (int v = 0; v < 5; ++v) sX[v * tileN + tix[j]] = s[j][v];
#pragma unroll
    for (int c = 0; c < 9; ++c) sX[(5 + c) * tileN + tix[j]] = vs[j][c];
    if (kEarlyF) {
      const Prim<T> w = prim_c(s[j], C);
      if (SPLIT) store_split_prims(s[j], w, C, sW + tix[j], tileN);
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        T F[5], fv[5];
        euler_flux(s[j], w, C.Hc, d, F);
        viscous_flux(vs[j], w.v, d, fv);
#pragma unroll
        for (int c = 0; c < 5; ++c) sF[(5 * d + c) * tileN + tix[j]] = SPLIT ? -fv[c] : F[c] - fv[c];
      }
    }
  };
  // halo: neighbours' stage state and face-normal viscous quantities on every face
  auto halo_gather = [&]() {
    for (int t = threadIdx.x; t < haloN; t += blockDim.x) {
      const Item<P> it = CUBE ? cube_item_of<P>(t) : item_of<P>(t);
      if (!CUBE && e0 + it.hl >= C.nel) continue;
      const int enb = CUBE ? cube_neighbour(bc, it.hl, C.K, it.d, it.side ? 1 : -1)
                           : neighbour_of(bc, it.hl, C.K, SLAB ? C.Kz : C.K, it.d, it.side ? 1 : -1);
      const long long gnb = (long long)enb * np + face_node<P>(it.d, it.side ? 0 : P, it.ab);
      switch (it.d) {
        case 0: load_face_data<0>(qf, vis, N, gnb, sH + t, haloN); break;
        case 1: load_face_data<1>(qf, vis, N, gnb, sH + t, haloN); break;
        default: load_face_data<2>(qf, vis, N, gnb, sH + t, haloN);
      }
    }
  };
  if (kHold) {
    // one node per thread: the own values stay in registers anyway, so their tile stores
    // wait until the halo gathers are issued and the two latencies overlap
#pragma unroll
    for (int j = 0; j < NPT; ++j)
      if (active[j]) own_loads(j);
    halo_gather();
#pragma unroll
    for (int j = 0; j < NPT; ++j)
      if (active[j]) own_stores(j);
  } else {
#pragma unroll
    for (int j = 0; j < NPT; ++j)
      if (active[j]) {
        own_loads(j);
        own_stores(j);
      }
    halo_gather();
  }
  __syncthreads();

  // interface terms, one work item per (element, face, face node); in a cube, the
  // external faces first, then one item per internal face node for both sides
  const int nItems = CUBE ? haloN + 12 * n2 : haloN;
  for (int t = threadIdx.x; t < nItems; t += blockDim.x) {
    if (!CUBE || t < haloN) {
      const Item<P> it = CUBE ? cube_item_of<P>(t) : item_of<P>(t);
      if (!CUBE && e0 + it.hl >= C.nel) continue;
      const int o = it.hl * np + face_node<P>(it.d, it.side ? P : 0, it.ab);
      T* out = sS + (CUBE ? item_index<P>(it.ab, it.side, it.d, it.hl) : t);
      T so[5], to[4], sn[5], tn[4];
#pragma unroll
      for (int v = 0; v < 5; ++v) so[v] = sX[v * tileN + o];
#pragma unroll
      for (int v = 0; v < 5; ++v) sn[v] = sH[v * haloN + t];
#pragma unroll
      for (int i = 0; i < 4; ++i) tn[i] = sH[(5 + i) * haloN + t];
      switch (it.d) {
        case 0:
#pragma unroll
          for (int i = 0; i < 4; ++i) to[i] = sX[(5 + face_vis_index(0, i)) * tileN + o];
          interface_item<0>(so, to, sn, tn, out, faceN, it.side, C);
          break;
        case 1:
#pragma unroll
          for (int i = 0; i < 4; ++i) to[i] = sX[(5 + face_vis_index(1, i)) * tileN + o];
          interface_item<1>(so, to, sn, tn, out, faceN, it.side, C);
          break;
        default:
#pragma unroll
          for (int i = 0; i < 4; ++i) to[i] = sX[(5 + face_vis_index(2, i)) * tileN + o];
          interface_item<2>(so, to, sn, tn, out, faceN, it.side, C);
      }
    } else {
      const int u = t - haloN;
      const int ab = u % n2, r = u / n2, d = r >> 2;
      const int hlL = cube_left_of_pair(r & 3, d), hlR = hlL | (1 << d);
      const int oL = hlL * np + face_node<P>(d, P, ab), oR = hlR * np + face_node<P>(d, 0, ab);
      T* outL = sS + item_index<P>(ab, 1, d, hlL);
      T* outR = sS + item_index<P>(ab, 0, d, hlR);
      T sl[5], tl[4], sr[5], tr[4];
#pragma unroll
      for (int v = 0; v < 5; ++v) sl[v] = sX[v * tileN + oL];
#pragma unroll
      for (int v = 0; v < 5; ++v) sr[v] = sX[v * tileN + oR];
      switch (d) {
        case 0:
#pragma unroll
          for (int i = 0; i < 4; ++i) tl[i] = sX[(5 + face_vis_index(0, i)) * tileN + oL];
#pragma unroll
          for (int i = 0; i < 4; ++i) tr[i] = sX[(5 + face_vis_index(0, i)) * tileN + oR];
          interface_pair<0>(sl, tl, sr, tr, outL, outR, faceN, C);
          break;
        case 1:
#pragma unroll
          for (int i = 0; i < 4; ++i) tl[i] = sX[(5 + face_vis_index(1, i)) * tileN + oL];
#pragma unroll
          for (int i = 0; i < 4; ++i) tr[i] = sX[(5 + face_vis_index(1, i)) * tileN + oR];
          interface_pair<1>(sl, tl, sr, tr, outL, outR, faceN, C);
          break;
        default:
#pragma unroll
          for (int i = 0; i < 4; ++i) tl[i] = sX[(5 + face_vis_index(2, i)) * tileN + oL];
#pragma unroll
          for (int i = 0; i < 4; ++i) tr[i] = sX[(5 + face_vis_index(2, i)) * tileN + oR];
          interface_pair<2>(sl, tl, sr, tr, outL, outR, faceN, C);
      }
    }
  }
  __syncthreads();  // own-data tile no longer needed: (late fluxes) it now takes the volume fluxes

#pragma unroll
  for (int j = 0; j < NPT; ++j) {
    if (kEarlyF || !active[j]) continue;
    if (!kHold) {
      load_rk(j);
#pragma unroll
      for (int v = 0; v < 5; ++v) s[j][v] = sX[v * tileN + tix[j]];
#pragma unroll
      for (int c = 0; c < 9; ++c) vs[j][c] = sX[(5 + c) * tileN + tix[j]];
    }
    const Prim<T> w = prim_c(s[j], C);
    if (SPLIT) store_split_prims(s[j], w, C, sW + tix[j], tileN);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      T F[5], fv[5];
      euler_flux(s[j], w, C.Hc, d, F);
      viscous_flux(vs[j], w.v, d, fv);
#pragma unroll
      for (int c = 0; c < 5; ++c) {
        const T fd = SPLIT ? -fv[c] : F[c] - fv[c];
        if (kShfl && d < 2) Fr[j][d][c] = fd;
        else sX[(5 * d + c) * tileN + tix[j]] = fd;
      }
    }
  }
  if (!kEarlyF) __syncthreads();

#pragma unroll
  for (int j = 0; j < NPT; ++j) {
    if (!active[j]) continue;
    const int nd = node[j], lj = le[j];
    const long long g = gi[j];
    // volume term -(2/h) sum_d D_d F_d, then the lifted interface terms (fixed order x, y, z)
    const int idx[3] = {nd % n, (nd / n) % n, nd / n2};
    const int stride[3] = {1, n, n2};
    T R[5] = {T(0), T(0), T(0), T(0), T(0)};
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const T* Drow = sD + idx[d] * n;
      const int base = lj * np + nd - idx[d] * stride[d];
#pragma unroll
      for (int c = 0; c < 5; ++c) {
        T acc = T(0);
        if (kShfl && d < 2) {
          const int l0 = (threadIdx.x & 31) - idx[d] * stride[d];
#pragma unroll
          for (int m = 0; m < n; ++m) acc += Drow[m] * __shfl_sync(0xffffffffu, Fr[j][d][c], l0 + m * stride[d]);
        } else {
#pragma unroll
          for (int m = 0; m < n; ++m) acc += Drow[m] * sF[(5 * d + c) * tileN + base + m * stride[d]];
        }
        R[c] -= C.s2h * acc;
      }
    }
    if (SPLIT) {
      const int ti = tix[j];
      T wi[6];
#pragma unroll
      for (int k = 0; k < 6; ++k) wi[k] = sW[k * tileN + ti];
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const T* Drow = sD + idx[d] * n;
        const int base = lj * np + nd - idx[d] * stride[d];
        T acc[5] = {T(0), T(0), T(0), T(0), T(0)};
#pragma unroll
        for (int m = 0; m < n; ++m) {
          const int o = base + m * stride[d];
          T wm[6];
#pragma unroll
          for (int k = 0; k < 6; ++k) wm[k] = sW[k * tileN + o];
          T F[5];
          kep_flux_prims(wi, wm, d, F);
#pragma unroll
          for (int c = 0; c < 5; ++c) acc[c] += Drow[m] * F[c];
        }
#pragma unroll
        for (int c = 0; c < 5; ++c) R[c] -= C.s2h * (T(2) * acc[c]);
      }
    }
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const bool right = (idx[d] == P), left = (idx[d] == 0);
      if (!(right || left)) continue;
      const int h = item_index<P>(face_ab<P>(d, idx), right ? 1 : 0, d, lj);
#pragma unroll
      for (int c = 0; c < 5; ++c) R[c] += sS[c * faceN + h];
    }

    if (fc.s != nullptr) {
      const long long base = (g / np) * fc.stride + nd;
#pragma unroll
      for (int c = 0; c < 5; ++c) {
        const int slot = c - fc.first_var;
        if (slot >= 0 && slot < fc.n_vars) R[c] += T(fc.s[base + (long long)slot * np]);
      }
    }

    if (MODE == 0) {
#pragma unroll
      for (int c = 0; c < 5; ++c) dqdt[c * N + g] = double(R[c]);
    } else if (MODE == 1) {
      // FP64 operator: plain 2N update of the FP64 state
#pragma unroll
      for (int c = 0; c < 5; ++c) {
        const long long o = c * N + g;
        T gnew = rk.dt * R[c];
        if (rk.A != T(0)) gnew = rk.A * gold[j][c] + gnew;
        greg[o] = gnew;
        q[o] = double(rk.B) * double(gnew) + q[o];
      }
    } else {
      // FP32 increment scheme
#pragma unroll
      for (int c = 0; c < 5; ++c) {
        const long long o = c * N + g;
        if (MODE == 2) {
          dlt[o] = float(rk.B * (rk.dt * R[c]));                 // g1 = dt R1; dlt1 = B1 g1
        } else if (MODE == 3) {
          const T g2 = rk.A * (dold[j][c] * rk.invB1) + rk.dt * R[c];
          greg[o] = g2;
          dlt[o] = float(dold[j][c] + rk.B * g2);
        } else {
          const T g3 = rk.A * gold[j][c] + rk.dt * R[c];
          const float d3 = float(dold[j][c] + rk.B * g3);
          q[o] = q[o] + f2d(d3);                                 // once per step, in FP64
        }
      }
    }
  }
}

template <int P, typename T, int MODE, bool CUBE = false, bool SPLIT = false, bool SLAB = false>
__global__ void __launch_bounds__(flux_max_threads(P), min_blocks_for(P, sizeof(T)))
k_flux(double* __restrict__ q, const T* __restrict__ qf, const T* __restrict__ vis, double* __restrict__ dqdt,
       T* __restrict__ greg, float* __restrict__ dlt, Forcing fc, const OpConst<T> C, RkArgs<T> rk) {
  pdl_wait();
  pdl_release();
  flux_block<P, T, MODE, CUBE, SPLIT, SLAB>(blockIdx.x, q, qf, vis, dqdt, greg, dlt, fc, C, rk);
}

// ---------------------------------------------------------------------------------------
// Batched launches: independent meshes of the same order P (different K, Re, closure,
// dt) share one launch.  Block b belongs to the instance whose block range holds it; the
// table travels as one kernel parameter, so its per-instance constants are read from the
// constant bank like the single-mesh kernels' own.
constexpr int kMaxBatch = 16;

template <typename T>
struct BatchTable {
  int n;                             // instances in this launch
  int block_start[kMaxBatch + 1];    // first block of each instance; block_start[n] = grid
  double* q[kMaxBatch];              // FP64 states
  float* qn32[kMaxBatch];            // FP32 operator: step-start image (NULL in FP64)
  float* dlt[kMaxBatch];             // FP32 operator: stage increment (NULL in FP64)
  T* qf[kMaxBatch];                  // stage state
  T* vis[kMaxBatch];                 // viscous quantities
  T* g[kMaxBatch];                   // RK register
  RkArgs<T> rk[kMaxBatch];
  OpConst<T> C[kMaxBatch];
  int bulk[kMaxBatch];               // streamed phase B: own tiles by TMA bulk copies (see StreamMesh)
  int* err[kMaxBatch];               // device error flag of the instance (may be NULL)
};

__device__ __forceinline__ int batch_instance(const int* start, int n, int b) {
  int i = 0;
  while (i + 1 < n && b >= start[i + 1]) ++i;
  return i;
}

template <int P, typename T, int SRC>
__global__ void __launch_bounds__(max_threads_for(P))
k_gradient_batch(const __grid_constant__ BatchTable<T> tb) {
  pdl_wait();
  pdl_release();
  const int i = batch_instance(tb.block_start, tb.n, blockIdx.x);
  gradient_block<P, T, SRC>(blockIdx.x - tb.block_start[i], tb.q[i], tb.qn32[i], tb.dlt[i], tb.qf[i],
                            SRC == 0 ? tb.qn32[i] : nullptr, tb.vis[i], tb.C[i]);
}

template <int P, typename T, int MODE>
__global__ void __launch_bounds__(flux_max_threads(P), min_blocks_for(P, sizeof(T)))
k_flux_batch(const __grid_constant__ BatchTable<T> tb) {
  pdl_wait();
  pdl_release();
  const int i = batch_instance(tb.block_start, tb.n, blockIdx.x);
  flux_block<P, T, MODE>(blockIdx.x - tb.block_start[i], tb.q[i], tb.qf[i], tb.vis[i], nullptr, tb.g[i],
                         tb.dlt[i], Forcing{}, tb.C[i], tb.rk[i]);
}

// ---------------------------------------------------------------------------------------
// Streamed phase B for high orders (FP32 operator, P >= 6, one element per work item).
//
// At P >= 6 an element's phase B is latency-bound when its loads and its arithmetic
// alternate: the block waits for the own tile and the face halo, then computes with no
// memory traffic in flight.  The streamed kernel is persistent: each block walks the
// elements blockIdx.x, blockIdx.x + gridDim.x, ... and, while it computes element k,
// copies element k + 1's tile (TMA bulk copies, one per component row) and face halo
// (4-byte cp.async) into the other half of a double buffer, straight to shared memory
// with no registers held.  The per-node and per-item arithmetic is flux_block's.

__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
               "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// TMA bulk copies (cp.async.bulk, global -> shared, completion counted in bytes on an
// mbarrier).  Addresses 16-byte aligned, size a multiple of 16 bytes.
__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void bulk_bar_init(unsigned long long* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ void bulk_bar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void bulk_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_copy(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_addr(dst)),
               "l"(src), "r"(bytes), "r"(smem_addr(bar))
               : "memory");
}
// Bounded wait for the phase with the given parity (about a second); false on expiry.
__device__ __forceinline__ bool bulk_wait(unsigned long long* bar, unsigned parity) {
  const long long t0 = clock64();
  for (;;) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n"
        " mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    if (ok) return true;
    if (clock64() - t0 > 2000000000LL) return false;
  }
}

// load_face_data with cp.async (no registers held while the copies fly).
template <int D>
__device__ __forceinline__ void copy_face_data(const float* qf, const float* vis, long long N, long long g,
                                               float* dst, int stride) {
  const float* s = qf + g;
  const float* w = vis + g;
#pragma unroll
  for (int v = 0; v < 5; ++v) cp_async4(dst + v * stride, s + v * N);
#pragma unroll
  for (int i = 0; i < 4; ++i) cp_async4(dst + (5 + i) * stride, w + face_vis_index(D, i) * N);
}

// Threads of a streamed block: one per node.
// One warp more where that saves a round of the 15 (P+1)^2 line-derivative tasks (P = 6:
// 735 tasks take two rounds of 384 threads instead of three of 352).
__host__ __device__ constexpr int stream_threads(int P) {
  return ((15 * (P + 1) * (P + 1) + ((((P + 1) * (P + 1) * (P + 1) + 31) / 32) * 32) - 1) /
              ((((P + 1) * (P + 1) * (P + 1) + 31) / 32) * 32) >
          (15 * (P + 1) * (P + 1) + ((((P + 1) * (P + 1) * (P + 1) + 31) / 32) * 32 + 32) - 1) /
              ((((P + 1) * (P + 1) * (P + 1) + 31) / 32) * 32 + 32))
             ? ((((P + 1) * (P + 1) * (P + 1) + 31) / 32) * 32 + 32)
             : ((((P + 1) * (P + 1) * (P + 1) + 31) / 32) * 32);
}
static_assert(stream_threads(6) == 384 && stream_threads(7) == 512 && stream_threads(8) == 736, "stream block sizes");
// Blocks per SM the streamed kernel is compiled for (shared memory allows two at P <= 7).
__host__ __device__ constexpr int stream_min_blocks(int P) { return P <= 7 ? 2 : 1; }

// One mesh's operands as seen by a streamed work item.
struct StreamItem {
  double* q;
  const float* qf;
  const float* vis;
  double* dqdt;
  float* greg;
  float* dlt;
  const OpConst<float>* C;
  const RkArgs<float>* rk;
  Forcing fc;
  int e;     // element
  int bulk;  // own tile by TMA bulk copies (every component row 16-byte aligned modulo the element shift)
  int* err;  // device error flag (may be NULL)
};

// Shared memory of the streamed kernel, in floats: two mbarriers (4 floats), the
// per-direction volume fluxes and then their derivatives [3][5][np], and two 16-byte
// aligned buffers of (own tile [14][kTS], halo [9][6 n2]); the interface items write
// their lifted terms over the halo slots they read (components 0-4), so that the
// footprint leaves room for the L1 cache that the halo gathers and RK loads go through.  An own-tile row has
// room for the element's 0-3 float misalignment (node nd of component c at c kTS + sh + nd,
// sh = (e np) mod 4), so that the bulk copies land on 16-byte boundaries.
template <int P>
__host__ __device__ constexpr int stream_tile_stride() { return ((P + 1) * (P + 1) * (P + 1) + 3 + 3) & ~3; }
template <int P>
__host__ __device__ constexpr int stream_buf_floats() {
  return (14 * stream_tile_stride<P>() + kFaceComponents * 6 * (P + 1) * (P + 1) + 3) & ~3;
}
template <int P>
__host__ __device__ constexpr int stream_buf_offset() {
  return (4 + 15 * (P + 1) * (P + 1) * (P + 1) + 3) & ~3;
}
template <int P>
__host__ __device__ constexpr int stream_smem_floats() {
  return stream_buf_offset<P>() + 2 * stream_buf_floats<P>();
}



template <int P, int MODE, class Src>
__device__ __forceinline__ void flux_stream(const Src& src, int n_items) {
  using T = float;
  constexpr int n = P + 1, n2 = n * n, np = n2 * n, haloN = 6 * n2;
  constexpr int FC = kFaceComponents;
  constexpr int kTS = stream_tile_stride<P>();
  constexpr int kBuf = stream_buf_floats<P>();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned long long* bar = reinterpret_cast<unsigned long long*>(smem_raw);  // one per buffer
  T* sV = reinterpret_cast<T*>(smem_raw) + 4;  // [3][5][np]: volume fluxes, then their derivatives
  T* buf0 = reinterpret_cast<T*>(smem_raw) + stream_buf_offset<P>();  // two buffers: own tile, halo

  // element k + 1's own tile and halo into buffer bi; the own tile's rows by one bulk
  // copy each (16-byte aligned interior, issued by thread 0, counted on bar[bi]) and their
  // 0-3 float ragged ends by 4-byte cp.async, or (unaligned layouts) all by cp.async
  auto prefetch = [&](int item, int bi) {
    const StreamItem m = src.at(item);
    T* b = buf0 + bi * kBuf;
    const long long N = m.C->N;
    const long long e0 = (long long)m.e * np;
    const int sh = (int)(e0 & 3);
    if (m.bulk) {
      const int hd = (4 - sh) & 3, tl = (sh + np) & 3, L = np - hd - tl;
      if (threadIdx.x == 0) {
        bulk_expect_tx(&bar[bi], 14u * 4u * (unsigned)L);
        for (int c = 0; c < 14; ++c) {
          const float* g = (c < 5 ? m.qf + c * N : m.vis + (c - 5) * N) + e0;
          bulk_copy(b + c * kTS + sh + hd, g + hd, 4u * (unsigned)L, &bar[bi]);
        }
      }
      for (int i = threadIdx.x; i < 14 * 8; i += blockDim.x) {
        const int c = i >> 3, j = i & 7;
        if (j < 4 ? j >= hd : j - 4 >= tl) continue;
        const int nd = j < 4 ? j : np - tl + (j - 4);
        const float* g = (c < 5 ? m.qf + c * N : m.vis + (c - 5) * N) + e0;
        cp_async4(b + c * kTS + sh + nd, g + nd);
      }
    } else {
      for (int nd = threadIdx.x; nd < np; nd += blockDim.x) {
#pragma unroll
        for (int v = 0; v < 5; ++v) cp_async4(b + v * kTS + sh + nd, m.qf + v * N + e0 + nd);
#pragma unroll
        for (int c = 0; c < 9; ++c) cp_async4(b + (5 + c) * kTS + sh + nd, m.vis + c * N + e0 + nd);
      }
    }
    const BlockCoords bc = block_coords(m.e, m.C->K);
    T* h = b + 14 * kTS;
    for (int t = threadIdx.x; t < haloN; t += blockDim.x) {
      const Item<P> it = item_of<P>(t);
      const int enb = neighbour_of(bc, 0, m.C->K, Src::kSlab ? m.C->Kz : m.C->K, it.d, it.side ? 1 : -1);
      const long long gnb = (long long)enb * np + face_node<P>(it.d, it.side ? 0 : P, it.ab);
      switch (it.d) {
        case 0: copy_face_data<0>(m.qf, m.vis, N, gnb, h + t, haloN); break;
        case 1: copy_face_data<1>(m.qf, m.vis, N, gnb, h + t, haloN); break;
        default: copy_face_data<2>(m.qf, m.vis, N, gnb, h + t, haloN);
      }
    }
    cp_async_commit();
  };

  pdl_wait();
  int item = blockIdx.x;
  if (item >= n_items) return;
  if (threadIdx.x == 0) {
    bulk_bar_init(&bar[0]);
    bulk_bar_init(&bar[1]);
    bulk_bar_fence_init();
  }
  __syncthreads();
  prefetch(item, 0);
  const int node = threadIdx.x;
  const bool active = node < np;
  const int idx[3] = {node % n, (node / n) % n, node / n2};

  unsigned phases = 0u;   // bit i: parity of buffer i's next bulk phase (members may mix modes)
  for (int k = 0; item < n_items; item += gridDim.x, ++k) {
    const StreamItem m = src.at(item);
    T* b = buf0 + (k & 1) * kBuf;
    cp_async_wait_all();
    bool landed = true;
    if (m.bulk) {
      landed = bulk_wait(&bar[k & 1], (phases >> (k & 1)) & 1u);
      phases ^= 1u << (k & 1);
    }
    if (__syncthreads_or(!landed)) {       // this item's data landed; the other buffer is free
      if (threadIdx.x == 0 && m.err) atomicExch(m.err, 1);
      break;                               // a bounded wait expired: give up (host reports it)
    }
    const int next = item + gridDim.x;
    if (next < n_items) prefetch(next, (k + 1) & 1);
    else pdl_release();   // this block's last element: the successor may launch

    const OpConst<T>& C = *m.C;
    const RkArgs<T>& rk = *m.rk;
    const long long N = C.N;
    const long long gi = (long long)m.e * np + node;
    T* sX = b + (int)(((long long)m.e * np) & 3);   // own tile: component c of node nd at sX[c kTS + nd]
    T* sH = b + 14 * kTS;

    // RK operands of this thread's node, loaded now and used at the end
    T gold[5], dold[5];
    double qold[5];
    if (active) {
      if (MODE == 3 || MODE == 4) {
#pragma unroll
        for (int v = 0; v < 5; ++v) dold[v] = m.dlt[v * N + gi];
      }
      if (MODE == 4) {
#pragma unroll
        for (int v = 0; v < 5; ++v) gold[v] = m.greg[v * N + gi];
#pragma unroll
        for (int v = 0; v < 5; ++v) qold[v] = m.q[v * N + gi];
      }
    }

    // volume fluxes of this thread's node into sV (the own tile stays intact for the
    // interface items, so no barrier separates the two)
    if (active) {
      T s[5], vs[9];
#pragma unroll
      for (int v = 0; v < 5; ++v) s[v] = sX[v * kTS + node];
#pragma unroll
      for (int c = 0; c < 9; ++c) vs[c] = sX[(5 + c) * kTS + node];
      const Prim<T> w = prim_c(s, C);
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        T F[5], fv[5];
        euler_flux(s, w, C.Hc, d, F);
        viscous_flux(vs, w.v, d, fv);
#pragma unroll
        for (int c = 0; c < 5; ++c) sV[(5 * d + c) * np + node] = F[c] - fv[c];
      }
    }

    // interface terms, one work item per (face, face node); each item reads its halo slot
    // and then writes its lifted terms over components 0-4 of that slot
    for (int t = threadIdx.x; t < haloN; t += blockDim.x) {
      const Item<P> it = item_of<P>(t);
      const int o = face_node<P>(it.d, it.side ? P : 0, it.ab);
      T so[5], to[4], sn[5], tn[4];
#pragma unroll
      for (int v = 0; v < 5; ++v) so[v] = sX[v * kTS + o];
#pragma unroll
      for (int v = 0; v < 5; ++v) sn[v] = sH[v * haloN + t];
#pragma unroll
      for (int i = 0; i < 4; ++i) tn[i] = sH[(5 + i) * haloN + t];
      switch (it.d) {
        case 0:
#pragma unroll
          for (int i = 0; i < 4; ++i) to[i] = sX[(5 + face_vis_index(0, i)) * kTS + o];
          interface_item<0>(so, to, sn, tn, sH + t, haloN, it.side, C);
          break;
        case 1:
#pragma unroll
          for (int i = 0; i < 4; ++i) to[i] = sX[(5 + face_vis_index(1, i)) * kTS + o];
          interface_item<1>(so, to, sn, tn, sH + t, haloN, it.side, C);
          break;
        default:
#pragma unroll
          for (int i = 0; i < 4; ++i) to[i] = sX[(5 + face_vis_index(2, i)) * kTS + o];
          interface_item<2>(so, to, sn, tn, sH + t, haloN, it.side, C);
      }
    }
    __syncthreads();

    // volume term: one task per (direction, component, line) replaces the line's fluxes
    // by their derivative; tasks are direction-major so that a warp shares d
    for (int task = threadIdx.x; task < 15 * n2; task += blockDim.x) {
      const int dc = task / n2, ab = task - dc * n2;
      float* f = sV + dc * np;
      if (dc < 5) line_derivative_inplace<P, 0>(f, ab);
      else if (dc < 10) line_derivative_inplace<P, 1>(f, ab);
      else line_derivative_inplace<P, 2>(f, ab);
    }
    __syncthreads();
    if (!active) continue;

    T R[5] = {T(0), T(0), T(0), T(0), T(0)};
#pragma unroll
    for (int d = 0; d < 3; ++d) {
#pragma unroll
      for (int c = 0; c < 5; ++c) R[c] -= C.s2h * sV[(5 * d + c) * np + node];
    }
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const bool right = (idx[d] == P), left = (idx[d] == 0);
      if (!(right || left)) continue;
      const int h = item_index<P>(face_ab<P>(d, idx), right ? 1 : 0, d, 0);
#pragma unroll
      for (int c = 0; c < 5; ++c) R[c] += sH[c * haloN + h];   // lifted terms over the halo slots
    }
    if (m.fc.s != nullptr) {
      const long long fb = (long long)m.e * m.fc.stride + node;
#pragma unroll
      for (int c = 0; c < 5; ++c) {
        const int slot = c - m.fc.first_var;
        if (slot >= 0 && slot < m.fc.n_vars) R[c] += T(m.fc.s[fb + (long long)slot * np]);
      }
    }
#pragma unroll
    for (int c = 0; c < 5; ++c) {
      const long long o = c * N + gi;
      if (MODE == 0) {
        m.dqdt[o] = double(R[c]);
      } else if (MODE == 2) {
        m.dlt[o] = float(rk.B * (rk.dt * R[c]));
      } else if (MODE == 3) {
        const T g2 = rk.A * (dold[c] * rk.invB1) + rk.dt * R[c];
        m.greg[o] = g2;
        m.dlt[o] = float(dold[c] + rk.B * g2);
      } else if (MODE == 4) {
        const T g3 = rk.A * gold[c] + rk.dt * R[c];
        const float d3 = float(dold[c] + rk.B * g3);
        m.q[o] = qold[c] + f2d(d3);
      }
    }
  }
  cp_async_wait_all();
}

// Operands of one mesh for the streamed kernel (kernel parameter).
struct StreamMesh {
  double* q;
  const float* qf;
  const float* vis;
  double* dqdt;
  float* greg;
  float* dlt;
  Forcing fc;
  OpConst<float> C;
  RkArgs<float> rk;
  int bulk;  // qf and vis 16-byte aligned and N a multiple of 4: own tiles by TMA bulk copies
  int* err;  // device error flag (may be NULL)
};

template <bool SLAB>
struct SingleSource {
  static constexpr bool kSlab = SLAB;
  const StreamMesh& m;
  __device__ __forceinline__ StreamItem at(int item) const {
    return StreamItem{m.q, m.qf, m.vis, m.dqdt, m.greg, m.dlt, &m.C, &m.rk, m.fc, (SLAB ? m.C.e_begin : 0) + item,
                      m.bulk, m.err};
  }
};

struct BatchSource {
  static constexpr bool kSlab = false;
  const BatchTable<float>& tb;
  __device__ __forceinline__ StreamItem at(int item) const {
    const int i = batch_instance(tb.block_start, tb.n, item);
    return StreamItem{tb.q[i], tb.qf[i], tb.vis[i], nullptr, tb.g[i], tb.dlt[i], &tb.C[i], &tb.rk[i], Forcing{},
                      item - tb.block_start[i], tb.bulk[i], tb.err[i]};
  }
};

template <int P, int MODE, bool SLAB = false>
__global__ void __launch_bounds__(stream_threads(P), stream_min_blocks(P))
k_flux_stream(const __grid_constant__ StreamMesh mesh) {
  flux_stream<P, MODE>(SingleSource<SLAB>{mesh}, mesh.C.nel - (SLAB ? mesh.C.e_begin : 0));
}

// Batched streamed phase B: members of order P, one element per work item
// (block_start counts elements).
template <int P, int MODE>
__global__ void __launch_bounds__(stream_threads(P), stream_min_blocks(P))
k_flux_stream_batch(const __grid_constant__ BatchTable<float> tb) {
  flux_stream<P, MODE>(BatchSource{tb}, tb.block_start[tb.n]);
}

}  // namespace dgnn
