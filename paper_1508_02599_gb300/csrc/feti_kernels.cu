// CUDA kernels (sm_103a) of the FETI solver: P1 element matrices, local
// assembly, dense local factorizations and operators, multiplier gathers,
// coarse projection and projected-CG vector updates.
//
// Design for GB300: FP64 arithmetic issues at about two FMAs per clock per SM,
// so every FP64 kernel here is bounded by the FP64 pipe or by HBM; gathers are
// row-major and deterministic (no floating-point atomics anywhere); every
// subdomain of uneven size is one batch element of a single launch.
#include "feti_internal.h"

#include <cmath>

namespace feti {

namespace {

constexpr int kThreads = 256;
constexpr int kPartials = 304;  // 2 x 152 SMs: fixed grid of the row kernels

__device__ __forceinline__ void set_status(int* status, int code) {
  atomicCAS(status, 0, code);
}

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Fixed-order CTA reduction (deterministic for a fixed launch shape).
__device__ double block_sum(double v, double* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double t = 0.0;
  if (wid == 0) {
    t = (lane < (int)(blockDim.x >> 5)) ? red[lane] : 0.0;
    t = warp_sum(t);
  }
  __syncthreads();
  if (threadIdx.x == 0) red[0] = t;
  __syncthreads();
  double r = red[0];
  __syncthreads();
  return r;
}

// ---------------------------------------------------------------------------
// P1 shape-function gradients: g[a][j] = dN_a/dX_j, volume V.
__device__ __forceinline__ bool p1_gradients(const double x[4][3], double g[4][3], double& V) {
  double Jm[3][3];  // columns x_k - x_0
  for (int i = 0; i < 3; ++i)
    for (int k = 0; k < 3; ++k) Jm[i][k] = x[k + 1][i] - x[0][i];
  const double c00 = Jm[1][1] * Jm[2][2] - Jm[1][2] * Jm[2][1];
  const double c01 = Jm[1][2] * Jm[2][0] - Jm[1][0] * Jm[2][2];
  const double c02 = Jm[1][0] * Jm[2][1] - Jm[1][1] * Jm[2][0];
  const double det = Jm[0][0] * c00 + Jm[0][1] * c01 + Jm[0][2] * c02;
  V = det / 6.0;
  if (!(det > 0.0)) return false;
  const double id = 1.0 / det;
  double Ji[3][3];  // inverse of Jm
  Ji[0][0] = c00 * id;
  Ji[1][0] = c01 * id;
  Ji[2][0] = c02 * id;
  Ji[0][1] = (Jm[0][2] * Jm[2][1] - Jm[0][1] * Jm[2][2]) * id;
  Ji[1][1] = (Jm[0][0] * Jm[2][2] - Jm[0][2] * Jm[2][0]) * id;
  Ji[2][1] = (Jm[0][1] * Jm[2][0] - Jm[0][0] * Jm[2][1]) * id;
  Ji[0][2] = (Jm[0][1] * Jm[1][2] - Jm[0][2] * Jm[1][1]) * id;
  Ji[1][2] = (Jm[0][2] * Jm[1][0] - Jm[0][0] * Jm[1][2]) * id;
  Ji[2][2] = (Jm[0][0] * Jm[1][1] - Jm[0][1] * Jm[1][0]) * id;
  // N_1..3 = xi_1..3 (rows of Ji), N_0 = 1 - sum
  for (int j = 0; j < 3; ++j) {
    g[1][j] = Ji[0][j];
    g[2][j] = Ji[1][j];
    g[3][j] = Ji[2][j];
    g[0][j] = -(Ji[0][j] + Ji[1][j] + Ji[2][j]);
  }
  return true;
}

__global__ void k_elem_linear(int n_tets, const double* __restrict__ coords, const int32_t* __restrict__ tets,
                              double E, double nu, double* __restrict__ Ke, int* status) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n_tets) return;
  double x[4][3], g[4][3], V;
  for (int a = 0; a < 4; ++a) {
    const int n = tets[4 * e + a];
    for (int i = 0; i < 3; ++i) x[a][i] = coords[3 * n + i];
  }
  if (!p1_gradients(x, g, V)) {
    set_status(status, DEV_INVERTED);
    return;
  }
  const double lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
  const double mu = E / (2.0 * (1.0 + nu));
  double* K = Ke + (size_t)e * ke_packed(12);
  for (int a = 0; a < 4; ++a)
    for (int b = a; b < 4; ++b) {
      const double gab = g[a][0] * g[b][0] + g[a][1] * g[b][1] + g[a][2] * g[b][2];
      for (int i = 0; i < 3; ++i)
        for (int j = (a == b ? i : 0); j < 3; ++j) {
          double v = lam * g[a][i] * g[b][j] + mu * g[a][j] * g[b][i];
          if (i == j) v += mu * gab;
          K[ke_idx(12, 3 * a + i, 3 * b + j)] = V * v;
        }
    }
}

// P2 element (10-node tetrahedron, straight edges; nodes: the vertices, then
// the midpoints of the edges (0,1) (0,2) (0,3) (1,2) (1,3) (2,3)) for Hooke's
// law, one warp per element: every lane evaluates the gradients of the
// barycentric coordinates, then takes node-pair blocks (a, b) = lane, lane +
// 32, .. of the 10 x 10 block grid and writes their 3 x 3 entries.  The
// gradients of N_a = L_a (2 L_a - 1) and N_ab = 4 L_a L_b are linear, so the
// degree-2 Gauss rule (four points (alpha, beta, beta, beta) and permutations,
// weights 1/4) integrates the stiffness exactly.  p0: the lambda term is
// carried by a piecewise-constant pressure condensed out of the element
// (Sec. 3.2, static condensation): lambda V bbar_a,i bbar_b,j with bbar_a the
// element mean of grad N_a, instead of the integral of lambda g_a,i g_b,j.
__device__ __forceinline__ void p2_grad(const double gL[4][3], const double Lq[4], int a, double g[3]) {
  if (a < 4) {
    const double f = 4.0 * Lq[a] - 1.0;
    g[0] = f * gL[a][0];
    g[1] = f * gL[a][1];
    g[2] = f * gL[a][2];
    return;
  }
  const int ea[6] = {0, 0, 0, 1, 1, 2}, eb[6] = {1, 2, 3, 2, 3, 3};
  const int u = ea[a - 4], v = eb[a - 4];
  for (int i = 0; i < 3; ++i) g[i] = 4.0 * (Lq[u] * gL[v][i] + Lq[v] * gL[u][i]);
}

__global__ void k_elem_linear_p2(int n_tets, const double* __restrict__ coords, const int32_t* __restrict__ tets,
                                 double E, double nu, int p0, double* __restrict__ Ke, int* status) {
  const int e = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (e >= n_tets) return;
  double x[4][3], gL[4][3], V;
  for (int a = 0; a < 4; ++a) {
    const int n = tets[10 * (size_t)e + a];
    for (int i = 0; i < 3; ++i) x[a][i] = coords[3 * (size_t)n + i];
  }
  if (!p1_gradients(x, gL, V)) {
    if (lane == 0) set_status(status, DEV_INVERTED);
    return;
  }
  const double lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
  const double mu = E / (2.0 * (1.0 + nu));
  const double al = (5.0 + 3.0 * sqrt(5.0)) / 20.0, be = (5.0 - sqrt(5.0)) / 20.0;
  double* K = Ke + (size_t)e * ke_packed(30);
  for (int blk = lane; blk < 100; blk += 32) {
    const int a = blk / 10, b = blk % 10;
    if (b < a) continue;  // upper triangle of node blocks
    double k9[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    double ma[3] = {0, 0, 0}, mb[3] = {0, 0, 0};
    for (int q = 0; q < 4; ++q) {
      double Lq[4];
      for (int c = 0; c < 4; ++c) Lq[c] = c == q ? al : be;
      double ga[3], gb[3];
      p2_grad(gL, Lq, a, ga);
      p2_grad(gL, Lq, b, gb);
      const double gab = ga[0] * gb[0] + ga[1] * gb[1] + ga[2] * gb[2];
      for (int i = 0; i < 3; ++i) {
        ma[i] += 0.25 * ga[i];
        mb[i] += 0.25 * gb[i];
        for (int j = 0; j < 3; ++j) {
          double v = mu * ga[j] * gb[i] + (p0 ? 0.0 : lam * ga[i] * gb[j]);
          if (i == j) v += mu * gab;
          k9[i][j] += 0.25 * v;
        }
      }
    }
    for (int i = 0; i < 3; ++i)
      for (int j = (a == b ? i : 0); j < 3; ++j)
        K[ke_idx(30, 3 * a + i, 3 * b + j)] = V * (k9[i][j] + (p0 ? lam * ma[i] * mb[j] : 0.0));
  }
}

// Two-fibre hyperelastic element (Sec. 3.1 energy, Sec. 3.2 tangent), one
// thread per element, evaluated in the current configuration.
//
// Material form.  With J23 = J^(-2/3), A_v = kappa (J-1) J and, per fibre
// family f, psi'_f, psi''_f the derivatives of its energy in I4bar = J23 I4:
//   S = A_v C^-1 + c J23 (I - I1/3 C^-1) + sum_f 2 psi'_f J23 (a a - I4/3 C^-1)
//   CC = 2 dS/dC = c_11 C^-1(x)C^-1 + c_Q Q + c_IC (I(x)C^-1 + C^-1(x)I)
//        + sum_f [4 psi''_f J23^2 B(x)B - (2/3) psi'_f J23 (C^-1(x)B + B(x)C^-1 + C^-1(x)aa + aa(x)C^-1)]
//   with Q_IJKL = (Ci_IK Ci_JL + Ci_IL Ci_JK)/2, B = a a - I4/3 C^-1 and
//   c_11 = kappa (2J-1) J + (2c/9) J23 I1, c_IC = -(2c/3) J23,
//   c_Q = -2 A_v + (2c/3) J23 I1 + sum_f (4/3) psi'_f J23 I4_f
//   (dC^-1/dC = -Q, dJ/dC = J/2 C^-1, dJ23/dC = -J23/3 C^-1, dI1/dC = I, dI4/dC = a a).
//
// Spatial evaluation.  The tangent block K[(a,i),(b,j)] = V (delta_ij g_a.S g_b
// + sum F_iI g_aJ CC_IJKL F_jK g_bL) is the same number when every tensor is
// pushed forward by F: with the current gradients h_a = F^-T g_a, C^-1 -> 1,
// I -> b = F F^T, a a -> A A (A = F a), Q -> the symmetric identity, S -> the
// Kirchhoff stress tau = F S F^T, and the tangent becomes
//   K[(a,i),(b,j)] = V [ c_11 h_ai h_bj + (c_Q/2)(delta_ij h_a.h_b + h_aj h_bi)
//       + c_IC ((b h_a)_i h_bj + h_ai (b h_b)_j)
//       + sum_f ( 4 psi''_f J23^2 (beta_f h_a)_i (beta_f h_b)_j
//                 - (2/3) psi'_f J23 (h_ai w_fbj + w_fai h_bj) )
//       + delta_ij h_a.tau h_b ],
//   beta_f = A A - I4/3 1,  w_fa = beta_f h_a + (A.h_a) A,
// and the internal force f_a = V tau h_a.  Every term is a product of
// per-node 3-vectors, about a fifth of the FP64 operations of contracting the
// material tensor entry by entry; all arrays stay in registers.
__global__ void __launch_bounds__(64) k_elem_hgo(int n_tets, const double* __restrict__ coords,
                                                 const int32_t* __restrict__ tets, const double* __restrict__ U,
                                                 const double* __restrict__ fibres, double cmat, double k1,
                                                 double k2, double kappa, double* __restrict__ Ke,
                                                 double* __restrict__ fe, int* status) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n_tets) return;
  double x[4][3], g[4][3], V, u[4][3];
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int n = tets[4 * e + a];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      x[a][i] = coords[3 * n + i];
      u[a][i] = U ? U[3 * n + i] : 0.0;
    }
  }
  if (!p1_gradients(x, g, V)) {
    set_status(status, DEV_INVERTED);
    return;
  }
  double F[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      double s = (i == j) ? 1.0 : 0.0;
#pragma unroll
      for (int a = 0; a < 4; ++a) s += u[a][i] * g[a][j];
      F[i][j] = s;
    }
  // cofactor matrix: cof(F) = J F^-T
  double cf[3][3];
  cf[0][0] = F[1][1] * F[2][2] - F[1][2] * F[2][1];
  cf[0][1] = F[1][2] * F[2][0] - F[1][0] * F[2][2];
  cf[0][2] = F[1][0] * F[2][1] - F[1][1] * F[2][0];
  cf[1][0] = F[0][2] * F[2][1] - F[0][1] * F[2][2];
  cf[1][1] = F[0][0] * F[2][2] - F[0][2] * F[2][0];
  cf[1][2] = F[0][1] * F[2][0] - F[0][0] * F[2][1];
  cf[2][0] = F[0][1] * F[1][2] - F[0][2] * F[1][1];
  cf[2][1] = F[0][2] * F[1][0] - F[0][0] * F[1][2];
  cf[2][2] = F[0][0] * F[1][1] - F[0][1] * F[1][0];
  const double J = F[0][0] * cf[0][0] + F[0][1] * cf[0][1] + F[0][2] * cf[0][2];
  if (!(J > 0.0)) {
    set_status(status, DEV_INVERTED);
    return;
  }
  const double iJ = 1.0 / J;
  double h[4][3];  // h_a = F^-T g_a
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int m = 0; m < 3; ++m) h[a][m] = (cf[m][0] * g[a][0] + cf[m][1] * g[a][1] + cf[m][2] * g[a][2]) * iJ;
  double bm[3][3];  // b = F F^T
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = i; j < 3; ++j) {
      bm[i][j] = F[i][0] * F[j][0] + F[i][1] * F[j][1] + F[i][2] * F[j][2];
      bm[j][i] = bm[i][j];
    }
  const double I1 = bm[0][0] + bm[1][1] + bm[2][2];
  const double J23 = rcbrt(J * J);
  const double Av = kappa * (J - 1.0) * J;
  // Kirchhoff stress: tau = t0 1 + c J23 b + sum_f 2 psi'_f J23 A_f A_f
  double t0 = Av - cmat * J23 * I1 / 3.0;
  double tau[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) tau[i][j] = cmat * J23 * bm[i][j];
  double Af[2][3], I4[2], dpsi[2], d2psi[2];
  double cQ = -2.0 * Av + 2.0 * cmat * J23 * I1 / 3.0;
#pragma unroll
  for (int f = 0; f < 2; ++f) {
    double a0[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) a0[i] = fibres[6 * e + 3 * f + i];
#pragma unroll
    for (int i = 0; i < 3; ++i) Af[f][i] = F[i][0] * a0[0] + F[i][1] * a0[1] + F[i][2] * a0[2];
    I4[f] = Af[f][0] * Af[f][0] + Af[f][1] * Af[f][1] + Af[f][2] * Af[f][2];
    const double dlt = J23 * I4[f] - 1.0;
    if (dlt > 1e-12) {
      const double ex = exp(k2 * dlt * dlt);
      dpsi[f] = k1 * dlt * ex;                            // dPsi/dI4bar
      d2psi[f] = k1 * ex * (1.0 + 2.0 * k2 * dlt * dlt);  // d2Psi/dI4bar2
    } else {
      dpsi[f] = d2psi[f] = 0.0;
    }
    const double m2 = 2.0 * dpsi[f] * J23;
    t0 -= m2 * I4[f] / 3.0;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) tau[i][j] += m2 * Af[f][i] * Af[f][j];
    cQ += 2.0 * m2 * I4[f] / 3.0;
  }
#pragma unroll
  for (int i = 0; i < 3; ++i) tau[i][i] += t0;
  const double c11 = kappa * (2.0 * J - 1.0) * J + 2.0 * cmat * J23 * I1 / 9.0;
  const double cIC = -2.0 * cmat * J23 / 3.0;
  // per-node vectors, scaled by V: P_a = V (c_IC b h_a - (2/3) sum_f psi'_f J23 w_fa),
  // Pv_a = P_a + V c_11 h_a, r_fa = sqrt(4 V psi''_f) J23 beta_f h_a; tau h_a
  double P[4][3], Pv[4][3], r[2][4][3], th[4][3];
#pragma unroll
  for (int a = 0; a < 4; ++a) {
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      th[a][i] = tau[i][0] * h[a][0] + tau[i][1] * h[a][1] + tau[i][2] * h[a][2];
      P[a][i] = cIC * (bm[i][0] * h[a][0] + bm[i][1] * h[a][1] + bm[i][2] * h[a][2]);
    }
#pragma unroll
    for (int f = 0; f < 2; ++f) {
      const double sa = Af[f][0] * h[a][0] + Af[f][1] * h[a][1] + Af[f][2] * h[a][2];
      const double cw = -(2.0 / 3.0) * dpsi[f] * J23;
      const double cr = 2.0 * J23 * sqrt(V * d2psi[f]);
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        const double bh = sa * Af[f][i] - I4[f] / 3.0 * h[a][i];  // beta_f h_a
        P[a][i] += cw * (bh + sa * Af[f][i]);
        r[f][a][i] = cr * bh;
      }
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      P[a][i] *= V;
      Pv[a][i] = P[a][i] + V * c11 * h[a][i];
    }
  }
  // diagonal-in-(i,j) part: D_ab = V ((c_Q/2) h_a.h_b + h_a.tau h_b)
  const double hq = 0.5 * cQ * V;
  double* Kout = Ke + (size_t)e * ke_packed(12);
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = a; b < 4; ++b) {
      const double D = hq * (h[a][0] * h[b][0] + h[a][1] * h[b][1] + h[a][2] * h[b][2]) +
                       V * (h[a][0] * th[b][0] + h[a][1] * th[b][1] + h[a][2] * th[b][2]);
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          if (a == b && j < i) continue;
          double v = Pv[a][i] * h[b][j] + h[a][i] * P[b][j] + hq * h[a][j] * h[b][i] + r[0][a][i] * r[0][b][j] +
                     r[1][a][i] * r[1][b][j];
          if (i == j) v += D;
          Kout[ke_idx(12, 3 * a + i, 3 * b + j)] = v;
        }
    }
  if (fe) {
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int i = 0; i < 3; ++i) fe[(size_t)e * 12 + 3 * a + i] = V * th[a][i];
  }
}

// ---------------------------------------------------------------------------
// T = double (FP64 factorization) or float (FP32 factorization: each entry
// is summed in FP32 in element order).
template <typename T>
__global__ void k_assemble(const SubLayout* __restrict__ lay, const int32_t* __restrict__ sub_elem_ptr,
                           const int32_t* __restrict__ sub_elems, const int32_t* __restrict__ elem_dense,
                           const double* __restrict__ Ke, int nde, T* __restrict__ Abase) {
  const int s = blockIdx.x;
  const SubLayout L = lay[s];
  T* A = Abase + L.aoff;
  const int kes = ke_packed(nde);
  for (int q = sub_elem_ptr[s]; q < sub_elem_ptr[s + 1]; ++q) {
    const int e = sub_elems[q];
    for (int t = threadIdx.x; t < kes; t += blockDim.x) {
      // packed entry t -> (i, j), i <= j; both (i, j) and (j, i) of the local matrix
      int i = 0, rem = t;
      while (rem >= nde - i) {
        rem -= nde - i;
        ++i;
      }
      const int j = i + rem;
      const int r = elem_dense[(size_t)nde * e + i], c = elem_dense[(size_t)nde * e + j];
      if (r >= 0 && c >= 0) {
        const T v = (T)Ke[(size_t)e * kes + t];
        A[(size_t)r * L.ld + c] += v;
        if (i != j) A[(size_t)c * L.ld + r] += v;
      }
    }
    __syncthreads();
  }
}

// Consistent nodal loads of one loaded face under constant pressure (kind 0,
// along the area vector) or traction (kind 1).  3-node faces: a third of the
// force to each vertex; 6-node (P2, flat) faces: the vertex shape functions
// integrate to zero and the midpoint ones to A/3, so a third of the force to
// each edge midpoint (nodes 3..5) and none to the vertices.
__global__ void k_face_forces(int n_faces, int fpn, const int32_t* __restrict__ tri, const double* __restrict__ coords,
                              const double* __restrict__ U, int kind, double scale,
                              const double* __restrict__ traction, double* __restrict__ out) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= n_faces) return;
  double x[3][3];
  for (int v = 0; v < 3; ++v) {
    const int n = tri[(size_t)fpn * f + v];
    for (int i = 0; i < 3; ++i) x[v][i] = coords[3 * n + i] + (U ? U[3 * n + i] : 0.0);
  }
  double e1[3], e2[3], av[3];
  for (int i = 0; i < 3; ++i) {
    e1[i] = x[1][i] - x[0][i];
    e2[i] = x[2][i] - x[0][i];
  }
  av[0] = 0.5 * (e1[1] * e2[2] - e1[2] * e2[1]);
  av[1] = 0.5 * (e1[2] * e2[0] - e1[0] * e2[2]);
  av[2] = 0.5 * (e1[0] * e2[1] - e1[1] * e2[0]);
  double force[3];
  if (kind == 0) {
    for (int i = 0; i < 3; ++i) force[i] = scale * av[i] / 3.0;
  } else {
    const double area = sqrt(av[0] * av[0] + av[1] * av[1] + av[2] * av[2]);
    for (int i = 0; i < 3; ++i) force[i] = scale * area * traction[i] / 3.0;
  }
  for (int v = 0; v < fpn; ++v)
    for (int i = 0; i < 3; ++i)
      out[3 * (size_t)fpn * f + 3 * v + i] = (fpn == 3 || v >= 3) ? force[i] : 0.0;
}

__global__ void k_assemble_rhs(const SubLayout* __restrict__ lay, const int32_t* __restrict__ sub_face_ptr,
                               const int32_t* __restrict__ face_dense, const double* __restrict__ face_force, int fdn,
                               const int32_t* __restrict__ sub_elem_ptr, const int32_t* __restrict__ sub_elems,
                               const int32_t* __restrict__ elem_dense, const double* __restrict__ elem_dirval,
                               const double* __restrict__ Ke, const double* __restrict__ fe, int nde, double tau,
                               double* __restrict__ fbase) {
  const int s = blockIdx.x;
  const SubLayout L = lay[s];
  double* f = fbase + L.voff;
  const int t = threadIdx.x;
  for (int i = t; i < L.n; i += blockDim.x) f[i] = 0.0;
  __syncthreads();
  for (int q = sub_face_ptr[s]; q < sub_face_ptr[s + 1]; ++q) {
    if (t < fdn) {
      const int r = face_dense[(size_t)fdn * q + t];
      if (r >= 0) f[r] += tau * face_force[(size_t)fdn * q + t];
    }
    __syncthreads();
  }
  const int kes = ke_packed(nde);
  for (int q = sub_elem_ptr[s]; q < sub_elem_ptr[s + 1]; ++q) {
    const int e = sub_elems[q];
    if (t < nde) {
      const int r = elem_dense[(size_t)nde * e + t];
      if (r >= 0) {
        double v = fe ? -fe[(size_t)e * nde + t] : 0.0;
        if (elem_dirval) {
          for (int b = 0; b < nde; ++b) {
            const double ud = elem_dirval[(size_t)nde * e + b];
            if (ud != 0.0) v -= Ke[(size_t)e * kes + ke_idx(nde, t, b)] * ud;
          }
        }
        f[r] += v;
      }
    }
    __syncthreads();
  }
}

template <typename T>
__global__ void k_augment(const SubLayout* __restrict__ lay, T* __restrict__ Abase) {
  const int s = blockIdx.x;
  const SubLayout L = lay[s];
  T* A = Abase + L.aoff;
  for (int j = threadIdx.x; j < L.nbp; j += blockDim.x) A[(size_t)(L.n + j) * L.ld + L.nI + j] = (T)1;
}

// Block sizes of the dense Cholesky kernels: 32-column panels, 64x64 update tiles.
constexpr int NB = 32;
constexpr int TT = 64;

__global__ void k_extract(const SubLayout* __restrict__ lay, int which, const double* __restrict__ Abase,
                          double* __restrict__ out) {
  const int s = blockIdx.x;
  const SubLayout L = lay[s];
  const double* A = Abase + L.aoff;
  const size_t ld = L.ld;
  if (which == 0) {
    const int nb = L.nbp + L.k;
    double* S = out + L.soff;
    for (int idx = threadIdx.x; idx < nb * nb; idx += blockDim.x) {
      const int i = idx / nb, j = idx % nb;
      const int ii = max(i, j), jj = min(i, j);
      S[idx] = A[(L.nI + ii) * ld + L.nI + jj];
    }
  } else {
    const int m = L.nbp;
    double* F = out + L.foff;
    for (int idx = threadIdx.x; idx < m * m; idx += blockDim.x) {
      const int i = idx / m, j = idx % m;
      const int ii = max(i, j), jj = min(i, j);
      F[idx] = -A[(L.n + ii) * ld + L.n + jj];
    }
  }
}

// x = K^+ g: forward L y = g_r, backward L^T x = y, both by 32-row blocks
// with two barriers per block.  Forward: the warps form the dot products of
// the block's rows with the part solved so far (one warp per row, lanes
// striding the columns), then one warp solves the 32 x 32 diagonal triangle
// with shuffles.  Backward: one warp solves the transposed diagonal triangle,
// then every thread subtracts the block's contributions from its columns of
// the unsolved part.  The fixing DOFs get zero.
__global__ void __launch_bounds__(kThreads) k_kplus(const SubLayout* __restrict__ lay,
                                                    const double* __restrict__ Abase,
                                                    const double* __restrict__ gbase, double* __restrict__ xbase,
                                                    const int* __restrict__ done) {
  if (done && *done) return;
  const int s = blockIdx.x;
  const SubLayout L = lay[s];
  const double* A = Abase + L.aoff;
  const size_t ld = L.ld;
  const double* g = gbase + L.voff;
  double* x = xbase + L.voff;
  const int nr = L.nI + L.nbp;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int kWarpsPerCta = kThreads / 32;
  __shared__ double D[32][33];
  __shared__ double t[32];
  __shared__ double xs[32];
  for (int i = nr + tid; i < L.n; i += blockDim.x) x[i] = 0.0;
  for (int I0 = 0; I0 < nr; I0 += 32) {
    const int nb = min(32, nr - I0);
    for (int idx = tid; idx < 32 * 32; idx += blockDim.x) {
      const int r = idx >> 5, c = idx & 31;
      D[r][c] = (r < nb && c <= r) ? A[(size_t)(I0 + r) * ld + I0 + c] : 0.0;
    }
    for (int r = warp; r < nb; r += kWarpsPerCta) {
      const double* row = A + (size_t)(I0 + r) * ld;
      double acc = 0.0;
#pragma unroll 4
      for (int j = lane; j < I0; j += 32) acc += row[j] * x[j];
      acc = warp_sum(acc);
      if (lane == 0) t[r] = acc;
    }
    __syncthreads();
    if (warp == 0) {
      double b = lane < nb ? g[I0 + lane] - t[lane] : 0.0;
      double xv = 0.0;
      for (int c = 0; c < nb; ++c) {
        if (lane == c) xv = b / D[c][c];
        const double xc = __shfl_sync(0xffffffffu, xv, c);
        if (lane > c) b -= D[lane][c] * xc;
      }
      if (lane < nb) x[I0 + lane] = xv;
    }
    __syncthreads();
  }
  for (int I0 = nr > 0 ? ((nr - 1) / 32) * 32 : -32; I0 >= 0; I0 -= 32) {
    const int nb = min(32, nr - I0);
    for (int idx = tid; idx < 32 * 32; idx += blockDim.x) {
      const int r = idx >> 5, c = idx & 31;
      D[r][c] = (r < nb && c <= r) ? A[(size_t)(I0 + r) * ld + I0 + c] : 0.0;
    }
    __syncthreads();
    if (warp == 0) {
      double b = lane < nb ? x[I0 + lane] : 0.0;
      double xv = 0.0;
      for (int c = nb - 1; c >= 0; --c) {
        if (lane == c) xv = b / D[c][c];
        const double xc = __shfl_sync(0xffffffffu, xv, c);
        if (lane < c) b -= D[c][lane] * xc;
      }
      if (lane < nb) x[I0 + lane] = xv;
      xs[lane] = xv;
    }
    __syncthreads();
    for (int j = tid; j < I0; j += blockDim.x) {
      double acc = 0.0;
      for (int r = 0; r < nb; ++r) acc += A[(size_t)(I0 + r) * ld + j] * xs[r];
      x[j] -= acc;
    }
  }
}

// ---------------------------------------------------------------------------
// Dense local operator apply on a pre-gathered local vector.  A CTA of 8
// warps owns `rpc` consecutive rows of one subdomain; each warp walks its
// rows R at a time, keeping R independent accumulators so each v element read
// from shared memory feeds R FMAs.  FP64 matrices: row stride m, one double
// per lane per step.  FP32 matrices: row stride padded to a multiple of 4
// floats (zero padding), one float4 per lane per step, the input vector
// already in FP32, sums kept in FP32 per lane and across the warp (the
// operator itself carries FP32 rounding; an FP64 cross-lane reduction costs
// about a quarter of the kernel on GB300's FP64 pipe).
__device__ __forceinline__ int pad4(int m) { return (m + 3) & ~3; }

__device__ __forceinline__ float warp_sumf(float v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Transposed warp reduction of R values per lane (R = 2, 4, 8): each of the
// log2 R halving steps keeps half of the values and adds the partner's copy of
// that half, then plain xor steps finish; lane (32 / R) j and its group hold
// the warp total of value j.  R - 1 + 5 - log2 R adds per lane instead of 5 R
// (FP64 adds occupy GB300's narrow FP64 pipe).
template <int R>
__device__ __forceinline__ double transposed_warp_sum(const double (&v)[R], int lane) {
  double cur[R];
#pragma unroll
  for (int i = 0; i < R; ++i) cur[i] = v[i];
  int n = R;
#pragma unroll
  for (int m = 16; m >= 32 / R; m >>= 1) {
    const bool up = lane & m;
    n >>= 1;
#pragma unroll
    for (int i = 0; i < R / 2; ++i)
      if (i < n) {
        const double send = up ? cur[i] : cur[i + n];
        const double keep = up ? cur[i + n] : cur[i];
        cur[i] = keep + __shfl_xor_sync(0xffffffffu, send, m);
      }
  }
  double t = cur[0];
#pragma unroll
  for (int m = 16 / R; m >= 1; m >>= 1) t += __shfl_xor_sync(0xffffffffu, t, m);
  return t;
}

template <typename T, int R>
__global__ void __launch_bounds__(kThreads) k_gemv_loc(const int32_t* __restrict__ blk_sub,
                                                       const int32_t* __restrict__ blk_row0, int rpc,
                                                       const SubLayout* __restrict__ lay, int which,
                                                       const T* __restrict__ M, const T* __restrict__ vloc,
                                                       double* __restrict__ y, const int* __restrict__ done) {
  if (*done) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* v = reinterpret_cast<T*>(smem_raw);
  const int s = blk_sub[blockIdx.x];
  const int r0 = blk_row0[blockIdx.x];
  const SubLayout L = lay[s];
  const int m = which == 0 ? L.nbp : L.nbp + L.k;
  constexpr bool f32 = sizeof(T) == 4;
  const int ldm = f32 ? pad4(m) : m;
  const T* Ms = M + (f32 ? (which == 0 ? L.foff32 : L.soff32) : (which == 0 ? L.foff : L.soff));
  for (int p = threadIdx.x; p < ldm; p += blockDim.x) v[p] = p < m ? vloc[L.boff + p] : (T)0;
  if (which == 0 && r0 == 0)
    for (int p = L.nbp + threadIdx.x; p < L.nbp + L.k; p += blockDim.x) y[L.boff + p] = 0.0;
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int rend = min(r0 + rpc, m);
  for (int rbase = r0 + wid * R; rbase < rend; rbase += (kThreads / 32) * R) {
    T acc[R];
#pragma unroll
    for (int j = 0; j < R; ++j) acc[j] = (T)0;
    const T* rows[R];
#pragma unroll
    for (int j = 0; j < R; ++j) rows[j] = Ms + (size_t)min(rbase + j, m - 1) * ldm;
    if constexpr (f32) {
      const int m4 = ldm >> 2;
      const float4* v4 = reinterpret_cast<const float4*>(v);
      for (int c = lane; c < m4; c += 32) {
        const float4 vv = v4[c];
        float4 a[R];
#pragma unroll
        for (int j = 0; j < R; ++j) a[j] = __ldg(reinterpret_cast<const float4*>(rows[j]) + c);
#pragma unroll
        for (int j = 0; j < R; ++j) acc[j] += a[j].x * vv.x + a[j].y * vv.y + a[j].z * vv.z + a[j].w * vv.w;
      }
#pragma unroll
      for (int j = 0; j < R; ++j) {
        const float t = warp_sumf(acc[j]);
        if (lane == 0 && rbase + j < rend) y[L.boff + rbase + j] = (double)t;
      }
    } else {
      for (int c = lane; c < m; c += 32) {
        const T vv = v[c];
        T a[R];
#pragma unroll
        for (int j = 0; j < R; ++j) a[j] = __ldg(rows[j] + c);
#pragma unroll
        for (int j = 0; j < R; ++j) acc[j] += a[j] * vv;
      }
      if constexpr (R >= 2) {
        // after the halving steps on lane bits 4, 3, .. the lanes of group
        // g = lane / (32 / R) hold the total of row g
        double accd[R];
#pragma unroll
        for (int j = 0; j < R; ++j) accd[j] = acc[j];
        const double t = transposed_warp_sum<R>(accd, lane);
        const int g = lane / (32 / R);
        if (lane % (32 / R) == 0 && rbase + g < rend) y[L.boff + rbase + g] = t;
      } else {
#pragma unroll
        for (int j = 0; j < R; ++j) {
          const double t = warp_sum(acc[j]);
          if (lane == 0 && rbase + j < rend) y[L.boff + rbase + j] = t;
        }
      }
    }
  }
}

// Signed gather onto the boundary positions in FP32 (input of the FP32 apply).
__global__ void k_gather32(Maps mp, const double* __restrict__ x, const double* __restrict__ wv,
                           float* __restrict__ y, const int* __restrict__ done) {
  if (*done) return;
  for (int gp = blockIdx.x * blockDim.x + threadIdx.x; gp < mp.nb_total; gp += gridDim.x * blockDim.x) {
    double val = 0.0;
    for (int e = mp.bt_ptr[gp]; e < mp.bt_ptr[gp + 1]; ++e) {
      const int row = mp.bt_row[e];
      val += mp.bt_sgn[e] * x[row] * (wv ? wv[row] : 1.0);
    }
    y[gp] = (float)val;
  }
}

// Symmetric FP32 local apply y = M v from the lower block-triangle only (half
// the bytes of the full rows).  A warp owns one panel I of PH = kSymPH rows
// and sweeps its stored columns in 128-column tiles (one float4 per lane per
// row): each lane keeps a partial row sum for the PH rows and, per tile, the
// column sums a_rc v_r over the panel's rows, which are the transposed
// products of the blocks left of the diagonal block (columns < PH I); those
// go to the partial buffer, the row sums (one warp reduction per row) to y.
template <int G, int PF>
__global__ void __launch_bounds__(kThreads, G == kSymPH ? 1 : 2) k_symv_f32(
    const int32_t* __restrict__ wsub, const int32_t* __restrict__ wpanel, int n_warps,
    const SubLayout* __restrict__ lay, int which, const float* __restrict__ M, const float* __restrict__ vloc,
    double* __restrict__ y, float* __restrict__ part, const int* __restrict__ done) {
  constexpr int PH = kSymPH;
  if (*done) return;
  const int gw = blockIdx.x * (kThreads / 32) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (gw >= n_warps) return;
  const int s = wsub[gw], I = wpanel[gw];
  const SubLayout L = lay[s];
  const int m = which == 0 ? L.nbp : L.nbp + L.k;
  const int w = PH * (I + 1);
  const int r0 = PH * I;
  const float* Pn = M + (which == 0 ? L.fsym32 : L.ssym32) + (size_t)(PH * PH / 2) * I * (I + 1);
  const float* v = vloc + L.boff;
  float* Pp = part + L.psym + (size_t)(PH / 2) * I * (I - 1);
  if (which == 0 && I == 0)
    for (int p = lane; p < L.k; p += 32) y[L.boff + L.nbp + p] = 0.0;
  const float vrow = (lane < PH && r0 + lane < m) ? v[r0 + lane] : 0.f;
  float acc[PH];
#pragma unroll
  for (int i = 0; i < PH; ++i) acc[i] = 0.f;
  if (PF > 0)  // the first PF tiles of row `lane` towards L2
    for (int q = 0; q < PF && q * 128 < w; ++q)
      if (lane < PH) {
        const int cq = q * 128;
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(Pn + (size_t)lane * w + cq),
                     "r"((uint32_t)min(128, w - cq) * 4u)
                     : "memory");
      }
  for (int c0 = 0; c0 < w; c0 += 128) {
    if (PF > 0 && lane < PH && c0 + PF * 128 < w) {
      // row `lane`'s segment PF tiles ahead (16-byte aligned, a multiple of 128 bytes)
      const int cq = c0 + PF * 128;
      asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(Pn + (size_t)lane * w + cq),
                   "r"((uint32_t)min(128, w - cq) * 4u)
                   : "memory");
    }
    const int c = c0 + 4 * lane;
    const bool ok = c < w;
    const float4 vv = make_float4(c < m ? v[c] : 0.f, c + 1 < m ? v[c + 1] : 0.f, c + 2 < m ? v[c + 2] : 0.f,
                                  c + 3 < m ? v[c + 3] : 0.f);
    float4 col = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int g = 0; g < PH / G; ++g) {
      float4 a[G];
#pragma unroll
      for (int j = 0; j < G; ++j)
        a[j] = ok ? __ldg(reinterpret_cast<const float4*>(Pn + (size_t)(g * G + j) * w + c))
                  : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
      for (int j = 0; j < G; ++j) {
        const int i = g * G + j;
        acc[i] += a[j].x * vv.x + a[j].y * vv.y + a[j].z * vv.z + a[j].w * vv.w;
        const float vi = __shfl_sync(0xffffffffu, vrow, i);
        col.x += a[j].x * vi;
        col.y += a[j].y * vi;
        col.z += a[j].z * vi;
        col.w += a[j].w * vi;
      }
    }
    if (ok && c < r0) *reinterpret_cast<float4*>(Pp + c) = col;
  }
  float mine = 0.f;
#pragma unroll
  for (int i = 0; i < PH; ++i) {
    const float t = warp_sumf(acc[i]);
    if (lane == i) mine = t;
  }
  if (lane < PH && r0 + lane < m) y[L.boff + r0 + lane] = (double)mine;
}

// Subdomain-per-CTA variant of the symmetric FP32 apply, with no second
// pass: CTA b takes subdomain order[b] (largest first), its eight warps take
// the panels in a snake order (w, 15 - w, 16 + w, ..), each warp sweeps its
// panel exactly as k_symv_f32 does, keeps the panel's row sums in shared
// memory (one owner per row) and adds the transposed products of the blocks
// left of the diagonal into its own shared-memory column buffer.  After a
// barrier every row c gets row sum + the eight warps' column sums in warp
// order (deterministic, no atomics).
template <int G>
__global__ void __launch_bounds__(kThreads, G == kSymPH ? 1 : 2) k_symv3_f32(const int32_t* __restrict__ order,
                                                          const SubLayout* __restrict__ lay, int which,
                                                          const float* __restrict__ M,
                                                          const float* __restrict__ vloc, double* __restrict__ y,
                                                          const int* __restrict__ done) {
  constexpr int PH = kSymPH;
  constexpr int W = kThreads / 32;
  if (*done) return;
  extern __shared__ float s3[];
  const int s = order[blockIdx.x];
  const SubLayout L = lay[s];
  const int m = which == 0 ? L.nbp : L.nbp + L.k;
  const int mp = (m + 3) & ~3;
  float* rowsum = s3;               // [mp]
  float* colsum = s3 + mp;          // [W][mp]
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int i = threadIdx.x; i < (W + 1) * mp; i += kThreads) s3[i] = 0.f;
  if (which == 0)
    for (int p = threadIdx.x; p < L.k; p += kThreads) y[L.boff + L.nbp + p] = 0.0;
  __syncthreads();
  const float* Mbase = M + (which == 0 ? L.fsym32 : L.ssym32);
  const float* v = vloc + L.boff;
  float* cs = colsum + (size_t)warp * mp;
  const int nP = (m + PH - 1) / PH;
  for (int q = 0;; ++q) {
    const int base = (q >> 1) * 2 * W;
    const int I = (q & 1) ? base + 2 * W - 1 - warp : base + warp;
    if (base >= nP) break;
    if (I >= nP) continue;
    const int w = PH * (I + 1);
    const int r0 = PH * I;
    const float* Pn = Mbase + (size_t)(PH * PH / 2) * I * (I + 1);
    const float vrow = (r0 + lane < m) ? v[r0 + lane] : 0.f;
    float acc[PH];
#pragma unroll
    for (int i = 0; i < PH; ++i) acc[i] = 0.f;
    for (int c0 = 0; c0 < w; c0 += 128) {
      const int c = c0 + 4 * lane;
      const bool ok = c < w;
      const float4 vv = make_float4(c < m ? v[c] : 0.f, c + 1 < m ? v[c + 1] : 0.f, c + 2 < m ? v[c + 2] : 0.f,
                                    c + 3 < m ? v[c + 3] : 0.f);
      float4 col = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
      for (int g = 0; g < PH / G; ++g) {
        float4 a[G];
#pragma unroll
        for (int j = 0; j < G; ++j)
          a[j] = ok ? __ldg(reinterpret_cast<const float4*>(Pn + (size_t)(g * G + j) * w + c))
                    : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int j = 0; j < G; ++j) {
          const int i = g * G + j;
          acc[i] += a[j].x * vv.x + a[j].y * vv.y + a[j].z * vv.z + a[j].w * vv.w;
          const float vi = __shfl_sync(0xffffffffu, vrow, i);
          col.x += a[j].x * vi;
          col.y += a[j].y * vi;
          col.z += a[j].z * vi;
          col.w += a[j].w * vi;
        }
      }
      if (ok && c < r0) {
        float4* d = reinterpret_cast<float4*>(cs + c);
        float4 t = *d;
        t.x += col.x;
        t.y += col.y;
        t.z += col.z;
        t.w += col.w;
        *d = t;
      }
    }
    float mine = 0.f;
#pragma unroll
    for (int i = 0; i < PH; ++i) {
      const float t = warp_sumf(acc[i]);
      if (lane == i) mine = t;
    }
    if (r0 + lane < m) rowsum[r0 + lane] = mine;
  }
  __syncthreads();
  for (int c = threadIdx.x; c < m; c += kThreads) {
    float t = rowsum[c];
#pragma unroll
    for (int q = 0; q < W; ++q) t += colsum[(size_t)q * mp + c];
    y[L.boff + c] = (double)t;
  }
}

// Streamed variant of the symmetric FP32 apply: the same panels, partials
// and fix kernel, but each warp streams its panel through a ring of SYM_NS
// shared-memory stages of 32 rows x 64 columns (8 KB): every lane copies one
// 256-byte row segment with cp.async.bulk (completion counted in bytes on the
// stage's mbarrier), so the next tiles are in flight while the current one is
// reduced, and the arithmetic reads shared memory instead of holding the
// loads in registers (16 row accumulators per lane: half-warp h takes rows
// 2j + h).  Warps are independent (no CTA barrier in the loop); all waits are
// bounded, and a warp whose wait runs out flags *err, issues nothing more and
// waits (bounded) for its copies in flight before it returns.  The main-loop
// waits give up after *spin_cycles SM clock cycles (the context's spin
// timeout); the drain waits keep a fixed budget of 2e8 clock cycles, so every
// copy issued has landed before the warp leaves.
constexpr int SYM_TW = 64;  // tile width (floats)
constexpr int SYM_NS = 3;   // stages per warp
constexpr int SYM_WPC = 4;  // warps per CTA
constexpr int SYM_STAGE = 32 * SYM_TW * 4;  // bytes

__device__ __forceinline__ uint32_t sym_su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ bool sym_try(uint64_t* b, uint32_t par) {
  uint32_t ok;
  asm volatile("{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
               : "=r"(ok)
               : "r"(sym_su32(b)), "r"(par)
               : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool sym_wait(uint64_t* b, uint32_t par) {
  const long long t0 = clock64();
  while (!sym_try(b, par))
    if (clock64() - t0 > 200000000LL) return false;
  return true;
}
// main-loop wait with a caller-set budget in SM clock cycles, checked before
// every try (a zero budget gives up at once)
__device__ __forceinline__ bool sym_wait_cycles(uint64_t* b, uint32_t par, long long budget) {
  const long long t0 = clock64();
  for (;;) {
    if (clock64() - t0 >= budget) return false;
    if (sym_try(b, par)) return true;
  }
}

__global__ void __launch_bounds__(SYM_WPC * 32) k_symv2_f32(const int32_t* __restrict__ wsub,
                                                           const int32_t* __restrict__ wpanel, int n_warps,
                                                           const SubLayout* __restrict__ lay, int which,
                                                           const float* __restrict__ M, const float* __restrict__ vloc,
                                                           double* __restrict__ y, float* __restrict__ part,
                                                           const int* __restrict__ done, int* __restrict__ err,
                                                           const unsigned long long* __restrict__ spin_cycles) {
  if (*done) return;
  extern __shared__ __align__(128) unsigned char sym_smem[];
  __shared__ uint64_t full[SYM_WPC][SYM_NS];
  const int wl = threadIdx.x >> 5, lane = threadIdx.x & 31, h = lane >> 4, l16 = lane & 15;
  const int gw = blockIdx.x * SYM_WPC + wl;
  if (gw >= n_warps) return;
  const int s = wsub[gw], I = wpanel[gw];
  const SubLayout L = lay[s];
  const int m = which == 0 ? L.nbp : L.nbp + L.k;
  const int w = 32 * (I + 1);
  const int r0 = 32 * I;
  const float* Pn = M + (which == 0 ? L.fsym32 : L.ssym32) + (size_t)512 * I * (I + 1);
  const float* v = vloc + L.boff;
  float* Pp = part + L.psym + (size_t)16 * I * (I - 1);
  unsigned char* ring = sym_smem + (size_t)wl * SYM_NS * SYM_STAGE;
  uint64_t* fb = full[wl];
  if (lane == 0) {
    for (int q = 0; q < SYM_NS; ++q)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(sym_su32(&fb[q])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();
  if (which == 0 && I == 0)
    for (int p = lane; p < L.k; p += 32) y[L.boff + L.nbp + p] = 0.0;
  const int nt = (w + SYM_TW - 1) / SYM_TW;
  // tile t -> stage t % NS: lane i copies row i's segment of the tile
  auto issue = [&](int t) {
    const int st = t % SYM_NS;
    const int c0 = t * SYM_TW;
    const uint32_t seg = (uint32_t)min(SYM_TW, w - c0) * 4u;
    if (lane == 0)
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(sym_su32(&fb[st])), "r"(seg * 32u)
                   : "memory");
    __syncwarp();
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     sym_su32(ring + st * SYM_STAGE + lane * SYM_TW * 4)),
                 "l"(Pn + (size_t)lane * w + c0), "r"(seg), "r"(sym_su32(&fb[st]))
                 : "memory");
  };
  int issued = 0;
  for (; issued < SYM_NS && issued < nt; ++issued) issue(issued);
  const float vrow = r0 + lane < m ? v[r0 + lane] : 0.f;
  float acc[16];
#pragma unroll
  for (int j = 0; j < 16; ++j) acc[j] = 0.f;
  bool bad = false;
  int t = 0;
  const long long budget = (long long)*spin_cycles;
  for (; t < nt; ++t) {
    const int st = t % SYM_NS;
    if (!sym_wait_cycles(&fb[st], (uint32_t)(t / SYM_NS) & 1u, budget)) bad = true;
    bad = __any_sync(0xffffffffu, bad);
    if (bad) break;
    const int c = t * SYM_TW + 4 * l16;
    const bool ok = c < w;
    const float4 vv = make_float4(c < m ? v[c] : 0.f, c + 1 < m ? v[c + 1] : 0.f, c + 2 < m ? v[c + 2] : 0.f,
                                  c + 3 < m ? v[c + 3] : 0.f);
    const float4* tile = reinterpret_cast<const float4*>(ring + st * SYM_STAGE);
    float4 col = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const int r = 2 * j + h;
      const float4 a = ok ? tile[r * (SYM_TW / 4) + l16] : make_float4(0.f, 0.f, 0.f, 0.f);
      acc[j] += a.x * vv.x + a.y * vv.y + a.z * vv.z + a.w * vv.w;
      const float vi = __shfl_sync(0xffffffffu, vrow, r);
      col.x += a.x * vi;
      col.y += a.y * vi;
      col.z += a.z * vi;
      col.w += a.w * vi;
    }
    col.x += __shfl_xor_sync(0xffffffffu, col.x, 16);
    col.y += __shfl_xor_sync(0xffffffffu, col.y, 16);
    col.z += __shfl_xor_sync(0xffffffffu, col.z, 16);
    col.w += __shfl_xor_sync(0xffffffffu, col.w, 16);
    if (h == 0 && ok && c < r0) *reinterpret_cast<float4*>(Pp + c) = col;
    // every lane has read the stage: order those reads before the refill
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncwarp();
    if (t + SYM_NS < nt) {
      issue(t + SYM_NS);
      issued = t + SYM_NS + 1;
    }
  }
  if (bad) {
    // copies in flight land before the warp leaves (fresh bounded waits)
    for (int j = t; j < issued; ++j) sym_wait(&fb[j % SYM_NS], (uint32_t)(j / SYM_NS) & 1u);
    if (lane == 0) atomicExch(err, 1);
    return;
  }
  // row 2j + h: reduce over the 16 lanes of half h
  float mine = 0.f;
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    float x = acc[j];
    x += __shfl_xor_sync(0xffffffffu, x, 8);
    x += __shfl_xor_sync(0xffffffffu, x, 4);
    x += __shfl_xor_sync(0xffffffffu, x, 2);
    x += __shfl_xor_sync(0xffffffffu, x, 1);
    if (l16 == j) mine = x;  // lane 16 h + j holds row 2j + h
  }
  const int row = r0 + 2 * l16 + h;
  if (row < m) y[L.boff + row] = (double)mine;
}

// y[c] += sum over the panels I below row c (I = c/PH + 1, ..) of their
// transposed products at column c, in that order.
__global__ void k_symv_fix(Maps mp, const SubLayout* __restrict__ lay, int which, const float* __restrict__ part,
                           double* __restrict__ y, const int* __restrict__ done) {
  constexpr int PH = kSymPH;
  if (*done) return;
  for (int gp = blockIdx.x * blockDim.x + threadIdx.x; gp < mp.nb_total; gp += gridDim.x * blockDim.x) {
    const SubLayout L = lay[mp.bpos_sub[gp]];
    const int m = which == 0 ? L.nbp : L.nbp + L.k;
    const int c = gp - L.boff;
    if (c >= m) continue;
    const int nP = (m + PH - 1) / PH;
    const float* ps = part + L.psym;
    // FP32 sum in panel order (the partials carry the FP32 operator's rounding;
    // FP64 adds and conversions would occupy GB300's narrow FP64 pipe), loads
    // requested sixteen at a time, one FP64 addition to y
    float t = 0.f;
    for (int I0 = c / PH + 1; I0 < nP; I0 += 16) {
      float f[16];
#pragma unroll
      for (int u = 0; u < 16; ++u) {
        const int I = I0 + u;
        f[u] = I < nP ? __ldg(ps + (size_t)(PH / 2) * I * (I - 1) + c) : 0.f;
      }
#pragma unroll
      for (int u = 0; u < 16; ++u) t += f[u];
    }
    y[gp] += (double)t;
  }
}

__global__ void k_vadd(int n, double* __restrict__ a, const double* __restrict__ b) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) a[i] += b[i];
}

__global__ void k_gather(Maps mp, const double* __restrict__ x, const double* __restrict__ wv,
                         double* __restrict__ y, const int* __restrict__ done) {
  if (*done) return;
  for (int gp = blockIdx.x * blockDim.x + threadIdx.x; gp < mp.nb_total; gp += gridDim.x * blockDim.x) {
    double val = 0.0;
    for (int e = mp.bt_ptr[gp]; e < mp.bt_ptr[gp + 1]; ++e) {
      const int row = mp.bt_row[e];
      val += mp.bt_sgn[e] * x[row] * (wv ? wv[row] : 1.0);
    }
    y[gp] = val;
  }
}

__global__ void __launch_bounds__(kThreads) k_scatter(Maps mp, const double* __restrict__ y,
                                                      const double* __restrict__ wv, double* __restrict__ q,
                                                      const double* __restrict__ a, double* __restrict__ partial,
                                                      const int* __restrict__ done) {
  if (*done) return;
  __shared__ double red[32];
  double dot = 0.0;
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < mp.n_lambda; r += gridDim.x * blockDim.x) {
    double val = 0.0;
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const int pos = mp.row_pos[2 * r + e];
      if (pos >= 0) val += mp.row_sgn[2 * r + e] * y[pos];
    }
    if (wv) val *= wv[r];
    q[r] = val;
    if (partial) dot += (a ? a[r] : val) * val;
  }
  if (partial) {
    dot = block_sum(dot, red);
    if (threadIdx.x == 0) partial[blockIdx.x] = dot;
  }
}

__global__ void __launch_bounds__(kThreads) k_gtv(const SubLayout* __restrict__ lay, const double* __restrict__ R,
                                                  Maps mp, const double* __restrict__ x, double* __restrict__ g,
                                                  const int* __restrict__ done) {
  if (*done) return;
  const int s = blockIdx.x;
  const SubLayout L = lay[s];
  if (L.k == 0) return;
  __shared__ double red[32];
  const int nb = L.nbp + L.k;
  double acc[6] = {0, 0, 0, 0, 0, 0};
  for (int p = threadIdx.x; p < nb; p += blockDim.x) {
    const int gp = L.boff + p;
    double val = 0.0;
    for (int e = mp.bt_ptr[gp]; e < mp.bt_ptr[gp + 1]; ++e) val += mp.bt_sgn[e] * x[mp.bt_row[e]];
    const double* Rr = R + L.roff + (size_t)(L.nI + p) * L.k;
    for (int a = 0; a < L.k; ++a) acc[a] += Rr[a] * val;
  }
  for (int a = 0; a < L.k; ++a) {
    const double t = block_sum(acc[a], red);
    if (threadIdx.x == 0) g[L.coff + a] = t;
  }
}

__device__ double reduce_partials(const double* partial, double* red) {
  double t = 0.0;
  for (int i = threadIdx.x; i < kPartials; i += blockDim.x) t += partial[i];
  return block_sum(t, red);
}

// G^T x split over chunks of 256 boundary positions (one CTA per chunk,
// several per subdomain): partial[c*6 + a] = sum over the chunk of
// R_b[p][a] (B^T x)[p].
// With q != NULL the input is the updated residual x - alpha q, alpha =
// rho / (p, q) evaluated by every CTA from the partial sums of (p, q) (the
// fused CG step); CTA 0 records alpha and flags a breakdown.
__global__ void __launch_bounds__(kThreads) k_gtv_part(const int32_t* __restrict__ chunk_sub,
                                                       const int32_t* __restrict__ chunk_p0, int n_chunks,
                                                       const SubLayout* __restrict__ lay,
                                                       const double* __restrict__ R, Maps mp,
                                                       const double* __restrict__ x, double* __restrict__ partial,
                                                       const int* __restrict__ done, const double* __restrict__ q,
                                                       const double* __restrict__ pq_partial, PcgScalars* sc,
                                                       double* __restrict__ alpha_hist) {
  if (*done) return;
  __shared__ double red[32];
  double alpha = 0.0;
  if (q) {
    const double pq = reduce_partials(pq_partial, red);
    alpha = sc->rho / pq;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      if (!(pq > 0.0) || !isfinite(pq)) {
        sc->status = DEV_BREAKDOWN;
        sc->done = 1;
      }
      sc->alpha = alpha;
      sc->pq = pq;
      alpha_hist[sc->it] = alpha;
    }
  }
  // one position per thread (the gathers' load chains run in parallel);
  // the six coarse columns are reduced by a transposed warp reduction (8
  // values -> one per lane group in 9 FP64 adds instead of 6 x 5 on GB300's
  // narrow FP64 pipe) and the eight warps' results summed in warp order
  const int c = blockIdx.x;
  if (c >= n_chunks) return;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const SubLayout L = lay[chunk_sub[c]];
  const int nb = L.nbp + L.k;
  const int p = chunk_p0[c] + threadIdx.x;
  double v8[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  if (p < nb) {
    const int gp = L.boff + p;
    double val = 0.0;
    for (int e = mp.bt_ptr[gp]; e < mp.bt_ptr[gp + 1]; ++e) {
      const int row = mp.bt_row[e];
      val += mp.bt_sgn[e] * (q ? x[row] - alpha * q[row] : x[row]);
    }
    const double* Rr = R + L.roff + (size_t)(L.nI + p) * L.k;
    for (int a = 0; a < L.k; ++a) v8[a] = Rr[a] * val;
  }
  // step 16: keep half the values, add the partner's copy of that half
  double v4[4], v2[2], v1;
  {
    const bool up = lane & 16;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const double send = up ? v8[i] : v8[i + 4];
      const double keep = up ? v8[i + 4] : v8[i];
      v4[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
    }
  }
  {
    const bool up = lane & 8;
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const double send = up ? v4[i] : v4[i + 2];
      const double keep = up ? v4[i + 2] : v4[i];
      v2[i] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
    }
  }
  {
    const bool up = lane & 4;
    const double send = up ? v2[0] : v2[1];
    const double keep = up ? v2[1] : v2[0];
    v1 = keep + __shfl_xor_sync(0xffffffffu, send, 4);
  }
  v1 += __shfl_xor_sync(0xffffffffu, v1, 2);
  v1 += __shfl_xor_sync(0xffffffffu, v1, 1);
  // lane 4 g holds column a = 4 (g >> 2 & 1) + 2 (g >> 1 & 1) + (g & 1), g = lane / 4
  __shared__ double wsum[kThreads / 32][8];
  if ((lane & 3) == 0) {
    const int g = lane >> 2;
    const int a = 4 * ((g >> 2) & 1) + 2 * ((g >> 1) & 1) + (g & 1);
    wsum[wid][a] = v1;
  }
  __syncthreads();
  if (threadIdx.x < L.k) {
    double t = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) t += wsum[w][threadIdx.x];
    partial[6 * c + threadIdx.x] = t;
  }
}

// c = Ginv g where g is first summed (fixed order) from the chunk partials of
// k_gtv_part into shared memory by every CTA.
__global__ void k_coarse_apply_part(int cd, const double* __restrict__ Ginv, const double* __restrict__ partial,
                                    const int32_t* __restrict__ sub_chunk_ptr, const int32_t* __restrict__ col_sub,
                                    const SubLayout* __restrict__ lay, double* __restrict__ c,
                                    const int* __restrict__ done) {
  if (*done) return;
  extern __shared__ double gsh[];
  for (int j = threadIdx.x; j < cd; j += blockDim.x) {
    const int s = col_sub[j];
    const int a = j - lay[s].coff;
    double t = 0.0;
    for (int q = sub_chunk_ptr[s]; q < sub_chunk_ptr[s + 1]; ++q) t += partial[6 * q + a];
    gsh[j] = t;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int r = warp; r < cd; r += nwarps) {
    double acc = 0.0;
    for (int j = lane; j < cd; j += 32) acc += Ginv[(size_t)r * cd + j] * gsh[j];
    acc = warp_sum(acc);
    if (lane == 0) c[r] = acc;
  }
}

__global__ void k_coarse_apply(int cd, const double* __restrict__ Ginv, const double* __restrict__ g,
                               double* __restrict__ c, const int* __restrict__ done) {
  if (*done) return;
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int r = warp; r < cd; r += nwarps) {
    double acc = 0.0;
    for (int j = lane; j < cd; j += 32) acc += Ginv[(size_t)r * cd + j] * g[j];
    acc = warp_sum(acc);
    if (lane == 0) c[r] = acc;
  }
}

// Fused CG update (upd != NULL): r <- r - alpha q and lam <- lam + alpha p
// in place (alpha = rho / (p, q) from the partial sums), then out = r - G c.
struct ExpandUpdate {
  double* r;
  double* lam;
  const double* p;
  const double* q;
  const double* pq_partial;
  PcgScalars* sc;
  double* alpha_hist;
};

__global__ void __launch_bounds__(kThreads) k_expand(Maps mp, const SubLayout* __restrict__ lay,
                                                     const double* __restrict__ R, const double* __restrict__ v,
                                                     const double* __restrict__ c, double* __restrict__ out,
                                                     const double* __restrict__ a, double* __restrict__ partial,
                                                     int with_dot, const int* __restrict__ done, ExpandUpdate upd) {
  if (*done) return;
  __shared__ double red[32];
  double alpha = 0.0;
  if (upd.r) {
    const double pq = reduce_partials(upd.pq_partial, red);
    alpha = upd.sc->rho / pq;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      if (!(pq > 0.0) || !isfinite(pq)) {
        upd.sc->status = DEV_BREAKDOWN;
        upd.sc->done = 1;
      }
      upd.sc->alpha = alpha;
      upd.sc->pq = pq;
      upd.alpha_hist[upd.sc->it] = alpha;
    }
  }
  double dot = 0.0;
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < mp.n_lambda; r += gridDim.x * blockDim.x) {
    double val;
    if (upd.r) {
      val = upd.r[r] - alpha * upd.q[r];
      upd.r[r] = val;
      upd.lam[r] += alpha * upd.p[r];
    } else {
      val = v[r];
    }
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const int gp = mp.row_pos[2 * r + e];
      if (gp >= 0) {
        const SubLayout L = lay[mp.bpos_sub[gp]];
        if (L.k) {
          const double* Rr = R + L.roff + (size_t)(L.nI + gp - L.boff) * L.k;
          double t = 0.0;
          for (int k = 0; k < L.k; ++k) t += Rr[k] * c[L.coff + k];
          val -= mp.row_sgn[2 * r + e] * t;
        }
      }
    }
    out[r] = val;
    if (with_dot) dot += (a ? a[r] : val) * val;
  }
  if (with_dot) {
    dot = block_sum(dot, red);
    if (threadIdx.x == 0) partial[blockIdx.x] = dot;
  }
}

// G^T G: one CTA per pair block (i, j), thread per entry, rows in fixed order.
__global__ void k_gtg(const int32_t* __restrict__ blk_i, const int32_t* __restrict__ blk_j,
                      const int32_t* __restrict__ blk_ptr, const int32_t* __restrict__ blk_rows,
                      const SubLayout* __restrict__ lay, const double* __restrict__ R, Maps mp, int cd,
                      double* __restrict__ GtG) {
  const int b = blockIdx.x;
  const int si = blk_i[b], sj = blk_j[b];
  const SubLayout Li = lay[si], Lj = lay[sj];
  const int t = threadIdx.x;
  if (t >= Li.k * Lj.k) return;
  const int a = t / Lj.k, c = t % Lj.k;
  double acc = 0.0;
  for (int q = blk_ptr[b]; q < blk_ptr[b + 1]; ++q) {
    const int r = blk_rows[q];
    double gi = 0.0, gj = 0.0;
    for (int e = 0; e < 2; ++e) {
      const int gp = mp.row_pos[2 * r + e];
      if (gp < 0) continue;
      const int s = mp.bpos_sub[gp];
      if (s == si) gi += mp.row_sgn[2 * r + e] * R[Li.roff + (size_t)(Li.nI + gp - Li.boff) * Li.k + a];
      if (s == sj) gj += mp.row_sgn[2 * r + e] * R[Lj.roff + (size_t)(Lj.nI + gp - Lj.boff) * Lj.k + c];
    }
    acc += gi * gj;
  }
  GtG[(size_t)(Li.coff + a) * cd + Lj.coff + c] = acc;
  GtG[(size_t)(Lj.coff + c) * cd + Li.coff + a] = acc;
}

// ---------------------------------------------------------------------------

__global__ void k_ctl_conv(PcgScalars* s, const double* __restrict__ partial, int first) {
  if (s->done) return;
  __shared__ double red[32];
  const double wn = sqrt(reduce_partials(partial, red));
  if (threadIdx.x == 0) {
    if (first) {
      s->wnorm0 = wn;
      s->wnorm = wn;
      if (!(wn > 0.0)) s->done = 1;
      if (!isfinite(wn)) {
        s->status = DEV_BREAKDOWN;
        s->done = 1;
      }
      return;
    }
    s->it += 1;
    s->wnorm = wn;
    if (!isfinite(wn)) {
      s->status = DEV_BREAKDOWN;
      s->done = 1;
    } else if (wn <= s->tol * s->wnorm0 || s->it >= s->maxit) {
      s->done = 1;
    }
  }
}

// Fused CG step: rho = (w, y) from the partial sums (every CTA), beta =
// rho / rho_prev (rho_prev kept in the slot of the previous iteration's
// parity), p = y + beta p; CTA 0 records rho and beta and flags a breakdown.
__global__ void __launch_bounds__(kThreads) k_axpby_rho(int n, double* __restrict__ p, const double* __restrict__ y,
                                                        PcgScalars* s, const double* __restrict__ partial,
                                                        double* __restrict__ beta_hist) {
  if (s->done) return;
  __shared__ double red[32];
  const double rho = reduce_partials(partial, red);
  const int it = s->it;
  const double beta = it > 0 ? rho / s->rho_slot[(it + 1) & 1] : 0.0;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    if (!(rho > 0.0) || !isfinite(rho)) {
      s->status = DEV_BREAKDOWN;
      s->done = 1;
    }
    s->rho_slot[it & 1] = rho;
    s->rho = rho;
    s->beta = beta;
    beta_hist[it] = beta;
  }
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    p[i] = it > 0 ? y[i] + beta * p[i] : y[i];
}

__global__ void k_vsub(int n, const double* a, const double* b, double* out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) out[i] = a[i] - b[i];
}

__global__ void k_owner_scatter(int n, const int32_t* __restrict__ gdof, const int32_t* __restrict__ vpos,
                                const double* __restrict__ x, double* __restrict__ U) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) U[gdof[i]] = x[vpos[i]];
}

__global__ void k_add_kernel(const SubLayout* __restrict__ lay, const double* __restrict__ R,
                             const double* __restrict__ gamma, double* __restrict__ xbase) {
  const int s = blockIdx.x;
  const SubLayout L = lay[s];
  if (L.k == 0) return;
  double* x = xbase + L.voff;
  for (int d = threadIdx.x; d < L.n; d += blockDim.x) {
    double t = 0.0;
    for (int a = 0; a < L.k; ++a) t += R[L.roff + (size_t)d * L.k + a] * gamma[L.coff + a];
    x[d] += t;
  }
}

__global__ void __launch_bounds__(kThreads) k_rtx(const SubLayout* __restrict__ lay, const double* __restrict__ R,
                                                  const double* __restrict__ xbase, double scale,
                                                  double* __restrict__ e) {
  const int s = blockIdx.x;
  const SubLayout L = lay[s];
  if (L.k == 0) return;
  __shared__ double red[32];
  const double* x = xbase + L.voff;
  double acc[6] = {0, 0, 0, 0, 0, 0};
  for (int d = threadIdx.x; d < L.n; d += blockDim.x) {
    const double* Rr = R + L.roff + (size_t)d * L.k;
    for (int a = 0; a < L.k; ++a) acc[a] += Rr[a] * x[d];
  }
  for (int a = 0; a < L.k; ++a) {
    const double t = block_sum(acc[a], red);
    if (threadIdx.x == 0) e[L.coff + a] = scale * t;
  }
}

__global__ void k_take_boundary(const SubLayout* __restrict__ lay, const double* __restrict__ xbase,
                                double* __restrict__ loc, const int* __restrict__ done) {
  if (done && *done) return;
  const int s = blockIdx.x;
  const SubLayout L = lay[s];
  for (int p = threadIdx.x; p < L.nbp + L.k; p += blockDim.x) loc[L.boff + p] = xbase[L.voff + L.nI + p];
}

__global__ void k_local_sub(const SubLayout* __restrict__ lay, const double* __restrict__ fbase,
                            const double* __restrict__ loc, double* __restrict__ obase) {
  const int s = blockIdx.x;
  const SubLayout L = lay[s];
  const double* f = fbase + L.voff;
  double* o = obase + L.voff;
  for (int d = threadIdx.x; d < L.n; d += blockDim.x)
    o[d] = d < L.nI ? f[d] : f[d] - loc[L.boff + d - L.nI];
}

inline int grid_for(long n, int threads = kThreads) {
  long b = (n + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > 65535) b = 65535;
  return (int)b;
}

}  // namespace

int scatter_partials() { return kPartials; }

void launch_elem_linear(int n_tets, const double* coords, const int32_t* tets, double E, double nu, double* Ke,
                        int* status, cudaStream_t st) {
  if (n_tets <= 0) return;
  k_elem_linear<<<(n_tets + 127) / 128, 128, 0, st>>>(n_tets, coords, tets, E, nu, Ke, status);
}

void launch_elem_hgo(int n_tets, const double* coords, const int32_t* tets, const double* U,
                     const double* fibres, double c, double k1, double k2, double kappa, double* Ke, double* fe,
                     int* status, cudaStream_t st) {
  if (n_tets <= 0) return;
  k_elem_hgo<<<(n_tets + 63) / 64, 64, 0, st>>>(n_tets, coords, tets, U, fibres, c, k1, k2, kappa, Ke, fe,
                                                status);
}

void launch_assemble(int P, const SubLayout* lay, const int32_t* sub_elem_ptr, const int32_t* sub_elems,
                     const int32_t* elem_dense, const double* Ke, int nde, double* A, cudaStream_t st) {
  k_assemble<double><<<P, nde > 12 ? 256 : 160, 0, st>>>(lay, sub_elem_ptr, sub_elems, elem_dense, Ke, nde, A);
}

void launch_assemble(int P, const SubLayout* lay, const int32_t* sub_elem_ptr, const int32_t* sub_elems,
                     const int32_t* elem_dense, const double* Ke, int nde, float* A, cudaStream_t st) {
  k_assemble<float><<<P, nde > 12 ? 256 : 160, 0, st>>>(lay, sub_elem_ptr, sub_elems, elem_dense, Ke, nde, A);
}

void launch_assemble_rhs(int P, const SubLayout* lay, const int32_t* sub_face_ptr, const int32_t* face_dense,
                         const double* face_force, int fdn, const int32_t* sub_elem_ptr, const int32_t* sub_elems,
                         const int32_t* elem_dense, const double* elem_dirval, const double* Ke, const double* fe,
                         int nde, double tau, double* f, cudaStream_t st) {
  k_assemble_rhs<<<P, 128, 0, st>>>(lay, sub_face_ptr, face_dense, face_force, fdn, sub_elem_ptr, sub_elems,
                                     elem_dense, elem_dirval, Ke, fe, nde, tau, f);
}

void launch_face_forces(int n_faces, int fpn, const int32_t* tri, const double* coords, const double* U, int kind,
                        double scale, const double* traction, double* out, cudaStream_t st) {
  if (n_faces <= 0) return;
  k_face_forces<<<(n_faces + 127) / 128, 128, 0, st>>>(n_faces, fpn, tri, coords, U, kind, scale, traction, out);
}

void launch_elem_linear_p2(int n_tets, const double* coords, const int32_t* tets, double E, double nu, int p0,
                           double* Ke, int* status, cudaStream_t st) {
  if (n_tets <= 0) return;
  const long threads = 32L * n_tets;
  k_elem_linear_p2<<<(unsigned)((threads + 127) / 128), 128, 0, st>>>(n_tets, coords, tets, E, nu, p0, Ke, status);
}

namespace {
// A_ii += delta * max_j A_jj over the rows [0, nI + nbp) of K_rr in each
// subdomain's dense workspace (a Levenberg-type shift of the local tangent).
__global__ void k_shift_diag(const SubLayout* __restrict__ lay, double* __restrict__ Abase, double delta) {
  const SubLayout L = lay[blockIdx.x];
  double* A = Abase + L.aoff;
  const int nr = L.nI + L.nbp;
  __shared__ double wmax[kThreads / 32];
  double m = 0.0;
  for (int i = threadIdx.x; i < nr; i += blockDim.x) m = fmax(m, A[(size_t)i * L.ld + i]);
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = m;
  __syncthreads();
  double mm = 0.0;
  for (int w = 0; w < (int)(blockDim.x / 32); ++w) mm = fmax(mm, wmax[w]);
  const double sh = delta * mm;
  for (int i = threadIdx.x; i < nr; i += blockDim.x) A[(size_t)i * L.ld + i] += sh;
}
}  // namespace

void launch_shift_diag(int P, const SubLayout* lay, double* A, double delta, cudaStream_t st) {
  k_shift_diag<<<P, kThreads, 0, st>>>(lay, A, delta);
}

void launch_augment(int P, const SubLayout* lay, double* A, cudaStream_t st) {
  k_augment<double><<<P, kThreads, 0, st>>>(lay, A);
}

void launch_augment(int P, const SubLayout* lay, float* A, cudaStream_t st) {
  k_augment<float><<<P, kThreads, 0, st>>>(lay, A);
}

void launch_extract(int P, const SubLayout* lay, int which, const double* A, double* out, cudaStream_t st) {
  k_extract<<<P, kThreads, 0, st>>>(lay, which, A, out);
}

void launch_kplus(int P, const SubLayout* lay, const double* A, const double* g, double* x, cudaStream_t st,
                  const int* done) {
  k_kplus<<<P, kThreads, 0, st>>>(lay, A, g, x, done);
}

void launch_gather(const Maps& mp, const double* x, const double* wv, double* y, const int* done,
                   cudaStream_t st) {
  k_gather<<<grid_for(mp.nb_total), kThreads, 0, st>>>(mp, x, wv, y, done);
}

void launch_scatter(const Maps& mp, const double* y, const double* wv, double* q, const double* a,
                    double* partial, const int* done, cudaStream_t st) {
  k_scatter<<<kPartials, kThreads, 0, st>>>(mp, y, wv, q, a, partial, done);
}

void launch_gtv(int P, const SubLayout* lay, const double* R, const Maps& mp, const double* x, double* g,
                const int* done, cudaStream_t st) {
  k_gtv<<<P, kThreads, 0, st>>>(lay, R, mp, x, g, done);
}

void launch_coarse_apply(int cd, const double* Ginv, const double* g, double* c, const int* done,
                         cudaStream_t st) {
  if (cd <= 0) return;
  const int warps = cd < 2432 ? cd : 2432;
  k_coarse_apply<<<(warps * 32 + kThreads - 1) / kThreads, kThreads, 0, st>>>(cd, Ginv, g, c, done);
}

void launch_expand(const Maps& mp, const SubLayout* lay, const double* R, const double* v, const double* c,
                   double* out, const double* a, double* partial, int with_dot, const int* done,
                   cudaStream_t st) {
  k_expand<<<kPartials, kThreads, 0, st>>>(mp, lay, R, v, c, out, a, partial, with_dot, done, ExpandUpdate{});
}

void launch_gtg(int n_blocks, const int32_t* blk_i, const int32_t* blk_j, const int32_t* blk_ptr,
                const int32_t* blk_rows, const SubLayout* lay, const double* R, const Maps& mp, int cd,
                double* GtG, cudaStream_t st) {
  if (n_blocks <= 0) return;
  k_gtg<<<n_blocks, 64, 0, st>>>(blk_i, blk_j, blk_ptr, blk_rows, lay, R, mp, cd, GtG);
}

void launch_ctl_conv(PcgScalars* s, const double* partial, int first, cudaStream_t st) {
  k_ctl_conv<<<1, kThreads, 0, st>>>(s, partial, first);
}
void launch_vsub(int n, const double* a, const double* b, double* out, cudaStream_t st) {
  k_vsub<<<grid_for(n), kThreads, 0, st>>>(n, a, b, out);
}
void launch_owner_scatter(int n_entries, const int32_t* gdof, const int32_t* vpos, const double* x, double* U,
                          cudaStream_t st) {
  if (n_entries <= 0) return;
  k_owner_scatter<<<grid_for(n_entries), kThreads, 0, st>>>(n_entries, gdof, vpos, x, U);
}
void launch_add_kernel(int P, const SubLayout* lay, const double* R, const double* gamma, double* x,
                       cudaStream_t st) {
  k_add_kernel<<<P, kThreads, 0, st>>>(lay, R, gamma, x);
}

void launch_rtx(int P, const SubLayout* lay, const double* R, const double* x, double scale, double* e,
                cudaStream_t st) {
  k_rtx<<<P, kThreads, 0, st>>>(lay, R, x, scale, e);
}
void launch_take_boundary(int P, const SubLayout* lay, const double* x, double* loc, cudaStream_t st,
                          const int* done) {
  k_take_boundary<<<P, kThreads, 0, st>>>(lay, x, loc, done);
}
void launch_local_sub(int P, const SubLayout* lay, const double* f, const double* loc, double* out,
                      cudaStream_t st) {
  k_local_sub<<<P, kThreads, 0, st>>>(lay, f, loc, out);
}

template <typename T, int R>
static void launch_gemv_t(int n_blocks, const int32_t* blk_sub, const int32_t* blk_row0, int rpc, const SubLayout* lay,
                          int which, const T* M, const T* vloc, double* y, int max_m, const int* done,
                          cudaStream_t st) {
  const size_t smem = (size_t)((max_m + 3) & ~3) * sizeof(T);
  if (smem > 48 * 1024) cudaFuncSetAttribute(k_gemv_loc<T, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k_gemv_loc<T, R><<<n_blocks, kThreads, smem, st>>>(blk_sub, blk_row0, rpc, lay, which, M, vloc, y, done);
}

void launch_gemv_loc(const GemvCfg& cfg, const SubLayout* lay, int which, const void* M, int f32, const void* vloc,
                     double* y, int max_m, const int* done, cudaStream_t st) {
  if (f32) {
    const float* Mf = static_cast<const float*>(M);
    const float* vf = static_cast<const float*>(vloc);
    switch (cfg.R) {
      case 2: launch_gemv_t<float, 2>(cfg.n_blocks, cfg.blk_sub, cfg.blk_row0, cfg.rpc, lay, which, Mf, vf, y, max_m, done, st); break;
      case 4: launch_gemv_t<float, 4>(cfg.n_blocks, cfg.blk_sub, cfg.blk_row0, cfg.rpc, lay, which, Mf, vf, y, max_m, done, st); break;
      default: launch_gemv_t<float, 8>(cfg.n_blocks, cfg.blk_sub, cfg.blk_row0, cfg.rpc, lay, which, Mf, vf, y, max_m, done, st); break;
    }
  } else {
    const double* Md = static_cast<const double*>(M);
    const double* vd = static_cast<const double*>(vloc);
    switch (cfg.R) {
      case 2: launch_gemv_t<double, 2>(cfg.n_blocks, cfg.blk_sub, cfg.blk_row0, cfg.rpc, lay, which, Md, vd, y, max_m, done, st); break;
      case 4: launch_gemv_t<double, 4>(cfg.n_blocks, cfg.blk_sub, cfg.blk_row0, cfg.rpc, lay, which, Md, vd, y, max_m, done, st); break;
      default: launch_gemv_t<double, 8>(cfg.n_blocks, cfg.blk_sub, cfg.blk_row0, cfg.rpc, lay, which, Md, vd, y, max_m, done, st); break;
    }
  }
}

void launch_symv_f32(int G, int n_warps, const int32_t* wsub, const int32_t* wpanel, const SubLayout* lay, int which,
                     const float* Msym, const float* vloc, double* y, float* part, const Maps& mp, const int* done,
                     cudaStream_t st) {
  const int blocks = (n_warps + kThreads / 32 - 1) / (kThreads / 32);
  // G: rows per load group (8, 16, 32); + 100 * PF: L2 prefetch PF tiles ahead (1, 2)
  switch (G) {
    case 8: k_symv_f32<8, 0><<<blocks, kThreads, 0, st>>>(wsub, wpanel, n_warps, lay, which, Msym, vloc, y, part, done); break;
    case 16: k_symv_f32<16, 0><<<blocks, kThreads, 0, st>>>(wsub, wpanel, n_warps, lay, which, Msym, vloc, y, part, done); break;
    case 108: k_symv_f32<8, 1><<<blocks, kThreads, 0, st>>>(wsub, wpanel, n_warps, lay, which, Msym, vloc, y, part, done); break;
    case 132: k_symv_f32<32, 1><<<blocks, kThreads, 0, st>>>(wsub, wpanel, n_warps, lay, which, Msym, vloc, y, part, done); break;
    case 232: k_symv_f32<32, 2><<<blocks, kThreads, 0, st>>>(wsub, wpanel, n_warps, lay, which, Msym, vloc, y, part, done); break;
    default: k_symv_f32<32, 0><<<blocks, kThreads, 0, st>>>(wsub, wpanel, n_warps, lay, which, Msym, vloc, y, part, done); break;
  }
  k_symv_fix<<<grid_for(mp.nb_total), kThreads, 0, st>>>(mp, lay, which, part, y, done);
}

void launch_symv3_f32(int G, int P, const int32_t* order, int max_m, const SubLayout* lay, int which,
                      const float* Msym, const float* vloc, double* y, const int* done, cudaStream_t st) {
  const size_t smem = (size_t)(kThreads / 32 + 1) * (((size_t)max_m + 3) & ~(size_t)3) * sizeof(float);
  static size_t attr[3] = {0, 0, 0};
  const int gi = G == 8 ? 0 : (G == 16 ? 1 : 2);
  if (smem > 48 * 1024 && smem > attr[gi]) {
    if (G == 8) cudaFuncSetAttribute(k_symv3_f32<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    else if (G == 16) cudaFuncSetAttribute(k_symv3_f32<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    else cudaFuncSetAttribute(k_symv3_f32<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    attr[gi] = smem;
  }
  if (G == 8) k_symv3_f32<8><<<P, kThreads, smem, st>>>(order, lay, which, Msym, vloc, y, done);
  else if (G == 16) k_symv3_f32<16><<<P, kThreads, smem, st>>>(order, lay, which, Msym, vloc, y, done);
  else k_symv3_f32<32><<<P, kThreads, smem, st>>>(order, lay, which, Msym, vloc, y, done);
}

void launch_symv2_f32(int n_warps, const int32_t* wsub, const int32_t* wpanel, const SubLayout* lay, int which,
                      const float* Msym, const float* vloc, double* y, float* part, const Maps& mp, const int* done,
                      int* err, const unsigned long long* spin_cycles, cudaStream_t st) {
  const size_t smem = (size_t)SYM_WPC * SYM_NS * SYM_STAGE;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_symv2_f32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    attr = true;
  }
  const int blocks = (n_warps + SYM_WPC - 1) / SYM_WPC;
  k_symv2_f32<<<blocks, SYM_WPC * 32, smem, st>>>(wsub, wpanel, n_warps, lay, which, Msym, vloc, y, part, done, err,
                                                  spin_cycles);
  k_symv_fix<<<grid_for(mp.nb_total), kThreads, 0, st>>>(mp, lay, which, part, y, done);
}

void launch_gather32(const Maps& mp, const double* x, const double* wv, float* y, const int* done, cudaStream_t st) {
  k_gather32<<<grid_for(mp.nb_total), kThreads, 0, st>>>(mp, x, wv, y, done);
}

void launch_vadd(int n, double* a, const double* b, cudaStream_t st) {
  k_vadd<<<grid_for(n), kThreads, 0, st>>>(n, a, b);
}

void launch_gtv_part(int n_chunks, const int32_t* chunk_sub, const int32_t* chunk_p0, const SubLayout* lay,
                     const double* R, const Maps& mp, const double* x, double* partial, const int* done,
                     cudaStream_t st, const double* q, const double* pq_partial, PcgScalars* sc,
                     double* alpha_hist) {
  if (n_chunks <= 0) return;
  k_gtv_part<<<n_chunks, kThreads, 0, st>>>(chunk_sub, chunk_p0, n_chunks, lay, R, mp, x, partial, done, q,
                                            pq_partial, sc, alpha_hist);
}

void launch_expand_update(const Maps& mp, const SubLayout* lay, const double* R, double* r, const double* c,
                          double* out, double* partial, double* lam, const double* p, const double* q,
                          const double* pq_partial, PcgScalars* sc, double* alpha_hist, cudaStream_t st) {
  ExpandUpdate u{r, lam, p, q, pq_partial, sc, alpha_hist};
  k_expand<<<kPartials, kThreads, 0, st>>>(mp, lay, R, r, c, out, nullptr, partial, 1, &sc->done, u);
}

void launch_axpby_rho(int n, double* p, const double* y, PcgScalars* s, const double* partial, double* beta_hist,
                      cudaStream_t st) {
  k_axpby_rho<<<grid_for(n), kThreads, 0, st>>>(n, p, y, s, partial, beta_hist);
}

void launch_coarse_apply_part(int cd, const double* Ginv, const double* partial, const int32_t* sub_chunk_ptr,
                              const int32_t* col_sub, const SubLayout* lay, double* c, const int* done,
                              cudaStream_t st) {
  if (cd <= 0) return;
  const size_t smem = (size_t)cd * sizeof(double);
  if (smem > 48 * 1024)
    cudaFuncSetAttribute(k_coarse_apply_part, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  const int warps = cd < 2432 ? cd : 2432;
  k_coarse_apply_part<<<(warps * 32 + kThreads - 1) / kThreads, kThreads, smem, st>>>(cd, Ginv, partial,
                                                                                        sub_chunk_ptr, col_sub, lay,
                                                                                        c, done);
}

namespace {
// Sum of squares of the assembled global vector sum_i A_i x_i on the listed
// global DOFs (copies summed in a fixed order), per-CTA partials.
__global__ void __launch_bounds__(kThreads) k_global_sumsq(int n, const int32_t* __restrict__ ptr,
                                                           const int32_t* __restrict__ pos,
                                                           const double* __restrict__ x, double* __restrict__ partial) {
  __shared__ double red[32];
  double acc = 0.0;
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < n; g += gridDim.x * blockDim.x) {
    double t = 0.0;
    for (int q = ptr[g]; q < ptr[g + 1]; ++q) t += x[pos[q]];
    acc += t * t;
  }
  acc = block_sum(acc, red);
  if (threadIdx.x == 0) partial[blockIdx.x] = acc;
}

__global__ void k_axpy_to(int n, const double* __restrict__ u, double a, const double* __restrict__ du,
                          double* __restrict__ out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) out[i] = u[i] + a * du[i];
}
}  // namespace

void launch_global_sumsq(int n, const int32_t* ptr, const int32_t* pos, const double* x, double* partial,
                         cudaStream_t st) {
  k_global_sumsq<<<kPartials, kThreads, 0, st>>>(n, ptr, pos, x, partial);
}

namespace {
// Newton-Krylov helpers on the non-Dirichlet global DOFs ("gs space": row j
// lists the local copies gs_pos[gs_ptr[j] .. gs_ptr[j + 1]), lowest
// subdomain first).
__global__ void k_gs_assemble(int n, const int32_t* __restrict__ ptr, const int32_t* __restrict__ pos,
                              const double* __restrict__ xloc, double* __restrict__ y) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
    double t = 0.0;
    for (int q = ptr[j]; q < ptr[j + 1]; ++q) t += xloc[pos[q]];
    y[j] = t;
  }
}
__global__ void k_gs_inject(int n, const int32_t* __restrict__ ptr, const int32_t* __restrict__ pos,
                            const double* __restrict__ r, double* __restrict__ floc) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) floc[pos[ptr[j]]] = r[j];
}
__global__ void k_gs_take(int n, const int32_t* __restrict__ ptr, const int32_t* __restrict__ pos,
                          const double* __restrict__ xloc, double* __restrict__ z) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) z[j] = xloc[pos[ptr[j]]];
}
// y = K v with K the sum of the element tangents Ke (row-major 12x12 per
// element): row j gathers, over its incident (element, local row) pairs
// inc[inc_ptr[j] ..], the 12-term products with v at the element's gs DOFs
// (-1 = Dirichlet, skipped).  Fixed order per row: deterministic.
__global__ void k_gs_elem_matvec(int n, const int32_t* __restrict__ inc_ptr, const int32_t* __restrict__ inc,
                                 const int32_t* __restrict__ elem_gs, const double* __restrict__ Ke,
                                 const double* __restrict__ v, double* __restrict__ y) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
    double t = 0.0;
    for (int q = inc_ptr[j]; q < inc_ptr[j + 1]; ++q) {
      const int ea = inc[q];
      const int e = ea / 12, a = ea % 12;
      const double* K = Ke + (size_t)e * ke_packed(12);
      const int32_t* d = elem_gs + (size_t)e * 12;
#pragma unroll
      for (int b = 0; b < 12; ++b) {
        const int g = d[b];
        if (g >= 0) t += K[ke_idx(12, a, b)] * v[g];
      }
    }
    y[j] = t;
  }
}
__global__ void __launch_bounds__(kThreads) k_gs_dot(int n, const double* __restrict__ a, const double* __restrict__ b,
                                                     double* __restrict__ partial) {
  __shared__ double red[32];
  double acc = 0.0;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) acc += a[j] * b[j];
  acc = block_sum(acc, red);
  if (threadIdx.x == 0) partial[blockIdx.x] = acc;
}
__global__ void k_gs_to_global(int n, const int32_t* __restrict__ gdof, const double* __restrict__ x,
                               double* __restrict__ out) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) out[gdof[j]] = x[j];
}
}  // namespace

void launch_gs_assemble(int n, const int32_t* ptr, const int32_t* pos, const double* xloc, double* y, cudaStream_t st) {
  k_gs_assemble<<<grid_for(n), kThreads, 0, st>>>(n, ptr, pos, xloc, y);
}
void launch_gs_inject(int n, const int32_t* ptr, const int32_t* pos, const double* r, double* floc, cudaStream_t st) {
  k_gs_inject<<<grid_for(n), kThreads, 0, st>>>(n, ptr, pos, r, floc);
}
void launch_gs_take(int n, const int32_t* ptr, const int32_t* pos, const double* xloc, double* z, cudaStream_t st) {
  k_gs_take<<<grid_for(n), kThreads, 0, st>>>(n, ptr, pos, xloc, z);
}
void launch_gs_elem_matvec(int n, const int32_t* inc_ptr, const int32_t* inc, const int32_t* elem_gs, const double* Ke,
                           const double* v, double* y, cudaStream_t st) {
  k_gs_elem_matvec<<<grid_for(n), kThreads, 0, st>>>(n, inc_ptr, inc, elem_gs, Ke, v, y);
}
void launch_gs_dot(int n, const double* a, const double* b, double* partial, cudaStream_t st) {
  k_gs_dot<<<kPartials, kThreads, 0, st>>>(n, a, b, partial);
}
void launch_gs_to_global(int n, const int32_t* gdof, const double* x, double* out, cudaStream_t st) {
  k_gs_to_global<<<grid_for(n), kThreads, 0, st>>>(n, gdof, x, out);
}

void launch_axpy_to(int n, const double* u, double a, const double* du, double* out, cudaStream_t st) {
  k_axpy_to<<<grid_for(n), kThreads, 0, st>>>(n, u, a, du, out);
}

namespace {
__global__ void k_zero_list(int n, const int32_t* __restrict__ idx, double* __restrict__ x) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) x[idx[i]] = 0.0;
}
}  // namespace

void launch_zero_list(int n, const int32_t* idx, double* x, cudaStream_t st) {
  if (n <= 0) return;
  k_zero_list<<<grid_for(n), kThreads, 0, st>>>(n, idx, x);
}

namespace {
// Multi-CTA right-looking Cholesky of one large dense matrix (the coarse
// G^T G, augmented by its identity coupling), lower triangle, row-major:
// per block column a diagonal-block kernel, a panel-solve kernel over row
// chunks and a trailing-update kernel over the lower-triangular 64x64 tiles.
__global__ void k_big_diag(double* __restrict__ A, size_t ld, int kb, int nk, int* status) {
  __shared__ double D[NB][NB + 1];
  __shared__ int bad;
  const int tid = threadIdx.x;
  if (tid == 0) bad = 0;
  for (int idx = tid; idx < NB * NB; idx += blockDim.x) {
    const int i = idx / NB, j = idx % NB;
    D[i][j] = (i < nk && j <= i) ? A[(kb + i) * ld + kb + j] : 0.0;
  }
  __syncthreads();
  if (tid < 32) {
    const int i = tid;
    for (int j = 0; j < nk; ++j) {
      if (i == j) {
        const double d = D[j][j];
        if (!(d > 0.0) || !isfinite(d)) bad = 1;
        D[j][j] = sqrt(d);
      }
      __syncwarp();
      if (bad) break;
      if (i > j && i < nk) D[i][j] /= D[j][j];
      __syncwarp();
      if (i > j && i < nk)
        for (int l = j + 1; l <= i; ++l) D[i][l] -= D[i][j] * D[l][j];
      __syncwarp();
    }
  }
  __syncthreads();
  if (bad) {
    if (tid == 0) set_status(status, DEV_LOCAL_SINGULAR);
    return;
  }
  for (int idx = tid; idx < nk * nk; idx += blockDim.x) {
    const int i = idx / nk, j = idx % nk;
    if (j <= i) A[(kb + i) * ld + kb + j] = D[i][j];
  }
}

__global__ void k_big_trsm(double* __restrict__ A, size_t ld, int kb, int nk, int n_act, const int* status) {
  if (*status) return;
  __shared__ double D[NB][NB + 1];
  __shared__ double Pa[TT][NB + 1];
  const int tid = threadIdx.x;
  for (int idx = tid; idx < NB * NB; idx += blockDim.x) {
    const int i = idx / NB, j = idx % NB;
    D[i][j] = (i < nk && j <= i) ? A[(kb + i) * ld + kb + j] : 0.0;
  }
  const int base = kb + nk + blockIdx.x * TT;
  const int nr = min(TT, n_act - base);
  for (int idx = tid; idx < TT * NB; idx += blockDim.x) {
    const int r = idx / NB, l = idx % NB;
    Pa[r][l] = (r < nr && l < nk) ? A[(base + r) * ld + kb + l] : 0.0;
  }
  __syncthreads();
  if (tid < nr) {
    double xr[NB];
#pragma unroll
    for (int j = 0; j < NB; ++j) xr[j] = Pa[tid][j];
#pragma unroll
    for (int j = 0; j < NB; ++j) {
      if (j < nk) {
        double v = xr[j];
#pragma unroll
        for (int l = 0; l < NB; ++l)
          if (l < j) v -= xr[l] * D[j][l];
        xr[j] = v / D[j][j];
      }
    }
#pragma unroll
    for (int j = 0; j < NB; ++j) Pa[tid][j] = xr[j];
  }
  __syncthreads();
  for (int idx = tid; idx < TT * NB; idx += blockDim.x) {
    const int r = idx / NB, l = idx % NB;
    if (r < nr && l < nk) A[(base + r) * ld + kb + l] = Pa[r][l];
  }
}

__global__ void __launch_bounds__(kThreads) k_big_update(double* __restrict__ A, size_t ld, int kb, int nk,
                                                         int n_act, const int* status) {
  if (*status) return;
  __shared__ double Pa[TT][NB + 1];
  __shared__ double Pb[TT][NB + 1];
  const long b = blockIdx.x;
  // lower-triangular tile index b -> (ti, tj), tj <= ti
  int ti = (int)((sqrt(8.0 * (double)b + 1.0) - 1.0) * 0.5);
  while ((long)(ti + 1) * (ti + 2) / 2 <= b) ++ti;
  while ((long)ti * (ti + 1) / 2 > b) --ti;
  const int tj = (int)(b - (long)ti * (ti + 1) / 2);
  const int r0 = kb + nk;
  const int ib = r0 + ti * TT, jb = r0 + tj * TT;
  const int tid = threadIdx.x;
  for (int idx = tid; idx < TT * NB; idx += blockDim.x) {
    const int r = idx / NB, l = idx % NB;
    Pa[r][l] = (ib + r < n_act && l < nk) ? A[(ib + r) * ld + kb + l] : 0.0;
    Pb[r][l] = (jb + r < n_act && l < nk) ? A[(jb + r) * ld + kb + l] : 0.0;
  }
  __syncthreads();
  const int tr = (tid / 16) * 4, tc = (tid % 16) * 4;
  double acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[a][c] = 0.0;
  for (int l = 0; l < nk; ++l) {
    double av[4], bv[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      av[a] = Pa[tr + a][l];
      bv[a] = Pb[tc + a][l];
    }
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[a][c] += av[a] * bv[c];
  }
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int i = ib + tr + a, j = jb + tc + c;
      if (i < n_act && j < n_act && j <= i) A[i * ld + j] -= acc[a][c];
    }
}
}  // namespace

void launch_dense_chol_big(double* A, int ld, int c0, int c1, int n_act, int aug0, int* status, cudaStream_t st) {
  for (int kb = c0; kb < c1; kb += NB) {
    const int nk = min(NB, c1 - kb);
    k_big_diag<<<1, kThreads, 0, st>>>(A, (size_t)ld, kb, nk, status);
    // augmentation rows of columns not yet eliminated are still zero there
    const int na = aug0 >= 0 ? min(n_act, aug0 + kb + nk - c0) : n_act;
    const int rows = na - (kb + nk);
    if (rows <= 0) continue;
    const int chunks = (rows + TT - 1) / TT;
    k_big_trsm<<<chunks, kThreads, 0, st>>>(A, (size_t)ld, kb, nk, na, status);
    const long tiles = (long)chunks * (chunks + 1) / 2;
    k_big_update<<<(unsigned)tiles, kThreads, 0, st>>>(A, (size_t)ld, kb, nk, na, status);
  }
}

namespace {
// Lumped preconditioner block K_bb in CSR over the boundary positions:
// values gathered from the assembled (unfactorized) local matrices.
template <typename T>
__global__ void k_lump_fill(long nnz, const int64_t* __restrict__ src, const T* __restrict__ A,
                            double* __restrict__ val) {
  for (long j = blockIdx.x * (long)blockDim.x + threadIdx.x; j < nnz; j += (long)gridDim.x * blockDim.x)
    val[j] = A[src[j]];
}

// y = K_bb v on every subdomain's boundary positions, one warp per row.
__global__ void __launch_bounds__(kThreads) k_spmv_lump(int n_rows, const int32_t* __restrict__ ptr,
                                                        const int32_t* __restrict__ col,
                                                        const double* __restrict__ val,
                                                        const double* __restrict__ v, double* __restrict__ y,
                                                        const int* __restrict__ done) {
  if (*done) return;
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int r = warp; r < n_rows; r += nwarps) {
    double acc = 0.0;
    for (int j = ptr[r] + lane; j < ptr[r + 1]; j += 32) acc += val[j] * v[col[j]];
    acc = warp_sum(acc);
    if (lane == 0) y[r] = acc;
  }
}
}  // namespace

void launch_lump_fill(long nnz, const int64_t* src, const double* A, double* val, cudaStream_t st) {
  if (nnz <= 0) return;
  k_lump_fill<double><<<grid_for(nnz), kThreads, 0, st>>>(nnz, src, A, val);
}

void launch_lump_fill(long nnz, const int64_t* src, const float* A, double* val, cudaStream_t st) {
  if (nnz <= 0) return;
  k_lump_fill<float><<<grid_for(nnz), kThreads, 0, st>>>(nnz, src, A, val);
}

void launch_spmv_lump(int n_rows, const int32_t* ptr, const int32_t* col, const double* val, const double* v,
                      double* y, const int* done, cudaStream_t st) {
  const int warps = n_rows < 65536 ? n_rows : 65536;
  k_spmv_lump<<<(warps * 32 + kThreads - 1) / kThreads, kThreads, 0, st>>>(n_rows, ptr, col, val, v, y, done);
}

namespace {
// Batched multi-CTA partial Cholesky: one launch per block-column step for
// all subdomains together (blockIdx.y = subdomain).  Phase 0 eliminates the
// interior columns [0, nI) with trailing rows/cols [.., n); phase 1 the
// boundary columns [nI, nI + nbp) with trailing rows/cols [.., ld).
struct PhaseRange {
  int c0, c1;
};
__device__ __forceinline__ PhaseRange phase_range(const SubLayout& L, int phase) {
  return phase == 0 ? PhaseRange{0, L.nI} : PhaseRange{L.nI, L.nI + L.nbp};
}
// Rows that block column [kb, kb + nk) can change, as an increasing map of
// 0 .. m - 1 onto matrix rows; the rows left out would receive exact zeros.
// Phase 0 (envelope of the interior columns: a row is zero left of the first
// interior column it couples to, and Cholesky fill stays inside that
// envelope): interior rows r0 .. eI - 1, the first nbact boundary rows (the
// boundary DOFs are ordered by envelope start) and the fixing rows, with
// (eI, nbact) per step and subdomain from the host.  Phase 1: rows r0 .. n - 1
// and the augmentation rows of the columns eliminated so far (augmentation
// row n + a starts as the unit row of column nI + a and stays zero left of
// that column until it is eliminated).
struct ActiveRows {
  int r0, lenA, lenB, bbase, cbase, m;
  __device__ __forceinline__ int row(int q) const {
    return q < lenA ? r0 + q : (q < lenA + lenB ? bbase + (q - lenA) : cbase + (q - lenA - lenB));
  }
};
__device__ __forceinline__ ActiveRows active_rows(const SubLayout& L, int phase, int step, int kb, int nk,
                                                  const int32_t* __restrict__ env0) {
  ActiveRows a;
  a.r0 = kb + nk;
  if (phase == 0) {
    const int32_t* ev = env0 + 2 * ((size_t)step * gridDim.y + blockIdx.y);
    const int eI = min(max(ev[0], a.r0), L.nI);
    const int nbact = min(max(ev[1], 0), L.nbp);
    a.lenA = eI - a.r0;
    a.lenB = nbact;
    a.bbase = L.nI;
    a.cbase = L.nI + L.nbp;
    a.m = a.lenA + a.lenB + L.k;
  } else {
    a.lenA = min(L.ld, L.n + a.r0 - L.nI) - a.r0;
    a.lenB = 0;
    a.bbase = a.cbase = a.r0;
    a.m = a.lenA;
  }
  return a;
}

template <typename T, int B>
__global__ void k_bat_diag(const SubLayout* __restrict__ lay, int phase, int step, T* __restrict__ Abase,
                           int* status) {
  const SubLayout L = lay[blockIdx.y];
  const PhaseRange pr = phase_range(L, phase);
  const int kb = pr.c0 + step * B;
  if (kb >= pr.c1) return;
  const int nk = min(B, pr.c1 - kb);
  T* A = Abase + L.aoff;
  const size_t ld = L.ld;
  __shared__ T D[B][B + 1];
  __shared__ int bad;
  const int tid = threadIdx.x;
  if (tid == 0) bad = 0;
  for (int idx = tid; idx < B * B; idx += blockDim.x) {
    const int i = idx / B, j = idx % B;
    D[i][j] = (i < nk && j <= i) ? A[(kb + i) * ld + kb + j] : (T)0;
  }
  __syncthreads();
  if (B == 32) {
    if (tid < 32) {
      const int i = tid;
      for (int j = 0; j < nk; ++j) {
        if (i == j) {
          const T d = D[j][j];
          if (!(d > 0.0) || !isfinite(d)) bad = 1;
          D[j][j] = sqrt(d);
        }
        __syncwarp();
        if (bad) break;
        if (i > j && i < nk) D[i][j] /= D[j][j];
        __syncwarp();
        if (i > j && i < nk)
          for (int l = j + 1; l <= i; ++l) D[i][l] -= D[i][j] * D[l][j];
        __syncwarp();
      }
    }
  } else {
    // wider blocks: row i by thread i, every thread through the block barriers
    const int i = tid;
    for (int j = 0; j < nk; ++j) {
      if (i == j) {
        const T d = D[j][j];
        if (!(d > 0.0) || !isfinite(d)) bad = 1;
        D[j][j] = sqrt(d);
      }
      __syncthreads();
      if (bad) break;
      if (i > j && i < nk) D[i][j] /= D[j][j];
      __syncthreads();
      if (i > j && i < nk)
        for (int l = j + 1; l <= i; ++l) D[i][l] -= D[i][j] * D[l][j];
      __syncthreads();
    }
  }
  __syncthreads();
  if (bad) {
    if (tid == 0) set_status(status, DEV_LOCAL_SINGULAR);
    return;
  }
  for (int idx = tid; idx < nk * nk; idx += blockDim.x) {
    const int i = idx / nk, j = idx % nk;
    if (j <= i) A[(kb + i) * ld + kb + j] = D[i][j];
  }
}

template <typename T, int B>
__global__ void k_bat_trsm(const SubLayout* __restrict__ lay, int phase, int step,
                           const int32_t* __restrict__ env0, T* __restrict__ Abase, const int* status) {
  if (*status) return;
  const SubLayout L = lay[blockIdx.y];
  const PhaseRange pr = phase_range(L, phase);
  const int kb = pr.c0 + step * B;
  if (kb >= pr.c1) return;
  const int nk = min(B, pr.c1 - kb);
  const ActiveRows ar = active_rows(L, phase, step, kb, nk, env0);
  const int q0 = blockIdx.x * TT;
  if (q0 >= ar.m) return;
  const int nr = min(TT, ar.m - q0);
  T* A = Abase + L.aoff;
  const size_t ld = L.ld;
  __shared__ T D[B][B + 1];
  __shared__ T Pa[TT][B + 1];
  const int tid = threadIdx.x;
  for (int idx = tid; idx < B * B; idx += blockDim.x) {
    const int i = idx / B, j = idx % B;
    D[i][j] = (i < nk && j <= i) ? A[(kb + i) * ld + kb + j] : (T)0;
  }
  for (int idx = tid; idx < TT * B; idx += blockDim.x) {
    const int r = idx / B, l = idx % B;
    Pa[r][l] = (r < nr && l < nk) ? A[(size_t)ar.row(q0 + r) * ld + kb + l] : (T)0;
  }
  __syncthreads();
  if (tid < nr) {
    T xr[B];
#pragma unroll
    for (int j = 0; j < B; ++j) xr[j] = Pa[tid][j];
#pragma unroll
    for (int j = 0; j < B; ++j) {
      if (j < nk) {
        T v = xr[j];
#pragma unroll
        for (int l = 0; l < B; ++l)
          if (l < j) v -= xr[l] * D[j][l];
        xr[j] = v / D[j][j];
      }
    }
#pragma unroll
    for (int j = 0; j < B; ++j) Pa[tid][j] = xr[j];
  }
  __syncthreads();
  for (int idx = tid; idx < TT * B; idx += blockDim.x) {
    const int r = idx / B, l = idx % B;
    if (r < nr && l < nk) A[(size_t)ar.row(q0 + r) * ld + kb + l] = Pa[r][l];
  }
}

template <typename T, int B>
__global__ void __launch_bounds__(kThreads) k_bat_update(const SubLayout* __restrict__ lay, int phase, int step,
                                                         const int32_t* __restrict__ env0,
                                                         T* __restrict__ Abase, const int* status) {
  if (*status) return;
  const SubLayout L = lay[blockIdx.y];
  const PhaseRange pr = phase_range(L, phase);
  const int kb = pr.c0 + step * B;
  if (kb >= pr.c1) return;
  const int nk = min(B, pr.c1 - kb);
  const ActiveRows ar = active_rows(L, phase, step, kb, nk, env0);
  const int m = ar.m;
  const int chunks = (m + TT - 1) / TT;
  const long b = blockIdx.x;
  if (b >= (long)chunks * (chunks + 1) / 2) return;
  int ti = (int)((sqrt(8.0 * (double)b + 1.0) - 1.0) * 0.5);
  while ((long)(ti + 1) * (ti + 2) / 2 <= b) ++ti;
  while ((long)ti * (ti + 1) / 2 > b) --ti;
  const int tj = (int)(b - (long)ti * (ti + 1) / 2);
  const int ib = ti * TT, jb = tj * TT;  // positions in the active-row list
  T* A = Abase + L.aoff;
  const size_t ld = L.ld;
  __shared__ T Pa[TT][B + 1];
  __shared__ T Pb[TT][B + 1];
  const int tid = threadIdx.x;
  for (int idx = tid; idx < TT * B; idx += blockDim.x) {
    const int r = idx / B, l = idx % B;
    Pa[r][l] = (ib + r < m && l < nk) ? A[(size_t)ar.row(ib + r) * ld + kb + l] : (T)0;
    Pb[r][l] = (jb + r < m && l < nk) ? A[(size_t)ar.row(jb + r) * ld + kb + l] : (T)0;
  }
  __syncthreads();
  const int tr = (tid / 16) * 4, tc = (tid % 16) * 4;
  T acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[a][c] = (T)0;
  for (int l = 0; l < nk; ++l) {
    T av[4], bv[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      av[a] = Pa[tr + a][l];
      bv[a] = Pb[tc + a][l];
    }
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[a][c] += av[a] * bv[c];
  }
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int qi = ib + tr + a, qj = jb + tc + c;  // increasing map: qj <= qi <=> j <= i
      if (qi < m && qj < m && qj <= qi) A[(size_t)ar.row(qi) * ld + ar.row(qj)] -= acc[a][c];
    }
}
}  // namespace

template <typename T, int B>
void chol_batched(int P, const SubLayout* lay, int phase, const int* step_chunks, int n_steps,
                  const int32_t* env0, T* A, int* status, cudaStream_t st) {
  for (int t = 0; t < n_steps; ++t) {
    const int chunks = step_chunks[t];
    k_bat_diag<T, B><<<dim3(1, P), kThreads, 0, st>>>(lay, phase, t, A, status);
    if (chunks <= 0) continue;
    k_bat_trsm<T, B><<<dim3(chunks, P), kThreads, 0, st>>>(lay, phase, t, env0, A, status);
    const long tiles = (long)chunks * (chunks + 1) / 2;
    k_bat_update<T, B><<<dim3((unsigned)tiles, P), kThreads, 0, st>>>(lay, phase, t, env0, A, status);
  }
}

void launch_chol_batched(int P, const SubLayout* lay, int phase, const int* step_chunks, int n_steps,
                         const int32_t* env0, double* A, int* status, cudaStream_t st) {
  chol_batched<double, 32>(P, lay, phase, step_chunks, n_steps, env0, A, status, st);
}

void launch_chol_batched(int P, const SubLayout* lay, int phase, const int* step_chunks, int n_steps,
                         const int32_t* env0, float* A, int* status, cudaStream_t st) {
  chol_batched<float, kChol32Block>(P, lay, phase, step_chunks, n_steps, env0, A, status, st);
}

namespace {
__global__ void k_ke_unpack(long n, int nde, const double* __restrict__ Kp, double* __restrict__ K) {
  const int kes = nde * nde;
  for (long x = blockIdx.x * (long)blockDim.x + threadIdx.x; x < n; x += (long)gridDim.x * blockDim.x) {
    const long e = x / kes;
    const int t = (int)(x - e * kes);
    K[x] = Kp[e * ke_packed(nde) + ke_idx(nde, t / nde, t % nde)];
  }
}
}  // namespace

void launch_ke_unpack(int n_el, int nde, const double* Kp, double* K, cudaStream_t st) {
  const long n = (long)n_el * nde * nde;
  if (n <= 0) return;
  long b = (n + kThreads - 1) / kThreads;
  if (b > 65535) b = 65535;
  k_ke_unpack<<<(int)b, kThreads, 0, st>>>(n, nde, Kp, K);
}

}  // namespace feti
