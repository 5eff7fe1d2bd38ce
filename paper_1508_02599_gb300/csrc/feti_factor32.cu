// FP32 local factorizations with FP64 iterative refinement of K^+.
//
// In the FETI_MIXED_F32FACTOR form the dense local elimination of Sec. 4.3 /
// 4.4 (K_rr = L L^T with the interior columns first, the Schur complement S_i
// as its trailing block, F_i = (S_i[b',b'])^-1 through an identity
// augmentation) runs in FP32 (the batched Cholesky kernels instantiated for
// float).  The FP32 explicit operators F_i and S_i drive the inner PCG as in
// the mixed form; every FP64-accurate use of the generalized inverse (the
// dual right-hand side d~, the outer dual residual, the recovery of u_i)
// goes through K^+ refined in FP64 (classical mixed-precision iterative
// refinement, Moler 1967):
//   x = L^-T L^-1 g (FP32);  repeat: r = g - K_rr x (FP64, from the element
//   matrices);  x += L^-T L^-1 r,
// with zero on the fixing DOFs, which is K^+ g of the fixing-DOF generalized
// inverse of Sec. 5.2 ("regularization by fixing nodes").  Each FP32
// correction sweeps only the interior block of L and reaches the boundary
// block through the explicit F_i (k_kp_fwd_* / k_kp_bwd_*); the FP64
// residual is an element pass and a row pass (k_elem_kx / k_row_resid).
#include "feti_internal.h"

#include <algorithm>

namespace feti {
namespace {

constexpr int kT = 256;

// The dense local operators out of the eliminated workspace in one pass, one
// CTA per 32 x 32 output tile (I, J) of one subdomain: the source tile
// (max(I,J), min(I,J)) of the workspace's lower triangle is read row by row
// into shared memory and written transposed or not into each requested
// layout: FP64 row-major (out64, stride m), the FP32 copy with rows padded to
// 4 (out32), and for J <= I the FP32 32-row lower panels of the symmetric
// apply (sym32; zero beyond the matrix).  which 0: the preconditioner block
// S_i (m = n_b' + k), which 1: F_i = minus the eliminated augmentation block
// (m = n_b').
template <typename TS>
__global__ void __launch_bounds__(256) k_extract_tiles(const SubLayout* __restrict__ lay, int which,
                                                       const TS* __restrict__ Abase, double* __restrict__ out64,
                                                       float* __restrict__ out32, float* __restrict__ sym32) {
  const SubLayout L = lay[blockIdx.y];
  const int m = which == 0 ? L.nbp + L.k : L.nbp;
  const int nT = (m + 31) / 32;
  const int I = blockIdx.x / nT, J = blockIdx.x - (blockIdx.x / nT) * nT;
  if (I >= nT) return;
  const size_t ld = L.ld;
  const int base = which == 0 ? L.nI : L.n;
  const TS sgn = which == 0 ? (TS)1 : (TS)-1;
  const TS* A = Abase + L.aoff + (size_t)base * ld + base;
  __shared__ TS T[32][33];
  const int Ts = max(I, J), Tc = min(I, J);
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 8 rows per pass
  for (int r = ty; r < 32; r += 8) {
    const int gr = 32 * Ts + r, gc = 32 * Tc + tx;
    // lower triangle only (the diagonal tile's upper half is filled by symmetry)
    T[r][tx] = (gr < m && gc < m && gc <= gr) ? A[(size_t)gr * ld + gc] : (TS)0;
  }
  __syncthreads();
  const int ldo = (m + 3) & ~3;
  double* o64 = out64 ? out64 + (which == 0 ? L.soff : L.foff) : nullptr;
  float* o32 = out32 ? out32 + (which == 0 ? L.soff32 : L.foff32) : nullptr;
  float* sp = sym32 ? sym32 + (which == 0 ? L.ssym32 : L.fsym32) + (size_t)512 * I * (I + 1) : nullptr;
  const int w = 32 * (I + 1);
  for (int r = ty; r < 32; r += 8) {
    const int gr = 32 * I + r, gc = 32 * J + tx;
    TS v;
    if (I > J) v = T[r][tx];
    else if (I < J) v = T[tx][r];
    else v = tx <= r ? T[r][tx] : T[tx][r];
    v *= sgn;
    if (o64 && gr < m && gc < m) o64[(size_t)gr * m + gc] = (double)v;
    if (o32 && gr < m && gc < ldo) o32[(size_t)gr * ldo + gc] = gc < m ? (float)v : 0.0f;
    if (sp && J <= I) sp[(size_t)r * w + 32 * J + tx] = (gr < m && gc < m) ? (float)v : 0.0f;
  }
}

// One FP32 correction x (+)= L^-T L^-1 r on the rows [0, n_I + n_b'), with
// the triangular sweeps confined to the interior: with K_rr = L L^T and L = [[L_II, 0], [L_bI, L_bb]] (interior rows first,
// then the boundary rows b' that are not fixing DOFs),
//   y_I = L_II^-1 r_I,   z_b = r_b - L_bI y_I,   x_b = (L_bb L_bb^T)^-1 z_b = F_i z_b,
//   x_I = L_II^-T (y_I - L_bI^T x_b),
// and F_i = S_i[b',b']^-1 is the explicit FP32 operator the PCG already
// applies.  The dependent 32-row block chains shrink from n_I + n_b' rows to
// n_I rows; the boundary panel products carry no chain.
// The sweeps in four kernels: the two triangular chains over L_II run one
// CTA per subdomain (k_kp_fwd_interior, k_kp_bwd_interior: 32-row blocks one
// after another), and the two products with L_bI, which carry no chain and
// hold most of the factor's bytes, run many CTAs per subdomain
// (k_kp_fwd_boundary: 32 boundary rows per CTA; k_kp_bwd_boundary: 32
// interior columns per CTA).  T is the factor's precision; every kernel reads
// the compact interior factor (rows [0, n_I + n_b') x columns [0, n_I) at
// L.loff, row stride kp_ld).
template <typename T>
__device__ __forceinline__ T kp_warp_sum(T v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Diagonal block [I0, I0 + 32) of L_II (lower triangle, zero elsewhere) into D.
template <typename T>
__device__ __forceinline__ void kp_load_diag(const T* __restrict__ A, size_t ld, int nI, int I0, T (*D)[33]) {
  const int nb = min(32, nI - I0);
  for (int idx = threadIdx.x; idx < 32 * 32; idx += kT) {
    const int rr = idx >> 5, c = idx & 31;
    D[rr][c] = (rr < nb && c <= rr) ? A[(size_t)(I0 + rr) * ld + I0 + c] : (T)0;
  }
}

// ys[i] -= L[i, I0 : I0 + 32] . xs for the rows i in [i0, nI), a thread per
// row, the 32 entries read as 16-byte vectors (rows and I0 are multiples of 4
// elements apart from an aligned base).
__device__ __forceinline__ void kp_row_update(const float* __restrict__ A, size_t ld, int I0, int i0, int nI,
                                              const float* xs, float* ys) {
  // two halves of 16 entries: the FP32 sweeps run 8 CTAs of 256 threads per
  // SM (one wave over a thousand subdomains), 32 registers a thread
  for (int i = i0 + threadIdx.x; i < nI; i += kT) {
    const float4* row = reinterpret_cast<const float4*>(A + (size_t)i * ld + I0);
    float acc = 0.0f;
#pragma unroll 1
    for (int h = 0; h < 2; ++h) {
      float4 a[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) a[u] = __ldg(row + 4 * h + u);
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const float* xv = xs + 16 * h + 4 * u;
        acc += a[u].x * xv[0] + a[u].y * xv[1] + a[u].z * xv[2] + a[u].w * xv[3];
      }
    }
    ys[i] -= acc;
  }
}
__device__ __forceinline__ void kp_row_update(const double* __restrict__ A, size_t ld, int I0, int i0, int nI,
                                              const double* xs, double* ys) {
  for (int i = i0 + threadIdx.x; i < nI; i += kT) {
    const double2* row = reinterpret_cast<const double2*>(A + (size_t)i * ld + I0);
    double2 a[16];
#pragma unroll
    for (int u = 0; u < 16; ++u) a[u] = __ldg(row + u);
    double acc = 0.0;
#pragma unroll
    for (int u = 0; u < 16; ++u) acc += a[u].x * xs[2 * u] + a[u].y * xs[2 * u + 1];
    ys[i] -= acc;
  }
}

// y_I = L_II^-1 r_I (into yI at the subdomain's local offset), right-looking
// by 32-column blocks: warp 0 solves the diagonal block, then every thread
// updates the rows below it with the block's 32 solved values while the next
// diagonal block is fetched into the other buffer.
template <typename T>
__global__ void __launch_bounds__(kT, sizeof(T) == 4 ? 8 : 4)
    k_kp_fwd_interior(const SubLayout* __restrict__ lay, const T* __restrict__ Lbase, const double* __restrict__ rbase,
                      T* __restrict__ yIbase) {
  extern __shared__ __align__(16) unsigned char kp_smem[];
  T* ys = reinterpret_cast<T*>(kp_smem);
  const SubLayout L = lay[blockIdx.x];
  const T* A = Lbase + L.loff;
  const size_t ld = kp_ld(L);
  const double* r = rbase + L.voff;
  const int nI = L.nI;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  __shared__ T Db[2][32][33];
  __shared__ __align__(16) T xs[32];
  for (int i = tid; i < nI; i += kT) ys[i] = (T)r[i];
  if (nI > 0) kp_load_diag(A, ld, nI, 0, Db[0]);
  __syncthreads();
  for (int I0 = 0, k = 0; I0 < nI; I0 += 32, ++k) {
    const int nb = min(32, nI - I0);
    T (*D)[33] = Db[k & 1];
    if (warp == 0) {
      T b = lane < nb ? ys[I0 + lane] : (T)0;
      T xv = 0;
      for (int c = 0; c < nb; ++c) {
        if (lane == c) xv = b / D[c][c];
        const T xc = __shfl_sync(0xffffffffu, xv, c);
        if (lane > c) b -= D[lane][c] * xc;
      }
      if (lane < nb) ys[I0 + lane] = xv;
      xs[lane] = lane < nb ? xv : (T)0;
    }
    __syncthreads();
    const int I1 = I0 + 32;
    if (I1 < nI) {  // then nb == 32
      kp_load_diag(A, ld, nI, I1, Db[(k + 1) & 1]);
      kp_row_update(A, ld, I0, I1, nI, xs, ys);
    }
    __syncthreads();
  }
  T* yI = yIbase + L.voff;
  for (int i = tid; i < nI; i += kT) yI[i] = ys[i];
}

// z_b = r_b - L_bI y_I for 32 boundary rows per CTA (grid.x over row blocks,
// grid.y over subdomains; warp w takes rows w, w + 8, w + 16, w + 24 of the
// block, four column strides at a time); the CTA with block 0 also zeros z on
// the fixing positions.
template <typename T>
__global__ void __launch_bounds__(kT, sizeof(T) == 4 ? 8 : 4)
    k_kp_fwd_boundary(const SubLayout* __restrict__ lay, const T* __restrict__ Lbase, const double* __restrict__ rbase,
                      const T* __restrict__ yIbase, T* __restrict__ zb) {
  extern __shared__ __align__(16) unsigned char kp_smem[];
  T* ys = reinterpret_cast<T*>(kp_smem);
  const SubLayout L = lay[blockIdx.y];
  const int nI = L.nI, nbp = L.nbp;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int kW = kT / 32;
  if (blockIdx.x == 0)
    for (int p = nbp + tid; p < nbp + L.k; p += kT) zb[L.boff + p] = (T)0;
  const int p0 = blockIdx.x * 32;
  if (p0 >= nbp) return;
  const T* yI = yIbase + L.voff;
  for (int i = tid; i < nI; i += kT) ys[i] = yI[i];
  __syncthreads();
  const size_t ld = kp_ld(L);
  const T* rp = Lbase + L.loff + (size_t)(nI + p0) * ld;
  const double* r = rbase + L.voff;
  int ro[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) ro[q] = min(warp + kW * q, nbp - 1 - p0) * (int)ld;
  T acc[4] = {0, 0, 0, 0};
  int j = lane;
  for (; j + 96 < nI; j += 128) {
    T a[4][4];
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int u = 0; u < 4; ++u) a[q][u] = __ldg(rp + ro[q] + j + 32 * u);
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const T yv = ys[j + 32 * u];
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[q] += a[q][u] * yv;
    }
  }
  for (; j < nI; j += 32) {
    const T yv = ys[j];
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[q] += __ldg(rp + ro[q] + j) * yv;
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const T v = kp_warp_sum(acc[q]);
    const int p = p0 + warp + kW * q;
    if (lane == 0 && p < min(nbp, p0 + 32)) zb[L.boff + p] = (T)(r[nI + p] - (double)v);
  }
}

// t_I = y_I - L_bI^T x_b in place in yI, 32 interior columns per CTA: lane =
// column, warp w = boundary rows w, w + 8, ..., eight rows in flight per
// thread, the eight warps' partial sums added in a fixed order.
template <typename T>
__global__ void __launch_bounds__(kT, sizeof(T) == 4 ? 8 : 4)
    k_kp_bwd_boundary(const SubLayout* __restrict__ lay, const T* __restrict__ Lbase, const double* __restrict__ xb,
                      T* __restrict__ yIbase) {
  extern __shared__ __align__(16) unsigned char kp_smem[];
  T* xbs = reinterpret_cast<T*>(kp_smem);
  const SubLayout L = lay[blockIdx.y];
  const int nI = L.nI, nbp = L.nbp;
  const int c0 = blockIdx.x * 32;
  if (c0 >= nI) return;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int kW = kT / 32;
  __shared__ T part[kW][32];
  for (int p = tid; p < nbp; p += kT) xbs[p] = (T)xb[L.boff + p];
  __syncthreads();
  const size_t ld = kp_ld(L);
  const int c = c0 + lane;
  const T* col = Lbase + L.loff + (size_t)nI * ld + min(c, nI - 1);
  T acc = 0;
  int p = warp;
  for (; p + 7 * kW < nbp; p += 8 * kW) {
    T a[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) a[u] = __ldg(col + (size_t)(p + kW * u) * ld);
#pragma unroll
    for (int u = 0; u < 8; ++u) acc += a[u] * xbs[p + kW * u];
  }
  for (; p < nbp; p += kW) acc += __ldg(col + (size_t)p * ld) * xbs[p];
  part[warp][lane] = acc;
  __syncthreads();
  if (warp == 0 && c < nI) {
    T s = part[0][lane];
#pragma unroll
    for (int w = 1; w < kW; ++w) s += part[w][lane];
    T* yI = yIbase + L.voff;
    yI[c] -= s;
  }
}

// x_I = L_II^-T t_I (t_I in yI after k_kp_bwd_boundary), by 32-column
// blocks from the last: warp 0 solves the transposed diagonal block, then a
// thread per column j below the block's start subtracts L[I0 : I0 + 32, j]^T
// times the block's solved values (32 loads in flight per thread) while the
// previous diagonal block is fetched into the other buffer; then x (+)= x on
// rows [0, n_I + n_b') (x_b from the F_i apply, FP64 at the boundary offset),
// and with init x = that correction, zero on the fixing rows.
template <typename T>
__global__ void __launch_bounds__(kT, sizeof(T) == 4 ? 8 : 4)
    k_kp_bwd_interior(const SubLayout* __restrict__ lay, const T* __restrict__ Lbase, const T* __restrict__ yIbase,
                      const double* __restrict__ xb, double* __restrict__ xbase, int init) {
  extern __shared__ __align__(16) unsigned char kp_smem[];
  T* ys = reinterpret_cast<T*>(kp_smem);
  const SubLayout L = lay[blockIdx.x];
  const T* A = Lbase + L.loff;
  const size_t ld = kp_ld(L);
  double* x = xbase + L.voff;
  const int nI = L.nI, nbp = L.nbp;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  __shared__ T Db[2][32][33];
  __shared__ T xs[32];
  const T* yI = yIbase + L.voff;
  for (int i = tid; i < nI; i += kT) ys[i] = yI[i];
  const int Ilast = nI > 0 ? ((nI - 1) / 32) * 32 : -32;
  if (Ilast >= 0) kp_load_diag(A, ld, nI, Ilast, Db[0]);
  __syncthreads();
  for (int I0 = Ilast, k = 0; I0 >= 0; I0 -= 32, ++k) {
    const int nb = min(32, nI - I0);
    T (*D)[33] = Db[k & 1];
    if (warp == 0) {
      T b = lane < nb ? ys[I0 + lane] : (T)0;
      T xv = 0;
      for (int c = nb - 1; c >= 0; --c) {
        if (lane == c) xv = b / D[c][c];
        const T xc = __shfl_sync(0xffffffffu, xv, c);
        if (lane < c) b -= D[c][lane] * xc;
      }
      if (lane < nb) ys[I0 + lane] = xv;
      xs[lane] = lane < nb ? xv : (T)0;
    }
    __syncthreads();
    if (I0 > 0) {
      kp_load_diag(A, ld, nI, I0 - 32, Db[(k + 1) & 1]);
      const T* blk = A + (size_t)I0 * ld;
      for (int j = tid; j < I0; j += kT) {
        T acc = 0;
#pragma unroll 1
        for (int h = 0; h < 2; ++h) {
          T a[16];
#pragma unroll
          for (int u = 0; u < 16; ++u) {
            const int rr = 16 * h + u;
            a[u] = rr < nb ? __ldg(blk + (size_t)rr * ld + j) : (T)0;
          }
#pragma unroll
          for (int u = 0; u < 16; ++u) acc += a[u] * xs[16 * h + u];
        }
        ys[j] -= acc;
      }
    }
    __syncthreads();
  }
  for (int i = tid; i < nI; i += kT) x[i] = (init ? 0.0 : x[i]) + (double)ys[i];
  for (int p = tid; p < nbp; p += kT) x[nI + p] = (init ? 0.0 : x[nI + p]) + xb[L.boff + p];
  if (init)
    for (int i = nI + nbp + tid; i < L.n; i += kT) x[i] = 0.0;
}

// Compact interior factor: one CTA per 32 rows of one subdomain, a warp per
// row, lanes along the columns (coalesced on both sides).
template <typename T>
__global__ void __launch_bounds__(256) k_compact_factor(const SubLayout* __restrict__ lay, const T* __restrict__ Abase,
                                                        T* __restrict__ Lbase) {
  const SubLayout L = lay[blockIdx.y];
  const int rows = L.nI + L.nbp;
  const int r0 = blockIdx.x * 32;
  if (r0 >= rows) return;
  const int ldo = kp_ld(L);
  const size_t ld = L.ld;
  const T* A = Abase + L.aoff;
  T* out = Lbase + L.loff;
  for (int r = r0 + (threadIdx.x >> 5); r < min(r0 + 32, rows); r += 8) {
    const int cmax = r < L.nI ? r : L.nI - 1;  // L_II lower triangle, L_bI whole rows
    for (int c = threadIdx.x & 31; c < ldo; c += 32)
      out[(size_t)r * ldo + c] = c <= cmax ? A[(size_t)r * ld + c] : (T)0;
  }
}

// r = g - K_rr x in FP64 on the rows [0, n_I + n_b') (zero on the fixing
// rows), in two deterministic passes: ye[nde e + a] = (K_e x_e)_a
// for every element (its dense map and the local vector of its subdomain,
// columns of eliminated DOFs skipped), then per local row r = g - the sum of
// its (element, row) entries in the order of its incidence list.
template <int NDE>
__global__ void __launch_bounds__(128) k_elem_kx(int n_el, const int32_t* __restrict__ elem_sub,
                                                 const SubLayout* __restrict__ lay,
                                                 const int32_t* __restrict__ elem_dense, const double* __restrict__ Ke,
                                                 const double* __restrict__ xbase, double* __restrict__ ye) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n_el) return;
  const double* x = xbase + lay[elem_sub[e]].voff;
  const int32_t* dm = elem_dense + (size_t)NDE * e;
  const double* ke = Ke + (size_t)e * ke_packed(NDE);
  double xe[NDE];
#pragma unroll
  for (int b = 0; b < NDE; ++b) {
    const int c = dm[b];
    xe[b] = c >= 0 ? x[c] : 0.0;
  }
#pragma unroll
  for (int a = 0; a < NDE; ++a) {
    double t = 0.0;
#pragma unroll
    for (int b = 0; b < NDE; ++b) t += ke[ke_idx(NDE, a, b)] * xe[b];
    ye[(size_t)NDE * e + a] = t;
  }
}

__global__ void k_row_resid(int n, const int32_t* __restrict__ row_sub, const SubLayout* __restrict__ lay,
                            const int32_t* __restrict__ kinc_ptr, const int32_t* __restrict__ kinc,
                            const double* __restrict__ ye, const double* __restrict__ g, double* __restrict__ r) {
  for (int gi = blockIdx.x * blockDim.x + threadIdx.x; gi < n; gi += gridDim.x * blockDim.x) {
    const SubLayout L = lay[row_sub[gi]];
    double acc = 0.0;
    if (gi - L.voff < L.nI + L.nbp) {
      acc = g[gi];
      const int q1 = kinc_ptr[gi + 1];
      int q = kinc_ptr[gi];
      for (; q + 4 <= q1; q += 4) {
        const int e0 = kinc[q], e1 = kinc[q + 1], e2 = kinc[q + 2], e3 = kinc[q + 3];
        const double v0 = ye[e0], v1 = ye[e1], v2 = ye[e2], v3 = ye[e3];
        acc -= v0;
        acc -= v1;
        acc -= v2;
        acc -= v3;
      }
      for (; q < q1; ++q) acc -= ye[kinc[q]];
    }
    r[gi] = acc;
  }
}

// out (full local vectors) = the boundary vector loc at the boundary
// positions [nI, n), zero on the interior.
__global__ void k_place(const SubLayout* __restrict__ lay, const double* __restrict__ loc, double* __restrict__ out,
                        const int* __restrict__ done) {
  if (done && *done) return;
  const SubLayout L = lay[blockIdx.x];
  for (int i = threadIdx.x; i < L.n; i += blockDim.x)
    out[L.voff + i] = i < L.nI ? 0.0 : loc[L.boff + i - L.nI];
}

// Per subdomain: out[2 s] = sum of r_i^2, out[2 s + 1] = sum of g_i^2 over [0, nr).
__global__ void k_sub_norm2(const SubLayout* __restrict__ lay, const double* __restrict__ r,
                            const double* __restrict__ g, double* __restrict__ out) {
  const SubLayout L = lay[blockIdx.x];
  const int nr = L.nI + L.nbp;
  __shared__ double sr[kT / 32], sg[kT / 32];
  double a = 0.0, b = 0.0;
  for (int i = threadIdx.x; i < nr; i += kT) {
    a += r[L.voff + i] * r[L.voff + i];
    b += g[L.voff + i] * g[L.voff + i];
  }
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
  if ((threadIdx.x & 31) == 0) {
    sr[threadIdx.x >> 5] = a;
    sg[threadIdx.x >> 5] = b;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double ta = 0.0, tb = 0.0;
    for (int w = 0; w < kT / 32; ++w) {
      ta += sr[w];
      tb += sg[w];
    }
    out[2 * blockIdx.x] = ta;
    out[2 * blockIdx.x + 1] = tb;
  }
}

// Deterministic test vector in [-1, 1) from a 64-bit mix of the index
// (splitmix64 finaliser).
__global__ void k_fill_mix(long n, double* __restrict__ x) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    unsigned long long z = (unsigned long long)i + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    x[i] = (double)(z >> 11) * (2.0 / 9007199254740992.0) - 1.0;
  }
}

}  // namespace

void launch_extract_tiles(int P, int max_m, const SubLayout* lay, int which, const float* A, double* out64, float* out32,
                          float* sym32, cudaStream_t st) {
  const int nT = (max_m + 31) / 32;
  if (P > 0 && nT > 0) k_extract_tiles<float><<<dim3(nT * nT, P), 256, 0, st>>>(lay, which, A, out64, out32, sym32);
}

void launch_extract_tiles(int P, int max_m, const SubLayout* lay, int which, const double* A, double* out64,
                          float* out32, float* sym32, cudaStream_t st) {
  const int nT = (max_m + 31) / 32;
  if (P > 0 && nT > 0) k_extract_tiles<double><<<dim3(nT * nT, P), 256, 0, st>>>(lay, which, A, out64, out32, sym32);
}

template <typename K>
void kp_smem_attr(K kern, size_t smem) {
  if (smem > 48 * 1024) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

template <typename T>
void kp_forward(int P, const SubLayout* lay, const T* Lc, const double* r, T* yI, T* zb, int max_nr, cudaStream_t st) {
  if (P <= 0) return;
  const size_t smem = (size_t)std::max(max_nr, 1) * sizeof(T);
  kp_smem_attr(k_kp_fwd_interior<T>, smem);
  kp_smem_attr(k_kp_fwd_boundary<T>, smem);
  k_kp_fwd_interior<T><<<P, kT, smem, st>>>(lay, Lc, r, yI);
  const int nblk = std::max(1, (max_nr + 31) / 32);
  k_kp_fwd_boundary<T><<<dim3(nblk, P), kT, smem, st>>>(lay, Lc, r, yI, zb);
}

template <typename T>
void kp_backward(int P, const SubLayout* lay, const T* Lc, T* yI, const double* xb, double* x, int init,
                 int max_nr, cudaStream_t st) {
  if (P <= 0) return;
  const size_t smem = (size_t)std::max(max_nr, 1) * sizeof(T);
  kp_smem_attr(k_kp_bwd_boundary<T>, smem);
  kp_smem_attr(k_kp_bwd_interior<T>, smem);
  const int nblk = std::max(1, (max_nr + 31) / 32);
  k_kp_bwd_boundary<T><<<dim3(nblk, P), kT, smem, st>>>(lay, Lc, xb, yI);
  k_kp_bwd_interior<T><<<P, kT, smem, st>>>(lay, Lc, yI, xb, x, init);
}

void launch_kp_forward(int P, const SubLayout* lay, const float* Lc, const double* r, float* yI, float* zb, int max_nr,
                       cudaStream_t st) {
  kp_forward<float>(P, lay, Lc, r, yI, zb, max_nr, st);
}

void launch_kp_backward(int P, const SubLayout* lay, const float* Lc, float* yI, const double* xb, double* x,
                        int init, int max_nr, cudaStream_t st) {
  kp_backward<float>(P, lay, Lc, yI, xb, x, init, max_nr, st);
}

void launch_kp_forward(int P, const SubLayout* lay, const double* Lc, const double* r, double* yI, double* zb,
                       int max_nr, cudaStream_t st) {
  kp_forward<double>(P, lay, Lc, r, yI, zb, max_nr, st);
}

void launch_kp_backward(int P, const SubLayout* lay, const double* Lc, double* yI, const double* xb, double* x,
                        int init, int max_nr, cudaStream_t st) {
  kp_backward<double>(P, lay, Lc, yI, xb, x, init, max_nr, st);
}

void launch_compact_factor(int P, int max_rows, const SubLayout* lay, const double* A, double* Lc, cudaStream_t st) {
  const int nt = (max_rows + 31) / 32;
  if (P > 0 && nt > 0) k_compact_factor<double><<<dim3(nt, P), 256, 0, st>>>(lay, A, Lc);
}

void launch_compact_factor(int P, int max_rows, const SubLayout* lay, const float* A, float* Lc, cudaStream_t st) {
  const int nt = (max_rows + 31) / 32;
  if (P > 0 && nt > 0) k_compact_factor<float><<<dim3(nt, P), 256, 0, st>>>(lay, A, Lc);
}

void launch_kresid2(int n_el, int nde, const int32_t* elem_sub, const int32_t* row_sub, int n_rows, const SubLayout* lay,
                    const int32_t* kinc_ptr, const int32_t* kinc, const int32_t* elem_dense, const double* Ke,
                    const double* g, const double* x, double* ye, double* r, cudaStream_t st) {
  if (n_el > 0) {
    if (nde == 30)
      k_elem_kx<30><<<(n_el + 127) / 128, 128, 0, st>>>(n_el, elem_sub, lay, elem_dense, Ke, x, ye);
    else
      k_elem_kx<12><<<(n_el + 127) / 128, 128, 0, st>>>(n_el, elem_sub, lay, elem_dense, Ke, x, ye);
  }
  long b = ((long)n_rows + kT - 1) / kT;
  if (b > 65535) b = 65535;
  if (n_rows > 0) k_row_resid<<<(int)b, kT, 0, st>>>(n_rows, row_sub, lay, kinc_ptr, kinc, ye, g, r);
}

void launch_place(int P, const SubLayout* lay, const double* loc, double* out, cudaStream_t st, const int* done) {
  k_place<<<P, kT, 0, st>>>(lay, loc, out, done);
}

void launch_sub_norm2(int P, const SubLayout* lay, const double* r, const double* g, double* out, cudaStream_t st) {
  k_sub_norm2<<<P, kT, 0, st>>>(lay, r, g, out);
}

void launch_fill_mix(long n, double* x, cudaStream_t st) {
  if (n <= 0) return;
  k_fill_mix<<<(unsigned)std::min<long>((n + kT - 1) / kT, 4096), kT, 0, st>>>(n, x);
}

}  // namespace feti
