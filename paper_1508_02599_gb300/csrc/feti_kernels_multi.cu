// Block form of the projected PCG: up to kMaxRhs independent CG recurrences
// sharing every operator apply (the RHS of several load cases, Sec. 3.2 /
// Sec. 4.3).  Multiplier-space vectors are row-major [n_lambda][nrhs] and
// local vectors [n_b][nrhs], so each gather, scatter and projection reads a
// row's nrhs values contiguously, and every dense local operator entry read
// from HBM feeds nrhs FMAs (a batched GEMM with N = nrhs instead of a GEMV).
// Scalars (rho, alpha, beta, norms) are per right-hand side; a converged
// right-hand side is frozen (alpha = beta = 0 for it) while the others run on.
#include "feti_internal.h"

#include <cuda.h>

#include <cmath>

namespace feti {

namespace {

constexpr int kThreads = 256;
constexpr int kPartials = 304;

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_sumf(float v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Per-RHS CTA reduction of acc[k] (k < nrhs): result valid in thread 0's out[k].
// red: shared [8][kMaxRhs].
__device__ void block_sum_vec(const double* acc, int nrhs, double (*red)[kMaxRhs], double* out) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int k = 0; k < nrhs; ++k) {
    const double t = warp_sum(acc[k]);
    if (lane == 0) red[wid][k] = t;
  }
  __syncthreads();
  if (threadIdx.x < nrhs) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w][threadIdx.x];
    out[threadIdx.x] = t;
  }
  __syncthreads();
}

// Sum of the kPartials partial sums of right-hand side k (fixed order).
__device__ double reduce_partials_k(const double* partial, int k, double* red1) {
  double t = 0.0;
  for (int i = threadIdx.x; i < kPartials; i += blockDim.x) t += partial[k * kPartials + i];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  t = warp_sum(t);
  __syncthreads();
  if (lane == 0) red1[wid] = t;
  __syncthreads();
  double s = 0.0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red1[w];
  __syncthreads();
  return s;
}

template <typename T>
__global__ void k_gather_m(Maps mp, int nrhs, const double* __restrict__ x, const double* __restrict__ wv,
                           T* __restrict__ y, const int* __restrict__ done) {
  if (*done) return;
  for (int gp = blockIdx.x * blockDim.x + threadIdx.x; gp < mp.nb_total; gp += gridDim.x * blockDim.x) {
    double val[kMaxRhs];
    for (int k = 0; k < nrhs; ++k) val[k] = 0.0;
    for (int e = mp.bt_ptr[gp]; e < mp.bt_ptr[gp + 1]; ++e) {
      const int row = mp.bt_row[e];
      const double sw = mp.bt_sgn[e] * (wv ? wv[row] : 1.0);
      for (int k = 0; k < nrhs; ++k) val[k] += sw * x[(size_t)row * nrhs + k];
    }
    for (int k = 0; k < nrhs; ++k) y[(size_t)gp * nrhs + k] = (T)val[k];
  }
}

// Y (m x nrhs) = M_i V (m x nrhs) for every subdomain.  V is staged in shared
// memory transposed ([k][column], padded to 4), each warp keeps R x nrhs
// accumulators: every matrix entry loaded from HBM feeds nrhs FMAs.
template <typename T, int R>
__global__ void __launch_bounds__(kThreads) k_gemm_loc(const int32_t* __restrict__ blk_sub,
                                                       const int32_t* __restrict__ blk_row0, int rpc,
                                                       const SubLayout* __restrict__ lay, int which,
                                                       const T* __restrict__ M, int nrhs,
                                                       const T* __restrict__ vloc, double* __restrict__ y,
                                                       const int* __restrict__ done) {
  if (*done) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* v = reinterpret_cast<T*>(smem_raw);
  const int s = blk_sub[blockIdx.x];
  const int r0 = blk_row0[blockIdx.x];
  const SubLayout L = lay[s];
  const int m = which == 0 ? L.nbp : L.nbp + L.k;
  constexpr bool f32 = sizeof(T) == 4;
  const int ldm = f32 ? ((m + 3) & ~3) : m;
  const T* Ms = M + (f32 ? (which == 0 ? L.foff32 : L.soff32) : (which == 0 ? L.foff : L.soff));
  for (int idx = threadIdx.x; idx < ldm * nrhs; idx += blockDim.x) {
    const int c = idx / nrhs, k = idx % nrhs;
    v[k * ldm + c] = c < m ? vloc[(size_t)(L.boff + c) * nrhs + k] : (T)0;
  }
  if (which == 0 && r0 == 0)
    for (int idx = threadIdx.x; idx < L.k * nrhs; idx += blockDim.x) y[(size_t)(L.boff + L.nbp) * nrhs + idx] = 0.0;
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int rend = min(r0 + rpc, m);
  for (int rbase = r0 + wid * R; rbase < rend; rbase += (kThreads / 32) * R) {
    T acc[R][kMaxRhs];
#pragma unroll
    for (int j = 0; j < R; ++j)
#pragma unroll
      for (int k = 0; k < kMaxRhs; ++k) acc[j][k] = (T)0;
    const T* rows[R];
#pragma unroll
    for (int j = 0; j < R; ++j) rows[j] = Ms + (size_t)min(rbase + j, m - 1) * ldm;
    if constexpr (f32) {
      const int m4 = ldm >> 2;
      for (int c = lane; c < m4; c += 32) {
        float4 a[R];
#pragma unroll
        for (int j = 0; j < R; ++j) a[j] = __ldg(reinterpret_cast<const float4*>(rows[j]) + c);
#pragma unroll
        for (int k = 0; k < kMaxRhs; ++k) {
          if (k < nrhs) {
            const float4 vv = reinterpret_cast<const float4*>(v + k * ldm)[c];
#pragma unroll
            for (int j = 0; j < R; ++j) acc[j][k] += a[j].x * vv.x + a[j].y * vv.y + a[j].z * vv.z + a[j].w * vv.w;
          }
        }
      }
    } else {
      for (int c = lane; c < m; c += 32) {
        T a[R];
#pragma unroll
        for (int j = 0; j < R; ++j) a[j] = __ldg(rows[j] + c);
#pragma unroll
        for (int k = 0; k < kMaxRhs; ++k) {
          if (k < nrhs) {
            const T vv = v[k * ldm + c];
#pragma unroll
            for (int j = 0; j < R; ++j) acc[j][k] += a[j] * vv;
          }
        }
      }
    }
#pragma unroll
    for (int j = 0; j < R; ++j)
#pragma unroll
      for (int k = 0; k < kMaxRhs; ++k) {
        if (k < nrhs) {
          double t;
          if constexpr (f32) t = (double)warp_sumf(acc[j][k]);
          else t = warp_sum(acc[j][k]);
          if (lane == 0 && rbase + j < rend) y[(size_t)(L.boff + rbase + j) * nrhs + k] = t;
        }
      }
  }
}

__global__ void __launch_bounds__(kThreads) k_scatter_m(Maps mp, int nrhs, const double* __restrict__ y,
                                                        const double* __restrict__ wv, double* __restrict__ q,
                                                        const double* __restrict__ a, double* __restrict__ partial,
                                                        const int* __restrict__ done) {
  if (*done) return;
  __shared__ double red[8][kMaxRhs];
  __shared__ double out[kMaxRhs];
  double dot[kMaxRhs];
  for (int k = 0; k < nrhs; ++k) dot[k] = 0.0;
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < mp.n_lambda; r += gridDim.x * blockDim.x) {
    double val[kMaxRhs];
    for (int k = 0; k < nrhs; ++k) val[k] = 0.0;
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const int pos = mp.row_pos[2 * r + e];
      if (pos >= 0) {
        const double sg = mp.row_sgn[2 * r + e];
        for (int k = 0; k < nrhs; ++k) val[k] += sg * y[(size_t)pos * nrhs + k];
      }
    }
    const double w = wv ? wv[r] : 1.0;
    for (int k = 0; k < nrhs; ++k) {
      const double v = w * val[k];
      q[(size_t)r * nrhs + k] = v;
      if (partial) dot[k] += (a ? a[(size_t)r * nrhs + k] : v) * v;
    }
  }
  if (partial) {
    block_sum_vec(dot, nrhs, red, out);
    if (threadIdx.x < nrhs) partial[threadIdx.x * kPartials + blockIdx.x] = out[threadIdx.x];
  }
}

// G^T x per chunk of 256 boundary positions: partial[(c * 6 + a) * nrhs + k].
// With q != NULL the input is x - alpha_k q (fused CG update).
__global__ void __launch_bounds__(kThreads) k_gtv_part_m(const int32_t* __restrict__ chunk_sub,
                                                         const int32_t* __restrict__ chunk_p0,
                                                         const SubLayout* __restrict__ lay,
                                                         const double* __restrict__ R, Maps mp, int nrhs,
                                                         const double* __restrict__ x, double* __restrict__ partial,
                                                         const double* __restrict__ q, const PcgScalarsM* sc,
                                                         const int* __restrict__ done) {
  if (*done) return;
  __shared__ double acc_sh[kThreads][6];
  const int c = blockIdx.x;
  const SubLayout L = lay[chunk_sub[c]];
  const int nb = L.nbp + L.k;
  const int k = threadIdx.x % nrhs;
  const int slot = threadIdx.x / nrhs;
  const int nslots = kThreads / nrhs;
  const double alpha = q ? sc->alpha[k] : 0.0;
  double acc[6] = {0, 0, 0, 0, 0, 0};
  if (slot < nslots) {
    for (int pp = slot; pp < 256; pp += nslots) {
      const int p = chunk_p0[c] + pp;
      if (p >= nb) break;
      const int gp = L.boff + p;
      double val = 0.0;
      for (int e = mp.bt_ptr[gp]; e < mp.bt_ptr[gp + 1]; ++e) {
        const int row = mp.bt_row[e];
        const double xv = x[(size_t)row * nrhs + k];
        val += mp.bt_sgn[e] * (q ? xv - alpha * q[(size_t)row * nrhs + k] : xv);
      }
      const double* Rr = R + L.roff + (size_t)(L.nI + p) * L.k;
      for (int a = 0; a < L.k; ++a) acc[a] += Rr[a] * val;
    }
  }
  for (int a = 0; a < 6; ++a) acc_sh[threadIdx.x][a] = (slot < nslots) ? acc[a] : 0.0;
  __syncthreads();
  if (threadIdx.x < L.k * nrhs) {
    const int a = threadIdx.x / nrhs, kk = threadIdx.x % nrhs;
    double t = 0.0;
    for (int sl = 0; sl < nslots; ++sl) t += acc_sh[sl * nrhs + kk][a];
    partial[((size_t)c * 6 + a) * nrhs + kk] = t;
  }
}

// g[j][k] = sum over the chunks of column j's subdomain.
__global__ void k_gsum_m(int cd, int nrhs, const double* __restrict__ partial,
                         const int32_t* __restrict__ sub_chunk_ptr, const int32_t* __restrict__ col_sub,
                         const SubLayout* __restrict__ lay, double* __restrict__ g, const int* __restrict__ done) {
  if (*done) return;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < cd * nrhs; idx += gridDim.x * blockDim.x) {
    const int j = idx / nrhs, k = idx % nrhs;
    const int s = col_sub[j];
    const int a = j - lay[s].coff;
    double t = 0.0;
    for (int qc = sub_chunk_ptr[s]; qc < sub_chunk_ptr[s + 1]; ++qc) t += partial[((size_t)qc * 6 + a) * nrhs + k];
    g[idx] = t;
  }
}

// C (cd x nrhs) = Ginv G, warp per row.
__global__ void k_coarse_gemm_m(int cd, int nrhs, const double* __restrict__ Ginv, const double* __restrict__ g,
                                double* __restrict__ c, const int* __restrict__ done) {
  if (*done) return;
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int r = warp; r < cd; r += nwarps) {
    double acc[kMaxRhs];
    for (int k = 0; k < nrhs; ++k) acc[k] = 0.0;
    for (int j = lane; j < cd; j += 32) {
      const double gv = Ginv[(size_t)r * cd + j];
      for (int k = 0; k < nrhs; ++k) acc[k] += gv * g[(size_t)j * nrhs + k];
    }
    for (int k = 0; k < nrhs; ++k) {
      const double t = warp_sum(acc[k]);
      if (lane == 0) c[(size_t)r * nrhs + k] = t;
    }
  }
}

// out = v - G c row-wise (v = r - alpha q with the fused update, r and lam
// updated in place), partial sums of (a, out) or (out, out) per RHS.
__global__ void __launch_bounds__(kThreads) k_expand_m(Maps mp, const SubLayout* __restrict__ lay,
                                                       const double* __restrict__ R, int nrhs, int has_coarse,
                                                       const double* __restrict__ v, const double* __restrict__ c,
                                                       double* __restrict__ out, const double* __restrict__ a,
                                                       double* __restrict__ partial, double* __restrict__ r_upd,
                                                       double* __restrict__ lam, const double* __restrict__ p,
                                                       const double* __restrict__ q, const PcgScalarsM* sc,
                                                       const int* __restrict__ done) {
  if (*done) return;
  __shared__ double red[8][kMaxRhs];
  __shared__ double outs[kMaxRhs];
  double alpha[kMaxRhs];
  for (int k = 0; k < nrhs; ++k) alpha[k] = r_upd ? sc->alpha[k] : 0.0;
  double dot[kMaxRhs];
  for (int k = 0; k < nrhs; ++k) dot[k] = 0.0;
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < mp.n_lambda; r += gridDim.x * blockDim.x) {
    double val[kMaxRhs];
    for (int k = 0; k < nrhs; ++k) {
      const size_t i = (size_t)r * nrhs + k;
      if (r_upd) {
        const double rv = r_upd[i] - alpha[k] * q[i];
        r_upd[i] = rv;
        lam[i] += alpha[k] * p[i];
        val[k] = rv;
      } else {
        val[k] = v[i];
      }
    }
    if (has_coarse) {
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const int gp = mp.row_pos[2 * r + e];
        if (gp < 0) continue;
        const SubLayout L = lay[mp.bpos_sub[gp]];
        if (!L.k) continue;
        const double sg = mp.row_sgn[2 * r + e];
        const double* Rr = R + L.roff + (size_t)(L.nI + gp - L.boff) * L.k;
        for (int kk = 0; kk < L.k; ++kk) {
          const double ra = sg * Rr[kk];
          const double* cr = c + (size_t)(L.coff + kk) * nrhs;
          for (int k = 0; k < nrhs; ++k) val[k] -= ra * cr[k];
        }
      }
    }
    for (int k = 0; k < nrhs; ++k) {
      out[(size_t)r * nrhs + k] = val[k];
      dot[k] += (a ? a[(size_t)r * nrhs + k] : val[k]) * val[k];
    }
  }
  block_sum_vec(dot, nrhs, red, outs);
  if (threadIdx.x < nrhs) partial[threadIdx.x * kPartials + blockIdx.x] = outs[threadIdx.x];
}

// rho_k = (w, y)_k, beta_k, p = y + beta p (frozen right-hand sides keep p).
__global__ void __launch_bounds__(kThreads) k_axpby_rho_m(int n, int nrhs, double* __restrict__ p,
                                                          const double* __restrict__ y, PcgScalarsM* s,
                                                          const double* __restrict__ partial) {
  if (s->done) return;
  __shared__ double red1[8];
  const int it = s->it;
  double beta[kMaxRhs];
  int act[kMaxRhs];
  for (int k = 0; k < nrhs; ++k) {
    const double rho = reduce_partials_k(partial, k, red1);
    act[k] = s->active[k];
    beta[k] = (it > 0 && act[k]) ? rho / s->rho_slot[(it + 1) & 1][k] : 0.0;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      if (act[k] && (!(rho > 0.0) || !isfinite(rho))) {
        s->status = DEV_BREAKDOWN;
        s->done = 1;
      }
      s->rho_slot[it & 1][k] = rho;
      s->rho[k] = rho;
      s->beta[k] = beta[k];
    }
  }
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    for (int k = 0; k < nrhs; ++k) {
      if (!act[k]) continue;
      const size_t j = (size_t)i * nrhs + k;
      p[j] = it > 0 ? y[j] + beta[k] * p[j] : y[j];
    }
}

// alpha_k = rho_k / (p, q)_k for active right-hand sides, 0 for frozen ones.
__global__ void k_alpha_m(int nrhs, PcgScalarsM* s, const double* __restrict__ partial, double* alpha_hist) {
  if (s->done) return;
  __shared__ double red1[8];
  for (int k = 0; k < nrhs; ++k) {
    const double pq = reduce_partials_k(partial, k, red1);
    if (threadIdx.x == 0) {
      double al = 0.0;
      if (s->active[k]) {
        if (!(pq > 0.0) || !isfinite(pq)) {
          s->status = DEV_BREAKDOWN;
          s->done = 1;
        } else {
          al = s->rho[k] / pq;
        }
      }
      s->alpha[k] = al;
      s->pq[k] = pq;
      alpha_hist[(size_t)s->it * kMaxRhs + k] = al;
    }
  }
}

// Stopping test per right-hand side; done when all are frozen or at maxit.
__global__ void k_conv_m(int nrhs, PcgScalarsM* s, const double* __restrict__ partial, int first) {
  if (s->done) return;
  __shared__ double red1[8];
  double wn[kMaxRhs];
  for (int k = 0; k < nrhs; ++k) wn[k] = sqrt(reduce_partials_k(partial, k, red1));
  if (threadIdx.x != 0) return;
  int any = 0;
  if (first) {
    for (int k = 0; k < nrhs; ++k) {
      s->wnorm0[k] = wn[k];
      s->wnorm[k] = wn[k];
      if (!isfinite(wn[k])) s->status = DEV_BREAKDOWN;
      s->active[k] = (s->active[k] && wn[k] > 0.0) ? 1 : 0;
      any |= s->active[k];
    }
    if (!any || s->status) s->done = 1;
    return;
  }
  s->it += 1;
  for (int k = 0; k < nrhs; ++k) {
    if (!s->active[k]) continue;
    s->wnorm[k] = wn[k];
    if (!isfinite(wn[k])) {
      s->status = DEV_BREAKDOWN;
    } else if (wn[k] <= s->tol[k] * s->wnorm0[k]) {
      s->active[k] = 0;
    }
    any |= s->active[k];
  }
  if (!any || s->status || s->it >= s->maxit) s->done = 1;
}

__global__ void k_spmv_lump_m(int n_rows, int nrhs, const int32_t* __restrict__ ptr, const int32_t* __restrict__ col,
                              const double* __restrict__ val, const double* __restrict__ v, double* __restrict__ y,
                              const int* __restrict__ done) {
  if (*done) return;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n_rows * nrhs; idx += gridDim.x * blockDim.x) {
    const int r = idx / nrhs, k = idx % nrhs;
    double acc = 0.0;
    for (int j = ptr[r]; j < ptr[r + 1]; ++j) acc += val[j] * v[(size_t)col[j] * nrhs + k];
    y[idx] = acc;
  }
}

// Strided column copies between [n][nrhs] blocks and contiguous vectors.
__global__ void k_col_get(int n, int nrhs, int k, const double* __restrict__ blk, double* __restrict__ v) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) v[i] = blk[(size_t)i * nrhs + k];
}
__global__ void k_col_set(int n, int nrhs, int k, double scale, const double* __restrict__ v,
                          double* __restrict__ blk) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    blk[(size_t)i * nrhs + k] = scale * v[i];
}

// ---------------------------------------------------------------------------
// Tensor-core block GEMM (tcgen05, kind::tf32, 3xTF32): Y (m x nrhs) = M_i V
// for the FP32 copies.  A CTA owns 128 rows of one subdomain; K runs in
// chunks of 32 columns through two shared-memory stages.  Each operand tile
// is split into a TF32 head and a tail (x = hi + lo, lo exact in FP32) while
// it is staged, and the three products hi*hi + hi*lo + lo*hi accumulate in
// FP32 in tensor memory (128 lanes x 16 columns), which gives FP32-level
// accuracy from TF32 tensor-core passes.  Staged tiles use the 128-byte
// swizzled K-major layout (8 rows x 128 B atoms), so the row-contiguous
// global loads map onto conflict-free shared-memory stores.  One thread
// issues the MMAs and commits them to an mbarrier per stage; all waits are
// bounded (about 0.1 s of clock cycles) and report a timeout in *err.
__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t c) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(b)), "r"(c) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint64_t* b, uint32_t par) {
  uint32_t ok;
  asm volatile("{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
               : "=r"(ok)
               : "r"(su32(b)), "r"(par)
               : "memory");
  return ok != 0;
}

// Shared-memory matrix descriptor: 128-byte swizzle, K-major, 1024 B between
// 8-row groups.
__device__ __forceinline__ uint64_t sw128_desc(const void* p) {
  uint64_t d = (su32(p) >> 4) & 0x3FFF;
  d |= (uint64_t)1 << 16;            // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;  // stride byte offset
  d |= (uint64_t)1 << 46;            // descriptor version
  d |= (uint64_t)2 << 61;            // 128-byte swizzle
  return d;
}

__device__ __forceinline__ int sw_off(int r, int c) { return r * 128 + ((c ^ (r & 7)) << 4); }

__device__ __forceinline__ void split_tf32(float x, float& hi, float& lo) {
  hi = __uint_as_float(__float_as_uint(x) & 0xFFFFE000u);
  lo = x - hi;
}

__device__ __forceinline__ void tc_mma(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile("{ .reg .pred p; setp.ne.b32 p, %4, 0; tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p; }" ::"r"(
                   tmem),
               "l"(a), "l"(b), "r"(idesc), "r"(acc)
               : "memory");
}

constexpr int TC_A_BYTES = 128 * 128;
constexpr int TC_B_BYTES = 16 * 128;
constexpr int TC_STAGE = 2 * TC_A_BYTES + 2 * TC_B_BYTES;
constexpr int TC_SMEM = 2 * TC_STAGE + 1024;

__global__ void __launch_bounds__(kThreads) k_gemm_tc(const int32_t* __restrict__ blk_sub,
                                                      const int32_t* __restrict__ blk_row0,
                                                      const SubLayout* __restrict__ lay, int which,
                                                      const float* __restrict__ M, int nrhs,
                                                      const float* __restrict__ vloc, double* __restrict__ y,
                                                      const int* __restrict__ done, int* __restrict__ err) {
  if (*done) return;
  extern __shared__ __align__(1024) unsigned char tc_smem_dyn[];
  unsigned char* smem = tc_smem_dyn + ((1024 - (su32(tc_smem_dyn) & 1023)) & 1023);
  __shared__ uint64_t mbar[2];
  __shared__ uint32_t tmem_base;
  const int s_id = blk_sub[blockIdx.x];
  const int r0 = blk_row0[blockIdx.x];
  const SubLayout L = lay[s_id];
  const int m = which == 0 ? L.nbp : L.nbp + L.k;
  const int ldm = (m + 3) & ~3;
  const float* Ms = M + (which == 0 ? L.foff32 : L.soff32);
  const int tid = threadIdx.x, wid = tid >> 5, lane = tid & 31;
  if (which == 0 && r0 == 0)
    for (int idx = tid; idx < L.k * nrhs; idx += blockDim.x) y[(size_t)(L.boff + L.nbp) * nrhs + idx] = 0.0;
  if (wid == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 32;" ::"r"(su32(&tmem_base)) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    mbar_init(&mbar[0], 1);
    mbar_init(&mbar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;
  // instruction descriptor: D FP32, A and B TF32, both K-major, N = 16, M = 128
  const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((16u >> 3) << 17) | ((128u >> 4) << 24);
  const int nk = (m + 31) / 32;
  bool timed_out = false;
  // register prefetch: each thread holds the 4 A chunks (16 B each) and up to
  // one B chunk of the next K step while the current step is staged and
  // multiplied
  float4 ra[4], rb;
  auto load_chunk = [&](int kc2) {
    const int k0 = kc2 * 32;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int idx = tid + q * kThreads;
      const int r = idx >> 3, c = idx & 7;
      const int row = r0 + r, col = k0 + 4 * c;
      ra[q] = (row < m && col < ldm) ? __ldg(reinterpret_cast<const float4*>(Ms + (size_t)row * ldm + col))
                                     : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    if (tid < 16 * 8) {
      const int n = tid >> 3, c = tid & 7;
      float v4[4];
      for (int e = 0; e < 4; ++e) {
        const int kk = k0 + 4 * c + e;
        v4[e] = (kk < m && n < nrhs) ? vloc[(size_t)(L.boff + kk) * nrhs + n] : 0.f;
      }
      rb = make_float4(v4[0], v4[1], v4[2], v4[3]);
    }
  };
  if (nk > 0) load_chunk(0);
  for (int kc = 0; kc < nk; ++kc) {
    const int st = kc & 1;
    float4 ca[4], cb = rb;
#pragma unroll
    for (int q = 0; q < 4; ++q) ca[q] = ra[q];
    if (kc + 1 < nk) load_chunk(kc + 1);
    if (kc >= 2) {
      const uint32_t par = ((kc - 2) >> 1) & 1;
      const long long t0 = clock64();
      while (!timed_out && !mbar_try(&mbar[st], par))
        if (clock64() - t0 > 200000000LL) timed_out = true;
    }
    unsigned char* sb = smem + st * TC_STAGE;
    unsigned char* Ahi = sb;
    unsigned char* Alo = sb + TC_A_BYTES;
    unsigned char* Bhi = sb + 2 * TC_A_BYTES;
    unsigned char* Blo = Bhi + TC_B_BYTES;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int idx = tid + q * kThreads;
      const int r = idx >> 3, c = idx & 7;
      float4 h, l;
      split_tf32(ca[q].x, h.x, l.x);
      split_tf32(ca[q].y, h.y, l.y);
      split_tf32(ca[q].z, h.z, l.z);
      split_tf32(ca[q].w, h.w, l.w);
      *reinterpret_cast<float4*>(Ahi + sw_off(r, c)) = h;
      *reinterpret_cast<float4*>(Alo + sw_off(r, c)) = l;
    }
    if (tid < 16 * 8) {
      const int n = tid >> 3, c = tid & 7;
      float4 h, l;
      split_tf32(cb.x, h.x, l.x);
      split_tf32(cb.y, h.y, l.y);
      split_tf32(cb.z, h.z, l.z);
      split_tf32(cb.w, h.w, l.w);
      *reinterpret_cast<float4*>(Bhi + sw_off(n, c)) = h;
      *reinterpret_cast<float4*>(Blo + sw_off(n, c)) = l;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      for (int j = 0; j < 4; ++j) {
        const uint64_t ah = sw128_desc(Ahi + 32 * j), al = sw128_desc(Alo + 32 * j);
        const uint64_t bh = sw128_desc(Bhi + 32 * j), bl = sw128_desc(Blo + 32 * j);
        tc_mma(tmem, ah, bh, idesc, (kc > 0 || j > 0) ? 1u : 0u);
        tc_mma(tmem, ah, bl, idesc, 1u);
        tc_mma(tmem, al, bh, idesc, 1u);
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(&mbar[st]))
                   : "memory");
    }
  }
  if (nk > 0) {
    const int st = (nk - 1) & 1;
    const uint32_t par = ((nk - 1) >> 1) & 1;
    const long long t0 = clock64();
    while (!timed_out && !mbar_try(&mbar[st], par))
      if (clock64() - t0 > 200000000LL) timed_out = true;
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (timed_out && lane == 0) atomicExch(err, 1);
  if (wid < 4) {
    uint32_t r[16];
    const uint32_t taddr = tmem + ((uint32_t)(wid * 32) << 16);
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    const int row = r0 + wid * 32 + lane;
    if (row < m && !timed_out)
      for (int n = 0; n < nrhs; ++n) y[(size_t)(L.boff + row) * nrhs + n] = (double)__uint_as_float(r[n]);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (wid == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 32;" ::"r"(tmem) : "memory");
}

// Bulk-copy staged variant: the FP32 rows of M_i are streamed into NRAW
// shared-memory stages by cp.async.bulk (one 128-byte row segment per thread,
// completion counted in bytes on a per-stage mbarrier), so several K chunks
// are in flight per CTA without holding registers; each chunk is then split
// into the TF32 head and tail from shared memory into the one swizzled MMA
// stage.  The timeout flag is made CTA-uniform at every step; after a timeout
// no further copies are issued, and the copies and MMAs already in flight
// are drained (with fresh bounded waits) before tensor memory is freed.
constexpr int TC2_NRAW = 3;
constexpr int TC2_RAW = 128 * 128;
constexpr int TC2_SMEM = TC_STAGE + TC2_NRAW * TC2_RAW + 1024;

__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(b)), "r"(bytes) : "memory");
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* b) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   su32(dst)),
               "l"(src), "r"(bytes), "r"(su32(b))
               : "memory");
}

__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* b, uint32_t par) {
  const long long t0 = clock64();
  while (!mbar_try(b, par))
    if (clock64() - t0 > 200000000LL) return false;
  return true;
}

__global__ void __launch_bounds__(kThreads) k_gemm_tc2(const int32_t* __restrict__ blk_sub,
                                                       const int32_t* __restrict__ blk_row0,
                                                       const SubLayout* __restrict__ lay, int which,
                                                       const float* __restrict__ M, int nrhs,
                                                       const float* __restrict__ vloc, double* __restrict__ y,
                                                       const int* __restrict__ done, int* __restrict__ err) {
  if (*done) return;
  extern __shared__ __align__(1024) unsigned char tc_smem_dyn[];
  unsigned char* smem = tc_smem_dyn + ((1024 - (su32(tc_smem_dyn) & 1023)) & 1023);
  unsigned char* Ahi = smem;
  unsigned char* Alo = smem + TC_A_BYTES;
  unsigned char* Bhi = smem + 2 * TC_A_BYTES;
  unsigned char* Blo = Bhi + TC_B_BYTES;
  unsigned char* raw0 = smem + TC_STAGE;
  __shared__ uint64_t mbar;
  __shared__ uint64_t rbar[TC2_NRAW];
  __shared__ uint32_t tmem_base;
  const int s_id = blk_sub[blockIdx.x];
  const int r0 = blk_row0[blockIdx.x];
  const SubLayout L = lay[s_id];
  const int m = which == 0 ? L.nbp : L.nbp + L.k;
  const int ldm = (m + 3) & ~3;
  const float* Ms = M + (which == 0 ? L.foff32 : L.soff32);
  const int tid = threadIdx.x, wid = tid >> 5, lane = tid & 31;
  if (which == 0 && r0 == 0)
    for (int idx = tid; idx < L.k * nrhs; idx += blockDim.x) y[(size_t)(L.boff + L.nbp) * nrhs + idx] = 0.0;
  if (wid == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 32;" ::"r"(su32(&tmem_base)) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    mbar_init(&mbar, 1);
    for (int i = 0; i < TC2_NRAW; ++i) mbar_init(&rbar[i], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;
  const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((16u >> 3) << 17) | ((128u >> 4) << 24);
  const int nk = (m + 31) / 32;
  const int nrows = min(128, m - r0);
  // chunk kc2 of rows r0 .. r0 + nrows - 1 into raw stage kc2 % NRAW; the
  // row segments start on 16-byte boundaries (row stride and chunk offset are
  // multiples of 4 floats) and are multiples of 16 bytes long
  auto issue_raw = [&](int kc2) {
    const int k0 = kc2 * 32;
    const uint32_t seg = (uint32_t)min(32, ldm - k0) * 4u;
    uint64_t* b = &rbar[kc2 % TC2_NRAW];
    unsigned char* dst = raw0 + (kc2 % TC2_NRAW) * TC2_RAW;
    if (tid == 0) mbar_expect_tx(b, seg * (uint32_t)nrows);
    if (tid < nrows) bulk_g2s(dst + tid * 128, Ms + (size_t)(r0 + tid) * ldm + k0, seg, b);
  };
  int issued = 0;
  for (; issued < TC2_NRAW && issued < nk; ++issued) issue_raw(issued);
  float4 rb = make_float4(0.f, 0.f, 0.f, 0.f);
  auto load_b = [&](int kc2) {
    if (tid < 16 * 8) {
      const int n = tid >> 3, c = tid & 7, k0 = kc2 * 32;
      float v4[4];
      for (int e = 0; e < 4; ++e) {
        const int kk = k0 + 4 * c + e;
        v4[e] = (kk < m && n < nrhs) ? vloc[(size_t)(L.boff + kk) * nrhs + n] : 0.f;
      }
      rb = make_float4(v4[0], v4[1], v4[2], v4[3]);
    }
  };
  if (nk > 0) load_b(0);
  bool timed_out = false;
  int n_mma = 0, kc = 0;
  for (; kc < nk; ++kc) {
    const float4 cb = rb;
    if (kc + 1 < nk) load_b(kc + 1);
    if (!mbar_wait_bounded(&rbar[kc % TC2_NRAW], (uint32_t)(kc / TC2_NRAW) & 1u)) timed_out = true;
    const unsigned char* raw = raw0 + (kc % TC2_NRAW) * TC2_RAW;
    const int k0 = kc * 32;
    float4 ca[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int idx = tid + q * kThreads;
      const int r = idx >> 3, c = idx & 7;
      ca[q] = (!timed_out && r < nrows && k0 + 4 * c < ldm) ? *reinterpret_cast<const float4*>(raw + r * 128 + c * 16)
                                                          : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    if (kc >= 1 && !timed_out && !mbar_wait_bounded(&mbar, (uint32_t)(kc - 1) & 1u)) timed_out = true;
    if (!timed_out) {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int idx = tid + q * kThreads;
        const int r = idx >> 3, c = idx & 7;
        float4 h, l;
        split_tf32(ca[q].x, h.x, l.x);
        split_tf32(ca[q].y, h.y, l.y);
        split_tf32(ca[q].z, h.z, l.z);
        split_tf32(ca[q].w, h.w, l.w);
        *reinterpret_cast<float4*>(Ahi + sw_off(r, c)) = h;
        *reinterpret_cast<float4*>(Alo + sw_off(r, c)) = l;
      }
      if (tid < 16 * 8) {
        const int n = tid >> 3, c = tid & 7;
        float4 h, l;
        split_tf32(cb.x, h.x, l.x);
        split_tf32(cb.y, h.y, l.y);
        split_tf32(cb.z, h.z, l.z);
        split_tf32(cb.w, h.w, l.w);
        *reinterpret_cast<float4*>(Bhi + sw_off(n, c)) = h;
        *reinterpret_cast<float4*>(Blo + sw_off(n, c)) = l;
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    timed_out = __syncthreads_or(timed_out ? 1 : 0) != 0;
    if (timed_out) break;
    if (kc + TC2_NRAW < nk) {
      issue_raw(kc + TC2_NRAW);
      issued = kc + TC2_NRAW + 1;
    }
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      for (int j = 0; j < 4; ++j) {
        const uint64_t ah = sw128_desc(Ahi + 32 * j), al = sw128_desc(Alo + 32 * j);
        const uint64_t bh = sw128_desc(Bhi + 32 * j), bl = sw128_desc(Blo + 32 * j);
        tc_mma(tmem, ah, bh, idesc, (kc > 0 || j > 0) ? 1u : 0u);
        tc_mma(tmem, ah, bl, idesc, 1u);
        tc_mma(tmem, al, bh, idesc, 1u);
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(&mbar))
                   : "memory");
    }
    n_mma = kc + 1;
  }
  // drain: copies issued for chunks not consumed (only after a timeout) and
  // the last MMA group, each with its own bounded wait
  bool drained = true;
  for (int j = kc; j < issued; ++j)
    if (!mbar_wait_bounded(&rbar[j % TC2_NRAW], (uint32_t)(j / TC2_NRAW) & 1u)) drained = false;
  if (n_mma > 0 && !mbar_wait_bounded(&mbar, (uint32_t)(n_mma - 1) & 1u)) drained = false;
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if ((timed_out || !drained) && lane == 0) atomicExch(err, 1);
  if (wid < 4) {
    uint32_t r[16];
    const uint32_t taddr = tmem + ((uint32_t)(wid * 32) << 16);
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    const int row = r0 + wid * 32 + lane;
    if (row < m && !timed_out && drained)
      for (int n = 0; n < nrhs; ++n) y[(size_t)(L.boff + row) * nrhs + n] = (double)__uint_as_float(r[n]);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (wid == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 32;" ::"r"(tmem) : "memory");
}

// TMA-fed variant: each K chunk of M_i (128 rows x 32 columns, FP32) is one
// 2-D tensor-map load (cp.async.bulk.tensor) into a 128B-swizzled stage, rows
// and columns beyond the block zero-filled by the copy engine.  The tensor
// core reads an FP32 operand of kind::tf32 through its TF32 part (the low 13
// mantissa bits are dropped, i.e. truncation toward zero), so the loaded
// tile is the head operand as it is and threads only write the tail
// x - trunc(x) beside it at the same swizzled offsets.  TC3_NS stages with a
// full and an MMA-done mbarrier each: thread 0 refills the stage of chunk
// kc - 1 as soon as its MMAs complete, while chunk kc's MMAs run.  The
// three products of a K step accumulate into separate tensor-memory columns
// (summed in the epilogue), so consecutive MMAs do not wait on one
// accumulator.  Timeouts are CTA-uniform; copies and MMAs in flight are
// drained with fresh bounded waits before tensor memory is freed.
constexpr int TC3_NS = 3;
constexpr int TC3_NACC = 3;  // hi*hi, hi*lo, lo*hi each in its own accumulator
constexpr int TC3_TCOLS = TC3_NACC == 1 ? 32 : (TC3_NACC * 16 <= 64 ? 64 : (TC3_NACC * 16 <= 128 ? 128 : 256));
constexpr int TC3_SMEM = TC3_NS * TC_STAGE + 1024;

__device__ __forceinline__ float tf32_trunc(float x) { return __uint_as_float(__float_as_uint(x) & 0xFFFFE000u); }

__global__ void __launch_bounds__(kThreads) k_gemm_tc3(const int32_t* __restrict__ blk_sub,
                                                       const int32_t* __restrict__ blk_row0,
                                                       const SubLayout* __restrict__ lay, int which,
                                                       const CUtensorMap* __restrict__ maps, int nrhs,
                                                       const float* __restrict__ vloc, double* __restrict__ y,
                                                       const int* __restrict__ done, int* __restrict__ err) {
  if (*done) return;
  extern __shared__ __align__(1024) unsigned char tc_smem_dyn[];
  unsigned char* smem = tc_smem_dyn + ((1024 - (su32(tc_smem_dyn) & 1023)) & 1023);
  __shared__ uint64_t full[TC3_NS], mdone[TC3_NS];
  __shared__ uint32_t tmem_base;
  const int s_id = blk_sub[blockIdx.x];
  const int r0 = blk_row0[blockIdx.x];
  const SubLayout L = lay[s_id];
  const int m = which == 0 ? L.nbp : L.nbp + L.k;
  const CUtensorMap* tm = maps + s_id;
  const int tid = threadIdx.x, wid = tid >> 5, lane = tid & 31;
  if (which == 0 && r0 == 0)
    for (int idx = tid; idx < L.k * nrhs; idx += blockDim.x) y[(size_t)(L.boff + L.nbp) * nrhs + idx] = 0.0;
  if (wid == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&tmem_base)),
                 "r"(TC3_TCOLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    for (int i = 0; i < TC3_NS; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&mdone[i], 1);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(tm) : "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;
  const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((16u >> 3) << 17) | ((128u >> 4) << 24);
  const int nk = (m + 31) / 32;
  // chunk kc2 -> stage kc2 % NS: box (32 columns from kc2 * 32, 128 rows from
  // r0); the x coordinate is a multiple of 32 floats (128 bytes)
  auto issue = [&](int kc2) {
    const int st = kc2 % TC3_NS;
    mbar_expect_tx(&full[st], (uint32_t)TC_A_BYTES);
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            su32(smem + st * TC_STAGE)),
        "l"(tm), "r"(kc2 * 32), "r"(r0), "r"(su32(&full[st]))
        : "memory");
  };
  if (tid == 0)
    for (int j = 0; j < TC3_NS && j < nk; ++j) issue(j);
  int issued = min(TC3_NS, nk);
  float4 rb = make_float4(0.f, 0.f, 0.f, 0.f);
  auto load_b = [&](int kc2) {
    if (tid < 16 * 8) {
      const int n = tid >> 3, c = tid & 7, k0 = kc2 * 32;
      float v4[4];
      for (int e = 0; e < 4; ++e) {
        const int kk = k0 + 4 * c + e;
        v4[e] = (kk < m && n < nrhs) ? vloc[(size_t)(L.boff + kk) * nrhs + n] : 0.f;
      }
      rb = make_float4(v4[0], v4[1], v4[2], v4[3]);
    }
  };
  if (nk > 0) load_b(0);
  bool timed_out = false;
  int kc = 0, n_mma = 0;
  for (; kc < nk; ++kc) {
    const int st = kc % TC3_NS;
    const float4 cb = rb;
    if (kc + 1 < nk) load_b(kc + 1);
    if (!mbar_wait_bounded(&full[st], (uint32_t)(kc / TC3_NS) & 1u)) timed_out = true;
    unsigned char* Ahi = smem + st * TC_STAGE;
    unsigned char* Alo = Ahi + TC_A_BYTES;
    unsigned char* Bhi = Ahi + 2 * TC_A_BYTES;
    unsigned char* Blo = Bhi + TC_B_BYTES;
    if (!timed_out) {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int off = (tid + q * kThreads) * 16;
        const float4 x = *reinterpret_cast<const float4*>(Ahi + off);
        const float4 l = make_float4(x.x - tf32_trunc(x.x), x.y - tf32_trunc(x.y), x.z - tf32_trunc(x.z),
                                     x.w - tf32_trunc(x.w));
        *reinterpret_cast<float4*>(Alo + off) = l;
      }
      if (tid < 16 * 8) {
        const int n = tid >> 3, c = tid & 7;
        const float4 l = make_float4(cb.x - tf32_trunc(cb.x), cb.y - tf32_trunc(cb.y), cb.z - tf32_trunc(cb.z),
                                     cb.w - tf32_trunc(cb.w));
        *reinterpret_cast<float4*>(Bhi + sw_off(n, c)) = cb;
        *reinterpret_cast<float4*>(Blo + sw_off(n, c)) = l;
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    timed_out = __syncthreads_or(timed_out ? 1 : 0) != 0;
    if (timed_out) break;
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      for (int j = 0; j < 4; ++j) {
        const uint64_t ah = sw128_desc(Ahi + 32 * j), al = sw128_desc(Alo + 32 * j);
        const uint64_t bh = sw128_desc(Bhi + 32 * j), bl = sw128_desc(Blo + 32 * j);
        const int a0 = (3 * j) % TC3_NACC, a1 = (3 * j + 1) % TC3_NACC, a2 = (3 * j + 2) % TC3_NACC;
        // an accumulator is initialised by its first product of the first chunk
        const uint32_t f0 = (kc > 0 || 3 * j >= TC3_NACC) ? 1u : 0u;
        const uint32_t f1 = (kc > 0 || 3 * j + 1 >= TC3_NACC) ? 1u : 0u;
        const uint32_t f2 = (kc > 0 || 3 * j + 2 >= TC3_NACC) ? 1u : 0u;
        tc_mma(tmem + 16u * a0, ah, bh, idesc, f0);
        tc_mma(tmem + 16u * a1, ah, bl, idesc, f1);
        tc_mma(tmem + 16u * a2, al, bh, idesc, f2);
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       su32(&mdone[st]))
                   : "memory");
      if (kc >= 1 && kc - 1 + TC3_NS < nk) {
        if (mbar_wait_bounded(&mdone[(kc - 1) % TC3_NS], (uint32_t)((kc - 1) / TC3_NS) & 1u))
          issue(kc - 1 + TC3_NS);
        else
          atomicExch(err, 1);
      }
    }
    if (kc >= 1 && kc - 1 + TC3_NS < nk) issued = kc + TC3_NS;
    n_mma = kc + 1;
  }
  // drain: loads issued but not consumed (only after a timeout), then the
  // last MMA groups, each with its own bounded wait
  bool drained = true;
  if (tid == 0)
    for (int j = kc; j < issued; ++j)
      if (!mbar_wait_bounded(&full[j % TC3_NS], (uint32_t)(j / TC3_NS) & 1u)) drained = false;
  for (int j = max(0, n_mma - TC3_NS); j < n_mma; ++j)
    if (!mbar_wait_bounded(&mdone[j % TC3_NS], (uint32_t)(j / TC3_NS) & 1u)) drained = false;
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if ((timed_out || !drained) && lane == 0) atomicExch(err, 1);
  if (wid < 4) {
    float acc[16];
#pragma unroll
    for (int n = 0; n < 16; ++n) acc[n] = 0.f;
    for (int a = 0; a < TC3_NACC; ++a) {
      uint32_t r[16];
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
            "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
          : "r"(tmem + ((uint32_t)(wid * 32) << 16) + 16u * (uint32_t)a));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
      for (int n = 0; n < 16; ++n) acc[n] += __uint_as_float(r[n]);
    }
    const int row = r0 + wid * 32 + lane;
    if (row < m && !timed_out && drained)
      for (int n = 0; n < nrhs; ++n) y[(size_t)(L.boff + row) * nrhs + n] = (double)acc[n];
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (wid == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC3_TCOLS) : "memory");
}

// Warp-specialised TMA-fed variant: the same stages, operands and products
// as k_gemm_tc3, but the roles run concurrently and meet only on per-stage
// mbarriers, with no CTA barrier per chunk: warp 0 (one lane) issues the
// tensor-map loads as soon as a stage is free (empty), warp 1 (one lane)
// issues the MMAs of a chunk once its tails are ready and commits them to the
// stage's empty barrier, warps 4..7 wait for a stage's tile (full), write
// the tails and the V tile and arrive on ready (one arrival per warp).  Any
// bounded wait that runs out sets a shared abort flag that ends every role's
// loop; the producer then waits (bounded) for its own loads in flight and
// the MMA lane for its last commit before tensor memory is freed.  The
// main-loop waits give up after *spin_cycles SM clock cycles (the context's
// spin timeout); those drain waits keep a fixed 2e8-cycle budget, so every
// load and MMA issued has completed before tensor memory is released.
constexpr int TC4_TCOLS = 64;  // three 16-column accumulators

// Main-loop wait: gives up after `budget` SM clock cycles (the context's spin
// timeout; checked before every try, so a zero budget gives up at once) or
// when another role has aborted.
__device__ __forceinline__ bool wait_or_abort(uint64_t* b, uint32_t par, volatile int* abort_flag, long long budget) {
  const long long t0 = clock64();
  for (;;) {
    if (*abort_flag) return false;
    if (clock64() - t0 >= budget) {
      *abort_flag = 1;
      return false;
    }
    if (mbar_try(b, par)) return true;
  }
}

template <int NS>
__global__ void __launch_bounds__(kThreads) k_gemm_tc4(const int32_t* __restrict__ blk_sub,
                                                       const int32_t* __restrict__ blk_row0,
                                                       const SubLayout* __restrict__ lay, int which,
                                                       const CUtensorMap* __restrict__ maps, int nrhs,
                                                       const float* __restrict__ vloc, double* __restrict__ y,
                                                       const int* __restrict__ done, int* __restrict__ err,
                                                       const unsigned long long* __restrict__ spin_cycles) {
  if (*done) return;
  extern __shared__ __align__(1024) unsigned char tc_smem_dyn[];
  unsigned char* smem = tc_smem_dyn + ((1024 - (su32(tc_smem_dyn) & 1023)) & 1023);
  __shared__ uint64_t full[NS], ready[NS], empty[NS];
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag;
  const int s_id = blk_sub[blockIdx.x];
  const int r0 = blk_row0[blockIdx.x];
  const SubLayout L = lay[s_id];
  const int m = which == 0 ? L.nbp : L.nbp + L.k;
  const CUtensorMap* tm = maps + s_id;
  const int tid = threadIdx.x, wid = tid >> 5, lane = tid & 31;
  if (which == 0 && r0 == 0)
    for (int idx = tid; idx < L.k * nrhs; idx += blockDim.x) y[(size_t)(L.boff + L.nbp) * nrhs + idx] = 0.0;
  if (wid == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&tmem_base)),
                 "r"(TC4_TCOLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    abort_flag = 0;
    for (int i = 0; i < NS; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&ready[i], 4);
      mbar_init(&empty[i], 1);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(tm) : "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;
  const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((16u >> 3) << 17) | ((128u >> 4) << 24);
  const int nk = (m + 31) / 32;
  volatile int* ab = &abort_flag;
  const long long budget = (long long)*spin_cycles;
  if (wid == 0) {
    if (lane == 0) {  // producer: chunk kc -> stage kc % NS once the MMAs of chunk kc - NS are done
      int issued = 0;
      for (int kc = 0; kc < nk; ++kc) {
        const int st = kc % NS;
        if (kc >= NS && !wait_or_abort(&empty[st], (uint32_t)((kc / NS) - 1) & 1u, ab, budget)) break;
        mbar_expect_tx(&full[st], (uint32_t)TC_A_BYTES);
        asm volatile(
            "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
            "[%4];" ::"r"(su32(smem + st * TC_STAGE)),
            "l"(tm), "r"(kc * 32), "r"(r0), "r"(su32(&full[st]))
            : "memory");
        issued = kc + 1;
      }
      for (int j = max(0, issued - NS); j < issued; ++j)
        if (!mbar_wait_bounded(&full[j % NS], (uint32_t)(j / NS) & 1u)) atomicExch(err, 1);
    }
    __syncwarp();
  } else if (wid == 1) {
    if (lane == 0) {  // MMA issuer
      int n_mma = 0;
      for (int kc = 0; kc < nk; ++kc) {
        const int st = kc % NS;
        if (!wait_or_abort(&ready[st], (uint32_t)(kc / NS) & 1u, ab, budget)) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        unsigned char* Ahi = smem + st * TC_STAGE;
        unsigned char* Alo = Ahi + TC_A_BYTES;
        unsigned char* Bhi = Ahi + 2 * TC_A_BYTES;
        unsigned char* Blo = Bhi + TC_B_BYTES;
        for (int j = 0; j < 4; ++j) {
          const uint64_t ah = sw128_desc(Ahi + 32 * j), al = sw128_desc(Alo + 32 * j);
          const uint64_t bh = sw128_desc(Bhi + 32 * j), bl = sw128_desc(Blo + 32 * j);
          const uint32_t f = (kc > 0 || j > 0) ? 1u : 0u;
          tc_mma(tmem, ah, bh, idesc, f);
          tc_mma(tmem + 16u, ah, bl, idesc, f);
          tc_mma(tmem + 32u, al, bh, idesc, f);
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         su32(&empty[st]))
                     : "memory");
        n_mma = kc + 1;
      }
      if (n_mma > 0 && !mbar_wait_bounded(&empty[(n_mma - 1) % NS], (uint32_t)((n_mma - 1) / NS) & 1u))
        atomicExch(err, 1);
    }
    __syncwarp();
  } else if (wid >= 4) {  // tail workers (128 threads)
    const int t = tid - 128;
    float4 rb = make_float4(0.f, 0.f, 0.f, 0.f);
    auto load_b = [&](int kc2) {
      const int n = t >> 3, c = t & 7, k0 = kc2 * 32;
      float v4[4];
      for (int e = 0; e < 4; ++e) {
        const int kk = k0 + 4 * c + e;
        v4[e] = (kk < m && n < nrhs) ? vloc[(size_t)(L.boff + kk) * nrhs + n] : 0.f;
      }
      rb = make_float4(v4[0], v4[1], v4[2], v4[3]);
    };
    if (nk > 0) load_b(0);
    for (int kc = 0; kc < nk; ++kc) {
      const int st = kc % NS;
      const float4 cb = rb;
      if (kc + 1 < nk) load_b(kc + 1);
      if (!wait_or_abort(&full[st], (uint32_t)(kc / NS) & 1u, ab, budget)) break;
      unsigned char* Ahi = smem + st * TC_STAGE;
      unsigned char* Alo = Ahi + TC_A_BYTES;
      unsigned char* Bhi = Ahi + 2 * TC_A_BYTES;
      unsigned char* Blo = Bhi + TC_B_BYTES;
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int off = (t + q * 128) * 16;
        const float4 x = *reinterpret_cast<const float4*>(Ahi + off);
        *reinterpret_cast<float4*>(Alo + off) = make_float4(x.x - tf32_trunc(x.x), x.y - tf32_trunc(x.y),
                                                            x.z - tf32_trunc(x.z), x.w - tf32_trunc(x.w));
      }
      {
        const int n = t >> 3, c = t & 7;
        *reinterpret_cast<float4*>(Bhi + sw_off(n, c)) = cb;
        *reinterpret_cast<float4*>(Blo + sw_off(n, c)) = make_float4(
            cb.x - tf32_trunc(cb.x), cb.y - tf32_trunc(cb.y), cb.z - tf32_trunc(cb.z), cb.w - tf32_trunc(cb.w));
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(&ready[st])) : "memory");
    }
  }
  // the epilogue warps wait for the last MMA group (issued after every earlier one completed)
  bool ok = true;
  if (wid >= 4 && nk > 0) {
    const int j = nk - 1;
    const long long t0 = clock64();
    while (!mbar_try(&empty[j % NS], (uint32_t)(j / NS) & 1u))
      if (*ab || clock64() - t0 > 200000000LL) {
        ok = false;
        break;
      }
  }
  if (*ab) ok = false;
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (wid >= 4) {
    if (!ok && lane == 0) atomicExch(err, 1);
    const int w4 = wid - 4;
    float acc[16];
#pragma unroll
    for (int n = 0; n < 16; ++n) acc[n] = 0.f;
    for (int a = 0; a < 3; ++a) {
      uint32_t r[16];
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
            "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
          : "r"(tmem + ((uint32_t)(w4 * 32) << 16) + 16u * (uint32_t)a));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
      for (int n = 0; n < 16; ++n) acc[n] += __uint_as_float(r[n]);
    }
    const int row = r0 + w4 * 32 + lane;
    if (row < m && ok)
      for (int n = 0; n < nrhs; ++n) y[(size_t)(L.boff + row) * nrhs + n] = (double)acc[n];
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (wid == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC4_TCOLS) : "memory");
}

// Persistent warp-specialised tensor-core block GEMM: a fixed grid walks the
// 128-row tiles round-robin, and the K-chunk pipeline runs on across tile
// boundaries, so the per-tile costs of the one-tile kernel (tensor-memory
// allocation, barrier set-up, pipeline fill, an epilogue that nothing
// overlaps) are paid once per CTA.  The raw A chunks (16 KB, the TF32 head
// read by the MMAs straight from the copy) live in a ring of R slots, the
// TF32 tails of A and B (20 KB) in a separate ring of Q slots, so that many
// copies are in flight while only a few tails exist.  Roles: warp 0 lane 0
// issues the tensor-map copies of A, warp 1 lane 0 the MMAs, warps 4-7 load
// the B chunk and write the tails, warps 8-11 (one per tensor-memory lane
// quadrant) drain the accumulators into y.  Two accumulator sets alternate
// between tiles: the MMAs of tile i + 1 run while the epilogue reads tile i.
// Every wait is bounded; a wait that runs out stops all roles, the copies and
// MMAs already issued are drained, and *err is set.
constexpr int TC5_THREADS = 384;
constexpr int TC5_TCOLS = 128;  // two accumulator sets of 3 x 16 columns, 64 apart
constexpr int TC5_OP = TC_A_BYTES + 2 * TC_B_BYTES;  // A tail, B head and tail
__host__ __device__ constexpr int tc5_smem(int R, int Q) { return R * TC_A_BYTES + Q * TC5_OP + 1024; }

template <int R, int Q>
__global__ void __launch_bounds__(TC5_THREADS) k_gemm_tc5(const int32_t* __restrict__ blk_sub,
                                                         const int32_t* __restrict__ blk_row0, int n_tiles,
                                                         const SubLayout* __restrict__ lay, int which,
                                                         const CUtensorMap* __restrict__ maps, int nrhs,
                                                         const float* __restrict__ vloc, double* __restrict__ y,
                                                         const int* __restrict__ done, int* __restrict__ err,
                                                         const unsigned long long* __restrict__ spin_cycles) {
  if (*done) return;
  extern __shared__ __align__(1024) unsigned char tc_smem_dyn[];
  unsigned char* smem = tc_smem_dyn + ((1024 - (su32(tc_smem_dyn) & 1023)) & 1023);
  unsigned char* raw = smem;                      // R x 16 KB
  unsigned char* ops = smem + R * TC_A_BYTES;     // Q x (A tail, B head, B tail)
  __shared__ uint64_t rfull[R], rempty[R], oready[Q], oempty[Q], tfull[2], tempty[2];
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag;
  const int tid = threadIdx.x, wid = tid >> 5, lane = tid & 31;
  if (wid == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&tmem_base)),
                 "r"(TC5_TCOLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    abort_flag = 0;
    for (int i = 0; i < R; ++i) {
      mbar_init(&rfull[i], 1);
      mbar_init(&rempty[i], 1);
    }
    for (int i = 0; i < Q; ++i) {
      mbar_init(&oready[i], 4);
      mbar_init(&oempty[i], 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&tfull[i], 1);
      mbar_init(&tempty[i], 4);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;
  const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((16u >> 3) << 17) | ((128u >> 4) << 24);
  volatile int* ab = &abort_flag;
  const long long budget = (long long)*spin_cycles;
  auto rows_of = [&](const SubLayout& L) { return which == 0 ? L.nbp : L.nbp + L.k; };
  if (wid == 0) {
    if (lane == 0) {  // producer: chunk g -> raw slot g % R once the MMAs of chunk g - R are done
      int g = 0, prev = -1;
      bool stop = false;
      for (int t = blockIdx.x; t < n_tiles && !stop; t += gridDim.x) {
        const int s_id = blk_sub[t], r0 = blk_row0[t];
        const int nk = (rows_of(lay[s_id]) + 31) / 32;
        const CUtensorMap* tm = maps + s_id;
        if (s_id != prev) {
          asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(tm) : "memory");
          prev = s_id;
        }
        for (int kc = 0; kc < nk; ++kc) {
          const int st = g % R;
          if (g >= R && !wait_or_abort(&rempty[st], (uint32_t)((g / R) - 1) & 1u, ab, budget)) {
            stop = true;
            break;
          }
          mbar_expect_tx(&rfull[st], (uint32_t)TC_A_BYTES);
          asm volatile(
              "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
              "[%4];" ::"r"(su32(raw + st * TC_A_BYTES)),
              "l"(tm), "r"(kc * 32), "r"(r0), "r"(su32(&rfull[st]))
              : "memory");
          ++g;
        }
      }
      // drain: every copy issued has landed before shared memory is released
      for (int j = max(0, g - R); j < g; ++j)
        if (!mbar_wait_bounded(&rfull[j % R], (uint32_t)(j / R) & 1u)) atomicExch(err, 1);
    }
    __syncwarp();
  } else if (wid == 1) {
    if (lane == 0) {  // MMA issuer
      int g = 0, n_commit = 0, i = 0;
      bool stop = false;
      for (int t = blockIdx.x; t < n_tiles && !stop; t += gridDim.x, ++i) {
        const int nk = (rows_of(lay[blk_sub[t]]) + 31) / 32;
        const int abuf = i & 1;
        if (i >= 2 && !wait_or_abort(&tempty[abuf], (uint32_t)((i / 2) - 1) & 1u, ab, budget)) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t acc = tmem + 64u * (uint32_t)abuf;
        for (int kc = 0; kc < nk; ++kc) {
          const int rs = g % R, os = g % Q;
          // the tails are written after the copy landed: one wait covers both
          if (!wait_or_abort(&oready[os], (uint32_t)(g / Q) & 1u, ab, budget)) {
            stop = true;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          unsigned char* Ahi = raw + rs * TC_A_BYTES;
          unsigned char* Alo = ops + os * TC5_OP;
          unsigned char* Bhi = Alo + TC_A_BYTES;
          unsigned char* Blo = Bhi + TC_B_BYTES;
          for (int j = 0; j < 4; ++j) {
            const uint64_t ah = sw128_desc(Ahi + 32 * j), al = sw128_desc(Alo + 32 * j);
            const uint64_t bh = sw128_desc(Bhi + 32 * j), bl = sw128_desc(Blo + 32 * j);
            const uint32_t f = (kc > 0 || j > 0) ? 1u : 0u;
            tc_mma(acc, ah, bh, idesc, f);
            tc_mma(acc + 16u, ah, bl, idesc, f);
            tc_mma(acc + 32u, al, bh, idesc, f);
          }
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                           su32(&rempty[rs]))
                       : "memory");
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                           su32(&oempty[os]))
                       : "memory");
          ++g;
          n_commit = g;
        }
        if (stop) break;
        // the tile's accumulator is complete once every MMA issued so far is
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         su32(&tfull[abuf]))
                     : "memory");
      }
      if (n_commit > 0 && !mbar_wait_bounded(&oempty[(n_commit - 1) % Q], (uint32_t)((n_commit - 1) / Q) & 1u))
        atomicExch(err, 1);
    }
    __syncwarp();
  } else if (wid >= 4 && wid < 8) {  // A and B tails, B chunk loads
    const int t4 = tid - 128;
    int g = 0;
    bool stop = false;
    for (int t = blockIdx.x; t < n_tiles && !stop; t += gridDim.x) {
      const SubLayout L = lay[blk_sub[t]];
      const int m = rows_of(L);
      const int nk = (m + 31) / 32;
      float4 rb = make_float4(0.f, 0.f, 0.f, 0.f);
      auto load_b = [&](int kc2) {
        const int n = t4 >> 3, c = t4 & 7, k0 = kc2 * 32;
        float v4[4];
        for (int e = 0; e < 4; ++e) {
          const int kk = k0 + 4 * c + e;
          v4[e] = (kk < m && n < nrhs) ? vloc[(size_t)(L.boff + kk) * nrhs + n] : 0.f;
        }
        rb = make_float4(v4[0], v4[1], v4[2], v4[3]);
      };
      if (nk > 0) load_b(0);
      for (int kc = 0; kc < nk; ++kc) {
        const int rs = g % R, os = g % Q;
        const float4 cb = rb;
        if (kc + 1 < nk) load_b(kc + 1);
        if (!wait_or_abort(&rfull[rs], (uint32_t)(g / R) & 1u, ab, budget)) {
          stop = true;
          break;
        }
        if (g >= Q && !wait_or_abort(&oempty[os], (uint32_t)((g / Q) - 1) & 1u, ab, budget)) {
          stop = true;
          break;
        }
        unsigned char* Ahi = raw + rs * TC_A_BYTES;
        unsigned char* Alo = ops + os * TC5_OP;
        unsigned char* Bhi = Alo + TC_A_BYTES;
        unsigned char* Blo = Bhi + TC_B_BYTES;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int off = (t4 + q * 128) * 16;
          const float4 x = *reinterpret_cast<const float4*>(Ahi + off);
          *reinterpret_cast<float4*>(Alo + off) = make_float4(x.x - tf32_trunc(x.x), x.y - tf32_trunc(x.y),
                                                              x.z - tf32_trunc(x.z), x.w - tf32_trunc(x.w));
        }
        {
          const int n = t4 >> 3, c = t4 & 7;
          *reinterpret_cast<float4*>(Bhi + sw_off(n, c)) = cb;
          *reinterpret_cast<float4*>(Blo + sw_off(n, c)) = make_float4(
              cb.x - tf32_trunc(cb.x), cb.y - tf32_trunc(cb.y), cb.z - tf32_trunc(cb.z), cb.w - tf32_trunc(cb.w));
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(&oready[os])) : "memory");
        ++g;
      }
    }
  } else if (wid >= 8) {  // epilogue: warp 8 + q reads tensor-memory lanes 32 q .. 32 q + 31
    const int q = wid - 8, te = tid - 256;
    int i = 0;
    for (int t = blockIdx.x; t < n_tiles; t += gridDim.x, ++i) {
      const SubLayout L = lay[blk_sub[t]];
      const int r0 = blk_row0[t], m = rows_of(L);
      if (which == 0 && r0 == 0)  // the fixing rows of F_i's output are zero
        for (int idx = te; idx < L.k * nrhs; idx += 128) y[(size_t)(L.boff + L.nbp) * nrhs + idx] = 0.0;
      const int abuf = i & 1;
      if (!wait_or_abort(&tfull[abuf], (uint32_t)(i / 2) & 1u, ab, budget)) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      float acc[16];
#pragma unroll
      for (int n = 0; n < 16; ++n) acc[n] = 0.f;
      for (int a = 0; a < 3; ++a) {
        uint32_t r[16];
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
            : "r"(tmem + ((uint32_t)(q * 32) << 16) + 64u * (uint32_t)abuf + 16u * (uint32_t)a));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int n = 0; n < 16; ++n) acc[n] += __uint_as_float(r[n]);
      }
      // the accumulator set is free again for tile i + 2
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(&tempty[abuf])) : "memory");
      const int row = r0 + q * 32 + lane;
      if (row < m)
        for (int n = 0; n < nrhs; ++n) y[(size_t)(L.boff + row) * nrhs + n] = (double)acc[n];
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (*ab) {
    if (tid == 0) atomicExch(err, 1);
  }
  if (wid == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC5_TCOLS) : "memory");
}

template <int R, int Q>
void launch_tc5(int ctas_per_sm, const GemvCfg& cfg, const SubLayout* lay, int which, const CUtensorMap* maps, int nrhs,
                const float* vloc, double* y, const int* done, int* err, const unsigned long long* spin_cycles,
                cudaStream_t st) {
  static int n_sm = 0;
  if (!n_sm) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    if (n_sm <= 0) n_sm = 1;
    cudaFuncSetAttribute(k_gemm_tc5<R, Q>, cudaFuncAttributeMaxDynamicSharedMemorySize, tc5_smem(R, Q));
  }
  const int grid = std::min(cfg.n_blocks, ctas_per_sm * n_sm);
  if (grid > 0)
    k_gemm_tc5<R, Q><<<grid, TC5_THREADS, tc5_smem(R, Q), st>>>(cfg.blk_sub, cfg.blk_row0, cfg.n_blocks, lay, which,
                                                               maps, nrhs, vloc, y, done, err, spin_cycles);
}

inline int grid_for(long n) {
  long b = (n + kThreads - 1) / kThreads;
  if (b < 1) b = 1;
  if (b > 65535) b = 65535;
  return (int)b;
}

template <typename T, int R>
void launch_gemm_t(const GemvCfg& cfg, const SubLayout* lay, int which, const T* M, int nrhs, const T* vloc, double* y,
                   int max_m, const int* done, cudaStream_t st) {
  const size_t smem = (size_t)((max_m + 3) & ~3) * nrhs * sizeof(T);
  if (smem > 48 * 1024) cudaFuncSetAttribute(k_gemm_loc<T, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k_gemm_loc<T, R><<<cfg.n_blocks, kThreads, smem, st>>>(cfg.blk_sub, cfg.blk_row0, cfg.rpc, lay, which, M, nrhs, vloc,
                                                        y, done);
}

}  // namespace

void launch_gather_m(const Maps& mp, int nrhs, const double* x, const double* wv, void* y, int f32, const int* done,
                     cudaStream_t st) {
  if (f32)
    k_gather_m<float><<<grid_for(mp.nb_total), kThreads, 0, st>>>(mp, nrhs, x, wv, static_cast<float*>(y), done);
  else
    k_gather_m<double><<<grid_for(mp.nb_total), kThreads, 0, st>>>(mp, nrhs, x, wv, static_cast<double*>(y), done);
}

void launch_gemm_loc(const GemvCfg& cfg, const SubLayout* lay, int which, const void* M, int f32, int nrhs,
                     const void* vloc, double* y, int max_m, const int* done, cudaStream_t st) {
  if (f32) {
    if (cfg.R >= 4)
      launch_gemm_t<float, 4>(cfg, lay, which, static_cast<const float*>(M), nrhs, static_cast<const float*>(vloc), y,
                              max_m, done, st);
    else if (cfg.R >= 2)
      launch_gemm_t<float, 2>(cfg, lay, which, static_cast<const float*>(M), nrhs, static_cast<const float*>(vloc), y,
                              max_m, done, st);
    else
      launch_gemm_t<float, 1>(cfg, lay, which, static_cast<const float*>(M), nrhs, static_cast<const float*>(vloc), y,
                              max_m, done, st);
  } else {
    if (cfg.R >= 2)
      launch_gemm_t<double, 2>(cfg, lay, which, static_cast<const double*>(M), nrhs, static_cast<const double*>(vloc), y,
                               max_m, done, st);
    else
      launch_gemm_t<double, 1>(cfg, lay, which, static_cast<const double*>(M), nrhs, static_cast<const double*>(vloc), y,
                               max_m, done, st);
  }
}

void launch_gemm_tc(const GemvCfg& cfg, const SubLayout* lay, int which, const float* M, int nrhs, const float* vloc,
                    double* y, const int* done, int* err, int variant, const void* tmaps,
                    const unsigned long long* spin_cycles, cudaStream_t st) {
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_gemm_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM);
    cudaFuncSetAttribute(k_gemm_tc2, cudaFuncAttributeMaxDynamicSharedMemorySize, TC2_SMEM);
    cudaFuncSetAttribute(k_gemm_tc3, cudaFuncAttributeMaxDynamicSharedMemorySize, TC3_SMEM);
    attr = true;
  }
  if (variant >= 6 && variant <= 8) {
    const CUtensorMap* mp = static_cast<const CUtensorMap*>(tmaps);
    if (variant == 6)  // 3 raw + 2 tail slots, two CTAs per SM
      launch_tc5<3, 2>(2, cfg, lay, which, mp, nrhs, vloc, y, done, err, spin_cycles, st);
    else if (variant == 7)  // 3 raw + 3 tail slots, two CTAs per SM
      launch_tc5<3, 3>(2, cfg, lay, which, mp, nrhs, vloc, y, done, err, spin_cycles, st);
    else  // 2 raw + 2 tail slots, three CTAs per SM
      launch_tc5<2, 2>(3, cfg, lay, which, mp, nrhs, vloc, y, done, err, spin_cycles, st);
    return;
  }
  if (variant == 4 || variant == 5) {
    static bool attr4 = false;
    if (!attr4) {
      cudaFuncSetAttribute(k_gemm_tc4<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, 3 * TC_STAGE + 1024);
      cudaFuncSetAttribute(k_gemm_tc4<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * TC_STAGE + 1024);
      attr4 = true;
    }
    const CUtensorMap* mp = static_cast<const CUtensorMap*>(tmaps);
    if (variant == 4)
      k_gemm_tc4<3><<<cfg.n_blocks, kThreads, 3 * TC_STAGE + 1024, st>>>(cfg.blk_sub, cfg.blk_row0, lay, which, mp,
                                                                        nrhs, vloc, y, done, err, spin_cycles);
    else
      k_gemm_tc4<2><<<cfg.n_blocks, kThreads, 2 * TC_STAGE + 1024, st>>>(cfg.blk_sub, cfg.blk_row0, lay, which, mp,
                                                                        nrhs, vloc, y, done, err, spin_cycles);
  } else if (variant == 3)
    k_gemm_tc3<<<cfg.n_blocks, kThreads, TC3_SMEM, st>>>(cfg.blk_sub, cfg.blk_row0, lay, which,
                                                         static_cast<const CUtensorMap*>(tmaps), nrhs, vloc, y, done,
                                                         err);
  else if (variant == 2)
    k_gemm_tc2<<<cfg.n_blocks, kThreads, TC2_SMEM, st>>>(cfg.blk_sub, cfg.blk_row0, lay, which, M, nrhs, vloc, y, done,
                                                         err);
  else
    k_gemm_tc<<<cfg.n_blocks, kThreads, TC_SMEM, st>>>(cfg.blk_sub, cfg.blk_row0, lay, which, M, nrhs, vloc, y, done,
                                                       err);
}

void launch_scatter_m(const Maps& mp, int nrhs, const double* y, const double* wv, double* q, const double* a,
                      double* partial, const int* done, cudaStream_t st) {
  k_scatter_m<<<kPartials, kThreads, 0, st>>>(mp, nrhs, y, wv, q, a, partial, done);
}

void launch_project_m(int n_chunks, const int32_t* chunk_sub, const int32_t* chunk_p0, const int32_t* sub_chunk_ptr,
                      const int32_t* col_sub, const SubLayout* lay, const double* R, const Maps& mp, int nrhs, int cd,
                      const double* Ginv, const double* x, const double* q, const PcgScalarsM* sc, double* gpart,
                      double* g, double* c, const int* done, cudaStream_t st) {
  if (cd <= 0 || n_chunks <= 0) return;
  k_gtv_part_m<<<n_chunks, kThreads, 0, st>>>(chunk_sub, chunk_p0, lay, R, mp, nrhs, x, gpart, q, sc, done);
  if (!Ginv) return;  // sparse coarse problem: the caller solves from the partials
  k_gsum_m<<<grid_for((long)cd * nrhs), kThreads, 0, st>>>(cd, nrhs, gpart, sub_chunk_ptr, col_sub, lay, g, done);
  const int warps = cd < 2432 ? cd : 2432;
  k_coarse_gemm_m<<<(warps * 32 + kThreads - 1) / kThreads, kThreads, 0, st>>>(cd, nrhs, Ginv, g, c, done);
}

void launch_expand_m(const Maps& mp, const SubLayout* lay, const double* R, int nrhs, int has_coarse, const double* v,
                     const double* c, double* out, const double* a, double* partial, double* r_upd, double* lam,
                     const double* p, const double* q, const PcgScalarsM* sc, const int* done, cudaStream_t st) {
  k_expand_m<<<kPartials, kThreads, 0, st>>>(mp, lay, R, nrhs, has_coarse, v, c, out, a, partial, r_upd, lam, p, q, sc,
                                             done);
}

void launch_axpby_rho_m(int n, int nrhs, double* p, const double* y, PcgScalarsM* s, const double* partial,
                        cudaStream_t st) {
  k_axpby_rho_m<<<grid_for(n), kThreads, 0, st>>>(n, nrhs, p, y, s, partial);
}

void launch_alpha_m(int nrhs, PcgScalarsM* s, const double* partial, double* alpha_hist, cudaStream_t st) {
  k_alpha_m<<<1, kThreads, 0, st>>>(nrhs, s, partial, alpha_hist);
}

void launch_conv_m(int nrhs, PcgScalarsM* s, const double* partial, int first, cudaStream_t st) {
  k_conv_m<<<1, kThreads, 0, st>>>(nrhs, s, partial, first);
}

void launch_spmv_lump_m(int n_rows, int nrhs, const int32_t* ptr, const int32_t* col, const double* val,
                        const double* v, double* y, const int* done, cudaStream_t st) {
  k_spmv_lump_m<<<grid_for((long)n_rows * nrhs), kThreads, 0, st>>>(n_rows, nrhs, ptr, col, val, v, y, done);
}

void launch_col_get(int n, int nrhs, int k, const double* blk, double* v, cudaStream_t st) {
  k_col_get<<<grid_for(n), kThreads, 0, st>>>(n, nrhs, k, blk, v);
}

void launch_col_set(int n, int nrhs, int k, double scale, const double* v, double* blk, cudaStream_t st) {
  k_col_set<<<grid_for(n), kThreads, 0, st>>>(n, nrhs, k, scale, v, blk);
}

}  // namespace feti
