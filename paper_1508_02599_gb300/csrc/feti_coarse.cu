// Sparse coarse problem on the device (Sec. 4.3: every projection
// P = I - G (G^T G)^-1 G^T solves with G^T G).
//
// Factorization (setup, FP64, multifrontal over the supernodes of a
// nested-dissection order of the subdomain graph, assembly level by level):
//   front of supernode s = [own columns | panel rows | w identity rows]; the
//   G^T G pair blocks are written into the fronts, each child's trailing block
//   (its update matrix) is added into its parent's front through the child's
//   index map (one launch per child slot: deterministic, no atomics), and the
//   own columns are eliminated by blocked right-looking Cholesky over all
//   rows.  Eliminating the identity rows with the rest leaves L_ss^-T there
//   (row e_i^T becomes e_i^T L_ss^-T), so the inverted diagonal blocks used
//   by the sweeps come out of the same elimination.  L_ss^-1, L_ss^-T, L_ps
//   and L_ps^T are then copied into compact row-major arrays.
// Solve (every projection, FP64): forward L y = g, backward L^T x = y as one
// kernel over a task graph: each CTA takes the next ticket, waits (bounded)
// for the tickets its task needs, runs it and publishes its flag; tasks wait
// only on lower tickets, which CTAs already running hold, so the graph
// always drains.  Flags carry an epoch, advanced by the last CTA to finish,
// so nothing is reset between launches.
#include "feti_internal.h"

#include <algorithm>

namespace feti {
namespace {

constexpr int kCT = 256;
constexpr int CNB = 32;  // column block of the front elimination
constexpr int CTT = 64;  // row tile

__global__ void k_cf_aug(const CoarseFront* __restrict__ fr, double* __restrict__ ws) {
  const CoarseFront F = fr[blockIdx.x];
  const int64_t f = F.w + F.p;
  double* A = ws + F.off;
  for (int i = threadIdx.x; i < F.w; i += blockDim.x) A[(f + i) * f + i] = 1.0;
}

// G^T G pair block b (subdomains blk_i <= blk_j): one CTA, thread per entry,
// multiplier rows in fixed order; written into the front given by place[b].
__global__ void k_cf_gtg(const int32_t* __restrict__ blk_i, const int32_t* __restrict__ blk_j,
                         const int32_t* __restrict__ blk_ptr, const int32_t* __restrict__ blk_rows,
                         const CoarsePlace* __restrict__ place, const SubLayout* __restrict__ lay,
                         const double* __restrict__ R, Maps mp, double* __restrict__ ws) {
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
  const CoarsePlace pl = place[b];
  const int row = pl.swap ? pl.row0 + c : pl.row0 + a;
  const int col = pl.swap ? pl.col0 + a : pl.col0 + c;
  ws[pl.off + (int64_t)row * pl.ld + col] = acc;
}

// Child slot `slot` of every front in the level list: parent += child's
// update matrix (lower triangle), warp per child row.
__global__ void k_cf_extend(const CoarseFront* __restrict__ fr, const CoarseChild* __restrict__ ch,
                            const int32_t* __restrict__ map, const int32_t* __restrict__ lvl, int slot,
                            double* __restrict__ ws) {
  const CoarseFront F = fr[lvl[blockIdx.y]];
  if (F.ch0 + slot >= F.ch1) return;
  const CoarseChild C = ch[F.ch0 + slot];
  const CoarseFront Fc = fr[C.c];
  const int lane = threadIdx.x & 31;
  const int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (r >= Fc.p) return;
  const int64_t fc = Fc.w + Fc.p, fp = F.w + F.p;
  const int32_t* mp = map + C.map;
  const double* U = ws + Fc.off + (Fc.w + r) * fc + Fc.w;
  double* A = ws + F.off + (int64_t)mp[r] * fp;
  for (int c = lane; c <= r; c += 32) A[mp[c]] += U[c];
}

// Rows of the front that step kb touches: [kb + nk, f + min(w, kb + nk)) —
// the identity rows of columns not yet reached are still zero there.
__global__ void k_cf_diag(const CoarseFront* __restrict__ fr, const int32_t* __restrict__ lvl, int kb,
                          double* __restrict__ ws, int* status) {
  const CoarseFront F = fr[lvl[blockIdx.y]];
  if (kb >= F.w) return;
  const int nk = min(CNB, F.w - kb);
  const int64_t ld = F.w + F.p;
  double* A = ws + F.off;
  __shared__ double D[CNB][CNB + 1];
  __shared__ int bad;
  const int tid = threadIdx.x;
  if (tid == 0) bad = 0;
  for (int idx = tid; idx < CNB * CNB; idx += blockDim.x) {
    const int i = idx / CNB, j = idx % CNB;
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
    if (tid == 0) atomicCAS(status, 0, (int)DEV_LOCAL_SINGULAR);
    return;
  }
  for (int idx = tid; idx < nk * nk; idx += blockDim.x) {
    const int i = idx / nk, j = idx % nk;
    if (j <= i) A[(kb + i) * ld + kb + j] = D[i][j];
  }
}

__global__ void k_cf_trsm(const CoarseFront* __restrict__ fr, const int32_t* __restrict__ lvl, int kb,
                          double* __restrict__ ws, const int* status) {
  if (*status) return;
  const CoarseFront F = fr[lvl[blockIdx.y]];
  if (kb >= F.w) return;
  const int nk = min(CNB, F.w - kb);
  const int64_t ld = F.w + F.p;
  const int n_act = F.w + F.p + min(F.w, kb + nk);
  const int base = kb + nk + blockIdx.x * CTT;
  if (base >= n_act) return;
  const int nr = min(CTT, n_act - base);
  double* A = ws + F.off;
  __shared__ double D[CNB][CNB + 1];
  __shared__ double Pa[CTT][CNB + 1];
  const int tid = threadIdx.x;
  for (int idx = tid; idx < CNB * CNB; idx += blockDim.x) {
    const int i = idx / CNB, j = idx % CNB;
    D[i][j] = (i < nk && j <= i) ? A[(kb + i) * ld + kb + j] : 0.0;
  }
  for (int idx = tid; idx < CTT * CNB; idx += blockDim.x) {
    const int r = idx / CNB, l = idx % CNB;
    Pa[r][l] = (r < nr && l < nk) ? A[(base + r) * ld + kb + l] : 0.0;
  }
  __syncthreads();
  if (tid < nr) {
    double xr[CNB];
#pragma unroll
    for (int j = 0; j < CNB; ++j) xr[j] = Pa[tid][j];
#pragma unroll
    for (int j = 0; j < CNB; ++j) {
      if (j < nk) {
        double v = xr[j];
#pragma unroll
        for (int l = 0; l < CNB; ++l)
          if (l < j) v -= xr[l] * D[j][l];
        xr[j] = v / D[j][j];
      }
    }
#pragma unroll
    for (int j = 0; j < CNB; ++j) Pa[tid][j] = xr[j];
  }
  __syncthreads();
  for (int idx = tid; idx < CTT * CNB; idx += blockDim.x) {
    const int r = idx / CNB, l = idx % CNB;
    if (r < nr && l < nk) A[(base + r) * ld + kb + l] = Pa[r][l];
  }
}

// Trailing update of step kb: rows [r0, n_act) x columns [r0, f), lower
// triangle, the identity rows only on the own columns; 64 x 64 tiles over
// the row-tile x column-tile rectangle (tiles above the diagonal exit).
__global__ void __launch_bounds__(kCT) k_cf_update(const CoarseFront* __restrict__ fr,
                                                   const int32_t* __restrict__ lvl, int kb,
                                                   double* __restrict__ ws, const int* status) {
  if (*status) return;
  const CoarseFront F = fr[lvl[blockIdx.y]];
  if (kb >= F.w) return;
  const int nk = min(CNB, F.w - kb);
  const int f = F.w + F.p;
  const int n_act = f + min(F.w, kb + nk);
  const int r0 = kb + nk;
  const int n_ct = (f - r0 + CTT - 1) / CTT;
  const int n_rt = (n_act - r0 + CTT - 1) / CTT;
  if (n_ct <= 0) return;
  const int b = blockIdx.x;
  if (b >= n_rt * n_ct) return;
  const int ib = r0 + (b / n_ct) * CTT, jb = r0 + (b % n_ct) * CTT;
  if (jb > ib + CTT - 1) return;
  if (ib >= f && jb >= F.w) return;
  const int64_t ld = f;
  double* A = ws + F.off;
  __shared__ double Pa[CTT][CNB + 1];
  __shared__ double Pb[CTT][CNB + 1];
  const int tid = threadIdx.x;
  for (int idx = tid; idx < CTT * CNB; idx += blockDim.x) {
    const int r = idx / CNB, l = idx % CNB;
    Pa[r][l] = (ib + r < n_act && l < nk) ? A[(ib + r) * ld + kb + l] : 0.0;
    Pb[r][l] = (jb + r < f && l < nk) ? A[(jb + r) * ld + kb + l] : 0.0;
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
      if (i < n_act && j < f && j <= i && (i < f || j < F.w)) A[i * ld + j] -= acc[a][c];
    }
}

// Compact copies: L_ss^-1 and L_ss^-T from the identity rows, L_ps and L_ps^T.
__global__ void k_cf_extract(const CoarseFront* __restrict__ fr, const double* __restrict__ ws,
                             double* __restrict__ Dm, double* __restrict__ Lm) {
  const CoarseFront F = fr[blockIdx.y];
  const int64_t f = F.w + F.p;
  const double* A = ws + F.off;
  const int64_t nd = (int64_t)F.w * F.w, nl = (int64_t)F.w * F.p;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nd + nl; e += (int64_t)gridDim.x * blockDim.x) {
    if (e < nd) {
      const int i = (int)(e / F.w), j = (int)(e % F.w);
      const double x = j >= i ? A[(f + i) * f + j] : 0.0;
      Dm[F.doff + nd + e] = x;                  // L_ss^-T (i, j)
      Dm[F.doff + (int64_t)j * F.w + i] = x;    // L_ss^-1 (j, i)
    } else {
      const int64_t q = e - nd;
      const int r = (int)(q / F.w), i = (int)(q % F.w);
      const double v = A[(F.w + r) * f + i];
      Lm[F.loff + q] = v;                        // L_ps (r, i)
      Lm[F.loff + nl + (int64_t)i * F.p + r] = v;  // L_ps^T (i, r)
    }
  }
}

__device__ __forceinline__ unsigned ld_relaxed_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_u32(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void cp_async8(void* s, const void* g) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(s);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(sa), "l"(g) : "memory");
}
__device__ __forceinline__ void cp_async4(void* s, const void* g) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(s);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(sa), "l"(g) : "memory");
}

// Stages rows [0, nr) x columns [c0, c0 + width) of a row-major global block
// (row stride gld) into shared memory (row stride coarse_odd(width)), only
// the columns with lo(r) <= c < hi(r); asynchronous (cp.async), all threads.
template <typename Lo, typename Hi>
__device__ __forceinline__ void stage(double* dst, const double* __restrict__ src, int64_t gld, int nr, int c0,
                                      int width, Lo lo, Hi hi) {
  const int n = nr * width;
  const int sld = (int)coarse_odd(width);
  for (int e = threadIdx.x; e < n; e += kCT) {
    const int r = e / width, j = e - r * width, cc = c0 + j;
    if (cc >= lo(r) && cc < hi(r)) cp_async8(dst + r * sld + j, src + (int64_t)r * gld + cc);
  }
}
__device__ __forceinline__ void stage_ints(int32_t* dst, const int32_t* __restrict__ src, int n) {
  for (int e = threadIdx.x; e < n; e += kCT) cp_async4(dst + e, src + e);
}

// Products from shared memory: for rows i in [r0, r1), the sum over j in
// [lo(i), hi(i)) of M(i)[j] v[j][k] (k < nrhs), handed to emit(i, k, value).
// Each row goes to a group of lanes: the widest power of two (up to a warp)
// with which the CTA covers every row in one pass, one lane per row for
// long lists.
template <int NR, typename Row, typename Lo, typename Hi, typename Emit>
__device__ __forceinline__ void rows_times(Row M, int r0, int r1, const double* v, int nrhs, Lo lo, Hi hi,
                                           Emit emit) {
  const int R = r1 - r0;
  int lg = 32;  // the widest group that still covers every row in one pass
  while (lg > 1 && R * lg > kCT) lg >>= 1;
  const int gid = threadIdx.x / lg, gl = threadIdx.x - gid * lg, ng = kCT / lg;
  const int passes = (R + ng - 1) / ng;
  for (int t = 0; t < passes; ++t) {
    const int i = r0 + gid + t * ng;
    const bool valid = i < r1;
    double s[NR];
#pragma unroll
    for (int k = 0; k < NR; ++k) s[k] = 0.0;
    if (valid) {
      const double* Mi = M(i);
      const int j1 = hi(i);
      for (int j = lo(i) + gl; j < j1; j += lg) {
        const double m = Mi[j];
#pragma unroll
        for (int k = 0; k < NR; ++k)
          if (k < nrhs) s[k] += m * v[j * nrhs + k];
      }
    }
    for (int off = lg >> 1; off > 0; off >>= 1)
#pragma unroll
      for (int k = 0; k < NR; ++k)
        if (k < nrhs) s[k] += __shfl_xor_sync(0xffffffffu, s[k], off);
    if (valid && gl == 0)
#pragma unroll
      for (int k = 0; k < NR; ++k)
        if (k < nrhs) emit(i, k, s[k]);
  }
}

template <int NR>
__global__ void __launch_bounds__(kCT) k_coarse_dag(CoarseDag dag, int nrhs, const double* __restrict__ g,
                                                    const double* __restrict__ partial,
                                                    const int32_t* __restrict__ sub_chunk_ptr,
                                                    const int32_t* __restrict__ col_sub,
                                                    const SubLayout* __restrict__ lay, double* __restrict__ c,
                                                    const int* __restrict__ done, int* __restrict__ err,
                                                    const unsigned long long* __restrict__ spin_cycles) {
  if (*done) return;
  extern __shared__ __align__(16) double csm[];
  __shared__ int s_ticket;
  __shared__ unsigned s_ep;
  const int tid = threadIdx.x, lane = tid & 31;
  if (tid == 0) {
    s_ticket = (int)atomicAdd(&dag.ctr[0], 1u);
    s_ep = *(volatile unsigned*)&dag.ctr[2];
  }
  __syncthreads();
  const int q = s_ticket;
  const unsigned target = s_ep + 1u;
  const CoarseTask T = dag.task[q];
  const CoarseFront F = dag.fr[T.s];
  const int w = F.w, p = F.p, f = w + p, kind = T.kind;
  const int r0 = T.r0, r1 = T.r1, nr = r1 - r0;
  const double* Dg = dag.Dm + F.doff;  // L_ss^-1, then L_ss^-T
  const double* Lg = dag.Lm + F.loff;  // L_ps, then L_ps^T
  // shared layout: staged factor block | index words | vectors (as planned)
  int64_t slab_sz;
  switch (kind) {
    case 0: slab_sz = (int64_t)nr * coarse_odd(r1); break;
    case 1: slab_sz = (int64_t)nr * coarse_odd(w); break;
    case 2: slab_sz = (int64_t)nr * coarse_odd(p); break;
    case 3: slab_sz = (int64_t)nr * coarse_odd(w - r0); break;
    case 4: slab_sz = (int64_t)w * coarse_odd(w) + (int64_t)p * coarse_odd(w); break;
    default: slab_sz = (int64_t)w * coarse_odd(p) + (int64_t)w * coarse_odd(w); break;
  }
  int g0 = 0, g1 = 0;  // front rows whose children's update rows this task gathers
  if (kind == 0) g1 = r1;
  else if (kind == 1) { g0 = w + r0; g1 = w + r1; }
  else if (kind == 4) g1 = f;
  const int32_t* gp = dag.gptr + F.gofs;
  const int gbase = g1 > g0 ? gp[g0] : 0;
  const int nsrc = g1 > g0 ? gp[g1] - gbase : 0;
  const int n_int = f + (g1 > g0 ? (g1 - g0 + 1) + nsrc : 0);
  double* slab = csm;
  int32_t* s_nat = reinterpret_cast<int32_t*>(csm + slab_sz);
  int32_t* s_gp = s_nat + f;
  int32_t* s_gs = s_gp + (g1 - g0 + 1);
  double* vec = csm + slab_sz + (n_int + 1) / 2;
  // 1. constant data into shared memory before the wait: the task's factor
  // block, the front's natural indices and the gather lists of its rows
  auto all = [](int) { return 0; };
  if (kind == 0) {
    stage(slab, Dg + (int64_t)r0 * w, w, nr, 0, r1, all, [r0](int r) { return r0 + r + 1; });
  } else if (kind == 1) {
    stage(slab, Lg + (int64_t)r0 * w, w, nr, 0, w, all, [w](int) { return w; });
  } else if (kind == 2) {
    stage(slab, Lg + (int64_t)w * p + (int64_t)r0 * p, p, nr, 0, p, all, [p](int) { return p; });
  } else if (kind == 3) {
    stage(slab, Dg + (int64_t)w * w + (int64_t)r0 * w, w, nr, r0, w - r0, [r0](int r) { return r0 + r; },
          [w](int) { return w; });
  } else if (kind == 4) {
    stage(slab, Dg, w, w, 0, w, all, [](int r) { return r + 1; });
    stage(slab + (int64_t)w * coarse_odd(w), Lg, w, p, 0, w, all, [w](int) { return w; });
  } else {
    stage(slab, Lg + (int64_t)w * p, p, w, 0, p, all, [p](int) { return p; });
    stage(slab + (int64_t)w * coarse_odd(p), Dg + (int64_t)w * w, w, w, 0, w, [](int r) { return r; },
          [w](int) { return w; });
  }
  stage_ints(s_nat, dag.nat + F.nat, f);
  if (g1 > g0) {
    stage_ints(s_gp, gp + g0, g1 - g0 + 1);
    stage_ints(s_gs, dag.gsrc + gbase, nsrc);
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
  asm volatile("cp.async.wait_all;" ::: "memory");
  __syncthreads();
  // 2. forward tasks: g on the own columns (ready before this kernel)
  if (kind == 0 || kind == 4) {
    const int wl = kind == 0 ? r1 : w;  // L_ss^-1 is lower: rows < r1 read columns < r1
    for (int idx = tid; idx < wl * nrhs; idx += kCT) {
      const int i = idx / nrhs, k = idx - i * nrhs;
      const int j = s_nat[i];
      double v;
      if (g) {
        v = g[(size_t)j * nrhs + k];
      } else {
        const int s = col_sub[j];
        const int a = j - lay[s].coff;
        v = 0.0;
        for (int qq = sub_chunk_ptr[s]; qq < sub_chunk_ptr[s + 1]; ++qq) v += partial[((size_t)qq * 6 + a) * nrhs + k];
      }
      vec[idx] = v;
    }
    if (kind == 4)
      for (int idx = w * nrhs + tid; idx < f * nrhs; idx += kCT) vec[idx] = 0.0;
  } else if (kind == 1) {
    for (int idx = w * nrhs + tid; idx < (w + nr) * nrhs; idx += kCT) vec[idx] = 0.0;
  }
  // 3. bounded wait for the tickets this task reads (warp 0): relaxed polls
  // with a short back-off, then an acquire load of each awaited flag
  if (tid < 32) {
    const long long budget = (long long)*spin_cycles;
    const long long t0 = clock64();
    bool ok = true;
    for (int d = T.dep0; d < T.dep1 && ok; ++d) {
      const int a = dag.dep[2 * d], n = dag.dep[2 * d + 1];
      for (int x = a + lane; x < a + n && ok; x += 32) {
        for (;;) {
          if (clock64() - t0 >= budget) { ok = false; break; }
          if (ld_relaxed_u32(&dag.flag[x]) == target) break;
          __nanosleep(20);
        }
        if (ok) (void)ld_acquire_u32(&dag.flag[x]);
      }
    }
    ok = __all_sync(0xffffffffu, ok);
    if (!ok && lane == 0) atomicExch(err, 1);
  }
  __syncthreads();
  // 4. vectors written by the tasks waited for (read from L2): every thread
  // gathers whole front rows (children's update rows in child order)
  if (g1 > g0) {
    // kind 0 / 4: into vec rows g; kind 1: into rows w + (g - g0) (after y)
    const int vrow0 = kind == 1 ? w - g0 : 0;
    for (int idx = tid; idx < (g1 - g0) * nrhs; idx += kCT) {
      const int m = idx / nrhs, k = idx - m * nrhs;
      double a = 0.0;
      for (int e = s_gp[m] - gbase; e < s_gp[m + 1] - gbase; ++e) a += __ldcg(dag.out + (size_t)s_gs[e] * nrhs + k);
      vec[(size_t)(vrow0 + g0 + m) * nrhs + k] += a;
    }
  }
  if (kind == 1) {
    for (int idx = tid; idx < w * nrhs; idx += kCT) {
      const int i = idx / nrhs, k = idx - i * nrhs;
      vec[idx] = __ldcg(dag.yt + (size_t)s_nat[i] * nrhs + k);
    }
  } else if (kind == 2 || kind == 5) {
    for (int idx = tid; idx < p * nrhs; idx += kCT) {
      const int r = idx / nrhs, k = idx - r * nrhs;
      vec[idx] = __ldcg(c + (size_t)s_nat[w + r] * nrhs + k);
    }
    if (kind == 5)
      for (int idx = tid; idx < w * nrhs; idx += kCT) {
        const int i = idx / nrhs, k = idx - i * nrhs;
        vec[(size_t)p * nrhs + idx] = __ldcg(dag.yt + (size_t)s_nat[i] * nrhs + k);
      }
  } else if (kind == 3) {
    for (int idx = tid; idx < (w - r0) * nrhs; idx += kCT) {
      const int i = r0 + idx / nrhs, k = idx % nrhs;
      vec[idx] = __ldcg(dag.yt + (size_t)s_nat[i] * nrhs + k);
    }
  }
  __syncthreads();
  // 5. products from shared memory
  double* yt = dag.yt;
  double* o = dag.out + (size_t)F.out * nrhs;
  if (kind == 0) {
    const int ld = (int)coarse_odd(r1);
    rows_times<NR>([&](int i) { return slab + (size_t)(i - r0) * ld; }, r0, r1, vec, nrhs, all,
                   [](int i) { return i + 1; },
                   [&](int i, int k, double v) { yt[(size_t)s_nat[i] * nrhs + k] = v; });
  } else if (kind == 1) {
    const int ld = (int)coarse_odd(w);
    const double* accp = vec + (size_t)w * nrhs;
    rows_times<NR>([&](int i) { return slab + (size_t)(i - r0) * ld; }, r0, r1, vec, nrhs, all,
                   [w](int) { return w; },
                   [&](int i, int k, double v) { o[(size_t)i * nrhs + k] = accp[(i - r0) * nrhs + k] - v; });
  } else if (kind == 2) {
    const int ld = (int)coarse_odd(p);
    rows_times<NR>([&](int i) { return slab + (size_t)(i - r0) * ld; }, r0, r1, vec, nrhs, all,
                   [p](int) { return p; }, [&](int i, int k, double v) {
                     double* dst = yt + (size_t)s_nat[i] * nrhs + k;
                     *dst = __ldcg(dst) - v;
                   });
  } else if (kind == 3) {
    // slab row i - r0 holds columns r0 .. w - 1; vec holds t from row r0
    const int ld = (int)coarse_odd(w - r0);
    rows_times<NR>([&](int i) { return slab + (size_t)(i - r0) * ld - r0; }, r0, r1, vec - (size_t)r0 * nrhs,
                   nrhs, [](int i) { return i; }, [w](int) { return w; },
                   [&](int i, int k, double v) { c[(size_t)s_nat[i] * nrhs + k] = v; });
  } else if (kind == 4) {
    // y = L_ss^-1 t (kept in shared memory after the front vector), then the update vector
    const int ld = (int)coarse_odd(w);
    double* y = vec + (size_t)f * nrhs;
    rows_times<NR>([&](int i) { return slab + (size_t)i * ld; }, 0, w, vec, nrhs, all, [](int i) { return i + 1; },
                   [&](int i, int k, double v) {
                     y[i * nrhs + k] = v;
                     yt[(size_t)s_nat[i] * nrhs + k] = v;
                   });
    __syncthreads();
    const double* Ls = slab + (size_t)w * ld;
    rows_times<NR>([&](int i) { return Ls + (size_t)i * ld; }, 0, p, y, nrhs, all, [w](int) { return w; },
                   [&](int i, int k, double v) { o[(size_t)i * nrhs + k] = vec[(w + i) * nrhs + k] - v; });
  } else {
    // t = y - L_ps^T x_panel (in shared memory), then x = L_ss^-T t
    const int ldp = (int)coarse_odd(p), ldw = (int)coarse_odd(w);
    double* t = vec + (size_t)f * nrhs;
    const double* yv = vec + (size_t)p * nrhs;
    rows_times<NR>([&](int i) { return slab + (size_t)i * ldp; }, 0, w, vec, nrhs, all, [p](int) { return p; },
                   [&](int i, int k, double v) { t[i * nrhs + k] = yv[i * nrhs + k] - v; });
    __syncthreads();
    const double* Us = slab + (size_t)w * ldp;
    rows_times<NR>([&](int i) { return Us + (size_t)i * ldw; }, 0, w, t, nrhs, [](int i) { return i; },
                   [w](int) { return w; }, [&](int i, int k, double v) { c[(size_t)s_nat[i] * nrhs + k] = v; });
  }
  // 6. publish: every thread's stores, then the flag (release), then the count
  __syncthreads();
  if (tid == 0) {
    st_release_u32(&dag.flag[q], target);
    const unsigned old = atomicAdd(&dag.ctr[1], 1u);
    if (old == (unsigned)dag.n_tasks - 1u) {
      atomicExch(&dag.ctr[0], 0u);
      atomicExch(&dag.ctr[1], 0u);
      atomicExch(&dag.ctr[2], target);
    }
  }
}

}  // namespace

void launch_coarse_factor(const CoarsePlan& cp, const CoarseDev& dv, const int32_t* blk_i, const int32_t* blk_j,
                          const int32_t* blk_ptr, const int32_t* blk_rows, int n_blocks, const SubLayout* lay,
                          const double* R, const Maps& mp, double* ws, int* status, cudaStream_t st) {
  const int S = (int)cp.fronts.size();
  if (S == 0) return;
  cudaMemsetAsync(ws, 0, (size_t)cp.ws * sizeof(double), st);
  k_cf_aug<<<S, kCT, 0, st>>>(dv.fr, ws);
  if (n_blocks > 0)
    k_cf_gtg<<<n_blocks, 64, 0, st>>>(blk_i, blk_j, blk_ptr, blk_rows, dv.place, lay, R, mp, ws);
  for (int l = 0; l < cp.height; ++l) {
    const std::vector<int32_t>& L = cp.level_fronts[l];
    const int nf = (int)L.size();
    if (nf == 0) continue;
    const int32_t* lvl = dv.lvl + dv.lvl_off[l];
    for (int slot = 0; slot < cp.max_children; ++slot) {
      int maxp = 0;
      for (int32_t s : L) {
        const CoarseFront& F = cp.fronts[s];
        if (F.ch0 + slot < F.ch1) maxp = std::max(maxp, cp.fronts[cp.child[F.ch0 + slot].c].p);
      }
      if (maxp == 0) continue;
      k_cf_extend<<<dim3((maxp + kCT / 32 - 1) / (kCT / 32), nf), kCT, 0, st>>>(dv.fr, dv.child, dv.map, lvl, slot,
                                                                               ws);
    }
    int maxw = 0;
    for (int32_t s : L) maxw = std::max(maxw, cp.fronts[s].w);
    for (int kb = 0; kb < maxw; kb += CNB) {
      int trsm = 0, upd = 0;
      for (int32_t s : L) {
        const CoarseFront& F = cp.fronts[s];
        if (kb >= F.w) continue;
        const int nk = std::min(CNB, F.w - kb);
        const int f = F.w + F.p;
        const int n_act = f + std::min(F.w, kb + nk);
        const int r0 = kb + nk;
        trsm = std::max(trsm, (n_act - r0 + CTT - 1) / CTT);
        upd = std::max(upd, ((n_act - r0 + CTT - 1) / CTT) * ((f - r0 + CTT - 1) / CTT));
      }
      k_cf_diag<<<dim3(1, nf), kCT, 0, st>>>(dv.fr, lvl, kb, ws, status);
      if (trsm > 0) k_cf_trsm<<<dim3(trsm, nf), kCT, 0, st>>>(dv.fr, lvl, kb, ws, status);
      if (upd > 0) k_cf_update<<<dim3(upd, nf), kCT, 0, st>>>(dv.fr, lvl, kb, ws, status);
    }
  }
  k_cf_extract<<<dim3(64, S), kCT, 0, st>>>(dv.fr, ws, dv.Dm, dv.Lm);
}

void launch_coarse_solve(const CoarseDag& dag, int nrhs, const double* g, const double* partial,
                         const int32_t* sub_chunk_ptr, const int32_t* col_sub, const SubLayout* lay, double* c,
                         const int* done, int* err, const unsigned long long* spin_cycles, cudaStream_t st) {
  if (dag.n_tasks <= 0) return;
  const size_t smem = (size_t)(nrhs == 1 ? dag.smem1 : dag.smem16) * sizeof(double);
  if (nrhs == 1) {
    if (smem > 48 * 1024) cudaFuncSetAttribute(k_coarse_dag<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_coarse_dag<1><<<dag.n_tasks, kCT, smem, st>>>(dag, 1, g, partial, sub_chunk_ptr, col_sub, lay, c, done, err,
                                                   spin_cycles);
  } else {
    if (smem > 48 * 1024)
      cudaFuncSetAttribute(k_coarse_dag<kMaxRhs>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_coarse_dag<kMaxRhs><<<dag.n_tasks, kCT, smem, st>>>(dag, nrhs, g, partial, sub_chunk_ptr, col_sub, lay, c,
                                                          done, err, spin_cycles);
  }
}

}  // namespace feti
