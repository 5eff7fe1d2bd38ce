// Internal interface between the host driver (feti_host.cpp) and the CUDA
// kernels (feti_kernels.cu).  Not part of the public ABI.
#pragma once
#include <cstdint>
#include <string>
#include <vector>
#include <cuda_runtime.h>

#include "feti.h"

namespace feti {

// Status codes written by kernels into a device word (first error wins).
enum DevStatus : int {
  DEV_OK = 0,
  DEV_LOCAL_SINGULAR = 1,   // non-positive pivot in a local Cholesky factorization
  DEV_INVERTED = 2,         // element with non-positive volume or det F
  DEV_BREAKDOWN = 3,        // (p, F p) <= 0 or not finite
};

// Per-subdomain dense layout.  Dense local order: [interior | boundary minus
// fixing (nbp) | fixing (k) | augmentation (nbp)].  The augmentation block
// holds the identity coupling used to obtain F_i = (S_i[b',b'])^-1 by block
// elimination.  Offsets are in doubles.
struct SubLayout {
  int32_t n;      // free local DOFs (interior + boundary)
  int32_t nI;     // interior DOFs
  int32_t nbp;    // boundary DOFs that are not fixing DOFs
  int32_t k;      // kernel dimension = number of fixing DOFs
  int32_t ld;     // leading dimension of the dense matrix = n + nbp
  int32_t boff;   // offset of this subdomain's boundary vector (sum of nb)
  int32_t voff;   // offset of this subdomain's full local vector (sum of n)
  int32_t coff;   // first coarse column of this subdomain
  int64_t aoff;   // offset of the dense (ld x ld) matrix
  int64_t soff;   // offset of the nb x nb preconditioner block
  int64_t foff;   // offset of the nbp x nbp dense F_i
  int64_t roff;   // offset of R_i (n x k, row-major) in dense local order
  int64_t foff32; // offset (floats) of the FP32 copy of F_i, row stride padded to 4
  int64_t soff32; // offset (floats) of the FP32 copy of the preconditioner block
  // FP32 lower block-triangles of the symmetric F_i and preconditioner block:
  // panels of kSymPH rows, panel I = rows PH I .. PH I + PH - 1 by columns
  // 0 .. PH (I + 1) - 1, row-major, at panel offset PH^2 I (I + 1) / 2; zero
  // beyond the matrix
  int64_t fsym32;
  int64_t ssym32;
  int64_t psym;   // offset (floats) of the transposed-product partials: PH I floats per panel I
  int64_t loff;   // offset of the compact interior factor: rows [0, nI + nbp) x columns [0, nI)
                  // of the Cholesky factor (L_II lower, L_bI), row stride kp_ld
};
// Row stride of the compact interior factor (a multiple of 4 elements).
__host__ __device__ inline int kp_ld(const SubLayout& L) { return (L.nI + 3) & ~3; }
constexpr int kSymPH = 32;  // panel height of the symmetric FP32 apply

// Element kernels ------------------------------------------------------------
// Element matrices are symmetric and stored as their upper triangle, row by
// row: ke_packed(nde) doubles per element, entry (i, j) at ke_idx(nde, i, j).
__host__ __device__ constexpr int ke_packed(int nde) { return nde * (nde + 1) / 2; }
__host__ __device__ inline int ke_idx(int nde, int i, int j) {
  const int a = i < j ? i : j, b = i < j ? j : i;
  return a * nde - a * (a - 1) / 2 + (b - a);
}
// Full (nde x nde, row-major) copies of the packed element matrices.
void launch_ke_unpack(int n_el, int nde, const double* Kp, double* K, cudaStream_t st);
void launch_elem_linear(int n_tets, const double* coords, const int32_t* tets, double E, double nu,
                        double* Ke, int* status, cudaStream_t st);
void launch_elem_hgo(int n_tets, const double* coords, const int32_t* tets, const double* U,
                     const double* fibres, double c, double k1, double k2, double kappa,
                     double* Ke, double* fe, int* status, cudaStream_t st);

// P2 (10-node) linear element matrices [n_tets * 900] (tets: [n_tets * 10]);
// p0: volumetric part condensed to a piecewise-constant pressure (P2-P0).
void launch_elem_linear_p2(int n_tets, const double* coords, const int32_t* tets, double E, double nu, int p0,
                           double* Ke, int* status, cudaStream_t st);
// Local assembly: one CTA per subdomain walks its elements in order (no
// atomics); nde = DOFs per element (12 for P1, 30 for P2), Ke stride nde^2.
void launch_assemble(int P, const SubLayout* lay, const int32_t* sub_elem_ptr, const int32_t* sub_elems,
                     const int32_t* elem_dense, const double* Ke, int nde, double* A, cudaStream_t st);
// Local load vectors: surface loads (+ -f_int) (- K_iD u_D); fdn = DOFs per
// loaded face (9 or 18).
void launch_assemble_rhs(int P, const SubLayout* lay, const int32_t* sub_face_ptr, const int32_t* face_dense,
                         const double* face_force, int fdn, const int32_t* sub_elem_ptr, const int32_t* sub_elems,
                         const int32_t* elem_dense, const double* elem_dirval, const double* Ke,
                         const double* fe, int nde, double tau, double* f, cudaStream_t st);
// fpn = nodes per loaded face (3, or 6 for P2 faces).
void launch_face_forces(int n_faces, int fpn, const int32_t* tri, const double* coords, const double* U,
                        int kind, double scale, const double* traction, double* out, cudaStream_t st);
// The same into the FP32 workspace of the FP32-factor form (entries summed in FP32).
void launch_assemble(int P, const SubLayout* lay, const int32_t* sub_elem_ptr, const int32_t* sub_elems,
                     const int32_t* elem_dense, const double* Ke, int nde, float* A, cudaStream_t st);
// A_ii += delta * (largest diagonal entry of K_rr) on the K_rr rows of every
// subdomain's FP64 workspace.
void launch_shift_diag(int P, const SubLayout* lay, double* A, double delta, cudaStream_t st);
// Writes the identity coupling of the augmentation block and zeros the rest of it.
void launch_augment(int P, const SubLayout* lay, double* A, cudaStream_t st);
void launch_augment(int P, const SubLayout* lay, float* A, cudaStream_t st);
// Copies the trailing boundary block (nb x nb at [nI, nI)) into S (which=0),
// or minus the augmentation block into F (which=1).
void launch_extract(int P, const SubLayout* lay, int which, const double* A, double* out, cudaStream_t st);
// x = K_i^+ g per subdomain (fixing-DOF generalized inverse; zero on fixing DOFs).
void launch_kplus(int P, const SubLayout* lay, const double* A, const double* g, double* x, cudaStream_t st,
                  const int* done = nullptr);

// Multiplier maps ----------------------------------------------------------
struct Maps {
  int n_lambda;
  int nb_total;
  const int32_t* row_pos;   // [2*n_lambda] global boundary position or -1
  const double* row_sgn;    // [2*n_lambda] +-1 (0 for padding)
  const double* weight;     // [n_lambda]
  const int32_t* bt_ptr;    // [nb_total+1]
  const int32_t* bt_row;    // rows of each boundary position
  const double* bt_sgn;
  const int32_t* bpos_sub;  // [nb_total] owning subdomain of each boundary position
};

// y_b = (B_i^T (wv o x))_b: signed gather onto the boundary positions.
void launch_gather(const Maps& mp, const double* x, const double* wv, double* y, const int* done,
                   cudaStream_t st);
// q = wv o (B y) row-wise (deterministic), optional partial sums of (a, q).
void launch_scatter(const Maps& mp, const double* y, const double* wv, double* q, const double* a,
                    double* partial, const int* done, cudaStream_t st);

// Coarse space ---------------------------------------------------------------
// g_i = R_b,i^T (B_i^T x)  for every subdomain with k > 0.
void launch_gtv(int P, const SubLayout* lay, const double* R, const Maps& mp, const double* x, double* g,
                const int* done, cudaStream_t st);
// c = Ginv g (dense coarse inverse, row-major cd x cd).
void launch_coarse_apply(int cd, const double* Ginv, const double* g, double* c, const int* done,
                         cudaStream_t st);
// out = v - G c row-wise; optional partial sums of (a, out) (a NULL: (out,out)).
void launch_expand(const Maps& mp, const SubLayout* lay, const double* R, const double* v, const double* c,
                   double* out, const double* a, double* partial, int with_dot, const int* done,
                   cudaStream_t st);
// G^T G assembled per pair block, deterministic (one CTA per block).
void launch_gtg(int n_blocks, const int32_t* blk_i, const int32_t* blk_j, const int32_t* blk_ptr,
                const int32_t* blk_rows, const SubLayout* lay, const double* R, const Maps& mp, int cd,
                double* GtG, cudaStream_t st);

// PCG control ------------------------------------------------------------------
// Device scalar block.
struct PcgScalars {
  double rho, rho_prev, alpha, beta, pq, wnorm0, wnorm, tol;
  int it, done, status, maxit;
  double rho_slot[2];  // rho of the last two iterations, by parity
};
int scatter_partials();  // number of partial sums the row kernels produce
void launch_ctl_conv(PcgScalars* s, const double* partial, int first, cudaStream_t st);
void launch_vsub(int n, const double* a, const double* b, double* out, cudaStream_t st);

// Global displacement by the owner rule.
void launch_owner_scatter(int n_entries, const int32_t* gdof, const int32_t* vpos, const double* x,
                          double* U, cudaStream_t st);
// x_local += R_i gamma_i.
void launch_add_kernel(int P, const SubLayout* lay, const double* R, const double* gamma, double* x,
                       cudaStream_t st);

}  // namespace feti

namespace feti {
// e_i = scale * R_i^T x_i on full local vectors (dense local order).
void launch_rtx(int P, const SubLayout* lay, const double* R, const double* x, double scale, double* e,
                cudaStream_t st);
// loc_b = boundary slice of the full local vectors x.
void launch_take_boundary(int P, const SubLayout* lay, const double* x, double* loc, cudaStream_t st,
                          const int* done = nullptr);
// rhs_i = f_i - (boundary vector loc placed at the boundary positions).
void launch_local_sub(int P, const SubLayout* lay, const double* f, const double* loc, double* out,
                      cudaStream_t st);
}  // namespace feti

namespace feti {
// Launch schedule of the dense local apply: R rows per warp step, rpc rows
// per CTA, and the (subdomain, first row) table of its n_blocks CTAs.
struct GemvCfg {
  int R = 4;
  int rpc = 64;
  int n_blocks = 0;
  const int32_t* blk_sub = nullptr;
  const int32_t* blk_row0 = nullptr;
};
// y_b = M_i v_b on a pre-gathered local vector; M is the FP64 (f32 = 0, v
// double) or padded FP32 (f32 = 1, v float) copy of F_i (which 0) or the
// preconditioner block (which 1).
void launch_gemv_loc(const GemvCfg& cfg, const SubLayout* lay, int which, const void* M, int f32, const void* vloc,
                     double* y, int max_m, const int* done, cudaStream_t st);
// Symmetric FP32 apply from the lower block-triangle: one warp per (subdomain,
// panel) of the work list, row sums into y and, for the blocks left of the
// diagonal block, the transposed products into the partial buffer; then
// k_symv_fix adds the partials of the panels below each row in a fixed order.
// G = rows per load group (8, 16 or 32).
void launch_symv_f32(int G, int n_warps, const int32_t* wsub, const int32_t* wpanel, const SubLayout* lay, int which,
                     const float* Msym, const float* vloc, double* y, float* part, const Maps& mp, const int* done,
                     cudaStream_t st);
// The same product with each warp streaming its panel through shared memory
// (cp.async.bulk row segments, bounded waits; a timeout sets *err).
// spin_cycles: device word, the main-loop wait budget in SM clock cycles.
void launch_symv2_f32(int n_warps, const int32_t* wsub, const int32_t* wpanel, const SubLayout* lay, int which,
                      const float* Msym, const float* vloc, double* y, float* part, const Maps& mp, const int* done,
                      int* err, const unsigned long long* spin_cycles, cudaStream_t st);
// The same product with one CTA per subdomain (order: subdomains largest
// first) and the transposed partial sums reduced in shared memory, no second
// pass; max_m: the largest operator size.  G = 8, 16 or 32.
void launch_symv3_f32(int G, int P, const int32_t* order, int max_m, const SubLayout* lay, int which,
                      const float* Msym, const float* vloc, double* y, const int* done, cudaStream_t st);
// FP32 signed gather (input of the FP32 apply).
void launch_gather32(const Maps& mp, const double* x, const double* wv, float* y, const int* done, cudaStream_t st);
// a += b
void launch_vadd(int n, double* a, const double* b, cudaStream_t st);
}  // namespace feti

namespace feti {
// G^T x over chunks of 256 boundary positions of the subdomains with k > 0:
// partial[6 c + a] for chunk c.
// With q != NULL the gathered input is x - alpha q (fused CG update, alpha
// from the (p, q) partial sums; CTA 0 stores alpha in sc and alpha_hist).
void launch_gtv_part(int n_chunks, const int32_t* chunk_sub, const int32_t* chunk_p0, const SubLayout* lay,
                     const double* R, const Maps& mp, const double* x, double* partial, const int* done,
                     cudaStream_t st, const double* q = nullptr, const double* pq_partial = nullptr,
                     PcgScalars* sc = nullptr, double* alpha_hist = nullptr);
// Fused CG update + projection expand: r -= alpha q, lam += alpha p in place,
// out = r - G c, partial sums of ||out||^2.
void launch_expand_update(const Maps& mp, const SubLayout* lay, const double* R, double* r, const double* c,
                          double* out, double* partial, double* lam, const double* p, const double* q,
                          const double* pq_partial, PcgScalars* sc, double* alpha_hist, cudaStream_t st);
// Fused CG step: rho from partial sums, beta, p = y + beta p.
void launch_axpby_rho(int n, double* p, const double* y, PcgScalars* s, const double* partial, double* beta_hist,
                      cudaStream_t st);
// c = Ginv (sum of chunk partials per coarse column).
void launch_coarse_apply_part(int cd, const double* Ginv, const double* partial, const int32_t* sub_chunk_ptr,
                              const int32_t* col_sub, const SubLayout* lay, double* c, const int* done,
                              cudaStream_t st);
}  // namespace feti

namespace feti {
// partial[b] = partial sums of (sum of local copies)^2 over n global DOFs (kPartials CTAs).
void launch_global_sumsq(int n, const int32_t* ptr, const int32_t* pos, const double* x, double* partial,
                         cudaStream_t st);
// out = u + a du
void launch_axpy_to(int n, const double* u, double a, const double* du, double* out, cudaStream_t st);
// Newton-Krylov on the non-Dirichlet global DOFs (gs rows: local copies,
// lowest subdomain first): assembled sum of the copies, owner injection into
// (pre-zeroed) local vectors, owner copy back, element-wise tangent matvec
// (node-incidence gather, deterministic), fixed-order dot partials (one per
// CTA of scatter_partials()), and scatter to the 3N global vector.
void launch_gs_assemble(int n, const int32_t* ptr, const int32_t* pos, const double* xloc, double* y, cudaStream_t st);
void launch_gs_inject(int n, const int32_t* ptr, const int32_t* pos, const double* r, double* floc, cudaStream_t st);
void launch_gs_take(int n, const int32_t* ptr, const int32_t* pos, const double* xloc, double* z, cudaStream_t st);
void launch_gs_elem_matvec(int n, const int32_t* inc_ptr, const int32_t* inc, const int32_t* elem_gs, const double* Ke,
                           const double* v, double* y, cudaStream_t st);
void launch_gs_dot(int n, const double* a, const double* b, double* partial, cudaStream_t st);
void launch_gs_to_global(int n, const int32_t* gdof, const double* x, double* out, cudaStream_t st);
}  // namespace feti

namespace feti {
// x[idx[i]] = 0
void launch_zero_list(int n, const int32_t* idx, double* x, cudaStream_t st);
}  // namespace feti

namespace feti {
// Multi-CTA partial Cholesky of one dense lower-triangular row-major matrix
// (leading dimension ld): columns [c0, c1), trailing update on [c1, n_act).
void launch_dense_chol_big(double* A, int ld, int c0, int c1, int n_act, int aug0, int* status, cudaStream_t st);
}  // namespace feti

namespace feti {
// Lumped preconditioner K_bb (Sec. 4.4, Eq. LumpedVK) in CSR over the
// boundary positions: values gathered from the assembled local matrices,
// then y = K_bb v (one warp per row).
void launch_lump_fill(long nnz, const int64_t* src, const double* A, double* val, cudaStream_t st);
void launch_lump_fill(long nnz, const int64_t* src, const float* A, double* val, cudaStream_t st);
void launch_spmv_lump(int n_rows, const int32_t* ptr, const int32_t* col, const double* val, const double* v,
                      double* y, const int* done, cudaStream_t st);
}  // namespace feti

namespace feti {
// Batched multi-CTA partial Cholesky of every subdomain's dense matrix, one
// launch triple (diagonal block, panel solve, tiled trailing update) per
// 32-column step; phase 0: interior columns, phase 1: boundary minus fixing
// columns.  Each step updates only the rows its block column can reach:
// phase 0 the envelope given by env0 ([step][subdomain] pairs (eI, nbact):
// interior rows up to eI, the first nbact boundary rows, the fixing rows),
// phase 1 the remaining rows plus the augmentation rows of the columns
// eliminated so far (env0 unused).  step_chunks[t] (host array, n_steps
// entries): the largest number of 64-row chunks of those rows over the
// subdomains at step t (idle CTAs exit at once).
void launch_chol_batched(int P, const SubLayout* lay, int phase, const int* step_chunks, int n_steps,
                         const int32_t* env0, double* A, int* status, cudaStream_t st);
// The same steps on the FP32 workspace (FP32 factorization), in blocks of
// kChol32Block columns (the step and envelope tables use that width).  64
// columns halve the passes over the trailing matrix (112 against 140 ms of
// elimination on the 1024-subdomain tube) but the FP32 factor then needs one
// more refinement correction and three more inner PCG iterations, which
// costs more than it saves: 32.
constexpr int kChol32Block = 32;
void launch_chol_batched(int P, const SubLayout* lay, int phase, const int* step_chunks, int n_steps,
                         const int32_t* env0, float* A, int* status, cudaStream_t st);
}  // namespace feti

namespace feti {
// ---- FP32 factorization with FP64-refined K^+ (feti_factor32.cu) ----
// Eliminated workspace (FP32 or FP64) -> the dense local operator in each
// requested layout (NULL: skipped) in one tiled pass: FP64 row-major (out64),
// the FP32 copy with rows padded to 4 (out32), the FP32 symmetric-apply
// panels (sym32); which 0: the preconditioner block (S_i), which 1: F_i;
// max_m: the largest operator size over the subdomains.
void launch_extract_tiles(int P, int max_m, const SubLayout* lay, int which, const float* A, double* out64, float* out32,
                          float* sym32, cudaStream_t st);
void launch_extract_tiles(int P, int max_m, const SubLayout* lay, int which, const double* A, double* out64,
                          float* out32, float* sym32, cudaStream_t st);
// One FP32 correction x (+)= L^-T L^-1 r of the FP32-factor K^+ (L the FP32
// Cholesky factor of K_rr), the sweeps confined to the interior rows:
// forward: y_I = L_II^-1 r_I (FP32 into yI, local offsets) and
// z_b = r_b - L_bI y_I (FP32 into zb, boundary offsets, zero on the fixing
// positions); the caller then applies the FP32 F_i to zb (x_b, FP64 at the
// boundary offsets); backward: x_I = L_II^-T (y_I - L_bI^T x_b) and
// x (+)= [x_I, x_b] (init: x = that, zero on the fixing rows).
// Both read the compact interior factor (SubLayout::loff, row stride kp_ld);
// the backward sweep overwrites yI (with y_I - L_bI^T x_b).
// The FP64 overloads give the FP64 K^+ of the FP64 factorizations in one
// pass (forward, FP64 F_i apply, backward: K_rr^-1 by its block form with
// the Schur complement inverse F_i).
void launch_kp_forward(int P, const SubLayout* lay, const float* Lc, const double* r, float* yI, float* zb, int max_nr,
                       cudaStream_t st);
void launch_kp_backward(int P, const SubLayout* lay, const float* Lc, float* yI, const double* xb, double* x,
                        int init, int max_nr, cudaStream_t st);
void launch_kp_forward(int P, const SubLayout* lay, const double* Lc, const double* r, double* yI, double* zb,
                       int max_nr, cudaStream_t st);
void launch_kp_backward(int P, const SubLayout* lay, const double* Lc, double* yI, const double* xb, double* x,
                        int init, int max_nr, cudaStream_t st);
// Copies rows [0, nI + nbp) x columns [0, nI) of each eliminated workspace
// matrix (at lay[s].aoff in A) into the compact interior factor Lc (at
// lay[s].loff, row stride kp_ld; zero above the diagonal of L_II and in the
// padding).  max_rows: the largest nI + nbp over the P subdomains.
void launch_compact_factor(int P, int max_rows, const SubLayout* lay, const double* A, double* Lc, cudaStream_t st);
void launch_compact_factor(int P, int max_rows, const SubLayout* lay, const float* A, float* Lc, cudaStream_t st);
// r = g - K_rr x in FP64 from the element matrices (zero on the fixing rows),
// in two passes: ye (nde doubles per element) = K_e x_e
// for all elements (elem_sub: the subdomain of each element), then per local
// row (row_sub: the subdomain of each of the n_rows local rows) g minus its
// incidence entries of ye in list order (kinc entries index ye directly).
void launch_kresid2(int n_el, int nde, const int32_t* elem_sub, const int32_t* row_sub, int n_rows, const SubLayout* lay,
                    const int32_t* kinc_ptr, const int32_t* kinc, const int32_t* elem_dense, const double* Ke,
                    const double* g, const double* x, double* ye, double* r, cudaStream_t st);
// out = boundary vector loc placed at the boundary positions, zero interior.
void launch_place(int P, const SubLayout* lay, const double* loc, double* out, cudaStream_t st,
                  const int* done = nullptr);
// out[2 s], out[2 s + 1] = squared norms of r and g over rows [0, nI + nbp) of subdomain s.
void launch_sub_norm2(int P, const SubLayout* lay, const double* r, const double* g, double* out, cudaStream_t st);
// x[i] = deterministic pseudo-random value in [-1, 1).
void launch_fill_mix(long n, double* x, cudaStream_t st);
}  // namespace feti

namespace feti {
// ---- block form: up to kMaxRhs right-hand sides, vectors [n][nrhs] ----
constexpr int kMaxRhs = 16;
struct PcgScalarsM {
  double tol[kMaxRhs];
  double rho[kMaxRhs];
  double rho_slot[2][kMaxRhs];
  double alpha[kMaxRhs];
  double beta[kMaxRhs];
  double pq[kMaxRhs];
  double wnorm0[kMaxRhs];
  double wnorm[kMaxRhs];
  int active[kMaxRhs];
  int it, done, status, maxit;
};
void launch_gather_m(const Maps& mp, int nrhs, const double* x, const double* wv, void* y, int f32, const int* done,
                     cudaStream_t st);
// Y = M_i V per subdomain (batched GEMM, N = nrhs), FP64 or FP32 copies.
void launch_gemm_loc(const GemvCfg& cfg, const SubLayout* lay, int which, const void* M, int f32, int nrhs,
                     const void* vloc, double* y, int max_m, const int* done, cudaStream_t st);
// Tensor-core (tcgen05, 3xTF32) variant of the FP32 block GEMM; cfg must be
// the 128-rows-per-CTA table; nrhs <= 16; *err is set if a bounded wait
// timed out.
// Tensor-core block GEMM on the FP32 copies: variant 1 register-staged,
// 2 bulk-copy staged, 3 tensor-map (TMA) fed, 4 / 5 warp-specialised
// TMA-fed with 3 / 2 stages, 6 / 7 / 8 persistent warp-specialised over all
// tiles (3 / 3 / 2 raw A slots and 2 / 3 / 2 tail slots; two / two / three
// CTAs per SM);
// tmaps = one CUtensorMap per subdomain for the matrix `which` (variants 3-8).
// spin_cycles: device word, the main-loop wait budget (SM clock cycles) of the
// warp-specialised variants (4-8); their drain waits keep a fixed budget.
void launch_gemm_tc(const GemvCfg& cfg, const SubLayout* lay, int which, const float* M, int nrhs, const float* vloc,
                    double* y, const int* done, int* err, int variant, const void* tmaps,
                    const unsigned long long* spin_cycles, cudaStream_t st);
void launch_scatter_m(const Maps& mp, int nrhs, const double* y, const double* wv, double* q, const double* a,
                      double* partial, const int* done, cudaStream_t st);
// c = (G^T G)^-1 G^T (x - alpha q), q optional (fused CG update); with
// Ginv == NULL only the chunk partials of G^T (x - alpha q) into gpart.
void launch_project_m(int n_chunks, const int32_t* chunk_sub, const int32_t* chunk_p0, const int32_t* sub_chunk_ptr,
                      const int32_t* col_sub, const SubLayout* lay, const double* R, const Maps& mp, int nrhs, int cd,
                      const double* Ginv, const double* x, const double* q, const PcgScalarsM* sc, double* gpart,
                      double* g, double* c, const int* done, cudaStream_t st);
void launch_expand_m(const Maps& mp, const SubLayout* lay, const double* R, int nrhs, int has_coarse, const double* v,
                     const double* c, double* out, const double* a, double* partial, double* r_upd, double* lam,
                     const double* p, const double* q, const PcgScalarsM* sc, const int* done, cudaStream_t st);
void launch_axpby_rho_m(int n, int nrhs, double* p, const double* y, PcgScalarsM* s, const double* partial,
                        cudaStream_t st);
void launch_alpha_m(int nrhs, PcgScalarsM* s, const double* partial, double* alpha_hist, cudaStream_t st);
void launch_conv_m(int nrhs, PcgScalarsM* s, const double* partial, int first, cudaStream_t st);
void launch_spmv_lump_m(int n_rows, int nrhs, const int32_t* ptr, const int32_t* col, const double* val,
                        const double* v, double* y, const int* done, cudaStream_t st);
void launch_col_get(int n, int nrhs, int k, const double* blk, double* v, cudaStream_t st);
// blk[:, k] = scale * v
void launch_col_set(int n, int nrhs, int k, double scale, const double* v, double* blk, cudaStream_t st);
}  // namespace feti

namespace feti {
// Records msg as the context's last error and returns st.
feti_status set_error(feti_ctx* ctx, feti_status st, const std::string& msg);
// Device address and capacity (doubles) of the static no-alloc scratch on the
// current device (cudaGetSymbolAddress; loads the module that holds it).
cudaError_t noalloc_scratch_lookup(double** out, size_t* capacity);
// q = F v, z = M^-1 q with the local scratch vectors placed in the static
// scratch looked up at feti_create instead of context memory; enqueued on the
// context's stream, no allocation, no graph, no event.
feti_status dual_apply_noalloc(feti_ctx* ctx, const double* v, double* q, double* z);
}  // namespace feti

namespace feti {
// ---- sparse coarse problem: supernodal Cholesky of G^T G (Sec. 4.3) ----
// Dynamic shared memory a sweep task may use (doubles, 224 KiB).
constexpr int64_t kCoarseSmemDoubles = 224 * 1024 / 8;
// Row stride of a staged factor block in shared memory: odd, so that rows
// read column by column by neighbouring threads fall in different banks.
__host__ __device__ constexpr int64_t coarse_odd(int64_t n) { return n | 1; }
// Front of a supernode: its own coarse columns (w), then its panel rows (p),
// as natural coarse indices nat[nat .. nat + w + p).
struct CoarseFront {
  int32_t w, p;
  int32_t parent;  // -1: root of the assembly tree
  int32_t level;   // height in the assembly tree (leaves 0)
  int32_t nat;     // offset of the front's natural indices
  int32_t out;     // first row of the update vector in the out scratch (p rows)
  int32_t ch0, ch1;  // children: range of the child list
  int32_t gofs;    // gather lists of the front rows: gptr[gofs .. gofs + w + p]
                   // bound the children's update rows (gsrc, rows of the out
                   // scratch) that add into each front row, children in order
  int32_t pad;
  int64_t off;     // numeric workspace, (f + w) x f row-major (f = w + p); the
                   // last w rows start as the identity on the own columns
  int64_t doff;    // L_ss^-1 (w x w, lower) then L_ss^-T (w x w, upper), row-major
  int64_t loff;    // L_ps (p x w) then L_ps^T (w x p), row-major
};
// A child of a front: its p front indices in the parent's front start at
// map; the first n_own of them are own columns of the parent.
struct CoarseChild {
  int32_t c, map, n_own, pad;
};
// One task of the triangular sweeps: rows [r0, r1) of kind 0 (forward:
// y = L_ss^-1 t on own rows), 1 (forward: update vector on panel rows),
// 2 (backward: t = y - L_ps^T x_panel on own rows), 3 (backward:
// x = L_ss^-T t on own rows), or a whole front: 4 (kinds 0 and 1), 5
// (kinds 2 and 3); it waits for the ticket ranges dep[2 d], dep[2 d + 1]
// (first, count) for d in [dep0, dep1).
struct CoarseTask {
  int32_t s, kind, r0, r1, dep0, dep1;
};
// Destination of a G^T G pair block (blk_i <= blk_j natural subdomain
// numbers) in a front: rows row0.., columns col0..; swap: the blk_i columns
// are the front's columns.
struct CoarsePlace {
  int64_t off;
  int32_t ld, row0, col0, swap;
};
struct CoarsePlan {
  std::vector<CoarseFront> fronts;
  std::vector<CoarseChild> child;
  std::vector<int32_t> map, nat, dep, gptr, gsrc;
  std::vector<CoarseTask> tasks;
  std::vector<CoarsePlace> place;
  std::vector<std::vector<int32_t>> level_fronts;
  int64_t ws = 0, nD = 0, nL = 0;
  int32_t n_out = 0;
  int max_w = 0, max_p = 0, max_children = 0, height = 0;
  // shared memory of the largest task (doubles: its staged factor block plus
  // its vectors) for one and for kMaxRhs right-hand sides
  int64_t smem1 = 1, smem16 = 1;
  double flops = 0.0;
};
// Nested-dissection order of the subdomain graph (pair blocks gi[b] <= gj[b]
// of the subdomains with k > 0), supernodes of at most leaf_max subdomains
// below the separators, fronts, child maps, block placements and the task
// graph of the sweeps (a front of at most merge_bytes of factor per sweep as
// one task, larger ones in row tasks of about task_bytes).  Host only.
bool coarse_plan(int P, const int32_t* k, const int32_t* coff, const std::vector<int32_t>& gi,
                 const std::vector<int32_t>& gj, int leaf_max, int task_bytes, int merge_bytes, CoarsePlan* out,
                 std::string* err);
}  // namespace feti

namespace feti {
// Device views of a coarse plan (feti_coarse.cu).
struct CoarseDag {
  const CoarseFront* fr;
  const CoarseChild* child;
  const int32_t* map;
  const int32_t* nat;
  const CoarseTask* task;
  const int32_t* dep;
  const int32_t* gptr;
  const int32_t* gsrc;
  const double* Dm;  // L_ss^-1, L_ss^-T per front
  const double* Lm;  // L_ps, L_ps^T per front
  double* yt;        // y, then t, by natural coarse index (cd x nrhs)
  double* out;       // update vectors (n_out x nrhs)
  unsigned* flag;    // per task: epoch of its last completion
  unsigned* ctr;     // ticket counter, completed count, epoch
  int n_tasks;
  int64_t smem1, smem16;  // dynamic shared memory (doubles) for 1 and up to kMaxRhs vectors
};
struct CoarseDev {
  const CoarseFront* fr;
  const CoarseChild* child;
  const int32_t* map;
  const CoarsePlace* place;
  const int32_t* lvl;            // level lists, concatenated
  std::vector<int64_t> lvl_off;  // host: start of each level list
  double* Dm;
  double* Lm;
};
// Numeric multifrontal factorization of G^T G into dv.Dm / dv.Lm (workspace
// ws of cp.ws doubles, pair blocks as for launch_gtg); a non-positive pivot
// sets DEV_LOCAL_SINGULAR in *status.
void launch_coarse_factor(const CoarsePlan& cp, const CoarseDev& dv, const int32_t* blk_i, const int32_t* blk_j,
                          const int32_t* blk_ptr, const int32_t* blk_rows, int n_blocks, const SubLayout* lay,
                          const double* R, const Maps& mp, double* ws, int* status, cudaStream_t st);
// c = (G^T G)^-1 g for nrhs vectors ([j][k] layout, natural coarse index j):
// g given, or (g == NULL) summed from the chunk partials of the G^T x
// kernels (partial[(chunk * 6 + a) * nrhs + k]).  One launch of dag.n_tasks
// CTAs; a wait that exceeds *spin_cycles sets *err.
void launch_coarse_solve(const CoarseDag& dag, int nrhs, const double* g, const double* partial,
                         const int32_t* sub_chunk_ptr, const int32_t* col_sub, const SubLayout* lay, double* c,
                         const int* done, int* err, const unsigned long long* spin_cycles, cudaStream_t st);
}  // namespace feti
