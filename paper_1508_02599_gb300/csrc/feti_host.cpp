// Host driver and C ABI of the FETI solver.
//
// Host side (once per mesh): the decomposition of Sec. 4 -- local numbering,
// fully redundant multiplier rows (Sec. 4.1, Fig. 3a), all-floating Dirichlet
// rows (Sec. 4.2), multiplicity weights (Sec. 4.4), rigid-body kernels and
// their detection for classical subdomains touching the Dirichlet boundary
// (Sec. 4.3), fixing DOFs of the generalized inverses (Sec. 5.2), dense local
// orderings and device layouts.  Device side: everything numerical, on one
// stream; the projected PCG runs as a captured CUDA graph of `chunk`
// iterations with the stopping test evaluated on the device.
#include "feti.h"
#include "feti_internal.h"

#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <atomic>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <numeric>
#include <string>
#include <vector>

using feti::SubLayout;

namespace {

struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

}  // namespace

struct feti_ctx {
  // problem (host copies)
  int N = 0, E = 0, P = 0;
  // nodes per element (4: P1, 10: P2), DOFs per element, nodes per loaded face
  int npe = 4, nde = 12, fpn = 3;
  std::vector<double> coords;
  std::vector<int32_t> tets, part;
  feti_material mat{};
  std::vector<double> fibres;
  std::vector<int32_t> dir_dof;
  std::vector<double> dir_val;
  std::vector<int32_t> face_tri;    // pressure faces then traction faces
  std::vector<int32_t> face_owner;
  std::vector<int32_t> face_kind;   // 0 pressure, 1 traction, per grouped face
  int n_press = 0, n_trac = 0;
  double pressure = 0.0, traction[3] = {0, 0, 0};
  feti_options opt{};
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  // the coarse-problem setup runs on a second stream, overlapping the local
  // factorizations: stream, completion event, its own device status word and
  // its workspace (freed once joined)
  cudaStream_t stream2 = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_coarse = nullptr;
  int* d_status2 = nullptr;
  void* coarse_ws[2] = {nullptr, nullptr};
  bool coarse_pending = false;
  std::string err;
  int device = -1;  // the CUDA device current at feti_create
  // static scratch of feti_dual_apply_noalloc on that device (looked up at
  // feti_create), its capacity in doubles, and the lookup's error if it failed
  double* noalloc_scratch = nullptr;
  size_t noalloc_cap = 0;
  std::string noalloc_err;

  // decomposition (host)
  std::vector<std::vector<int32_t>> nodes;
  std::vector<int32_t> row_sub, row_ldof;
  std::vector<int8_t> row_sign;
  std::vector<double> weight, bvec;
  std::vector<SubLayout> lay;
  std::vector<int32_t> fix_ptr, fix_ldof;
  int64_t n_lambda = 0, nb_total = 0, nloc_total = 0, cd = 0;
  int max_nb = 0;
  bool af = true;
  bool any_dirval = false;

  // device
  std::vector<DevBuf> bufs;
  double *d_coords = nullptr, *d_fibres = nullptr, *d_Ke = nullptr, *d_fe = nullptr, *d_A = nullptr;
  float *d_F32 = nullptr, *d_S32 = nullptr;
  double *d_vloc = nullptr, *d_dl = nullptr;
  double *d_S = nullptr, *d_F = nullptr, *d_R = nullptr, *d_f = nullptr, *d_x = nullptr, *d_x2 = nullptr;
  double *d_face_force = nullptr, *d_traction = nullptr, *d_elem_dirval = nullptr;
  int32_t *d_tets = nullptr, *d_face_tri = nullptr;
  SubLayout* d_lay = nullptr;
  int32_t *d_sub_elem_ptr = nullptr, *d_sub_elems = nullptr, *d_elem_dense = nullptr;
  int32_t *d_sub_face_ptr = nullptr, *d_face_dense = nullptr;
  int32_t *d_row_pos = nullptr, *d_bt_ptr = nullptr, *d_bt_row = nullptr, *d_bpos_sub = nullptr;
  double *d_row_sgn = nullptr, *d_weight = nullptr, *d_bt_sgn = nullptr, *d_b = nullptr;
  // CTA tables of the dense local applies for rows-per-CTA 32, 64, 128
  // ([which][k]), and the schedules picked by the autotuner
  feti::GemvCfg tab[2][3];
  std::vector<int32_t> tab_ptr[2][3];  // first CTA of each subdomain in tab[which][k] (p + 1 entries)
  feti::GemvCfg cfg64[2], cfg32[2];
  feti::GemvCfg cfgm64[2], cfgm32[2];  // block form (N = nrhs) schedules
  // FP32 block GEMM on the tensor cores: 0 no, 1 register-staged, 2 bulk-copy staged, 3 TMA-fed,
  // 4 / 5 warp-specialised TMA-fed with 3 / 2 stages
  int tc_m[2] = {0, 0};
  CUtensorMap* d_tmap[2] = {nullptr, nullptr};  // per-subdomain tensor maps of the FP32 F_i and S_i copies
  int* d_tc_err = nullptr;
  int tuned_m = 0;                     // nrhs the block schedules were tuned for
  bool tuned = false;
  float* d_vloc32 = nullptr;
  int32_t *d_chunk_sub = nullptr, *d_chunk_p0 = nullptr, *d_sub_chunk_ptr = nullptr, *d_col_sub = nullptr;
  double* d_gpart = nullptr;
  int32_t *d_gs_ptr = nullptr, *d_gs_pos = nullptr, *d_dir_dof = nullptr;
  int32_t *d_gs_gdof = nullptr, *d_elem_gs = nullptr, *d_inc_ptr = nullptr, *d_inc = nullptr;
  double* d_nk = nullptr;  // Newton-Krylov vectors: 5 x n_gs
  int32_t *d_lump_ptr = nullptr, *d_lump_col = nullptr;
  int64_t* d_lump_src = nullptr;
  double* d_lump_val = nullptr;
  int64_t lump_nnz = 0;
  int n_gs = 0;
  double *d_dU = nullptr, *d_Utrial = nullptr, *d_fl = nullptr;
  std::vector<double> h_partial;
  int n_chunks = 0;
  int32_t *d_gtg_i = nullptr, *d_gtg_j = nullptr, *d_gtg_ptr = nullptr, *d_gtg_rows = nullptr;
  int n_gtg = 0;
  double *d_GtG = nullptr, *d_Ginv = nullptr, *d_Acoarse = nullptr;
  SubLayout* d_lay_coarse = nullptr;
  // sparse coarse problem (supernodal Cholesky of G^T G) in place of the
  // dense inverse: plan, device views, and the flag of its bounded waits
  bool coarse_sparse = false;
  feti::CoarsePlan cplan;
  feti::CoarseDev cdev{};
  feti::CoarseDag cdag{};
  int* d_coarse_err = nullptr;
  int32_t *d_own_gdof = nullptr, *d_own_vpos = nullptr;
  int n_own = 0;
  std::vector<double> U_init;  // classical: Dirichlet values at their DOFs
  double *d_U = nullptr, *d_Uinit = nullptr, *d_Uout = nullptr;
  // PCG vectors
  double *d_lam = nullptr, *d_r = nullptr, *d_w = nullptr, *d_z = nullptr, *d_y = nullptr, *d_p = nullptr;
  double *d_q = nullptr, *d_d = nullptr, *d_loc = nullptr, *d_g = nullptr, *d_c = nullptr, *d_e = nullptr;
  double *d_partial_wy = nullptr, *d_partial_pq = nullptr;
  double *d_partial = nullptr, *d_alpha_hist = nullptr, *d_beta_hist = nullptr;
  feti::PcgScalars* d_sc = nullptr;
  feti::PcgScalars* h_sc = nullptr;  // pinned
  int *d_status = nullptr, *d_zero = nullptr;
  int *h_status = nullptr;  // pinned
  feti::Maps maps{};
  bool prepared = false;
  // host plan (feti_create_plan): the decomposition without any device state;
  // only the host getters accept it
  bool dry = false;
  cudaGraphExec_t pcg_graph = nullptr;
  int pcg_graph_chunk = 0;
  bool pcg_graph_mixed = false;
  double t_setup_ms = 0.0;
  // interior elimination restricted to the envelope: per step and subdomain
  // the end eI of the interior rows and the count nbact of boundary rows that
  // the step's block column can reach ([step][subdomain][2])
  // ([step][subdomain of the group][2] per elimination group, the groups'
  // tables one after another from env_off[g])
  std::vector<int32_t> env0;
  std::vector<int64_t> env_off;
  int32_t* d_env0 = nullptr;
  // the same for the FP32 elimination's kChol32Block-column steps
  std::vector<int32_t> env0_32;
  std::vector<int64_t> env32_off;
  int32_t* d_env0_32 = nullptr;
  // local factorizations in groups: subdomains [grp[g], grp[g + 1]) are
  // eliminated together in the one workspace d_A / d_A32 of ws_elems
  // elements (ws_full: every subdomain at once); d_lay_ws holds the layouts
  // with aoff relative to the group's first matrix.  keep_factor: the whole
  // factor stays (implicit local form; one group, no compact copy), else the
  // compact interior factor d_Lc / d_Lc32 (lc_elems) serves every K^+.
  std::vector<int32_t> grp;
  SubLayout* d_lay_ws = nullptr;
  int64_t ws_elems = 0, ws_full = 0, lc_elems = 0;
  bool keep_factor = false;
  double* d_Lc = nullptr;
  float* d_Lc32 = nullptr;
  double *d_kyI64 = nullptr, *d_kzb64 = nullptr;  // FP64 K^+: y_I and z_b
  std::vector<int64_t> lump_grp;  // first lumped-preconditioner entry of each group
  double gemv_ms = 0.0, gemv_bytes = 0.0, gemv_flops = 0.0;
  double elem_ms = 0.0, elem_bytes = 0.0;
  // sizes (elements) of d_A, d_S, d_F, d_F32, d_S32, d_F32s, d_S32s, d_symp
  int64_t op_elems[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  // symmetric FP32 local applies: lower block-triangles, transposed-product
  // partials, work lists, and the load-group size picked by the autotuner
  // per matrix (0: the full-row kernel is used)
  float *d_F32s = nullptr, *d_S32s = nullptr, *d_symp = nullptr;
  int32_t *d_sym_sub[2] = {nullptr, nullptr}, *d_sym_panel[2] = {nullptr, nullptr};
  // subdomain-per-CTA symmetric apply: subdomains by operator size, largest
  // first, and the largest size, per matrix
  int32_t* d_sym_order[2] = {nullptr, nullptr};
  int sym_max_m[2] = {0, 0};
  int sym_n[2] = {0, 0};
  // 8 / 16 / 32: register-staged load groups (+ 100 x L2-prefetch distance in
  // tiles); 64: streamed through shared memory
  int sym32[2] = {0, 0};
  int* d_sym_err = nullptr;  // set by a streamed symmetric apply whose bounded wait ran out
  // main-loop wait budget (SM clock cycles) of the streamed symmetric apply
  // and the warp-specialised tensor-core GEMM: a device word read at every launch
  unsigned long long* d_spin = nullptr;
  // FP32-factor form: FP32 elimination workspace (the group workspace, as d_A), per
  // local row its (element, element row) incidences for the FP64 residual of
  // the refined K^+, refinement scratch, per-subdomain norms, and the number
  // of refinement corrections chosen at setup (with the residual they reach)
  float* d_A32 = nullptr;
  int32_t *d_kinc_ptr = nullptr, *d_kinc = nullptr;
  double *d_kr = nullptr, *d_kg = nullptr, *d_knorm = nullptr;
  // interior-sweep corrections: y_I (FP32, local offsets), z_b (FP32) and
  // x_b = F_i z_b (FP64) at the boundary offsets
  float *d_kyI = nullptr, *d_kzb = nullptr;
  double* d_kxb = nullptr;
  // implicit local form: the placed boundary vector and K^+ of it (full local vectors)
  double *d_ix = nullptr, *d_ix2 = nullptr;
  // two-pass FP64 residual: subdomain of each element and of each local row,
  // and the per-(element, row) products K_e x_e
  int32_t *d_elem_sub = nullptr, *d_row_sub = nullptr;
  double* d_kye = nullptr;
  int refine_steps = 0;
  // Newton preconditioner: relative diagonal shift of the local tangents of
  // the last assembly (0 = exact local tangents)
  double shift = 0.0;
  double refine_res = 0.0;
  int max_nr = 0;
  cudaEvent_t elem_ev[2] = {nullptr, nullptr};
  // block form (several right-hand sides)
  int m_cap = 0;  // allocated nrhs capacity of the block buffers
  double *dm_lam = nullptr, *dm_r = nullptr, *dm_w = nullptr, *dm_z = nullptr, *dm_y = nullptr, *dm_p = nullptr;
  double *dm_q = nullptr, *dm_d = nullptr, *dm_dl = nullptr, *dm_loc = nullptr, *dm_vloc = nullptr;
  float* dm_vloc32 = nullptr;
  double *dm_part_wy = nullptr, *dm_part_pq = nullptr, *dm_part_ww = nullptr, *dm_gpart = nullptr;
  double *dm_g = nullptr, *dm_c = nullptr, *dm_alpha_hist = nullptr;
  feti::PcgScalarsM* dm_sc = nullptr;
  feti::PcgScalarsM* hm_sc = nullptr;  // pinned
  cudaGraphExec_t pcgm_graph = nullptr;
  int pcgm_chunk = 0, pcgm_nrhs = 0;
  bool pcgm_mixed = false;
  cudaGraphExec_t dualm_graph = nullptr;
  const double* dualm_v = nullptr;
  const double* dualm_q = nullptr;
  const double* dualm_z = nullptr;
  int dualm_n = 0, dualm_nrhs = 0;
  std::vector<cudaEvent_t> dualm_events;
  cudaGraphExec_t dual_graph = nullptr;
  const double* dual_v = nullptr;
  const double* dual_q = nullptr;
  const double* dual_z = nullptr;
  int dual_n = 0;
  std::vector<cudaEvent_t> dual_events;
};

namespace {

#define FETI_CK(call)                                                                            \
  do {                                                                                           \
    cudaError_t e_ = (call);                                                                     \
    if (e_ != cudaSuccess) {                                                                     \
      ctx->err = std::string(#call) + ": " + cudaGetErrorString(e_);                           \
      return e_ == cudaErrorMemoryAllocation ? FETI_ERR_OOM : FETI_ERR_CUDA;                     \
    }                                                                                            \
  } while (0)

#define FETI_TRY(expr)              \
  do {                              \
    feti_status s_ = (expr);        \
    if (s_ != FETI_OK) return s_;   \
  } while (0)

feti_status fail(feti_ctx* ctx, feti_status st, const std::string& msg) {
  ctx->err = msg;
  return st;
}

// Entry points that need device state refuse a host plan.
feti_status need_device(feti_ctx* ctx) {
  if (ctx->dry) return fail(ctx, FETI_ERR_STATE, "host plan context (feti_create_plan): no device state");
  return FETI_OK;
}

// Precision forms: FP32 elimination (refined K^+); FP32 operators inside the
// PCG (both mixed forms); FP64 explicit F_i and S_i (FP64 and mixed forms).
bool f32_factor(const feti_ctx* ctx) { return ctx->opt.precision == FETI_MIXED_F32FACTOR; }
bool f32_ops(const feti_ctx* ctx) { return ctx->opt.precision != FETI_FP64; }
bool fp64_ops(const feti_ctx* ctx) { return ctx->opt.precision != FETI_MIXED_F32FACTOR; }

template <class T>
feti_status dev_alloc(feti_ctx* ctx, T** out, size_t count) {
  if (ctx->dry) {
    *out = nullptr;
    return FETI_OK;
  }
  void* p = nullptr;
  const size_t bytes = std::max<size_t>(count, 1) * sizeof(T);
  cudaError_t e = cudaMalloc(&p, bytes);
  if (e != cudaSuccess) {
    ctx->err = std::string("cudaMalloc of ") + std::to_string(bytes) + " bytes: " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? FETI_ERR_OOM : FETI_ERR_CUDA;
  }
  ctx->bufs.push_back({p, bytes});
  *out = static_cast<T*>(p);
  return FETI_OK;
}

// Allocator that leaves the elements of a resized vector uninitialised: for
// large host arrays that are written completely before they are read.
template <class T>
struct NoInitAlloc : std::allocator<T> {
  template <class U>
  struct rebind {
    using other = NoInitAlloc<U>;
  };
  NoInitAlloc() = default;
  template <class U>
  NoInitAlloc(const NoInitAlloc<U>&) noexcept {}
  template <class U>
  void construct(U* p) noexcept {
    ::new (static_cast<void*>(p)) U;
  }
  template <class U, class... A>
  void construct(U* p, A&&... a) {
    ::new (static_cast<void*>(p)) U(std::forward<A>(a)...);
  }
};
template <class T>
using hvec = std::vector<T, NoInitAlloc<T>>;

template <class T, class Al>
feti_status upload(feti_ctx* ctx, T** out, const std::vector<T, Al>& v) {
  if (ctx->dry) return FETI_OK;
  FETI_TRY(dev_alloc(ctx, out, v.size()));
  if (!v.empty()) FETI_CK(cudaMemcpyAsync(*out, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, ctx->stream));
  return FETI_OK;
}

// Symmetric 6x6 eigen-decomposition by cyclic Jacobi rotations.
void jacobi6(double A[6][6], double V[6][6], double w[6]) {
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < 6; ++j) V[i][j] = (i == j) ? 1.0 : 0.0;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0;
    for (int i = 0; i < 6; ++i)
      for (int j = i + 1; j < 6; ++j) off += A[i][j] * A[i][j];
    if (off < 1e-300) break;
    for (int p = 0; p < 6; ++p)
      for (int q = p + 1; q < 6; ++q) {
        if (std::fabs(A[p][q]) < 1e-300) continue;
        const double theta = (A[q][q] - A[p][p]) / (2.0 * A[p][q]);
        const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < 6; ++k) {
          const double akp = A[k][p], akq = A[k][q];
          A[k][p] = c * akp - s * akq;
          A[k][q] = s * akp + c * akq;
        }
        for (int k = 0; k < 6; ++k) {
          const double apk = A[p][k], aqk = A[q][k];
          A[p][k] = c * apk - s * aqk;
          A[q][k] = s * apk + c * aqk;
        }
        for (int k = 0; k < 6; ++k) {
          const double vkp = V[k][p], vkq = V[k][q];
          V[k][p] = c * vkp - s * vkq;
          V[k][q] = s * vkp + c * vkq;
        }
      }
  }
  for (int i = 0; i < 6; ++i) w[i] = A[i][i];
}

// Extreme eigenvalues of the symmetric tridiagonal (diag a, offdiag b) by
// Sturm-sequence bisection.
double sturm_count(const std::vector<double>& a, const std::vector<double>& b, double x) {
  int cnt = 0;
  double d = 1.0;
  for (size_t i = 0; i < a.size(); ++i) {
    const double bb = i ? b[i - 1] * b[i - 1] : 0.0;
    d = a[i] - x - (i ? bb / (d == 0.0 ? 1e-300 : d) : 0.0);
    if (d < 0) ++cnt;
  }
  return cnt;
}

double lanczos_cond(const std::vector<double>& alpha, const std::vector<double>& beta) {
  const size_t m = alpha.size();
  if (m == 0) return 1.0;
  std::vector<double> a(m), b(m > 0 ? m - 1 : 0);
  for (size_t j = 0; j < m; ++j) {
    a[j] = 1.0 / alpha[j] + (j > 0 ? beta[j] / alpha[j - 1] : 0.0);
    if (j + 1 < m) b[j] = std::sqrt(beta[j + 1]) / alpha[j];
  }
  double lo = 1e300, hi = -1e300;
  for (size_t i = 0; i < m; ++i) {
    const double r = (i ? std::fabs(b[i - 1]) : 0.0) + (i + 1 < m ? std::fabs(b[i]) : 0.0);
    lo = std::min(lo, a[i] - r);
    hi = std::max(hi, a[i] + r);
  }
  auto kth = [&](int k) {  // k-th smallest eigenvalue (0-based)
    double l = lo, h = hi;
    for (int it = 0; it < 200; ++it) {
      const double mid = 0.5 * (l + h);
      if (sturm_count(a, b, mid) > k) h = mid; else l = mid;
    }
    return 0.5 * (l + h);
  };
  const double emin = kth(0), emax = kth((int)m - 1);
  return emin > 0 ? emax / emin : INFINITY;
}

// ---------------------------------------------------------------------------
// FETI_LOG=2 (or more) in the environment: wall time of each setup stage on
// stderr (the stream is synchronised after each stage, only then).
// Runs f(i) for i in [0, n) on up to 16 host threads, chunks taken in order
// from a shared counter.  Every caller writes only the slots of its own
// index, so the result does not depend on the number of threads.
template <class F>
void par_for(int64_t n, int64_t chunk, F&& f) {
  const int64_t nchunks = (n + chunk - 1) / std::max<int64_t>(chunk, 1);
  int T = (int)std::min<int64_t>(nchunks, std::min(16u, std::max(1u, std::thread::hardware_concurrency())));
  if (T <= 1) {
    for (int64_t i = 0; i < n; ++i) f(i);
    return;
  }
  std::atomic<int64_t> next(0);
  auto work = [&]() {
    for (;;) {
      const int64_t c = next.fetch_add(1);
      if (c >= nchunks) break;
      const int64_t e = std::min(n, (c + 1) * chunk);
      for (int64_t i = c * chunk; i < e; ++i) f(i);
    }
  };
  std::vector<std::thread> pool;
  for (int t = 1; t < T; ++t) pool.emplace_back(work);
  work();
  for (auto& t : pool) t.join();
}

struct StageLog {
  feti_ctx* ctx;
  bool on;
  std::chrono::steady_clock::time_point t;
  explicit StageLog(feti_ctx* c) : ctx(c) {
    const char* e = std::getenv("FETI_LOG");
    on = e && e[0] >= '2' && e[0] <= '9';
    t = std::chrono::steady_clock::now();
  }
  void mark(const char* what) {
    if (!on) return;
    cudaStreamSynchronize(ctx->stream);
    const auto now = std::chrono::steady_clock::now();
    std::fprintf(stderr, "feti: %-28s %9.2f ms\n", what, std::chrono::duration<double, std::milli>(now - t).count());
    t = now;
  }
};

// Main-loop wait budget of the kernels with bounded mbarrier waits: ns,
// converted to SM clock cycles at the device's maximum clock (rounded down)
// and written to the context's device word; 0 cycles = give up at the first
// check.
constexpr unsigned long long kDefaultSpinNs = 100000000ull;

// Sparse coarse problem: used from this many coarse columns on (automatic
// form); supernodes of at most kCoarseLeaf subdomains below the separators;
// a front with at most kCoarseMergeBytes of factor per sweep runs each sweep
// as one task, larger fronts in row tasks of about kCoarseTaskBytes.
constexpr int64_t kCoarseSparseMin = 1536;
constexpr int kCoarseLeaf = 8;
constexpr int kCoarseTaskBytes = 49152;
constexpr int kCoarseMergeBytes = 98304;

// Uploads the coarse plan and allocates the factor, the sweep scratch (for up
// to kMaxRhs vectors), the task flags and counters (zero) and the wait flag.
feti_status upload_coarse(feti_ctx* ctx) {
  if (ctx->dry) return FETI_OK;
  const feti::CoarsePlan& cp = ctx->cplan;
  std::vector<int32_t> lvl;
  ctx->cdev.lvl_off.clear();
  for (const auto& L : cp.level_fronts) {
    ctx->cdev.lvl_off.push_back((int64_t)lvl.size());
    lvl.insert(lvl.end(), L.begin(), L.end());
  }
  feti::CoarseFront* fr = nullptr;
  feti::CoarseChild* ch = nullptr;
  feti::CoarseTask* tk = nullptr;
  feti::CoarsePlace* pl = nullptr;
  int32_t *map = nullptr, *nat = nullptr, *dep = nullptr, *dlvl = nullptr, *gptr = nullptr, *gsrc = nullptr;
  FETI_TRY(upload(ctx, &fr, cp.fronts));
  FETI_TRY(upload(ctx, &ch, cp.child));
  FETI_TRY(upload(ctx, &map, cp.map));
  FETI_TRY(upload(ctx, &nat, cp.nat));
  FETI_TRY(upload(ctx, &tk, cp.tasks));
  FETI_TRY(upload(ctx, &dep, cp.dep));
  FETI_TRY(upload(ctx, &pl, cp.place));
  FETI_TRY(upload(ctx, &dlvl, lvl));
  FETI_TRY(upload(ctx, &gptr, cp.gptr));
  FETI_TRY(upload(ctx, &gsrc, cp.gsrc));
  double *Dm = nullptr, *Lm = nullptr, *yt = nullptr, *out = nullptr;
  unsigned *flag = nullptr, *ctr = nullptr;
  FETI_TRY(dev_alloc(ctx, &Dm, cp.nD));
  FETI_TRY(dev_alloc(ctx, &Lm, cp.nL));
  FETI_TRY(dev_alloc(ctx, &yt, (size_t)ctx->cd * feti::kMaxRhs));
  FETI_TRY(dev_alloc(ctx, &out, (size_t)std::max<int32_t>(cp.n_out, 1) * feti::kMaxRhs));
  FETI_TRY(dev_alloc(ctx, &flag, cp.tasks.size()));
  FETI_TRY(dev_alloc(ctx, &ctr, 3));
  FETI_TRY(dev_alloc(ctx, &ctx->d_coarse_err, 1));
  FETI_CK(cudaMemsetAsync(flag, 0, std::max<size_t>(cp.tasks.size(), 1) * sizeof(unsigned), ctx->stream));
  FETI_CK(cudaMemsetAsync(ctr, 0, 3 * sizeof(unsigned), ctx->stream));
  FETI_CK(cudaMemsetAsync(ctx->d_coarse_err, 0, sizeof(int), ctx->stream));
  ctx->cdev.fr = fr;
  ctx->cdev.child = ch;
  ctx->cdev.map = map;
  ctx->cdev.place = pl;
  ctx->cdev.lvl = dlvl;
  ctx->cdev.Dm = Dm;
  ctx->cdev.Lm = Lm;
  feti::CoarseDag& d = ctx->cdag;
  d.fr = fr;
  d.child = ch;
  d.map = map;
  d.nat = nat;
  d.task = tk;
  d.dep = dep;
  d.gptr = gptr;
  d.gsrc = gsrc;
  d.Dm = Dm;
  d.Lm = Lm;
  d.yt = yt;
  d.out = out;
  d.flag = flag;
  d.ctr = ctr;
  d.n_tasks = (int)cp.tasks.size();
  d.smem1 = cp.smem1;
  d.smem16 = cp.smem16;
  return FETI_OK;
}
feti_status set_spin_budget(feti_ctx* ctx, uint64_t ns) {
  int khz = 0;
  FETI_CK(cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, ctx->device));
  const double cyc = (double)ns * (khz > 0 ? khz : 2000000) * 1e-6;
  const unsigned long long v = cyc > 9.0e18 ? 9000000000000000000ull : (unsigned long long)cyc;
  FETI_CK(cudaMemcpyAsync(ctx->d_spin, &v, sizeof(v), cudaMemcpyHostToDevice, ctx->stream));
  FETI_CK(cudaStreamSynchronize(ctx->stream));
  return FETI_OK;
}

feti_status build_decomposition(feti_ctx* ctx) {
  StageLog lg(ctx);
  const int N = ctx->N, E = ctx->E, P = ctx->P;
  ctx->af = ctx->opt.method == FETI_ALL_FLOATING;
  // elements grouped by subdomain (ascending), then the local nodes of each
  // subdomain (ascending), subdomains in parallel
  std::vector<int32_t> sub_elem_ptr(P + 1, 0), sub_elems(E);
  for (int e = 0; e < E; ++e) sub_elem_ptr[ctx->part[e] + 1]++;
  for (int s = 0; s < P; ++s) {
    if (sub_elem_ptr[s + 1] == 0) return fail(ctx, FETI_ERR_PARTITION, "subdomain " + std::to_string(s) + " has no elements");
    sub_elem_ptr[s + 1] += sub_elem_ptr[s];
  }
  {
    std::vector<int32_t> f2(sub_elem_ptr.begin(), sub_elem_ptr.end() - 1);
    for (int e = 0; e < E; ++e) sub_elems[f2[ctx->part[e]]++] = e;
  }
  ctx->nodes.assign(P, {});
  par_for(P, 4, [&](int64_t s) {
    // first visits marked in a per-thread table (cleared again below), so
    // only the distinct nodes are sorted
    thread_local std::vector<char> seen;
    if (seen.size() < (size_t)N) seen.assign(N, 0);
    auto& v = ctx->nodes[s];
    for (int q = sub_elem_ptr[s]; q < sub_elem_ptr[s + 1]; ++q)
      for (int a = 0; a < ctx->npe; ++a) {
        const int n = ctx->tets[(size_t)ctx->npe * sub_elems[q] + a];
        if (!seen[n]) {
          seen[n] = 1;
          v.push_back(n);
        }
      }
    for (int n : v) seen[n] = 0;
    std::sort(v.begin(), v.end());
  });
  lg.mark("create:   local node lists");
  // node -> subdomains (ascending)
  std::vector<int32_t> nptr(N + 1, 0);
  for (int s = 0; s < P; ++s)
    for (int n : ctx->nodes[s]) nptr[n + 1]++;
  for (int n = 0; n < N; ++n) nptr[n + 1] += nptr[n];
  // nsub[a]: the subdomains of each node (ascending); lcopy[a]: the node's
  // local index in subdomain nsub[a]
  std::vector<int32_t> nsub(nptr[N]), lcopy(nptr[N]), fill(nptr.begin(), nptr.end() - 1);
  for (int s = 0; s < P; ++s)
    for (size_t l = 0; l < ctx->nodes[s].size(); ++l) {
      const int n = ctx->nodes[s][l];
      lcopy[fill[n]] = (int32_t)l;
      nsub[fill[n]++] = s;
    }
  auto lnode = [&](int s, int n) {
    for (int a = nptr[n]; a < nptr[n + 1]; ++a)
      if (nsub[a] == s) return (int)lcopy[a];
    return -1;
  };
  lg.mark("create:   node -> subdomains");
  std::vector<char> is_dir(3 * (size_t)N, 0);
  std::vector<double> dval(3 * (size_t)N, 0.0);
  for (size_t i = 0; i < ctx->dir_dof.size(); ++i) {
    is_dir[ctx->dir_dof[i]] = 1;
    dval[ctx->dir_dof[i]] = ctx->dir_val[i];
  }
  const bool af = ctx->af;
  // multiplier rows in canonical order
  auto& rs = ctx->row_sub;
  auto& rl = ctx->row_ldof;
  auto& rg = ctx->row_sign;
  auto& rw = ctx->weight;
  auto& rb = ctx->bvec;
  rs.clear(); rl.clear(); rg.clear(); rw.clear(); rb.clear();
  {
    // row count first: every node shared by m subdomains gives m (m - 1) / 2
    // rows per component (all-floating: plus one per subdomain copy of a
    // Dirichlet DOF)
    int64_t nrow = 0;
    for (int n = 0; n < N; ++n) {
      const int64_t m = nptr[n + 1] - nptr[n];
      nrow += 3 * (m * (m - 1) / 2);
    }
    if (af)
      for (size_t q = 0; q < ctx->dir_dof.size(); ++q) nrow += nptr[ctx->dir_dof[q] / 3 + 1] - nptr[ctx->dir_dof[q] / 3];
    rs.reserve(2 * nrow); rl.reserve(2 * nrow); rg.reserve(2 * nrow); rw.reserve(nrow); rb.reserve(nrow);
  }
  for (int n = 0; n < N; ++n) {
    const int m = nptr[n + 1] - nptr[n];
    if (m < 2) continue;
    for (int c = 0; c < 3; ++c) {
      const int dof = 3 * n + c;
      if (!af && is_dir[dof]) continue;
      const double w = (af && is_dir[dof]) ? 0.0 : 1.0 / m;
      for (int a = nptr[n]; a < nptr[n + 1]; ++a)
        for (int b = a + 1; b < nptr[n + 1]; ++b) {
          const int i = nsub[a], j = nsub[b];
          rs.push_back(i); rs.push_back(j);
          rl.push_back(3 * lcopy[a] + c); rl.push_back(3 * lcopy[b] + c);
          rg.push_back(1); rg.push_back(-1);
          rw.push_back(w);
          rb.push_back(0.0);
        }
    }
  }
  if (af) {
    for (size_t q = 0; q < ctx->dir_dof.size(); ++q) {
      const int dof = ctx->dir_dof[q], n = dof / 3, c = dof % 3;
      for (int a = nptr[n]; a < nptr[n + 1]; ++a) {
        const int i = nsub[a];
        rs.push_back(i); rs.push_back(-1);
        rl.push_back(3 * lcopy[a] + c); rl.push_back(-1);
        rg.push_back(1); rg.push_back(0);
        rw.push_back(1.0);
        rb.push_back(ctx->dir_val[q]);
      }
    }
  }
  lg.mark("create: local nodes, multipliers");
  ctx->n_lambda = (int64_t)rw.size();
  if (ctx->n_lambda == 0) return fail(ctx, FETI_ERR_PARTITION, "decomposition has no multipliers");
  // boundary flags per subdomain local DOF
  std::vector<std::vector<char>> bflag(P);
  for (int s = 0; s < P; ++s) bflag[s].assign(3 * ctx->nodes[s].size(), 0);
  for (int64_t r = 0; r < ctx->n_lambda; ++r)
    for (int e = 0; e < 2; ++e)
      if (rs[2 * r + e] >= 0) bflag[rs[2 * r + e]][rl[2 * r + e]] = 1;
  lg.mark("create:   boundary flags, element groups");
  // per subdomain: free DOFs, kernels, fixing DOFs, dense order
  ctx->lay.assign(P, SubLayout{});
  std::vector<std::vector<int32_t>> env0(P);  // per interior-elimination step: (eI, nbact)
  std::vector<std::vector<int32_t>> env0w(P);  // the same for kChol32Block-column steps
  ctx->fix_ptr.assign(P + 1, 0);
  ctx->fix_ldof.clear();
  std::vector<std::vector<int32_t>> dense_ldof(P);  // dense index -> local DOF
  std::vector<std::vector<double>> Rd(P);           // R in dense order, n x k
  int64_t aoff = 0, soff = 0, foff = 0, roff = 0, foff32 = 0, soff32 = 0, fsym = 0, ssym = 0, psym = 0;
  int boff = 0, voff = 0, coff = 0;
  // per subdomain (in parallel): free DOFs, kernel basis, fixing DOFs, dense
  // order, envelope and R in dense order; sizes and offsets after
  struct SubInfo {
    int k = 0, nI = 0, nbp = 0, n = 0;
    std::vector<int32_t> fix;
    feti_status err = FETI_OK;
    const char* msg = nullptr;
  };
  std::vector<SubInfo> info(P);
  par_for(P, 1, [&](int64_t s) {
    SubInfo& si = info[s];
    const auto& nod = ctx->nodes[s];
    const int nl = (int)nod.size(), nd = 3 * nl;
    std::vector<char> free(nd, 1);
    if (!af)
      for (int l = 0; l < nl; ++l)
        for (int c = 0; c < 3; ++c)
          if (is_dir[3 * (size_t)nod[l] + c]) free[3 * l + c] = 0;
    // rigid-body modes about the mean node position (Sec. 4.3)
    double cx = 0, cy = 0, cz = 0;
    for (int n : nod) {
      cx += ctx->coords[3 * (size_t)n];
      cy += ctx->coords[3 * (size_t)n + 1];
      cz += ctx->coords[3 * (size_t)n + 2];
    }
    cx /= nl; cy /= nl; cz /= nl;
    std::vector<double> rbm((size_t)nd * 6, 0.0);
    for (int l = 0; l < nl; ++l) {
      const double dx = ctx->coords[3 * (size_t)nod[l]] - cx, dy = ctx->coords[3 * (size_t)nod[l] + 1] - cy,
                   dz = ctx->coords[3 * (size_t)nod[l] + 2] - cz;
      double* r0 = &rbm[(3 * l + 0) * 6];
      double* r1 = &rbm[(3 * l + 1) * 6];
      double* r2 = &rbm[(3 * l + 2) * 6];
      r0[0] = 1.0; r1[1] = 1.0; r2[2] = 1.0;
      r0[3] = -dy; r1[3] = dx;   // e_z x d
      r1[4] = -dz; r2[4] = dy;   // e_x x d
      r2[5] = -dx; r0[5] = dz;   // e_y x d
    }
    // kernel basis N (6 x k): all-floating -> identity; classical -> null
    // space of the modes restricted to the Dirichlet DOFs (Sec. 4.3).
    std::vector<double> Nb;
    int k = 6;
    if (af) {
      Nb.assign(36, 0.0);
      for (int i = 0; i < 6; ++i) Nb[i * 6 + i] = 1.0;
    } else {
      double M[6][6] = {};
      int ncons = 0;
      for (int d = 0; d < nd; ++d)
        if (!free[d]) {
          ++ncons;
          for (int i = 0; i < 6; ++i)
            for (int j = 0; j < 6; ++j) M[i][j] += rbm[d * 6 + i] * rbm[d * 6 + j];
        }
      double V[6][6], w[6];
      jacobi6(M, V, w);
      double wmax = 0.0;
      for (int i = 0; i < 6; ++i) wmax = std::max(wmax, w[i]);
      std::vector<int> nullc;
      for (int i = 0; i < 6; ++i)
        if (ncons == 0 || w[i] <= 1e-12 * wmax) nullc.push_back(i);
      k = (int)nullc.size();
      Nb.assign(6 * (size_t)k, 0.0);
      for (int i = 0; i < 6; ++i)
        for (int a = 0; a < k; ++a) Nb[i * k + a] = V[i][nullc[a]];
    }
    // R on local DOFs (nd x k)
    std::vector<double> Rl((size_t)nd * k, 0.0);
    for (int d = 0; d < nd; ++d)
      for (int a = 0; a < k; ++a) {
        double t = 0.0;
        for (int i = 0; i < 6; ++i) t += rbm[d * 6 + i] * Nb[i * k + a];
        Rl[(size_t)d * k + a] = t;
      }
    // boundary DOFs ascending, then pivoted selection of k fixing DOFs
    std::vector<int32_t> bl;
    for (int d = 0; d < nd; ++d)
      if (free[d] && bflag[s][d]) bl.push_back(d);
    std::vector<int32_t> fix;
    if (k > 0) {
      if ((int)bl.size() < k) {
        si.err = FETI_ERR_KERNEL_DETECT;
        si.msg = "too few boundary DOFs to fix the kernel";
        return;
      }
      std::vector<double> W((size_t)bl.size() * k);
      for (size_t i = 0; i < bl.size(); ++i)
        for (int a = 0; a < k; ++a) W[i * k + a] = Rl[(size_t)bl[i] * k + a];
      std::vector<char> chosen(bl.size(), 0);
      for (int it = 0; it < k; ++it) {
        double top = -1.0;
        std::vector<double> nrm(bl.size(), -1.0);
        for (size_t i = 0; i < bl.size(); ++i) {
          if (chosen[i]) continue;
          double t = 0.0;
          for (int a = 0; a < k; ++a) t += W[i * k + a] * W[i * k + a];
          nrm[i] = t;
          top = std::max(top, t);
        }
        size_t j = 0;
        for (size_t i = 0; i < bl.size(); ++i)
          if (!chosen[i] && nrm[i] >= top * (1.0 - 1e-10)) { j = i; break; }
        if (!(top > 0.0)) {
          si.err = FETI_ERR_KERNEL_DETECT;
          si.msg = "kernel basis vanishes on the boundary";
          return;
        }
        chosen[j] = 1;
        fix.push_back(bl[j]);
        std::vector<double> qv(k);
        const double inv = 1.0 / std::sqrt(nrm[j]);
        for (int a = 0; a < k; ++a) qv[a] = W[j * k + a] * inv;
        for (size_t i = 0; i < bl.size(); ++i) {
          double t = 0.0;
          for (int a = 0; a < k; ++a) t += W[i * k + a] * qv[a];
          for (int a = 0; a < k; ++a) W[i * k + a] -= t * qv[a];
        }
      }
    }
    std::vector<char> isfix(nd, 0);
    for (int d : fix) isfix[d] = 1;
    auto& dl = dense_ldof[s];
    for (int d = 0; d < nd; ++d)
      if (free[d] && !bflag[s][d]) dl.push_back(d);
    const int nI = (int)dl.size();
    // Envelope of the interior columns: per local DOF, the first interior
    // dense position it couples to through an element of this subdomain (nI
    // if none).  Cholesky fill stays inside the envelope, so a row is zero in
    // every interior column left of that position.
    std::vector<int32_t> dof_first(nd, nI);
    {
      std::vector<int32_t> own(nl, nI), node_first(nl, nI);
      for (int i = 0; i < nI; ++i) own[dl[i] / 3] = std::min(own[dl[i] / 3], i);
      for (int q = sub_elem_ptr[s]; q < sub_elem_ptr[s + 1]; ++q) {
        const int e = sub_elems[q];
        int ln[10], m = nI;
        for (int a = 0; a < ctx->npe; ++a) {
          ln[a] = lnode(s, ctx->tets[(size_t)ctx->npe * e + a]);
          m = std::min(m, own[ln[a]]);
        }
        for (int a = 0; a < ctx->npe; ++a) node_first[ln[a]] = std::min(node_first[ln[a]], m);
      }
      for (int d = 0; d < nd; ++d) dof_first[d] = node_first[d / 3];
    }
    // boundary DOFs (fixing DOFs excepted) by envelope start, so that the rows
    // an interior block column can reach form a prefix of the boundary block
    std::vector<int32_t> bsort;
    for (int d : bl)
      if (!isfix[d]) bsort.push_back(d);
    std::stable_sort(bsort.begin(), bsort.end(),
                     [&](int32_t a, int32_t b) { return dof_first[a] < dof_first[b]; });
    for (int d : bsort) dl.push_back(d);
    const int nbp = (int)dl.size() - nI;
    {
      // last[v] = the last interior row whose envelope starts left of column v
      std::vector<int32_t> last(nI + 1, -1);
      for (int r = 0; r < nI; ++r) last[dof_first[dl[r]] + 1] = std::max(last[dof_first[dl[r]] + 1], r);
      for (int v = 1; v <= nI; ++v) last[v] = std::max(last[v], last[v - 1]);
      std::vector<int32_t> bfirst(nbp);
      for (int i = 0; i < nbp; ++i) bfirst[i] = dof_first[bsort[i]];
      for (int w = 0; w < 2; ++w) {
        auto& ev = w == 0 ? env0[s] : env0w[s];
        const int B = w == 0 ? 32 : feti::kChol32Block;
        for (int kb = 0; kb < nI; kb += B) {
          const int r0 = kb + std::min(B, nI - kb);
          ev.push_back(std::max(r0, last[r0] + 1));
          ev.push_back((int32_t)(std::lower_bound(bfirst.begin(), bfirst.end(), r0) - bfirst.begin()));
        }
      }
    }
    for (int d : fix) dl.push_back(d);
    const int n = (int)dl.size();
    Rd[s].assign((size_t)n * k, 0.0);
    for (int i = 0; i < n; ++i)
      for (int a = 0; a < k; ++a) Rd[s][(size_t)i * k + a] = Rl[(size_t)dl[i] * k + a];
    si.k = k;
    si.nI = nI;
    si.nbp = nbp;
    si.n = n;
    si.fix = std::move(fix);
  });
  for (int s = 0; s < P; ++s)
    if (info[s].err != FETI_OK) return fail(ctx, info[s].err, info[s].msg);
  for (int s = 0; s < P; ++s) {
    const SubInfo& si = info[s];
    const int n = si.n, nI = si.nI, nbp = si.nbp, k = si.k;
    SubLayout L{};
    L.n = n; L.nI = nI; L.nbp = nbp; L.k = k; L.ld = n + nbp;
    L.boff = boff; L.voff = voff; L.coff = coff;
    L.aoff = aoff; L.soff = soff; L.foff = foff; L.roff = roff;
    L.foff32 = foff32; L.soff32 = soff32;
    L.fsym32 = fsym; L.ssym32 = ssym; L.psym = psym;
    ctx->lay[s] = L;
    const int nb = nbp + k;
    {
      constexpr int64_t PH = feti::kSymPH;
      const int64_t pf = (nbp + PH - 1) / PH, ps = (nb + PH - 1) / PH;
      fsym += PH * PH / 2 * pf * (pf + 1);
      ssym += PH * PH / 2 * ps * (ps + 1);
      psym += PH / 2 * ps * (ps - 1);  // sized for the larger (preconditioner) block
    }
    boff += nb;
    voff += n;
    coff += k;
    aoff += (int64_t)L.ld * L.ld;
    soff += (int64_t)nb * nb;
    foff += (int64_t)nbp * nbp;
    roff += (int64_t)n * k;
    foff32 += (int64_t)nbp * ((nbp + 3) & ~3);
    soff32 += (int64_t)nb * ((nb + 3) & ~3);
    ctx->max_nb = std::max(ctx->max_nb, nb);
    for (int d : si.fix) ctx->fix_ldof.push_back(d);
    ctx->fix_ptr[s + 1] = (int32_t)ctx->fix_ldof.size();
  }
  lg.mark("create: kernels, fixing, dense order");
  ctx->nb_total = boff;
  // compact interior factor: rows [0, nI + nbp) x columns [0, nI) per subdomain
  {
    int64_t lo = 0;
    for (auto& L : ctx->lay) {
      L.loff = lo;
      lo += (int64_t)(L.nI + L.nbp) * feti::kp_ld(L);
    }
    ctx->lc_elems = lo;
  }
  // elimination groups: consecutive subdomains whose dense matrices fit the
  // workspace budget (at least one per group)
  {
    ctx->keep_factor = ctx->opt.local_form == 2;
    const int64_t esz = ctx->opt.precision == FETI_MIXED_F32FACTOR ? 4 : 8;
    const int64_t mb = ctx->opt.workspace_mb == 0 ? 12288 : ctx->opt.workspace_mb;
    const int64_t cap = (ctx->keep_factor || mb < 0) ? INT64_MAX : (mb << 20) / esz;
    ctx->grp.assign(1, 0);
    ctx->ws_full = aoff;
    ctx->ws_elems = 0;
    int64_t acc = 0;
    for (int s = 0; s < P; ++s) {
      const int64_t m = (int64_t)ctx->lay[s].ld * ctx->lay[s].ld;
      if (acc > 0 && acc + m > cap) {
        ctx->grp.push_back(s);
        acc = 0;
      }
      acc += m;
      ctx->ws_elems = std::max(ctx->ws_elems, acc);
    }
    ctx->grp.push_back(P);
  }
  const int n_grp = (int)ctx->grp.size() - 1;
  std::vector<SubLayout> lay_ws(ctx->lay);
  for (int g = 0; g < n_grp; ++g)
    for (int s = ctx->grp[g]; s < ctx->grp[g + 1]; ++s) lay_ws[s].aoff -= ctx->lay[ctx->grp[g]].aoff;
  FETI_TRY(upload(ctx, &ctx->d_lay_ws, lay_ws));
  // envelope tables of the interior elimination, [step][subdomain of the group][2] per group
  auto env_tables = [&](const std::vector<std::vector<int32_t>>& ev, std::vector<int32_t>& tab,
                        std::vector<int64_t>& off) {
    tab.clear();
    off.assign(n_grp, 0);
    for (int g = 0; g < n_grp; ++g) {
      const int s0 = ctx->grp[g], pg = ctx->grp[g + 1] - s0;
      int steps = 0;
      for (int s = s0; s < s0 + pg; ++s) steps = std::max(steps, (int)ev[s].size() / 2);
      off[g] = (int64_t)tab.size();
      tab.resize(tab.size() + 2 * (size_t)steps * pg, 0);
      for (int s = s0; s < s0 + pg; ++s)
        for (size_t t = 0; t < ev[s].size() / 2; ++t) {
          tab[off[g] + 2 * (t * pg + (s - s0))] = ev[s][2 * t];
          tab[off[g] + 2 * (t * pg + (s - s0)) + 1] = ev[s][2 * t + 1];
        }
    }
  };
  env_tables(env0, ctx->env0, ctx->env_off);
  FETI_TRY(upload(ctx, &ctx->d_env0, ctx->env0));
  if (ctx->opt.precision == FETI_MIXED_F32FACTOR) {
    env_tables(env0w, ctx->env0_32, ctx->env32_off);
    FETI_TRY(upload(ctx, &ctx->d_env0_32, ctx->env0_32));
  }
  for (const auto& L : ctx->lay) ctx->max_nr = std::max(ctx->max_nr, L.nI + L.nbp);
  ctx->nloc_total = voff;
  ctx->cd = coff;
  // dense position lookup per subdomain: local DOF -> dense index
  std::vector<std::vector<int32_t>> pos_of(P);
  for (int s = 0; s < P; ++s) {
    pos_of[s].assign(3 * ctx->nodes[s].size(), -1);
    for (size_t i = 0; i < dense_ldof[s].size(); ++i) pos_of[s][dense_ldof[s][i]] = (int32_t)i;
  }
  lg.mark("create:   dense positions");
  // device maps
  std::vector<int32_t> row_pos(2 * ctx->n_lambda, -1);
  std::vector<double> row_sgn(2 * ctx->n_lambda, 0.0);
  std::vector<int32_t> bt_cnt(ctx->nb_total + 1, 0);
  for (int64_t r = 0; r < ctx->n_lambda; ++r)
    for (int e = 0; e < 2; ++e) {
      const int s = rs[2 * r + e];
      if (s < 0) continue;
      const SubLayout& L = ctx->lay[s];
      const int di = pos_of[s][rl[2 * r + e]];
      if (di < L.nI) return fail(ctx, FETI_ERR_PARTITION, "internal: multiplier on an interior DOF");
      row_pos[2 * r + e] = L.boff + di - L.nI;
      row_sgn[2 * r + e] = rg[2 * r + e];
      bt_cnt[L.boff + di - L.nI + 1]++;
    }
  for (int64_t i = 0; i < ctx->nb_total; ++i) bt_cnt[i + 1] += bt_cnt[i];
  std::vector<int32_t> bt_row(bt_cnt[ctx->nb_total]);
  std::vector<double> bt_sgn(bt_cnt[ctx->nb_total]);
  {
    std::vector<int32_t> f2(bt_cnt.begin(), bt_cnt.end() - 1);
    for (int64_t r = 0; r < ctx->n_lambda; ++r)
      for (int e = 0; e < 2; ++e) {
        const int gp = row_pos[2 * r + e];
        if (gp < 0) continue;
        bt_row[f2[gp]] = (int32_t)r;
        bt_sgn[f2[gp]] = row_sgn[2 * r + e];
        f2[gp]++;
      }
  }
  std::vector<int32_t> bpos_sub(ctx->nb_total);
  for (int s = 0; s < P; ++s)
    for (int p = 0; p < ctx->lay[s].nbp + ctx->lay[s].k; ++p) bpos_sub[ctx->lay[s].boff + p] = s;
  lg.mark("create:   multiplier maps");
  // dense maps of the elements (grouped by subdomain above)
  const int npe = ctx->npe, nde = ctx->nde, fpn = ctx->fpn;
  hvec<int32_t> elem_dense((size_t)nde * E);  // every entry written below
  std::vector<double> elem_dirval;
  ctx->any_dirval = false;
  if (!af)
    for (double v : ctx->dir_val)
      if (v != 0.0) ctx->any_dirval = true;
  if (ctx->any_dirval) elem_dirval.assign((size_t)nde * E, 0.0);
  par_for(P, 4, [&](int64_t s) {
    // the subdomain's local node numbers in a per-thread table (cleared again below)
    thread_local std::vector<int32_t> lof;
    if (lof.size() < (size_t)N) lof.assign(N, -1);
    const auto& nd = ctx->nodes[s];
    for (size_t l = 0; l < nd.size(); ++l) lof[nd[l]] = (int32_t)l;
    for (int q = sub_elem_ptr[s]; q < sub_elem_ptr[s + 1]; ++q) {
      const int e = sub_elems[q];
      for (int a = 0; a < npe; ++a) {
        const int n = ctx->tets[(size_t)npe * e + a];
        const int l = lof[n];
        for (int c = 0; c < 3; ++c) {
          elem_dense[(size_t)nde * e + 3 * a + c] = pos_of[s][3 * l + c];
          if (ctx->any_dirval && is_dir[3 * (size_t)n + c])
            elem_dirval[(size_t)nde * e + 3 * a + c] = dval[3 * (size_t)n + c];
        }
      }
    }
    for (int n : nd) lof[n] = -1;
  });
  lg.mark("create:   element dense maps");
  // FP32-factor form: per local row (global local index voff + dense row) the
  // (element, element row) pairs of its subdomain's elements, ascending
  // (encoded nde e + a)
  if (ctx->opt.precision == FETI_MIXED_F32FACTOR) {
    // a subdomain's rows are touched only by its own elements: count and fill
    // per subdomain in parallel, elements ascending (each row's list ascends
    // in nde e + a)
    std::vector<int32_t> kptr(voff + 1, 0);
    par_for(P, 4, [&](int64_t s) {
      const SubLayout& L = ctx->lay[s];
      for (int q = sub_elem_ptr[s]; q < sub_elem_ptr[s + 1]; ++q) {
        const int e = sub_elems[q];
        for (int a = 0; a < nde; ++a) {
          const int r = elem_dense[(size_t)nde * e + a];
          if (r >= 0) kptr[L.voff + r + 1]++;
        }
      }
    });
    for (int i = 0; i < voff; ++i) kptr[i + 1] += kptr[i];
    hvec<int32_t> kinc(kptr[voff]);  // every slot written below
    std::vector<int32_t> kf(kptr.begin(), kptr.end() - 1);
    par_for(P, 4, [&](int64_t s) {
      const SubLayout& L = ctx->lay[s];
      for (int q = sub_elem_ptr[s]; q < sub_elem_ptr[s + 1]; ++q) {
        const int e = sub_elems[q];
        for (int a = 0; a < nde; ++a) {
          const int r = elem_dense[(size_t)nde * e + a];
          if (r >= 0) kinc[kf[L.voff + r]++] = nde * e + a;
        }
      }
    });
    FETI_TRY(upload(ctx, &ctx->d_kinc_ptr, kptr));
    FETI_TRY(upload(ctx, &ctx->d_kinc, kinc));
    {
      hvec<int32_t> es(E), rsub(voff);  // every element and every local row belongs to one subdomain
      par_for(P, 16, [&](int64_t s) {
        for (int q = sub_elem_ptr[s]; q < sub_elem_ptr[s + 1]; ++q) es[sub_elems[q]] = (int32_t)s;
        for (int i = 0; i < ctx->lay[s].n; ++i) rsub[ctx->lay[s].voff + i] = (int32_t)s;
      });
      FETI_TRY(upload(ctx, &ctx->d_elem_sub, es));
      FETI_TRY(upload(ctx, &ctx->d_row_sub, rsub));
    }
  }
  lg.mark("create:   refinement incidences");
  // lumped preconditioner: CSR pattern of K_bb over the global boundary
  // positions, from the boundary DOF pairs that share an element
  std::vector<int32_t> lump_ptr, lump_col;
  std::vector<int64_t> lump_src;
  if (ctx->opt.precond == FETI_PREC_LUMPED) {
    std::vector<std::vector<int32_t>> rows(ctx->nb_total);
    for (int e = 0; e < E; ++e) {
      const SubLayout& L = ctx->lay[ctx->part[e]];
      int bp[30], nbq = 0;
      for (int a = 0; a < nde; ++a) {
        const int di = elem_dense[(size_t)nde * e + a];
        if (di >= L.nI) bp[nbq++] = di - L.nI;
      }
      for (int x = 0; x < nbq; ++x)
        for (int y = 0; y < nbq; ++y) rows[L.boff + bp[x]].push_back(L.boff + bp[y]);
    }
    lump_ptr.assign(1, 0);
    ctx->lump_grp.clear();
    for (int s = 0; s < P; ++s) {
      const SubLayout& L = lay_ws[s];
      if (std::binary_search(ctx->grp.begin(), ctx->grp.end(), s)) ctx->lump_grp.push_back((int64_t)lump_col.size());
      for (int p = 0; p < L.nbp + L.k; ++p) {
        auto& r = rows[L.boff + p];
        std::sort(r.begin(), r.end());
        r.erase(std::unique(r.begin(), r.end()), r.end());
        for (int gq : r) {
          const int q = gq - L.boff;
          const int i = std::max(p, q), j = std::min(p, q);
          lump_col.push_back(gq);
          lump_src.push_back(L.aoff + (int64_t)(L.nI + i) * L.ld + (L.nI + j));
        }
        lump_ptr.push_back((int32_t)lump_col.size());
      }
    }
    ctx->lump_nnz = (int64_t)lump_col.size();
    ctx->lump_grp.push_back(ctx->lump_nnz);
  }
  // faces grouped by owning subdomain
  const int nf = ctx->n_press + ctx->n_trac;
  std::vector<int32_t> sub_face_ptr(P + 1, 0), face_order(nf), face_dense(3 * (size_t)fpn * nf, -1);
  for (int f = 0; f < nf; ++f) sub_face_ptr[ctx->part[ctx->face_owner[f]] + 1]++;
  for (int s = 0; s < P; ++s) sub_face_ptr[s + 1] += sub_face_ptr[s];
  {
    std::vector<int32_t> f2(sub_face_ptr.begin(), sub_face_ptr.end() - 1);
    for (int f = 0; f < nf; ++f) face_order[f2[ctx->part[ctx->face_owner[f]]]++] = f;
  }
  // face_dense indexed by the grouped position; face forces are permuted to it
  std::vector<int32_t> face_tri_grouped((size_t)fpn * nf);
  std::vector<int32_t> face_kind(nf);
  for (int q = 0; q < nf; ++q) {
    const int f = face_order[q];
    const int s = ctx->part[ctx->face_owner[f]];
    for (int v = 0; v < fpn; ++v) {
      const int n = ctx->face_tri[(size_t)fpn * f + v];
      const auto& nod = ctx->nodes[s];
      auto it = std::lower_bound(nod.begin(), nod.end(), n);
      if (it == nod.end() || *it != n) return fail(ctx, FETI_ERR_INVALID_ARG, "loaded face not on its owner element");
      const int l = (int)(it - nod.begin());
      for (int c = 0; c < 3; ++c) face_dense[3 * (size_t)fpn * q + 3 * v + c] = pos_of[s][3 * l + c];
      face_tri_grouped[(size_t)fpn * q + v] = n;
    }
    face_kind[q] = f < ctx->n_press ? 0 : 1;
  }
  // owner rule for the global displacement: lowest subdomain id per free DOF
  std::vector<int32_t> own_gdof, own_vpos;
  {
    std::vector<char> taken(3 * (size_t)N, 0);
    for (int s = 0; s < P; ++s) {
      const SubLayout& L = ctx->lay[s];
      for (int i = 0; i < L.n; ++i) {
        const int d = dense_ldof[s][i];
        const int g = 3 * ctx->nodes[s][d / 3] + d % 3;
        if (taken[g]) continue;
        taken[g] = 1;
        own_gdof.push_back(g);
        own_vpos.push_back(L.voff + i);
      }
    }
  }
  ctx->n_own = (int)own_gdof.size();
  lg.mark("create:   lumped pattern, faces, owners");
  // global non-Dirichlet DOF -> local copies (for residual norms)
  std::vector<int32_t> gs_ptr, gs_pos;
  {
    std::vector<int32_t> cnt(3 * (size_t)N + 1, 0);
    for (int s = 0; s < P; ++s)
      for (int i = 0; i < ctx->lay[s].n; ++i) {
        const int d = dense_ldof[s][i];
        const int g = 3 * ctx->nodes[s][d / 3] + d % 3;
        if (!is_dir[g]) cnt[g + 1]++;
      }
    std::vector<int32_t> gid(3 * (size_t)N, -1);
    gs_ptr.push_back(0);
    for (size_t g = 0; g < 3 * (size_t)N; ++g)
      if (cnt[g + 1] > 0) {
        gid[g] = (int32_t)gs_ptr.size() - 1;
        gs_ptr.push_back(gs_ptr.back() + cnt[g + 1]);
      }
    gs_pos.assign(gs_ptr.back(), 0);
    std::vector<int32_t> fill2(gs_ptr.begin(), gs_ptr.end() - 1);
    for (int s = 0; s < P; ++s)
      for (int i = 0; i < ctx->lay[s].n; ++i) {
        const int d = dense_ldof[s][i];
        const int g = 3 * ctx->nodes[s][d / 3] + d % 3;
        if (!is_dir[g]) gs_pos[fill2[gid[g]]++] = ctx->lay[s].voff + i;
      }
    if (ctx->mat.kind == FETI_HGO_TWO_FIBRE) {
      // Newton-Krylov maps: gs row -> global DOF, element DOF -> gs row (-1:
      // Dirichlet), and per gs row its incident (element, local row) pairs
      std::vector<int32_t> gs_gdof;
      for (size_t g = 0; g < 3 * (size_t)N; ++g)
        if (gid[g] >= 0) gs_gdof.push_back((int32_t)g);
      std::vector<int32_t> elem_gs(12 * (size_t)E), inc_ptr(gs_gdof.size() + 1, 0), inc;
      for (int e = 0; e < E; ++e)
        for (int a = 0; a < 12; ++a) {
          const int j = gid[3 * ctx->tets[4 * (size_t)e + a / 3] + a % 3];
          elem_gs[12 * (size_t)e + a] = j;
          if (j >= 0) inc_ptr[j + 1]++;
        }
      for (size_t j = 0; j < gs_gdof.size(); ++j) inc_ptr[j + 1] += inc_ptr[j];
      inc.assign(inc_ptr.back(), 0);
      std::vector<int32_t> fill3(inc_ptr.begin(), inc_ptr.end() - 1);
      for (int e = 0; e < E; ++e)
        for (int a = 0; a < 12; ++a) {
          const int j = elem_gs[12 * (size_t)e + a];
          if (j >= 0) inc[fill3[j]++] = 12 * e + a;
        }
      FETI_TRY(upload(ctx, &ctx->d_gs_gdof, gs_gdof));
      FETI_TRY(upload(ctx, &ctx->d_elem_gs, elem_gs));
      FETI_TRY(upload(ctx, &ctx->d_inc_ptr, inc_ptr));
      FETI_TRY(upload(ctx, &ctx->d_inc, inc));
    }
  }
  ctx->n_gs = (int)gs_ptr.size() - 1;
  ctx->U_init.assign(3 * (size_t)N, 0.0);
  if (!af)
    for (size_t i = 0; i < ctx->dir_dof.size(); ++i) ctx->U_init[ctx->dir_dof[i]] = ctx->dir_val[i];
  lg.mark("create:   global-DOF and Newton maps, uploads");
  // coarse G^T G pair blocks (i <= j, ascending), each with the multiplier
  // rows that couple them, ascending
  std::vector<int32_t> gi, gj, gptr(1, 0), grows;
  {
    // per subdomain i with a kernel (in parallel): the multiplier rows of its
    // boundary positions, ascending, grouped by the other subdomain j of each
    // row (j > i with a kernel; the diagonal block takes every row), so the
    // blocks come out in (i, j) order; then concatenated
    struct SubBlocks {
      std::vector<int32_t> j, ptr, rows;
    };
    std::vector<SubBlocks> sb(P);
    par_for(P, 4, [&](int64_t i) {
      const SubLayout& L = ctx->lay[i];
      if (L.k == 0) return;
      std::vector<int32_t> rr;
      for (int p = 0; p < L.nbp + L.k; ++p)
        for (int e = bt_cnt[L.boff + p]; e < bt_cnt[L.boff + p + 1]; ++e) rr.push_back(bt_row[e]);
      std::sort(rr.begin(), rr.end());
      rr.erase(std::unique(rr.begin(), rr.end()), rr.end());
      // (other subdomain, row) for the off-diagonal blocks
      std::vector<std::pair<int32_t, int32_t>> od;
      for (int32_t r : rr) {
        const int a0 = rs[2 * (int64_t)r], a1 = rs[2 * (int64_t)r + 1];
        const int j = a0 == (int)i ? a1 : a0;
        if (j > (int)i && ctx->lay[j].k > 0) od.emplace_back(j, r);
      }
      std::sort(od.begin(), od.end());
      SubBlocks& B = sb[i];
      B.j.push_back((int32_t)i);
      B.ptr.push_back(0);
      B.rows = rr;
      for (size_t q = 0; q < od.size(); ++q) {
        if (q == 0 || od[q].first != od[q - 1].first) {
          B.ptr.push_back((int32_t)B.rows.size());
          B.j.push_back(od[q].first);
        }
        B.rows.push_back(od[q].second);
      }
      B.ptr.push_back((int32_t)B.rows.size());
    });
    for (int i = 0; i < P; ++i) {
      const SubBlocks& B = sb[i];
      for (size_t q = 0; q < B.j.size(); ++q) {
        gi.push_back(i);
        gj.push_back(B.j[q]);
        grows.insert(grows.end(), B.rows.begin() + B.ptr[q], B.rows.begin() + B.ptr[q + 1]);
        gptr.push_back((int32_t)grows.size());
      }
    }
  }
  ctx->n_gtg = (int)gi.size();
  lg.mark("create: maps, coarse blocks");
  {
    const int form = ctx->opt.coarse_form;
    ctx->coarse_sparse = ctx->cd > 0 && (form == 2 || (form == 0 && ctx->cd >= kCoarseSparseMin));
    if (ctx->coarse_sparse) {
      std::vector<int32_t> kk(P), co(P);
      for (int s = 0; s < P; ++s) {
        kk[s] = ctx->lay[s].k;
        co[s] = ctx->lay[s].coff;
      }
      std::string e;
      if (!feti::coarse_plan(P, kk.data(), co.data(), gi, gj, kCoarseLeaf, kCoarseTaskBytes, kCoarseMergeBytes,
                              &ctx->cplan, &e))
        return fail(ctx, FETI_ERR_PARTITION, e);
      lg.mark("create: coarse ordering and supernodes");
    }
  }
  // gemv block tables
  std::vector<int32_t> tab_sub[2][3], tab_row[2][3];
  const int rpcs[3] = {32, 64, 128};
  for (int w = 0; w < 2; ++w)
    for (int t = 0; t < 3; ++t)
      for (int s = 0; s < P; ++s) {
        const SubLayout& L = ctx->lay[s];
        const int m = w == 0 ? std::max(L.nbp, 1) : L.nbp + L.k;
        ctx->tab_ptr[w][t].push_back((int32_t)tab_sub[w][t].size());
        for (int r0 = 0; r0 < m; r0 += rpcs[t]) { tab_sub[w][t].push_back(s); tab_row[w][t].push_back(r0); }
        if (s == P - 1) ctx->tab_ptr[w][t].push_back((int32_t)tab_sub[w][t].size());
      }
  // chunks of 256 boundary positions for the projection's G^T v
  std::vector<int32_t> chunk_sub, chunk_p0, sub_chunk_ptr(P + 1, 0), col_sub(std::max<int64_t>(ctx->cd, 1), 0);
  for (int s = 0; s < P; ++s) {
    const SubLayout& L = ctx->lay[s];
    if (L.k > 0)
      for (int p0 = 0; p0 < L.nbp + L.k; p0 += 256) { chunk_sub.push_back(s); chunk_p0.push_back(p0); }
    sub_chunk_ptr[s + 1] = (int32_t)chunk_sub.size();
    for (int a = 0; a < L.k; ++a) col_sub[L.coff + a] = s;
  }
  ctx->n_chunks = (int)chunk_sub.size();
  hvec<double> Rall(roff);  // every subdomain's n x k block copied below
  par_for(P, 8, [&](int64_t s) { std::copy(Rd[s].begin(), Rd[s].end(), Rall.begin() + ctx->lay[s].roff); });

  lg.mark("create: tables");
  // ---- uploads and allocations
  FETI_TRY(upload(ctx, &ctx->d_coords, ctx->coords));
  FETI_TRY(upload(ctx, &ctx->d_tets, ctx->tets));
  if (!ctx->fibres.empty()) FETI_TRY(upload(ctx, &ctx->d_fibres, ctx->fibres));
  FETI_TRY(upload(ctx, &ctx->d_lay, ctx->lay));
  FETI_TRY(upload(ctx, &ctx->d_sub_elem_ptr, sub_elem_ptr));
  FETI_TRY(upload(ctx, &ctx->d_sub_elems, sub_elems));
  FETI_TRY(upload(ctx, &ctx->d_elem_dense, elem_dense));
  if (ctx->any_dirval) FETI_TRY(upload(ctx, &ctx->d_elem_dirval, elem_dirval));
  FETI_TRY(upload(ctx, &ctx->d_sub_face_ptr, sub_face_ptr));
  FETI_TRY(upload(ctx, &ctx->d_face_dense, face_dense));
  FETI_TRY(upload(ctx, &ctx->d_face_tri, face_tri_grouped));
  {
    std::vector<double> tr(ctx->traction, ctx->traction + 3);
    FETI_TRY(upload(ctx, &ctx->d_traction, tr));
  }
  FETI_TRY(upload(ctx, &ctx->d_row_pos, row_pos));
  FETI_TRY(upload(ctx, &ctx->d_row_sgn, row_sgn));
  FETI_TRY(upload(ctx, &ctx->d_weight, ctx->weight));
  FETI_TRY(upload(ctx, &ctx->d_b, ctx->bvec));
  FETI_TRY(upload(ctx, &ctx->d_bt_ptr, bt_cnt));
  FETI_TRY(upload(ctx, &ctx->d_bt_row, bt_row));
  FETI_TRY(upload(ctx, &ctx->d_bt_sgn, bt_sgn));
  FETI_TRY(upload(ctx, &ctx->d_bpos_sub, bpos_sub));
  for (int w = 0; w < 2; ++w)
    for (int t = 0; t < 3; ++t) {
      int32_t *ds = nullptr, *dr = nullptr;
      FETI_TRY(upload(ctx, &ds, tab_sub[w][t]));
      FETI_TRY(upload(ctx, &dr, tab_row[w][t]));
      feti::GemvCfg& c = ctx->tab[w][t];
      c.rpc = rpcs[t];
      c.n_blocks = (int)tab_sub[w][t].size();
      c.blk_sub = ds;
      c.blk_row0 = dr;
    }
  for (int w = 0; w < 2; ++w) {
    ctx->cfg64[w] = ctx->tab[w][0];  // R=4, 32 rows per CTA
    ctx->cfg64[w].R = 4;
    ctx->cfg32[w] = ctx->tab[w][1];  // R=8, 64 rows per CTA
    ctx->cfg32[w].R = 8;
  }
  FETI_TRY(upload(ctx, &ctx->d_chunk_sub, chunk_sub));
  FETI_TRY(upload(ctx, &ctx->d_chunk_p0, chunk_p0));
  FETI_TRY(upload(ctx, &ctx->d_sub_chunk_ptr, sub_chunk_ptr));
  FETI_TRY(upload(ctx, &ctx->d_col_sub, col_sub));
  FETI_TRY(dev_alloc(ctx, &ctx->d_gpart, 6 * (size_t)std::max(ctx->n_chunks, 1)));
  FETI_TRY(upload(ctx, &ctx->d_gtg_i, gi));
  FETI_TRY(upload(ctx, &ctx->d_gtg_j, gj));
  FETI_TRY(upload(ctx, &ctx->d_gtg_ptr, gptr));
  FETI_TRY(upload(ctx, &ctx->d_gtg_rows, grows));
  if (ctx->coarse_sparse) FETI_TRY(upload_coarse(ctx));
  FETI_TRY(upload(ctx, &ctx->d_R, Rall));
  FETI_TRY(upload(ctx, &ctx->d_own_gdof, own_gdof));
  FETI_TRY(upload(ctx, &ctx->d_gs_ptr, gs_ptr));
  if (ctx->opt.precond == FETI_PREC_LUMPED) {
    FETI_TRY(upload(ctx, &ctx->d_lump_ptr, lump_ptr));
    FETI_TRY(upload(ctx, &ctx->d_lump_col, lump_col));
    FETI_TRY(upload(ctx, &ctx->d_lump_src, lump_src));
    FETI_TRY(dev_alloc(ctx, &ctx->d_lump_val, ctx->lump_nnz));
  }
  FETI_TRY(upload(ctx, &ctx->d_dir_dof, ctx->dir_dof));
  FETI_TRY(upload(ctx, &ctx->d_gs_pos, gs_pos));
  FETI_TRY(upload(ctx, &ctx->d_own_vpos, own_vpos));
  FETI_TRY(upload(ctx, &ctx->d_Uinit, ctx->U_init));
  FETI_TRY(dev_alloc(ctx, &ctx->d_Uout, 3 * (size_t)N));
  ctx->face_kind.swap(face_kind);
  FETI_TRY(dev_alloc(ctx, &ctx->d_face_force, 3 * (size_t)fpn * std::max(nf, 1)));
  FETI_TRY(dev_alloc(ctx, &ctx->d_Ke, (size_t)feti::ke_packed(nde) * E));
  if (ctx->mat.kind == FETI_HGO_TWO_FIBRE) {
    FETI_TRY(dev_alloc(ctx, &ctx->d_fe, 12 * (size_t)E));
    FETI_TRY(dev_alloc(ctx, &ctx->d_U, 3 * (size_t)N));
    FETI_TRY(dev_alloc(ctx, &ctx->d_dU, 3 * (size_t)N));
    FETI_TRY(dev_alloc(ctx, &ctx->d_Utrial, 3 * (size_t)N));
    FETI_TRY(dev_alloc(ctx, &ctx->d_fl, ctx->nloc_total));
  }
  // the dense local operators (the bulk of the memory) are allocated by the
  // first setup, so that element-only use of a context does not hold them
  ctx->op_elems[0] = ctx->ws_elems;
  ctx->op_elems[1] = ctx->opt.precond == FETI_PREC_DIRICHLET ? soff : 1;
  ctx->op_elems[2] = foff;
  ctx->op_elems[3] = foff32;
  ctx->op_elems[4] = ctx->opt.precond == FETI_PREC_DIRICHLET ? soff32 : 1;
  ctx->op_elems[5] = fsym;
  ctx->op_elems[6] = ctx->opt.precond == FETI_PREC_DIRICHLET ? ssym : 1;
  ctx->op_elems[7] = psym;
  for (int w = 0; w < 2; ++w) {
    // symmetric-apply work lists: one warp per (subdomain, kSymPH-row panel).
    // Panel I carries I + 1 blocks, so the list runs from the longest panels
    // to the shortest and the eight warps of a CTA take the same panel index
    // of eight subdomains: balanced CTAs, longest work first.
    std::vector<int32_t> ws, wp;
    int max_np = 0;
    for (int q = 0; q < P; ++q) {
      const int m = w == 0 ? ctx->lay[q].nbp : ctx->lay[q].nbp + ctx->lay[q].k;
      max_np = std::max(max_np, (m + feti::kSymPH - 1) / feti::kSymPH);
    }
    for (int I = max_np - 1; I >= 0; --I)
      for (int q = 0; q < P; ++q) {
        const int m = w == 0 ? ctx->lay[q].nbp : ctx->lay[q].nbp + ctx->lay[q].k;
        if (I < (m + feti::kSymPH - 1) / feti::kSymPH) {
          ws.push_back(q);
          wp.push_back(I);
        }
      }
    ctx->sym_n[w] = (int)ws.size();
    FETI_TRY(upload(ctx, &ctx->d_sym_sub[w], ws));
    FETI_TRY(upload(ctx, &ctx->d_sym_panel[w], wp));
    std::vector<int32_t> ord(P);
    std::iota(ord.begin(), ord.end(), 0);
    auto msz = [&](int q) { return w == 0 ? ctx->lay[q].nbp : ctx->lay[q].nbp + ctx->lay[q].k; };
    std::stable_sort(ord.begin(), ord.end(), [&](int32_t a, int32_t b) { return msz(a) > msz(b); });
    ctx->sym_max_m[w] = P > 0 ? msz(ord[0]) : 0;
    FETI_TRY(upload(ctx, &ctx->d_sym_order[w], ord));
  }
  FETI_TRY(dev_alloc(ctx, &ctx->d_f, ctx->nloc_total));
  FETI_TRY(dev_alloc(ctx, &ctx->d_x, ctx->nloc_total));
  FETI_TRY(dev_alloc(ctx, &ctx->d_x2, ctx->nloc_total));
  const size_t nlam = ctx->n_lambda;
  for (double** v : {&ctx->d_lam, &ctx->d_r, &ctx->d_w, &ctx->d_z, &ctx->d_y, &ctx->d_p, &ctx->d_q, &ctx->d_d})
    FETI_TRY(dev_alloc(ctx, v, nlam));
  FETI_TRY(dev_alloc(ctx, &ctx->d_loc, ctx->nb_total));
  FETI_TRY(dev_alloc(ctx, &ctx->d_vloc, ctx->nb_total));
  FETI_TRY(dev_alloc(ctx, &ctx->d_vloc32, ctx->nb_total + 4));
  FETI_TRY(dev_alloc(ctx, &ctx->d_dl, ctx->n_lambda));
  FETI_TRY(dev_alloc(ctx, &ctx->d_g, std::max<int64_t>(ctx->cd, 1)));
  FETI_TRY(dev_alloc(ctx, &ctx->d_c, std::max<int64_t>(ctx->cd, 1)));
  FETI_TRY(dev_alloc(ctx, &ctx->d_e, std::max<int64_t>(ctx->cd, 1)));
  FETI_TRY(dev_alloc(ctx, &ctx->d_partial, feti::scatter_partials()));
  FETI_TRY(dev_alloc(ctx, &ctx->d_partial_wy, feti::scatter_partials()));
  FETI_TRY(dev_alloc(ctx, &ctx->d_partial_pq, feti::scatter_partials()));
  FETI_TRY(dev_alloc(ctx, &ctx->d_alpha_hist, ctx->opt.maxit + 2));
  FETI_TRY(dev_alloc(ctx, &ctx->d_beta_hist, ctx->opt.maxit + 2));
  FETI_TRY(dev_alloc(ctx, &ctx->d_sc, 1));
  FETI_TRY(dev_alloc(ctx, &ctx->d_status, 1));
  FETI_TRY(dev_alloc(ctx, &ctx->d_zero, 1));
  FETI_TRY(dev_alloc(ctx, &ctx->d_spin, 1));
  if (ctx->dry) return FETI_OK;  // host plan: nothing on a device
  FETI_TRY(set_spin_budget(ctx, ctx->opt.spin_timeout_ns ? ctx->opt.spin_timeout_ns : kDefaultSpinNs));
  FETI_CK(cudaMemsetAsync(ctx->d_zero, 0, sizeof(int), ctx->stream));
  FETI_CK(cudaMemsetAsync(ctx->d_status, 0, sizeof(int), ctx->stream));
  if (ctx->cd > 0 && !ctx->coarse_sparse) {
    FETI_TRY(dev_alloc(ctx, &ctx->d_Ginv, (size_t)ctx->cd * ctx->cd));
    SubLayout Lc{};
    Lc.n = (int)ctx->cd; Lc.nI = 0; Lc.nbp = (int)ctx->cd; Lc.k = 0; Lc.ld = 2 * (int)ctx->cd;
    std::vector<SubLayout> lc(1, Lc);
    FETI_TRY(upload(ctx, &ctx->d_lay_coarse, lc));
  }
  FETI_CK(cudaMallocHost(&ctx->h_sc, sizeof(feti::PcgScalars)));
  FETI_CK(cudaMallocHost(&ctx->h_status, sizeof(int)));
  ctx->maps.n_lambda = (int)ctx->n_lambda;
  ctx->maps.nb_total = (int)ctx->nb_total;
  ctx->maps.row_pos = ctx->d_row_pos;
  ctx->maps.row_sgn = ctx->d_row_sgn;
  ctx->maps.weight = ctx->d_weight;
  ctx->maps.bt_ptr = ctx->d_bt_ptr;
  ctx->maps.bt_row = ctx->d_bt_row;
  ctx->maps.bt_sgn = ctx->d_bt_sgn;
  ctx->maps.bpos_sub = ctx->d_bpos_sub;
  FETI_CK(cudaStreamSynchronize(ctx->stream));
  return FETI_OK;
}

feti_status check_status(feti_ctx* ctx, const char* where) {
  FETI_CK(cudaMemcpyAsync(ctx->h_status, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  FETI_CK(cudaStreamSynchronize(ctx->stream));
  const int s = *ctx->h_status;
  if (s != 0) {
    FETI_CK(cudaMemsetAsync(ctx->d_status, 0, sizeof(int), ctx->stream));
    FETI_CK(cudaStreamSynchronize(ctx->stream));
  }
  if (s == feti::DEV_LOCAL_SINGULAR) return fail(ctx, FETI_ERR_LOCAL_SINGULAR, std::string(where) + ": non-positive pivot");
  if (s == feti::DEV_INVERTED) return fail(ctx, FETI_ERR_ELEMENT_INVERTED, std::string(where) + ": inverted element");
  if (s != 0) return fail(ctx, FETI_ERR_CUDA, std::string(where) + ": device status " + std::to_string(s));
  return FETI_OK;
}

// A bounded device wait that ran out (flag set by the kernel): FETI_ERR_TIMEOUT,
// flag cleared so the context stays usable.
feti_status check_wait_flag(feti_ctx* ctx, int* d_flag, const char* where) {
  if (!d_flag) return FETI_OK;
  int herr = 0;
  FETI_CK(cudaMemcpyAsync(&herr, d_flag, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  FETI_CK(cudaStreamSynchronize(ctx->stream));
  if (!herr) return FETI_OK;
  FETI_CK(cudaMemsetAsync(d_flag, 0, sizeof(int), ctx->stream));
  FETI_CK(cudaStreamSynchronize(ctx->stream));
  return fail(ctx, FETI_ERR_TIMEOUT, std::string(where) + ": a bounded wait ran out");
}

// Element matrices at U (device pointer or NULL), local assembly, loads.
// Element matrices at dU (device or NULL): the two-fibre tangent and force,
// Hooke P1 (linear, and P2-P0 on P1 where the element mean of div u is div u),
// or Hooke P2 / P2-P0 on 10-node tetrahedra.
void launch_elements(feti_ctx* ctx, const double* dU) {
  cudaStream_t st = ctx->stream;
  if (ctx->mat.kind == FETI_HGO_TWO_FIBRE)
    feti::launch_elem_hgo(ctx->E, ctx->d_coords, ctx->d_tets, dU, ctx->d_fibres, ctx->mat.c, ctx->mat.k1,
                          ctx->mat.k2, ctx->mat.kappa, ctx->d_Ke, ctx->d_fe, ctx->d_status, st);
  else if (ctx->npe == 10)
    feti::launch_elem_linear_p2(ctx->E, ctx->d_coords, ctx->d_tets, ctx->mat.E, ctx->mat.nu,
                                ctx->mat.kind == FETI_LINEAR_ISO_P0 ? 1 : 0, ctx->d_Ke, ctx->d_status, st);
  else
    feti::launch_elem_linear(ctx->E, ctx->d_coords, ctx->d_tets, ctx->mat.E, ctx->mat.nu, ctx->d_Ke,
                             ctx->d_status, st);
}

feti_status assemble_all(feti_ctx* ctx, const double* dU, double tau) {
  cudaStream_t st = ctx->stream;
  const bool hgo = ctx->mat.kind == FETI_HGO_TWO_FIBRE;
  launch_elements(ctx, dU);
  FETI_CK(cudaGetLastError());
  // face forces (grouped order; kind per face)
  const int nf = ctx->n_press + ctx->n_trac;
  if (nf > 0) {
    // faces are grouped by subdomain, so the two kinds may interleave: launch
    // one force pass per run of equal kind
    int q = 0;
    while (q < nf) {
      const int kind = ctx->face_kind[q];
      int q1 = q;
      while (q1 < nf && ctx->face_kind[q1] == kind) ++q1;
      feti::launch_face_forces(q1 - q, ctx->fpn, ctx->d_face_tri + (size_t)ctx->fpn * q, ctx->d_coords,
                               (hgo && ctx->opt.follower) ? dU : nullptr, kind, kind == 0 ? ctx->pressure : 1.0,
                               ctx->d_traction, ctx->d_face_force + 3 * (size_t)ctx->fpn * q, st);
      q = q1;
    }
  }
  feti::launch_assemble_rhs(ctx->P, ctx->d_lay, ctx->d_sub_face_ptr, ctx->d_face_dense, ctx->d_face_force,
                            3 * ctx->fpn, ctx->d_sub_elem_ptr, ctx->d_sub_elems, ctx->d_elem_dense,
                            ctx->d_elem_dirval, ctx->d_Ke, hgo ? ctx->d_fe : nullptr, ctx->nde, tau, ctx->d_f, st);
  FETI_CK(cudaGetLastError());
  return check_status(ctx, "element/assembly");
}

// Dense local apply of F_i (which 0) or the preconditioner block (which 1)
// on a gathered local vector (default: d_vloc / d_vloc32) into yout
// (default: d_loc).
void gemv_apply(feti_ctx* ctx, int which, const int* done, bool f32, const void* vin = nullptr,
                double* yout = nullptr);

// r = g - K_rr x in FP64 from the element matrices (zero on the fixing rows).
void kresid(feti_ctx* ctx, const double* g, const double* x, double* r) {
  feti::launch_kresid2(ctx->E, ctx->nde, ctx->d_elem_sub, ctx->d_row_sub, (int)ctx->nloc_total, ctx->d_lay,
                       ctx->d_kinc_ptr, ctx->d_kinc, ctx->d_elem_dense, ctx->d_Ke, g, x, ctx->d_kye, r, ctx->stream);
}

// One FP32 correction x (+)= L^-T L^-1 r (init: x = it) with the triangular
// sweeps confined to the interior rows and the boundary block through the
// explicit FP32 F_i (the autotuned operator kernel of the PCG).
void kplus_corr(feti_ctx* ctx, const double* r, double* x, bool init) {
  feti::launch_kp_forward(ctx->P, ctx->d_lay, ctx->d_Lc32, r, ctx->d_kyI, ctx->d_kzb, ctx->max_nr, ctx->stream);
  gemv_apply(ctx, 0, ctx->d_zero, true, ctx->d_kzb, ctx->d_kxb);
  feti::launch_kp_backward(ctx->P, ctx->d_lay, ctx->d_Lc32, ctx->d_kyI, ctx->d_kxb, x, init ? 1 : 0, ctx->max_nr,
                           ctx->stream);
}

// x = K^+ g on full local vectors (zero on the fixing DOFs).  FP64
// factorizations: sweeps over the whole factor where it is kept (implicit
// local form), else K_rr^-1 in its block form from the compact interior
// factor and the FP64 F_i = S_i[b',b']^-1: y_I = L_II^-1 g_I,
// z_b = g_b - L_bI y_I, x_b = F_i z_b, x_I = L_II^-T (y_I - L_bI^T x_b).
// FP32 factorizations: the same block form in FP32, refined against the FP64
// element matrices (refine_steps corrections; d_kr is scratch).
void kplus(feti_ctx* ctx, const double* g, double* x) {
  cudaStream_t st = ctx->stream;
  if (ctx->keep_factor) {
    feti::launch_kplus(ctx->P, ctx->d_lay, ctx->d_A, g, x, st);
    return;
  }
  if (!f32_factor(ctx)) {
    feti::launch_kp_forward(ctx->P, ctx->d_lay, ctx->d_Lc, g, ctx->d_kyI64, ctx->d_kzb64, ctx->max_nr, st);
    gemv_apply(ctx, 0, ctx->d_zero, false, ctx->d_kzb64, ctx->d_kxb);
    feti::launch_kp_backward(ctx->P, ctx->d_lay, ctx->d_Lc, ctx->d_kyI64, ctx->d_kxb, x, 1, ctx->max_nr, st);
    return;
  }
  kplus_corr(ctx, g, x, true);
  for (int k = 1; k < ctx->refine_steps; ++k) {
    kresid(ctx, g, x, ctx->d_kr);
    kplus_corr(ctx, ctx->d_kr, x, false);
  }
}

// Number of refinement corrections of the FP32-factor K^+: applied to a fixed
// pseudo-random vector, corrections are added while the largest relative
// residual over the subdomains, ||g - K_rr x|| / ||g||, still falls by at
// least half and is above 1e-14 (at most 12).
feti_status tune_refinement(feti_ctx* ctx) {
  cudaStream_t st = ctx->stream;
  const int P = ctx->P;
  feti::launch_fill_mix(ctx->nloc_total, ctx->d_kg, st);
  kplus_corr(ctx, ctx->d_kg, ctx->d_x2, true);
  std::vector<double> nrm(2 * (size_t)P);
  double prev = 1e300;
  int steps = 1;
  for (; steps <= 12; ++steps) {
    kresid(ctx, ctx->d_kg, ctx->d_x2, ctx->d_kr);
    feti::launch_sub_norm2(P, ctx->d_lay, ctx->d_kr, ctx->d_kg, ctx->d_knorm, st);
    FETI_CK(cudaGetLastError());
    FETI_CK(cudaMemcpyAsync(nrm.data(), ctx->d_knorm, nrm.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
    FETI_CK(cudaStreamSynchronize(st));
    double worst = 0.0;
    for (int q = 0; q < P; ++q)
      if (nrm[2 * q + 1] > 0.0) worst = std::max(worst, std::sqrt(nrm[2 * q] / nrm[2 * q + 1]));
    if (!std::isfinite(worst)) return fail(ctx, FETI_ERR_LOCAL_SINGULAR, "FP32 factor: refinement diverged");
    ctx->refine_res = worst;
    if (worst <= 1e-14 || worst > 0.5 * prev || steps == 12) break;
    prev = worst;
    kplus_corr(ctx, ctx->d_kr, ctx->d_x2, false);
  }
  if (ctx->refine_res > 1e-6)
    return fail(ctx, FETI_ERR_LOCAL_SINGULAR, "FP32 factor: refinement does not converge (residual " +
                                                  std::to_string(ctx->refine_res) + ")");
  ctx->refine_steps = steps;
  const char* e = std::getenv("FETI_LOG");
  if (e && e[0] >= '2' && e[0] <= '9') {  // one correction and one residual, timed
    cudaEvent_t a, b, c;
    FETI_CK(cudaEventCreate(&a));
    FETI_CK(cudaEventCreate(&b));
    FETI_CK(cudaEventCreate(&c));
    FETI_CK(cudaEventRecord(a, st));
    kplus_corr(ctx, ctx->d_kr, ctx->d_x2, false);
    FETI_CK(cudaEventRecord(b, st));
    kresid(ctx, ctx->d_kg, ctx->d_x2, ctx->d_kr);
    FETI_CK(cudaEventRecord(c, st));
    FETI_CK(cudaEventSynchronize(c));
    float t1 = 0.f, t2 = 0.f;
    FETI_CK(cudaEventElapsedTime(&t1, a, b));
    FETI_CK(cudaEventElapsedTime(&t2, b, c));
    std::fprintf(stderr, "feti: refinement %d corrections, residual %.2e; correction %.3f ms, residual %.3f ms\n",
                 steps, ctx->refine_res, t1, t2);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaEventDestroy(c);
  }
  return FETI_OK;
}

// Local factorizations, dense local operators, coarse problem.
// One elimination group in the workspace: assembly of the dense matrices,
// interior elimination, S_i, boundary elimination, F_i, and the compact
// interior factor.  T is the factorization's precision.  Returns the first
// error of the enqueueing calls.
template <typename T>
cudaError_t factorize_group(feti_ctx* ctx, int g, T* A, const std::vector<int32_t>& envt, const std::vector<int64_t>& eoff,
                     const int32_t* d_env, int B, double* S64, float* S32,
                     float* S32s, double* F64, float* F32, float* F32s, T* Lc) {
  cudaStream_t st = ctx->stream;
  const int s0 = ctx->grp[g], pg = ctx->grp[g + 1] - s0;
  const SubLayout* lw = ctx->d_lay_ws + s0;
  int64_t elems = 0;
  for (int s = s0; s < s0 + pg; ++s) elems += (int64_t)ctx->lay[s].ld * ctx->lay[s].ld;
  const cudaError_t e = cudaMemsetAsync(A, 0, (size_t)elems * sizeof(T), st);
  if (e != cudaSuccess) return e;
  feti::launch_assemble(pg, lw, ctx->d_sub_elem_ptr + s0, ctx->d_sub_elems, ctx->d_elem_dense, ctx->d_Ke, ctx->nde,
                        A, st);
  if constexpr (sizeof(T) == 8) {
    if (ctx->shift > 0.0) feti::launch_shift_diag(pg, lw, A, ctx->shift, st);
  }
  feti::launch_augment(pg, lw, A, st);
  if (ctx->opt.precond == FETI_PREC_LUMPED) {
    const int64_t i0 = ctx->lump_grp[g], i1 = ctx->lump_grp[g + 1];
    feti::launch_lump_fill((long)(i1 - i0), ctx->d_lump_src + i0, A, ctx->d_lump_val + i0, st);
  }
  // per step, the largest trailing chunk count over the group's subdomains
  // (steps of B columns)
  std::vector<int> chunks[2];
  for (int phase = 0; phase < 2; ++phase)
    for (int s = s0; s < s0 + pg; ++s) {
      const SubLayout& L = ctx->lay[s];
      const int c0 = phase == 0 ? 0 : L.nI, c1 = phase == 0 ? L.nI : L.nI + L.nbp;
      for (int t = 0, kb = c0; kb < c1; ++t, kb += B) {
        const int r0 = kb + std::min(B, c1 - kb);
        // phase 0: the rows inside the envelope (interior rows up to eI, the
        // first nbact boundary rows, the fixing rows); phase 1: all remaining
        // rows plus the augmentation rows of the columns eliminated so far
        int m;
        if (phase == 0) {
          const int32_t* ev = &envt[eoff[g] + 2 * ((size_t)t * pg + (s - s0))];
          m = (ev[0] - r0) + ev[1] + L.k;
        } else {
          m = std::min(L.ld, L.n + r0 - L.nI) - r0;
        }
        const int ch = (m + 63) / 64;
        if ((int)chunks[phase].size() <= t) chunks[phase].push_back(0);
        chunks[phase][t] = std::max(chunks[phase][t], ch);
      }
    }
  feti::launch_chol_batched(pg, lw, 0, chunks[0].data(), (int)chunks[0].size(), d_env + eoff[g], A, ctx->d_status,
                            st);
  if (ctx->opt.precond == FETI_PREC_DIRICHLET)
    feti::launch_extract_tiles(pg, ctx->max_nb, lw, 0, A, S64, S32, S32s, st);
  feti::launch_chol_batched(pg, lw, 1, chunks[1].data(), (int)chunks[1].size(), nullptr, A, ctx->d_status, st);
  feti::launch_extract_tiles(pg, ctx->max_nb, lw, 1, A, F64, F32, F32s, st);
  if (Lc) feti::launch_compact_factor(pg, ctx->max_nr, lw, A, Lc, st);
  return cudaGetLastError();
}

feti_status factorize_all(feti_ctx* ctx) {
  const int n_grp = (int)ctx->grp.size() - 1;
  if (f32_factor(ctx)) {
    // FP32 elimination; S_i and F_i go straight into the FP32 operator layouts
    for (int g = 0; g < n_grp; ++g)
      FETI_CK(factorize_group<float>(ctx, g, ctx->d_A32, ctx->env0_32, ctx->env32_off, ctx->d_env0_32,
                             feti::kChol32Block, nullptr, ctx->d_S32, ctx->d_S32s, nullptr, ctx->d_F32, ctx->d_F32s,
                             ctx->d_Lc32));
    FETI_TRY(check_status(ctx, "local factorization (FP32)"));
    return FETI_OK;
  }
  // FP64 operators, and in the FP32-local form their FP32 copies, in one pass each
  const bool mix = ctx->opt.precision == FETI_MIXED;
  for (int g = 0; g < n_grp; ++g)
    FETI_CK(factorize_group<double>(ctx, g, ctx->d_A, ctx->env0, ctx->env_off, ctx->d_env0, 32, ctx->d_S,
                            mix ? ctx->d_S32 : nullptr, mix ? ctx->d_S32s : nullptr, ctx->d_F,
                            mix ? ctx->d_F32 : nullptr, mix ? ctx->d_F32s : nullptr,
                            ctx->keep_factor ? nullptr : ctx->d_Lc));
  FETI_TRY(check_status(ctx, "local factorization"));
  return FETI_OK;
}

// Coarse problem, enqueued on the second stream (it needs only R_i and the
// multiplier maps, not the local factorizations, so it overlaps them; the
// FP64 elimination and an FP32 local factorization use different pipes).
// G^T G and the elimination workspace (5 cd^2 doubles) exist until
// coarse_join; the context keeps (G^T G)^-1.
feti_status coarse_begin(feti_ctx* ctx) {
  if (ctx->cd == 0) return FETI_OK;
  const size_t cd = ctx->cd;
  if (!ctx->stream2) {
    FETI_CK(cudaStreamCreateWithFlags(&ctx->stream2, cudaStreamNonBlocking));
    FETI_CK(cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming));
    FETI_CK(cudaEventCreateWithFlags(&ctx->ev_coarse, cudaEventDisableTiming));
    FETI_TRY(dev_alloc(ctx, &ctx->d_status2, 1));
  }
  if (ctx->coarse_sparse) {
    // supernodal factorization: fronts workspace only until joined
    cudaError_t e = cudaMalloc(&ctx->coarse_ws[0], std::max<int64_t>(ctx->cplan.ws, 1) * sizeof(double));
    if (e != cudaSuccess) {
      (void)cudaGetLastError();
      ctx->coarse_ws[0] = nullptr;
      return fail(ctx, e == cudaErrorMemoryAllocation ? FETI_ERR_OOM : FETI_ERR_CUDA,
                  std::string("coarse workspace: ") + cudaGetErrorString(e));
    }
    cudaStream_t st = ctx->stream2;
    FETI_CK(cudaEventRecord(ctx->ev_fork, ctx->stream));
    FETI_CK(cudaStreamWaitEvent(st, ctx->ev_fork, 0));
    FETI_CK(cudaMemsetAsync(ctx->d_status2, 0, sizeof(int), st));
    feti::launch_coarse_factor(ctx->cplan, ctx->cdev, ctx->d_gtg_i, ctx->d_gtg_j, ctx->d_gtg_ptr, ctx->d_gtg_rows,
                               ctx->n_gtg, ctx->d_lay, ctx->d_R, ctx->maps, static_cast<double*>(ctx->coarse_ws[0]),
                               ctx->d_status2, st);
    FETI_CK(cudaGetLastError());
    FETI_CK(cudaEventRecord(ctx->ev_coarse, st));
    ctx->coarse_pending = true;
    return FETI_OK;
  }
  {
    cudaError_t e = cudaMalloc(&ctx->coarse_ws[0], cd * cd * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&ctx->coarse_ws[1], 4 * cd * cd * sizeof(double));
    if (e != cudaSuccess) {
      (void)cudaGetLastError();
      for (void*& q : ctx->coarse_ws)
        if (q) { cudaFree(q); q = nullptr; }
      return fail(ctx, e == cudaErrorMemoryAllocation ? FETI_ERR_OOM : FETI_ERR_CUDA,
                  std::string("coarse workspace: ") + cudaGetErrorString(e));
    }
  }
  cudaStream_t st = ctx->stream2;
  FETI_CK(cudaEventRecord(ctx->ev_fork, ctx->stream));
  FETI_CK(cudaStreamWaitEvent(st, ctx->ev_fork, 0));
  double* GtG = static_cast<double*>(ctx->coarse_ws[0]);
  double* Ac = static_cast<double*>(ctx->coarse_ws[1]);
  FETI_CK(cudaMemsetAsync(ctx->d_status2, 0, sizeof(int), st));
  FETI_CK(cudaMemsetAsync(GtG, 0, cd * cd * sizeof(double), st));
  feti::launch_gtg(ctx->n_gtg, ctx->d_gtg_i, ctx->d_gtg_j, ctx->d_gtg_ptr, ctx->d_gtg_rows, ctx->d_lay, ctx->d_R,
                   ctx->maps, (int)cd, GtG, st);
  // [[G^T G, I], [I, 0]] eliminated over the first cd columns leaves -(G^T G)^-1
  FETI_CK(cudaMemsetAsync(Ac, 0, 4 * cd * cd * sizeof(double), st));
  FETI_CK(cudaMemcpy2DAsync(Ac, 2 * cd * sizeof(double), GtG, cd * sizeof(double), cd * sizeof(double), cd,
                            cudaMemcpyDeviceToDevice, st));
  feti::launch_augment(1, ctx->d_lay_coarse, Ac, st);
  feti::launch_dense_chol_big(Ac, 2 * (int)cd, 0, (int)cd, 2 * (int)cd, (int)cd, ctx->d_status2, st);
  // extract into Ginv: F layout of the coarse "subdomain" has foff = 0
  feti::launch_extract(1, ctx->d_lay_coarse, 1, Ac, ctx->d_Ginv, st);
  FETI_CK(cudaGetLastError());
  FETI_CK(cudaEventRecord(ctx->ev_coarse, st));
  ctx->coarse_pending = true;
  return FETI_OK;
}

// Joins the coarse setup into the context's stream, checks its status and
// frees its workspace.
feti_status coarse_join(feti_ctx* ctx) {
  if (!ctx->coarse_pending) return FETI_OK;
  ctx->coarse_pending = false;
  FETI_CK(cudaStreamWaitEvent(ctx->stream, ctx->ev_coarse, 0));
  int h = 0;
  FETI_CK(cudaMemcpyAsync(&h, ctx->d_status2, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream2));
  FETI_CK(cudaStreamSynchronize(ctx->stream2));
  for (void*& q : ctx->coarse_ws)
    if (q) { cudaFree(q); q = nullptr; }
  if (h == feti::DEV_LOCAL_SINGULAR) return fail(ctx, FETI_ERR_KERNEL_DETECT, "coarse factorization: G^T G not positive definite");
  if (h != 0) return fail(ctx, FETI_ERR_CUDA, "coarse factorization: device status " + std::to_string(h));
  return FETI_OK;
}

// c = (G^T G)^-1 g (one vector): dense inverse or sparse sweeps.
void coarse_apply_g(feti_ctx* ctx, const double* g, double* c, const int* done) {
  if (ctx->coarse_sparse)
    feti::launch_coarse_solve(ctx->cdag, 1, g, nullptr, ctx->d_sub_chunk_ptr, ctx->d_col_sub, ctx->d_lay, c, done,
                              ctx->d_coarse_err, ctx->d_spin, ctx->stream);
  else
    feti::launch_coarse_apply((int)ctx->cd, ctx->d_Ginv, g, c, done, ctx->stream);
}

// d_c = (G^T G)^-1 G^T x from the chunk partials in d_gpart.
void coarse_apply_part(feti_ctx* ctx, const int* done) {
  if (ctx->coarse_sparse)
    feti::launch_coarse_solve(ctx->cdag, 1, nullptr, ctx->d_gpart, ctx->d_sub_chunk_ptr, ctx->d_col_sub, ctx->d_lay,
                              ctx->d_c, done, ctx->d_coarse_err, ctx->d_spin, ctx->stream);
  else
    feti::launch_coarse_apply_part((int)ctx->cd, ctx->d_Ginv, ctx->d_gpart, ctx->d_sub_chunk_ptr, ctx->d_col_sub,
                                   ctx->d_lay, ctx->d_c, done, ctx->stream);
}

// P v -> out (with optional partial dot with a, or the squared norm, into
// partial, by default d_partial)
void project(feti_ctx* ctx, const double* v, double* out, const double* a, bool with_dot, const int* done,
             double* partial = nullptr) {
  cudaStream_t st = ctx->stream;
  if (!partial) partial = ctx->d_partial;
  if (ctx->cd == 0) {
    // no coarse space: out = v (the expand kernel with c unused)
    feti::launch_expand(ctx->maps, ctx->d_lay, ctx->d_R, v, ctx->d_c, out, a, partial, with_dot, done, st);
    return;
  }
  feti::launch_gtv_part(ctx->n_chunks, ctx->d_chunk_sub, ctx->d_chunk_p0, ctx->d_lay, ctx->d_R, ctx->maps, v,
                        ctx->d_gpart, done, st);
  coarse_apply_part(ctx, done);
  feti::launch_expand(ctx->maps, ctx->d_lay, ctx->d_R, v, ctx->d_c, out, a, partial, with_dot, done, st);
}

// Dense local apply of F_i (which 0) or the preconditioner block (which 1)
// on the gathered local vector (d_vloc / d_vloc32) into d_loc: one batched
// launch over all subdomains, or, in the plain form, the same kernel and
// schedule launched once per subdomain.
void gemv_apply(feti_ctx* ctx, int which, const int* done, bool f32, const void* vin, double* yout) {
  const feti::GemvCfg& cfg = f32 ? ctx->cfg32[which] : ctx->cfg64[which];
  const void* M = f32 ? (which == 0 ? (const void*)ctx->d_F32 : (const void*)ctx->d_S32)
                      : (which == 0 ? (const void*)ctx->d_F : (const void*)ctx->d_S);
  const void* v = vin ? vin : f32 ? (const void*)ctx->d_vloc32 : (const void*)ctx->d_vloc;
  const float* v32 = static_cast<const float*>(v);
  double* yo = yout ? yout : ctx->d_loc;
  if (f32 && ctx->sym32[which] == 64 && !ctx->opt.per_subdomain) {
    feti::launch_symv2_f32(ctx->sym_n[which], ctx->d_sym_sub[which], ctx->d_sym_panel[which], ctx->d_lay, which,
                           which == 0 ? ctx->d_F32s : ctx->d_S32s, v32, yo, ctx->d_symp, ctx->maps,
                           done, ctx->d_sym_err, ctx->d_spin, ctx->stream);
    return;
  }
  if (f32 && ctx->sym32[which] >= 300 && !ctx->opt.per_subdomain) {
    feti::launch_symv3_f32(ctx->sym32[which] - 300, ctx->P, ctx->d_sym_order[which], ctx->sym_max_m[which],
                           ctx->d_lay, which, which == 0 ? ctx->d_F32s : ctx->d_S32s, v32, yo,
                           done, ctx->stream);
    return;
  }
  if (f32 && ctx->sym32[which] && !ctx->opt.per_subdomain) {
    feti::launch_symv_f32(ctx->sym32[which], ctx->sym_n[which], ctx->d_sym_sub[which], ctx->d_sym_panel[which],
                          ctx->d_lay, which, which == 0 ? ctx->d_F32s : ctx->d_S32s, v32, yo,
                          ctx->d_symp, ctx->maps, done, ctx->stream);
    return;
  }
  if (!ctx->opt.per_subdomain) {
    feti::launch_gemv_loc(cfg, ctx->d_lay, which, M, f32, v, yo, ctx->max_nb, done, ctx->stream);
    return;
  }
  int t = 0;
  while (t < 2 && ctx->tab[which][t].rpc != cfg.rpc) ++t;
  const std::vector<int32_t>& ptr = ctx->tab_ptr[which][t];
  for (size_t s = 0; s + 1 < ptr.size(); ++s) {
    feti::GemvCfg c = cfg;
    c.n_blocks = ptr[s + 1] - ptr[s];
    c.blk_sub = cfg.blk_sub + ptr[s];
    c.blk_row0 = cfg.blk_row0 + ptr[s];
    if (c.n_blocks > 0) feti::launch_gemv_loc(c, ctx->d_lay, which, M, f32, v, yo, ctx->max_nb, done, ctx->stream);
  }
}

// Signed gather of x (weights wv or none) and the dense local apply of F_i
// (which 0) or the preconditioner block (which 1) into d_loc.
void local_apply(feti_ctx* ctx, int which, const double* x, const double* wv, const int* done, bool f32) {
  if (which == 0 && !f32 && ctx->opt.local_form == 2) {
    // implicit: y_b = [K^+ (0 ; B^T x)]_b by the triangular sweeps of the factor
    feti::launch_gather(ctx->maps, x, wv, ctx->d_vloc, done, ctx->stream);
    feti::launch_place(ctx->P, ctx->d_lay, ctx->d_vloc, ctx->d_ix, ctx->stream, done);
    feti::launch_kplus(ctx->P, ctx->d_lay, ctx->d_A, ctx->d_ix, ctx->d_ix2, ctx->stream, done);
    feti::launch_take_boundary(ctx->P, ctx->d_lay, ctx->d_ix2, ctx->d_loc, ctx->stream, done);
    return;
  }
  if (f32)
    feti::launch_gather32(ctx->maps, x, wv, ctx->d_vloc32, done, ctx->stream);
  else
    feti::launch_gather(ctx->maps, x, wv, ctx->d_vloc, done, ctx->stream);
  gemv_apply(ctx, which, done, f32);
}

// q = F x: signed gather B_i^T x, dense F_i apply, row-major gather back;
// optional partial dot with a.  f32 selects the FP32 copies of F_i.
void apply_F(feti_ctx* ctx, const double* x, double* q, const double* a, bool with_dot, const int* done,
             bool f32 = false) {
  if (!f32 && f32_factor(ctx)) {
    // FP64-accurate F x without FP64 explicit operators: B K^+ B^T x with the
    // refined K^+ on full local vectors (boundary values placed, interior zero)
    feti::launch_gather(ctx->maps, x, nullptr, ctx->d_loc, done, ctx->stream);
    feti::launch_place(ctx->P, ctx->d_lay, ctx->d_loc, ctx->d_kg, ctx->stream);
    kplus(ctx, ctx->d_kg, ctx->d_x2);
    feti::launch_take_boundary(ctx->P, ctx->d_lay, ctx->d_x2, ctx->d_loc, ctx->stream);
    feti::launch_scatter(ctx->maps, ctx->d_loc, nullptr, q, a, with_dot ? ctx->d_partial : nullptr, done,
                         ctx->stream);
    return;
  }
  local_apply(ctx, 0, x, nullptr, done, f32);
  feti::launch_scatter(ctx->maps, ctx->d_loc, nullptr, q, a, with_dot ? ctx->d_partial : nullptr, done, ctx->stream);
}

// z = M^-1 w = W B Y B^T W w.
void apply_M(feti_ctx* ctx, const double* w, double* z, const int* done, bool f32 = false) {
  if (ctx->opt.precond == FETI_PREC_IDENTITY) {
    feti::launch_gather(ctx->maps, w, ctx->d_weight, ctx->d_loc, done, ctx->stream);
  } else if (ctx->opt.precond == FETI_PREC_LUMPED) {
    feti::launch_gather(ctx->maps, w, ctx->d_weight, ctx->d_vloc, done, ctx->stream);
    feti::launch_spmv_lump((int)ctx->nb_total, ctx->d_lump_ptr, ctx->d_lump_col, ctx->d_lump_val, ctx->d_vloc,
                           ctx->d_loc, done, ctx->stream);
  } else {
    local_apply(ctx, 1, w, ctx->d_weight, done, f32);
  }
  feti::launch_scatter(ctx->maps, ctx->d_loc, ctx->d_weight, z, nullptr, nullptr, done, ctx->stream);
}

// Autotuner: times every (rows per warp step, rows per CTA) schedule of the
// dense local applies on the real operators and keeps the fastest.
feti_status autotune_run(feti_ctx* ctx);

// Schedules picked by the autotuner, remembered per process for decompositions
// with the same signature (sizes of every subdomain layout, options that
// change the operators), so that a new context on the same mesh and
// partition skips the timing runs.
struct TunedPick {
  int t64[2], r64[2], t32[2], r32[2], sym[2];
};
std::mutex g_tune_mu;
std::unordered_map<uint64_t, TunedPick> g_tune_cache;

uint64_t tune_signature(const feti_ctx* ctx) {
  uint64_t h = 1469598103934665603ull;
  auto add = [&](int64_t v) {
    for (int b = 0; b < 8; ++b) {
      h ^= (uint64_t)((v >> (8 * b)) & 0xff);
      h *= 1099511628211ull;
    }
  };
  add(ctx->P);
  add(ctx->n_lambda);
  add(ctx->nb_total);
  add(ctx->opt.precision);
  add(ctx->opt.precond);
  add(ctx->opt.symmetric);
  add(ctx->opt.per_subdomain);
  add(ctx->device);
  for (const auto& L : ctx->lay) {
    add(L.n);
    add(L.nI);
    add(L.nbp);
    add(L.k);
  }
  return h;
}

int tab_index(const feti_ctx* ctx, int w, const feti::GemvCfg& c) {
  for (int t = 0; t < 3; ++t)
    if (ctx->tab[w][t].blk_sub == c.blk_sub) return t;
  return 0;
}

feti_status autotune(feti_ctx* ctx) {
  const uint64_t sig = tune_signature(ctx);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune_cache.find(sig);
    if (it != g_tune_cache.end()) {
      const TunedPick& tp = it->second;
      for (int w = 0; w < 2; ++w) {
        ctx->cfg64[w] = ctx->tab[w][tp.t64[w]];
        ctx->cfg64[w].R = tp.r64[w];
        ctx->cfg32[w] = ctx->tab[w][tp.t32[w]];
        ctx->cfg32[w].R = tp.r32[w];
        ctx->sym32[w] = tp.sym[w];
      }
      ctx->tuned = true;
      return FETI_OK;
    }
  }
  FETI_TRY(autotune_run(ctx));
  TunedPick tp{};
  for (int w = 0; w < 2; ++w) {
    tp.t64[w] = tab_index(ctx, w, ctx->cfg64[w]);
    tp.r64[w] = ctx->cfg64[w].R;
    tp.t32[w] = tab_index(ctx, w, ctx->cfg32[w]);
    tp.r32[w] = ctx->cfg32[w].R;
    tp.sym[w] = ctx->sym32[w];
  }
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune_cache[sig] = tp;
  return FETI_OK;
}

feti_status autotune_run(feti_ctx* ctx) {
  cudaStream_t st = ctx->stream;
  cudaEvent_t e0, e1;
  FETI_CK(cudaEventCreate(&e0));
  FETI_CK(cudaEventCreate(&e1));
  const int Rs[3] = {2, 4, 8};
  const bool mixed = f32_ops(ctx);
  FETI_CK(cudaMemsetAsync(ctx->d_vloc, 0, ctx->nb_total * sizeof(double), st));
  FETI_CK(cudaMemsetAsync(ctx->d_vloc32, 0, ctx->nb_total * sizeof(float), st));
  for (int prec = fp64_ops(ctx) ? 0 : 1; prec < (mixed ? 2 : 1); ++prec) {
    const bool f32 = prec == 1;
    for (int w = 0; w < 2; ++w) {
      if (w == 1 && ctx->opt.precond != FETI_PREC_DIRICHLET) continue;
      const void* M = f32 ? (w == 0 ? (const void*)ctx->d_F32 : (const void*)ctx->d_S32)
                          : (w == 0 ? (const void*)ctx->d_F : (const void*)ctx->d_S);
      const void* v = f32 ? (const void*)ctx->d_vloc32 : (const void*)ctx->d_vloc;
      float best = 1e30f;
      feti::GemvCfg bestc = f32 ? ctx->cfg32[w] : ctx->cfg64[w];
      for (int t = 0; t < 3; ++t)
        for (int ri = 0; ri < 3; ++ri) {
          feti::GemvCfg c = ctx->tab[w][t];
          c.R = Rs[ri];
          feti::launch_gemv_loc(c, ctx->d_lay, w, M, f32, v, ctx->d_loc, ctx->max_nb, ctx->d_zero, st);
          FETI_CK(cudaEventRecord(e0, st));
          for (int rep = 0; rep < 3; ++rep)
            feti::launch_gemv_loc(c, ctx->d_lay, w, M, f32, v, ctx->d_loc, ctx->max_nb, ctx->d_zero, st);
          FETI_CK(cudaEventRecord(e1, st));
          FETI_CK(cudaEventSynchronize(e1));
          float ms = 0.f;
          FETI_CK(cudaEventElapsedTime(&ms, e0, e1));
          if (ms < best) { best = ms; bestc = c; }
        }
      (f32 ? ctx->cfg32[w] : ctx->cfg64[w]) = bestc;
      if (f32 && ctx->d_F32s && !ctx->opt.per_subdomain) {  // the plain form launches full rows
        // symmetric lower block-triangle kernel: load groups of 8 / 16 / 32 rows,
        // + 100 x (tiles of L2 prefetch ahead)
        ctx->sym32[w] = 0;
        const int Gs[6] = {8, 16, 32, 108, 132, 232};
        const float* Ms = w == 0 ? ctx->d_F32s : ctx->d_S32s;
        float best_sym = 1e30f;
        int gbest = 8;
        for (int gi = 0; gi < 6; ++gi) {
          feti::launch_symv_f32(Gs[gi], ctx->sym_n[w], ctx->d_sym_sub[w], ctx->d_sym_panel[w], ctx->d_lay, w, Ms,
                                ctx->d_vloc32, ctx->d_loc, ctx->d_symp, ctx->maps, ctx->d_zero, st);
          FETI_CK(cudaEventRecord(e0, st));
          for (int rep = 0; rep < 3; ++rep)
            feti::launch_symv_f32(Gs[gi], ctx->sym_n[w], ctx->d_sym_sub[w], ctx->d_sym_panel[w], ctx->d_lay, w, Ms,
                                  ctx->d_vloc32, ctx->d_loc, ctx->d_symp, ctx->maps, ctx->d_zero, st);
          FETI_CK(cudaEventRecord(e1, st));
          FETI_CK(cudaEventSynchronize(e1));
          float ms = 0.f;
          FETI_CK(cudaEventElapsedTime(&ms, e0, e1));
          if (ms < best_sym) {
            best_sym = ms;
            gbest = Gs[gi];
          }
        }
        for (int g3 : {8, 16, 32}) {  // subdomain-per-CTA variant (no second pass)
          feti::launch_symv3_f32(g3, ctx->P, ctx->d_sym_order[w], ctx->sym_max_m[w], ctx->d_lay, w, Ms,
                                 ctx->d_vloc32, ctx->d_loc, ctx->d_zero, st);
          FETI_CK(cudaEventRecord(e0, st));
          for (int rep = 0; rep < 3; ++rep)
            feti::launch_symv3_f32(g3, ctx->P, ctx->d_sym_order[w], ctx->sym_max_m[w], ctx->d_lay, w, Ms,
                                   ctx->d_vloc32, ctx->d_loc, ctx->d_zero, st);
          FETI_CK(cudaEventRecord(e1, st));
          FETI_CK(cudaEventSynchronize(e1));
          float ms = 0.f;
          FETI_CK(cudaEventElapsedTime(&ms, e0, e1));
          if (ms < best_sym) {
            best_sym = ms;
            gbest = 300 + g3;
          }
        }
        {  // streamed variant (shared-memory ring), kept only if no bounded wait ran out
          FETI_CK(cudaMemsetAsync(ctx->d_sym_err, 0, sizeof(int), st));
          feti::launch_symv2_f32(ctx->sym_n[w], ctx->d_sym_sub[w], ctx->d_sym_panel[w], ctx->d_lay, w, Ms,
                                 ctx->d_vloc32, ctx->d_loc, ctx->d_symp, ctx->maps, ctx->d_zero, ctx->d_sym_err,
                                 ctx->d_spin, st);
          FETI_CK(cudaEventRecord(e0, st));
          for (int rep = 0; rep < 3; ++rep)
            feti::launch_symv2_f32(ctx->sym_n[w], ctx->d_sym_sub[w], ctx->d_sym_panel[w], ctx->d_lay, w, Ms,
                                   ctx->d_vloc32, ctx->d_loc, ctx->d_symp, ctx->maps, ctx->d_zero, ctx->d_sym_err,
                                   ctx->d_spin, st);
          FETI_CK(cudaEventRecord(e1, st));
          FETI_CK(cudaEventSynchronize(e1));
          float ms = 0.f;
          FETI_CK(cudaEventElapsedTime(&ms, e0, e1));
          int herr = 0;
          FETI_CK(cudaMemcpy(&herr, ctx->d_sym_err, sizeof(int), cudaMemcpyDeviceToHost));
          if (herr == 0 && ms < best_sym && ctx->opt.symmetric != 3) {
            best_sym = ms;
            gbest = 64;
          }
          FETI_CK(cudaMemsetAsync(ctx->d_sym_err, 0, sizeof(int), st));
        }
        if (ctx->opt.symmetric == 3) gbest = 64;
        if (ctx->opt.symmetric == 4 && gbest < 300) {  // fastest subdomain-per-CTA load group
          float b3 = 1e30f;
          for (int g3 : {8, 16, 32}) {
            FETI_CK(cudaEventRecord(e0, st));
            feti::launch_symv3_f32(g3, ctx->P, ctx->d_sym_order[w], ctx->sym_max_m[w], ctx->d_lay, w, Ms,
                                   ctx->d_vloc32, ctx->d_loc, ctx->d_zero, st);
            FETI_CK(cudaEventRecord(e1, st));
            FETI_CK(cudaEventSynchronize(e1));
            float ms = 0.f;
            FETI_CK(cudaEventElapsedTime(&ms, e0, e1));
            if (ms < b3) {
              b3 = ms;
              gbest = 300 + g3;
            }
          }
        }
        if (best_sym < best || ctx->opt.symmetric >= 2) ctx->sym32[w] = gbest;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  FETI_CK(cudaGetLastError());
  ctx->tuned = true;
  return FETI_OK;
}

// One projected PCG iteration, 14 launches:
//   z = M^-1 w (gather, local apply, scatter); y = P z with (w, y) partials
//   (G^T z, coarse apply, expand); rho, beta and p = y + beta p in one kernel;
//   q = F p with (p, q) partials; alpha, r -= alpha q, lam += alpha p fused
//   into w = P r (G^T r, coarse apply, expand) with ||w||^2 partials;
//   stopping test.  Separate partial buffers keep readers and writers of one
//   launch apart.
void pcg_iteration(feti_ctx* ctx, double* lam, bool f32) {
  cudaStream_t st = ctx->stream;
  const int* done = &ctx->d_sc->done;
  const int nl = (int)ctx->n_lambda;
  apply_M(ctx, ctx->d_w, ctx->d_z, done, f32);                                   // z = M^-1 w
  project(ctx, ctx->d_z, ctx->d_y, ctx->d_w, true, done, ctx->d_partial_wy);      // y = P z
  feti::launch_axpby_rho(nl, ctx->d_p, ctx->d_y, ctx->d_sc, ctx->d_partial_wy, ctx->d_beta_hist, st);
  local_apply(ctx, 0, ctx->d_p, nullptr, done, f32);                              // q = F p, (p, q)
  feti::launch_scatter(ctx->maps, ctx->d_loc, nullptr, ctx->d_q, ctx->d_p, ctx->d_partial_pq, done, st);
  if (ctx->cd > 0) {
    feti::launch_gtv_part(ctx->n_chunks, ctx->d_chunk_sub, ctx->d_chunk_p0, ctx->d_lay, ctx->d_R, ctx->maps,
                          ctx->d_r, ctx->d_gpart, done, st, ctx->d_q, ctx->d_partial_pq, ctx->d_sc,
                          ctx->d_alpha_hist);
    coarse_apply_part(ctx, done);
  }
  feti::launch_expand_update(ctx->maps, ctx->d_lay, ctx->d_R, ctx->d_r, ctx->d_c, ctx->d_w, ctx->d_partial, lam,
                             ctx->d_p, ctx->d_q, ctx->d_partial_pq, ctx->d_sc, ctx->d_alpha_hist, st);
  feti::launch_ctl_conv(ctx->d_sc, ctx->d_partial, 0, st);
}

feti_status build_pcg_graph(feti_ctx* ctx, int chunk, bool mixed) {
  if (ctx->pcg_graph && ctx->pcg_graph_chunk == chunk && ctx->pcg_graph_mixed == mixed) return FETI_OK;
  if (ctx->pcg_graph) {
    cudaGraphExecDestroy(ctx->pcg_graph);
    ctx->pcg_graph = nullptr;
  }
  cudaGraph_t g = nullptr;
  FETI_CK(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
  for (int i = 0; i < chunk; ++i) pcg_iteration(ctx, mixed ? ctx->d_dl : ctx->d_lam, mixed);
  cudaError_t e = cudaStreamEndCapture(ctx->stream, &g);
  if (e != cudaSuccess) return fail(ctx, FETI_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
  e = cudaGraphInstantiate(&ctx->pcg_graph, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return fail(ctx, FETI_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
  ctx->pcg_graph_chunk = chunk;
  ctx->pcg_graph_mixed = mixed;
  return FETI_OK;
}

// Dense local matrices (factorized in place), S_i, F_i and their FP32 copies.
feti_status alloc_operators(feti_ctx* ctx) {
  if (ctx->d_A || ctx->d_A32) return FETI_OK;
  if (f32_factor(ctx)) {
    FETI_TRY(dev_alloc(ctx, &ctx->d_A32, (size_t)ctx->op_elems[0]));
    FETI_TRY(dev_alloc(ctx, &ctx->d_kr, (size_t)ctx->nloc_total));
    FETI_TRY(dev_alloc(ctx, &ctx->d_kg, (size_t)ctx->nloc_total));
    FETI_TRY(dev_alloc(ctx, &ctx->d_knorm, 2 * (size_t)ctx->P));
    FETI_TRY(dev_alloc(ctx, &ctx->d_kyI, (size_t)ctx->nloc_total));
    FETI_TRY(dev_alloc(ctx, &ctx->d_kzb, (size_t)ctx->nb_total));
    FETI_TRY(dev_alloc(ctx, &ctx->d_kxb, (size_t)ctx->nb_total));
    FETI_TRY(dev_alloc(ctx, &ctx->d_kye, (size_t)ctx->nde * ctx->E));
    FETI_TRY(dev_alloc(ctx, &ctx->d_Lc32, (size_t)ctx->lc_elems));
  } else {
    FETI_TRY(dev_alloc(ctx, &ctx->d_A, (size_t)ctx->op_elems[0]));
    FETI_TRY(dev_alloc(ctx, &ctx->d_S, (size_t)ctx->op_elems[1]));
    FETI_TRY(dev_alloc(ctx, &ctx->d_F, (size_t)ctx->op_elems[2]));
    if (!ctx->keep_factor) {
      FETI_TRY(dev_alloc(ctx, &ctx->d_Lc, (size_t)ctx->lc_elems));
      FETI_TRY(dev_alloc(ctx, &ctx->d_kyI64, (size_t)ctx->nloc_total));
      FETI_TRY(dev_alloc(ctx, &ctx->d_kzb64, (size_t)ctx->nb_total));
      FETI_TRY(dev_alloc(ctx, &ctx->d_kxb, (size_t)ctx->nb_total));
    }
  }
  if (f32_ops(ctx)) {
    FETI_TRY(dev_alloc(ctx, &ctx->d_F32, (size_t)ctx->op_elems[3]));
    FETI_TRY(dev_alloc(ctx, &ctx->d_S32, (size_t)ctx->op_elems[4]));
    if (ctx->opt.symmetric != 1) {
      FETI_TRY(dev_alloc(ctx, &ctx->d_F32s, (size_t)ctx->op_elems[5]));
      FETI_TRY(dev_alloc(ctx, &ctx->d_S32s, (size_t)ctx->op_elems[6]));
      FETI_TRY(dev_alloc(ctx, &ctx->d_symp, (size_t)ctx->op_elems[7] + 4));
      FETI_TRY(dev_alloc(ctx, &ctx->d_sym_err, 1));
      FETI_CK(cudaMemsetAsync(ctx->d_sym_err, 0, sizeof(int), ctx->stream));
    }
  }
  if (ctx->opt.local_form == 2) {
    FETI_TRY(dev_alloc(ctx, &ctx->d_ix, (size_t)ctx->nloc_total));
    FETI_TRY(dev_alloc(ctx, &ctx->d_ix2, (size_t)ctx->nloc_total));
  }
  return FETI_OK;
}

// Setup: element matrices through the coarse inverse.
feti_status prepare(feti_ctx* ctx, const double* dU, double tau) {
  StageLog lg(ctx);
  FETI_TRY(alloc_operators(ctx));
  lg.mark("setup: allocation");
  FETI_TRY(assemble_all(ctx, dU, tau));
  lg.mark("setup: elements + assembly");
  if (!ctx->prepared) FETI_TRY(coarse_begin(ctx));
  feti_status fs = factorize_all(ctx);
  lg.mark("setup: local factorization");
  const feti_status cs = coarse_join(ctx);
  FETI_TRY(fs);
  FETI_TRY(cs);
  lg.mark("setup: coarse problem (joined)");
  if (!ctx->tuned) FETI_TRY(autotune(ctx));
  lg.mark("setup: autotuning");
  // the refinement count of the FP32-factor K^+ (its corrections apply the
  // tuned F_i kernel)
  if (f32_factor(ctx) && ctx->refine_steps == 0) {
    FETI_TRY(tune_refinement(ctx));
    lg.mark("setup: refinement count");
  }
  ctx->prepared = true;
  return FETI_OK;
}

// Runs graph chunks of the PCG recurrence (scalars already initialised and the
// first projected residual computed) until the device reports done.
feti_status run_pcg_chunks(feti_ctx* ctx, bool mixed, int maxit) {
  const int chunk = ctx->opt.chunk > 0 ? ctx->opt.chunk : 16;
  FETI_TRY(build_pcg_graph(ctx, chunk, mixed));
  const int max_launch = maxit / chunk + 2;
  for (int l = 0; l < max_launch; ++l) {
    FETI_CK(cudaGraphLaunch(ctx->pcg_graph, ctx->stream));
    FETI_CK(cudaMemcpyAsync(ctx->h_sc, ctx->d_sc, sizeof(feti::PcgScalars), cudaMemcpyDeviceToHost, ctx->stream));
    FETI_CK(cudaStreamSynchronize(ctx->stream));
    if (ctx->h_sc->done) break;
  }
  return FETI_OK;
}

// Resets the scalar block, projects r into w and evaluates ||w|| (as wnorm0).
feti_status start_pcg(feti_ctx* ctx, double tol, int maxit) {
  feti::PcgScalars h{};
  h.tol = tol;
  h.maxit = maxit;
  FETI_CK(cudaMemcpyAsync(ctx->d_sc, &h, sizeof(h), cudaMemcpyHostToDevice, ctx->stream));
  FETI_CK(cudaMemsetAsync(ctx->d_p, 0, ctx->n_lambda * sizeof(double), ctx->stream));
  project(ctx, ctx->d_r, ctx->d_w, nullptr, true, &ctx->d_sc->done);
  feti::launch_ctl_conv(ctx->d_sc, ctx->d_partial, 1, ctx->stream);
  FETI_CK(cudaGetLastError());
  FETI_CK(cudaMemcpyAsync(ctx->h_sc, ctx->d_sc, sizeof(feti::PcgScalars), cudaMemcpyDeviceToHost, ctx->stream));
  FETI_CK(cudaStreamSynchronize(ctx->stream));
  return FETI_OK;
}

// Right-hand sides, projected PCG, recovery.  Leaves the local solutions in d_x.
//
// FP64 form: one PCG on P F P with the FP64 operators.
// Mixed form: iterative refinement on the dual problem -- the true projected
// residual r = P(d~ - F lambda) is evaluated with the FP64 operators, the
// correction P F P delta = r is solved by PCG with the FP32 copies of F_i and
// S_i (vectors, dots, projection and coarse solve stay FP64) to a relative
// tolerance inner_tol, and lambda += delta, until ||r|| <= tol ||r_0||.
// d~ = sum B K^+ f - b into d_d and lambda_0 = G (G^T G)^-1 e into d_lam.
feti_status rhs_setup(feti_ctx* ctx) {
  cudaStream_t st = ctx->stream;
  const int nl = (int)ctx->n_lambda;
  const int* zero = ctx->d_zero;
  kplus(ctx, ctx->d_f, ctx->d_x);
  feti::launch_take_boundary(ctx->P, ctx->d_lay, ctx->d_x, ctx->d_loc, st);
  feti::launch_scatter(ctx->maps, ctx->d_loc, nullptr, ctx->d_q, nullptr, nullptr, zero, st);
  feti::launch_vsub(nl, ctx->d_q, ctx->d_b, ctx->d_d, st);
  // e = R^T f, lambda_0 = G (G^T G)^-1 e
  FETI_CK(cudaMemsetAsync(ctx->d_lam, 0, nl * sizeof(double), st));
  if (ctx->cd > 0) {
    feti::launch_rtx(ctx->P, ctx->d_lay, ctx->d_R, ctx->d_f, -1.0, ctx->d_e, st);
    coarse_apply_g(ctx, ctx->d_e, ctx->d_c, zero);
    feti::launch_expand(ctx->maps, ctx->d_lay, ctx->d_R, ctx->d_lam, ctx->d_c, ctx->d_lam, nullptr, nullptr, 0,
                        zero, st);
  }
  FETI_CK(cudaGetLastError());
  return FETI_OK;
}

feti_status dual_solve(feti_ctx* ctx, feti_report* rep, float* pcg_ms) {
  cudaStream_t st = ctx->stream;
  const int nl = (int)ctx->n_lambda;
  const int* zero = ctx->d_zero;
  const bool mixed = f32_ops(ctx);
  FETI_TRY(rhs_setup(ctx));
  cudaEvent_t e0, e1;
  FETI_CK(cudaEventCreate(&e0));
  FETI_CK(cudaEventCreate(&e1));
  FETI_CK(cudaEventRecord(e0, st));
  int total_it = 0, outer = 0, last_it = 0;
  bool conv = false, breakdown = false;
  double nrm0 = -1.0, nrm = 0.0;
  if (!mixed) {
    apply_F(ctx, ctx->d_lam, ctx->d_q, nullptr, false, zero);       // r0 = d~ - F lambda_0
    feti::launch_vsub(nl, ctx->d_d, ctx->d_q, ctx->d_r, st);
    FETI_TRY(start_pcg(ctx, ctx->opt.tol, ctx->opt.maxit));
    nrm0 = ctx->h_sc->wnorm0;
    if (!ctx->h_sc->done) FETI_TRY(run_pcg_chunks(ctx, false, ctx->opt.maxit));
    const feti::PcgScalars& sc = *ctx->h_sc;
    total_it = last_it = sc.it;
    breakdown = sc.status == feti::DEV_BREAKDOWN;
    nrm = sc.wnorm;
    conv = !breakdown && (sc.wnorm <= sc.tol * sc.wnorm0 || sc.wnorm0 == 0.0);
  } else {
    const double inner_tol = ctx->opt.inner_tol > 0.0 ? ctx->opt.inner_tol : 1e-4;
    const int max_outer = ctx->opt.max_outer > 0 ? ctx->opt.max_outer : 20;
    for (;;) {
      apply_F(ctx, ctx->d_lam, ctx->d_q, nullptr, false, zero);     // FP64 residual
      feti::launch_vsub(nl, ctx->d_d, ctx->d_q, ctx->d_r, st);
      FETI_TRY(start_pcg(ctx, inner_tol, std::max(1, ctx->opt.maxit - total_it)));
      nrm = ctx->h_sc->wnorm0;
      if (nrm0 < 0.0) nrm0 = nrm;
      if (!std::isfinite(nrm)) { breakdown = true; break; }
      if (nrm <= ctx->opt.tol * nrm0 || nrm == 0.0) { conv = true; break; }
      if (outer >= max_outer || total_it >= ctx->opt.maxit) break;
      // inner tolerance: no tighter than needed to reach tol on this pass
      const double tin = std::max(inner_tol, 0.5 * ctx->opt.tol * nrm0 / nrm);
      FETI_CK(cudaMemcpyAsync(&ctx->d_sc->tol, &tin, sizeof(double), cudaMemcpyHostToDevice, st));
      FETI_CK(cudaMemsetAsync(ctx->d_dl, 0, nl * sizeof(double), st));
      FETI_TRY(run_pcg_chunks(ctx, true, ctx->opt.maxit - total_it));
      const feti::PcgScalars& sc = *ctx->h_sc;
      total_it += sc.it;
      last_it = sc.it;
      if (sc.status == feti::DEV_BREAKDOWN) { breakdown = true; break; }
      feti::launch_vadd(nl, ctx->d_lam, ctx->d_dl, st);
      ++outer;
    }
  }
  FETI_CK(cudaEventRecord(e1, st));
  FETI_CK(cudaEventSynchronize(e1));
  float ms = 0.f;
  FETI_CK(cudaEventElapsedTime(&ms, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (pcg_ms) *pcg_ms = ms;
  // Lanczos estimate from the last CG recurrence
  double cond = 1.0;
  if (last_it > 0) {
    std::vector<double> al(last_it), be(last_it);
    FETI_CK(cudaMemcpy(al.data(), ctx->d_alpha_hist, last_it * sizeof(double), cudaMemcpyDeviceToHost));
    FETI_CK(cudaMemcpy(be.data(), ctx->d_beta_hist, last_it * sizeof(double), cudaMemcpyDeviceToHost));
    cond = lanczos_cond(al, be);
  }
  if (rep) {
    rep->iterations = total_it;
    rep->outer_iterations = outer;
    rep->rel_residual = nrm0 > 0 ? nrm / nrm0 : 0.0;
    rep->converged = conv ? 1 : 0;
    rep->cond_est = cond;
    rep->t_pcg_ms = ms;
    rep->n_lambda = ctx->n_lambda;
    rep->coarse_dim = ctx->cd;
  }
  FETI_TRY(check_wait_flag(ctx, ctx->d_sym_err, "streamed symmetric local apply"));
  FETI_TRY(check_wait_flag(ctx, ctx->d_coarse_err, "sparse coarse solve"));
  if (breakdown) return fail(ctx, FETI_ERR_BREAKDOWN, "PCG breakdown");
  // recovery: gamma = (G^T G)^-1 G^T (F lambda - d~), u_i = K^+(f_i - B_i^T lambda) + R_i gamma_i
  apply_F(ctx, ctx->d_lam, ctx->d_q, nullptr, false, zero);
  feti::launch_vsub(nl, ctx->d_q, ctx->d_d, ctx->d_z, st);
  if (ctx->cd > 0) {
    feti::launch_gtv(ctx->P, ctx->d_lay, ctx->d_R, ctx->maps, ctx->d_z, ctx->d_g, zero, st);
    coarse_apply_g(ctx, ctx->d_g, ctx->d_c, zero);
  }
  feti::launch_gather(ctx->maps, ctx->d_lam, nullptr, ctx->d_loc, zero, st);
  feti::launch_local_sub(ctx->P, ctx->d_lay, ctx->d_f, ctx->d_loc, ctx->d_x2, st);
  kplus(ctx, ctx->d_x2, ctx->d_x);
  if (ctx->cd > 0) feti::launch_add_kernel(ctx->P, ctx->d_lay, ctx->d_R, ctx->d_c, ctx->d_x, st);
  FETI_CK(cudaGetLastError());
  FETI_TRY(check_wait_flag(ctx, ctx->d_sym_err, "streamed symmetric local apply"));
  FETI_TRY(check_wait_flag(ctx, ctx->d_coarse_err, "sparse coarse solve"));
  if (!conv) return fail(ctx, FETI_ERR_NOT_CONVERGED, "PCG reached maxit");
  return FETI_OK;
}

feti_status write_displacement(feti_ctx* ctx, double* u_out, int on_device, double* d_target);

// ---------------------------------------------------------------------------
// Block form: nrhs right-hand sides share every operator apply.
// Times the block-form local GEMM schedules (rows per warp step {1, 2, 4},
// rows per CTA {32, 64}) on the real operators and keeps the fastest.
// One 2-D tensor map per subdomain over its FP32 copy of F_i (which 0) or of
// the preconditioner block (which 1): (columns, rows) = (m, m), row pitch the
// padded stride, 32 x 128 boxes, 128-byte swizzle, out-of-range elements
// zero-filled.  Encoded through the runtime's driver entry point.
feti_status build_tensor_maps(feti_ctx* ctx) {
  if (ctx->d_tmap[0]) return FETI_OK;
  void* fn = nullptr;
  cudaDriverEntryPointQueryResult q{};
  FETI_CK(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q));
  if (!fn || q != cudaDriverEntryPointSuccess) return fail(ctx, FETI_ERR_CUDA, "cuTensorMapEncodeTiled unavailable");
  auto encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  for (int w = 0; w < 2; ++w) {
    if (w == 1 && ctx->opt.precond != FETI_PREC_DIRICHLET) break;  // no dense preconditioner block
    std::vector<CUtensorMap> maps(ctx->P);
    const float* base = w == 0 ? ctx->d_F32 : ctx->d_S32;
    for (int s = 0; s < ctx->P; ++s) {
      const SubLayout& L = ctx->lay[s];
      const int m = w == 0 ? std::max(L.nbp, 1) : std::max(L.nbp + L.k, 1);
      const cuuint64_t ld = (cuuint64_t)((m + 3) & ~3);
      const cuuint64_t dim[2] = {(cuuint64_t)m, (cuuint64_t)m};
      const cuuint64_t stride[1] = {ld * sizeof(float)};
      const cuuint32_t box[2] = {32, 128};
      const cuuint32_t estr[2] = {1, 1};
      void* addr = (void*)(base + (w == 0 ? L.foff32 : L.soff32));
      const CUresult r = encode(&maps[s], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, addr, dim, stride, box, estr,
                                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                                CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
      if (r != CUDA_SUCCESS)
        return fail(ctx, FETI_ERR_CUDA, "tensor map of subdomain " + std::to_string(s) + ": error " + std::to_string((int)r));
    }
    FETI_TRY(upload(ctx, &ctx->d_tmap[w], maps));
  }
  return FETI_OK;
}

feti_status autotune_m(feti_ctx* ctx, int nrhs) {
  if (ctx->tuned_m == nrhs) return FETI_OK;
  cudaStream_t st = ctx->stream;
  cudaEvent_t e0, e1;
  FETI_CK(cudaEventCreate(&e0));
  FETI_CK(cudaEventCreate(&e1));
  const bool mixed = f32_ops(ctx);
  FETI_CK(cudaMemsetAsync(ctx->dm_vloc, 0, (size_t)ctx->nb_total * nrhs * sizeof(double), st));
  FETI_CK(cudaMemsetAsync(ctx->dm_vloc32, 0, (size_t)ctx->nb_total * nrhs * sizeof(float), st));
  const int Rs[3] = {1, 2, 4};
  for (int prec = fp64_ops(ctx) ? 0 : 1; prec < (mixed ? 2 : 1); ++prec) {
    const bool f32 = prec == 1;
    for (int w = 0; w < 2; ++w) {
      feti::GemvCfg best = ctx->tab[w][0];
      best.R = 2;
      if (!(w == 1 && ctx->opt.precond != FETI_PREC_DIRICHLET)) {
        const void* M = f32 ? (w == 0 ? (const void*)ctx->d_F32 : (const void*)ctx->d_S32)
                            : (w == 0 ? (const void*)ctx->d_F : (const void*)ctx->d_S);
        const void* v = f32 ? (const void*)ctx->dm_vloc32 : (const void*)ctx->dm_vloc;
        float bt = 1e30f;
        for (int t = 0; t < 2; ++t)
          for (int ri = 0; ri < 3; ++ri) {
            if (!f32 && Rs[ri] == 4) continue;
            feti::GemvCfg c = ctx->tab[w][t];
            c.R = Rs[ri];
            feti::launch_gemm_loc(c, ctx->d_lay, w, M, f32, nrhs, v, ctx->dm_loc, ctx->max_nb, ctx->d_zero, st);
            FETI_CK(cudaEventRecord(e0, st));
            for (int rep = 0; rep < 3; ++rep)
              feti::launch_gemm_loc(c, ctx->d_lay, w, M, f32, nrhs, v, ctx->dm_loc, ctx->max_nb, ctx->d_zero, st);
            FETI_CK(cudaEventRecord(e1, st));
            FETI_CK(cudaEventSynchronize(e1));
            float ms = 0.f;
            FETI_CK(cudaEventElapsedTime(&ms, e0, e1));
            if (ms < bt) { bt = ms; best = c; }
          }
        if (f32 && ctx->opt.no_tensor_cores != 1) {
          // tensor-core candidate: kept only if faster and no bounded wait timed out
          if (!ctx->d_tc_err) FETI_TRY(dev_alloc(ctx, &ctx->d_tc_err, 1));
          FETI_CK(cudaMemsetAsync(ctx->d_tc_err, 0, sizeof(int), st));
          const float* Mf = static_cast<const float*>(M);
          const float* vf = static_cast<const float*>(v);
          float bt_tc = 1e30f;
          ctx->tc_m[w] = 0;
          const int ntc = ctx->opt.no_tensor_cores;
          FETI_TRY(build_tensor_maps(ctx));
          for (int variant = 1; variant <= 8; ++variant) {
            if (ntc >= 3 && variant != ntc - 2) continue;
            FETI_CK(cudaMemsetAsync(ctx->d_tc_err, 0, sizeof(int), st));
            feti::launch_gemm_tc(ctx->tab[w][2], ctx->d_lay, w, Mf, nrhs, vf, ctx->dm_loc, ctx->d_zero, ctx->d_tc_err,
                                 variant, ctx->d_tmap[w], ctx->d_spin, st);
            FETI_CK(cudaEventRecord(e0, st));
            for (int rep = 0; rep < 3; ++rep)
              feti::launch_gemm_tc(ctx->tab[w][2], ctx->d_lay, w, Mf, nrhs, vf, ctx->dm_loc, ctx->d_zero,
                                   ctx->d_tc_err, variant, ctx->d_tmap[w], ctx->d_spin, st);
            FETI_CK(cudaEventRecord(e1, st));
            FETI_CK(cudaEventSynchronize(e1));
            float ms = 0.f;
            FETI_CK(cudaEventElapsedTime(&ms, e0, e1));
            int herr = 0;
            FETI_CK(cudaMemcpy(&herr, ctx->d_tc_err, sizeof(int), cudaMemcpyDeviceToHost));
            if (herr == 0 && ms < bt_tc) {
              bt_tc = ms;
              if (ms < bt || ntc >= 2) ctx->tc_m[w] = variant;
            }
          }
          FETI_CK(cudaMemsetAsync(ctx->d_tc_err, 0, sizeof(int), st));
        }
      }
      (f32 ? ctx->cfgm32[w] : ctx->cfgm64[w]) = best;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  FETI_CK(cudaGetLastError());
  ctx->tuned_m = nrhs;
  return FETI_OK;
}

feti_status alloc_multi(feti_ctx* ctx, int nrhs) {
  if (ctx->m_cap >= nrhs) return autotune_m(ctx, nrhs);
  if (ctx->m_cap > 0) return fail(ctx, FETI_ERR_STATE, "block buffers were sized for fewer right-hand sides");
  const size_t nl = (size_t)ctx->n_lambda * nrhs, nb = (size_t)ctx->nb_total * nrhs;
  for (double** v : {&ctx->dm_lam, &ctx->dm_r, &ctx->dm_w, &ctx->dm_z, &ctx->dm_y, &ctx->dm_p, &ctx->dm_q, &ctx->dm_d,
                     &ctx->dm_dl})
    FETI_TRY(dev_alloc(ctx, v, nl));
  FETI_TRY(dev_alloc(ctx, &ctx->dm_loc, nb));
  FETI_TRY(dev_alloc(ctx, &ctx->dm_vloc, nb));
  FETI_TRY(dev_alloc(ctx, &ctx->dm_vloc32, nb + 4));
  const size_t np = (size_t)feti::scatter_partials() * feti::kMaxRhs;
  FETI_TRY(dev_alloc(ctx, &ctx->dm_part_wy, np));
  FETI_TRY(dev_alloc(ctx, &ctx->dm_part_pq, np));
  FETI_TRY(dev_alloc(ctx, &ctx->dm_part_ww, np));
  FETI_TRY(dev_alloc(ctx, &ctx->dm_gpart, (size_t)std::max(ctx->n_chunks, 1) * 6 * nrhs));
  FETI_TRY(dev_alloc(ctx, &ctx->dm_g, (size_t)std::max<int64_t>(ctx->cd, 1) * nrhs));
  FETI_TRY(dev_alloc(ctx, &ctx->dm_c, (size_t)std::max<int64_t>(ctx->cd, 1) * nrhs));
  FETI_TRY(dev_alloc(ctx, &ctx->dm_alpha_hist, (size_t)(ctx->opt.maxit + 2) * feti::kMaxRhs));
  FETI_TRY(dev_alloc(ctx, &ctx->dm_sc, 1));
  FETI_CK(cudaMallocHost(&ctx->hm_sc, sizeof(feti::PcgScalarsM)));
  ctx->m_cap = nrhs;
  return autotune_m(ctx, nrhs);
}

// Y = W B M B^T W X on blocks (which 0: F_i, no weights; which 1: preconditioner).
void local_apply_m(feti_ctx* ctx, int which, int nrhs, const double* x, const double* wv, const int* done, bool f32) {
  cudaStream_t st = ctx->stream;
  if (which == 1 && ctx->opt.precond == FETI_PREC_IDENTITY) {
    feti::launch_gather_m(ctx->maps, nrhs, x, wv, ctx->dm_loc, 0, done, st);
    return;
  }
  if (which == 1 && ctx->opt.precond == FETI_PREC_LUMPED) {
    feti::launch_gather_m(ctx->maps, nrhs, x, wv, ctx->dm_vloc, 0, done, st);
    feti::launch_spmv_lump_m((int)ctx->nb_total, nrhs, ctx->d_lump_ptr, ctx->d_lump_col, ctx->d_lump_val, ctx->dm_vloc,
                             ctx->dm_loc, done, st);
    return;
  }
  const feti::GemvCfg& cfg = f32 ? ctx->cfgm32[which] : ctx->cfgm64[which];
  const void* M = f32 ? (which == 0 ? (const void*)ctx->d_F32 : (const void*)ctx->d_S32)
                      : (which == 0 ? (const void*)ctx->d_F : (const void*)ctx->d_S);
  void* v = f32 ? (void*)ctx->dm_vloc32 : (void*)ctx->dm_vloc;
  feti::launch_gather_m(ctx->maps, nrhs, x, wv, v, f32 ? 1 : 0, done, st);
  if (f32 && ctx->tc_m[which])
    feti::launch_gemm_tc(ctx->tab[which][2], ctx->d_lay, which, static_cast<const float*>(M), nrhs,
                         static_cast<const float*>(v), ctx->dm_loc, done, ctx->d_tc_err, ctx->tc_m[which],
                         ctx->d_tmap[which], ctx->d_spin, st);
  else
    feti::launch_gemm_loc(cfg, ctx->d_lay, which, M, f32 ? 1 : 0, nrhs, v, ctx->dm_loc, ctx->max_nb, done, st);
}

void apply_F_m(feti_ctx* ctx, int nrhs, const double* x, double* q, const double* a, double* partial, const int* done,
               bool f32) {
  local_apply_m(ctx, 0, nrhs, x, nullptr, done, f32);
  feti::launch_scatter_m(ctx->maps, nrhs, ctx->dm_loc, nullptr, q, a, partial, done, ctx->stream);
}

void apply_M_m(feti_ctx* ctx, int nrhs, const double* w, double* z, const int* done, bool f32) {
  local_apply_m(ctx, 1, nrhs, w, ctx->d_weight, done, f32);
  feti::launch_scatter_m(ctx->maps, nrhs, ctx->dm_loc, ctx->d_weight, z, nullptr, nullptr, done, ctx->stream);
}

// out = P (v - alpha q)  (q optional: fused CG update of r and lam, see launch_expand_m)
void project_m(feti_ctx* ctx, int nrhs, const double* v, double* out, const double* a, double* partial,
               double* r_upd, double* lam, const double* p, const double* q, const int* done) {
  const bool coarse = ctx->cd > 0;
  if (coarse) {
    // dense: G^T x partials, their sums, Ginv G; sparse: G^T x partials, then the sweeps
    feti::launch_project_m(ctx->n_chunks, ctx->d_chunk_sub, ctx->d_chunk_p0, ctx->d_sub_chunk_ptr, ctx->d_col_sub,
                           ctx->d_lay, ctx->d_R, ctx->maps, nrhs, (int)ctx->cd,
                           ctx->coarse_sparse ? nullptr : ctx->d_Ginv, r_upd ? r_upd : v, r_upd ? q : nullptr,
                           ctx->dm_sc, ctx->dm_gpart, ctx->dm_g, ctx->dm_c, done, ctx->stream);
    if (ctx->coarse_sparse)
      feti::launch_coarse_solve(ctx->cdag, nrhs, nullptr, ctx->dm_gpart, ctx->d_sub_chunk_ptr, ctx->d_col_sub,
                                ctx->d_lay, ctx->dm_c, done, ctx->d_coarse_err, ctx->d_spin, ctx->stream);
  }
  feti::launch_expand_m(ctx->maps, ctx->d_lay, ctx->d_R, nrhs, coarse ? 1 : 0, v, ctx->dm_c, out, a, partial, r_upd,
                        lam, p, q, ctx->dm_sc, done, ctx->stream);
}

void pcg_iteration_m(feti_ctx* ctx, int nrhs, double* lam, bool f32) {
  cudaStream_t st = ctx->stream;
  const int* done = &ctx->dm_sc->done;
  const int nl = (int)ctx->n_lambda;
  apply_M_m(ctx, nrhs, ctx->dm_w, ctx->dm_z, done, f32);
  project_m(ctx, nrhs, ctx->dm_z, ctx->dm_y, ctx->dm_w, ctx->dm_part_wy, nullptr, nullptr, nullptr, nullptr, done);
  feti::launch_axpby_rho_m(nl, nrhs, ctx->dm_p, ctx->dm_y, ctx->dm_sc, ctx->dm_part_wy, st);
  apply_F_m(ctx, nrhs, ctx->dm_p, ctx->dm_q, ctx->dm_p, ctx->dm_part_pq, done, f32);
  feti::launch_alpha_m(nrhs, ctx->dm_sc, ctx->dm_part_pq, ctx->dm_alpha_hist, st);
  project_m(ctx, nrhs, ctx->dm_r, ctx->dm_w, nullptr, ctx->dm_part_ww, ctx->dm_r, lam, ctx->dm_p, ctx->dm_q, done);
  feti::launch_conv_m(nrhs, ctx->dm_sc, ctx->dm_part_ww, 0, st);
}

feti_status run_pcg_chunks_m(feti_ctx* ctx, int nrhs, bool mixed, int maxit) {
  const int chunk = ctx->opt.chunk > 0 ? ctx->opt.chunk : 16;
  if (!(ctx->pcgm_graph && ctx->pcgm_chunk == chunk && ctx->pcgm_nrhs == nrhs && ctx->pcgm_mixed == mixed)) {
    if (ctx->pcgm_graph) cudaGraphExecDestroy(ctx->pcgm_graph);
    ctx->pcgm_graph = nullptr;
    cudaGraph_t g = nullptr;
    FETI_CK(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
    for (int i = 0; i < chunk; ++i) pcg_iteration_m(ctx, nrhs, mixed ? ctx->dm_dl : ctx->dm_lam, mixed);
    cudaError_t e = cudaStreamEndCapture(ctx->stream, &g);
    if (e != cudaSuccess) return fail(ctx, FETI_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    e = cudaGraphInstantiate(&ctx->pcgm_graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(ctx, FETI_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    ctx->pcgm_chunk = chunk;
    ctx->pcgm_nrhs = nrhs;
    ctx->pcgm_mixed = mixed;
  }
  const int max_launch = maxit / chunk + 2;
  for (int l = 0; l < max_launch; ++l) {
    FETI_CK(cudaGraphLaunch(ctx->pcgm_graph, ctx->stream));
    FETI_CK(cudaMemcpyAsync(ctx->hm_sc, ctx->dm_sc, sizeof(feti::PcgScalarsM), cudaMemcpyDeviceToHost, ctx->stream));
    FETI_CK(cudaStreamSynchronize(ctx->stream));
    if (ctx->hm_sc->done) break;
  }
  return FETI_OK;
}

// Resets the block scalars (active[k] for k < nrhs unless frozen[k]), projects
// r into w and evaluates the per-RHS norms (wnorm0).
feti_status start_pcg_m(feti_ctx* ctx, int nrhs, const double* tol, const std::vector<int>& frozen, int maxit) {
  feti::PcgScalarsM h{};
  for (int k = 0; k < nrhs; ++k) {
    h.tol[k] = tol[k];
    h.active[k] = frozen.empty() || !frozen[k] ? 1 : 0;
  }
  h.maxit = maxit;
  FETI_CK(cudaMemcpyAsync(ctx->dm_sc, &h, sizeof(h), cudaMemcpyHostToDevice, ctx->stream));
  FETI_CK(cudaMemsetAsync(ctx->dm_p, 0, (size_t)ctx->n_lambda * nrhs * sizeof(double), ctx->stream));
  project_m(ctx, nrhs, ctx->dm_r, ctx->dm_w, nullptr, ctx->dm_part_ww, nullptr, nullptr, nullptr, nullptr,
            &ctx->dm_sc->done);
  feti::launch_conv_m(nrhs, ctx->dm_sc, ctx->dm_part_ww, 1, ctx->stream);
  FETI_CK(cudaGetLastError());
  FETI_CK(cudaMemcpyAsync(ctx->hm_sc, ctx->dm_sc, sizeof(feti::PcgScalarsM), cudaMemcpyDeviceToHost, ctx->stream));
  FETI_CK(cudaStreamSynchronize(ctx->stream));
  return FETI_OK;
}

// Block solve of nrhs load cases f_k = scale_k f (homogeneous Dirichlet data):
// right-hand sides from the single-RHS setup, scaled; one PCG (or one
// refinement loop) over the block; recovery per right-hand side.
feti_status dual_solve_multi(feti_ctx* ctx, const double* scale, int nrhs, double* u_out, int u_on_device,
                             feti_report* rep) {
  cudaStream_t st = ctx->stream;
  const int nl = (int)ctx->n_lambda;
  const int* zero = ctx->d_zero;
  const bool mixed = f32_ops(ctx);
  FETI_TRY(alloc_multi(ctx, nrhs));
  FETI_TRY(rhs_setup(ctx));
  for (int k = 0; k < nrhs; ++k) {
    feti::launch_col_set(nl, nrhs, k, scale[k], ctx->d_lam, ctx->dm_lam, st);
    feti::launch_col_set(nl, nrhs, k, scale[k], ctx->d_d, ctx->dm_d, st);
  }
  FETI_CK(cudaGetLastError());
  cudaEvent_t e0, e1;
  FETI_CK(cudaEventCreate(&e0));
  FETI_CK(cudaEventCreate(&e1));
  FETI_CK(cudaEventRecord(e0, st));
  const int nlb = nl * nrhs;
  int total_it = 0, outer = 0;
  bool conv = false, breakdown = false;
  std::vector<double> nrm0(nrhs, -1.0), tolv(nrhs, ctx->opt.tol);
  std::vector<int> frozen(nrhs, 0);
  if (!mixed) {
    apply_F_m(ctx, nrhs, ctx->dm_lam, ctx->dm_q, nullptr, nullptr, zero, false);
    feti::launch_vsub(nlb, ctx->dm_d, ctx->dm_q, ctx->dm_r, st);
    FETI_TRY(start_pcg_m(ctx, nrhs, tolv.data(), frozen, ctx->opt.maxit));
    if (!ctx->hm_sc->done) FETI_TRY(run_pcg_chunks_m(ctx, nrhs, false, ctx->opt.maxit));
    const feti::PcgScalarsM& sc = *ctx->hm_sc;
    total_it = sc.it;
    breakdown = sc.status != 0;
    conv = !breakdown;
    for (int k = 0; k < nrhs; ++k)
      if (!(sc.wnorm[k] <= sc.tol[k] * sc.wnorm0[k] || sc.wnorm0[k] == 0.0)) conv = false;
  } else {
    const double inner_tol = ctx->opt.inner_tol > 0.0 ? ctx->opt.inner_tol : 1e-4;
    const int max_outer = ctx->opt.max_outer > 0 ? ctx->opt.max_outer : 20;
    for (;;) {
      if (f32_factor(ctx)) {   // FP64 residuals by the refined K^+, one right-hand side at a time
        for (int k = 0; k < nrhs; ++k) {
          feti::launch_col_get(nl, nrhs, k, ctx->dm_lam, ctx->d_lam, st);
          apply_F(ctx, ctx->d_lam, ctx->d_q, nullptr, false, zero);
          feti::launch_col_set(nl, nrhs, k, 1.0, ctx->d_q, ctx->dm_q, st);
        }
      } else {
        apply_F_m(ctx, nrhs, ctx->dm_lam, ctx->dm_q, nullptr, nullptr, zero, false);   // FP64 residuals
      }
      feti::launch_vsub(nlb, ctx->dm_d, ctx->dm_q, ctx->dm_r, st);
      std::vector<int> none;
      FETI_TRY(start_pcg_m(ctx, nrhs, tolv.data(), none, std::max(1, ctx->opt.maxit - total_it)));
      bool all = true;
      std::vector<double> tin(nrhs);
      for (int k = 0; k < nrhs; ++k) {
        const double nr = ctx->hm_sc->wnorm0[k];
        if (nrm0[k] < 0.0) nrm0[k] = nr;
        if (!std::isfinite(nr)) breakdown = true;
        frozen[k] = (nr <= ctx->opt.tol * nrm0[k] || nr == 0.0) ? 1 : 0;
        all = all && frozen[k];
        tin[k] = nr > 0.0 ? std::max(inner_tol, 0.5 * ctx->opt.tol * nrm0[k] / nr) : inner_tol;
      }
      if (breakdown) break;
      if (all) { conv = true; break; }
      if (outer >= max_outer || total_it >= ctx->opt.maxit) break;
      // inner solve on the unconverged right-hand sides only
      feti::PcgScalarsM h = *ctx->hm_sc;
      for (int k = 0; k < nrhs; ++k) {
        h.tol[k] = tin[k];
        h.active[k] = frozen[k] ? 0 : 1;
      }
      FETI_CK(cudaMemcpyAsync(ctx->dm_sc, &h, sizeof(h), cudaMemcpyHostToDevice, st));
      FETI_CK(cudaMemsetAsync(ctx->dm_dl, 0, (size_t)nlb * sizeof(double), st));
      FETI_TRY(run_pcg_chunks_m(ctx, nrhs, true, ctx->opt.maxit - total_it));
      total_it += ctx->hm_sc->it;
      if (ctx->hm_sc->status) { breakdown = true; break; }
      feti::launch_vadd(nlb, ctx->dm_lam, ctx->dm_dl, st);
      ++outer;
    }
  }
  FETI_CK(cudaEventRecord(e1, st));
  FETI_CK(cudaEventSynchronize(e1));
  float ms = 0.f;
  FETI_CK(cudaEventElapsedTime(&ms, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rep) {
    rep->iterations = total_it;
    rep->outer_iterations = outer;
    rep->converged = conv ? 1 : 0;
    rep->t_pcg_ms = ms;
    rep->n_lambda = ctx->n_lambda;
    rep->coarse_dim = ctx->cd;
  }
  FETI_TRY(check_wait_flag(ctx, ctx->d_tc_err, "tensor-core block GEMM"));
  FETI_TRY(check_wait_flag(ctx, ctx->d_coarse_err, "sparse coarse solve"));
  if (breakdown) return fail(ctx, FETI_ERR_BREAKDOWN, "PCG breakdown (block form)");
  // recovery, one right-hand side at a time (single-RHS kernels on column k)
  const size_t n3 = 3 * (size_t)ctx->N;
  for (int k = 0; k < nrhs; ++k) {
    feti::launch_col_get(nl, nrhs, k, ctx->dm_lam, ctx->d_lam, st);
    apply_F(ctx, ctx->d_lam, ctx->d_q, nullptr, false, zero);
    feti::launch_axpy_to(nl, ctx->d_q, -scale[k], ctx->d_d, ctx->d_z, st);       // F lambda_k - d~_k
    if (ctx->cd > 0) {
      feti::launch_gtv(ctx->P, ctx->d_lay, ctx->d_R, ctx->maps, ctx->d_z, ctx->d_g, zero, st);
      coarse_apply_g(ctx, ctx->d_g, ctx->d_c, zero);
    }
    feti::launch_gather(ctx->maps, ctx->d_lam, nullptr, ctx->d_loc, zero, st);
    feti::launch_axpy_to((int)ctx->nloc_total, ctx->d_f, scale[k] - 1.0, ctx->d_f, ctx->d_x2, st);   // scale_k f
    feti::launch_local_sub(ctx->P, ctx->d_lay, ctx->d_x2, ctx->d_loc, ctx->d_x2, st);
    kplus(ctx, ctx->d_x2, ctx->d_x);
    if (ctx->cd > 0) feti::launch_add_kernel(ctx->P, ctx->d_lay, ctx->d_R, ctx->d_c, ctx->d_x, st);
    FETI_CK(cudaGetLastError());
    double* out_k = u_out + k * n3;
    FETI_TRY(write_displacement(ctx, out_k, u_on_device, u_on_device ? out_k : ctx->d_Uout));
  }
  if (!conv) return fail(ctx, FETI_ERR_NOT_CONVERGED, "PCG reached maxit (block form)");
  return FETI_OK;
}

feti_status write_displacement(feti_ctx* ctx, double* u_out, int on_device, double* d_target) {
  cudaStream_t st = ctx->stream;
  const size_t n3 = 3 * (size_t)ctx->N;
  double* dst = d_target;
  FETI_CK(cudaMemcpyAsync(dst, ctx->d_Uinit, n3 * sizeof(double), cudaMemcpyDeviceToDevice, st));
  feti::launch_owner_scatter(ctx->n_own, ctx->d_own_gdof, ctx->d_own_vpos, ctx->d_x, dst, st);
  FETI_CK(cudaGetLastError());
  if (u_out && u_out != dst) {
    FETI_CK(cudaMemcpyAsync(u_out, dst, n3 * sizeof(double), on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
  }
  FETI_CK(cudaStreamSynchronize(st));
  return FETI_OK;
}

}  // namespace

namespace feti {

feti_status set_error(feti_ctx* ctx, feti_status st, const std::string& msg) { return fail(ctx, st, msg); }

feti_status dual_apply_noalloc(feti_ctx* ctx, const double* v, double* q, double* z) {
  FETI_TRY(need_device(ctx));
  if (!v || !q || !z) return fail(ctx, FETI_ERR_INVALID_ARG, "feti_dual_apply_noalloc: null vector");
  if (!ctx->noalloc_scratch)
    return fail(ctx, FETI_ERR_CUDA, "feti_dual_apply_noalloc: static scratch unavailable (" + ctx->noalloc_err + ")");
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    (void)cudaGetLastError();
    return fail(ctx, FETI_ERR_CUDA, "feti_dual_apply_noalloc: no current CUDA device");
  }
  if (dev != ctx->device)
    return fail(ctx, FETI_ERR_INVALID_ARG, "feti_dual_apply_noalloc: current device " + std::to_string(dev) +
                                               " is not the context's device " + std::to_string(ctx->device));
  double* scratch = ctx->noalloc_scratch;
  const size_t capacity = ctx->noalloc_cap;
  // scratch: local input (doubles, or floats for the FP32 copies) + local output
  const size_t nb = (size_t)ctx->nb_total;
  const size_t need = nb + (nb + 7) / 2 + 4 + nb;
  if (need > capacity)
    return fail(ctx, FETI_ERR_INVALID_ARG,
                "feti_dual_apply_noalloc: this decomposition needs " + std::to_string(need) +
                    " doubles of scratch (about 2.5 per boundary DOF), the static scratch holds " +
                    std::to_string(capacity));
  if (!ctx->prepared) return fail(ctx, FETI_ERR_STATE, "call feti_prepare or feti_solve first");
  {
    // an error left pending by earlier work is reported, not cleared
    const cudaError_t pend = cudaPeekAtLastError();
    if (pend != cudaSuccess)
      return fail(ctx, FETI_ERR_CUDA, std::string("feti_dual_apply_noalloc: pending CUDA error: ") +
                                          cudaGetErrorString(pend));
  }
  cudaStream_t st = ctx->stream;
  const int* zero = ctx->d_zero;
  double* vloc = scratch;                                          // nb doubles
  float* vloc32 = reinterpret_cast<float*>(scratch + nb);          // nb floats, 16-byte aligned
  double* loc = scratch + nb + (nb + 7) / 2 + 4;                   // nb doubles
  vloc32 = reinterpret_cast<float*>(reinterpret_cast<uintptr_t>(vloc32 + 3) & ~uintptr_t(15));
  const bool f32 = f32_ops(ctx);
  // q = F v
  if (f32) {
    feti::launch_gather32(ctx->maps, v, nullptr, vloc32, zero, st);
    feti::launch_gemv_loc(ctx->cfg32[0], ctx->d_lay, 0, ctx->d_F32, 1, vloc32, loc, ctx->max_nb, zero, st);
  } else {
    feti::launch_gather(ctx->maps, v, nullptr, vloc, zero, st);
    feti::launch_gemv_loc(ctx->cfg64[0], ctx->d_lay, 0, ctx->d_F, 0, vloc, loc, ctx->max_nb, zero, st);
  }
  feti::launch_scatter(ctx->maps, loc, nullptr, q, nullptr, nullptr, zero, st);
  // z = W B Y B^T W q
  if (ctx->opt.precond == FETI_PREC_IDENTITY) {
    feti::launch_gather(ctx->maps, q, ctx->d_weight, loc, zero, st);
  } else if (ctx->opt.precond == FETI_PREC_LUMPED) {
    feti::launch_gather(ctx->maps, q, ctx->d_weight, vloc, zero, st);
    feti::launch_spmv_lump((int)ctx->nb_total, ctx->d_lump_ptr, ctx->d_lump_col, ctx->d_lump_val, vloc, loc, zero, st);
  } else if (f32) {
    feti::launch_gather32(ctx->maps, q, ctx->d_weight, vloc32, zero, st);
    feti::launch_gemv_loc(ctx->cfg32[1], ctx->d_lay, 1, ctx->d_S32, 1, vloc32, loc, ctx->max_nb, zero, st);
  } else {
    feti::launch_gather(ctx->maps, q, ctx->d_weight, vloc, zero, st);
    feti::launch_gemv_loc(ctx->cfg64[1], ctx->d_lay, 1, ctx->d_S, 0, vloc, loc, ctx->max_nb, zero, st);
  }
  feti::launch_scatter(ctx->maps, loc, ctx->d_weight, z, nullptr, nullptr, zero, st);
  FETI_CK(cudaGetLastError());
  return FETI_OK;
}

}  // namespace feti

extern "C" {

}  // extern "C"

namespace {

// feti_create and feti_create_plan: argument checks, then (dry = false) the
// device and stream set-up, then the host decomposition and its upload.
feti_status create_context(feti_ctx** out, const feti_mesh* mesh, const feti_material* mat, const feti_bc* bc,
                           const feti_options* opt, void* stream, bool dry) {
  if (!out) return FETI_ERR_INVALID_ARG;
  *out = nullptr;
  feti_ctx* ctx = new (std::nothrow) feti_ctx();
  if (!ctx) return FETI_ERR_OOM;
  *out = ctx;
  ctx->dry = dry;
  if (!mesh || !mat || !bc || !opt) return fail(ctx, FETI_ERR_INVALID_ARG, "null argument");
  if (mesh->n_nodes <= 0 || mesh->n_tets <= 0 || mesh->n_parts <= 0 || !mesh->coords || !mesh->tets || !mesh->part)
    return fail(ctx, FETI_ERR_INVALID_ARG, "empty or missing mesh arrays");
  if (opt->method != FETI_CLASSICAL && opt->method != FETI_ALL_FLOATING)
    return fail(ctx, FETI_ERR_INVALID_ARG, "unknown method");
  if (opt->precond < FETI_PREC_IDENTITY || opt->precond > FETI_PREC_DIRICHLET)
    return fail(ctx, FETI_ERR_INVALID_ARG, "unknown preconditioner");
  if (opt->precision != FETI_FP64 && opt->precision != FETI_MIXED && opt->precision != FETI_MIXED_F32FACTOR)
    return fail(ctx, FETI_ERR_INVALID_ARG, "unsupported precision");
  if (opt->coarse_form < 0 || opt->coarse_form > 2) return fail(ctx, FETI_ERR_INVALID_ARG, "unsupported coarse_form");
  if (opt->local_form < 0 || opt->local_form > 2) return fail(ctx, FETI_ERR_INVALID_ARG, "unsupported local_form");
  if (opt->local_form == 2 && opt->precision != FETI_FP64)
    return fail(ctx, FETI_ERR_INVALID_ARG, "the implicit local form needs FETI_FP64");
  if (opt->workspace_mb < -1) return fail(ctx, FETI_ERR_INVALID_ARG, "workspace_mb must be >= -1");
  if (!(opt->tol > 0.0) || opt->maxit <= 0) return fail(ctx, FETI_ERR_INVALID_ARG, "tol and maxit must be positive");
  if (mat->kind != FETI_LINEAR_ISO && mat->kind != FETI_HGO_TWO_FIBRE && mat->kind != FETI_LINEAR_ISO_P0)
    return fail(ctx, FETI_ERR_INVALID_ARG, "unknown material");
  if (mat->kind == FETI_HGO_TWO_FIBRE && !mat->fibres) return fail(ctx, FETI_ERR_INVALID_ARG, "fibres required");
  ctx->N = mesh->n_nodes;
  ctx->E = mesh->n_tets;
  ctx->P = mesh->n_parts;
  ctx->coords.assign(mesh->coords, mesh->coords + 3 * (size_t)ctx->N);
  ctx->npe = mesh->nodes_per_tet == 0 ? 4 : mesh->nodes_per_tet;
  if (ctx->npe != 4 && ctx->npe != 10) return fail(ctx, FETI_ERR_INVALID_ARG, "nodes_per_tet must be 4 or 10");
  ctx->nde = 3 * ctx->npe;
  ctx->fpn = ctx->npe == 10 ? 6 : 3;
  if (ctx->npe == 10 && mat->kind == FETI_HGO_TWO_FIBRE)
    return fail(ctx, FETI_ERR_INVALID_ARG, "10-node tetrahedra are built for the linear materials");
  ctx->tets.assign(mesh->tets, mesh->tets + (size_t)ctx->npe * ctx->E);
  ctx->part.assign(mesh->part, mesh->part + ctx->E);
  for (int32_t v : ctx->tets)
    if (v < 0 || v >= ctx->N) return fail(ctx, FETI_ERR_INVALID_ARG, "tetrahedron node out of range");
  for (int32_t v : ctx->part)
    if (v < 0 || v >= ctx->P) return fail(ctx, FETI_ERR_INVALID_ARG, "subdomain id out of range");
  for (double v : ctx->coords)
    if (!std::isfinite(v)) return fail(ctx, FETI_ERR_INVALID_ARG, "non-finite coordinate");
  ctx->mat = *mat;
  if (mat->fibres) ctx->fibres.assign(mat->fibres, mat->fibres + 6 * (size_t)ctx->E);
  if (bc->n_dir < 0 || bc->n_press < 0 || bc->n_trac < 0) return fail(ctx, FETI_ERR_INVALID_ARG, "negative count");
  if (bc->n_dir > 0 && (!bc->dir_dof || !bc->dir_val)) return fail(ctx, FETI_ERR_INVALID_ARG, "missing Dirichlet arrays");
  ctx->dir_dof.assign(bc->dir_dof, bc->dir_dof + bc->n_dir);
  ctx->dir_val.assign(bc->dir_val, bc->dir_val + bc->n_dir);
  for (int i = 0; i < bc->n_dir; ++i) {
    if (ctx->dir_dof[i] < 0 || ctx->dir_dof[i] >= 3 * ctx->N) return fail(ctx, FETI_ERR_INVALID_ARG, "Dirichlet DOF out of range");
    if (i && ctx->dir_dof[i] <= ctx->dir_dof[i - 1]) return fail(ctx, FETI_ERR_INVALID_ARG, "Dirichlet DOFs must increase");
  }
  ctx->n_press = bc->n_press;
  ctx->n_trac = bc->n_trac;
  ctx->pressure = bc->pressure;
  for (int i = 0; i < 3; ++i) ctx->traction[i] = bc->traction[i];
  if ((bc->n_press && (!bc->press_tri || !bc->press_owner)) || (bc->n_trac && (!bc->trac_tri || !bc->trac_owner)))
    return fail(ctx, FETI_ERR_INVALID_ARG, "missing face arrays");
  ctx->face_tri.assign(bc->press_tri, bc->press_tri + (size_t)ctx->fpn * bc->n_press);
  ctx->face_tri.insert(ctx->face_tri.end(), bc->trac_tri, bc->trac_tri + (size_t)ctx->fpn * bc->n_trac);
  ctx->face_owner.assign(bc->press_owner, bc->press_owner + bc->n_press);
  ctx->face_owner.insert(ctx->face_owner.end(), bc->trac_owner, bc->trac_owner + bc->n_trac);
  for (int32_t v : ctx->face_owner)
    if (v < 0 || v >= ctx->E) return fail(ctx, FETI_ERR_INVALID_ARG, "face owner out of range");
  for (int32_t v : ctx->face_tri)
    if (v < 0 || v >= ctx->N) return fail(ctx, FETI_ERR_INVALID_ARG, "face node out of range");
  ctx->opt = *opt;
  if (dry) return build_decomposition(ctx);
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    (void)cudaGetLastError();
    return fail(ctx, FETI_ERR_CUDA, "no CUDA device");
  }
  (void)cudaGetLastError();
  if (stream) {
    ctx->stream = static_cast<cudaStream_t>(stream);
  } else {
    FETI_CK(cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking));
    ctx->own_stream = true;
  }
  StageLog lg(ctx);
  FETI_CK(cudaGetDevice(&ctx->device));
  {
    // set-up of feti_dual_apply_noalloc on this device: the static scratch's
    // device address (this loads its module here, not in a later call)
    const cudaError_t e = feti::noalloc_scratch_lookup(&ctx->noalloc_scratch, &ctx->noalloc_cap);
    if (e != cudaSuccess) {
      ctx->noalloc_err = std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e);
      (void)cudaGetLastError();
    }
  }
  lg.mark("create: arguments");
  const feti_status st = build_decomposition(ctx);
  lg.mark("create: decomposition + upload");
  return st;
}

}  // namespace

extern "C" {

feti_status feti_create(feti_ctx** out, const feti_mesh* mesh, const feti_material* mat, const feti_bc* bc,
                        const feti_options* opt, void* stream) {
  return create_context(out, mesh, mat, bc, opt, stream, false);
}

feti_status feti_create_plan(feti_ctx** out, const feti_mesh* mesh, const feti_material* mat, const feti_bc* bc,
                             const feti_options* opt) {
  return create_context(out, mesh, mat, bc, opt, nullptr, true);
}

feti_status feti_prepare(feti_ctx* ctx) {
  if (!ctx) return FETI_ERR_INVALID_ARG;
  FETI_TRY(need_device(ctx));
  (void)cudaGetLastError();  // drop a non-sticky error left by an earlier, unrelated runtime call
  auto t0 = std::chrono::steady_clock::now();
  ctx->shift = 0.0;  // exact local operators (a Newton run may have left a shift)
  FETI_TRY(prepare(ctx, nullptr, 1.0));
  ctx->t_setup_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  return FETI_OK;
}

feti_status feti_solve(feti_ctx* ctx, double* u_out, int32_t u_on_device, feti_report* report) {
  if (!ctx) return FETI_ERR_INVALID_ARG;
  FETI_TRY(need_device(ctx));
  (void)cudaGetLastError();
  if (!u_out) return fail(ctx, FETI_ERR_INVALID_ARG, "null output");
  auto t0 = std::chrono::steady_clock::now();
  if (report) std::memset(report, 0, sizeof(*report));
  if (ctx->mat.kind == FETI_HGO_TWO_FIBRE) return fail(ctx, FETI_ERR_INVALID_ARG, "feti_solve needs a linear material");
  FETI_TRY(feti_prepare(ctx));
  float pcg_ms = 0.f;
  feti_status s = dual_solve(ctx, report, &pcg_ms);
  if (s != FETI_OK && s != FETI_ERR_NOT_CONVERGED) return s;
  FETI_TRY(write_displacement(ctx, u_out, u_on_device, (u_on_device ? u_out : ctx->d_Uout)));
  if (report) {
    report->t_setup_ms = ctx->t_setup_ms;
    report->t_total_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  }
  return s;
}

// ||sum_i A_i x_i|| over the non-Dirichlet global DOFs (device reduction,
// fixed-order sum of the per-CTA partials on the host).
static feti_status global_norm(feti_ctx* ctx, const double* x, double* out) {
  const int np = feti::scatter_partials();
  feti::launch_global_sumsq(ctx->n_gs, ctx->d_gs_ptr, ctx->d_gs_pos, x, ctx->d_partial, ctx->stream);
  FETI_CK(cudaGetLastError());
  ctx->h_partial.resize(np);
  FETI_CK(cudaMemcpyAsync(ctx->h_partial.data(), ctx->d_partial, np * sizeof(double), cudaMemcpyDeviceToHost,
                          ctx->stream));
  FETI_CK(cudaStreamSynchronize(ctx->stream));
  double t = 0.0;
  for (double v : ctx->h_partial) t += v;
  *out = std::sqrt(t);
  return FETI_OK;
}

// Relative residual ||f_int(U) - tau f_ext(U)|| / ||tau f_ext(U)|| from the
// local vectors of the last assembly (d_f = tau f_ext - f_int per subdomain).
static feti_status newton_residual(feti_ctx* ctx, const double* dU, double tau, double* rel) {
  double rn = 0.0, fn = 0.0;
  FETI_TRY(global_norm(ctx, ctx->d_f, &rn));
  feti::launch_assemble_rhs(ctx->P, ctx->d_lay, ctx->d_sub_face_ptr, ctx->d_face_dense, ctx->d_face_force,
                            3 * ctx->fpn, ctx->d_sub_elem_ptr, ctx->d_sub_elems, ctx->d_elem_dense, nullptr,
                            ctx->d_Ke, nullptr, ctx->nde, tau, ctx->d_fl, ctx->stream);
  FETI_TRY(global_norm(ctx, ctx->d_fl, &fn));
  (void)dU;
  *rel = fn > 0.0 ? rn / fn : rn;
  return FETI_OK;
}

// (a, b) over the non-Dirichlet global DOFs: per-CTA partials, fixed-order
// host sum.
static feti_status gs_dot(feti_ctx* ctx, const double* a, const double* b, double* out) {
  const int np = feti::scatter_partials();
  feti::launch_gs_dot(ctx->n_gs, a, b, ctx->d_partial, ctx->stream);
  FETI_CK(cudaGetLastError());
  ctx->h_partial.resize(np);
  FETI_CK(cudaMemcpyAsync(ctx->h_partial.data(), ctx->d_partial, np * sizeof(double), cudaMemcpyDeviceToHost,
                          ctx->stream));
  FETI_CK(cudaStreamSynchronize(ctx->stream));
  double t = 0.0;
  for (double v : ctx->h_partial) t += v;
  *out = t;
  return FETI_OK;
}

// Newton increment dU (3N, zero on Dirichlet DOFs) from the local residuals
// d_f of the last assembly: flexible CG on the assembled tangent system
// K dU = R over the non-Dirichlet DOFs, with the FETI solve as the
// preconditioner (residual injected into the owner copies, dual PCG,
// recovery, owner copies taken back) and K applied element by element from
// the stored element tangents.  When the FETI increment is exact the first
// iteration already meets the tolerance; when the reference rigid modes are
// no longer exact kernels of the prestressed local tangents, the outer
// iteration supplies what the FETI increment misses.  Stops at
// ||R - K dU|| <= eta ||R|| or after max_it FETI solves.
static feti_status newton_increment(feti_ctx* ctx, double eta, int max_it, int* pcg_its, double* pcg_ms,
                                    int* krylov_its, double* krylov_rel) {
  cudaStream_t st = ctx->stream;
  const int n = ctx->n_gs;
  if (!ctx->d_nk) FETI_TRY(dev_alloc(ctx, &ctx->d_nk, 5 * (size_t)std::max(n, 1)));
  double *x = ctx->d_nk, *r = x + n, *z = r + n, *p = z + n, *q = p + n;
  feti::launch_gs_assemble(n, ctx->d_gs_ptr, ctx->d_gs_pos, ctx->d_f, r, st);
  FETI_CK(cudaMemsetAsync(x, 0, (size_t)n * sizeof(double), st));
  double bb = 0.0;
  FETI_TRY(gs_dot(ctx, r, r, &bb));
  const double bnorm = std::sqrt(bb);
  double pq_prev = 0.0, rn = bnorm;
  *krylov_its = 0;
  for (int it = 0; it < max_it && rn > 0.0; ++it) {
    FETI_CK(cudaMemsetAsync(ctx->d_f, 0, (size_t)ctx->nloc_total * sizeof(double), st));
    feti::launch_gs_inject(n, ctx->d_gs_ptr, ctx->d_gs_pos, r, ctx->d_f, st);
    feti_report rep{};
    float ms = 0.f;
    {
      // the FETI solve is only the preconditioner here: an inner PCG that
      // stops at maxit (possible on shifted local tangents) still gives a
      // usable direction for the flexible CG
      const feti_status ds = dual_solve(ctx, &rep, &ms);
      if (ds != FETI_OK && ds != FETI_ERR_NOT_CONVERGED) return ds;
    }
    *pcg_its += rep.iterations;
    *pcg_ms += ms;
    feti::launch_gs_take(n, ctx->d_gs_ptr, ctx->d_gs_pos, ctx->d_x, z, st);
    if (it == 0) {
      FETI_CK(cudaMemcpyAsync(p, z, (size_t)n * sizeof(double), cudaMemcpyDeviceToDevice, st));
    } else {
      double zq = 0.0;
      FETI_TRY(gs_dot(ctx, z, q, &zq));  // q = K p of the previous direction
      feti::launch_axpy_to(n, z, -zq / pq_prev, p, p, st);
    }
    feti::launch_gs_elem_matvec(n, ctx->d_inc_ptr, ctx->d_inc, ctx->d_elem_gs, ctx->d_Ke, p, q, st);
    double pq = 0.0, pr = 0.0;
    FETI_TRY(gs_dot(ctx, p, q, &pq));
    FETI_TRY(gs_dot(ctx, p, r, &pr));
    if (!(pq > 0.0) || !std::isfinite(pq)) {
      if (it == 0) {  // tangent not positive along the FETI increment: keep that increment
        FETI_CK(cudaMemcpyAsync(x, z, (size_t)n * sizeof(double), cudaMemcpyDeviceToDevice, st));
        *krylov_its = 1;
      }
      break;
    }
    const double alpha = pr / pq;
    feti::launch_axpy_to(n, x, alpha, p, x, st);
    feti::launch_axpy_to(n, r, -alpha, q, r, st);
    double rr = 0.0;
    FETI_TRY(gs_dot(ctx, r, r, &rr));
    rn = std::sqrt(rr);
    *krylov_its = it + 1;
    pq_prev = pq;
    if (rn <= eta * bnorm) break;
  }
  *krylov_rel = bnorm > 0.0 ? rn / bnorm : 0.0;
  FETI_CK(cudaMemsetAsync(ctx->d_dU, 0, 3 * (size_t)ctx->N * sizeof(double), st));
  feti::launch_gs_to_global(n, ctx->d_gs_gdof, x, ctx->d_dU, st);
  FETI_CK(cudaGetLastError());
  return FETI_OK;
}

// Setup of a Newton iteration at U: element tangents, local assembly and
// factorization.  A local tangent that is not positive definite (possible
// under prestress: rigid rotations stop being kernel vectors of a
// subdomain's tangent, and its quadratic form along them can turn negative)
// is shifted, A_ii += delta max_j A_jj with delta = 1e-6, 1e-5, .. 1e-1, until
// every local Cholesky factorization succeeds; the FETI solve is then only
// the preconditioner of the flexible CG on the exact element-assembled
// tangent (newton_increment), which still converges to the Newton increment.
static feti_status prepare_newton(feti_ctx* ctx, const double* dU, double tau, bool log) {
  ctx->shift = 0.0;
  feti_status s = prepare(ctx, dU, tau);
  for (double d = 1e-6; s == FETI_ERR_LOCAL_SINGULAR && d <= 0.11; d *= 10.0) {
    ctx->shift = d;
    if (log) std::fprintf(stderr, "feti_newton: local tangent not positive definite; shift %.0e\n", d);
    s = prepare(ctx, dU, tau);
  }
  return s;
}

// Load steps first..last of the load-stepped Newton method (Sec. 3.2, Eq.
// loadStepping: tau = s / n_load_steps), starting from U_start (device, host
// or NULL = zero) -- the state after load step first - 1.
static feti_status newton_run(feti_ctx* ctx, const double* U_start, int32_t u_start_on_device, int first, int last,
                              double* u_out, int32_t u_on_device, int32_t* pcg_per_step, int32_t* newton_per_step,
                              feti_report* report) {
  if (!u_out) return fail(ctx, FETI_ERR_INVALID_ARG, "null output");
  (void)cudaGetLastError();
  if (ctx->mat.kind != FETI_HGO_TWO_FIBRE) return fail(ctx, FETI_ERR_INVALID_ARG, "feti_newton needs HGO_TWO_FIBRE");
  if (ctx->npe != 4) return fail(ctx, FETI_ERR_INVALID_ARG, "feti_newton is built for 4-node tetrahedra");
  if (f32_factor(ctx))
    return fail(ctx, FETI_ERR_INVALID_ARG, "feti_newton: FETI_MIXED_F32FACTOR is for linear solves");
  for (double v : ctx->dir_val)
    if (v != 0.0) return fail(ctx, FETI_ERR_INVALID_ARG, "feti_newton needs homogeneous Dirichlet data");
  const int nsteps = ctx->opt.n_load_steps > 0 ? ctx->opt.n_load_steps : 1;
  if (first < 1 || last > nsteps || first > last)
    return fail(ctx, FETI_ERR_INVALID_ARG, "load steps must satisfy 1 <= first <= last <= n_load_steps");
  if (report) std::memset(report, 0, sizeof(*report));
  auto t0 = std::chrono::steady_clock::now();
  cudaStream_t st = ctx->stream;
  const int n3 = 3 * ctx->N;
  const int maxit = ctx->opt.newton_maxit > 0 ? ctx->opt.newton_maxit : 25;
  const double ntol = ctx->opt.newton_tol > 0 ? ctx->opt.newton_tol : 1e-8;
  if (U_start)
    FETI_CK(cudaMemcpyAsync(ctx->d_U, U_start, n3 * sizeof(double),
                            u_start_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
  else
    FETI_CK(cudaMemsetAsync(ctx->d_U, 0, n3 * sizeof(double), st));
  // FETI_LOG=1 in the environment prints one line per Newton iteration to stderr
  const char* log_env = std::getenv("FETI_LOG");
  const bool log = log_env && log_env[0] && log_env[0] != '0';
  int newton_total = 0, pcg_total = 0;
  double rel = 0.0;
  double t_pcg = 0.0;
  for (int step = first; step <= last; ++step) {
    const double tau = (double)step / nsteps;
    int step_newton = 0, step_pcg_total = 0;
    FETI_TRY(prepare_newton(ctx, ctx->d_U, tau, log));
    FETI_TRY(newton_residual(ctx, ctx->d_U, tau, &rel));
    if (log) std::fprintf(stderr, "feti_newton: load step %d tau %.4f start rel %.3e\n", step, tau, rel);
    for (int k = 0;; ++k) {
      if (rel <= ntol) break;
      if (k >= maxit) {
        if (report) { report->newton_iters = newton_total; report->newton_rel_res = rel; report->iterations = pcg_total; }
        return fail(ctx, FETI_ERR_NEWTON_DIVERGED, "Newton reached its iteration limit at load step " + std::to_string(step));
      }
      int step_pcg = 0, kits = 0;
      double krel = 0.0;
      FETI_TRY(newton_increment(ctx, 1e-4, 12, &step_pcg, &t_pcg, &kits, &krel));
      pcg_total += step_pcg;
      step_pcg_total += step_pcg;
      feti_status s = FETI_OK;
      // the full Newton step (Sec. 3.2, Eq. NewtonRecursion); the step is
      // halved only while an element inverts (down to 1/64).  Local tangents
      // that are not positive definite at the new state are shifted for the
      // FETI preconditioner (prepare_newton).
      double a = 1.0;
      for (;;) {
        feti::launch_axpy_to(n3, ctx->d_U, a, ctx->d_dU, ctx->d_Utrial, st);
        feti::launch_zero_list((int)ctx->dir_dof.size(), ctx->d_dir_dof, ctx->d_Utrial, st);
        s = prepare_newton(ctx, ctx->d_Utrial, tau, log);
        if (s == FETI_OK) break;
        if (log) std::fprintf(stderr, "feti_newton: step %d it %d step length %.4f rejected (%s)\n", step, k + 1, a,
                              ctx->err.c_str());
        if (s != FETI_ERR_ELEMENT_INVERTED) return s;
        a *= 0.5;
        if (a < 1.0 / 64) return fail(ctx, FETI_ERR_NEWTON_DIVERGED, "every step length inverts an element");
      }
      FETI_CK(cudaMemcpyAsync(ctx->d_U, ctx->d_Utrial, n3 * sizeof(double), cudaMemcpyDeviceToDevice, st));
      ++newton_total;
      ++step_newton;
      FETI_TRY(newton_residual(ctx, ctx->d_U, tau, &rel));
      if (log) {
        std::fprintf(stderr,
                     "feti_newton: step %d it %d: %d FETI solves (%d PCG iterations), increment residual %.2e, "
                     "step length %.4f -> rel %.3e\n",
                     step, k + 1, kits, step_pcg, krel, a, rel);
      }
    }
    if (pcg_per_step) pcg_per_step[step - first] = step_pcg_total;
    if (newton_per_step) newton_per_step[step - first] = step_newton;
  }
  FETI_CK(cudaMemcpyAsync(u_out, ctx->d_U, n3 * sizeof(double), u_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
  FETI_CK(cudaStreamSynchronize(st));
  if (report) {
    report->newton_iters = newton_total;
    report->newton_rel_res = rel;
    report->iterations = pcg_total;
    report->converged = 1;
    report->t_pcg_ms = t_pcg;
    report->n_lambda = ctx->n_lambda;
    report->coarse_dim = ctx->cd;
    report->t_total_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  }
  return FETI_OK;
}

feti_status feti_newton(feti_ctx* ctx, double* u_out, int32_t u_on_device, feti_report* report) {
  if (!ctx) return FETI_ERR_INVALID_ARG;
  FETI_TRY(need_device(ctx));
  const int nsteps = ctx->opt.n_load_steps > 0 ? ctx->opt.n_load_steps : 1;
  return newton_run(ctx, nullptr, 0, 1, nsteps, u_out, u_on_device, nullptr, nullptr, report);
}

feti_status feti_newton_steps(feti_ctx* ctx, const double* U_start, int32_t first_step, int32_t last_step,
                              double* u_out, int32_t u_on_device, int32_t* pcg_per_step, int32_t* newton_per_step,
                              feti_report* report) {
  if (!ctx) return FETI_ERR_INVALID_ARG;
  FETI_TRY(need_device(ctx));
  return newton_run(ctx, U_start, u_on_device, first_step, last_step, u_out, u_on_device, pcg_per_step,
                    newton_per_step, report);
}

feti_status feti_elements(feti_ctx* ctx, const double* U, int32_t u_on_device, double* Ke_out, double* fe_out,
                          int32_t out_on_device) {
  if (!ctx) return FETI_ERR_INVALID_ARG;
  FETI_TRY(need_device(ctx));
  if (!Ke_out) return fail(ctx, FETI_ERR_INVALID_ARG, "null Ke_out");
  (void)cudaGetLastError();
  cudaStream_t st = ctx->stream;
  const bool hgo = ctx->mat.kind == FETI_HGO_TWO_FIBRE;
  const size_t n3 = 3 * (size_t)ctx->N;
  if (hgo && !ctx->d_U) FETI_TRY(dev_alloc(ctx, &ctx->d_U, n3));
  const double* dU = nullptr;
  if (hgo && U) {
    FETI_CK(cudaMemcpyAsync(ctx->d_U, U, n3 * sizeof(double), u_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
    dU = ctx->d_U;
  }
  FETI_CK(cudaMemsetAsync(ctx->d_status, 0, sizeof(int), st));
  if (!ctx->elem_ev[0]) {
    FETI_CK(cudaEventCreate(&ctx->elem_ev[0]));
    FETI_CK(cudaEventCreate(&ctx->elem_ev[1]));
  }
  FETI_CK(cudaEventRecord(ctx->elem_ev[0], st));
  launch_elements(ctx, dU);
  FETI_CK(cudaGetLastError());
  FETI_CK(cudaEventRecord(ctx->elem_ev[1], st));
  FETI_TRY(check_status(ctx, "element matrices"));
  {
    float ms = 0.f;
    FETI_CK(cudaEventElapsedTime(&ms, ctx->elem_ev[0], ctx->elem_ev[1]));
    ctx->elem_ms = ms;
    // connectivity, fibres (hyperelastic), packed symmetric tangent and force
    // per element; coordinates (+ displacement) per node
    const double nd = ctx->nde;
    const double per_elem = 4.0 * ctx->npe + nd * (nd + 1) / 2 * 8.0 + (hgo ? 48.0 + 12.0 * 8.0 : 0.0);
    const double per_node = hgo ? 48.0 : 24.0;
    ctx->elem_bytes = per_elem * (double)ctx->E + per_node * (double)ctx->N;
  }
  const cudaMemcpyKind kind = out_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  // full nde x nde copies of the packed (upper-triangle) element matrices
  const size_t full = (size_t)ctx->nde * ctx->nde * ctx->E;
  if (out_on_device) {
    feti::launch_ke_unpack(ctx->E, ctx->nde, ctx->d_Ke, Ke_out, st);
    FETI_CK(cudaGetLastError());
  } else {
    double* tmp = nullptr;
    FETI_CK(cudaMalloc(&tmp, std::max<size_t>(full, 1) * sizeof(double)));
    feti::launch_ke_unpack(ctx->E, ctx->nde, ctx->d_Ke, tmp, st);
    cudaError_t e = cudaMemcpyAsync(Ke_out, tmp, full * sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(tmp);
    FETI_CK(e);
  }
  if (fe_out && hgo) FETI_CK(cudaMemcpyAsync(fe_out, ctx->d_fe, 12 * (size_t)ctx->E * sizeof(double), kind, st));
  FETI_CK(cudaStreamSynchronize(st));
  return FETI_OK;
}

feti_status feti_solve_multi(feti_ctx* ctx, const double* load_scale, int32_t nrhs, double* u_out,
                             int32_t u_on_device, feti_report* report) {
  if (!ctx) return FETI_ERR_INVALID_ARG;
  FETI_TRY(need_device(ctx));
  if (!u_out || !load_scale) return fail(ctx, FETI_ERR_INVALID_ARG, "null argument");
  if (nrhs < 1 || nrhs > feti::kMaxRhs) return fail(ctx, FETI_ERR_INVALID_ARG, "nrhs must be in [1, 16]");
  (void)cudaGetLastError();
  if (report) std::memset(report, 0, sizeof(*report));
  if (ctx->mat.kind == FETI_HGO_TWO_FIBRE)
    return fail(ctx, FETI_ERR_INVALID_ARG, "feti_solve_multi needs a linear material");
  for (double v : ctx->dir_val)
    if (v != 0.0) return fail(ctx, FETI_ERR_INVALID_ARG, "feti_solve_multi needs homogeneous Dirichlet data");
  auto t0 = std::chrono::steady_clock::now();
  FETI_TRY(feti_prepare(ctx));
  feti_status s = dual_solve_multi(ctx, load_scale, nrhs, u_out, u_on_device, report);
  if (report) {
    report->t_setup_ms = ctx->t_setup_ms;
    report->t_total_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  }
  return s;
}

feti_status feti_dual_apply_multi(feti_ctx* ctx, const double* v, double* q, double* z, int32_t nrhs,
                                  int32_t n_apply, double* ms_per_apply) {
  if (!ctx) return FETI_ERR_INVALID_ARG;
  FETI_TRY(need_device(ctx));
  if (!v || !q || !z || n_apply <= 0 || nrhs < 1 || nrhs > feti::kMaxRhs)
    return fail(ctx, FETI_ERR_INVALID_ARG, "bad dual_apply_multi arguments");
  if (!ctx->prepared) return fail(ctx, FETI_ERR_STATE, "call feti_prepare or feti_solve first");
  (void)cudaGetLastError();
  FETI_TRY(alloc_multi(ctx, nrhs));
  cudaStream_t st = ctx->stream;
  const int* zero = ctx->d_zero;
  const bool f32 = f32_ops(ctx);
  if (!(ctx->dualm_graph && ctx->dualm_v == v && ctx->dualm_q == q && ctx->dualm_z == z && ctx->dualm_n == n_apply &&
        ctx->dualm_nrhs == nrhs)) {
    if (ctx->dualm_graph) cudaGraphExecDestroy(ctx->dualm_graph);
    ctx->dualm_graph = nullptr;
    for (auto ev : ctx->dualm_events) cudaEventDestroy(ev);
    ctx->dualm_events.assign(2 * (size_t)n_apply + 2, nullptr);
    for (auto& ev : ctx->dualm_events) FETI_CK(cudaEventCreate(&ev));
    const feti::GemvCfg cfg = f32 ? ctx->cfgm32[0] : ctx->cfgm64[0];
    cudaGraph_t g = nullptr;
    FETI_CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    for (int i = 0; i < n_apply; ++i) {
      void* vl = f32 ? (void*)ctx->dm_vloc32 : (void*)ctx->dm_vloc;
      feti::launch_gather_m(ctx->maps, nrhs, v, nullptr, vl, f32 ? 1 : 0, zero, st);
      FETI_CK(cudaEventRecordWithFlags(ctx->dualm_events[2 + 2 * i], st, cudaEventRecordExternal));
      if (f32 && ctx->tc_m[0])
        feti::launch_gemm_tc(ctx->tab[0][2], ctx->d_lay, 0, ctx->d_F32, nrhs, static_cast<const float*>(vl), ctx->dm_loc,
                             zero, ctx->d_tc_err, ctx->tc_m[0], ctx->d_tmap[0], ctx->d_spin, st);
      else
        feti::launch_gemm_loc(cfg, ctx->d_lay, 0, f32 ? (const void*)ctx->d_F32 : (const void*)ctx->d_F, f32 ? 1 : 0,
                              nrhs, vl, ctx->dm_loc, ctx->max_nb, zero, st);
      FETI_CK(cudaEventRecordWithFlags(ctx->dualm_events[3 + 2 * i], st, cudaEventRecordExternal));
      feti::launch_scatter_m(ctx->maps, nrhs, ctx->dm_loc, nullptr, q, nullptr, nullptr, zero, st);
      apply_M_m(ctx, nrhs, q, z, zero, f32);
    }
    FETI_CK(cudaStreamEndCapture(st, &g));
    cudaError_t e = cudaGraphInstantiate(&ctx->dualm_graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(ctx, FETI_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    ctx->dualm_v = v;
    ctx->dualm_q = q;
    ctx->dualm_z = z;
    ctx->dualm_n = n_apply;
    ctx->dualm_nrhs = nrhs;
  }
  FETI_CK(cudaEventRecord(ctx->dualm_events[0], st));
  FETI_CK(cudaGraphLaunch(ctx->dualm_graph, st));
  FETI_CK(cudaEventRecord(ctx->dualm_events[1], st));
  FETI_CK(cudaEventSynchronize(ctx->dualm_events[1]));
  float ms = 0.f;
  FETI_CK(cudaEventElapsedTime(&ms, ctx->dualm_events[0], ctx->dualm_events[1]));
  double kern = 0.0;
  for (int i = 0; i < n_apply; ++i) {
    float t = 0.f;
    FETI_CK(cudaEventElapsedTime(&t, ctx->dualm_events[2 + 2 * i], ctx->dualm_events[3 + 2 * i]));
    kern += t;
  }
  if (ms_per_apply) *ms_per_apply = ms / n_apply;
  double entries = 0.0, vec = 0.0;
  for (const auto& L : ctx->lay) {
    entries += (double)L.nbp * L.nbp;
    vec += (double)L.nbp;
  }
  ctx->gemv_ms = kern / n_apply;
  const double esz = f32 ? 4.0 : 8.0;
  ctx->gemv_bytes = entries * esz + vec * (esz + 8.0) * nrhs;
  ctx->gemv_flops = 2.0 * entries * nrhs;
  return FETI_OK;
}

feti_status feti_get_sizes(const feti_ctx* ctx, int64_t out[5]) {
  if (!ctx || !out) return FETI_ERR_INVALID_ARG;
  out[0] = ctx->n_lambda;
  out[1] = ctx->cd;
  out[2] = ctx->nloc_total;
  out[3] = ctx->nb_total;
  out[4] = ctx->P;
  return FETI_OK;
}

feti_status feti_get_coarse_info(const feti_ctx* ctx, int64_t out[6]) {
  if (!ctx || !out) return FETI_ERR_INVALID_ARG;
  for (int i = 0; i < 6; ++i) out[i] = 0;
  if (ctx->cd == 0) return FETI_OK;
  out[0] = ctx->coarse_sparse ? 2 : 1;
  if (!ctx->coarse_sparse) {
    out[3] = ctx->cd * ctx->cd;
    return FETI_OK;
  }
  const feti::CoarsePlan& cp = ctx->cplan;
  out[1] = (int64_t)cp.fronts.size();
  out[2] = cp.height;
  for (const auto& F : cp.fronts) out[3] += (int64_t)F.w * (F.w + 1) / 2 + (int64_t)F.w * F.p;
  out[4] = (int64_t)cp.tasks.size();
  out[5] = cp.ws;
  return FETI_OK;
}

feti_status feti_get_factor_info(const feti_ctx* ctx, int64_t out[5]) {
  if (!ctx || !out) return FETI_ERR_INVALID_ARG;
  out[0] = (int64_t)ctx->grp.size() - 1;
  out[1] = ctx->ws_elems;
  out[2] = ctx->ws_full;
  out[3] = ctx->keep_factor ? 0 : ctx->lc_elems;
  out[4] = ctx->opt.precision == FETI_MIXED_F32FACTOR ? 4 : 8;
  return FETI_OK;
}

feti_status feti_get_index_maps(const feti_ctx* ctx, int32_t* row_sub, int32_t* row_ldof, int8_t* row_sign,
                                double* weight, double* b) {
  if (!ctx) return FETI_ERR_INVALID_ARG;
  const size_t n = ctx->n_lambda;
  if (row_sub) std::memcpy(row_sub, ctx->row_sub.data(), 2 * n * sizeof(int32_t));
  if (row_ldof) std::memcpy(row_ldof, ctx->row_ldof.data(), 2 * n * sizeof(int32_t));
  if (row_sign) std::memcpy(row_sign, ctx->row_sign.data(), 2 * n * sizeof(int8_t));
  if (weight) std::memcpy(weight, ctx->weight.data(), n * sizeof(double));
  if (b) std::memcpy(b, ctx->bvec.data(), n * sizeof(double));
  return FETI_OK;
}

feti_status feti_get_fixing(const feti_ctx* ctx, int32_t* fix_ptr, int32_t* fix_ldof) {
  if (!ctx) return FETI_ERR_INVALID_ARG;
  if (fix_ptr) std::memcpy(fix_ptr, ctx->fix_ptr.data(), ctx->fix_ptr.size() * sizeof(int32_t));
  if (fix_ldof) std::memcpy(fix_ldof, ctx->fix_ldof.data(), ctx->fix_ldof.size() * sizeof(int32_t));
  return FETI_OK;
}

feti_status feti_dual_apply(feti_ctx* ctx, const double* v, double* q, double* z, int32_t n_apply,
                            double* ms_per_apply) {
  if (!ctx) return FETI_ERR_INVALID_ARG;
  FETI_TRY(need_device(ctx));
  if (!v || !q || !z || n_apply <= 0) return fail(ctx, FETI_ERR_INVALID_ARG, "bad dual_apply arguments");
  if (!ctx->prepared) return fail(ctx, FETI_ERR_STATE, "call feti_prepare or feti_solve first");
  (void)cudaGetLastError();
  cudaStream_t st = ctx->stream;
  const int* zero = ctx->d_zero;
  const bool same = ctx->dual_graph && ctx->dual_v == v && ctx->dual_q == q && ctx->dual_z == z &&
                    ctx->dual_n == n_apply;
  if (!same) {
    if (ctx->dual_graph) cudaGraphExecDestroy(ctx->dual_graph);
    ctx->dual_graph = nullptr;
    for (auto ev : ctx->dual_events) cudaEventDestroy(ev);
    ctx->dual_events.assign(2 * (size_t)n_apply + 2, nullptr);
    for (auto& ev : ctx->dual_events) FETI_CK(cudaEventCreate(&ev));
    // The graph brackets every F-gemv launch with event-record nodes so the
    // dominant kernel is timed inside the same run as the whole apply.
    cudaGraph_t g = nullptr;
    FETI_CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    const bool f32 = f32_ops(ctx);
    const bool implicit = !f32 && ctx->opt.local_form == 2;
    for (int i = 0; i < n_apply; ++i) {
      if (implicit) {
        // the timed span is the whole implicit local apply (gather, sweeps, boundary take)
        FETI_CK(cudaEventRecordWithFlags(ctx->dual_events[2 + 2 * i], st, cudaEventRecordExternal));
        local_apply(ctx, 0, v, nullptr, zero, false);
        FETI_CK(cudaEventRecordWithFlags(ctx->dual_events[3 + 2 * i], st, cudaEventRecordExternal));
        feti::launch_scatter(ctx->maps, ctx->d_loc, nullptr, q, nullptr, nullptr, zero, st);
        apply_M(ctx, q, z, zero, f32);
        continue;
      }
      if (f32)
        feti::launch_gather32(ctx->maps, v, nullptr, ctx->d_vloc32, zero, st);
      else
        feti::launch_gather(ctx->maps, v, nullptr, ctx->d_vloc, zero, st);
      FETI_CK(cudaEventRecordWithFlags(ctx->dual_events[2 + 2 * i], st, cudaEventRecordExternal));
      gemv_apply(ctx, 0, zero, f32);
      FETI_CK(cudaEventRecordWithFlags(ctx->dual_events[3 + 2 * i], st, cudaEventRecordExternal));
      feti::launch_scatter(ctx->maps, ctx->d_loc, nullptr, q, nullptr, nullptr, zero, st);
      apply_M(ctx, q, z, zero, f32);
    }
    FETI_CK(cudaStreamEndCapture(st, &g));
    cudaError_t e = cudaGraphInstantiate(&ctx->dual_graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(ctx, FETI_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    ctx->dual_v = v;
    ctx->dual_q = q;
    ctx->dual_z = z;
    ctx->dual_n = n_apply;
  }
  FETI_CK(cudaEventRecord(ctx->dual_events[0], st));
  FETI_CK(cudaGraphLaunch(ctx->dual_graph, st));
  FETI_CK(cudaEventRecord(ctx->dual_events[1], st));
  FETI_CK(cudaEventSynchronize(ctx->dual_events[1]));
  float ms = 0.f;
  FETI_CK(cudaEventElapsedTime(&ms, ctx->dual_events[0], ctx->dual_events[1]));
  double kern = 0.0;
  for (int i = 0; i < n_apply; ++i) {
    float t = 0.f;
    FETI_CK(cudaEventElapsedTime(&t, ctx->dual_events[2 + 2 * i], ctx->dual_events[3 + 2 * i]));
    kern += t;
  }
  if (ms_per_apply) *ms_per_apply = ms / n_apply;
  double entries = 0.0, half = 0.0, vec = 0.0;
  for (const auto& L : ctx->lay) {
    entries += (double)L.nbp * L.nbp;
    half += 0.5 * (double)L.nbp * (L.nbp + 1);
    vec += (double)L.nbp;
  }
  ctx->gemv_ms = kern / n_apply;
  // algorithmic bytes of one F_i apply: the n(n+1)/2 distinct entries of the
  // symmetric F_i once (8 B in FP64, 4 B in the FP32 copy), the gathered
  // local input (8 B) and the local output (8 B) per boundary DOF; flops: 2
  // per entry of the full matrix
  const double esz = f32_ops(ctx) ? 4.0 : 8.0;
  ctx->gemv_bytes = half * esz + vec * 16.0;
  ctx->gemv_flops = 2.0 * entries;
  return FETI_OK;
}

feti_status feti_element_stats(const feti_ctx* ctx, double* elem_ms, double* elem_bytes, double* n_elements) {
  if (!ctx || !elem_ms || !elem_bytes || !n_elements) return FETI_ERR_INVALID_ARG;
  const bool run = ctx->elem_ms > 0.0;
  *elem_ms = ctx->elem_ms;
  *elem_bytes = ctx->elem_bytes;
  *n_elements = run ? (double)ctx->E : 0.0;
  return FETI_OK;
}

feti_status feti_get_schedule(const feti_ctx* ctx, int32_t out[12]) {
  if (!ctx || !out) return FETI_ERR_INVALID_ARG;
  for (int i = 8; i < 12; ++i) out[i] = -1;
  for (int w = 0; w < 2; ++w) {
    out[2 * w] = ctx->cfg64[w].R;
    out[2 * w + 1] = ctx->cfg64[w].rpc;
    out[4 + 2 * w] = ctx->sym32[w] ? -ctx->sym32[w] : ctx->cfg32[w].R;
    out[4 + 2 * w + 1] = ctx->sym32[w] ? feti::kSymPH : ctx->cfg32[w].rpc;
    if (ctx->tuned_m) {
      out[8 + 2 * w] = ctx->tc_m[w] ? 1 - ctx->tc_m[w] : ctx->cfgm32[w].R;  // 0 .. -4: tensor-core variants
      out[8 + 2 * w + 1] = ctx->tc_m[w] ? 128 : ctx->cfgm32[w].rpc;
    }
  }
  return FETI_OK;
}

feti_status feti_kernel_stats(const feti_ctx* ctx, double* gemv_ms, double* gemv_bytes, double* gemv_flops) {
  if (!ctx) return FETI_ERR_INVALID_ARG;
  if (gemv_ms) *gemv_ms = ctx->gemv_ms;
  if (gemv_bytes) *gemv_bytes = ctx->gemv_bytes;
  if (gemv_flops) *gemv_flops = ctx->gemv_flops;
  return FETI_OK;
}

const char* feti_last_error(const feti_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

feti_status feti_get_refinement(const feti_ctx* ctx, int32_t* steps, double* residual) {
  if (!ctx) return FETI_ERR_INVALID_ARG;
  if (steps) *steps = ctx->refine_steps;
  if (residual) *residual = ctx->refine_res;
  return FETI_OK;
}

feti_status feti_set_spin_timeout(feti_ctx* ctx, uint64_t spin_timeout_ns) {
  if (!ctx) return FETI_ERR_INVALID_ARG;
  if (!ctx->d_spin) return fail(ctx, FETI_ERR_STATE, "context not set up");
  return set_spin_budget(ctx, spin_timeout_ns);
}

void feti_destroy(feti_ctx* ctx) {
  if (!ctx) return;
  if (ctx->coarse_pending && ctx->stream2) cudaStreamSynchronize(ctx->stream2);
  if (ctx->pcg_graph) cudaGraphExecDestroy(ctx->pcg_graph);
  if (ctx->dual_graph) cudaGraphExecDestroy(ctx->dual_graph);
  for (auto ev : ctx->dual_events) cudaEventDestroy(ev);
  for (auto ev : ctx->elem_ev)
    if (ev) cudaEventDestroy(ev);
  if (ctx->pcgm_graph) cudaGraphExecDestroy(ctx->pcgm_graph);
  if (ctx->dualm_graph) cudaGraphExecDestroy(ctx->dualm_graph);
  for (auto ev : ctx->dualm_events) cudaEventDestroy(ev);
  if (ctx->hm_sc) cudaFreeHost(ctx->hm_sc);
  for (auto& b : ctx->bufs) cudaFree(b.p);
  if (ctx->h_sc) cudaFreeHost(ctx->h_sc);
  if (ctx->h_status) cudaFreeHost(ctx->h_status);
  if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
  for (void* q : ctx->coarse_ws)
    if (q) cudaFree(q);
  if (ctx->stream2) cudaStreamDestroy(ctx->stream2);
  if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
  if (ctx->ev_coarse) cudaEventDestroy(ctx->ev_coarse);
  delete ctx;
}

}  // extern "C"
