// Symbolic analysis of the sparse coarse problem G^T G (Sec. 4.3, the
// projection P = I - G (G^T G)^-1 G^T).
//
// G = [B_1 R_1, ..., B_p R_p] has one block of columns per subdomain with a
// kernel, so G^T G is block-sparse: block (i, j) is nonzero only where
// subdomains i and j share a Lagrange multiplier.  Its Cholesky factor is
// computed over supernodes of a nested-dissection order of that subdomain
// graph:
//   * the graph is split recursively by a level set of a breadth-first search
//     from a pseudo-peripheral subdomain (the separator), parts first, the
//     separator last; parts of at most leaf_max subdomains and separators
//     become supernodes, each with a dense diagonal block;
//   * the rows of a supernode's factor panel are its neighbours ordered after
//     it plus the panels of its children (the fill of the elimination), the
//     parent is the supernode of the first panel row (the assembly tree);
//   * the front of a supernode lists its own columns, then its panel rows,
//     each as natural coarse indices, and every child's panel rows map into it
//     by increasing front index (multifrontal extend-add);
//   * the triangular sweeps of each solve are a task graph in ticket order
//     (tasks wait only on tasks with lower tickets): per assembly level the
//     forward tasks (y = L_ss^-1 t and the update vector passed to the
//     parent), and in reverse level order the backward tasks
//     (t = y - L_ps^T x_panel and x = L_ss^-T t); small fronts do a whole
//     sweep in one task, large ones split each step into row tasks.
// Pure host code, no CUDA calls.
#include "feti_internal.h"

#include <algorithm>
#include <cstdio>
#include <numeric>
#include <vector>

namespace feti {
namespace {

struct Nd {
  const std::vector<std::vector<int32_t>>& adj;
  int leaf_max;
  std::vector<int32_t> stamp;  // set membership by stamp value
  std::vector<int32_t> lev;
  int32_t cur = 0;
  std::vector<int32_t> order;                  // output node sequence
  std::vector<std::pair<int32_t, int32_t>> sn;  // supernode ranges in order

  Nd(const std::vector<std::vector<int32_t>>& a, int lm)
      : adj(a), leaf_max(lm), stamp(a.size(), -1), lev(a.size(), -1) {}

  void emit(const std::vector<int32_t>& s) {
    if (s.empty()) return;
    const int32_t b = (int32_t)order.size();
    order.insert(order.end(), s.begin(), s.end());
    sn.emplace_back(b, (int32_t)order.size());
  }

  // breadth-first levels from root over the nodes stamped st; returns the
  // level sets (lev[] written for the reached nodes)
  std::vector<std::vector<int32_t>> bfs(int32_t root, int32_t st) {
    std::vector<std::vector<int32_t>> L(1, std::vector<int32_t>(1, root));
    const int32_t mark = ++cur;  // visited marks live in lev as -(mark)
    lev[root] = -mark;
    for (;;) {
      std::vector<int32_t> nxt;
      for (int32_t v : L.back())
        for (int32_t u : adj[v])
          if (stamp[u] == st && lev[u] != -mark) {
            lev[u] = -mark;
            nxt.push_back(u);
          }
      if (nxt.empty()) break;
      std::sort(nxt.begin(), nxt.end());
      L.push_back(std::move(nxt));
    }
    return L;
  }

  int32_t degree_in(int32_t v, int32_t st) const {
    int32_t d = 0;
    for (int32_t u : adj[v]) d += stamp[u] == st;
    return d;
  }

  void run(std::vector<int32_t> S) {
    std::sort(S.begin(), S.end());
    if ((int)S.size() <= leaf_max) {
      emit(S);
      return;
    }
    const int32_t st = ++cur;
    for (int32_t v : S) stamp[v] = st;
    // connected components are ordered one after the other
    std::vector<std::vector<int32_t>> L = bfs(S[0], st);
    size_t reached = 0;
    for (auto& l : L) reached += l.size();
    if (reached < S.size()) {
      std::vector<int32_t> comp, rest;
      const int32_t mark = lev[S[0]];
      for (int32_t v : S) (lev[v] == mark ? comp : rest).push_back(v);
      run(comp);
      run(rest);
      return;
    }
    // pseudo-peripheral root: restart from a lowest-degree node of the last
    // level while the eccentricity grows
    int32_t root = S[0];
    for (int round = 0; round < 6; ++round) {
      const std::vector<int32_t>& last = L.back();
      int32_t cand = last[0], cd = degree_in(last[0], st);
      for (int32_t v : last) {
        const int32_t d = degree_in(v, st);
        if (d < cd) { cd = d; cand = v; }
      }
      std::vector<std::vector<int32_t>> L2 = bfs(cand, st);
      if (L2.size() <= L.size() && round > 0) break;
      L = std::move(L2);
      root = cand;
    }
    (void)root;
    const int m = (int)L.size() - 1;
    if (m < 2) {  // no level set separates two non-empty parts
      emit(S);
      return;
    }
    // separator level: the first level at which half of the nodes are reached
    size_t cum = 0;
    int ell = 1;
    for (int l = 0; l <= m; ++l) {
      cum += L[l].size();
      if (2 * cum >= S.size()) { ell = l; break; }
    }
    ell = std::min(std::max(ell, 1), m - 1);
    std::vector<int32_t> A, B, sep;
    for (int l = 0; l < ell; ++l) A.insert(A.end(), L[l].begin(), L[l].end());
    for (int l = ell + 1; l <= m; ++l) B.insert(B.end(), L[l].begin(), L[l].end());
    // thin the separator: a node with no neighbour beyond it joins A
    const int32_t sb = ++cur;
    for (int32_t v : B) stamp[v] = sb;
    for (int32_t v : L[ell]) {
      bool nb = false;
      for (int32_t u : adj[v]) nb |= stamp[u] == sb;
      (nb ? sep : A).push_back(v);
    }
    run(A);
    run(B);
    std::sort(sep.begin(), sep.end());
    emit(sep);
  }
};

}  // namespace

bool coarse_plan(int P, const int32_t* k, const int32_t* coff, const std::vector<int32_t>& gi,
                 const std::vector<int32_t>& gj, int leaf_max, int task_bytes, int merge_bytes, CoarsePlan* out,
                 std::string* err) {
  CoarsePlan& cp = *out;
  cp = CoarsePlan{};
  // graph over the subdomains with a kernel
  std::vector<std::vector<int32_t>> adj(P);
  for (size_t b = 0; b < gi.size(); ++b)
    if (gi[b] != gj[b]) {
      adj[gi[b]].push_back(gj[b]);
      adj[gj[b]].push_back(gi[b]);
    }
  std::vector<int32_t> nodes;
  for (int s = 0; s < P; ++s)
    if (k[s] > 0) {
      nodes.push_back(s);
      std::sort(adj[s].begin(), adj[s].end());
      adj[s].erase(std::unique(adj[s].begin(), adj[s].end()), adj[s].end());
    }
  if (nodes.empty()) return true;
  Nd nd(adj, std::max(1, leaf_max));
  nd.run(nodes);
  const int n = (int)nd.order.size();
  const int S = (int)nd.sn.size();
  std::vector<int32_t> pos(P, -1), sup(n);
  for (int x = 0; x < n; ++x) pos[nd.order[x]] = x;
  for (int s = 0; s < S; ++s)
    for (int x = nd.sn[s].first; x < nd.sn[s].second; ++x) sup[x] = s;
  // column offset of each node inside its supernode's own columns
  std::vector<int32_t> own_off(n);
  cp.fronts.resize(S);
  for (int s = 0; s < S; ++s) {
    int32_t w = 0;
    for (int x = nd.sn[s].first; x < nd.sn[s].second; ++x) {
      own_off[x] = w;
      w += k[nd.order[x]];
    }
    cp.fronts[s].w = w;
  }
  // panels (node positions after the supernode), parents, children
  std::vector<std::vector<int32_t>> panel(S), kids(S);
  for (int s = 0; s < S; ++s) {
    const int32_t b = nd.sn[s].first, e = nd.sn[s].second;
    std::vector<int32_t>& pr = panel[s];
    for (int x = b; x < e; ++x)
      for (int32_t u : adj[nd.order[x]]) {
        const int32_t y = pos[u];
        if (y >= e) pr.push_back(y);
        else if (y < b && sup[y] >= s) {
          *err = "coarse ordering: neighbour ordered before its supernode";
          return false;
        }
      }
    for (int32_t c : kids[s])
      for (int32_t y : panel[c]) {
        if (y < b) {
          *err = "coarse ordering: child panel row before its parent";
          return false;
        }
        if (y >= e) pr.push_back(y);
      }
    std::sort(pr.begin(), pr.end());
    pr.erase(std::unique(pr.begin(), pr.end()), pr.end());
    cp.fronts[s].parent = pr.empty() ? -1 : sup[pr[0]];
    if (!pr.empty()) kids[cp.fronts[s].parent].push_back(s);
  }
  // levels (height in the assembly tree), front index data
  int64_t ws = 0, nD = 0, nL = 0;
  int32_t nout = 0;
  cp.max_children = 0;
  for (int s = 0; s < S; ++s) {
    CoarseFront& F = cp.fronts[s];
    int32_t lv = 0;
    for (int32_t c : kids[s]) lv = std::max(lv, cp.fronts[c].level + 1);
    F.level = lv;
    F.nat = (int32_t)cp.nat.size();
    for (int x = nd.sn[s].first; x < nd.sn[s].second; ++x) {
      const int32_t v = nd.order[x];
      for (int a = 0; a < k[v]; ++a) cp.nat.push_back(coff[v] + a);
    }
    int32_t p = 0;
    for (int32_t y : panel[s]) {
      const int32_t v = nd.order[y];
      for (int a = 0; a < k[v]; ++a) cp.nat.push_back(coff[v] + a);
      p += k[v];
    }
    F.p = p;
    const int64_t f = (int64_t)F.w + p;
    F.off = ws;
    ws += (f + F.w) * f;
    F.doff = nD;
    nD += 2 * (int64_t)F.w * F.w;
    F.loff = nL;
    nL += 2 * (int64_t)F.w * p;
    F.out = nout;
    nout += p;
    cp.max_w = std::max(cp.max_w, F.w);
    cp.max_p = std::max(cp.max_p, p);
    cp.max_children = std::max(cp.max_children, (int)kids[s].size());
    cp.height = std::max(cp.height, lv + 1);
  }
  cp.ws = ws;
  cp.nD = nD;
  cp.nL = nL;
  cp.n_out = nout;
  // children with their index maps into the parent's front
  for (int s = 0; s < S; ++s) {
    CoarseFront& F = cp.fronts[s];
    F.ch0 = (int32_t)cp.child.size();
    const int32_t b = nd.sn[s].first, e = nd.sn[s].second;
    // panel node -> first front row
    std::vector<int32_t> prow(panel[s].size());
    {
      int32_t r = F.w;
      for (size_t q = 0; q < panel[s].size(); ++q) {
        prow[q] = r;
        r += k[nd.order[panel[s][q]]];
      }
    }
    for (int32_t c : kids[s]) {
      CoarseChild ch{};
      ch.c = c;
      ch.map = (int32_t)cp.map.size();
      int32_t n_own = 0;
      for (int32_t y : panel[c]) {
        int32_t r0;
        if (y >= b && y < e) {
          r0 = own_off[y];
        } else {
          auto it = std::lower_bound(panel[s].begin(), panel[s].end(), y);
          if (it == panel[s].end() || *it != y) {
            *err = "coarse ordering: child panel row missing from the parent front";
            return false;
          }
          r0 = prow[it - panel[s].begin()];
        }
        for (int a = 0; a < k[nd.order[y]]; ++a) {
          cp.map.push_back(r0 + a);
          if (r0 + a < F.w) ++n_own;
        }
      }
      ch.n_own = n_own;
      cp.child.push_back(ch);
    }
    F.ch1 = (int32_t)cp.child.size();
    // gather lists: per front row, the children's update rows adding into it
    const int32_t f = F.w + F.p;
    std::vector<int32_t> cnt(f + 1, 0);
    for (int32_t ch = F.ch0; ch < F.ch1; ++ch) {
      const CoarseChild& C = cp.child[ch];
      for (int32_t r = 0; r < cp.fronts[C.c].p; ++r) cnt[cp.map[C.map + r] + 1]++;
    }
    F.gofs = (int32_t)cp.gptr.size();
    const int32_t base = (int32_t)cp.gsrc.size();
    for (int32_t m = 0; m < f; ++m) cnt[m + 1] += cnt[m];
    for (int32_t m = 0; m <= f; ++m) cp.gptr.push_back(base + cnt[m]);
    cp.gsrc.resize(base + cnt[f]);
    for (int32_t ch = F.ch0; ch < F.ch1; ++ch) {
      const CoarseChild& C = cp.child[ch];
      const CoarseFront& Fc = cp.fronts[C.c];
      for (int32_t r = 0; r < Fc.p; ++r) cp.gsrc[base + cnt[cp.map[C.map + r]]++] = Fc.out + r;
    }
  }
  // where each G^T G pair block lands: the front of the earlier node, rows of
  // the later node, columns of the earlier one (lower triangle)
  cp.place.resize(gi.size());
  for (size_t bk = 0; bk < gi.size(); ++bk) {
    const int32_t xi = pos[gi[bk]], xj = pos[gj[bk]];
    const int32_t xa = std::min(xi, xj), xb = std::max(xi, xj);
    const int s = sup[xa];
    const CoarseFront& F = cp.fronts[s];
    CoarsePlace pl{};
    pl.off = F.off;
    pl.ld = F.w + F.p;
    pl.col0 = own_off[xa];
    if (sup[xb] == s) {
      pl.row0 = own_off[xb];
    } else {
      auto it = std::lower_bound(panel[s].begin(), panel[s].end(), xb);
      if (it == panel[s].end() || *it != xb) {
        *err = "coarse ordering: coupled block outside the front";
        return false;
      }
      int32_t r = F.w;
      for (auto q = panel[s].begin(); q != it; ++q) r += k[nd.order[*q]];
      pl.row0 = r;
    }
    // the kernel computes the block with gi's columns as rows; swap when gi
    // is the earlier node (its columns are the front's columns)
    pl.swap = (xi < xj) ? 1 : 0;
    cp.place[bk] = pl;
  }
  // level lists
  cp.level_fronts.assign(cp.height, {});
  for (int s = 0; s < S; ++s) cp.level_fronts[cp.fronts[s].level].push_back(s);
  // task graph.  A front whose whole factor (L_ss^-1 and L_ps, or their
  // transposes) fits in merge_bytes runs each sweep as one task (kind 4
  // forward, 5 backward); larger fronts split each sweep into row tasks of
  // about task_bytes of matrix (kinds 0, 1 forward; 2, 3 backward).  Every
  // task must fit in shared memory with kMaxRhs vectors.
  const int64_t smem_cap = kCoarseSmemDoubles;
  auto slab_of = [&](const CoarseFront& F, int kind, int64_t r0, int64_t r1) -> int64_t {
    const int64_t w = F.w, p = F.p, nr = r1 - r0;
    switch (kind) {
      case 0: return nr * coarse_odd(r1);
      case 1: return nr * coarse_odd(w);
      case 2: return nr * coarse_odd(p);
      case 3: return nr * coarse_odd(w - r0);
      default: return w * coarse_odd(w) + (kind == 4 ? p * coarse_odd(w) : w * coarse_odd(p));
    }
  };
  auto vec_of = [&](const CoarseFront& F, int kind, int64_t r0, int64_t r1) -> int64_t {
    const int64_t w = F.w, p = F.p;
    switch (kind) {
      case 0: return r1;
      case 1: return w + (r1 - r0);
      case 2: return p;
      case 3: return w - r0;
      default: return 2 * w + p;
    }
  };
  // gather rows of a task: front rows [g0, g1) whose children's update rows it adds
  auto grows = [&](const CoarseFront& F, int kind, int64_t r0, int64_t r1, int64_t* g0, int64_t* g1) {
    *g0 = 0;
    *g1 = 0;
    if (kind == 0) { *g1 = r1; }
    else if (kind == 1) { *g0 = F.w + r0; *g1 = F.w + r1; }
    else if (kind == 4) { *g1 = F.w + F.p; }
  };
  // index words staged in shared memory: natural indices of the front, then
  // the gather pointers and sources of the task's rows (in doubles, rounded up)
  auto ints_of = [&](const CoarseFront& F, int kind, int64_t r0, int64_t r1) -> int64_t {
    int64_t g0, g1;
    grows(F, kind, r0, r1, &g0, &g1);
    int64_t n = F.w + F.p;
    if (g1 > g0) n += (g1 - g0 + 1) + (cp.gptr[F.gofs + g1] - cp.gptr[F.gofs + g0]);
    return (n + 1) / 2;
  };
  auto fits = [&](const CoarseFront& F, int kind, int64_t r0, int64_t r1) {
    return slab_of(F, kind, r0, r1) + vec_of(F, kind, r0, r1) * kMaxRhs + ints_of(F, kind, r0, r1) <= smem_cap;
  };
  auto rows_per = [&](int64_t width, int32_t rows) {
    const int64_t r = std::max<int64_t>(8, task_bytes / std::max<int64_t>(8 * width, 1));
    return (int32_t)std::min<int64_t>(std::max<int32_t>(rows, 1), (r + 7) / 8 * 8);
  };
  std::vector<char> merged(S, 0);
  for (int s = 0; s < S; ++s) {
    const int64_t w = cp.fronts[s].w, p = cp.fronts[s].p;
    merged[s] = 8 * w * (w + p) <= merge_bytes && fits(cp.fronts[s], 4, 0, 1) && fits(cp.fronts[s], 5, 0, 1);
  }
  std::vector<int32_t> first(6 * (size_t)S, 0), count(6 * (size_t)S, 0);
  bool too_big = false;
  auto add_tasks = [&](int s, int kind, int32_t rows, int32_t rpt) {
    const CoarseFront& F = cp.fronts[s];
    first[6 * s + kind] = (int32_t)cp.tasks.size();
    for (int32_t r0 = 0; r0 < rows;) {
      int32_t r1 = std::min(rows, r0 + rpt);
      while (r1 > r0 + 1 && !fits(F, kind, r0, r1)) r1 = r0 + (r1 - r0) / 2;
      if (!fits(F, kind, r0, r1)) too_big = true;
      CoarseTask t{};
      t.s = s;
      t.kind = kind;
      t.r0 = r0;
      t.r1 = r1;
      cp.tasks.push_back(t);
      r0 = r1;
    }
    count[6 * s + kind] = (int32_t)cp.tasks.size() - first[6 * s + kind];
  };
  for (int l = 0; l < cp.height; ++l) {
    for (int32_t s : cp.level_fronts[l]) {
      const CoarseFront& F = cp.fronts[s];
      if (merged[s]) add_tasks(s, 4, 1, 1);
      else add_tasks(s, 0, F.w, rows_per(F.w, F.w));
    }
    for (int32_t s : cp.level_fronts[l])
      if (!merged[s]) add_tasks(s, 1, cp.fronts[s].p, rows_per(cp.fronts[s].w, cp.fronts[s].p));
  }
  for (int l = cp.height - 1; l >= 0; --l) {
    for (int32_t s : cp.level_fronts[l]) {
      const CoarseFront& F = cp.fronts[s];
      if (merged[s]) add_tasks(s, 5, 1, 1);
      else add_tasks(s, 2, F.w, rows_per(F.p, F.w));
    }
    for (int32_t s : cp.level_fronts[l])
      if (!merged[s]) add_tasks(s, 3, cp.fronts[s].w, rows_per(cp.fronts[s].w, cp.fronts[s].w));
  }
  if (too_big) {
    *err = "coarse sweeps: a front's panel is too large for shared memory";
    return false;
  }
  auto dep = [&](CoarseTask& t, int s, int kind) {
    if (count[6 * s + kind] == 0) return;
    cp.dep.push_back(first[6 * s + kind]);
    cp.dep.push_back(count[6 * s + kind]);
    t.dep1 += 1;
  };
  // the tasks that complete a front's forward (update vector) and backward (x) sweep
  auto fwd_done = [&](CoarseTask& t, int s) { dep(t, s, merged[s] ? 4 : (cp.fronts[s].p > 0 ? 1 : 0)); };
  auto bwd_done = [&](CoarseTask& t, int s) { dep(t, s, merged[s] ? 5 : 3); };
  cp.smem1 = 1;
  cp.smem16 = 1;
  for (size_t q = 0; q < cp.tasks.size(); ++q) {
    CoarseTask& t = cp.tasks[q];
    const CoarseFront& F = cp.fronts[t.s];
    t.dep0 = (int32_t)cp.dep.size() / 2;
    t.dep1 = t.dep0;
    switch (t.kind) {
      case 0:
      case 4:
        for (int32_t c = F.ch0; c < F.ch1; ++c) fwd_done(t, cp.child[c].c);
        break;
      case 1: dep(t, t.s, 0); break;
      case 2:
      case 5:
        dep(t, t.s, merged[t.s] ? 4 : 0);
        if (F.parent >= 0) bwd_done(t, F.parent);
        break;
      default: dep(t, t.s, 2); break;
    }
    const int64_t sl = slab_of(F, t.kind, t.r0, t.r1) + ints_of(F, t.kind, t.r0, t.r1);
    const int64_t ve = vec_of(F, t.kind, t.r0, t.r1);
    cp.smem1 = std::max(cp.smem1, sl + ve);
    cp.smem16 = std::max(cp.smem16, sl + ve * kMaxRhs);
    for (int32_t d = t.dep0; d < t.dep1; ++d)
      if (cp.dep[2 * d] + cp.dep[2 * d + 1] > (int32_t)q) {
        *err = "coarse task graph: dependency on a later ticket";
        return false;
      }
  }
  for (int s = 0; s < S; ++s) cp.flops += (double)cp.fronts[s].w * cp.fronts[s].w * (cp.fronts[s].w / 3.0 + cp.fronts[s].p) +
                                          (double)cp.fronts[s].w * cp.fronts[s].p * cp.fronts[s].p;
  return true;
}

}  // namespace feti
