// Symbolic phase of DDPS (host): Fig. 2 steps 1, 3 and 5 on the pattern, plus
// the ordering and layout that the numeric steps 2 and 4 run on.
//
//  * Eq. (1)-(2), Fig. 2 step 1: every stored entry of A is either in a
//    diagonal block A_ii (same block row and block column) or in R.
//  * Fig. 2 step 3 and the Sec. 3 dropping rule: entries of R are kept or
//    dropped (column rule with delta, or the element-wise absolute rule).
//  * Fig. 2 step 5: c = sorted set of the kept columns of R (the nonzero
//    columns of G = D^-1 R~); the reduced system of Fig. 3 (6.2) is indexed
//    by positions in c, and the rows of G^ owned by block i form one range.
//  * Fig. 2 step 2 runs as a multifrontal LU without pivoting.  Each A_ii is
//    ordered by nested dissection of its symmetrised graph (recursive BFS
//    level-structure bisection); every dissection-tree node becomes a front:
//    a dense m x m matrix whose first k rows/columns are the node's pivots
//    and whose last r = m - k rows/columns are the later indices its pivots
//    couple to.  Fronts are grouped by tree depth so that the device can
//    process one depth of all blocks of all systems per launch.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <exception>
#include <mutex>
#include <numeric>
#include <sstream>
#include <system_error>
#include <thread>

#ifdef __linux__
#include <sched.h>
#endif

#include "ddps_internal.h"

namespace ddps {
namespace {

// An error found inside the analysis (also inside a worker thread); its
// message is the analysis' result.
struct AnalyzeError {
  std::string msg;
};

// Host threads of the analysis: DDPS_ANALYZE_THREADS if set (>= 1), else the
// CPUs this process may run on (its affinity mask; the hardware threads where
// that is not available), at most 64.
int analysis_threads() {
  if (const char* s = std::getenv("DDPS_ANALYZE_THREADS")) {
    const int v = std::atoi(s);
    if (v >= 1) return std::min(v, 256);
  }
  int hw = 0;
#ifdef __linux__
  cpu_set_t set;
  CPU_ZERO(&set);
  if (sched_getaffinity(0, sizeof(set), &set) == 0) hw = CPU_COUNT(&set);
#endif
  if (hw <= 0) hw = (int)std::thread::hardware_concurrency();
  return hw <= 0 ? 1 : std::min(hw, 64);
}

// Runs body(i) for every i in [0, count), items handed out in order from a
// counter to the calling thread and up to analysis_threads() - 1 others (if
// a thread cannot be started, the ones running take its share).  Every item
// writes only its own outputs, so the result does not depend on the number
// of threads.  The exception of the lowest failing item is rethrown here.
template <class Body>
void parallel_items(int64_t count, const Body& body) {
  if (count <= 0) return;
  const int nt = (int)std::min<int64_t>(analysis_threads(), count);
  std::atomic<int64_t> next{0};
  std::mutex mu;
  int64_t err_item = -1;
  std::exception_ptr err;
  auto work = [&]() {
    for (;;) {
      const int64_t i = next.fetch_add(1);
      if (i >= count) return;
      try {
        body(i);
      } catch (...) {
        std::lock_guard<std::mutex> lk(mu);
        if (err_item < 0 || i < err_item) {
          err_item = i;
          err = std::current_exception();
        }
      }
    }
  };
  std::vector<std::thread> pool;
  for (int t = 1; t < nt; ++t) {
    try {
      pool.emplace_back(work);
    } catch (const std::system_error&) {
      break;
    }
  }
  work();
  for (auto& th : pool) th.join();
  if (err) std::rethrow_exception(err);
}

struct Graph {
  int32_t nv = 0;
  std::vector<int64_t> xadj;
  std::vector<int32_t> adj;
};

// Symmetrised pattern of A(r0:r1, r0:r1) without the diagonal, local indices.
Graph block_graph(const int32_t* rowptr, const int32_t* colind, int64_t r0, int64_t r1) {
  Graph g;
  g.nv = (int32_t)(r1 - r0);
  std::vector<int64_t> deg(g.nv + 1, 0);
  for (int64_t i = r0; i < r1; ++i)
    for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) {
      int64_t j = colind[e];
      if (j >= r0 && j < r1 && j != i) {
        deg[i - r0]++;
        deg[j - r0]++;
      }
    }
  std::vector<int64_t> start(g.nv + 1, 0);
  for (int32_t v = 0; v < g.nv; ++v) start[v + 1] = start[v] + deg[v];
  std::vector<int32_t> tmp(start[g.nv]);
  std::vector<int64_t> fill(start.begin(), start.end() - 1);
  for (int64_t i = r0; i < r1; ++i)
    for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) {
      int64_t j = colind[e];
      if (j >= r0 && j < r1 && j != i) {
        tmp[fill[i - r0]++] = (int32_t)(j - r0);
        tmp[fill[j - r0]++] = (int32_t)(i - r0);
      }
    }
  g.xadj.assign(g.nv + 1, 0);
  g.adj.reserve(tmp.size());
  for (int32_t v = 0; v < g.nv; ++v) {
    auto b = tmp.begin() + start[v], e = tmp.begin() + start[v + 1];
    std::sort(b, e);
    auto u = std::unique(b, e);
    g.adj.insert(g.adj.end(), b, u);
    g.xadj[v + 1] = (int64_t)g.adj.size();
  }
  return g;
}

struct NDNode {
  std::vector<int32_t> piv;       // local (old) vertex ids, ascending
  std::vector<int32_t> children;  // node ids
  int32_t p0 = 0;                 // first new local index of the pivots
  std::vector<int32_t> upd;       // new local indices > pivots coupled to the front
};

class NestedDissection {
 public:
  NestedDissection(const Graph& g, int leaf) : g_(g), leaf_(leaf) {
    inset_.assign(g.nv, 0);
    cstamp_.assign(g.nv, 0);
    vis_.assign(g.nv, 0);
    lev_.assign(g.nv, 0);
  }

  void run() {
    std::vector<int32_t> V(g_.nv);
    std::iota(V.begin(), V.end(), 0);
    build(V, roots);
  }

  std::vector<NDNode> nodes;
  std::vector<int32_t> roots;

 private:
  const Graph& g_;
  int leaf_;
  std::vector<int32_t> inset_, cstamp_, vis_, lev_;
  int32_t set_id_ = 0, bfs_id_ = 0, comp_id_ = 0;

  int32_t make_node(std::vector<int32_t> piv, std::vector<int32_t> ch) {
    std::sort(piv.begin(), piv.end());
    NDNode nd;
    nd.piv = std::move(piv);
    nd.children = std::move(ch);
    nodes.push_back(std::move(nd));
    return (int32_t)nodes.size() - 1;
  }

  // BFS from src inside the current set; returns the visit order, levels in lev_.
  int32_t bfs(int32_t src, int32_t sid, std::vector<int32_t>& order) {
    int32_t bid = ++bfs_id_;
    order.clear();
    order.push_back(src);
    vis_[src] = bid;
    lev_[src] = 0;
    int32_t nlev = 1;
    for (size_t h = 0; h < order.size(); ++h) {
      int32_t v = order[h];
      for (int64_t e = g_.xadj[v]; e < g_.xadj[v + 1]; ++e) {
        int32_t u = g_.adj[e];
        if (inset_[u] == sid && vis_[u] != bid) {
          vis_[u] = bid;
          lev_[u] = lev_[v] + 1;
          nlev = std::max(nlev, lev_[u] + 1);
          order.push_back(u);
        }
      }
    }
    return nlev;
  }

  void build(std::vector<int32_t>& V, std::vector<int32_t>& out) {
    if ((int)V.size() <= leaf_) {
      if (!V.empty()) out.push_back(make_node(V, {}));
      return;
    }
    int32_t sid = ++set_id_;
    for (int32_t v : V) inset_[v] = sid;
    std::vector<int32_t> order;
    // connected components: dissect each large one on its own, pack small ones into leaves
    {
      std::vector<std::vector<int32_t>> comps;
      int32_t cid = ++comp_id_;
      for (int32_t v : V) {
        if (cstamp_[v] == cid) continue;
        bfs(v, sid, order);
        for (int32_t u : order) cstamp_[u] = cid;
        comps.push_back(order);
      }
      if (comps.size() > 1) {
        std::vector<int32_t> pack;
        for (auto& cpt : comps) {
          if ((int)cpt.size() > leaf_) {
            build(cpt, out);
            continue;
          }
          if ((int)(pack.size() + cpt.size()) > leaf_) {
            out.push_back(make_node(pack, {}));
            pack.clear();
          }
          pack.insert(pack.end(), cpt.begin(), cpt.end());
        }
        if (!pack.empty()) out.push_back(make_node(pack, {}));
        return;
      }
    }
    // pseudo-peripheral start vertex (George & Liu)
    auto degree = [&](int32_t v) { return g_.xadj[v + 1] - g_.xadj[v]; };
    int32_t s = V[0];
    for (int32_t v : V)
      if (degree(v) < degree(s)) s = v;
    int32_t nlev = bfs(s, sid, order);
    for (int it = 0; it < 6; ++it) {
      int32_t t = -1;
      for (auto it2 = order.rbegin(); it2 != order.rend() && lev_[*it2] == nlev - 1; ++it2)
        if (t < 0 || degree(*it2) < degree(t)) t = *it2;
      std::vector<int32_t> order2;
      int32_t nlev2 = bfs(t, sid, order2);
      if (nlev2 > nlev) {
        nlev = nlev2;
        order.swap(order2);
      } else {
        bfs(s, sid, order);  // restore lev_ of the kept structure
        break;
      }
      s = t;
    }
    if (nlev < 3) {  // too small a diameter to dissect: one dense front
      out.push_back(make_node(V, {}));
      return;
    }
    std::vector<int64_t> cnt(nlev, 0);
    for (int32_t v : order) cnt[lev_[v]]++;
    // separator level: the median level, kept away from both ends
    int64_t half = (int64_t)V.size() / 2, acc = 0;
    int32_t l = 1;
    for (int32_t q = 0; q < nlev; ++q) {
      if (acc + cnt[q] > half) {
        l = q;
        break;
      }
      acc += cnt[q];
    }
    l = std::max(1, std::min(l, nlev - 2));
    std::vector<int32_t> S, V1, V2;
    for (int32_t v : order) {
      int32_t lv = lev_[v];
      if (lv < l) {
        V1.push_back(v);
      } else if (lv > l) {
        V2.push_back(v);
      } else {
        bool touches_next = false;
        for (int64_t e = g_.xadj[v]; e < g_.xadj[v + 1] && !touches_next; ++e) {
          int32_t u = g_.adj[e];
          touches_next = inset_[u] == sid && lev_[u] == l + 1;
        }
        (touches_next ? S : V1).push_back(v);
      }
    }
    std::vector<int32_t> ch;
    build(V1, ch);
    build(V2, ch);
    out.push_back(make_node(S, ch));
  }
};

}  // namespace

static std::string analyze_impl(int64_t n, int64_t nnz, const int32_t* rowptr,
                                const int32_t* colind, int32_t p, const int64_t* block_ptr,
                                int32_t nsys, const int32_t* sys_block_ptr, const double* values,
                                const ddps_options& opt, Analysis& A) {
  std::ostringstream err;
  if (n <= 0 || nnz < 0 || !rowptr || (nnz > 0 && !colind) || p <= 0 || !block_ptr)
    return "ddps_analyze: invalid sizes or null pattern pointers";
  if (n >= (int64_t)1 << 31 || nnz >= (int64_t)1 << 31)
    return "ddps_analyze: n and nnz must fit in int32";
  if (rowptr[0] != 0 || rowptr[n] != nnz) return "ddps_analyze: rowptr must start at 0 and end at nnz";
  for (int64_t i = 0; i < n; ++i) {
    if (rowptr[i + 1] < rowptr[i]) return "ddps_analyze: rowptr is not monotone";
    for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) {
      if (colind[e] < 0 || colind[e] >= n) return "ddps_analyze: column index out of range";
      if (e > rowptr[i] && colind[e] <= colind[e - 1])
        return "ddps_analyze: columns must be sorted and unique within a row";
    }
  }
  if (block_ptr[0] != 0 || block_ptr[p] != n) return "ddps_analyze: block_ptr must span [0, n]";
  for (int32_t b = 0; b < p; ++b)
    if (block_ptr[b + 1] <= block_ptr[b]) return "ddps_analyze: empty or decreasing block";
  if (nsys <= 0) return "ddps_analyze: nsys must be positive";
  if (opt.drop_mode != DDPS_DROP_NONE && !values)
    return "ddps_analyze: the drop rule needs the values on the host";
  if (opt.drop_mode < 0 || opt.drop_mode > 2) return "ddps_analyze: unknown drop mode";

  A.n = n;
  A.nnz = nnz;
  A.p = p;
  A.nsys = nsys;
  A.block_ptr.assign(block_ptr, block_ptr + p + 1);
  if (sys_block_ptr) {
    A.sys_block_ptr.assign(sys_block_ptr, sys_block_ptr + nsys + 1);
  } else {
    if (nsys != 1) return "ddps_analyze: sys_block_ptr is required when nsys > 1";
    A.sys_block_ptr = {0, p};
  }
  if (A.sys_block_ptr[0] != 0 || A.sys_block_ptr[nsys] != p)
    return "ddps_analyze: sys_block_ptr must span [0, p]";
  for (int32_t s = 0; s < nsys; ++s)
    if (A.sys_block_ptr[s + 1] <= A.sys_block_ptr[s]) return "ddps_analyze: system without blocks";
  A.sys_row_ptr.resize(nsys + 1);
  A.block_sys.resize(p);
  for (int32_t s = 0; s <= nsys; ++s) A.sys_row_ptr[s] = block_ptr[A.sys_block_ptr[s]];
  for (int32_t s = 0; s < nsys; ++s)
    for (int32_t b = A.sys_block_ptr[s]; b < A.sys_block_ptr[s + 1]; ++b) A.block_sys[b] = s;

  // ---- Fig. 2 steps 1 and 3: split and drop -------------------------------
  std::vector<int32_t> row_block(n);
  for (int32_t b = 0; b < p; ++b)
    for (int64_t i = block_ptr[b]; i < block_ptr[b + 1]; ++i) row_block[i] = b;
  std::vector<uint8_t> keep_r(nnz, 0);
  std::vector<uint8_t> is_d(nnz, 0);
  // blocks in parallel: each one sets the flags of its own rows' entries
  parallel_items(p, [&](int64_t bi) {
    const int32_t b = (int32_t)bi;
    int64_t r0 = block_ptr[b], r1 = block_ptr[b + 1];
    int32_t s = A.block_sys[b];
    int64_t s0 = A.sys_row_ptr[s], s1 = A.sys_row_ptr[s + 1];
    std::vector<std::pair<int32_t, double>> colnorm;  // (column, max |r|) for the column rule
    for (int64_t i = r0; i < r1; ++i)
      for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) {
        int64_t j = colind[e];
        if (j >= r0 && j < r1) {
          is_d[e] = 1;
          continue;
        }
        if (j < s0 || j >= s1) {
          std::ostringstream why;
          why << "ddps_analyze: entry (" << i << ", " << j << ") couples two systems";
          throw AnalyzeError{why.str()};
        }
        if (opt.drop_mode == DDPS_DROP_ABS)
          keep_r[e] = std::fabs(values[e]) >= opt.drop_tol;
        else
          keep_r[e] = 1;
        if (opt.drop_mode == DDPS_DROP_COLUMN) colnorm.push_back({(int32_t)j, std::fabs(values[e])});
      }
    if (opt.drop_mode == DDPS_DROP_COLUMN && !colnorm.empty()) {
      std::sort(colnorm.begin(), colnorm.end());
      std::vector<std::pair<int32_t, double>> cmax;
      for (auto& cv : colnorm) {
        if (cmax.empty() || cmax.back().first != cv.first)
          cmax.push_back(cv);
        else
          cmax.back().second = std::max(cmax.back().second, cv.second);
      }
      double mx = 0;
      for (auto& cv : cmax) mx = std::max(mx, cv.second);
      for (int64_t i = r0; i < r1; ++i)
        for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) {
          if (is_d[e]) continue;
          int32_t j = colind[e];
          auto it = std::lower_bound(cmax.begin(), cmax.end(), std::make_pair(j, -1.0));
          keep_r[e] = !(it->second <= opt.drop_tol * mx);
        }
    }
  });

  // ---- Fig. 2 step 5: c ------------------------------------------------------
  std::vector<uint8_t> inc(n, 0);
  for (int64_t e = 0; e < nnz; ++e)
    if (keep_r[e]) inc[colind[e]] = 1;
  std::vector<int32_t> qpos(n, -1);
  for (int64_t j = 0; j < n; ++j)
    if (inc[j]) {
      qpos[j] = (int32_t)A.c.size();
      A.c.push_back(j);
    }
  const int64_t m = (int64_t)A.c.size();
  A.sys_c_ptr.resize(nsys + 1);
  for (int32_t s = 0; s <= nsys; ++s)
    A.sys_c_ptr[s] = std::lower_bound(A.c.begin(), A.c.end(), A.sys_row_ptr[s]) - A.c.begin();

  // ---- Fig. 2 step 2 structure: nested dissection + multifrontal symbolic ----
  const int leaf = opt.leaf_size > 0 ? opt.leaf_size : 64;
  A.perm.assign(n, 0);
  A.iperm.assign(n, 0);
  struct FrontTmp {
    int32_t k;
    int64_t row0;
    std::vector<int32_t> upd;  // global new indices
    std::vector<int32_t> ch;
    int32_t parent = -1;
    int32_t block;
  };
  std::vector<FrontTmp> F;
  std::vector<int32_t> roots;
  A.ilu = opt.factor_kind == DDPS_FACTOR_ILU0;
  if (A.ilu) {
    // ILU(0) keeps every block in its own row order: no dissection, no fronts
    for (int64_t i = 0; i < n; ++i) A.perm[i] = A.iperm[i] = (int32_t)i;
  }
  // The blocks are ordered and analysed independently (Sec. 3: each diagonal
  // block is factored on its own), in parallel: a block writes only its own
  // rows of perm / iperm and its own list of fronts, numbered from 0 in
  // postorder; the lists are then appended in block order.
  const int32_t nblk = A.ilu ? 0 : p;
  std::vector<std::vector<FrontTmp>> BF(nblk);
  std::vector<std::vector<int32_t>> BR(nblk);
  parallel_items(nblk, [&](int64_t bi) {
    const int32_t b = (int32_t)bi;
    const int64_t r0 = block_ptr[b], r1 = block_ptr[b + 1];
    std::vector<FrontTmp>& Fb = BF[b];
    Graph g = block_graph(rowptr, colind, r0, r1);
    NestedDissection nd(g, leaf);
    nd.run();
    // postorder numbering: children first, then the node's pivots
    int32_t next = 0;
    std::vector<int32_t> node2front(nd.nodes.size(), -1);
    std::vector<std::pair<int32_t, int32_t>> stack;
    for (int32_t root : nd.roots) {
      stack.push_back({root, 0});
      while (!stack.empty()) {
        auto& top = stack.back();
        NDNode& nd_ = nd.nodes[top.first];
        if (top.second < (int32_t)nd_.children.size()) {
          int32_t c = nd_.children[top.second++];
          stack.push_back({c, 0});
          continue;
        }
        nd_.p0 = next;
        for (int32_t v : nd_.piv) {
          A.perm[r0 + next] = (int32_t)(r0 + v);
          A.iperm[r0 + v] = (int32_t)(r0 + next);
          ++next;
        }
        FrontTmp ft;
        ft.k = (int32_t)nd_.piv.size();
        ft.row0 = r0 + nd_.p0;
        ft.block = b;
        for (int32_t c : nd_.children) ft.ch.push_back(node2front[c]);
        node2front[top.first] = (int32_t)Fb.size();
        Fb.push_back(std::move(ft));
        stack.pop_back();
      }
    }
    if (next != g.nv) throw AnalyzeError{"ddps_analyze: internal error in the dissection numbering"};
    for (int32_t root : nd.roots) BR[b].push_back(node2front[root]);
    // symbolic factorisation, bottom-up (the fronts are in postorder); mark[u
    // - r0] holds the last front that listed row u
    std::vector<int32_t> mark(g.nv, -1);
    for (int32_t f = 0; f < (int32_t)Fb.size(); ++f) {
      FrontTmp& ft = Fb[f];
      const int64_t end = ft.row0 + ft.k;
      std::vector<int32_t> upd;
      for (int64_t q = ft.row0; q < end; ++q) {
        int64_t vloc = A.perm[q] - r0;
        for (int64_t e = g.xadj[vloc]; e < g.xadj[vloc + 1]; ++e) {
          int32_t u = A.iperm[r0 + g.adj[e]];
          if (u >= end && mark[u - r0] != f) {
            mark[u - r0] = f;
            upd.push_back(u);
          }
        }
      }
      for (int32_t c : ft.ch) {
        Fb[c].parent = f;
        for (int32_t u : Fb[c].upd)
          if (u >= end && mark[u - r0] != f) {
            mark[u - r0] = f;
            upd.push_back(u);
          }
      }
      std::sort(upd.begin(), upd.end());
      ft.upd = std::move(upd);
    }
  });
  for (int32_t b = 0; b < nblk; ++b) {
    const int32_t base = (int32_t)F.size();
    for (FrontTmp& ft : BF[b]) {
      for (int32_t& c : ft.ch) c += base;
      if (ft.parent >= 0) ft.parent += base;
      F.push_back(std::move(ft));
    }
    for (int32_t r : BR[b]) roots.push_back(r + base);
    std::vector<FrontTmp>().swap(BF[b]);
  }
  std::vector<int32_t> owner(n, -1);  // new index -> front id
  for (int32_t f = 0; f < (int32_t)F.size(); ++f)
    for (int64_t q = F[f].row0; q < F[f].row0 + F[f].k; ++q) owner[q] = (int32_t)f;

  // depths, levels, storage offsets
  const int32_t nf = (int32_t)F.size();
  A.f_k.resize(nf);
  A.f_m.resize(nf);
  A.f_block.resize(nf);
  A.f_parent.resize(nf);
  A.f_depth.assign(nf, 0);
  A.f_cbeg.resize(nf);
  A.f_cend.resize(nf);
  A.f_row0.resize(nf);
  A.f_arena.resize(nf);
  A.f_idx.resize(nf);
  A.f_upd.resize(nf);
  A.f_rel.assign(nf, -1);
  // fronts were created in postorder, so parents come after children: walk backwards
  int32_t maxdepth = 0;
  for (int32_t f = nf - 1; f >= 0; --f) {
    if (F[f].parent >= 0) A.f_depth[f] = A.f_depth[F[f].parent] + 1;
    maxdepth = std::max(maxdepth, A.f_depth[f]);
  }
  A.nlevels = maxdepth + 1;
  int64_t arena = 0, updsz = 0, idxsz = 0;
  A.max_children = 1;
  for (int32_t f = 0; f < nf; ++f) {
    const FrontTmp& ft = F[f];
    int32_t r = (int32_t)ft.upd.size();
    int32_t mm = ft.k + r;
    A.f_k[f] = ft.k;
    A.f_m[f] = mm;
    A.f_block[f] = ft.block;
    A.f_parent[f] = ft.parent;
    A.f_row0[f] = ft.row0;
    A.f_arena[f] = arena;
    arena += (int64_t)mm * mm;
    A.f_idx[f] = idxsz;
    idxsz += mm;
    A.f_upd[f] = updsz;
    updsz += r;
    A.f_cbeg[f] = (int32_t)A.children.size();
    for (int32_t c : ft.ch) A.children.push_back(c);
    A.f_cend[f] = (int32_t)A.children.size();
    A.max_children = std::max<int32_t>(A.max_children, (int32_t)ft.ch.size());
    A.max_front = std::max<int64_t>(A.max_front, mm);
    const double kk = ft.k, md = mm;
    A.factor_flops += 2.0 * (kk * md * md - kk * kk * md + kk * kk * kk / 3.0);
    A.factor_lu_entries += (int64_t)ft.k * (2 * (int64_t)mm - ft.k);
  }
  A.arena_size = arena;
  A.upd_size = updsz;
  A.idx.resize(idxsz);
  for (int32_t f = 0; f < nf; ++f) {
    int64_t o = A.f_idx[f];
    for (int32_t i = 0; i < F[f].k; ++i) A.idx[o + i] = (int32_t)(F[f].row0 + i);
    for (size_t i = 0; i < F[f].upd.size(); ++i) A.idx[o + F[f].k + i] = F[f].upd[i];
  }
  // relative positions of each child's update rows inside its parent's front
  // (offsets first, then the fronts in parallel chunks)
  int64_t nrel = 0;
  for (int32_t f = 0; f < nf; ++f) {
    if (F[f].parent < 0) {
      if (!F[f].upd.empty()) return "ddps_analyze: internal error (root front with update rows)";
      continue;
    }
    A.f_rel[f] = nrel;
    nrel += (int64_t)F[f].upd.size();
  }
  A.rel.resize(nrel);
  constexpr int32_t kFrontChunk = 256;
  parallel_items((nf + kFrontChunk - 1) / kFrontChunk, [&](int64_t it) {
    const int32_t f1 = (int32_t)std::min<int64_t>(nf, (it + 1) * kFrontChunk);
    for (int32_t f = (int32_t)it * kFrontChunk; f < f1; ++f) {
      if (F[f].parent < 0) continue;
      const FrontTmp& pf = F[F[f].parent];
      int32_t* out = A.rel.data() + A.f_rel[f];
      for (int32_t u : F[f].upd) {
        int64_t pos;
        if (u >= pf.row0 && u < pf.row0 + pf.k) {
          pos = u - pf.row0;
        } else {
          auto it2 = std::lower_bound(pf.upd.begin(), pf.upd.end(), u);
          if (it2 == pf.upd.end() || *it2 != u)
            throw AnalyzeError{"ddps_analyze: internal error (update row not in parent)"};
          pos = pf.k + (it2 - pf.upd.begin());
        }
        *out++ = (int32_t)pos;
      }
    }
  });
  // level lists and the extend-add schedule
  A.level_ptr.assign(A.nlevels + 1, 0);
  for (int32_t f = 0; f < nf; ++f) A.level_ptr[A.f_depth[f] + 1]++;
  for (int32_t d = 0; d < A.nlevels; ++d) A.level_ptr[d + 1] += A.level_ptr[d];
  A.level_fronts.resize(nf);
  {
    std::vector<int32_t> fill(A.level_ptr.begin(), A.level_ptr.end() - 1);
    for (int32_t f = 0; f < nf; ++f) A.level_fronts[fill[A.f_depth[f]]++] = f;
  }
  const int32_t S = A.max_children;
  A.ea_ptr.assign((int64_t)A.nlevels * S + 1, 0);
  {
    std::vector<std::vector<int32_t>> lists((int64_t)A.nlevels * S);
    for (int32_t f = 0; f < nf; ++f)
      for (int32_t s = 0; s < (int32_t)F[f].ch.size(); ++s)
        lists[(int64_t)A.f_depth[f] * S + s].push_back(F[f].ch[s]);
    for (size_t q = 0; q < lists.size(); ++q) {
      A.ea_ptr[q + 1] = A.ea_ptr[q] + (int32_t)lists[q].size();
      A.ea_list.insert(A.ea_list.end(), lists[q].begin(), lists[q].end());
    }
  }

  // ---- assembly map: D entries -> front positions; R entries -> -1 ----------
  A.amap.assign(nnz, -1);
  if (A.ilu) {
    // ILU(0): the D entries of each row, in order, form the factor's CSR; the
    // map sends entry e to its position there
    A.il_rp.assign(n + 1, 0);
    A.il_diag.assign(n, -1);
    A.il_row_block.assign(n, 0);
    for (int64_t i = 0; i < n; ++i) {
      A.il_row_block[i] = row_block[i];
      for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) {
        if (!is_d[e]) continue;
        if (colind[e] == i) A.il_diag[i] = (int32_t)A.il_col.size();
        A.amap[e] = (int64_t)A.il_col.size();
        A.il_col.push_back(colind[e]);
      }
      A.il_rp[i + 1] = (int32_t)A.il_col.size();
      if (A.il_diag[i] < 0) {
        err << "ddps_analyze: ILU(0) needs every diagonal entry stored (row " << i << ")";
        return err.str();
      }
    }
    // levels: L dependencies (k < i) forward, U dependencies (j > i) backward
    std::vector<int32_t> lf(n, 0), lb(n, 0);
    int32_t nlf = 0, nlb = 0;
    for (int64_t i = 0; i < n; ++i) {
      for (int32_t e = A.il_rp[i]; e < A.il_diag[i]; ++e) lf[i] = std::max(lf[i], lf[A.il_col[e]] + 1);
      nlf = std::max(nlf, lf[i] + 1);
    }
    for (int64_t i = n - 1; i >= 0; --i) {
      for (int32_t e = A.il_diag[i] + 1; e < A.il_rp[i + 1]; ++e)
        lb[i] = std::max(lb[i], lb[A.il_col[e]] + 1);
      nlb = std::max(nlb, lb[i] + 1);
    }
    auto bucket = [&](const std::vector<int32_t>& lev, int32_t nl, std::vector<int32_t>& rows,
                      std::vector<int32_t>& ptr) {
      ptr.assign(nl + 1, 0);
      for (int64_t i = 0; i < n; ++i) ptr[lev[i] + 1]++;
      for (int32_t l = 0; l < nl; ++l) ptr[l + 1] += ptr[l];
      rows.resize(n);
      std::vector<int32_t> fill(ptr.begin(), ptr.end() - 1);
      for (int64_t i = 0; i < n; ++i) rows[fill[lev[i]]++] = (int32_t)i;
    };
    bucket(lf, nlf, A.il_lf, A.il_lf_ptr);
    bucket(lb, nlb, A.il_lb, A.il_lb_ptr);
    // flops of the factorisation (1 division and 2 per update) and entries a solve streams
    for (int64_t i = 0; i < n; ++i)
      for (int32_t e = A.il_rp[i]; e < A.il_diag[i]; ++e) {
        const int32_t k = A.il_col[e];
        int32_t q = e + 1, upd = 0;
        for (int32_t u = A.il_diag[k] + 1; u < A.il_rp[k + 1]; ++u) {
          while (q < A.il_rp[i + 1] && A.il_col[q] < A.il_col[u]) ++q;
          if (q < A.il_rp[i + 1] && A.il_col[q] == A.il_col[u]) ++upd;
        }
        A.factor_flops += 1.0 + 2.0 * upd;
      }
    A.factor_lu_entries = (int64_t)A.il_col.size();
  }
  constexpr int64_t kRowChunk = 4096;
  parallel_items(A.ilu ? 0 : (n + kRowChunk - 1) / kRowChunk, [&](int64_t it) {
    const int64_t i1 = std::min(n, (it + 1) * kRowChunk);
    for (int64_t i = it * kRowChunk; i < i1; ++i) {
      for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) {
        if (!is_d[e]) continue;
        int32_t a = A.iperm[i], bn = A.iperm[colind[e]];
        int32_t piv = std::min(a, bn);
        int32_t f = owner[piv];
        const FrontTmp& ft = F[f];
        auto posf = [&](int32_t u) -> int64_t {
          if (u < ft.row0 + ft.k) return u - ft.row0;
          auto it2 = std::lower_bound(ft.upd.begin(), ft.upd.end(), u);
          return ft.k + (it2 - ft.upd.begin());
        };
        A.amap[e] = A.f_arena[f] + posf(a) + posf(bn) * (int64_t)A.f_m[f];
      }
    }
  });

  // ---- R~ as CSR with reduced column indices; spike right-hand sides --------
  A.rt_rowptr.assign(n + 1, 0);
  A.gq0.resize(p);
  A.gq1.resize(p);
  A.gcol_ptr.assign(p + 1, 0);
  A.ghat_off.assign(p + 1, 0);
  A.gld.assign(p, 0);
  std::vector<std::vector<int32_t>> bcols(p);
  // stored L and U entries of each block's fronts, summed in front order
  std::vector<double> blk_lu(p, 0.0);
  for (int32_t f = 0; f < nf; ++f)
    blk_lu[A.f_block[f]] += (double)A.f_k[f] * (2.0 * A.f_m[f] - A.f_k[f]);
  // coupling columns of each block (sorted reduced indices), blocks in parallel
  parallel_items(p, [&](int64_t b) {
    std::vector<int32_t>& cols = bcols[b];
    for (int64_t i = block_ptr[b]; i < block_ptr[b + 1]; ++i)
      for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e)
        if (keep_r[e]) cols.push_back(qpos[colind[e]]);
    std::sort(cols.begin(), cols.end());
    cols.erase(std::unique(cols.begin(), cols.end()), cols.end());
  });
  for (int32_t b = 0; b < p; ++b) {
    int64_t r0 = block_ptr[b], r1 = block_ptr[b + 1];
    const std::vector<int32_t>& cols = bcols[b];
    A.gq0[b] = std::lower_bound(A.c.begin(), A.c.end(), r0) - A.c.begin();
    A.gq1[b] = std::lower_bound(A.c.begin(), A.c.end(), r1) - A.c.begin();
    A.gcol_ptr[b + 1] = A.gcol_ptr[b] + (int64_t)cols.size();
    A.gcols.insert(A.gcols.end(), cols.begin(), cols.end());
    // rows are padded to a multiple of 8 entries so that every row starts on a
    // 16-byte boundary in every storage precision
    A.gld[b] = ((int64_t)cols.size() + 7) / 8 * 8;
    A.ghat_off[b + 1] = A.ghat_off[b] + (A.gq1[b] - A.gq0[b]) * A.gld[b];
    A.ghat_entries += (A.gq1[b] - A.gq0[b]) * (int64_t)cols.size();
    A.max_rhs = std::max<int64_t>(A.max_rhs, (int64_t)cols.size());
    const double lu = A.ilu ? (double)(A.il_rp[r1] - A.il_rp[r0]) / 2.0 : blk_lu[b];
    A.spike_flops += 4.0 * lu * (double)cols.size();
  }
  // row pointers first, then the rows in parallel chunks
  for (int64_t i = 0; i < n; ++i) {
    int32_t kept = 0;
    for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) kept += keep_r[e];
    A.rt_rowptr[i + 1] = A.rt_rowptr[i] + kept;
  }
  const int64_t nrt = A.rt_rowptr[n];
  A.rt_col.resize(nrt);
  A.rt_src.resize(nrt);
  A.rt_rhscol.resize(nrt);
  A.rt_rownew.resize(nrt);
  parallel_items((n + kRowChunk - 1) / kRowChunk, [&](int64_t it) {
    const int64_t i1 = std::min(n, (it + 1) * kRowChunk);
    for (int64_t i = it * kRowChunk; i < i1; ++i) {
      const std::vector<int32_t>& cols = bcols[row_block[i]];
      int64_t o = A.rt_rowptr[i];
      for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) {
        if (!keep_r[e]) continue;
        int32_t q = qpos[colind[e]];
        A.rt_col[o] = q;
        A.rt_src[o] = e;
        A.rt_rhscol[o] = (int32_t)(std::lower_bound(cols.begin(), cols.end(), q) - cols.begin());
        A.rt_rownew[o] = A.iperm[i];
        ++o;
      }
    }
  });
  A.c_rownew.resize(m);
  for (int64_t q = 0; q < m; ++q) A.c_rownew[q] = A.iperm[A.c[q]];

  if (opt.verbose) {
    fprintf(stderr,
            "ddps_analyze: n=%lld nnz=%lld p=%d nsys=%d |c|=%lld nnz(R~)=%zu fronts=%d levels=%d "
            "max_front=%lld arena=%lld lu_entries=%lld factor_flops=%.3g ghat=%lld max_rhs=%lld "
            "spike_flops=%.3g\n",
            (long long)n, (long long)nnz, p, nsys, (long long)m, A.rt_col.size(), nf, A.nlevels,
            (long long)A.max_front, (long long)A.arena_size, (long long)A.factor_lu_entries,
            A.factor_flops, (long long)A.ghat_entries, (long long)A.max_rhs, A.spike_flops);
  }
  return "";
}

std::string analyze(int64_t n, int64_t nnz, const int32_t* rowptr, const int32_t* colind,
                    int32_t p, const int64_t* block_ptr, int32_t nsys,
                    const int32_t* sys_block_ptr, const double* values,
                    const ddps_options& opt, Analysis& A) {
  try {
    return analyze_impl(n, nnz, rowptr, colind, p, block_ptr, nsys, sys_block_ptr, values, opt, A);
  } catch (const AnalyzeError& e) {
    return e.msg;
  } catch (const std::bad_alloc&) {
    return "ddps_analyze: host allocation failed";
  } catch (const std::exception& e) {
    return std::string("ddps_analyze: ") + e.what();
  }
}

}  // namespace ddps
