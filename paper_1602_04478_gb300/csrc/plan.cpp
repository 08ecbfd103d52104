// Query validation, decomposition into blocks, and aut(Q).
//
// Decomposition (Section 4.1): repeatedly pick a block of the current query
// -- a leaf edge (a, b) with b of degree one, or an induced cycle with at
// most two boundary nodes -- and contract it:
//   Case 1 (cycle, one boundary node a): drop the rest of the cycle, the
//          block annotates a;
//   Case 2 (cycle, boundary nodes a, b): drop the rest, add edge (a, b)
//          annotated with the block (an existing a-b edge is a cycle edge,
//          since the cycle is induced, so no parallel edge arises);
//   Case 3 (leaf edge (a, b)): drop b, the block annotates a.
// Annotations present on the contracted nodes and edges become the block's
// children.  The loop ends with one node (root = its annotation) or one
// induced cycle holding every remaining node (the root cycle).  Lemma 4.1
// guarantees a block at every step for treewidth-2 queries, so "no block"
// means treewidth above 2.
//
// Several orders are usually possible (Section 5.3).  plan_query explores
// them depth-first (bounded) and keeps the best by: kernels available for
// every block first, then the paper's factors in order -- longest cycle
// block, number of boundary nodes, number of annotations.
#include <algorithm>
#include <cstring>
#include <functional>
#include <map>

#include "cc_internal.h"

namespace cc {
namespace {


struct QS {
  int k = 0;
  uint32_t alive = 0;
  uint32_t adj[kMaxK];
  int node_ann[kMaxK];
  int edge_ann[kMaxK][kMaxK];
  int edge_first[kMaxK][kMaxK];
};

struct Cand {
  bool leaf = false;
  int L = 0;
  int nodes[kMaxK];
  int nb = 0;
  int bd[2] = {-1, -1};
};

int popc(uint32_t x) { return __builtin_popcount(x); }

void init_state(QS &s, int k, const std::vector<std::pair<int, int>> &edges) {
  s.k = k;
  s.alive = (k >= 32) ? 0xFFFFFFFFu : ((1u << k) - 1);
  for (int i = 0; i < kMaxK; i++) {
    s.adj[i] = 0;
    s.node_ann[i] = -1;
    for (int j = 0; j < kMaxK; j++) s.edge_ann[i][j] = -1, s.edge_first[i][j] = -1;
  }
  for (auto &e : edges) {
    s.adj[e.first] |= 1u << e.second;
    s.adj[e.second] |= 1u << e.first;
  }
}

// Simple cycles of the current query; each listed once with its smallest
// node first and nodes[1] < nodes[L-1].
void cycles(const QS &s, std::vector<std::vector<int>> &out) {
  std::vector<int> path;
  std::function<void(int, uint32_t)> ext = [&](int start, uint32_t used) {
    int v = path.back();
    uint32_t nb = s.adj[v] & s.alive;
    for (int w = 0; w < s.k; w++) {
      if (!(nb >> w & 1)) continue;
      if (w == start) {
        if (path.size() >= 3 && path[1] < path.back()) out.push_back(path);
        continue;
      }
      if (w < start || (used >> w & 1)) continue;
      path.push_back(w);
      ext(start, used | (1u << w));
      path.pop_back();
    }
  };
  for (int st = 0; st < s.k; st++) {
    if (!(s.alive >> st & 1)) continue;
    path.assign(1, st);
    ext(st, 1u << st);
  }
}

std::vector<Cand> candidates(const QS &s) {
  std::vector<Cand> c;
  for (int b = 0; b < s.k; b++) {
    if (!(s.alive >> b & 1)) continue;
    uint32_t nb = s.adj[b] & s.alive;
    if (popc(nb) != 1) continue;
    Cand x;
    x.leaf = true;
    x.L = 2;
    x.nodes[0] = __builtin_ctz(nb);
    x.nodes[1] = b;
    x.nb = 1;
    x.bd[0] = x.nodes[0];
    c.push_back(x);
  }
  std::vector<std::vector<int>> cyc;
  cycles(s, cyc);
  for (auto &cy : cyc) {
    int L = (int)cy.size();
    uint32_t cm = 0;
    for (int a : cy) cm |= 1u << a;
    bool induced = true;
    for (int i = 0; i < L && induced; i++) {
      uint32_t want = (1u << cy[(i + 1) % L]) | (1u << cy[(i + L - 1) % L]);
      if ((s.adj[cy[i]] & cm) != want) induced = false;
    }
    if (!induced) continue;
    Cand x;
    x.L = L;
    for (int i = 0; i < L; i++) x.nodes[i] = cy[i];
    for (int a : cy) {
      if (s.adj[a] & s.alive & ~cm) {
        if (x.nb < 2) x.bd[x.nb] = a;
        x.nb++;
      }
    }
    if (x.nb <= 2) c.push_back(x);
  }
  return c;
}

uint32_t stage_sq(const std::vector<Stage> &st, int idx) { return idx < 0 ? 0u : st[idx].sq_mask; }

// Contract candidate x: append its stage and update the state.
void apply(QS &s, const Cand &x, std::vector<Stage> &st, bool is_root) {
  Stage g;
  int id = (int)st.size();
  g.L = x.L;
  for (int i = 0; i < kMaxK; i++) g.node_child[i] = -1, g.edge_child[i] = -1, g.edge_fwd[i] = true;
  for (int i = 0; i < x.L; i++) g.nodes[i] = x.nodes[i];
  g.nb = x.nb;
  g.bd[0] = x.bd[0];
  g.bd[1] = x.bd[1];
  uint32_t sq = 0;
  int ne = x.leaf ? 1 : x.L;
  for (int i = 0; i < x.L; i++) {
    int a = x.nodes[i];
    sq |= 1u << a;
    g.node_child[i] = s.node_ann[a];
    sq |= stage_sq(st, s.node_ann[a]);
  }
  for (int i = 0; i < ne; i++) {
    int a = x.nodes[i], b = x.nodes[(i + 1) % x.L];
    g.edge_child[i] = s.edge_ann[a][b];
    g.edge_fwd[i] = s.edge_first[a][b] == a;
    sq |= stage_sq(st, s.edge_ann[a][b]);
  }
  g.sq_mask = sq;
  g.s = popc(sq);
  if (!x.leaf && x.nb == 2 && !is_root) {
    // Case 2: the table is keyed by data edges only when the boundary nodes
    // are joined by a cycle edge whose images are data edges
    int i0 = 0, i1 = 0;
    for (int i = 0; i < x.L; i++) {
      if (x.nodes[i] == x.bd[0]) i0 = i;
      if (x.nodes[i] == x.bd[1]) i1 = i;
    }
    int e = -1;
    if ((i0 + 1) % x.L == i1) e = i0;
    else if ((i1 + 1) % x.L == i0) e = i1;
    g.pair_out = e < 0 || (g.edge_child[e] >= 0 && st[g.edge_child[e]].pair_out);
  }
  if (x.leaf) g.kind = ST_LEAF;
  else if (x.L == 3) g.kind = ST_TRI;
  else g.kind = is_root ? (int)ST_CYCLE_ROOT : (int)ST_CYCLE_NONROOT;
  st.push_back(g);
  // update the query (Cases 1-3)
  for (int i = 0; i < ne; i++) {
    int a = x.nodes[i], b = x.nodes[(i + 1) % x.L];
    s.adj[a] &= ~(1u << b);
    s.adj[b] &= ~(1u << a);
    s.edge_ann[a][b] = s.edge_ann[b][a] = -1;
    s.edge_first[a][b] = s.edge_first[b][a] = -1;
  }
  if (x.leaf) {
    int a = x.nodes[0], b = x.nodes[1];
    s.alive &= ~(1u << b);
    s.node_ann[b] = -1;
    s.node_ann[a] = id;
    return;
  }
  for (int i = 0; i < x.L; i++) {
    int a = x.nodes[i];
    s.node_ann[a] = -1;
    if (a != x.bd[0] && a != x.bd[1]) s.alive &= ~(1u << a);
  }
  if (is_root) {
    s.alive = 0;
    return;
  }
  if (x.nb == 1) {
    s.node_ann[x.bd[0]] = id;
  } else {
    int a = x.bd[0], b = x.bd[1];
    s.adj[a] |= 1u << b;
    s.adj[b] |= 1u << a;
    s.edge_ann[a][b] = s.edge_ann[b][a] = id;
    s.edge_first[a][b] = s.edge_first[b][a] = a;
  }
}

// If the state is at its root, append the root stage and return true.
bool try_root(QS &s, std::vector<Stage> &st, bool *ok) {
  *ok = true;
  int na = popc(s.alive);
  if (na == 1) {
    int a = __builtin_ctz(s.alive);
    if (s.node_ann[a] < 0) { *ok = false; return true; }
    Stage g;
    for (int i = 0; i < kMaxK; i++) g.node_child[i] = -1, g.edge_child[i] = -1, g.edge_fwd[i] = true;
    g.kind = ST_ROOT_NODE;
    g.L = 1;
    g.nodes[0] = a;
    g.node_child[0] = s.node_ann[a];
    g.sq_mask = st[s.node_ann[a]].sq_mask;
    g.s = popc(g.sq_mask);
    st.push_back(g);
    s.alive = 0;
    return true;
  }
  // one induced cycle over every remaining node: the root cycle
  std::vector<std::vector<int>> cyc;
  cycles(s, cyc);
  for (auto &cy : cyc) {
    if ((int)cy.size() != na) continue;
    uint32_t edges = 0;
    int ecount = 0;
    for (int a = 0; a < s.k; a++)
      if (s.alive >> a & 1) ecount += popc(s.adj[a] & s.alive);
    (void)edges;
    if (ecount != 2 * na) continue;  // extra edges: not just the cycle
    Cand x;
    x.L = na;
    for (int i = 0; i < na; i++) x.nodes[i] = cy[i];
    x.nb = 0;
    apply(s, x, st, true);
    return true;
  }
  return false;
}

// Ranking of a decomposition tree.  The paper's factors, in its order
// (Section 5.3): longest cycle block, boundary nodes, annotations.  The
// library inserts one engine-aware factor after the longest cycle (see
// join_cost) unless `paper_only`.
struct Score {
  int unsupported, longest, nonroot_long;
  double cost;
  int boundary, annotations, stages;
  bool paper_only;
  bool operator<(const Score &o) const {
    if (unsupported != o.unsupported) return unsupported < o.unsupported;
    if (longest != o.longest) return longest < o.longest;
    // non-root cycles of length >= 4 run on the general per-source kernel
    if (!paper_only && nonroot_long != o.nonroot_long) return nonroot_long < o.nonroot_long;
    if (!paper_only && cost != o.cost) return cost < o.cost;
    if (boundary != o.boundary) return boundary < o.boundary;
    if (annotations != o.annotations) return annotations < o.annotations;
    return stages < o.stages;
  }
};

int64_t binom_i(int a, int b) {
  if (b < 0 || a < 0 || b > a) return 0;
  int64_t r = 1;
  for (int i = 1; i <= b; i++) r = r * (a - b + i) / i;
  return r;
}

// Engine-aware cost of the triangle and leaf blocks, in units of one table
// entry joined per data edge: a triangle block joins, per data triangle and
// for each of its six node assignments, the rows of all its annotating
// blocks (their product of row lengths; four times that when two or more
// annotate it, the partial-list form; twice when its output is keyed by
// edge); a leaf block joins per data edge one row of each annotating block.
// Data triangles are taken as three per edge, the order of the heavy-tailed
// benchmark graphs (about 3.4 on the Chung-Lu n = 10^6 graph).
double join_cost(const std::vector<Stage> &st, int k) {
  auto row_len = [&](int c) -> double {
    const Stage &b = st[c];
    return (double)(b.nb == 2 ? binom_i(k - 2, b.s - 2) : binom_i(k - 1, b.s - 1));
  };
  double tot = 0.0;
  for (auto &g : st) {
    if (g.kind != ST_TRI && g.kind != ST_LEAF) continue;
    const int ne = g.kind == ST_LEAF ? 1 : g.L;
    double prod = 1.0;
    int kids = 0;
    for (int i = 0; i < g.L; i++)
      if (g.node_child[i] >= 0) prod *= row_len(g.node_child[i]), kids++;
    for (int i = 0; i < ne; i++)
      if (g.edge_child[i] >= 0) prod *= row_len(g.edge_child[i]), kids++;
    if (g.kind == ST_LEAF) tot += prod;
    else tot += 3.0 * 6.0 * prod * (kids >= 2 ? 4.0 : 1.0) * (g.nb == 2 ? 2.0 : 1.0);
  }
  return tot;
}

Score score_of(const std::vector<Stage> &st, int k = 0, bool paper_only = false) {
  Score sc{0, 0, 0, 0.0, 0, 0, (int)st.size(), paper_only};
  for (auto &g : st) {
    if (g.kind == ST_CYCLE_NONROOT && g.L > kMaxCycle) sc.unsupported = 1;
    if (g.kind == ST_CYCLE_NONROOT && g.nb == 2) {
      // cut at the boundary nodes: the longer half must fit the kernel's levels
      int i0 = 0, i1 = 0;
      for (int i = 0; i < g.L; i++) {
        if (g.nodes[i] == g.bd[0]) i0 = i;
        if (g.nodes[i] == g.bd[1]) i1 = i;
      }
      const int d = (i1 - i0 + g.L) % g.L;
      if (g.L - std::min(d, g.L - d) > kMaxHalf) sc.unsupported = 1;
    }
    // pair-keyed tables: produced and read by the cycle kernel only
    int ne_g = g.kind == ST_LEAF ? 1 : (g.kind == ST_ROOT_NODE ? 0 : g.L), pair_edges = 0;
    for (int i = 0; i < ne_g; i++) pair_edges += edge_pair_keyed(st, g, i);
    if (pair_edges > kMaxPairGraphs) sc.unsupported = 1;
    if (g.kind == ST_CYCLE_NONROOT) sc.nonroot_long++;
    if (g.kind == ST_CYCLE_ROOT && g.L > kMaxCycle) sc.unsupported = 1;
    if (g.kind == ST_TRI || g.kind == ST_CYCLE_ROOT || g.kind == ST_CYCLE_NONROOT)
      sc.longest = std::max(sc.longest, g.L);
    sc.boundary += g.nb;
    int ne = g.kind == ST_LEAF ? 1 : (g.kind == ST_ROOT_NODE ? 0 : g.L);
    for (int i = 0; i < g.L; i++) sc.annotations += g.node_child[i] >= 0;
    for (int i = 0; i < ne; i++) sc.annotations += g.edge_child[i] >= 0;
  }
  if (k > 0 && !paper_only) sc.cost = join_cost(st, k);
  return sc;
}

int validate(int k, const std::vector<std::pair<int, int>> &edges) {
  if (k < 2 || k > kMaxK) return CC_ERR_K_RANGE;
  uint32_t adj[kMaxK] = {0};
  for (auto &e : edges) {
    if (e.first < 0 || e.second < 0 || e.first >= k || e.second >= k || e.first == e.second)
      return CC_ERR_INVALID_ARG;
    if (adj[e.first] >> e.second & 1) return CC_ERR_INVALID_ARG;
    adj[e.first] |= 1u << e.second;
    adj[e.second] |= 1u << e.first;
  }
  uint32_t seen = 1, frontier = 1;
  while (frontier) {
    uint32_t nxt = 0;
    for (int a = 0; a < k; a++)
      if (frontier >> a & 1) nxt |= adj[a];
    frontier = nxt & ~seen;
    seen |= nxt;
  }
  if (seen != ((1u << k) - 1)) return CC_ERR_NOT_CONNECTED;
  return CC_OK;
}

// Structural signature of each block: kind, size, boundary count and the
// annotating children by position (cycle positions relative to the block's
// own node order).  Two blocks with equal signatures represent isomorphic
// subqueries with the same boundary roles, so their tables are equal.
void signatures(Plan &p) {
  for (auto &st : p.stages) {
    std::string g = std::to_string(st.kind) + "/" + std::to_string(st.L) + "/" + std::to_string(st.s) + "/" +
                    std::to_string(st.nb) + "[";
    int ne = st.kind == ST_LEAF ? 1 : (st.kind == ST_ROOT_NODE ? 0 : st.L);
    for (int i = 0; i < st.L; i++) {
      bool bdn = st.nb > 0 && (st.nodes[i] == st.bd[0] || (st.nb > 1 && st.nodes[i] == st.bd[1]));
      g += (bdn ? "b" : "n");
      g += st.node_child[i] >= 0 ? "(" + p.stages[st.node_child[i]].sig + ")" : "-";
      if (i < ne) {
        g += st.edge_child[i] >= 0 ? std::string(st.edge_fwd[i] ? "F" : "R") + "(" + p.stages[st.edge_child[i]].sig + ")"
                                   : "e";
      }
      g += ",";
    }
    st.sig = g + "]";
  }
}

void finish(Plan &p, int k, const std::vector<std::pair<int, int>> &edges) {
  signatures(p);
  p.k = k;
  p.edges = edges;
  p.aut = count_automorphisms(k, edges);
  Score sc = score_of(p.stages);
  p.longest_cycle = sc.longest;
  p.supported = sc.unsupported == 0;
}

}  // namespace

int64_t count_automorphisms(int k, const std::vector<std::pair<int, int>> &edges) {
  uint32_t adj[kMaxK] = {0};
  for (auto &e : edges) {
    adj[e.first] |= 1u << e.second;
    adj[e.second] |= 1u << e.first;
  }
  int img[kMaxK];
  int64_t count = 0;
  std::function<void(int, uint32_t)> rec = [&](int i, uint32_t used) {
    if (i == k) { count++; return; }
    for (int c = 0; c < k; c++) {
      if (used >> c & 1) continue;
      if (popc(adj[c]) != popc(adj[i])) continue;
      bool ok = true;
      for (int j = 0; j < i && ok; j++)
        if (((adj[i] >> j) & 1) != ((adj[c] >> img[j]) & 1)) ok = false;
      if (!ok) continue;
      img[i] = c;
      rec(i + 1, used | (1u << c));
    }
  };
  rec(0, 0);
  return count;
}

int plan_query(int k, const std::vector<std::pair<int, int>> &edges, Plan &out, bool paper_only) {
  int rc = validate(k, edges);
  if (rc != CC_OK) return rc;
  QS s0;
  init_state(s0, k, edges);
  bool found = false, any_block_failure = false;
  Score best{};
  std::vector<Stage> best_st;
  int explored = 0;
  const int kCap = 600;
  std::function<void(QS &, std::vector<Stage> &)> dfs = [&](QS &s, std::vector<Stage> &st) {
    if (explored >= kCap) return;
    bool ok = true;
    size_t mark = st.size();
    QS saved = s;
    if (try_root(s, st, &ok)) {
      if (ok) {
        explored++;
        Score sc = score_of(st, k, paper_only);
        if (!found || sc < best) { best = sc; best_st = st; found = true; }
      }
      st.resize(mark);
      s = saved;
      return;
    }
    std::vector<Cand> cs = candidates(s);
    if (cs.empty()) { any_block_failure = true; return; }
    // leaves first, then shorter cycles: good plans are met early
    std::stable_sort(cs.begin(), cs.end(), [](const Cand &a, const Cand &b) {
      if (a.leaf != b.leaf) return a.leaf;
      if (a.L != b.L) return a.L < b.L;
      return a.nb > b.nb;
    });
    for (auto &c : cs) {
      QS t = s;
      apply(t, c, st, false);
      dfs(t, st);
      st.resize(mark);
      if (explored >= kCap) return;
    }
  };
  std::vector<Stage> st;
  dfs(s0, st);
  if (!found) return any_block_failure ? CC_ERR_NOT_TW2 : CC_ERR_NOT_TW2;
  out = Plan();
  out.stages = best_st;
  finish(out, k, edges);
  return out.supported ? CC_OK : CC_ERR_UNSUPPORTED;
}

// Every decomposition tree of the query (Section 5.3: one tree per sequence
// of choices; sequences that differ only in the order of independent
// contractions give the same tree, kept once by the root block's structural
// signature), each as the contraction sequence cc_set_decomposition takes,
// with the paper's ranking factors.
int plan_enumerate(int k, const std::vector<std::pair<int, int>> &edges, std::vector<PlanChoice> &out) {
  int rc = validate(k, edges);
  if (rc != CC_OK) return rc;
  Plan def, pap;
  int drc = plan_query(k, edges, def, false);
  int prc = plan_query(k, edges, pap, true);
  const std::string def_sig = (drc == CC_OK || drc == CC_ERR_UNSUPPORTED) && !def.stages.empty()
                                  ? def.stages.back().sig : std::string();
  const std::string pap_sig = (prc == CC_OK || prc == CC_ERR_UNSUPPORTED) && !pap.stages.empty()
                                  ? pap.stages.back().sig : std::string();
  QS s0;
  init_state(s0, k, edges);
  std::map<std::string, size_t> seen;
  int explored = 0;
  const int kCap = 20000;
  std::function<void(QS &, std::vector<Stage> &)> dfs = [&](QS &s, std::vector<Stage> &st) {
    if (explored >= kCap) return;
    bool ok = true;
    size_t mark = st.size();
    QS saved = s;
    if (try_root(s, st, &ok)) {
      if (ok) {
        explored++;
        Plan p;
        p.stages = st;
        finish(p, k, edges);
        const std::string &sig = p.stages.back().sig;
        if (!seen.count(sig)) {
          PlanChoice c;
          for (size_t i = 0; i + 1 < p.stages.size(); i++) {
            const Stage &g = p.stages[i];
            c.seq.push_back(g.kind == ST_LEAF ? 0 : g.L);
            for (int j = 0; j < g.L; j++) c.seq.push_back(g.nodes[j]);
          }
          Score sc = score_of(p.stages, k);
          c.supported = sc.unsupported == 0;
          c.longest = sc.longest;
          c.boundary = sc.boundary;
          c.annotations = sc.annotations;
          c.cost = sc.cost;
          c.is_default = sig == def_sig;
          c.is_paper = sig == pap_sig;
          seen[sig] = out.size();
          out.push_back(c);
        }
      }
      st.resize(mark);
      s = saved;
      return;
    }
    std::vector<Cand> cs = candidates(s);
    for (auto &c : cs) {
      QS t = s;
      apply(t, c, st, false);
      dfs(t, st);
      st.resize(mark);
      if (explored >= kCap) return;
    }
  };
  std::vector<Stage> st;
  dfs(s0, st);
  return out.empty() ? CC_ERR_NOT_TW2 : CC_OK;
}

int plan_explicit(int k, const std::vector<std::pair<int, int>> &edges,
                  const std::vector<int> &seq, Plan &out) {
  int rc = validate(k, edges);
  if (rc != CC_OK) return rc;
  QS s;
  init_state(s, k, edges);
  std::vector<Stage> st;
  size_t i = 0;
  while (i < seq.size()) {
    int L = seq[i];
    int len = (L == 0) ? 2 : L;
    if (L == 1 || L < 0 || L > kMaxK || i + 1 + len > seq.size()) return CC_ERR_INVALID_ARG;
    std::vector<int> want(seq.begin() + i + 1, seq.begin() + i + 1 + len);
    i += 1 + len;
    std::vector<Cand> cs = candidates(s);
    int pick = -1;
    for (size_t c = 0; c < cs.size() && pick < 0; c++) {
      const Cand &x = cs[c];
      if (L == 0) {
        if (x.leaf && x.nodes[0] == want[0] && x.nodes[1] == want[1]) pick = (int)c;
        continue;
      }
      if (x.leaf || x.L != L) continue;
      // same cycle: equal node sets with equal cyclic neighbours
      bool same = true;
      for (int a = 0; a < L && same; a++) {
        int p = -1;
        for (int b = 0; b < L; b++) if (x.nodes[b] == want[a]) p = b;
        if (p < 0) { same = false; break; }
        int nx = want[(a + 1) % L];
        if (x.nodes[(p + 1) % L] != nx && x.nodes[(p + L - 1) % L] != nx) same = false;
      }
      if (same) pick = (int)c;
    }
    if (pick < 0) return CC_ERR_INVALID_ARG;
    // the cycle keeps the caller's orientation
    Cand x = cs[pick];
    if (L > 0)
      for (int a = 0; a < L; a++) x.nodes[a] = want[a];
    if (!x.leaf && popc(s.alive) == x.L && x.nb == 0) return CC_ERR_INVALID_ARG;  // root is implied
    apply(s, x, st, false);
  }
  bool ok = true;
  if (!try_root(s, st, &ok) || !ok) return CC_ERR_INVALID_ARG;
  out = Plan();
  out.stages = st;
  finish(out, k, edges);
  return out.supported ? CC_OK : CC_ERR_UNSUPPORTED;
}

}  // namespace cc
