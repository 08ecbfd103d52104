// CPU oracle for colour-coding subgraph counting of treewidth-2 queries.
//
// TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
// baseline leg of the benchmark may load this library.  It shares no code with
// the CUDA library: its own graph structures, colouring hash, query
// decomposition, automorphism count and dynamic program.
//
// What it computes (Chakaravarthy et al., "Subgraph Counting: Color Coding
// Beyond Trees", arXiv 1602.04478):
//   * brute_colorful: the number of colourful matches, straight from the
//     definitions of Section 2 ("Subgraph counting problem", "Color coding and
//     colorful matches"): maps pi: V_Q -> V_G with every query edge on a data
//     edge and the k images carrying k distinct colours.
//   * brute_matches: the number of matches (injective edge-preserving maps),
//     Section 2, used for the estimator identity (k^k/k!) E[n_colorful] = n.
//   * automorphisms: aut(Q) by enumerating the k! permutations (Section 2).
//   * decompose: the decomposition tree of Section 4.1 (Cases 1-3).
//   * dp_count: the bottom-up traversal of Section 4.2 (Figure "Overall
//     Algorithm") with projection tables as hash maps keyed by boundary images
//     and signature (Section 4.2), cycle blocks by the DB procedure of
//     Section 5 (Procedures 1-2 and the NodeJoin / EdgeJoin procedure for
//     general cycles, all highest-node choices h, Eq. 1), or by the PS
//     split without any vertex order; leaf blocks and the root as in
//     Section 5.2.
// Readings of points the paper leaves open:
//   * colours are 0..k-1 (bit c of a mask) instead of 1..k;
//   * the colour of vertex v in trial t is hi64(mix(seed ^ G*(t+1) ^ mix(v)) * k)
//     with mix = SplitMix64's output function applied to x + G,
//     G = 0x9E3779B97F4A7C15 (an explicit colour array may be passed instead);
//   * the DB first edge also requires u > w in the order (as in Procedure 1);
//   * the general-cycle join loop runs NodeJoin/EdgeJoin for a_{h+1}..a_{d-1}
//     and then NodeJoin(a_d) once; P- joins a_h's node block and P+ joins
//     a_d's, so every node block is joined exactly once per h;
//   * the degree order is (degree, caller id) ascending (Section 5.1 tie rule).
// Counts are accumulated in unsigned 128-bit integers; any table entry or the
// final count above 2^64-1 sets the overflow flag.
#include <algorithm>
#include <chrono>
#include <cstdint>
#include <cstring>
#include <functional>
#include <map>
#include <set>
#include <unordered_map>
#include <vector>

typedef unsigned __int128 u128;
typedef uint32_t Mask;

static const u128 U64MAX = (u128)(~0ULL);

// ------------------------------- data graph -------------------------------
struct DGraph {
  int64_t n = 0;
  std::vector<std::vector<int32_t>> adj;  // sorted neighbour lists
  std::vector<std::unordered_map<int32_t, int>> pos;  // unused for small graphs
  bool has_edge(int32_t a, int32_t b) const {
    const auto &r = adj[a];
    return std::binary_search(r.begin(), r.end(), b);
  }
};

static void load_graph(DGraph &g, int64_t n, const int64_t *row_ptr, const int32_t *col) {
  g.n = n;
  g.adj.assign((size_t)n, {});
  for (int64_t v = 0; v < n; v++) {
    g.adj[v].assign(col + row_ptr[v], col + row_ptr[v + 1]);
    std::sort(g.adj[v].begin(), g.adj[v].end());
  }
}

// ------------------------------- query graph -------------------------------
struct QGraph {
  int k = 0;
  std::vector<std::vector<int>> adj;
  std::vector<std::vector<bool>> am;
};

static bool load_query(QGraph &q, int k, int ne, const int32_t *edges) {
  if (k < 1 || k > 16) return false;
  q.k = k;
  q.adj.assign(k, {});
  q.am.assign(k, std::vector<bool>(k, false));
  for (int i = 0; i < ne; i++) {
    int a = edges[2 * i], b = edges[2 * i + 1];
    if (a < 0 || b < 0 || a >= k || b >= k || a == b) return false;
    if (q.am[a][b]) return false;
    q.am[a][b] = q.am[b][a] = true;
    q.adj[a].push_back(b);
    q.adj[b].push_back(a);
  }
  return true;
}

// BFS order so every node after the first has an earlier neighbour.
static std::vector<int> bfs_order(const QGraph &q) {
  std::vector<int> order, seen(q.k, 0);
  order.push_back(0);
  seen[0] = 1;
  for (size_t i = 0; i < order.size(); i++)
    for (int b : q.adj[order[i]])
      if (!seen[b]) { seen[b] = 1; order.push_back(b); }
  return order;
}

// ------------------------------- colouring -------------------------------
static inline uint64_t sm_mix(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

// SplitMix64's next() for a generator whose state is x (exposed for its test vector).
extern "C" uint64_t or_splitmix64(uint64_t x) { return sm_mix(x); }

extern "C" int or_color(uint64_t seed, int64_t trial, int64_t v, int k) {
  uint64_t h = sm_mix(seed ^ (0x9E3779B97F4A7C15ULL * (uint64_t)(trial + 1)) ^ sm_mix((uint64_t)v));
  return (int)(uint64_t)(((u128)h * (u128)(uint64_t)k) >> 64);
}

extern "C" void or_colors(uint64_t seed, int64_t trial, int64_t n, int k, uint8_t *out) {
  for (int64_t v = 0; v < n; v++) out[v] = (uint8_t)or_color(seed, trial, v, k);
}

// ------------------------------- brute force -------------------------------
struct Brute {
  const DGraph *g;
  const QGraph *q;
  const uint8_t *col;  // nullptr: uncoloured (injective matches)
  std::vector<int> order, img;
  std::vector<int> used_vertex_stamp;  // for injectivity (uncoloured)
  u128 count = 0;
  int fixed_node = -1;
  int32_t fixed_vertex = -1;

  void rec(size_t i, Mask used_colors) {
    if (i == order.size()) { count += 1; return; }
    int a = order[i];
    // candidates: neighbours of an earlier-mapped neighbour, or all vertices
    int anchor = -1;
    for (size_t j = 0; j < i; j++)
      if (q->am[a][order[j]]) { anchor = order[j]; break; }
    auto try_v = [&](int32_t v) {
      if (a == fixed_node && v != fixed_vertex) return;
      Mask nc = used_colors;
      if (col) {
        Mask b = 1u << col[v];
        if (used_colors & b) return;
        nc |= b;
      } else {
        for (size_t j = 0; j < i; j++)
          if (img[order[j]] == v) return;
      }
      for (size_t j = 0; j < i; j++) {
        int b = order[j];
        if (q->am[a][b] && !g->has_edge(v, img[b])) return;
      }
      img[a] = v;
      rec(i + 1, nc);
      img[a] = -1;
    };
    if (anchor >= 0) {
      for (int32_t v : g->adj[img[anchor]]) try_v(v);
    } else if (a == fixed_node) {
      try_v(fixed_vertex);
    } else {
      for (int32_t v = 0; v < g->n; v++) try_v(v);
    }
  }
};

static u128 brute_count(const DGraph &g, const QGraph &q, const uint8_t *col, int fixed_node,
                        int32_t fixed_vertex) {
  Brute b;
  b.g = &g;
  b.q = &q;
  b.col = col;
  if (fixed_node >= 0) {
    // start the search at the fixed node so the root is pinned first
    std::vector<int> order{fixed_node}, seen(q.k, 0);
    seen[fixed_node] = 1;
    for (size_t i = 0; i < order.size(); i++)
      for (int c : q.adj[order[i]])
        if (!seen[c]) { seen[c] = 1; order.push_back(c); }
    b.order = order;
  } else {
    b.order = bfs_order(q);
  }
  b.img.assign(q.k, -1);
  b.fixed_node = fixed_node;
  b.fixed_vertex = fixed_vertex;
  b.rec(0, 0);
  return b.count;
}

static void put128(u128 v, uint64_t *out) {
  out[0] = (uint64_t)v;
  out[1] = (uint64_t)(v >> 64);
}

// Colourful matches (Section 2), optionally only those with pi(fixed_node) = fixed_vertex.
extern "C" int or_brute_colorful(int64_t n, const int64_t *row_ptr, const int32_t *col, int k,
                                 int ne, const int32_t *qedges, const uint8_t *colors,
                                 int fixed_node, int32_t fixed_vertex, uint64_t *out128) {
  DGraph g;
  QGraph q;
  if (!load_query(q, k, ne, qedges)) return -1;
  load_graph(g, n, row_ptr, col);
  put128(brute_count(g, q, colors, fixed_node, fixed_vertex), out128);
  return 0;
}

// Matches (injective, edge preserving), no colours.
extern "C" int or_brute_matches(int64_t n, const int64_t *row_ptr, const int32_t *col, int k,
                                int ne, const int32_t *qedges, uint64_t *out128) {
  DGraph g;
  QGraph q;
  if (!load_query(q, k, ne, qedges)) return -1;
  load_graph(g, n, row_ptr, col);
  put128(brute_count(g, q, nullptr, -1, -1), out128);
  return 0;
}

// aut(Q): permutations of V_Q that map E_Q onto itself.
extern "C" int64_t or_automorphisms(int k, int ne, const int32_t *qedges) {
  QGraph q;
  if (!load_query(q, k, ne, qedges)) return -1;
  std::vector<int> p(k);
  for (int i = 0; i < k; i++) p[i] = i;
  int64_t cnt = 0;
  do {
    bool ok = true;
    for (int a = 0; a < k && ok; a++)
      for (int b = 0; b < k && ok; b++)
        if (q.am[a][b] != q.am[p[a]][p[b]]) ok = false;
    cnt += ok;
  } while (std::next_permutation(p.begin(), p.end()));
  return cnt;
}

// --------------------------- decomposition tree ---------------------------
// Section 4.1: repeatedly contract a block (leaf edge, or an induced cycle
// with at most two boundary nodes), annotating what it leaves behind.
enum BlockKind { B_LEAF = 0, B_CYCLE = 1, B_ROOT_CYCLE = 2, B_ROOT_NODE = 3 };

struct EdgeAnn {
  int block = -1;
  int first = -1;  // query node the block's table uses as its first key
};

struct Block {
  int kind = 0;
  std::vector<int> nodes;     // leaf: {a, b} (b is the leaf); cycle: a_0..a_{L-1}
  std::vector<int> boundary;  // ordered boundary nodes (0, 1 or 2)
  std::map<int, int> node_ann;                   // query node -> child block
  std::map<std::pair<int, int>, EdgeAnn> edge_ann;  // (min,max) -> child block
  std::vector<int> sq;        // nodes of the represented subquery
};

struct QState {
  int k;
  std::vector<bool> alive;
  std::set<std::pair<int, int>> edges;  // (min, max)
  std::map<int, int> node_ann;
  std::map<std::pair<int, int>, EdgeAnn> edge_ann;
  bool edge(int a, int b) const { return edges.count({std::min(a, b), std::max(a, b)}) > 0; }
  int deg(int a) const {
    int d = 0;
    for (int b = 0; b < k; b++) if (alive[b] && b != a && edge(a, b)) d++;
    return d;
  }
  int n_alive() const {
    int c = 0;
    for (bool x : alive) c += x;
    return c;
  }
};

struct Candidate {
  int kind;               // B_LEAF or B_CYCLE
  std::vector<int> nodes;  // leaf {a, b}; cycle in cyclic order
  std::vector<int> boundary;
};

// All simple cycles of the alive query (each once: smallest node first, one direction).
static void enum_cycles(const QState &s, std::vector<std::vector<int>> &out) {
  int k = s.k;
  std::vector<int> path;
  std::vector<bool> on(k, false);
  std::function<void(int, int)> dfs = [&](int start, int v) {
    for (int w = 0; w < k; w++) {
      if (!s.alive[w] || !s.edge(v, w)) continue;
      if (w == start && path.size() >= 3) {
        if (path[1] < path.back()) out.push_back(path);  // one direction only
        continue;
      }
      if (on[w] || w < start) continue;
      on[w] = true;
      path.push_back(w);
      dfs(start, w);
      path.pop_back();
      on[w] = false;
    }
  };
  for (int st = 0; st < k; st++) {
    if (!s.alive[st]) continue;
    path = {st};
    on.assign(k, false);
    on[st] = true;
    dfs(st, st);
  }
}

static std::vector<Candidate> find_blocks(const QState &s) {
  std::vector<Candidate> c;
  int k = s.k;
  // leaf edges (a, b) with b of degree one; skip the symmetric duplicate of a lone edge
  for (int b = 0; b < k; b++) {
    if (!s.alive[b] || s.deg(b) != 1) continue;
    for (int a = 0; a < k; a++)
      if (s.alive[a] && a != b && s.edge(a, b)) c.push_back({B_LEAF, {a, b}, {a}});
  }
  std::vector<std::vector<int>> cyc;
  enum_cycles(s, cyc);
  for (auto &cy : cyc) {
    std::set<int> in(cy.begin(), cy.end());
    // induced: no edge between cycle nodes other than consecutive ones
    bool induced = true;
    int L = (int)cy.size();
    for (int i = 0; i < L && induced; i++)
      for (int j = i + 2; j < L && induced; j++) {
        if (i == 0 && j == L - 1) continue;
        if (s.edge(cy[i], cy[j])) induced = false;
      }
    if (!induced) continue;
    std::vector<int> bd;
    for (int a : cy) {
      bool out = false;
      for (int b = 0; b < k; b++)
        if (s.alive[b] && !in.count(b) && s.edge(a, b)) out = true;
      if (out) bd.push_back(a);
    }
    if (bd.size() <= 2) c.push_back({B_CYCLE, cy, bd});
  }
  return c;
}

struct Decomp {
  std::vector<Block> blocks;
  int root = -1;
  bool ok = false;
};

// choice: at step i the candidate index choice[i] (modulo the number of
// candidates) is contracted; choices beyond the vector pick candidate 0.
// n_choices receives the number of candidates at each step.
static Decomp decompose(const QGraph &q, const std::vector<int> &choice, std::vector<int> *n_choices) {
  Decomp D;
  QState s;
  s.k = q.k;
  s.alive.assign(q.k, true);
  for (int a = 0; a < q.k; a++)
    for (int b : q.adj[a])
      if (a < b) s.edges.insert({a, b});
  size_t step = 0;
  while (true) {
    int na = s.n_alive();
    if (na == 1) {
      int a = -1;
      for (int i = 0; i < q.k; i++) if (s.alive[i]) a = i;
      if (!s.node_ann.count(a)) return D;  // single-node query: nothing to count
      Block r;
      r.kind = B_ROOT_NODE;
      r.nodes = {a};
      r.node_ann[a] = s.node_ann[a];
      r.sq = D.blocks[s.node_ann[a]].sq;
      D.blocks.push_back(r);
      D.root = (int)D.blocks.size() - 1;
      D.ok = true;
      return D;
    }
    std::vector<Candidate> cand = find_blocks(s);
    // the whole remaining query is one induced cycle: it is the root block
    for (auto &c : cand) {
      if (c.kind == B_CYCLE && (int)c.nodes.size() == na && c.boundary.empty()) {
        Block r;
        r.kind = B_ROOT_CYCLE;
        r.nodes = c.nodes;
        std::set<int> sqs;
        int L = (int)c.nodes.size();
        for (int i = 0; i < L; i++) {
          int a = c.nodes[i], b = c.nodes[(i + 1) % L];
          sqs.insert(a);
          if (s.node_ann.count(a)) {
            r.node_ann[a] = s.node_ann[a];
            for (int x : D.blocks[s.node_ann[a]].sq) sqs.insert(x);
          }
          auto key = std::make_pair(std::min(a, b), std::max(a, b));
          if (s.edge_ann.count(key)) {
            r.edge_ann[key] = s.edge_ann[key];
            for (int x : D.blocks[s.edge_ann[key].block].sq) sqs.insert(x);
          }
        }
        r.sq.assign(sqs.begin(), sqs.end());
        D.blocks.push_back(r);
        D.root = (int)D.blocks.size() - 1;
        D.ok = true;
        return D;
      }
    }
    if (cand.empty()) return D;  // no block: treewidth above 2 (Lemma 4.1)
    if (n_choices) n_choices->push_back((int)cand.size());
    int ci = step < choice.size() ? choice[step] % (int)cand.size() : 0;
    step++;
    const Candidate &c = cand[ci];
    Block B;
    B.kind = c.kind;
    B.nodes = c.nodes;
    B.boundary = c.boundary;
    std::set<int> sqs;
    int id = (int)D.blocks.size();
    if (c.kind == B_LEAF) {
      int a = c.nodes[0], b = c.nodes[1];
      auto key = std::make_pair(std::min(a, b), std::max(a, b));
      for (int x : {a, b}) {
        sqs.insert(x);
        if (s.node_ann.count(x)) {
          B.node_ann[x] = s.node_ann[x];
          for (int y : D.blocks[s.node_ann[x]].sq) sqs.insert(y);
        }
      }
      if (s.edge_ann.count(key)) {
        B.edge_ann[key] = s.edge_ann[key];
        for (int y : D.blocks[s.edge_ann[key].block].sq) sqs.insert(y);
        s.edge_ann.erase(key);
      }
      // Case 3: drop b and the edge, annotate a with the new block
      s.alive[b] = false;
      s.edges.erase(key);
      s.node_ann.erase(b);
      s.node_ann[a] = id;
    } else {
      int L = (int)c.nodes.size();
      std::set<int> bd(c.boundary.begin(), c.boundary.end());
      for (int i = 0; i < L; i++) {
        int a = c.nodes[i], b = c.nodes[(i + 1) % L];
        sqs.insert(a);
        if (s.node_ann.count(a)) {
          B.node_ann[a] = s.node_ann[a];
          for (int y : D.blocks[s.node_ann[a]].sq) sqs.insert(y);
        }
        auto key = std::make_pair(std::min(a, b), std::max(a, b));
        if (s.edge_ann.count(key)) {
          B.edge_ann[key] = s.edge_ann[key];
          for (int y : D.blocks[s.edge_ann[key].block].sq) sqs.insert(y);
          s.edge_ann.erase(key);
        }
        s.edges.erase(key);
      }
      for (int a : c.nodes) {
        s.node_ann.erase(a);  // inherited by the block
        if (!bd.count(a)) s.alive[a] = false;
      }
      if (c.boundary.size() == 1) {
        s.node_ann[c.boundary[0]] = id;  // Case 1
      } else if (c.boundary.size() == 2) {
        int a = c.boundary[0], b = c.boundary[1];  // Case 2
        auto key = std::make_pair(std::min(a, b), std::max(a, b));
        s.edges.insert(key);
        s.edge_ann[key] = EdgeAnn{id, a};
      } else {
        return D;  // a cycle with no boundary that is not the whole query cannot occur
      }
    }
    B.sq.assign(sqs.begin(), sqs.end());
    D.blocks.push_back(B);
  }
}

// ------------------------------ projection tables ------------------------------
struct UKeyHash {
  size_t operator()(uint64_t x) const { return (size_t)sm_mix(x); }
};
// unary: (v, mask) -> count
typedef std::unordered_map<uint64_t, u128, UKeyHash> UTable;
static inline uint64_t ukey(int32_t v, Mask m) { return ((uint64_t)(uint32_t)v << 20) | m; }
static inline int32_t ukey_v(uint64_t key) { return (int32_t)(key >> 20); }
static inline Mask ukey_m(uint64_t key) { return (Mask)(key & 0xFFFFF); }

// binary: (x, y, mask) with x = image of the block's first boundary node
struct BKey {
  int32_t x, y;
  Mask m;
  bool operator==(const BKey &o) const { return x == o.x && y == o.y && m == o.m; }
};
struct BKeyHash {
  size_t operator()(const BKey &k) const {
    return (size_t)sm_mix(((uint64_t)(uint32_t)k.x << 32) ^ (uint64_t)(uint32_t)k.y ^ ((uint64_t)k.m << 44));
  }
};
typedef std::unordered_map<BKey, u128, BKeyHash> BTable;

struct Table {
  int arity = 0;  // 1 unary, 2 binary
  UTable u;
  BTable b;
  // index of the binary table by its first and by its second key
  std::unordered_map<int32_t, std::vector<std::pair<BKey, u128>>> by_first, by_second;
  // unary table by vertex
  std::unordered_map<int32_t, std::vector<std::pair<Mask, u128>>> by_vertex;
  void index() {
    by_first.clear();
    by_second.clear();
    by_vertex.clear();
    for (auto &e : b) {
      by_first[e.first.x].push_back(e);
      by_second[e.first.y].push_back(e);
    }
    for (auto &e : u) by_vertex[ukey_v(e.first)].push_back({ukey_m(e.first), e.second});
  }
};

struct Ctx {
  const DGraph *g;
  const QGraph *q;
  const uint8_t *col;
  const std::vector<int64_t> *rank;  // nullptr: no vertex order (PS)
  bool overflow = false;
  // optional restriction of the root cycle's highest vertex
  const std::vector<char> *root_sources = nullptr;
  std::vector<u128> *per_source = nullptr;  // root cycle: count by highest vertex
  Mask bit(int32_t v) const { return 1u << col[v]; }
  bool higher(int32_t u, int32_t w) const { return (*rank)[u] > (*rank)[w]; }
};

// A path-table entry of the DB procedure: endpoints u (image of a_h) and v
// (current end), recorded images of boundary nodes met on the path, signature.
struct PKey {
  int32_t u, v;
  int32_t rec[2];
  Mask m;
  bool operator==(const PKey &o) const {
    return u == o.u && v == o.v && rec[0] == o.rec[0] && rec[1] == o.rec[1] && m == o.m;
  }
};
struct PKeyHash {
  size_t operator()(const PKey &k) const {
    uint64_t h = sm_mix(((uint64_t)(uint32_t)k.u << 32) | (uint32_t)k.v);
    h = sm_mix(h ^ (((uint64_t)(uint32_t)k.rec[0] << 32) | (uint32_t)k.rec[1]));
    return (size_t)sm_mix(h ^ k.m);
  }
};
typedef std::unordered_map<PKey, u128, PKeyHash> PTable;

static inline void add_to(u128 &dst, u128 v) { dst += v; }

// Edge lookups for a cycle edge traversed from query node `from` to `to`:
// calls f(w, mask, value) for each annotated-table entry starting at data vertex v,
// or for each graph neighbour w of v (plain edge block B_G, Section 5.2).
static void for_each_edge_entry(const Ctx &C, const std::map<std::pair<int, int>, EdgeAnn> &eann,
                                const std::vector<Table> &tabs, int from, int to, int32_t v,
                                const std::function<void(int32_t, Mask, u128)> &f) {
  auto key = std::make_pair(std::min(from, to), std::max(from, to));
  auto it = eann.find(key);
  if (it == eann.end()) {
    // B_G: one colourful match per data edge whose ends differ in colour
    for (int32_t w : C.g->adj[v])
      if (C.col[w] != C.col[v]) f(w, C.bit(v) | C.bit(w), 1);
    return;
  }
  const Table &T = tabs[it->second.block];
  if (it->second.first == from) {
    auto jt = T.by_first.find(v);
    if (jt == T.by_first.end()) return;
    for (auto &e : jt->second) f(e.first.y, e.first.m, e.second);
  } else {
    auto jt = T.by_second.find(v);
    if (jt == T.by_second.end()) return;
    for (auto &e : jt->second) f(e.first.x, e.first.m, e.second);
  }
}

static const Table *node_table(const Block &B, const std::vector<Table> &tabs, int a) {
  auto it = B.node_ann.find(a);
  return it == B.node_ann.end() ? nullptr : &tabs[it->second];
}

// NodeJoin (general DB procedure): join each entry at its current end v with
// the unary table of the block annotating that query node.
static PTable node_join(const Ctx &C, const PTable &P, const Table *NT) {
  if (!NT) return P;
  PTable out;
  for (auto &e : P) {
    auto it = NT->by_vertex.find(e.first.v);
    if (it == NT->by_vertex.end()) continue;
    for (auto &ne : it->second) {
      if ((e.first.m & ne.first) != C.bit(e.first.v)) continue;
      PKey k = e.first;
      k.m = e.first.m | ne.first;
      out[k] += e.second * ne.second;
    }
  }
  return out;
}

// One DB/PS half path from a_h towards a_d in direction dir (+1 or -1).
static PTable build_half(const Ctx &C, const Block &B, const std::vector<Table> &tabs, int h,
                         int d, int dir, const std::vector<int> &bd, int32_t only_u) {
  const std::vector<int> &a = B.nodes;
  int L = (int)a.size();
  auto at = [&](int i) { return a[((i % L) + L) % L]; };
  auto record = [&](PKey &k, int qnode, int32_t img) {
    for (size_t i = 0; i < bd.size(); i++)
      if (bd[i] == qnode) k.rec[i] = img;
  };
  PTable P;
  // initial table: the (annotated or plain) edge a_h -> a_{h+dir}, high-starting
  int first = at(h), second = at(h + dir);
  for (int32_t u = 0; u < C.g->n; u++) {
    if (only_u >= 0 && u != only_u) continue;
    if (B.kind == B_ROOT_CYCLE && C.root_sources && !(*C.root_sources)[u]) continue;
    for_each_edge_entry(C, B.edge_ann, tabs, first, second, u, [&](int32_t w, Mask m, u128 val) {
      if (C.rank && !C.higher(u, w)) return;
      PKey k{u, w, {-1, -1}, m};
      record(k, first, u);
      record(k, second, w);
      P[k] += val;
    });
  }
  // P- includes the block annotating a_h (convention of Section 5.2)
  if (dir < 0) {
    const Table *NT = node_table(B, tabs, first);
    if (NT) {
      PTable out;
      for (auto &e : P) {
        auto it = NT->by_vertex.find(e.first.u);
        if (it == NT->by_vertex.end()) continue;
        for (auto &ne : it->second) {
          if ((e.first.m & ne.first) != C.bit(e.first.u)) continue;
          PKey k = e.first;
          k.m |= ne.first;
          out[k] += e.second * ne.second;
        }
      }
      P.swap(out);
    }
  }
  // interior nodes: NodeJoin(a_j) then EdgeJoin(a_j -> a_{j+dir})
  int steps = ((dir > 0 ? d - h : h - d) % L + L) % L;
  for (int s = 1; s < steps; s++) {
    int j = h + dir * s;
    P = node_join(C, P, node_table(B, tabs, at(j)));
    PTable out;
    int from = at(j), to = at(j + dir);
    for (auto &e : P) {
      for_each_edge_entry(C, B.edge_ann, tabs, from, to, e.first.v, [&](int32_t w, Mask m, u128 val) {
        if (C.rank && !C.higher(e.first.u, w)) return;
        if ((e.first.m & m) != C.bit(e.first.v)) return;
        PKey k = e.first;
        k.v = w;
        k.m = e.first.m | m;
        record(k, to, w);
        out[k] += e.second * val;
      });
    }
    P.swap(out);
  }
  // P+ includes the block annotating a_d
  if (dir > 0) P = node_join(C, P, node_table(B, tabs, at(d)));
  return P;
}

// A cycle block by DB (all highest-node choices h, Eq. 1) or by a single PS
// split without order.  Output: unary / binary table, or the root count.
static void solve_cycle(Ctx &C, const Block &B, const std::vector<Table> &tabs, Table &out,
                        u128 &root_count) {
  int L = (int)B.nodes.size();
  std::vector<int> bd = B.boundary;
  std::vector<int> hs;
  if (C.rank) for (int h = 0; h < L; h++) hs.push_back(h);
  else hs.push_back(0);
  int nb = (int)bd.size();
  out.arity = nb;
  std::vector<int> pos_of(C.q->k, -1);
  for (int i = 0; i < L; i++) pos_of[B.nodes[i]] = i;
  for (int h : hs) {
    int d = (h + L / 2) % L;
    PTable Pp = build_half(C, B, tabs, h, d, +1, bd, -1);
    PTable Pm = build_half(C, B, tabs, h, d, -1, bd, -1);
    // group P- by (u, v)
    std::unordered_map<uint64_t, std::vector<std::pair<PKey, u128>>, UKeyHash> gm;
    for (auto &e : Pm) gm[((uint64_t)(uint32_t)e.first.u << 32) | (uint32_t)e.first.v].push_back(e);
    // which half records each boundary node
    auto on_plus = [&](int qnode) {
      int p = pos_of[qnode];
      int off = ((p - h) % L + L) % L;
      return off <= (L / 2);
    };
    for (auto &e1 : Pp) {
      auto it = gm.find(((uint64_t)(uint32_t)e1.first.u << 32) | (uint32_t)e1.first.v);
      if (it == gm.end()) continue;
      Mask cuv = C.bit(e1.first.u) | C.bit(e1.first.v);
      for (auto &e2 : it->second) {
        if ((e1.first.m & e2.first.m) != cuv) continue;
        u128 val = e1.second * e2.second;
        Mask m = e1.first.m | e2.first.m;
        int32_t img[2] = {-1, -1};
        for (int i = 0; i < nb; i++) img[i] = on_plus(bd[i]) ? e1.first.rec[i] : e2.first.rec[i];
        if (nb == 0) {
          root_count += val;
          if (C.per_source) (*C.per_source)[e1.first.u] += val;
        } else if (nb == 1) {
          out.u[ukey(img[0], m)] += val;
        } else {
          out.b[BKey{img[0], img[1], m}] += val;
        }
      }
    }
  }
}

// Leaf block (a, b): join the tables on node a, edge (a, b) and node b.
static void solve_leaf(Ctx &C, const Block &B, const std::vector<Table> &tabs, Table &out) {
  int a = B.nodes[0], b = B.nodes[1];
  out.arity = 1;
  const Table *TA = node_table(B, tabs, a);
  const Table *TB = node_table(B, tabs, b);
  for (int32_t x = 0; x < C.g->n; x++) {
    std::vector<std::pair<Mask, u128>> arow;
    if (TA) {
      auto it = TA->by_vertex.find(x);
      if (it == TA->by_vertex.end()) continue;
      arow = it->second;
    } else {
      arow.push_back({C.bit(x), 1});
    }
    for_each_edge_entry(C, B.edge_ann, tabs, a, b, x, [&](int32_t y, Mask m2, u128 v2) {
      std::vector<std::pair<Mask, u128>> brow;
      if (TB) {
        auto it = TB->by_vertex.find(y);
        if (it == TB->by_vertex.end()) return;
        brow = it->second;
      } else {
        brow.push_back({C.bit(y), 1});
      }
      for (auto &ea : arow) {
        if ((ea.first & m2) != C.bit(x)) continue;
        for (auto &eb : brow) {
          if ((eb.first & m2) != C.bit(y)) continue;
          if (ea.first & eb.first) continue;
          out.u[ukey(x, ea.first | m2 | eb.first)] += ea.second * v2 * eb.second;
        }
      }
    });
  }
}

static bool table_overflow(const Table &t) {
  for (auto &e : t.u) if (e.second > U64MAX) return true;
  for (auto &e : t.b) if (e.second > U64MAX) return true;
  return false;
}

static u128 run_dp(Ctx &C, const Decomp &D, std::vector<u128> *per_vertex_root) {
  std::vector<Table> tabs(D.blocks.size());
  u128 root = 0;
  for (size_t i = 0; i < D.blocks.size(); i++) {
    const Block &B = D.blocks[i];
    if (B.kind == B_LEAF) {
      solve_leaf(C, B, tabs, tabs[i]);
    } else if (B.kind == B_CYCLE) {
      u128 dummy = 0;
      solve_cycle(C, B, tabs, tabs[i], dummy);
    } else if (B.kind == B_ROOT_CYCLE) {
      solve_cycle(C, B, tabs, tabs[i], root);
    } else {
      const Table &T = tabs[B.node_ann.begin()->second];
      for (auto &e : T.u) {
        root += e.second;
        if (per_vertex_root) (*per_vertex_root)[ukey_v(e.first)] += e.second;
      }
    }
    if (table_overflow(tabs[i])) C.overflow = true;
    tabs[i].index();
  }
  if (root > U64MAX) C.overflow = true;
  return root;
}

// Degree order of Section 5.1: ascending degree, ties by the smaller id first.
static std::vector<int64_t> degree_rank(const DGraph &g) {
  std::vector<int32_t> ord((size_t)g.n);
  for (int64_t v = 0; v < g.n; v++) ord[v] = (int32_t)v;
  std::stable_sort(ord.begin(), ord.end(), [&](int32_t x, int32_t y) {
    return g.adj[x].size() < g.adj[y].size();
  });
  std::vector<int64_t> rank((size_t)g.n);
  for (int64_t i = 0; i < g.n; i++) rank[ord[i]] = i;
  return rank;
}

// order_kind: 0 = PS (no order, one split), 1 = degree order, 2 = id order,
// 3 = caller-supplied rank array.
// choice/n_choice: decomposition choices (see decompose).
// per_source (optional, length n): root-cycle count by highest vertex, or the
// root-node table sum per vertex for a singleton root.
// root_filter (optional, length n, 0/1): restrict the root cycle's highest vertex.
extern "C" int or_dp_count(int64_t n, const int64_t *row_ptr, const int32_t *col, int k, int ne,
                           const int32_t *qedges, const uint8_t *colors, int order_kind,
                           const int64_t *rank_in, const int32_t *choice, int n_choice,
                           const uint8_t *root_filter, uint64_t *per_source128, uint64_t *out128,
                           int *overflow, double *dp_seconds) {
  DGraph g;
  QGraph q;
  if (!load_query(q, k, ne, qedges)) return -1;
  load_graph(g, n, row_ptr, col);
  std::vector<int> ch(choice, choice + (choice ? n_choice : 0));
  Decomp D = decompose(q, ch, nullptr);
  if (!D.ok) return -2;
  std::vector<int64_t> rank;
  if (order_kind == 1) rank = degree_rank(g);
  else if (order_kind == 2) { rank.resize((size_t)n); for (int64_t v = 0; v < n; v++) rank[v] = v; }
  else if (order_kind == 3) rank.assign(rank_in, rank_in + n);
  Ctx C;
  C.g = &g;
  C.q = &q;
  C.col = colors;
  C.rank = order_kind == 0 ? nullptr : &rank;
  std::vector<char> filt;
  if (root_filter) {
    filt.assign(root_filter, root_filter + n);
    C.root_sources = &filt;
  }
  std::vector<u128> ps;
  if (per_source128) {
    ps.assign((size_t)n, 0);
    C.per_source = &ps;
  }
  auto t0 = std::chrono::steady_clock::now();
  u128 r = run_dp(C, D, per_source128 ? &ps : nullptr);
  if (dp_seconds)
    *dp_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  put128(r, out128);
  if (per_source128)
    for (int64_t v = 0; v < n; v++) put128(ps[v], per_source128 + 2 * v);
  *overflow = C.overflow ? 1 : 0;
  return 0;
}

// Decomposition inspection: number of steps and candidates per step for a
// choice sequence; blocks written as (kind, n_nodes, nodes..., n_bd, bd...,
// n_children, children...) records.  Returns the number of blocks, -1 for
// an invalid query, -2 when no decomposition exists (treewidth > 2).
extern "C" int or_decompose(int k, int ne, const int32_t *qedges, const int32_t *choice,
                            int n_choice, int32_t *n_cand_out, int max_steps, int32_t *blocks_out,
                            int max_words, int32_t *root_out) {
  QGraph q;
  if (!load_query(q, k, ne, qedges)) return -1;
  std::vector<int> ch(choice, choice + (choice ? n_choice : 0)), nc;
  Decomp D = decompose(q, ch, &nc);
  for (int i = 0; i < max_steps; i++) n_cand_out[i] = i < (int)nc.size() ? nc[i] : 0;
  if (!D.ok) return -2;
  int w = 0;
  auto put = [&](int32_t x) { if (w < max_words) blocks_out[w] = x; w++; };
  for (auto &B : D.blocks) {
    put(B.kind);
    put((int32_t)B.nodes.size());
    for (int x : B.nodes) put(x);
    put((int32_t)B.boundary.size());
    for (int x : B.boundary) put(x);
    std::vector<int> kids;
    for (auto &e : B.node_ann) kids.push_back(e.second);
    for (auto &e : B.edge_ann) kids.push_back(e.second.block);
    put((int32_t)kids.size());
    for (int x : kids) put(x);
  }
  *root_out = D.root;
  return (int)D.blocks.size();
}

// Structural work of the DB procedure on a plain (unannotated) root cycle of
// length L with k colours, in edge-subset updates: for each source u and each
// half (depth floor(L/2) and ceil(L/2)), level sets L_0 = {u},
// L_{j+1} = lower-than-u neighbours of L_j; extending level j scans
// sum_{v in L_j} |{w in N(v): w < u}| edges, each against C(k-2, j-1) signature
// slots (level 0: one slot).  One highest-node choice (rotations of a plain
// cycle give equal counts).  A source with fewer than two lower neighbours
// closes no cycle and does no work.  Independent of the colouring.
// source_filter (nullable): only these sources; per_source (nullable): units by u;
// scans (nullable, 8 entries): edges scanned out of level j, both halves summed
// (the CSR reads behind the units).
extern "C" double or_cycle_units(int64_t n, const int64_t *row_ptr, const int32_t *col, int L, int k,
                                 const uint8_t *source_filter, double *per_source, double *scans) {
  DGraph g;
  load_graph(g, n, row_ptr, col);
  std::vector<int64_t> rank = degree_rank(g);
  auto binom = [](int a, int b) -> double {
    if (b < 0 || b > a) return 0.0;
    double r = 1;
    for (int i = 1; i <= b; i++) r = r * (a - b + i) / i;
    return r;
  };
  double total = 0;
  std::vector<int64_t> mark((size_t)n, -1);
  for (int64_t u = 0; u < n; u++) {
    if (source_filter && !source_filter[u]) continue;
    int lower = 0;
    for (int32_t w : g.adj[u]) lower += rank[w] < rank[u];
    if (lower < 2) continue;
    double mine = 0;
    for (int half = 0; half < 2; half++) {
      int depth = half == 0 ? L / 2 : L - L / 2;
      std::vector<int32_t> level{(int32_t)u};
      for (int j = 0; j < depth; j++) {
        double slots = j == 0 ? 1.0 : binom(k - 2, j - 1);
        std::vector<int32_t> next;
        int64_t tag = (int64_t)u * 16 + half * 8 + j;
        for (int32_t v : level)
          for (int32_t w : g.adj[v]) {
            if (rank[w] >= rank[u]) continue;
            mine += slots;
            if (scans && j < 8) scans[j] += 1.0;
            if (mark[w] != tag) { mark[w] = tag; next.push_back(w); }
          }
        level.swap(next);
      }
    }
    total += mine;
    if (per_source) per_source[u] = mine;
  }
  return total;
}
