// Graph partitioner for the non-overlapping partition Omega_Ii of Section 2.  The paper obtains it by
// applying ParMETIS to the graph of A^T + A (Section 4); this is a host-side multilevel recursive
// bisection of the same graph, written for this library:
//   - the graph: the off-diagonal pattern of A + A^T, unit vertex and edge weights;
//   - coarsening: heavy-edge matching (vertices visited in a seeded pseudo-random order, each matched
//     to its unmatched neighbour of largest edge weight), contracted until the graph is small or stops
//     shrinking;
//   - initial bisection of the coarsest graph: breadth-first growing from several start vertices, each
//     refined, the best cut kept;
//   - uncoarsening: the bisection projected level by level, each level refined by Fiduccia-Mattheyses
//     passes (single-vertex moves by gain, a balance window, roll-back to the best state seen);
//   - k parts: the vertex set split in the ratio floor(k/2) : ceil(k/2) and each side split again.
// Host code only: no kernels, no device memory.

#include "a2ls_internal.cuh"

#include <algorithm>
#include <cstdint>
#include <future>
#include <limits>
#include <new>
#include <numeric>
#include <queue>
#include <system_error>
#include <utility>
#include <vector>

namespace a2ls {
namespace {

// weighted undirected graph in CSR form (each edge stored in both directions, no self-loops)
struct WGraph {
  int n = 0;
  std::vector<int64_t> xadj;  // n + 1
  std::vector<int> adj;       // neighbours
  std::vector<int> ew;        // edge weights, parallel to adj
  std::vector<int> vw;        // vertex weights
  int64_t total_vw() const { return std::accumulate(vw.begin(), vw.end(), (int64_t)0); }
};

// splitmix64: a seeded order of the vertices for the matching
uint64_t mix64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

// graph of A + A^T from the CSR pattern of A (diagonal entries dropped, duplicates merged)
WGraph symmetrised_graph(int n, const int32_t* rowptr, const int32_t* colind) {
  WGraph g;
  g.n = n;
  std::vector<int64_t> deg(n, 0);
  for (int i = 0; i < n; ++i)
    for (int64_t q = rowptr[i]; q < rowptr[i + 1]; ++q) {
      const int j = colind[q];
      if (j == i) continue;
      ++deg[i];
      ++deg[j];
    }
  std::vector<int64_t> start(n + 1, 0);
  for (int i = 0; i < n; ++i) start[i + 1] = start[i] + deg[i];
  std::vector<int> raw(start[n]);
  std::vector<int64_t> fill(start.begin(), start.end() - 1);
  for (int i = 0; i < n; ++i)
    for (int64_t q = rowptr[i]; q < rowptr[i + 1]; ++q) {
      const int j = colind[q];
      if (j == i) continue;
      raw[fill[i]++] = j;
      raw[fill[j]++] = i;
    }
  g.xadj.assign(n + 1, 0);
  g.adj.reserve(raw.size());
  for (int i = 0; i < n; ++i) {
    auto b = raw.begin() + start[i], e = raw.begin() + start[i + 1];
    std::sort(b, e);
    e = std::unique(b, e);
    g.adj.insert(g.adj.end(), b, e);
    g.xadj[i + 1] = (int64_t)g.adj.size();
  }
  g.ew.assign(g.adj.size(), 1);
  g.vw.assign(n, 1);
  return g;
}

// subgraph induced by the vertices with side[v] == s; gid maps its vertices to the parent's
WGraph induced(const WGraph& g, const std::vector<int8_t>& side, int s, std::vector<int>& gid) {
  std::vector<int> local(g.n, -1);
  gid.clear();
  for (int v = 0; v < g.n; ++v)
    if (side[v] == s) {
      local[v] = (int)gid.size();
      gid.push_back(v);
    }
  WGraph h;
  h.n = (int)gid.size();
  h.xadj.assign(h.n + 1, 0);
  h.adj.reserve(g.adj.size());
  h.ew.reserve(g.adj.size());
  h.vw.resize(h.n);
  for (int a = 0; a < h.n; ++a) {
    const int v = gid[a];
    h.vw[a] = g.vw[v];
    for (int64_t q = g.xadj[v]; q < g.xadj[v + 1]; ++q) {
      const int u = local[g.adj[q]];
      if (u < 0) continue;
      h.adj.push_back(u);
      h.ew.push_back(g.ew[q]);
    }
    h.xadj[a + 1] = (int64_t)h.adj.size();
  }
  return h;
}

// heavy-edge matching and contraction: returns the coarse graph, cmap[v] = coarse vertex of v; no
// coarse vertex weighs more than max_vw (unless a fine one does)
WGraph coarsen(const WGraph& g, uint64_t seed, int64_t max_vw, std::vector<int>& cmap) {
  std::vector<int> order(g.n);
  std::iota(order.begin(), order.end(), 0);
  uint64_t state = seed;
  for (int v = g.n - 1; v > 0; --v) {  // Fisher-Yates shuffle driven by splitmix64
    state = mix64(state);
    std::swap(order[v], order[(int)(state % (uint64_t)(v + 1))]);
  }
  std::vector<int> match(g.n, -1);
  for (int v : order) {
    if (match[v] >= 0) continue;
    int best = v, bw = -1;
    for (int64_t q = g.xadj[v]; q < g.xadj[v + 1]; ++q) {
      const int u = g.adj[q];
      if (match[u] >= 0 || (int64_t)g.vw[v] + g.vw[u] > max_vw) continue;
      // heaviest edge; ties to the lighter vertex (keeps coarse weights even)
      if (g.ew[q] > bw || (g.ew[q] == bw && g.vw[u] < g.vw[best])) {
        best = u;
        bw = g.ew[q];
      }
    }
    match[v] = best;
    match[best] = v;
  }
  cmap.assign(g.n, -1);
  int nc = 0;
  for (int v = 0; v < g.n; ++v)
    if (cmap[v] < 0) {
      cmap[v] = nc;
      cmap[match[v]] = nc;
      ++nc;
    }
  WGraph c;
  c.n = nc;
  c.xadj.assign(nc + 1, 0);
  c.vw.assign(nc, 0);
  c.adj.reserve(g.adj.size());
  c.ew.reserve(g.adj.size());
  std::vector<int> slot(nc, -1);  // position of a coarse neighbour in the row being built
  std::vector<int> members;
  members.reserve(2);
  for (int v = 0, cv = 0; v < g.n; ++v) {
    if (cmap[v] != cv) continue;  // each coarse vertex built once, from its first fine vertex
    members.clear();
    members.push_back(v);
    if (match[v] != v) members.push_back(match[v]);
    const int64_t row0 = (int64_t)c.adj.size();
    for (int m : members) {
      c.vw[cv] += g.vw[m];
      for (int64_t q = g.xadj[m]; q < g.xadj[m + 1]; ++q) {
        const int cu = cmap[g.adj[q]];
        if (cu == cv) continue;
        if (slot[cu] < 0) {
          slot[cu] = (int)(c.adj.size() - row0);
          c.adj.push_back(cu);
          c.ew.push_back(g.ew[q]);
        } else {
          c.ew[row0 + slot[cu]] += g.ew[q];
        }
      }
    }
    for (int64_t q = row0; q < (int64_t)c.adj.size(); ++q) slot[c.adj[q]] = -1;
    c.xadj[cv + 1] = (int64_t)c.adj.size();
    ++cv;
  }
  return c;
}


// Bisection state: side[v] in {0, 1}, the weight of side 0 and the cut (sum of the weights of the
// edges between the sides).  The balance window [lo, hi] bounds the weight of side 0.
struct Bisection {
  std::vector<int8_t> side;
  int64_t w0 = 0;
  int64_t cut = 0;
};

int64_t excess(int64_t w0, int64_t lo, int64_t hi) { return w0 < lo ? lo - w0 : (w0 > hi ? w0 - hi : 0); }

void evaluate(const WGraph& g, Bisection& b) {
  b.w0 = 0;
  b.cut = 0;
  for (int v = 0; v < g.n; ++v) {
    if (b.side[v] == 0) b.w0 += g.vw[v];
    for (int64_t q = g.xadj[v]; q < g.xadj[v + 1]; ++q)
      if (b.side[g.adj[q]] != b.side[v]) b.cut += g.ew[q];
  }
  b.cut /= 2;
}

// Fiduccia-Mattheyses refinement.  A pass moves one unlocked vertex at a time: while side 0 is outside
// the window, the best-gain vertex of the heavy side; otherwise the best-gain vertex whose move keeps
// side 0 inside the window.  The pass stops after `patience` moves without a better state and rolls
// back to the best state, ordered by (distance outside the window, cut).  Passes repeat while they
// improve, at most max_passes.  Gains (cut decrease if v changes side) are computed once and kept up
// to date through the moves and the roll-backs.
void fm_refine(const WGraph& g, Bisection& b, int64_t lo, int64_t hi, int max_passes) {
  const int n = g.n;
  if (n < 2) return;
  std::vector<int64_t> gain(n), degw(n);
  for (int v = 0; v < n; ++v) {
    int64_t ext = 0, in = 0;
    for (int64_t q = g.xadj[v]; q < g.xadj[v + 1]; ++q) (b.side[g.adj[q]] != b.side[v] ? ext : in) += g.ew[q];
    gain[v] = ext - in;
    degw[v] = ext + in;
  }
  std::vector<char> locked(n);
  std::vector<int> moved;
  const int patience = std::max(50, std::min(1000, n / 10));
  using Item = std::pair<int64_t, int>;
  // v changes side: gains of v and its neighbours follow
  auto flip = [&](int v) {
    const int s = b.side[v];
    b.side[v] = (int8_t)(1 - s);
    b.w0 += s == 0 ? -g.vw[v] : g.vw[v];
    b.cut -= gain[v];
    gain[v] = -gain[v];
    for (int64_t q = g.xadj[v]; q < g.xadj[v + 1]; ++q) {
      const int u = g.adj[q];
      // u's edge to v was internal (u on s) and is now cut, or the reverse
      gain[u] += b.side[u] == s ? 2 * (int64_t)g.ew[q] : -2 * (int64_t)g.ew[q];
    }
  };
  for (int pass = 0; pass < max_passes; ++pass) {
    // candidates: the boundary vertices (ext > 0, i.e. gain > -degw), or every vertex while side 0 is
    // outside the window (a heavy side need not touch the boundary, e.g. a component of its own);
    // interior vertices enter the heaps when a neighbour moves
    std::vector<Item> init[2];
    const bool all = excess(b.w0, lo, hi) > 0;
    for (int v = 0; v < n; ++v)
      if (all || gain[v] > -degw[v]) init[b.side[v]].push_back({gain[v], v});
    std::priority_queue<Item> heap[2] = {std::priority_queue<Item>(std::less<Item>(), std::move(init[0])),
                                         std::priority_queue<Item>(std::less<Item>(), std::move(init[1]))};
    std::fill(locked.begin(), locked.end(), 0);
    moved.clear();
    int64_t best_ex = excess(b.w0, lo, hi), best_cut = b.cut;
    size_t best_len = 0;
    int since = 0;
    auto top = [&](int s) -> int {  // best unlocked vertex on side s (stale entries dropped)
      while (!heap[s].empty()) {
        const Item it = heap[s].top();
        const int v = it.second;
        if (!locked[v] && b.side[v] == s && gain[v] == it.first) return v;
        heap[s].pop();
      }
      return -1;
    };
    while (since < patience) {
      const int v0 = top(0), v1 = top(1);
      const int64_t w0 = b.w0;
      int v = -1;
      if (w0 > hi) {
        v = v0;
      } else if (w0 < lo) {
        v = v1;
      } else {
        const bool ok0 = v0 >= 0 && w0 - g.vw[v0] >= lo;
        const bool ok1 = v1 >= 0 && w0 + g.vw[v1] <= hi;
        if (ok0 && ok1)
          v = gain[v0] >= gain[v1] ? v0 : v1;
        else if (ok0)
          v = v0;
        else if (ok1)
          v = v1;
      }
      if (v < 0) break;
      heap[b.side[v]].pop();
      flip(v);
      locked[v] = 1;
      moved.push_back(v);
      for (int64_t q = g.xadj[v]; q < g.xadj[v + 1]; ++q) {
        const int u = g.adj[q];
        if (!locked[u]) heap[b.side[u]].push({gain[u], u});
      }
      const int64_t ex = excess(b.w0, lo, hi);
      if (ex < best_ex || (ex == best_ex && b.cut < best_cut)) {
        best_ex = ex;
        best_cut = b.cut;
        best_len = moved.size();
        since = 0;
      } else {
        ++since;
      }
    }
    for (size_t k = moved.size(); k > best_len; --k) flip(moved[k - 1]);  // roll back past the best state
    if (best_len == 0) break;
  }
}

// breadth-first order of all vertices, starting at r and restarting at the lowest unvisited vertex
// for the other components; *first receives the size of r's component, *ecc its number of levels
void bfs_order(const WGraph& g, int r, std::vector<int>& order, size_t* first = nullptr, int* ecc = nullptr) {
  std::vector<int> level(g.n, -1);
  order.clear();
  int next = 0;
  for (int root = r;;) {
    level[root] = 0;
    size_t head = order.size();
    order.push_back(root);
    while (head < order.size()) {
      const int v = order[head++];
      for (int64_t q = g.xadj[v]; q < g.xadj[v + 1]; ++q) {
        const int u = g.adj[q];
        if (level[u] < 0) {
          level[u] = level[v] + 1;
          order.push_back(u);
        }
      }
    }
    if (root == r) {
      if (first) *first = order.size();
      if (ecc) *ecc = level[order.back()];
    }
    while (next < g.n && level[next] >= 0) ++next;
    if (next >= g.n) break;
    root = next;
  }
}

// a vertex far from the others of its component (George and Liu's pseudo-peripheral node): BFS again
// from the last vertex reached while the number of levels grows
int pseudo_peripheral(const WGraph& g, int start) {
  std::vector<int> order;
  int r = start, ecc = -1;
  for (int it = 0; it < 8; ++it) {
    size_t comp = 0;
    int e = 0;
    bfs_order(g, r, order, &comp, &e);
    if (e <= ecc) break;
    ecc = e;
    r = order[comp - 1];
  }
  return r;
}

constexpr int COARSE_TARGET = 120;  // coarsening stops at this many vertices
constexpr int INIT_TRIES = 8;       // start vertices of the initial bisection
constexpr int FM_PASSES = 8;
constexpr int PARALLEL_DEPTH = 4;       // recursion levels whose halves run concurrently (up to 16 threads)
constexpr int PARALLEL_MIN_N = 20000;   // smaller subgraphs stay on the calling thread

// Multilevel bisection of g: side 0 gets the weight share k0 / k of the total, within
// tol = max(1, W / (50 k)) (2 % of an average final part), and at least k0 vertices while side 1
// keeps at least k - k0 (the finest level has unit weights, so every final part stays non-empty).
std::vector<int8_t> ml_bisect(const WGraph& g, int k0, int k, uint64_t seed) {
  const int64_t W = g.total_vw();
  const int64_t tW = (W * k0 + k / 2) / k;
  const int64_t tol = std::max<int64_t>(1, W / (50 * (int64_t)k));
  const int64_t lo = std::max<int64_t>(k0, tW - tol), hi = std::min<int64_t>(W - (k - k0), tW + tol);
  // coarsening
  std::vector<WGraph> levels;
  std::vector<std::vector<int>> cmaps;
  const int64_t max_vw = std::max<int64_t>(2, (3 * W) / (2 * COARSE_TARGET));
  const WGraph* cur = &g;
  for (int l = 0; cur->n > COARSE_TARGET && l < 64; ++l) {
    std::vector<int> cmap;
    WGraph c = coarsen(*cur, mix64(seed + 0x51ull * (uint64_t)(l + 1)), max_vw, cmap);
    if (c.n > cur->n - cur->n / 20) break;  // shrinks by less than 5 %: stop
    levels.push_back(std::move(c));
    cmaps.push_back(std::move(cmap));
    cur = &levels.back();
  }
  // window of a level: the finest level's [lo, hi]; a coarse level's widened to its heaviest vertex
  auto window = [&](const WGraph& h, int64_t& wlo, int64_t& whi) {
    if (&h == &g) {
      wlo = lo;
      whi = hi;
      return;
    }
    const int64_t t = std::max<int64_t>(tol, *std::max_element(h.vw.begin(), h.vw.end()));
    wlo = std::max<int64_t>(0, tW - t);
    whi = std::min<int64_t>(W, tW + t);
  };
  // initial bisection of the coarsest graph: BFS growing from several starts, each refined
  const WGraph& gc = *cur;
  int64_t clo, chi;
  window(gc, clo, chi);
  Bisection best;
  int64_t best_ex = std::numeric_limits<int64_t>::max(), best_cut = 0;
  std::vector<int> order;
  for (int t = 0; t < std::min(INIT_TRIES, gc.n); ++t) {
    const int start = t == 0 ? pseudo_peripheral(gc, 0) : (int)(((int64_t)t * gc.n) / INIT_TRIES);
    bfs_order(gc, start, order);
    Bisection b;
    b.side.assign(gc.n, 1);
    int64_t w0 = 0;
    for (int v : order) {
      if (w0 >= tW) break;
      b.side[v] = 0;
      w0 += gc.vw[v];
    }
    evaluate(gc, b);
    fm_refine(gc, b, clo, chi, FM_PASSES);
    const int64_t ex = excess(b.w0, clo, chi);
    if (ex < best_ex || (ex == best_ex && b.cut < best_cut)) {
      best_ex = ex;
      best_cut = b.cut;
      best = b;
    }
  }
  // uncoarsening: project to the next finer level and refine there
  for (int l = (int)levels.size() - 1; l >= 0; --l) {
    const WGraph& fine = l == 0 ? g : levels[l - 1];
    Bisection b;
    b.side.resize(fine.n);
    for (int v = 0; v < fine.n; ++v) b.side[v] = best.side[cmaps[l][v]];
    evaluate(fine, b);
    int64_t flo, fhi;
    window(fine, flo, fhi);
    fm_refine(fine, b, flo, fhi, FM_PASSES);
    best = std::move(b);
  }
  return best.side;
}

// k-way partition by recursive bisection: parts first .. first + k - 1 for the vertices of g, whose
// original numbers are orig.  The two halves are independent (own seeds, disjoint entries of part):
// near the top of the recursion the first runs on a thread of its own, so the result does not depend
// on the scheduling.
void recursive_bisection(const WGraph& g, const std::vector<int>& orig, int k, int first, uint64_t seed,
                         int32_t* part, int depth) {
  if (k == 1) {
    for (int v = 0; v < g.n; ++v) part[orig[v]] = first;
    return;
  }
  const int k0 = k / 2;
  const std::vector<int8_t> side = ml_bisect(g, k0, k, seed);
  auto half = [&, side](int s) {
    std::vector<int> gid;
    const WGraph h = induced(g, side, s, gid);
    std::vector<int> horig(gid.size());
    for (size_t a = 0; a < gid.size(); ++a) horig[a] = orig[gid[a]];
    recursive_bisection(h, horig, s == 0 ? k0 : k - k0, s == 0 ? first : first + k0, mix64(seed + 2 + s), part,
                        depth + 1);
  };
  std::future<void> f0;
  if (depth < PARALLEL_DEPTH && g.n >= PARALLEL_MIN_N) {
    try {
      f0 = std::async(std::launch::async, half, 0);
    } catch (const std::system_error&) {  // no thread to be had: the calling thread does both halves
    }
  }
  if (!f0.valid()) half(0);
  half(1);
  if (f0.valid()) f0.get();  // rethrows a failure of the other half
}

// Connected parts where the graph allows it: a part whose vertices fall into several pieces
// (connected components of its induced subgraph; Fiduccia-Mattheyses moves can cut a part in two)
// keeps its largest piece, and every other piece that touches another part moves to the part it
// shares the most edges with (ties to the lower part number).  A piece that is a whole component of
// the graph stays.  Repeated until nothing moves (at most 8 rounds); no part loses its largest piece,
// so none becomes empty.
void connect_parts(const WGraph& g, int nparts, int32_t* part) {
  std::vector<int> comp(g.n), order(g.n), start, size, owner, largest(nparts);
  std::vector<int64_t> links(nparts, 0);
  std::vector<int> touched;
  for (int round = 0; round < 8; ++round) {
    std::fill(comp.begin(), comp.end(), -1);
    start.clear();
    size.clear();
    owner.clear();
    size_t tail = 0;
    for (int r = 0; r < g.n; ++r) {
      if (comp[r] >= 0) continue;
      const int c = (int)size.size();
      const size_t head0 = tail;
      comp[r] = c;
      order[tail++] = r;
      for (size_t head = head0; head < tail; ++head) {
        const int v = order[head];
        for (int64_t q = g.xadj[v]; q < g.xadj[v + 1]; ++q) {
          const int u = g.adj[q];
          if (comp[u] < 0 && part[u] == part[r]) {
            comp[u] = c;
            order[tail++] = u;
          }
        }
      }
      start.push_back((int)head0);
      size.push_back((int)(tail - head0));
      owner.push_back(part[r]);
    }
    std::fill(largest.begin(), largest.end(), -1);
    for (int c = 0; c < (int)size.size(); ++c)
      if (largest[owner[c]] < 0 || size[c] > size[largest[owner[c]]]) largest[owner[c]] = c;
    bool moved = false;
    for (int c = 0; c < (int)size.size(); ++c) {
      if (largest[owner[c]] == c) continue;
      touched.clear();
      for (int a = start[c]; a < start[c] + size[c]; ++a) {
        const int v = order[a];
        for (int64_t q = g.xadj[v]; q < g.xadj[v + 1]; ++q) {
          const int pu = part[g.adj[q]];
          if (pu == owner[c]) continue;
          if (links[pu] == 0) touched.push_back(pu);
          links[pu] += g.ew[q];
        }
      }
      int best = -1;
      for (int pu : touched)
        if (best < 0 || links[pu] > links[best] || (links[pu] == links[best] && pu < best)) best = pu;
      for (int pu : touched) links[pu] = 0;
      if (best < 0) continue;  // a component of the graph on its own
      for (int a = start[c]; a < start[c] + size[c]; ++a) part[order[a]] = best;
      moved = true;
    }
    if (!moved) break;
  }
}

}  // namespace

void partition_graph(int32_t n, const int32_t* rowptr, const int32_t* colind, int32_t nparts, uint64_t seed,
                     int32_t* part) {
  if (n < 1 || !rowptr || !part || (rowptr[n] > 0 && !colind))
    fail(A2LS_ERR_ARG, "a2ls_partition: n = %d must be positive and rowptr, colind, part non-NULL", n);
  if (nparts < 1 || nparts > n) fail(A2LS_ERR_ARG, "a2ls_partition: nparts = %d must lie in [1, n = %d]", nparts, n);
  if (rowptr[0] != 0) fail(A2LS_ERR_ARG, "a2ls_partition: rowptr[0] = %d, expected 0", rowptr[0]);
  for (int i = 0; i < n; ++i)
    if (rowptr[i + 1] < rowptr[i]) fail(A2LS_ERR_ARG, "a2ls_partition: rowptr decreases at row %d", i);
  for (int64_t q = 0; q < rowptr[n]; ++q)
    if (colind[q] < 0 || colind[q] >= n)
      fail(A2LS_ERR_ARG, "a2ls_partition: colind[%lld] = %d outside [0, %d)", (long long)q, colind[q], n);
  std::fill(part, part + n, -1);
  try {
    const WGraph g = symmetrised_graph(n, rowptr, colind);
    std::vector<int> orig(n);
    std::iota(orig.begin(), orig.end(), 0);
    recursive_bisection(g, orig, nparts, 0, mix64(seed), part, 0);
    connect_parts(g, nparts, part);
  } catch (const std::bad_alloc&) {
    fail(A2LS_ERR_OOM, "a2ls_partition: out of host memory (n = %d, %d pattern entries)", n, rowptr[n]);
  }
  std::vector<int64_t> count(nparts, 0);
  for (int i = 0; i < n; ++i) {
    if (part[i] < 0 || part[i] >= nparts) fail(A2LS_ERR_STATE, "a2ls_partition: vertex %d left unassigned", i);
    ++count[part[i]];
  }
  for (int p = 0; p < nparts; ++p)
    if (count[p] == 0) fail(A2LS_ERR_STATE, "a2ls_partition: part %d came out empty", p);
}

}  // namespace a2ls
