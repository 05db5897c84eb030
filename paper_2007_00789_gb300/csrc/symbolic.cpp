// Symbolic phase of spaND on grid problems (host, C++).
//
// Builds the multilevel partition that the spaND algorithm (§3) runs on:
// geometric nested dissection of the coordinate box, then, for every stage
// k, the clusters alive at the stage start (interiors = the level-k
// separators or leaves, interfaces = pieces of the higher separators), their
// block adjacency before and after the interior eliminations (fill), a greedy
// colouring of the interfaces for the sparsification order, and the merge map
// to stage k+1.
//
// Partition rule.  The node at depth d cuts coordinate (d mod dim) at the
// floor(cnt/2)-th smallest distinct coordinate value of its box; the vertices
// on the cut are its separator (level nlevels-1-d), the others go to the lower
// (2i+1) or upper (2i+2) child; leaves are at depth nlevels-1 (level 0).  At
// stage k a vertex of level m > k on the separator of node S is keyed by a
// walk down S's lower subtree through the nodes of depth < nlevels-1-k: cuts
// parallel to S send the walk to the upper child unrecorded; other cuts record
// the comparison (0 below, 1 on, 2 above), go down on 0 / 2 and stop on 1.
// Clusters are the distinct (S, key) pairs, numbered in lexicographic order.
// The key is packed two bits per depth, most significant first, so that
// numeric order of (S, packed key) is that lexicographic order.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <limits>
#include <numeric>
#include <thread>
#include <unordered_map>

#include "spand_internal.h"

namespace spand {

static inline int node_depth(int i) { return 31 - __builtin_clz((unsigned)(i + 1)); }


// The distinct values of x in ascending order, in tmp.  Grid coordinates take
// few distinct values, which an open-addressing set collects in one pass; past
// kDistinct distinct values the values are sorted instead.
static void distinct_values(const std::vector<double>& x, std::vector<double>& tmp) {
  constexpr int kDistinct = 2048, kSlots = 4096;  // a power of two, at most half full
  uint64_t keys[kSlots];
  bool used[kSlots] = {};
  int nd = 0;
  bool small = true;
  for (double v : x) {
    if (v == 0.0) v = 0.0;  // -0 and +0 are one value
    uint64_t b;
    std::memcpy(&b, &v, sizeof b);
    uint32_t h = (uint32_t)((b * 0x9E3779B97F4A7C15ull) >> 52);
    while (used[h] && keys[h] != b) h = (h + 1) & (kSlots - 1);
    if (!used[h]) {
      if (nd == kDistinct) {
        small = false;
        break;
      }
      used[h] = true;
      keys[h] = b;
      ++nd;
    }
  }
  tmp.clear();
  if (small) {
    for (int h = 0; h < kSlots; ++h)
      if (used[h]) {
        double v;
        std::memcpy(&v, &keys[h], sizeof v);
        tmp.push_back(v);
      }
  } else {
    tmp.assign(x.begin(), x.end());
  }
  std::sort(tmp.begin(), tmp.end());
  tmp.erase(std::unique(tmp.begin(), tmp.end()), tmp.end());
}

// The floor(d/2)-th of the d distinct values of x (the cut plane of a box).
static double distinct_median(const std::vector<double>& x, std::vector<double>& tmp) {
  distinct_values(x, tmp);
  return tmp[tmp.size() / 2];
}

int build_tree(const double* coords, int n, int dim, int nlevels, Tree& t, std::string& err) {
  t.n = n;
  t.dim = dim;
  t.nlevels = nlevels;
  t.coords.resize((size_t)n * dim);
  parallel_copy(t.coords.data(), coords, (int64_t)n * dim);
  const int dmax = nlevels - 1;
  const int nint = (1 << dmax) - 1;
  t.cut_dim.assign(std::max(nint, 1), -1);
  t.cut_val.assign(std::max(nint, 1), 0.0);
  t.node_of.assign(n, -1);
  t.level_of.assign(n, -1);
  std::vector<int> verts(n);
  std::iota(verts.begin(), verts.end(), 0);
  // frontier of (node, [begin, end) in a vertex buffer); the boxes of a depth
  // are independent (disjoint vertex slices, their own nodes) and are cut in
  // parallel, each box's children stored at 2i, 2i + 1 as in a serial sweep
  struct Box { int node, b, e; };
  struct Scratch { std::vector<int> lo, hi; std::vector<double> vals, tmp; };
  std::vector<Box> frontier{{0, 0, n}}, next;
  std::vector<Scratch> scratch(16);
  const int nth = std::max(1, std::min(16, (int)std::thread::hardware_concurrency()));
  std::vector<int> vbuf;
  std::vector<std::vector<double>> pvals;
  // A box of the first depths, with fewer boxes than threads, is cut in pieces
  // on all threads: each piece's distinct values (merged into the box's), each
  // piece's lower/upper counts, then both children scattered in vertex order
  // (the serial sweep's order) through vbuf.
  auto cut_in_pieces = [&](int bi, int depth) {
    const Box bx = frontier[bi];
    const int c = depth % dim;
    const int64_t len = bx.e - bx.b;
    const int np = (int)std::max<int64_t>(1, std::min<int64_t>(4 * nth, len / 4096));
    auto piece = [&](int p) { return bx.b + (int)(len * p / np); };
    pvals.resize(np);
    parallel_for(np, [&](int p, int w) {
      std::vector<double>& vals = scratch[w].vals;
      vals.clear();
      for (int i = piece(p); i < piece(p + 1); ++i) vals.push_back(coords[(size_t)verts[i] * dim + c]);
      distinct_values(vals, pvals[p]);
    });
    std::vector<double>& all = scratch[0].vals;
    all.clear();
    for (int p = 0; p < np; ++p) all.insert(all.end(), pvals[p].begin(), pvals[p].end());
    std::sort(all.begin(), all.end());
    all.erase(std::unique(all.begin(), all.end()), all.end());
    const double cut = all[all.size() / 2];
    t.cut_dim[bx.node] = c;
    t.cut_val[bx.node] = cut;
    std::vector<int> nlo(np + 1, 0), nhi(np + 1, 0);
    parallel_for(np, [&](int p, int) {
      int a = 0, h = 0;
      for (int i = piece(p); i < piece(p + 1); ++i) {
        const int v = verts[i];
        const double x = coords[(size_t)v * dim + c];
        if (x < cut) ++a;
        else if (x > cut) ++h;
        else {
          t.node_of[v] = bx.node;
          t.level_of[v] = dmax - depth;
        }
      }
      nlo[p + 1] = a;
      nhi[p + 1] = h;
    });
    for (int p = 0; p < np; ++p) {
      nlo[p + 1] += nlo[p];
      nhi[p + 1] += nhi[p];
    }
    const int tlo = nlo[np], thi = nhi[np];
    vbuf.resize((size_t)tlo + thi);
    parallel_for(np, [&](int p, int) {
      int a = nlo[p], h = tlo + nhi[p];
      for (int i = piece(p); i < piece(p + 1); ++i) {
        const int v = verts[i];
        const double x = coords[(size_t)v * dim + c];
        if (x < cut) vbuf[a++] = v;
        else if (x > cut) vbuf[h++] = v;
      }
    });
    parallel_copy(verts.data() + bx.b, vbuf.data(), (int64_t)tlo + thi);
    next[2 * bi] = {2 * bx.node + 1, bx.b, bx.b + tlo};
    next[2 * bi + 1] = {2 * bx.node + 2, bx.b + tlo, bx.b + tlo + thi};
  };
  for (int depth = 0; depth <= dmax; ++depth) {
    next.assign(2 * frontier.size(), Box{0, 0, 0});
    // the first (lowest) empty box of the depth, as a serial sweep meets it
    std::atomic<int> empty_node(std::numeric_limits<int>::max());
    auto note_empty = [&](int node) {
      int cur = empty_node.load();
      while (node < cur && !empty_node.compare_exchange_weak(cur, node)) {
      }
    };
    if (depth < dmax && (int)frontier.size() < nth) {
      for (int bi = 0; bi < (int)frontier.size(); ++bi) {
        if (frontier[bi].e <= frontier[bi].b) note_empty(frontier[bi].node);
        else cut_in_pieces(bi, depth);
      }
    } else parallel_for((int)frontier.size(), [&](int bi, int w) {
      const Box bx = frontier[bi];
      if (bx.e <= bx.b) {
        note_empty(bx.node);
        return;
      }
      if (depth == dmax) {
        for (int i = bx.b; i < bx.e; ++i) {
          t.node_of[verts[i]] = bx.node;
          t.level_of[verts[i]] = 0;
        }
        return;
      }
      std::vector<int>& lo = scratch[w].lo;
      std::vector<int>& hi = scratch[w].hi;
      std::vector<double>& vals = scratch[w].vals;
      const int c = depth % dim;
      vals.clear();
      for (int i = bx.b; i < bx.e; ++i) vals.push_back(coords[(size_t)verts[i] * dim + c]);
      const double cut = distinct_median(vals, scratch[w].tmp);
      t.cut_dim[bx.node] = c;
      t.cut_val[bx.node] = cut;
      lo.clear();
      hi.clear();
      for (int i = bx.b; i < bx.e; ++i) {
        const int v = verts[i];
        const double x = coords[(size_t)v * dim + c];
        if (x < cut) lo.push_back(v);
        else if (x > cut) hi.push_back(v);
        else {
          t.node_of[v] = bx.node;
          t.level_of[v] = dmax - depth;
        }
      }
      // lower child's vertices, then upper child's, reuse the slice [b, e)
      int p = bx.b;
      for (int v : lo) verts[p++] = v;
      const int mid = p;
      for (int v : hi) verts[p++] = v;
      next[2 * bi] = {2 * bx.node + 1, bx.b, mid};
      next[2 * bi + 1] = {2 * bx.node + 2, mid, p};
    });
    if (empty_node.load() != std::numeric_limits<int>::max()) {
      err = "empty nested-dissection box at node " + std::to_string(empty_node.load());
      return SPAND_EINVAL;
    }
    frontier.swap(next);
  }
  return SPAND_OK;
}

// Packed cluster key of vertex v at stage k (0 for interiors).
static uint64_t vertex_key(const Tree& t, int v, int k) {
  const int ell = t.nlevels;
  const int node = t.node_of[v];
  if (t.level_of[v] <= k) return 0;
  uint64_t key = 0;
  const int sdim = t.cut_dim[node];
  const int limit = ell - 1 - k;
  int cur = 2 * node + 1;
  while (node_depth(cur) < limit) {
    const int cd = t.cut_dim[cur];
    if (cd == sdim) {
      cur = 2 * cur + 2;
      continue;
    }
    const double x = t.coords[(size_t)v * t.dim + cd];
    const double cv = t.cut_val[cur];
    const int cmp = x < cv ? 0 : (x > cv ? 2 : 1);
    const int d = node_depth(cur);
    key |= (uint64_t)(cmp + 1) << (2 * (ell - 1 - d));
    if (cmp == 1) break;
    cur = cmp == 0 ? 2 * cur + 1 : 2 * cur + 2;
  }
  return key;
}

// ---------------------------------------------------------------------------
// Algebraic partition (input without coordinates).  The node at depth d
// bisects its vertex set V by breadth-first distances in the subgraph induced
// on V: a first sweep from the smallest vertex finds the far vertex (smallest
// index at the largest distance), the second sweep's distances from it order
// V by (distance, index) with unreached vertices last; the distance of the
// median (position |V|/2) is the separator, smaller distances the lower child,
// larger ones and unreached vertices the upper child (an unreached median:
// empty separator, the reached vertices form the lower child).  Interfaces
// are keyed by reach: the leaves connected to a separator vertex through
// vertices of lower level; at stage k the key is the set of depth
// nlevels-1-k ancestors of those leaves.
// ---------------------------------------------------------------------------
namespace {

// The boxes of one depth are bisected in parallel.  stamp[v] names the box
// (node + 1) that holds v at the current depth, so a sweep stays inside its
// box; boxes of other threads only ever hold other stamps, and their writes
// are relaxed atomics.  dist is written and read only for the box's own
// vertices.
struct GraphBisector {
  const int32_t* rowptr;
  const int32_t* colind;
  std::vector<std::atomic<int>>& stamp;
  std::vector<std::atomic<int>>& dist;
  std::vector<int> front, next, hist;
  std::vector<std::vector<int>> found;  // per range of a wide level
  int reach_d = 0;                      // the largest distance of the last sweep
  int cur = 0;
  bool wide = false;  // the only box in work: its wide levels run on all threads

  bool inside(int u) const { return stamp[u].load(std::memory_order_relaxed) == cur; }
  int dist_of(int v) const { return dist[v].load(std::memory_order_relaxed); }

  // distances from root within the box (-1: not reached).  A wide level is
  // expanded in ranges on all threads, each vertex claimed by the one thread
  // whose exchange finds it unreached; the distances equal the serial ones
  // (only the order of the next level differs).
  void bfs(int root) {
    constexpr size_t kWide = 8192;  // level size from which it is expanded in parallel
    dist[root].store(0, std::memory_order_relaxed);
    front.assign(1, root);
    reach_d = 0;
    int d = 0;
    while (!front.empty()) {
      next.clear();
      ++d;
      if (!wide || front.size() < kWide) {
        for (int v : front)
          for (int64_t e = rowptr[v]; e < rowptr[v + 1]; ++e) {
            const int u = colind[e];
            if (inside(u) && dist_of(u) < 0) {
              dist[u].store(d, std::memory_order_relaxed);
              next.push_back(u);
            }
          }
      } else {
        const int nr = (int)std::min<size_t>(64, front.size() / 1024);
        found.resize(nr);
        parallel_for(nr, [&](int r, int) {
          std::vector<int>& mine = found[r];
          mine.clear();
          const size_t b = front.size() * r / nr, en = front.size() * (r + 1) / nr;
          for (size_t i = b; i < en; ++i) {
            const int v = front[i];
            for (int64_t e = rowptr[v]; e < rowptr[v + 1]; ++e) {
              const int u = colind[e];
              if (!inside(u) || dist_of(u) >= 0) continue;
              int unreached = -1;
              if (dist[u].compare_exchange_strong(unreached, d, std::memory_order_relaxed)) mine.push_back(u);
            }
          }
        });
        for (const auto& f : found) next.insert(next.end(), f.begin(), f.end());
      }
      if (!next.empty()) reach_d = d;
      front.swap(next);
    }
  }

  void bisect(int box, const std::vector<int>& verts, std::vector<int>& sep, std::vector<int>& lo,
              std::vector<int>& hi) {
    cur = box;
    for (int v : verts) {
      stamp[v].store(cur, std::memory_order_relaxed);
      dist[v].store(-1, std::memory_order_relaxed);
    }
    bfs(verts[0]);
    int far = -1, r1 = -1;
    for (int v : verts)
      if (dist_of(v) > far) {
        far = dist_of(v);
        r1 = v;
      }
    for (int v : verts) dist[v].store(-1, std::memory_order_relaxed);
    bfs(r1);
    // the median key: the (|V|/2)-th smallest distance, unreached vertices
    // last (counted per distance: the keys are levels of the sweep)
    const long big = 1L << 40;
    hist.assign(reach_d + 2, 0);
    for (int v : verts) ++hist[dist_of(v) < 0 ? reach_d + 1 : dist_of(v)];
    long med = big;
    for (int k = 0, below = 0; k <= reach_d; ++k) {
      below += hist[k];
      if (below > (int)verts.size() / 2) {
        med = k;
        break;
      }
    }
    sep.clear();
    lo.clear();
    hi.clear();
    for (int v : verts) {
      const long key = dist_of(v) < 0 ? big : (long)dist_of(v);
      if (med == big) {
        (key < big ? lo : hi).push_back(v);
      } else if (key == med) {
        sep.push_back(v);
      } else {
        (key < med ? lo : hi).push_back(v);
      }
    }
  }
};

inline int ancestor_at(int i, int depth) {
  while (node_depth(i) > depth) i = (i - 1) / 2;
  return i;
}

}  // namespace

int build_tree_graph(const int32_t* rowptr, const int32_t* colind, int n, int nlevels, Tree& t,
                     std::string& err) {
  t.n = n;
  t.dim = 0;
  t.nlevels = nlevels;
  t.algebraic = 1;
  t.coords.clear();
  t.node_of.assign(n, -1);
  t.level_of.assign(n, -1);
  const int dmax = nlevels - 1;
  std::vector<std::atomic<int>> stamp(n);
  parallel_for(n, [&](int v, int) { stamp[v].store(0, std::memory_order_relaxed); }, 65536);
  std::vector<std::atomic<int>> dist(n);
  std::vector<GraphBisector> gb;
  for (int w = 0; w < 16; ++w) gb.push_back(GraphBisector{rowptr, colind, stamp, dist, {}, {}, {}, {}, 0, false});
  const int nth = std::max(1, std::min(16, (int)std::thread::hardware_concurrency()));
  struct Part {
    int node;
    std::vector<int> verts;
  };
  std::vector<Part> frontier, next;
  frontier.push_back({0, {}});
  frontier[0].verts.resize(n);
  std::iota(frontier[0].verts.begin(), frontier[0].verts.end(), 0);
  std::vector<std::vector<int>> seps;
  for (int depth = 0; depth <= dmax; ++depth) {
    // the first (lowest) empty box of the depth, as a serial sweep meets it
    for (const Part& pt : frontier)
      if (pt.verts.empty()) {
        err = "empty nested-dissection subdomain at node " + std::to_string(pt.node);
        return SPAND_EINVAL;
      }
    if (depth == dmax) {
      parallel_for((int)frontier.size(), [&](int bi, int) {
        for (int v : frontier[bi].verts) {
          t.node_of[v] = frontier[bi].node;
          t.level_of[v] = 0;
        }
      });
      break;
    }
    next.assign(2 * frontier.size(), Part{0, {}});
    seps.resize(frontier.size());
    auto cut = [&](int bi, int w) {
      Part& pt = frontier[bi];
      gb[w].bisect(pt.node + 1, pt.verts, seps[bi], next[2 * bi].verts, next[2 * bi + 1].verts);
      for (int v : seps[bi]) {
        t.node_of[v] = pt.node;
        t.level_of[v] = dmax - depth;
      }
      next[2 * bi].node = 2 * pt.node + 1;
      next[2 * bi + 1].node = 2 * pt.node + 2;
      std::vector<int>().swap(pt.verts);
    };
    // fewer boxes than threads (the first depths): one box at a time, its
    // wide sweep levels on all threads; else the boxes in parallel
    const bool few = frontier.size() <= 2 && nth > 2;
    gb[0].wide = few;
    if (few) {
      for (int bi = 0; bi < (int)frontier.size(); ++bi) cut(bi, 0);
    } else {
      parallel_for((int)frontier.size(), cut);
    }
    frontier.swap(next);
  }
  // reach sets, by increasing level (a level's vertices in parallel: they read
  // the finished sets of lower levels only)
  std::vector<std::vector<int>> R(n);
  std::vector<int> lstart(dmax + 2, 0), bylevel(n);
  for (int v = 0; v < n; ++v) ++lstart[t.level_of[v] + 1];
  for (int l = 0; l <= dmax; ++l) lstart[l + 1] += lstart[l];
  {
    std::vector<int> at(lstart.begin(), lstart.end() - 1);
    for (int v = 0; v < n; ++v) bylevel[at[t.level_of[v]]++] = v;
  }
  for (int lvl = 1; lvl <= dmax; ++lvl)
    parallel_for(lstart[lvl + 1] - lstart[lvl], [&](int i, int) {
      const int v = bylevel[lstart[lvl] + i];
      auto& s = R[v];
      for (int64_t e = rowptr[v]; e < rowptr[v + 1]; ++e) {
        const int u = colind[e];
        if (t.level_of[u] == 0) s.push_back(t.node_of[u]);
        else if (t.level_of[u] < lvl) s.insert(s.end(), R[u].begin(), R[u].end());
      }
      std::sort(s.begin(), s.end());
      s.erase(std::unique(s.begin(), s.end()), s.end());
    }, 256);
  t.reach_ptr.assign(n + 1, 0);
  t.width = 1;
  for (int v = 0; v < n; ++v) {
    t.reach_ptr[v + 1] = t.reach_ptr[v] + (int)R[v].size();
    t.width = std::max(t.width, (int)R[v].size());
  }
  t.reach.resize(t.reach_ptr[n]);
  parallel_for(n, [&](int v, int) { std::copy(R[v].begin(), R[v].end(), t.reach.begin() + t.reach_ptr[v]); },
               4096);
  return SPAND_OK;
}

// Stage-k clusters of an algebraic tree: (node, sorted ancestor set padded
// with -1) in lexicographic order.
// Algebraic clusters of stage 0 in (node, key) order, ties by vertex: the
// vertices bucketed by node over contiguous vertex ranges (each node's
// vertices stay ascending), each node's vertices sorted by key (a separator
// vertex's reach, compared as a sequence; leaves have none), then numbered
// node by node.  node_of_cluster, key_of_cluster and members (optional):
// every cluster's node, key and vertices (ascending).
static int stage0_map_graph(const Tree& t, std::vector<int>& cl, std::vector<int>* level_of_cluster,
                            std::vector<int>* node_of_cluster = nullptr,
                            std::vector<std::vector<int>>* key_of_cluster = nullptr,
                            std::vector<std::vector<int>>* members = nullptr) {
  const int n = t.n;
  int nnode = 0;
  for (int v = 0; v < n; ++v) nnode = std::max(nnode, t.node_of[v] + 1);
  // vertex ranges of the counting sort (counts: nodes x ranges, within 8M entries)
  const int np = std::max(1, std::min({32, n / 65536, (1 << 23) / std::max(1, nnode)}));
  auto piece = [&](int p) { return (int)((int64_t)n * p / np); };
  std::vector<int> at((size_t)nnode * np, 0), start(nnode + 1, 0);
  parallel_for(np, [&](int p, int) {
    for (int v = piece(p); v < piece(p + 1); ++v) ++at[(size_t)t.node_of[v] * np + p];
  });
  int total = 0;
  for (int b = 0; b < nnode; ++b) {
    start[b] = total;
    for (int p = 0; p < np; ++p) {
      const int c = at[(size_t)b * np + p];
      at[(size_t)b * np + p] = total;
      total += c;
    }
  }
  start[nnode] = total;
  std::vector<int> order(n);
  parallel_for(np, [&](int p, int) {
    for (int v = piece(p); v < piece(p + 1); ++v) order[at[(size_t)t.node_of[v] * np + p]++] = v;
  });
  const int* R = t.reach.data();
  const int* Rp = t.reach_ptr.data();
  auto key_less = [&](int a, int b) {  // keys of two vertices of one node
    if (t.level_of[a] == 0) return false;  // a leaf's vertices: no keys
    return std::lexicographical_compare(R + Rp[a], R + Rp[a + 1], R + Rp[b], R + Rp[b + 1]);
  };
  auto key_eq = [&](int a, int b) {
    return t.level_of[a] == 0 || std::equal(R + Rp[a], R + Rp[a + 1], R + Rp[b], R + Rp[b + 1]);
  };
  std::vector<int> ncb(nnode + 1, 0);  // clusters of each node, then their prefix
  parallel_for(nnode, [&](int b, int) {
    const auto first = order.begin() + start[b], last = order.begin() + start[b + 1];
    std::sort(first, last, [&](int x, int y) { return key_less(x, y) || (!key_less(y, x) && x < y); });
    int c = 0;
    for (auto it = first; it != last; ++it)
      if (it == first || !key_eq(*it, *(it - 1))) ++c;
    ncb[b + 1] = c;
  }, 256);
  for (int b = 0; b < nnode; ++b) ncb[b + 1] += ncb[b];
  const int ncl = ncb[nnode];
  cl.assign(n, -1);
  if (level_of_cluster) level_of_cluster->assign(ncl, 0);
  if (node_of_cluster) node_of_cluster->assign(ncl, 0);
  if (key_of_cluster) key_of_cluster->assign(ncl, {});
  if (members) members->assign(ncl, {});
  parallel_for(nnode, [&](int b, int) {
    int id = ncb[b] - 1;
    const auto first = order.begin() + start[b], last = order.begin() + start[b + 1];
    for (auto it = first; it != last; ++it) {
      const int v = *it;
      if (it == first || !key_eq(v, *(it - 1))) {
        ++id;
        if (level_of_cluster) (*level_of_cluster)[id] = t.level_of[v];
        if (node_of_cluster) (*node_of_cluster)[id] = b;
        if (key_of_cluster && t.level_of[v] > 0) (*key_of_cluster)[id].assign(R + Rp[v], R + Rp[v + 1]);
      }
      cl[v] = id;
      if (members) (*members)[id].push_back(v);
    }
  }, 256);
  return ncl;
}

// Geometric clusters of stage k in (node, key) order: the live vertices
// counting-sorted by node over contiguous vertex pieces (each node's vertices
// stay ascending), each node's vertices sorted by key, then the clusters
// numbered node by node.  full: -1 for the vertices eliminated before stage
// k, else their entries are left as they were.  node_of_cluster,
// key_of_cluster and members (optional): every cluster's tree node, key and
// vertices (ascending).
struct KeyedVertex {
  uint64_t key;
  int v;
  bool operator<(const KeyedVertex& o) const { return key != o.key ? key < o.key : v < o.v; }
};
static int cluster_map_geo(const Tree& t, int k, std::vector<int>& cl, std::vector<int>* level_of_cluster,
                           bool full, std::vector<int>* node_of_cluster = nullptr,
                           std::vector<uint64_t>* key_of_cluster = nullptr,
                           std::vector<std::vector<int>>* members = nullptr) {
  const int n = t.n;
  const int np0 = std::max(1, std::min(32, n / 65536));
  std::vector<int> pmax(np0, 0);
  parallel_for(np0, [&](int p, int) {
    int mx = 0;
    for (int v = (int)((int64_t)n * p / np0); v < (int)((int64_t)n * (p + 1) / np0); ++v)
      if (t.level_of[v] >= k) mx = std::max(mx, t.node_of[v] + 1);
    pmax[p] = mx;
  });
  const int nnode = *std::max_element(pmax.begin(), pmax.end());
  // vertex ranges of the counting sort: fewer for many nodes, so that the
  // counts (nodes x ranges) stay within 8M entries
  const int np = std::max(1, std::min(np0, (1 << 23) / std::max(1, nnode)));
  auto piece = [&](int p) { return (int)((int64_t)n * p / np); };
  // for every live vertex of piece p in order: fn(v)
  auto each = [&](int p, auto&& fn) {
    for (int v = piece(p); v < piece(p + 1); ++v)
      if (t.level_of[v] >= k) fn(v);
  };
  // at[b * np + p]: vertices of node b in piece p, then where they go
  std::vector<int> at((size_t)nnode * np, 0), start(nnode + 1, 0);
  parallel_for(np, [&](int p, int) { each(p, [&](int v) { ++at[(size_t)t.node_of[v] * np + p]; }); });
  int total = 0;
  for (int b = 0; b < nnode; ++b) {
    start[b] = total;
    for (int p = 0; p < np; ++p) {
      const int c = at[(size_t)b * np + p];
      at[(size_t)b * np + p] = total;
      total += c;
    }
  }
  start[nnode] = total;
  host_vec<KeyedVertex> items(total);
  parallel_for(np, [&](int p, int) {
    each(p, [&](int v) { items[at[(size_t)t.node_of[v] * np + p]++] = {vertex_key(t, v, k), v}; });
  });
  std::vector<int> ncb(nnode + 1, 0);  // clusters of each node, then their prefix
  parallel_for(nnode, [&](int b, int) {
    const auto first = items.begin() + start[b], last = items.begin() + start[b + 1];
    if (!std::is_sorted(first, last)) std::sort(first, last);  // a leaf's: one key, in vertex order
    int c = 0;
    for (auto it = first; it != last; ++it)
      if (it == first || it->key != (it - 1)->key) ++c;
    ncb[b + 1] = c;
  }, 256);
  for (int b = 0; b < nnode; ++b) ncb[b + 1] += ncb[b];
  const int ncl = ncb[nnode];
  if (full) cl.assign(n, -1);
  else cl.resize(n);
  if (level_of_cluster) level_of_cluster->assign(ncl, 0);
  if (node_of_cluster) node_of_cluster->assign(ncl, 0);
  if (key_of_cluster) key_of_cluster->assign(ncl, 0);
  if (members) members->assign(ncl, {});
  parallel_for(nnode, [&](int b, int) {
    int id = ncb[b] - 1;
    const auto first = items.begin() + start[b], last = items.begin() + start[b + 1];
    for (auto it = first; it != last; ++it) {
      if (it == first || it->key != (it - 1)->key) {
        ++id;
        if (level_of_cluster) (*level_of_cluster)[id] = t.level_of[it->v];
        if (node_of_cluster) (*node_of_cluster)[id] = b;
        if (key_of_cluster) (*key_of_cluster)[id] = it->key;
      }
      cl[it->v] = id;
      if (members) (*members)[id].push_back(it->v);
    }
  }, 256);
  return ncl;
}

int stage0_cluster_map(const Tree& t, std::vector<int>& cl) {
  if (t.algebraic) return stage0_map_graph(t, cl, nullptr);
  return cluster_map_geo(t, 0, cl, nullptr, true);
}

int build_stages(const Tree& t, const int32_t* rowptr, const int32_t* colind, int skip,
                 std::vector<StageSym>& st, std::string& err) {
  const int ell = t.nlevels;
  st.assign(ell, StageSym());
  // Only stage 0 maps vertices to clusters, and records every cluster's tree
  // node, key and vertices.  Stage k + 1's clusters are stage k's interfaces grouped by
  // node and by their key at stage k + 1, numbered in (node, key) order as a
  // per-vertex map would number them.  Geometric: the key without its entries
  // of depth nlevels - 2 - k and deeper (a vertex's bisection walk at stage
  // k + 1 is a prefix of its walk at stage k).  Algebraic: the parents of the
  // key's nodes (the depth-d ancestors of the reach are the parents of its
  // depth-(d + 1) ones), empty for the level-(k + 1) separators.
  std::vector<std::vector<int>> maps(ell);
  std::vector<int> nmaps(ell, 0);
  std::vector<int> cnode;
  std::vector<uint64_t> ckey;            // geometric keys
  std::vector<std::vector<int>> gkey;    // algebraic keys
  if (t.algebraic) nmaps[0] = stage0_map_graph(t, maps[0], &st[0].level, &cnode, &gkey, &st[0].members0);
  else nmaps[0] = cluster_map_geo(t, 0, maps[0], &st[0].level, false, &cnode, &ckey, &st[0].members0);
  for (int k = 0; k < ell; ++k) {
    StageSym& S = st[k];
    S.ncl = nmaps[k];
    const std::vector<int>& cl = maps[k];
    S.interior.assign(S.ncl, 0);
    for (int c = 0; c < S.ncl; ++c) {
      if (S.level[c] == k) {
        S.interior[c] = 1;
        S.interiors.push_back(c);
      } else {
        S.ifaces.push_back(c);
      }
    }
    S.sparsify = (k >= skip) && (k < ell - 1);
    S.adj0.assign(S.ncl, {});
    if (k == 0) {
      // S.members0: from the stage-0 map
      // each cluster's neighbours from its own rows (clusters in parallel)
      parallel_for(S.ncl, [&](int a, int) {
        auto& N = S.adj0[a];
        for (int i : S.members0[a])
          for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) {
            const int b = cl[colind[e]];
            if (a != b) N.push_back(b);
          }
        std::sort(N.begin(), N.end());
        N.erase(std::unique(N.begin(), N.end()), N.end());
      }, 256);
    } else {
      StageSym& P = st[k - 1];
      S.children.assign(S.ncl, {});
      for (int p : P.ifaces) S.children[P.parent[p]].push_back(p);
      // a cluster's neighbours: the parents of its children's neighbours
      parallel_for(S.ncl, [&](int a, int) {
        auto& N = S.adj0[a];
        for (int p : S.children[a])
          for (int q : P.adj1[p]) {
            const int b = P.parent[q];
            if (a != b) N.push_back(b);
          }
        std::sort(N.begin(), N.end());
        N.erase(std::unique(N.begin(), N.end()), N.end());
      }, 256);
    }
    for (int s : S.interiors)
      for (int q : S.adj0[s])
        if (S.interior[q]) {
          err = "interiors of stage " + std::to_string(k) + " touch each other";
          return SPAND_EINVAL;
        }
    // adjacency among interfaces after eliminating the interiors (fill)
    // (p's interface neighbours, and every other neighbour of each interior next
    // to p; adj0 is symmetric, so each interface gathers its own list: in parallel)
    S.adj1.assign(S.ncl, {});
    parallel_for((int)S.ifaces.size(), [&](int i, int) {
      const int p = S.ifaces[i];
      auto& N1 = S.adj1[p];
      for (int q : S.adj0[p]) {
        if (!S.interior[q]) {
          N1.push_back(q);
        } else {
          for (int r : S.adj0[q])
            if (r != p) N1.push_back(r);
        }
      }
      std::sort(N1.begin(), N1.end());
      N1.erase(std::unique(N1.begin(), N1.end()), N1.end());
    }, 256);
    // greedy colouring of the interface graph in id order
    S.colour.assign(S.ncl, -1);
    S.ncolours = 0;
    std::vector<int> mark;
    for (int p : S.ifaces) {
      mark.assign(S.adj1[p].size() + 1, 0);
      for (int q : S.adj1[p])
        if (S.colour[q] >= 0 && S.colour[q] < (int)mark.size()) mark[S.colour[q]] = 1;
      int c = 0;
      while (mark[c]) ++c;
      S.colour[p] = c;
      S.ncolours = std::max(S.ncolours, c + 1);
    }
    S.by_colour.assign(S.ncolours, {});
    for (int p : S.ifaces) S.by_colour[S.colour[p]].push_back(p);
    // panel-row block lists
    S.rowsegs.assign(S.ncl, {});
    parallel_for(S.ncl, [&](int c, int) {
      auto& rs = S.rowsegs[c];
      rs = S.interior[c] ? S.adj0[c] : S.adj1[c];
      rs.insert(std::lower_bound(rs.begin(), rs.end(), c), c);
    }, 256);
    // Schur targets (q >= r) and their contributing interiors: the (r, s) of
    // every target row q bucketed by q (sizes counted first, interiors in
    // parallel), each bucket sorted, then the targets numbered in (q, r) order
    {
      std::vector<int64_t> qoff(S.ncl + 1, 0);
      for (int s : S.interiors) {
        const auto& N = S.adj0[s];
        for (size_t a = 0; a < N.size(); ++a) qoff[N[a] + 1] += (int64_t)a + 1;
      }
      for (int q = 0; q < S.ncl; ++q) qoff[q + 1] += qoff[q];
      const int64_t npairs = qoff[S.ncl];
      std::vector<uint64_t> items((size_t)npairs);  // (r << 32) | s
      std::unique_ptr<std::atomic<int64_t>[]> fill(new std::atomic<int64_t>[S.ncl]);
      for (int q = 0; q < S.ncl; ++q) fill[q].store(qoff[q], std::memory_order_relaxed);
      parallel_for((int)S.interiors.size(), [&](int i, int) {
        const int s = S.interiors[i];
        const auto& N = S.adj0[s];
        for (size_t a = 0; a < N.size(); ++a) {
          int64_t f = fill[N[a]].fetch_add((int64_t)a + 1, std::memory_order_relaxed);
          for (size_t b = 0; b <= a; ++b) items[f++] = ((uint64_t)N[b] << 32) | (uint32_t)s;
        }
      }, 256);
      std::vector<int> tq(S.ncl + 1, 0);  // targets of each row q, then their prefix
      parallel_for(S.ncl, [&](int q, int) {
        const auto first = items.begin() + qoff[q], last = items.begin() + qoff[q + 1];
        std::sort(first, last);
        int cnt = 0;
        for (auto it = first; it != last; ++it)
          if (it == first || (*it >> 32) != (*(it - 1) >> 32)) ++cnt;
        tq[q + 1] = cnt;
      }, 256);
      for (int q = 0; q < S.ncl; ++q) tq[q + 1] += tq[q];
      const int ntarget = tq[S.ncl];
      S.schur_q.resize(ntarget);
      S.schur_r.resize(ntarget);
      S.schur_ptr.resize((size_t)ntarget + 1);
      S.schur_s.resize((size_t)npairs);
      parallel_for(S.ncl, [&](int q, int) {
        int tg = tq[q];
        for (int64_t i = qoff[q]; i < qoff[q + 1]; ++i) {
          const int r = (int)(items[i] >> 32);
          if (i == qoff[q] || r != (int)(items[i - 1] >> 32)) {
            S.schur_q[tg] = q;
            S.schur_r[tg] = r;
            S.schur_ptr[tg] = (int)i;
            ++tg;
          }
          S.schur_s[i] = (int)(uint32_t)items[i];
        }
      }, 256);
      S.schur_ptr[ntarget] = (int)npairs;
    }
    // parents at stage k+1
    S.parent.assign(S.ncl, -1);
    if (k + 1 < ell && t.algebraic) {
      const int ni = (int)S.ifaces.size();
      std::vector<std::vector<int>> key2(ni);
      parallel_for(ni, [&](int i, int) {
        const int p = S.ifaces[i];
        if (S.level[p] == k + 1) return;  // separators eliminated at stage k + 1: no key
        auto& kk = key2[i];
        for (int a : gkey[p]) kk.push_back((a - 1) / 2);  // parents stay ascending
        kk.erase(std::unique(kk.begin(), kk.end()), kk.end());
      }, 256);
      std::vector<int> ord(ni);
      std::iota(ord.begin(), ord.end(), 0);
      std::sort(ord.begin(), ord.end(), [&](int x, int y) {
        const int nx = cnode[S.ifaces[x]], ny = cnode[S.ifaces[y]];
        if (nx != ny) return nx < ny;
        if (key2[x] != key2[y]) return key2[x] < key2[y];
        return x < y;
      });
      std::vector<int> node2;
      std::vector<std::vector<int>> gkey2;
      std::vector<int>& level2 = st[k + 1].level;
      level2.clear();
      for (int i = 0; i < ni; ++i) {
        const int x = ord[i], p = S.ifaces[x];
        if (i == 0 || cnode[p] != node2.back() || key2[x] != gkey2.back()) {
          node2.push_back(cnode[p]);
          gkey2.push_back(std::move(key2[x]));
          level2.push_back(S.level[p]);
        }
        S.parent[p] = (int)node2.size() - 1;
      }
      nmaps[k + 1] = (int)node2.size();
      cnode.swap(node2);
      gkey.swap(gkey2);
    } else if (k + 1 < ell) {
      const int drop = 2 * k + 4;  // key bits of the entries of depth nlevels - 2 - k and deeper
      const uint64_t keep = drop >= 64 ? 0 : ~((uint64_t(1) << drop) - 1);
      struct Group {
        int node;
        uint64_t key;
        int p;
        bool operator<(const Group& o) const {
          return node != o.node ? node < o.node : (key != o.key ? key < o.key : p < o.p);
        }
      };
      std::vector<Group> g;
      g.reserve(S.ifaces.size());
      for (int p : S.ifaces) g.push_back({cnode[p], ckey[p] & keep, p});
      std::sort(g.begin(), g.end());
      std::vector<int> node2;
      std::vector<uint64_t> key2;
      std::vector<int>& level2 = st[k + 1].level;
      level2.clear();
      for (size_t i = 0; i < g.size(); ++i) {
        if (i == 0 || g[i].node != g[i - 1].node || g[i].key != g[i - 1].key) {
          node2.push_back(g[i].node);
          key2.push_back(g[i].key);
          level2.push_back(S.level[g[i].p]);
        }
        S.parent[g[i].p] = (int)node2.size() - 1;
      }
      nmaps[k + 1] = (int)node2.size();
      cnode.swap(node2);
      ckey.swap(key2);
    } else if (!S.ifaces.empty()) {
      err = "interfaces left after the last stage";
      return SPAND_EINVAL;
    }
    std::vector<int>().swap(maps[k]);  // no later stage reads it
  }
  return SPAND_OK;
}

}  // namespace spand
