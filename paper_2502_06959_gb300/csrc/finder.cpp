// Automatic joint-cut blocks (Sec. V: the gates crossing the cut are regrouped into
// cascades that can be cut jointly, using the freedom that RZZ gates commute; Sec. IV-D,
// Example 4: a cascade of gates sharing one qubit keeps Schmidt rank 2).
//
//   1. The circuit is split into maximal runs of consecutive gates that are diagonal in
//      the computational basis (RZZ, CZ, RZ, S, T, Z, diagonal matrices): gates of a
//      run commute with one another, so any order of a run is the same circuit.
//   2. In a run, the crossing gates are two-qubit gates with one qubit on each side:
//      edges of a bipartite graph between a-qubits and b-qubits.  A set of hub qubits
//      that touches every edge is a vertex cover; every hub with its edges is one
//      cascade of rank 2, so the joint path count is 2^(number of hubs).  The fewest hubs
//      is a minimum vertex cover, which for a bipartite graph has the size of a maximum
//      matching (Koenig's theorem); it is built from an augmenting-path matching
//      (Kuhn's algorithm) and the alternating-path reachability of the unmatched
//      a-qubits.  (The paper uses a brute-force search; this gives the same optimum.)
//   3. Each edge goes to a hub it touches (the one with more cover edges when both are
//      hubs); a hub's edges form one block, split into blocks of at most `max_leaves`
//      edges (a cascade block may hold up to 8 qubits on the side opposite its hub).  Crossing gates of more than two
//      qubits, or outside diagonal runs, become singleton blocks (plain cuts).
//   4. Every run is reordered: its in-half gates first (they then sit before the
//      Schmidt factors and are shared by all paths), then the blocks one after another.
//      Blocks are listed in circuit order.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <functional>
#include <map>
#include <vector>

#include "plan.h"

using namespace hsf;

namespace {

bool gate_is_diagonal(const GateH &g) {
  const int d = 1 << g.nq;
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j)
      if (i != j && g.m[(size_t)i * d + j] != cd(0.0)) return false;
  return true;
}

// Minimum vertex cover of a bipartite graph (left ids 0..L-1, right ids 0..R-1).
// Returns (in_cover_left, in_cover_right).
void min_vertex_cover(int L, int R, const std::vector<std::vector<int>> &adj, std::vector<char> &cl,
                      std::vector<char> &cr) {
  std::vector<int> match_l(L, -1), match_r(R, -1);
  for (int u = 0; u < L; ++u) {
    std::vector<char> seen(R, 0);
    std::function<bool(int)> augment = [&](int x) -> bool {
      for (int y : adj[x]) {
        if (seen[y]) continue;
        seen[y] = 1;
        if (match_r[y] < 0 || augment(match_r[y])) {
          match_l[x] = y;
          match_r[y] = x;
          return true;
        }
      }
      return false;
    };
    augment(u);
  }
  // Z = vertices reachable from unmatched left vertices by alternating paths
  // (non-matching edges left -> right, matching edges right -> left); cover =
  // (left \ Z) u (right n Z)
  std::vector<char> zl(L, 0), zr(R, 0);
  std::vector<int> stack;
  for (int u = 0; u < L; ++u)
    if (match_l[u] < 0 && !adj[u].empty()) {
      zl[u] = 1;
      stack.push_back(u);
    }
  while (!stack.empty()) {
    const int x = stack.back();
    stack.pop_back();
    for (int y : adj[x]) {
      if (zr[y] || match_l[x] == y) continue;
      zr[y] = 1;
      const int x2 = match_r[y];
      if (x2 >= 0 && !zl[x2]) {
        zl[x2] = 1;
        stack.push_back(x2);
      }
    }
  }
  cl.assign(L, 0);
  cr.assign(R, 0);
  for (int u = 0; u < L; ++u) cl[u] = !adj[u].empty() && !zl[u];
  for (int y = 0; y < R; ++y) cr[y] = zr[y];
}

// What the finder needs of a gate.
struct GView {
  int nq = 0;
  int q[4] = {0, 0, 0, 0};
  bool diag = false;
  int side = 0;     // 0 = a, 1 = b, 2 = crossing
};

// The finder on gate views: fills the reordered gate list, the blocks (positions in it)
// and the number of hubs.
void find_core(const std::vector<GView> &gv, int cut_l, int max_leaves, std::vector<int> &out_order,
               std::vector<std::vector<int>> &blocks, int &hubs_total) {
  const int G = (int)gv.size();
  out_order.clear();
  blocks.clear();
  hubs_total = 0;
  int g0 = 0;
  while (g0 < G) {
    const bool diag = gv[g0].diag;
    int g1 = g0 + 1;
    if (diag)
      while (g1 < G && gv[g1].diag) ++g1;
    if (!diag) {
      out_order.push_back(g0);
      if (gv[g0].side == 2) blocks.push_back({(int)out_order.size() - 1});
      g0 = g1;
      continue;
    }
    // a diagonal run [g0, g1): crossing two-qubit gates are the bipartite edges
    std::map<int, int> lid, rid;             // a-qubit -> left id, b-qubit -> right id
    std::vector<int> lq, rq;
    struct Edge { int gi, l, r; };
    std::vector<Edge> edges;
    std::vector<int> singles, inside;
    for (int gi = g0; gi < g1; ++gi) {
      const GView &g = gv[gi];
      if (g.side != 2) {
        inside.push_back(gi);
        continue;
      }
      if (g.nq != 2) {
        singles.push_back(gi);
        continue;
      }
      const int qa = g.q[0] > cut_l ? g.q[0] : g.q[1], qb = g.q[0] > cut_l ? g.q[1] : g.q[0];
      if (!lid.count(qa)) { lid[qa] = (int)lq.size(); lq.push_back(qa); }
      if (!rid.count(qb)) { rid[qb] = (int)rq.size(); rq.push_back(qb); }
      edges.push_back({gi, lid[qa], rid[qb]});
    }
    const int L = (int)lq.size(), R = (int)rq.size();
    std::vector<std::vector<int>> adj(L);
    for (const Edge &e : edges)
      if (std::find(adj[e.l].begin(), adj[e.l].end(), e.r) == adj[e.l].end()) adj[e.l].push_back(e.r);
    std::vector<char> cl, cr;
    min_vertex_cover(L, R, adj, cl, cr);
    std::vector<int> deg_l(L, 0), deg_r(R, 0);
    for (const Edge &e : edges) {
      if (cl[e.l]) deg_l[e.l]++;
      if (cr[e.r]) deg_r[e.r]++;
    }
    // hub key: left ids as-is, right ids offset by L
    std::map<int, std::vector<int>> by_hub;     // hub -> gate indices, circuit order
    for (const Edge &e : edges) {
      int hub;
      if (cl[e.l] && cr[e.r]) hub = deg_l[e.l] >= deg_r[e.r] ? e.l : L + e.r;
      else hub = cl[e.l] ? e.l : L + e.r;
      by_hub[hub].push_back(e.gi);
    }
    for (int gi : inside) out_order.push_back(gi);
    // blocks in the order of their first gate
    std::vector<std::vector<int>> run_blocks;
    for (auto &kv : by_hub) {
      hubs_total++;
      const std::vector<int> &gs = kv.second;
      for (size_t i = 0; i < gs.size(); i += (size_t)max_leaves)
        run_blocks.push_back(std::vector<int>(gs.begin() + i, gs.begin() + std::min(gs.size(), i + (size_t)max_leaves)));
    }
    for (int gi : singles) run_blocks.push_back({gi});
    std::sort(run_blocks.begin(), run_blocks.end(),
              [](const std::vector<int> &x, const std::vector<int> &y) { return x.front() < y.front(); });
    for (auto &rb : run_blocks) {
      std::vector<int> pos;
      for (int gi : rb) {
        out_order.push_back(gi);
        pos.push_back((int)out_order.size() - 1);
      }
      blocks.push_back(pos);
    }
    g0 = g1;
  }
}

}  // namespace

extern "C" hsf_status hsf_find_blocks(const hsf_circuit *circuit, int32_t cut_l, int32_t max_leaves,
                                      int32_t *order, int32_t *offsets, int32_t *gate_idx, int32_t cap_blocks,
                                      int32_t *num_blocks, int32_t *num_hubs) {
  if (!circuit || !order || !offsets || !gate_idx || !num_blocks)
    return set_error(HSF_EINVAL, "hsf_find_blocks: NULL argument");
  if (circuit->n < 2 || circuit->n > 62) return set_error(HSF_EINVAL, "n = %d outside 2..62", circuit->n);
  if (cut_l < 0 || cut_l > circuit->n - 2) return set_error(HSF_EINVAL, "cut %d outside 0..n-2", cut_l);
  if (max_leaves < 1 || max_leaves > kMaxCascadeLeaves)
    return set_error(HSF_EINVAL, "max_leaves %d outside 1..%d", max_leaves, kMaxCascadeLeaves);
  if (cap_blocks < 0) return set_error(HSF_EINVAL, "cap_blocks < 0");
  hsf_plan p;
  p.n = circuit->n;
  p.cut = cut_l;
  p.nb = cut_l + 1;
  p.na = circuit->n - cut_l - 1;
  hsf_status st = load_gates(p, circuit, nullptr);
  if (st != HSF_OK) return st;
  const int G = (int)p.gates.size();
  std::vector<GView> gv(G);
  for (int gi = 0; gi < G; ++gi) {
    const GateH &g = p.gates[gi];
    gv[gi].nq = g.nq;
    for (int x = 0; x < 4; ++x) gv[gi].q[x] = g.q[x];
    gv[gi].diag = gate_is_diagonal(g);
    gv[gi].side = g.side;
  }
  std::vector<int> out_order;
  std::vector<std::vector<int>> blocks;
  int hubs_total = 0;
  find_core(gv, cut_l, max_leaves, out_order, blocks, hubs_total);
  if ((int)blocks.size() > cap_blocks)
    return set_error(HSF_ENOMEM, "%zu blocks found, room for %d", blocks.size(), cap_blocks);
  for (int i = 0; i < G; ++i) order[i] = out_order[i];
  int e = 0;
  offsets[0] = 0;
  for (size_t b = 0; b < blocks.size(); ++b) {
    for (int x : blocks[b]) gate_idx[e++] = x;
    offsets[b + 1] = e;
  }
  *num_blocks = (int32_t)blocks.size();
  if (num_hubs) *num_hubs = hubs_total;
  return HSF_OK;
}

// ---------------------------------------------------------------------------------
// Qubit-reordering search (Sec. VI names reordering the qubits to find better blocks
// as future work; the paper gives no method, this is one).  Which qubits lie on which
// side of the cut decides the crossing gates and so the joint path count; the order of
// the qubits within a side does not.  The search therefore moves over bipartitions with
// the sides' sizes fixed (n_b = cut_l + 1): the cost of a bipartition is log2 of the
// path count of the blocks hsf_find_blocks would form (a cascade of two or more gates
// has Schmidt rank 2, Example 4; a single crossing gate has the operator-Schmidt rank of
// its relabeled matrix, Sec. IV-A), and a local search swaps one a-qubit with one
// b-qubit at a time in Kernighan-Lin passes (best swap among unmoved qubits even when it
// does not improve, keep the best point of the pass, repeat while a pass improves);
// seeded random restarts keep the best bipartition found.
namespace {

// Rank of M (rows x cols, row-major) by Gaussian elimination with full pivoting; pivots
// below tol x max|M| count as zero.
int numeric_rank(std::vector<cd> M, int rows, int cols, double tol) {
  double mx = 0.0;
  for (const cd &z : M) mx = std::max(mx, std::abs(z));
  if (mx == 0.0) return 0;
  int rank = 0;
  std::vector<char> row_used(rows, 0), col_used(cols, 0);
  for (int step = 0; step < std::min(rows, cols); ++step) {
    int pr = -1, pc = -1;
    double best = tol * mx;
    for (int r = 0; r < rows; ++r) {
      if (row_used[r]) continue;
      for (int c = 0; c < cols; ++c)
        if (!col_used[c] && std::abs(M[(size_t)r * cols + c]) > best) {
          best = std::abs(M[(size_t)r * cols + c]);
          pr = r;
          pc = c;
        }
    }
    if (pr < 0) break;
    row_used[pr] = 1;
    col_used[pc] = 1;
    ++rank;
    const cd piv = M[(size_t)pr * cols + pc];
    for (int r = 0; r < rows; ++r) {
      if (row_used[r]) continue;
      const cd f = M[(size_t)r * cols + pc] / piv;
      if (f == cd(0.0)) continue;
      for (int c = 0; c < cols; ++c) M[(size_t)r * cols + c] -= f * M[(size_t)pr * cols + c];
    }
  }
  return rank;
}

// Operator-Schmidt rank of a gate across the cut (qubit x of the gate on side a when
// bit x of a_mask is set): the rank of its relabeled matrix R[(i_a j_a), (i_b j_b)]
// (Sec. IV-A).  Matrix index bit nq-1-x belongs to the gate's qubit x.
int gate_cut_rank(const GateH &g, unsigned a_mask) {
  const int nq = g.nq, d = 1 << nq;
  std::vector<int> xa, xb;
  for (int x = 0; x < nq; ++x) ((a_mask >> x) & 1u ? xa : xb).push_back(x);
  if (xa.empty() || xb.empty()) return 1;
  const int ka = (int)xa.size(), kb = (int)xb.size();
  const int rows = 1 << (2 * ka), cols = 1 << (2 * kb);
  std::vector<cd> R((size_t)rows * cols);
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j) {
      int ia = 0, ja = 0, ib = 0, jb = 0;
      for (int t = 0; t < ka; ++t) {
        const int bit = nq - 1 - xa[t];
        ia = (ia << 1) | ((i >> bit) & 1);
        ja = (ja << 1) | ((j >> bit) & 1);
      }
      for (int t = 0; t < kb; ++t) {
        const int bit = nq - 1 - xb[t];
        ib = (ib << 1) | ((i >> bit) & 1);
        jb = (jb << 1) | ((j >> bit) & 1);
      }
      R[(size_t)((ia << ka) | ja) * cols + ((ib << kb) | jb)] = g.m[(size_t)i * d + j];
    }
  return numeric_rank(R, rows, cols, 1e-10);
}

struct CutSearch {
  const hsf_plan &p;
  int n, cut_l, max_leaves;
  std::vector<GView> gv;
  std::vector<int> out_order;
  std::vector<std::vector<int>> blocks;
  std::map<std::pair<int, unsigned>, int> rank_cache;

  CutSearch(const hsf_plan &plan, int cut, int leaves) : p(plan), n(plan.n), cut_l(cut), max_leaves(leaves) {
    gv.resize(p.gates.size());
    for (size_t gi = 0; gi < p.gates.size(); ++gi) {
      gv[gi].nq = p.gates[gi].nq;
      gv[gi].diag = gate_is_diagonal(p.gates[gi]);
    }
  }

  // Search key: log2 of the joint path count, plus the number of crossing gates scaled
  // below one bit (a tie-break that gives the search a slope on the path count's
  // plateaus: fewer crossing gates leave fewer edges for the vertex cover)
  double cost(const std::vector<char> &on_a) {
    double crossing = 0.0;
    const double bits = path_bits(on_a, &crossing);
    return bits + crossing / (double)(gv.size() + 1);
  }

  // log2 of the joint path count with qubit q on side a iff on_a[q]
  double path_bits(const std::vector<char> &on_a, double *crossing = nullptr) {
    for (size_t gi = 0; gi < gv.size(); ++gi) {
      const GateH &g = p.gates[gi];
      // labels: b-qubits first (0..cut_l), then a-qubits, each in ascending old order;
      // the finder only looks at sides and at qubit identities
      bool any_a = false, any_b = false;
      for (int x = 0; x < g.nq; ++x) {
        gv[gi].q[x] = g.q[x];
        (on_a[g.q[x]] ? any_a : any_b) = true;
      }
      gv[gi].side = any_a && any_b ? 2 : (any_a ? 0 : 1);
      if (crossing && gv[gi].side == 2) *crossing += 1.0;
    }
    int hubs = 0;
    find_core_sided(on_a, hubs);
    double bits = 0.0;
    for (const auto &blk : blocks) {
      if (blk.size() >= 2) {
        bits += 1.0;
        continue;
      }
      const int gi = out_order[blk[0]];
      const GateH &g = p.gates[gi];
      unsigned mask = 0;
      for (int x = 0; x < g.nq; ++x)
        if (on_a[g.q[x]]) mask |= 1u << x;
      auto key = std::make_pair(gi, mask);
      auto it = rank_cache.find(key);
      const int r = it != rank_cache.end() ? it->second : (rank_cache[key] = gate_cut_rank(g, mask));
      bits += r > 1 ? std::log2((double)r) : 0.0;
    }
    return bits;
  }

  // find_core decides a gate's side by the qubit labels and cut_l; relabel so that the
  // a-qubits are the labels above cut_l
  void find_core_sided(const std::vector<char> &on_a, int &hubs) {
    std::vector<int> label(n);
    int nb = 0, na = 0;
    for (int q = 0; q < n; ++q) label[q] = on_a[q] ? -1 : nb++;
    for (int q = 0; q < n; ++q)
      if (on_a[q]) label[q] = cut_l + 1 + na++;
    for (auto &g : gv)
      for (int x = 0; x < g.nq; ++x) g.q[x] = label[g.q[x]];
    find_core(gv, cut_l, max_leaves, out_order, blocks, hubs);
  }
};

uint64_t splitmix64(uint64_t &s) {
  uint64_t z = (s += 0x9e3779b97f4a7c15ull);
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

}  // namespace

extern "C" hsf_status hsf_search_cut(const hsf_circuit *circuit, int32_t cut_l, int32_t max_leaves,
                                     int32_t restarts, uint64_t seed, int32_t *perm, double *log2_paths_before,
                                     double *log2_paths_after) {
  if (!circuit || !perm) return set_error(HSF_EINVAL, "hsf_search_cut: NULL argument");
  if (circuit->n < 2 || circuit->n > 62) return set_error(HSF_EINVAL, "n = %d outside 2..62", circuit->n);
  if (cut_l < 0 || cut_l > circuit->n - 2) return set_error(HSF_EINVAL, "cut %d outside 0..n-2", cut_l);
  if (max_leaves < 1 || max_leaves > kMaxCascadeLeaves)
    return set_error(HSF_EINVAL, "max_leaves %d outside 1..%d", max_leaves, kMaxCascadeLeaves);
  if (restarts < 0) return set_error(HSF_EINVAL, "restarts < 0");
  hsf_plan p;
  p.n = circuit->n;
  p.cut = cut_l;
  p.nb = cut_l + 1;
  p.na = circuit->n - cut_l - 1;
  hsf_status st = load_gates(p, circuit, nullptr);
  if (st != HSF_OK) return st;
  const int n = p.n;
  CutSearch cs(p, cut_l, max_leaves);
  std::vector<char> start(n);
  for (int q = 0; q < n; ++q) start[q] = q > cut_l;
  const double before = cs.path_bits(start);
  std::vector<char> best_side = start;
  double best = cs.cost(start);
  uint64_t rng = seed;
  for (int r = 0; r <= restarts; ++r) {
    std::vector<char> side = start;
    if (r > 0) {       // a seeded random bipartition with the same side sizes
      std::vector<int> qs(n);
      for (int q = 0; q < n; ++q) qs[q] = q;
      for (int i = n - 1; i > 0; --i) std::swap(qs[i], qs[(int)(splitmix64(rng) % (uint64_t)(i + 1))]);
      for (int i = 0; i < n; ++i) side[qs[i]] = i > cut_l;
    }
    double cur = cs.cost(side);
    // Kernighan-Lin passes: swap the best pair among the unlocked qubits (even when the
    // swap does not improve), lock both, repeat until every qubit of the smaller side has
    // moved; keep the best prefix of the pass; stop when a pass brings no improvement
    for (int pass = 0; pass < 64; ++pass) {
      std::vector<char> locked(n, 0), trial = side;
      double tcur = cur, pbest = cur;
      std::vector<char> pbest_side = side;
      const int moves = std::min(cut_l + 1, n - cut_l - 1);
      for (int mv = 0; mv < moves; ++mv) {
        int bi = -1, bj = -1;
        double bc = 1e300;
        for (int i = 0; i < n; ++i) {
          if (!trial[i] || locked[i]) continue;
          for (int j = 0; j < n; ++j) {
            if (trial[j] || locked[j]) continue;
            trial[i] = 0;
            trial[j] = 1;
            const double c = cs.cost(trial);
            trial[i] = 1;
            trial[j] = 0;
            if (c < bc) {
              bc = c;
              bi = i;
              bj = j;
            }
          }
        }
        if (bi < 0) break;
        trial[bi] = 0;
        trial[bj] = 1;
        locked[bi] = locked[bj] = 1;
        tcur = bc;
        if (tcur < pbest - 1e-9) {
          pbest = tcur;
          pbest_side = trial;
        }
      }
      if (pbest >= cur - 1e-9) break;
      cur = pbest;
      side = pbest_side;
    }
    if (cur < best - 1e-9) {
      best = cur;
      best_side = side;
    }
  }
  int nb = 0, na = 0;
  for (int q = 0; q < n; ++q)
    if (!best_side[q]) perm[q] = nb++;
  for (int q = 0; q < n; ++q)
    if (best_side[q]) perm[q] = cut_l + 1 + na++;
  if (log2_paths_before) *log2_paths_before = before;
  if (log2_paths_after) *log2_paths_after = cs.path_bits(best_side);
  return HSF_OK;
}
