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
  std::vector<int> out_order;
  std::vector<std::vector<int>> blocks;      // positions in out_order
  int hubs_total = 0;
  int g0 = 0;
  while (g0 < G) {
    const bool diag = gate_is_diagonal(p.gates[g0]);
    int g1 = g0 + 1;
    if (diag)
      while (g1 < G && gate_is_diagonal(p.gates[g1])) ++g1;
    if (!diag) {
      out_order.push_back(g0);
      if (p.gates[g0].side == 2) blocks.push_back({(int)out_order.size() - 1});
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
      const GateH &g = p.gates[gi];
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
