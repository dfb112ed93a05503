// C ABI of the joint-cut HSF library: planning (host) and run orchestration.
//
// Planning (Sec. II-B, III-A, IV-A, IV-D):
//   * classify gates by side of the cut (a: qubits l+1..n-1, b: qubits 0..l);
//   * check the blocks: every crossing gate in exactly one block, every block convex
//     in the gate DAG and listed in an order compatible with the dependencies;
//   * multiply and Schmidt-decompose every block on the GPU (svd.cu), read back ranks,
//     singular values and factors;
//   * give every in-half gate a tree level: the number of the last block whose
//     factor it depends on (gates that commute with a later factor are applied before
//     the branching, so the children of a path-tree node share as much work as the
//     dependencies allow);
//   * per side and level, build the gate program (Schmidt factor first, then gates),
//     merge runs of one-qubit gates, and split programs into tile passes when the
//     half state is larger than a shared-memory tile.
// Running: the path tree is walked level by level over chunks of paths (subtrees
// sized to the workspace); each level is one sweep launch per pass and side; the
// leaves are accumulated by gather_dot (bitstrings) or window (full output).
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <functional>
#include <map>
#include <memory>
#include <queue>
#include <set>
#include <string>
#include <vector>

#include "plan.h"

using namespace hsf;

namespace {

thread_local std::string g_err;
std::atomic<uint64_t> g_launches{0};
std::atomic<int> g_profiling{0};

hsf_status fail(hsf_status code, const char *fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

#define CUDA_TRY(expr)                                                                   \
  do {                                                                                   \
    cudaError_t e_ = (expr);                                                             \
    if (e_ != cudaSuccess)                                                               \
      return fail(HSF_ECUDA, "%s failed: %s", #expr, cudaGetErrorString(e_));            \
  } while (0)

// ---------------------------------------------------------------------------
// Gate matrices (host, FP64).  R_P(t) = exp(-i t P / 2).
// ---------------------------------------------------------------------------
hsf_status named_matrix(int kind, double t, std::vector<cd> &m, int &nq) {
  const cd I(0.0, 1.0);
  const double c = std::cos(t / 2), s = std::sin(t / 2);
  switch (kind) {
    case HSF_GATE_H: nq = 1; { const double r = 1.0 / std::sqrt(2.0); m = {r, r, r, -r}; } break;
    case HSF_GATE_X: nq = 1; m = {0.0, 1.0, 1.0, 0.0}; break;
    case HSF_GATE_Y: nq = 1; m = {0.0, -I, I, 0.0}; break;
    case HSF_GATE_Z: nq = 1; m = {1.0, 0.0, 0.0, -1.0}; break;
    case HSF_GATE_S: nq = 1; m = {1.0, 0.0, 0.0, I}; break;
    case HSF_GATE_T: nq = 1; m = {1.0, 0.0, 0.0, std::exp(I * (M_PI / 4))}; break;
    case HSF_GATE_RX: nq = 1; m = {c, -I * s, -I * s, c}; break;
    case HSF_GATE_RY: nq = 1; m = {c, -s, s, c}; break;
    case HSF_GATE_RZ: nq = 1; m = {std::exp(-I * (t / 2)), 0.0, 0.0, std::exp(I * (t / 2))}; break;
    case HSF_GATE_CX:
      nq = 2; m.assign(16, 0.0);
      m[0 * 4 + 0] = 1; m[1 * 4 + 1] = 1; m[2 * 4 + 3] = 1; m[3 * 4 + 2] = 1;
      break;
    case HSF_GATE_CZ:
      nq = 2; m.assign(16, 0.0);
      m[0] = 1; m[5] = 1; m[10] = 1; m[15] = -1;
      break;
    case HSF_GATE_SWAP:
      nq = 2; m.assign(16, 0.0);
      m[0] = 1; m[1 * 4 + 2] = 1; m[2 * 4 + 1] = 1; m[15] = 1;
      break;
    case HSF_GATE_ISWAP:
      nq = 2; m.assign(16, 0.0);
      m[0] = 1; m[1 * 4 + 2] = I; m[2 * 4 + 1] = I; m[15] = 1;
      break;
    case HSF_GATE_RZZ: {
      nq = 2; m.assign(16, 0.0);
      const cd em = std::exp(-I * (t / 2)), ep = std::exp(I * (t / 2));
      m[0] = em; m[5] = ep; m[10] = ep; m[15] = em;
      break;
    }
    default:
      return fail(HSF_EINVAL, "unknown gate kind %d", kind);
  }
  return HSF_OK;
}

std::vector<cd> matmul(const std::vector<cd> &a, const std::vector<cd> &b, int d) {
  std::vector<cd> r((size_t)d * d, 0.0);
  for (int i = 0; i < d; ++i)
    for (int k = 0; k < d; ++k) {
      const cd aik = a[(size_t)i * d + k];
      if (aik == 0.0) continue;
      for (int j = 0; j < d; ++j) r[(size_t)i * d + j] += aik * b[(size_t)k * d + j];
    }
  return r;
}

bool is_diagonal(const std::vector<cd> &m, int d) {
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j)
      if (i != j && m[(size_t)i * d + j] != 0.0) return false;
  return true;
}

// ---------------------------------------------------------------------------
// DAG with blocks contracted to single nodes.
// ---------------------------------------------------------------------------
struct Node {
  bool is_block;
  int id;                  // gate index or block index
  int key;                 // tie-break: smallest gate index
  std::vector<int> succ;
  int indeg = 0;
};

hsf_status execution_order(const hsf_plan &p, std::vector<std::pair<bool, int>> &order) {
  const int G = (int)p.gates.size();
  const int B = (int)p.blocks.size();
  std::vector<int> owner(G, -1);
  for (int b = 0; b < B; ++b)
    for (int gi : p.blocks[b].gates) owner[gi] = b;
  // node ids: blocks 0..B-1, free gates B + gi
  std::vector<Node> nodes(B + G);
  for (int b = 0; b < B; ++b) nodes[b] = Node{true, b, *std::min_element(p.blocks[b].gates.begin(), p.blocks[b].gates.end()), {}, 0};
  std::vector<char> used(B + G, 0);
  for (int b = 0; b < B; ++b) used[b] = 1;
  for (int gi = 0; gi < G; ++gi)
    if (owner[gi] < 0) { nodes[B + gi] = Node{false, gi, gi, {}, 0}; used[B + gi] = 1; }
  auto nid = [&](int gi) { return owner[gi] >= 0 ? owner[gi] : B + gi; };
  std::set<std::pair<int, int>> edges;
  std::vector<int> last(p.n, -1);
  for (int gi = 0; gi < G; ++gi) {
    const int v = nid(gi);
    for (int j = 0; j < p.gates[gi].nq; ++j) {
      const int q = p.gates[gi].q[j];
      if (last[q] >= 0) {
        const int u = nid(last[q]);
        if (u != v) edges.insert({u, v});
      }
      last[q] = gi;
    }
  }
  // the listed block order is part of the path numbering: enforce it as edges
  for (int b = 0; b + 1 < B; ++b) edges.insert({b, b + 1});
  for (auto &e : edges) { nodes[e.first].succ.push_back(e.second); nodes[e.second].indeg++; }
  using QE = std::pair<int, int>;  // (key, node)
  std::priority_queue<QE, std::vector<QE>, std::greater<QE>> pq;
  for (int v = 0; v < B + G; ++v)
    if (used[v] && nodes[v].indeg == 0) pq.push({nodes[v].key, v});
  order.clear();
  int count = 0, total = 0;
  for (int v = 0; v < B + G; ++v) total += used[v];
  while (!pq.empty()) {
    const int v = pq.top().second;
    pq.pop();
    ++count;
    order.push_back({nodes[v].is_block, nodes[v].id});
    for (int w : nodes[v].succ)
      if (--nodes[w].indeg == 0) pq.push({nodes[w].key, w});
  }
  if (count != total)
    return fail(HSF_EBLOCK, "a block is not convex in the circuit DAG, or the blocks are not listed "
                            "in an order compatible with the circuit");
  return HSF_OK;
}

// ---------------------------------------------------------------------------
// Side programs.
// ---------------------------------------------------------------------------
void merge_one_qubit_runs(std::vector<OpH> &ops) {
  std::vector<OpH> out;
  std::map<int, int> last;   // qubit -> index in out of the last op touching it
  for (auto &op : ops) {
    if (op.nq == 1 && op.digits == 1) {
      auto it = last.find(op.q[0]);
      if (it != last.end()) {
        OpH &prev = out[it->second];
        if (prev.nq == 1 && prev.digits == 1) {
          // prev then op: combined = op * prev
          std::vector<cd> a = op.m, b = prev.m;
          if (op.type == OP_DIAG) a = {op.m[0], 0.0, 0.0, op.m[1]};
          if (prev.type == OP_DIAG) b = {prev.m[0], 0.0, 0.0, prev.m[1]};
          std::vector<cd> c = matmul(a, b, 2);
          if (op.type == OP_DIAG && prev.type == OP_DIAG) {
            prev.m = {c[0], c[3]};
          } else {
            prev.type = OP_DENSE;
            prev.m = c;
          }
          continue;
        }
      }
    }
    out.push_back(op);
    for (int j = 0; j < op.nq; ++j) last[op.q[j]] = (int)out.size() - 1;
  }
  ops.swap(out);
}

int popcount64(uint64_t x) { return __builtin_popcountll(x); }

// Split a level program into passes whose dense ops only touch the tile's qubits.
void split_passes(LevelH &lv, int h, int tmax) {
  lv.passes.clear();
  const uint64_t full = (h >= 64) ? ~0ull : ((1ull << h) - 1ull);
  if (h <= tmax) {
    PassH ps;
    ps.active = full;
    ps.t = h;
    ps.ops = lv.ops;
    lv.passes.push_back(ps);
    return;
  }
  std::vector<OpH> rem = lv.ops;
  while (!rem.empty()) {
    uint64_t active = 0, blocked = 0;
    std::vector<OpH> here, later;
    for (auto &op : rem) {
      uint64_t qm = 0;
      for (int j = 0; j < op.nq; ++j) qm |= 1ull << op.q[j];
      if (qm & blocked) { later.push_back(op); blocked |= qm; continue; }
      if (op.type == OP_DENSE && (qm & ~active)) {
        if (popcount64(active | qm) <= tmax) {
          active |= qm;
        } else {
          later.push_back(op);
          blocked |= qm;
          continue;
        }
      }
      here.push_back(op);
    }
    // fill the tile with the lowest remaining qubits (long contiguous runs)
    for (int q = 0; q < h && popcount64(active) < tmax; ++q) active |= 1ull << q;
    PassH ps;
    ps.active = active;
    ps.t = popcount64(active);
    ps.ops = here;
    lv.passes.push_back(ps);
    rem.swap(later);
  }
  if (lv.passes.empty()) {
    PassH ps;
    ps.active = 0;
    for (int q = 0; q < tmax; ++q) ps.active |= 1ull << q;
    ps.t = tmax;
    lv.passes.push_back(ps);
  }
}

template <typename C>
void pack_pass(const PassH &ps, std::vector<DevOp> &dops, std::vector<C> &mats) {
  // tile bit of a storage bit
  int tile_bit[64];
  int tb = 0;
  for (int q = 0; q < 64; ++q) tile_bit[q] = (ps.active >> q) & 1ull ? tb++ : -1;
  for (auto &op : ps.ops) {
    DevOp d{};
    d.type = op.type;
    d.nq = op.nq;
    for (int j = 0; j < 3; ++j) d.pos[j] = 0;
    for (int j = 0; j < op.nq; ++j) {
      const int q = op.q[j];
      d.pos[j] = tile_bit[q] >= 0 ? tile_bit[q] : kFixedBit + q;
    }
    d.mat = (int32_t)mats.size();
    const int per = op.type == OP_DENSE ? (1 << (2 * op.nq)) : (1 << op.nq);
    d.digit_stride = op.digits > 1 ? per : 0;
    for (auto &z : op.m) {
      C c;
      c.x = (decltype(c.x))z.real();
      c.y = (decltype(c.y))z.imag();
      mats.push_back(c);
    }
    (void)per;
    dops.push_back(d);
  }
}

hsf_status build_programs(hsf_plan &p) {
  const int B = (int)p.blocks.size();
  std::vector<std::pair<bool, int>> order;
  hsf_status st = execution_order(p, order);
  if (st != HSF_OK) return st;
  for (int s = 0; s < 2; ++s) {
    SideH &sd = p.side[s];
    sd.h = s == 0 ? p.na : p.nb;
    sd.offset = s == 0 ? p.cut + 1 : 0;
    sd.levels.assign(B + 1, LevelH{});
    // Schmidt factors open levels 1..B
    for (int b = 0; b < B; ++b) {
      const BlockH &bk = p.blocks[b];
      const std::vector<int> &qs = s == 0 ? bk.qa : bk.qb;
      OpH op;
      op.type = OP_DENSE;
      op.nq = (int)qs.size();
      for (int j = 0; j < op.nq; ++j) op.q[j] = qs[j] - sd.offset;
      op.digits = bk.rank;
      op.block = b;
      op.m = s == 0 ? bk.x : bk.y;
      sd.levels[b + 1].ops.push_back(op);
    }
    std::vector<int> qlevel(sd.h, 0);
    int blocks_seen = 0;
    for (auto &item : order) {
      if (item.first) {
        const int b = item.second;
        const std::vector<int> &qs = s == 0 ? p.blocks[b].qa : p.blocks[b].qb;
        for (int q : qs) qlevel[q - sd.offset] = std::max(qlevel[q - sd.offset], b + 1);
        blocks_seen = std::max(blocks_seen, b + 1);
        continue;
      }
      const GateH &g = p.gates[item.second];
      if (g.side != s) continue;
      int lvl = 0;
      if (p.flags & HSF_FLAG_NO_LIGHTCONE) {
        lvl = blocks_seen;
      } else {
        for (int j = 0; j < g.nq; ++j) lvl = std::max(lvl, qlevel[g.q[j] - sd.offset]);
      }
      for (int j = 0; j < g.nq; ++j) qlevel[g.q[j] - sd.offset] = lvl;
      OpH op;
      op.type = g.diag ? OP_DIAG : OP_DENSE;
      op.nq = g.nq;
      for (int j = 0; j < g.nq; ++j) op.q[j] = g.q[j] - sd.offset;
      const int d = 1 << g.nq;
      if (g.diag) {
        op.m.resize(d);
        for (int i = 0; i < d; ++i) op.m[i] = g.m[(size_t)i * d + i];
      } else {
        op.m = g.m;
      }
      sd.levels[lvl].ops.push_back(op);
    }
    for (auto &lv : sd.levels) {
      merge_one_qubit_runs(lv.ops);
      split_passes(lv, sd.h, p.tile_max);
    }
  }
  return HSF_OK;
}

hsf_status upload_programs(hsf_plan &p) {
  // layout: for every side/level/pass: ops (DevOp[]) then matrices, 256-B aligned
  std::vector<unsigned char> host;
  auto align = [&](size_t a) { while (host.size() % a) host.push_back(0); };
  int64_t launches = 0;
  for (int s = 0; s < 2; ++s)
    for (auto &lv : p.side[s].levels)
      for (auto &ps : lv.passes) {
        std::vector<DevOp> dops;
        align(256);
        ps.ops_off = host.size();
        ps.num_ops = (int)ps.ops.size();
        if (p.precision == HSF_PREC_C64) {
          std::vector<float2> mats;
          pack_pass(ps, dops, mats);
          host.insert(host.end(), (unsigned char *)dops.data(), (unsigned char *)(dops.data() + dops.size()));
          align(256);
          ps.mats_off = host.size();
          host.insert(host.end(), (unsigned char *)mats.data(), (unsigned char *)(mats.data() + mats.size()));
        } else {
          std::vector<double2> mats;
          pack_pass(ps, dops, mats);
          host.insert(host.end(), (unsigned char *)dops.data(), (unsigned char *)(dops.data() + dops.size()));
          align(256);
          ps.mats_off = host.size();
          host.insert(host.end(), (unsigned char *)mats.data(), (unsigned char *)(mats.data() + mats.size()));
        }
        ++launches;
      }
  align(256);
  if (host.empty()) host.resize(256);
  CUDA_TRY(cudaMalloc(&p.dev_table, host.size()));
  p.dev_table_bytes = host.size();
  CUDA_TRY(cudaMemcpy(p.dev_table, host.data(), host.size(), cudaMemcpyHostToDevice));
  p.launches = launches / 2;
  return HSF_OK;
}

// Multiply and decompose every block on the device; read back ranks and factors.
hsf_status decompose_blocks(hsf_plan &p) {
  const int B = (int)p.blocks.size();
  if (B == 0) return HSF_OK;
  std::vector<int32_t> bk(3 * B), gbeg(B + 1, 0), gdesc;
  std::vector<double> gm;
  for (int b = 0; b < B; ++b) {
    BlockH &blk = p.blocks[b];
    const int k = (int)blk.qubits.size();
    bk[3 * b] = k;
    bk[3 * b + 1] = (int)blk.qa.size();
    bk[3 * b + 2] = (int)blk.qb.size();
    for (int gi : blk.gates) {
      const GateH &g = p.gates[gi];
      gdesc.push_back(g.nq);
      for (int j = 0; j < 3; ++j) {
        int pos = 0;
        if (j < g.nq) {
          const int idx = (int)(std::find(blk.qubits.begin(), blk.qubits.end(), g.q[j]) - blk.qubits.begin());
          pos = k - 1 - idx;      // qubits are listed most significant first
        }
        gdesc.push_back(pos);
      }
      gdesc.push_back((int32_t)(gm.size() / 2));
      for (auto &z : g.m) { gm.push_back(z.real()); gm.push_back(z.imag()); }
    }
    gbeg[b + 1] = (int32_t)(gdesc.size() / 5);
  }
  const size_t nf = (size_t)B * 64 * 64 * 2;
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t o = off; off += (bytes + 255) / 256 * 256; return o; };
  const size_t o_bk = take(bk.size() * 4), o_gb = take(gbeg.size() * 4), o_gd = take(gdesc.size() * 4 + 4),
               o_gm = take(gm.size() * 8 + 8), o_sig = take((size_t)B * 64 * 8), o_rank = take((size_t)B * 4),
               o_x = take(nf * 8), o_y = take(nf * 8), o_sw = take((size_t)B * 4);
  unsigned char *d = nullptr;
  CUDA_TRY(cudaMalloc(&d, off));
  std::unique_ptr<unsigned char, void (*)(unsigned char *)> guard(d, [](unsigned char *q) { cudaFree(q); });
  CUDA_TRY(cudaMemcpy(d + o_bk, bk.data(), bk.size() * 4, cudaMemcpyHostToDevice));
  CUDA_TRY(cudaMemcpy(d + o_gb, gbeg.data(), gbeg.size() * 4, cudaMemcpyHostToDevice));
  if (!gdesc.empty()) CUDA_TRY(cudaMemcpy(d + o_gd, gdesc.data(), gdesc.size() * 4, cudaMemcpyHostToDevice));
  if (!gm.empty()) CUDA_TRY(cudaMemcpy(d + o_gm, gm.data(), gm.size() * 8, cudaMemcpyHostToDevice));
  BlockSvdArgs a{};
  a.num_blocks = B;
  a.block_k = (const int32_t *)(d + o_bk);
  a.gate_begin = (const int32_t *)(d + o_gb);
  a.gate_desc = (const int32_t *)(d + o_gd);
  a.gate_mats = (const double *)(d + o_gm);
  a.rank_tol = p.rank_tol;
  a.max_sweeps = 60;
  a.sigma = (double *)(d + o_sig);
  a.rank = (int32_t *)(d + o_rank);
  a.xf = (double *)(d + o_x);
  a.yf = (double *)(d + o_y);
  a.sweeps_used = (int32_t *)(d + o_sw);
  CUDA_TRY(launch_block_svd(a, 0));
  g_launches++;
  CUDA_TRY(cudaDeviceSynchronize());
  std::vector<double> sig((size_t)B * 64), xf(nf), yf(nf);
  std::vector<int32_t> rank(B);
  CUDA_TRY(cudaMemcpy(sig.data(), d + o_sig, sig.size() * 8, cudaMemcpyDeviceToHost));
  CUDA_TRY(cudaMemcpy(rank.data(), d + o_rank, rank.size() * 4, cudaMemcpyDeviceToHost));
  CUDA_TRY(cudaMemcpy(xf.data(), d + o_x, nf * 8, cudaMemcpyDeviceToHost));
  CUDA_TRY(cudaMemcpy(yf.data(), d + o_y, nf * 8, cudaMemcpyDeviceToHost));
  for (int b = 0; b < B; ++b) {
    BlockH &blk = p.blocks[b];
    blk.rank = rank[b];
    if (blk.rank <= 0) return fail(HSF_ENUMERIC, "block %d decomposed to rank 0", b);
    blk.sigma.assign(sig.begin() + (size_t)b * 64, sig.begin() + (size_t)b * 64 + blk.rank);
    for (double s : blk.sigma)
      if (!std::isfinite(s)) return fail(HSF_ENUMERIC, "block %d: non-finite singular value", b);
    const int ea = 1 << (2 * (int)blk.qa.size()), eb = 1 << (2 * (int)blk.qb.size());
    blk.x.clear();
    blk.y.clear();
    for (int m = 0; m < blk.rank; ++m) {
      for (int e = 0; e < ea; ++e) {
        const size_t i = (((size_t)b * 64 + m) * 64 + e) * 2;
        blk.x.push_back(cd(xf[i], xf[i + 1]));
      }
      for (int e = 0; e < eb; ++e) {
        const size_t i = (((size_t)b * 64 + m) * 64 + e) * 2;
        blk.y.push_back(cd(yf[i], yf[i + 1]));
      }
    }
  }
  return HSF_OK;
}

hsf_status validate_and_load(hsf_plan &p, const hsf_circuit *c, int cut, const hsf_blocks *bl,
                             const hsf_plan_opts *o) {
  if (!c || !bl) return fail(HSF_EINVAL, "circuit and blocks must not be NULL");
  if (c->n < 2 || c->n > 62) return fail(HSF_EINVAL, "n = %d outside 2..62", c->n);
  if (cut < 0 || cut > c->n - 2) return fail(HSF_EINVAL, "cut %d outside 0..n-2", cut);
  if (c->num_gates < 0 || (c->num_gates > 0 && !c->gates)) return fail(HSF_EINVAL, "bad gate array");
  p.n = c->n;
  p.cut = cut;
  p.nb = cut + 1;
  p.na = c->n - cut - 1;
  if (o) {
    p.precision = o->precision;
    p.gemm_mode = o->gemm_mode;
    p.rank_tol = o->rank_tol > 0 ? o->rank_tol : 1e-12;
    p.max_paths = o->max_paths ? o->max_paths : (1ull << 40);
    p.flags = o->flags;
  } else {
    p.max_paths = 1ull << 40;
  }
  if (p.precision != HSF_PREC_C64 && p.precision != HSF_PREC_C128)
    return fail(HSF_EINVAL, "precision %d", p.precision);
  if (p.gemm_mode < 0 || p.gemm_mode > 3) return fail(HSF_EINVAL, "gemm_mode %d", p.gemm_mode);
  // a shared-memory tile holds 2^t amplitudes: 128 KB at most
  const int tcap = p.precision == HSF_PREC_C64 ? 14 : 13;
  p.tile_max = (o && o->tile_bits) ? o->tile_bits : tcap;
  if (p.tile_max < 3 || p.tile_max > tcap) return fail(HSF_EINVAL, "tile_bits %d outside 3..%d", p.tile_max, tcap);
  if (p.na > 40 || p.nb > 40) return fail(HSF_EINVAL, "half of %d/%d qubits is too large", p.na, p.nb);
  p.gates.resize(c->num_gates);
  for (int i = 0; i < c->num_gates; ++i) {
    const hsf_gate &g = c->gates[i];
    GateH &h = p.gates[i];
    h.kind = g.kind;
    h.param = g.param;
    h.param_id = g.param_id;
    if (g.param_id >= 0 && o && o->angles) {
      if (g.param_id >= o->num_angles) return fail(HSF_EINVAL, "gate %d: param_id %d >= num_angles", i, g.param_id);
      h.param = o->angles[g.param_id];
    }
    int nq = 0;
    if (g.kind == HSF_GATE_MATRIX) {
      nq = g.nq;
      if (nq < 1 || nq > 3) return fail(HSF_EINVAL, "gate %d: matrix gates take 1..3 qubits", i);
      if (!g.mat) return fail(HSF_EINVAL, "gate %d: matrix pointer is NULL", i);
      const int d = 1 << nq;
      h.m.resize((size_t)d * d);
      for (int e = 0; e < d * d; ++e) h.m[e] = cd(g.mat[2 * e], g.mat[2 * e + 1]);
      for (auto &z : h.m)
        if (!std::isfinite(z.real()) || !std::isfinite(z.imag())) return fail(HSF_EINVAL, "gate %d: non-finite matrix", i);
    } else {
      hsf_status st = named_matrix(g.kind, h.param, h.m, nq);
      if (st != HSF_OK) return st;
      if (g.nq != nq) return fail(HSF_EINVAL, "gate %d: kind %d takes %d qubits, got %d", i, g.kind, nq, g.nq);
    }
    h.nq = nq;
    for (int j = 0; j < nq; ++j) {
      h.q[j] = g.q[j];
      if (g.q[j] < 0 || g.q[j] >= c->n) return fail(HSF_EINVAL, "gate %d: qubit %d out of range", i, g.q[j]);
      for (int k = 0; k < j; ++k)
        if (g.q[k] == g.q[j]) return fail(HSF_EINVAL, "gate %d: repeated qubit %d", i, g.q[j]);
    }
    h.diag = is_diagonal(h.m, 1 << nq);
    bool hi = false, lo = false;
    for (int j = 0; j < nq; ++j) (h.q[j] > cut ? hi : lo) = true;
    h.side = (hi && lo) ? 2 : (hi ? 0 : 1);
  }
  // blocks
  if (bl->num_blocks < 0 || bl->num_blocks > 64) return fail(HSF_EINVAL, "num_blocks %d outside 0..64", bl->num_blocks);
  if (bl->num_blocks > 0 && (!bl->offsets || !bl->gate_idx)) return fail(HSF_EINVAL, "bad block arrays");
  std::vector<int> owner(c->num_gates, -1);
  p.blocks.resize(bl->num_blocks);
  for (int b = 0; b < bl->num_blocks; ++b) {
    const int lo = bl->offsets[b], hi = bl->offsets[b + 1];
    if (lo < 0 || hi < lo) return fail(HSF_EINVAL, "block %d: bad offsets", b);
    if (hi == lo) return fail(HSF_EBLOCK, "block %d is empty", b);
    BlockH &blk = p.blocks[b];
    std::set<int> qs;
    bool crossing = false;
    for (int e = lo; e < hi; ++e) {
      const int gi = bl->gate_idx[e];
      if (gi < 0 || gi >= c->num_gates) return fail(HSF_EINVAL, "block %d: gate index %d out of range", b, gi);
      if (owner[gi] >= 0) return fail(HSF_EBLOCK, "gate %d is in blocks %d and %d", gi, owner[gi], b);
      owner[gi] = b;
      blk.gates.push_back(gi);
      for (int j = 0; j < p.gates[gi].nq; ++j) qs.insert(p.gates[gi].q[j]);
      crossing |= p.gates[gi].side == 2;
    }
    if (!crossing) return fail(HSF_EBLOCK, "block %d holds no gate crossing the cut", b);
    std::sort(blk.gates.begin(), blk.gates.end());
    blk.qubits.assign(qs.rbegin(), qs.rend());
    for (int q : blk.qubits) (q > cut ? blk.qa : blk.qb).push_back(q);
    if (blk.qa.size() > 3 || blk.qb.size() > 3)
      return fail(HSF_ERANK, "block %d spans %zu|%zu qubits; at most 3 per side", b, blk.qa.size(), blk.qb.size());
  }
  for (int i = 0; i < c->num_gates; ++i)
    if (p.gates[i].side == 2 && owner[i] < 0)
      return fail(HSF_EBLOCK, "gate %d crosses the cut but is in no block", i);
  return HSF_OK;
}

struct RunLayout {
  uint64_t chunk = 0;          // leaves per chunk (a subtree size)
  size_t state_bytes[2] = {0, 0};
  size_t off_buf[2][2] = {{0, 0}, {0, 0}};
  size_t off_partial = 0, off_comp = 0, total = 0;
  int32_t ppg = 64, groups = 0;
};

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

RunLayout layout_for(const hsf_plan &p, size_t num_bits, uint64_t window, uint64_t chunk) {
  RunLayout L;
  L.chunk = chunk;
  const size_t csz = p.precision == HSF_PREC_C64 ? 8 : 16;
  const int B = (int)p.blocks.size();
  size_t off = 0;
  for (int s = 0; s < 2; ++s) {
    // the largest level held at once: nodes per level within one chunk
    uint64_t maxn = 1;
    for (int k = 0; k <= B; ++k) maxn = std::max<uint64_t>(maxn, (chunk + p.below[k] - 1) / p.below[k] + 1);
    maxn = std::min<uint64_t>(maxn, chunk);
    L.state_bytes[s] = ((size_t)1 << p.side[s].h) * csz;
    for (int j = 0; j < 2; ++j) {
      L.off_buf[s][j] = off;
      off += align256(maxn * L.state_bytes[s]);
    }
  }
  if (num_bits > 0) {
    L.ppg = 64;
    while ((chunk + L.ppg - 1) / L.ppg > 65535) L.ppg *= 2;
    L.groups = (int32_t)((chunk + L.ppg - 1) / L.ppg);
    L.off_partial = off;
    off += align256((size_t)L.groups * num_bits * 16);
    L.off_comp = off;
    off += align256(num_bits * 16);
  } else {
    const uint64_t count = window ? window : (1ull << p.n);
    L.off_comp = off;
    off += align256(count * 16);
  }
  L.total = off;
  return L;
}

bool choose_layout(const hsf_plan &p, size_t num_bits, uint64_t window, size_t budget, RunLayout &out) {
  const int B = (int)p.blocks.size();
  for (int k = 0; k <= B; ++k) {           // below[0] = all paths, below[B] = 1
    RunLayout L = layout_for(p, num_bits, window, p.below[k]);
    if (budget == 0 || L.total <= budget) { out = L; return true; }
  }
  return false;
}

// Launch one kernel (fn) and, with profiling on, bracket it with events on `st`.
template <typename F>
hsf_status launch(hsf_plan &p, int kind, double bytes, double flops, cudaStream_t st, F fn) {
  if (!g_profiling.load()) {
    CUDA_TRY(fn());
    g_launches++;
    return HSF_OK;
  }
  hsf_plan::ProfRec r{kind, nullptr, nullptr, bytes, flops};
  CUDA_TRY(cudaEventCreate(&r.e0));
  CUDA_TRY(cudaEventCreate(&r.e1));
  CUDA_TRY(cudaEventRecord(r.e0, st));
  CUDA_TRY(fn());
  g_launches++;
  CUDA_TRY(cudaEventRecord(r.e1, st));
  p.prof.push_back(r);
  return HSF_OK;
}

#define LAUNCH(kind, bytes, flops, call)                                                 \
  do {                                                                                   \
    hsf_status s_ = launch(*p, kind, bytes, flops, st, [&]() { return (call); });        \
    if (s_ != HSF_OK) return s_;                                                         \
  } while (0)

}  // namespace

extern "C" {

void hsf_set_profiling(int32_t on) { g_profiling.store(on ? 1 : 0); }

uint64_t hsf_launch_count(void) { return g_launches.load(); }

hsf_status hsf_profile_collect(hsf_plan *p, hsf_kernel_stat *stats, int32_t cap) {
  if (!p || (!stats && cap > 0)) return fail(HSF_EINVAL, "NULL argument");
  for (int i = 0; i < cap; ++i) stats[i] = hsf_kernel_stat{0, 0.0, 0.0, 0.0};
  for (auto &r : p->prof) {
    float ms = 0.f;
    CUDA_TRY(cudaEventSynchronize(r.e1));
    CUDA_TRY(cudaEventElapsedTime(&ms, r.e0, r.e1));
    if (r.kind < cap) {
      stats[r.kind].launches += 1;
      stats[r.kind].ms += ms;
      stats[r.kind].bytes += r.bytes;
      stats[r.kind].flops += r.flops;
    }
    cudaEventDestroy(r.e0);
    cudaEventDestroy(r.e1);
  }
  p->prof.clear();
  return HSF_OK;
}

const char *hsf_last_error(void) { return g_err.c_str(); }
const char *hsf_version(void) { return "hsf-gb300 0.1 (sm_103a)"; }

hsf_status hsf_plan_create(const hsf_circuit *circuit, int32_t cut_l, const hsf_blocks *blocks,
                           const hsf_plan_opts *opts, hsf_plan **out) {
  if (!out) return fail(HSF_EINVAL, "out must not be NULL");
  *out = nullptr;
  std::unique_ptr<hsf_plan> p(new (std::nothrow) hsf_plan());
  if (!p) return fail(HSF_ENOMEM, "host allocation failed");
  hsf_status st = validate_and_load(*p, circuit, cut_l, blocks, opts);
  if (st != HSF_OK) return st;
  {
    std::vector<std::pair<bool, int>> order;
    st = execution_order(*p, order);
    if (st != HSF_OK) return st;
  }
  st = decompose_blocks(*p);
  if (st != HSF_OK) return st;
  const int B = (int)p->blocks.size();
  p->radix.assign(B + 1, 1);
  p->below.assign(B + 1, 1);
  long double paths = 1;
  for (int b = 0; b < B; ++b) {
    p->radix[b + 1] = (uint64_t)p->blocks[b].rank;
    paths *= p->blocks[b].rank;
  }
  if (paths > (long double)p->max_paths || paths > (long double)(1ull << 62))
    return fail(HSF_ERANK, "%.0Lf paths exceed max_paths %llu", paths, (unsigned long long)p->max_paths);
  p->num_paths = (uint64_t)paths;
  for (int k = B - 1; k >= 0; --k) p->below[k] = p->below[k + 1] * p->radix[k + 1];
  int64_t nodes = 0;
  for (int k = 0; k <= B; ++k) nodes += (int64_t)(p->num_paths / p->below[k]);
  p->tree_nodes = nodes;
  st = build_programs(*p);
  if (st != HSF_OK) return st;
  st = upload_programs(*p);
  if (st != HSF_OK) return st;
  *out = p.release();
  return HSF_OK;
}

hsf_status hsf_plan_get_info(const hsf_plan *p, hsf_plan_info *info) {
  if (!p || !info) return fail(HSF_EINVAL, "NULL argument");
  std::memset(info, 0, sizeof *info);
  info->n = p->n;
  info->n_a = p->na;
  info->n_b = p->nb;
  info->num_blocks = (int)p->blocks.size();
  info->num_paths = p->num_paths;
  info->precision = p->precision;
  int mr = 0;
  for (auto &b : p->blocks) mr = std::max(mr, b.rank);
  info->max_rank = mr;
  info->tree_nodes = p->tree_nodes;
  info->num_launches = p->launches;
  return HSF_OK;
}

hsf_status hsf_plan_get_sigma(const hsf_plan *p, int32_t block, double *sigma, int32_t cap, int32_t *rank) {
  if (!p) return fail(HSF_EINVAL, "NULL plan");
  if (block < 0 || block >= (int)p->blocks.size()) return fail(HSF_EINVAL, "block %d out of range", block);
  const BlockH &b = p->blocks[block];
  if (rank) *rank = b.rank;
  if (sigma)
    for (int i = 0; i < std::min<int>(cap, b.rank); ++i) sigma[i] = b.sigma[i];
  return HSF_OK;
}

void hsf_plan_destroy(hsf_plan *p) {
  if (!p) return;
  for (auto &r : p->prof) { cudaEventDestroy(r.e0); cudaEventDestroy(r.e1); }
  if (p->dev_table) cudaFree(p->dev_table);
  delete p;
}

hsf_status hsf_workspace_size(const hsf_plan *p, size_t num_bits, uint64_t window, size_t budget, size_t *bytes) {
  if (!p || !bytes) return fail(HSF_EINVAL, "NULL argument");
  if (num_bits == 0 && window == 0 && p->n > 34) return fail(HSF_EINVAL, "full output of 2^%d amplitudes", p->n);
  RunLayout L;
  if (!choose_layout(*p, num_bits, window, budget, L))
    return fail(HSF_ENOMEM, "no path chunk fits a %zu-byte budget", budget);
  *bytes = L.total;
  return HSF_OK;
}

hsf_status hsf_run(hsf_plan *p, const uint64_t *bits, size_t num, uint64_t window, uint64_t path_begin,
                   uint64_t path_end, void *out, void *workspace, size_t ws_bytes, void *stream) {
  if (!p || !out || !workspace) return fail(HSF_EINVAL, "NULL plan, output or workspace");
  if (num > 0 && !bits) return fail(HSF_EINVAL, "num > 0 but bitstrings is NULL");
  if ((uintptr_t)workspace % 256) return fail(HSF_EINVAL, "workspace must be 256-byte aligned");
  if (path_begin == 0 && path_end == 0) path_end = p->num_paths;
  if (path_begin > path_end || path_end > p->num_paths)
    return fail(HSF_EINVAL, "path range [%llu, %llu) outside [0, %llu)", (unsigned long long)path_begin,
                (unsigned long long)path_end, (unsigned long long)p->num_paths);
  if (num == 0) {
    if (p->n > 34 && window == 0) return fail(HSF_EINVAL, "full output of 2^%d amplitudes", p->n);
    if (window > (1ull << std::min(p->n, 62))) return fail(HSF_EINVAL, "window larger than 2^n");
  }
  RunLayout L;
  if (!choose_layout(*p, num, window, ws_bytes, L))
    return fail(HSF_ENOMEM, "workspace of %zu bytes is too small for one path chunk", ws_bytes);
  cudaStream_t st = (cudaStream_t)stream;
  unsigned char *ws = (unsigned char *)workspace;
  double *outd = (double *)out;
  double *comp = (double *)(ws + L.off_comp);
  const uint64_t count = num > 0 ? num : (window ? window : (1ull << p->n));
  const double csz = p->precision == HSF_PREC_C64 ? 8.0 : 16.0;
  LAUNCH(HSF_KERNEL_OTHER, 16.0 * count, 0.0, launch_zero(outd, (int64_t)(2 * count), st));
  LAUNCH(HSF_KERNEL_OTHER, 16.0 * count, 0.0, launch_zero(comp, (int64_t)(2 * count), st));
  const int B = (int)p->blocks.size();
  const uint64_t C = L.chunk;
  for (uint64_t a0 = (path_begin / C) * C; a0 < path_end; a0 += C) {
    const uint64_t c0 = std::max(a0, path_begin), c1 = std::min(a0 + C, path_end);
    if (c0 >= c1) continue;
    const void *leaf[2] = {nullptr, nullptr};
    for (int s = 0; s < 2; ++s) {
      const SideH &sd = p->side[s];
      int64_t prev_lo = 0;
      for (int k = 0; k <= B; ++k) {
        const int64_t lo = (int64_t)(c0 / p->below[k]);
        const int64_t hi = (int64_t)((c1 - 1) / p->below[k]) + 1;
        void *dst = ws + L.off_buf[s][k & 1];
        const void *par = ws + L.off_buf[s][(k + 1) & 1];
        const LevelH &lv = sd.levels[k];
        for (size_t pi = 0; pi < lv.passes.size(); ++pi) {
          const PassH &ps = lv.passes[pi];
          SweepArgs a{};
          a.ops = (const DevOp *)((unsigned char *)p->dev_table + ps.ops_off);
          a.num_ops = ps.num_ops;
          a.h = sd.h;
          a.mats = (unsigned char *)p->dev_table + ps.mats_off;
          a.read_parent = (pi == 0 && k > 0) ? 1 : 0;
          a.init_zero = (pi == 0 && k == 0) ? 1 : 0;
          a.src = a.read_parent ? par : dst;
          a.dst = dst;
          a.active_mask = ps.active;
          a.t = ps.t;
          a.radix = (int32_t)p->radix[k];
          a.node_lo = lo;
          a.parent_lo = prev_lo;
          a.num_nodes = hi - lo;
          a.tiles_per_node = 1 << (sd.h - ps.t);
          const double amps = (double)a.num_nodes * (double)(1ull << sd.h);
          double fl = 0.0;
          for (const OpH &op : ps.ops) fl += amps * (op.type == OP_DENSE ? 8.0 * (1 << op.nq) : 6.0);
          LAUNCH(HSF_KERNEL_SWEEP, 2.0 * amps * csz, fl, launch_sweep(a, p->precision, st));
        }
        prev_lo = lo;
        if (k == B) leaf[s] = dst;
      }
    }
    const int64_t np = (int64_t)(c1 - c0);
    if (num > 0) {
      GatherArgs g{};
      g.A = leaf[0];
      g.B = leaf[1];
      g.num_paths = np;
      g.ha = p->na;
      g.hb = p->nb;
      g.bits = bits;
      g.S = (int64_t)num;
      g.paths_per_group = L.ppg;
      g.num_groups = (int32_t)((np + L.ppg - 1) / L.ppg);
      g.partial = (double *)(ws + L.off_partial);
      LAUNCH(HSF_KERNEL_GATHER, (double)np * g.S * 2.0 * csz + 16.0 * g.num_groups * g.S,
             8.0 * (double)np * g.S, launch_gather_dot(g, p->precision, st));
      LAUNCH(HSF_KERNEL_REDUCE, 16.0 * g.num_groups * g.S + 64.0 * g.S, 0.0,
             launch_reduce_partials(g.partial, g.num_groups, g.S, outd, comp, st));
    } else {
      WindowArgs w{};
      w.A = leaf[0];
      w.B = leaf[1];
      w.num_paths = np;
      w.ha = p->na;
      w.hb = p->nb;
      const uint64_t nbw = 1ull << p->nb;
      w.window = count;
      w.M = (int64_t)((count + nbw - 1) / nbw);
      w.N = (int64_t)std::min<uint64_t>(count, nbw);
      w.out = outd;
      w.comp = comp;
      LAUNCH(HSF_KERNEL_WINDOW, (double)np * (w.M + w.N) * csz + 64.0 * w.M * w.N,
             8.0 * (double)np * w.M * w.N, launch_window(w, p->precision, st));
    }
  }
  LAUNCH(HSF_KERNEL_OTHER, 48.0 * count, 0.0, launch_finalize(outd, comp, (int64_t)(2 * count), st));
  return HSF_OK;
}

}  // extern "C"
