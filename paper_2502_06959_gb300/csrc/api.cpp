// C ABI of the joint-cut HSF library: plan creation (see planner.cpp) and the run.
//
// Running (Sec. II-B): the path tree is walked level by level over chunks of paths
// (subtrees sized to the workspace).  Every level is one sweep launch per tile pass
// and side; the children of a node start from its state (prefix reuse).  The leaves
// are either contracted directly at the requested bitstrings (leaf_contract), or
// materialised and summed by gather_dot (bitstrings) / window (full output).  Path
// chunks are folded into the FP64 output with Neumaier-compensated additions.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <functional>
#include <map>
#include <memory>
#include <mutex>
#include <queue>
#include <set>
#include <string>
#include <vector>

#include "plan.h"

using namespace hsf;

namespace {

std::atomic<int> g_profiling{0};

// Allocator of plan-owned workspaces (hsf_set_allocator); NULL functions: cudaMalloc.
std::mutex g_alloc_mu;
hsf_alloc_fn g_alloc = nullptr;
hsf_free_fn g_release = nullptr;
void *g_alloc_ctx = nullptr;

#define CUDA_TRY(expr)                                                                   \
  do {                                                                                   \
    cudaError_t e_ = (expr);                                                             \
    if (e_ != cudaSuccess)                                                               \
      return set_error(HSF_ECUDA, "%s failed: %s", #expr, cudaGetErrorString(e_));       \
  } while (0)

struct RunLayout {
  uint64_t chunk = 0;          // leaves per chunk (a subtree size)
  bool leaf = false;           // leaf level contracted at the bitstrings
  bool tc = false;             // window output on the tensor cores
  size_t off_buf[2][2] = {{0, 0}, {0, 0}};
  size_t off_partial = 0, off_sync = 0, off_comp = 0, off_index = 0, off_gemm = 0, off_sort = 0, total = 0;
  size_t off_mask[2] = {0, 0};   // leaf contraction: segments of the deepest level that bitstrings read
  bool dots = false;             // leaf in the dot form (use_leaf_dots)
  size_t off_dots[2] = {0, 0};   // dot form: [nodes of the deepest level][bitstrings] x 32 bytes per side
  size_t off_dsort = 0;          // dot form: the bitstrings grouped by segment (dot_sort_layout)
  int32_t ppg = 64, groups = 0;
};

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

bool use_leaf(const hsf_plan &p, size_t num_bits) {
  return num_bits > 0 && p.leaf_c > 0 && !(p.flags & HSF_FLAG_NO_LEAF_CONTRACT);
}

// The dot form of the factored leaf (HSF_FLAG_LEAF_DOTS): the deepest level (FP16
// tensor-core kernel, nothing after its product) writes the leaf's four chunk dots per
// (child, bitstring) instead of its children, where the operators factor on 16-amplitude
// chunks (one segment of the kernel's rows) and the dots take no more memory than the
// children.
bool use_leaf_dots(const hsf_plan &p, size_t num_bits) {
  if (!use_leaf(p, num_bits) || !(p.flags & HSF_FLAG_LEAF_DOTS) || p.precision != HSF_PREC_C64) return false;
  const int B = (int)p.blocks.size(), top = B - 1;
  if (top < 1 || p.leaf_pf < 0 || p.leaf_pf > 3 || p.leaf_c != 4 || num_bits >= 65536) return false;
  if (p.radix[B] < 3 || p.radix[B] > 4) return false;     // the factored leaf's digit counts
  for (int s = 0; s < 2; ++s) {
    const SideH &sd = p.side[s];
    if (sd.h < kMmaMinH || sd.h > 24 || (uint64_t)num_bits * 4 > (1ull << sd.h)) return false;
    const LevelH &lv = sd.levels[top];
    if (!lv.mma || !lv.post.empty() || !lv.passes.empty()) return false;
  }
  return true;
}

RunLayout layout_for(const hsf_plan &p, size_t num_bits, uint64_t window, uint64_t chunk) {
  RunLayout L;
  L.chunk = chunk;
  L.leaf = use_leaf(p, num_bits);
  L.dots = use_leaf_dots(p, num_bits);
  const size_t csz = p.precision == HSF_PREC_C64 ? 8 : 16;
  const int B = (int)p.blocks.size();
  const int top = L.leaf ? B - 1 : B;          // deepest level held in memory
  auto nodes_in_chunk = [&](int k) {           // nodes of level k inside one chunk
    return std::min<uint64_t>(chunk, (chunk + p.below[k] - 1) / p.below[k] + 1);
  };
  size_t off = 0;
  for (int s = 0; s < 2; ++s) {
    uint64_t maxn = 1;
    // (dot form: the deepest level's children are not stored)
    for (int k = 0; k <= (L.dots ? top - 1 : top); ++k) maxn = std::max<uint64_t>(maxn, nodes_in_chunk(k));
    const size_t sb = ((size_t)1 << p.side[s].h) * csz;
    for (int j = 0; j < 2; ++j) {
      L.off_buf[s][j] = off;
      off += align256(maxn * sb);
    }
    if (L.dots) {
      L.off_dots[s] = off;
      off += align256(nodes_in_chunk(top) * num_bits * 32);
    }
  }
  if (L.dots) {
    L.off_dsort = off;
    off += align256(dot_sort_bytes((int64_t)num_bits, p.side[0].h, p.side[1].h));
  }
  if (num_bits > 0) {
    const uint64_t units = L.leaf ? (chunk + p.radix[B] - 1) / p.radix[B] + 1 : chunk;
    L.ppg = 64;
    while ((units + L.ppg - 1) / L.ppg > 65535) L.ppg *= 2;
    L.groups = (int32_t)((units + L.ppg - 1) / L.ppg);
    L.off_partial = off;
    off += align256((size_t)L.groups * num_bits * 16);
    L.off_sync = off;
    off += 256;
    L.off_index = off;
    off += align256(num_bits * 16);
    L.off_comp = off;
    off += align256(num_bits * 16);
    if (L.leaf && !L.dots && p.side[0].h >= 5 && p.side[1].h >= 5 && p.side[0].h <= 28 && p.side[1].h <= 28) {
      for (int s = 0; s < 2; ++s) {
        L.off_mask[s] = off;
        off += align256(std::max<size_t>(4, ((size_t)1 << (p.side[s].h - 4)) / 8));
      }
    }
    if (L.leaf && num_bits >= 65536) {       // the streaming leaf's sorted bitstrings
      L.off_sort = off;
      off += align256(num_bits * 24) + align256(((size_t)1 << kSortBits) * 4);
    }
  } else {
    const uint64_t count = window ? window : (1ull << p.n);
    const uint64_t nbw = 1ull << p.nb;
    const uint64_t M = (count + nbw - 1) / nbw, N = std::min<uint64_t>(count, nbw);
    L.off_index = off;
    off += align256((M + N) * 8);
    L.off_comp = off;
    off += align256(count * 16);
    if (p.gemm_mode != HSF_GEMM_FP32) {
      L.tc = true;
      L.off_gemm = off;
      off += align256(path_gemm_operand_bytes(p.gemm_mode, (int64_t)M, (int64_t)N, (int64_t)chunk));
    }
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

PermArgs perm_of(const SideH &sd) {
  PermArgs pa{};
  pa.h = sd.h;
  for (int q = 0; q < sd.h; ++q) pa.store[q] = sd.store[q];
  return pa;
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

// Schroedinger plan: the full 2^n state is swept in place in the workspace, pass by pass
// (the first pass starts every tile from |0...0>), then the requested amplitudes are read
// out (bit q of a bitstring is qubit q, identity storage order).
hsf_status run_schrodinger(hsf_plan &pl, const uint64_t *bits, size_t num, uint64_t window, double *outd,
                           void *workspace, size_t ws_bytes, cudaStream_t st) {
  hsf_plan *p = &pl;
  const size_t csz = p->precision == HSF_PREC_C64 ? 8 : 16;
  const size_t need = ((size_t)1 << p->n) * csz;
  if (ws_bytes < need) return set_error(HSF_ENOMEM, "workspace of %zu bytes cannot hold the %zu-byte state", ws_bytes, need);
  const SideH &sd = p->side[0];
  const LevelH &lv = sd.levels[0];
  const double amps = (double)(1ull << sd.h);
  for (size_t pi = 0; pi < lv.passes.size(); ++pi) {
    const PassH &ps = lv.passes[pi];
    SweepArgs a{};
    a.ops = (const DevOp *)((unsigned char *)p->dev_table + ps.ops_off);
    a.num_ops = ps.num_ops;
    a.h = sd.h;
    a.mats = (unsigned char *)p->dev_table + ps.mats_off;
    a.read_parent = 0;
    a.init_zero = pi == 0 ? 1 : 0;
    a.src = workspace;
    a.dst = workspace;
    a.active_mask = ps.active;
    a.t = ps.t;
    a.radix = 1;
    a.node_lo = 0;
    a.parent_lo = 0;
    a.num_nodes = 1;
    a.tiles_per_node = (int32_t)(1ll << (sd.h - ps.t));
    a.groups = ps.groups.empty() ? nullptr : (const DevGroup *)((unsigned char *)p->dev_table + ps.groups_off);
    a.num_groups = (int32_t)ps.groups.size();
    a.rbits = p->rbits;
    const size_t blk = ps.table_end - ps.ops_off;
    if (!ps.groups.empty() && blk <= (size_t)kMaxStageBytes) {
      a.stage_src = (unsigned char *)p->dev_table + ps.ops_off;
      a.stage_bytes = (int32_t)((blk + 15) / 16 * 16);
      a.stage_mats_off = (int32_t)(ps.mats_off - ps.ops_off);
      a.stage_groups_off = (int32_t)(ps.groups_off - ps.ops_off);
    }
    double fl = 0.0;
    for (const OpH &op : ps.ops) fl += amps * (op.type == OP_DENSE ? 8.0 * (1 << op.nq) : 6.0);
    // the first pass only writes (its tiles start from |0...0>)
    LAUNCH(HSF_KERNEL_SWEEP, (pi == 0 ? 1.0 : 2.0) * amps * csz, fl, launch_sweep(a, p->precision, st));
  }
  const int64_t count = num > 0 ? (int64_t)num : (int64_t)(window ? window : (1ull << p->n));
  LAUNCH(HSF_KERNEL_OTHER, (double)count * (16.0 + csz + (num ? 8.0 : 0.0)), 0.0,
         launch_state_gather(workspace, p->precision, num > 0 ? bits : nullptr, count, outd,
                             p->dev_status + kStatusNumeric, st));
  return HSF_OK;
}

}  // namespace

extern "C" {

void hsf_set_profiling(int32_t on) { g_profiling.store(on ? 1 : 0); }

void hsf_set_allocator(hsf_alloc_fn alloc, hsf_free_fn release, void *ctx) {
  std::lock_guard<std::mutex> lock(g_alloc_mu);
  g_alloc = (alloc && release) ? alloc : nullptr;
  g_release = (alloc && release) ? release : nullptr;
  g_alloc_ctx = (alloc && release) ? ctx : nullptr;
}

uint64_t hsf_launch_count(void) { return g_launches.load(); }

hsf_status hsf_profile_collect(hsf_plan *p, hsf_kernel_stat *stats, int32_t cap) {
  if (!p || (!stats && cap > 0)) return set_error(HSF_EINVAL, "NULL argument");
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

const char *hsf_last_error(void) { return hsf::last_error(); }
const char *hsf_version(void) { return "hsf-gb300 0.1 (sm_103a)"; }

hsf_status hsf_plan_create(const hsf_circuit *circuit, int32_t cut_l, const hsf_blocks *blocks,
                           const hsf_plan_opts *opts, hsf_plan **out) {
  if (!out) return set_error(HSF_EINVAL, "out must not be NULL");
  *out = nullptr;
  std::unique_ptr<hsf_plan> p(new (std::nothrow) hsf_plan());
  if (!p) return set_error(HSF_ENOMEM, "host allocation failed");
  hsf_status st = validate_and_load(*p, circuit, cut_l, blocks, opts);
  if (st != HSF_OK) return st;
  st = check_order(*p);
  if (st != HSF_OK) return st;
  st = decompose_blocks(*p);
  if (st != HSF_OK) return st;
  st = finish_plan(*p);
  if (st != HSF_OK) return st;
  *out = p.release();
  return HSF_OK;
}

hsf_status hsf_plan_create_schrodinger(const hsf_circuit *circuit, const hsf_plan_opts *opts, hsf_plan **out) {
  if (!out) return set_error(HSF_EINVAL, "out must not be NULL");
  *out = nullptr;
  std::unique_ptr<hsf_plan> p(new (std::nothrow) hsf_plan());
  if (!p) return set_error(HSF_ENOMEM, "host allocation failed");
  hsf_status st = build_schrodinger(*p, circuit, opts);
  if (st != HSF_OK) return st;
  *out = p.release();
  return HSF_OK;
}

hsf_status hsf_plan_get_info(const hsf_plan *p, hsf_plan_info *info) {
  if (!p || !info) return set_error(HSF_EINVAL, "NULL argument");
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
  info->leaf_bits = p->leaf_c;
  info->num_params = p->num_params;
  return HSF_OK;
}

hsf_status hsf_plan_get_sigma(const hsf_plan *p, int32_t block, double *sigma, int32_t cap, int32_t *rank) {
  if (!p) return set_error(HSF_EINVAL, "NULL plan");
  if (block < 0 || block >= (int)p->blocks.size()) return set_error(HSF_EINVAL, "block %d out of range", block);
  const BlockH &b = p->blocks[block];
  if (rank) *rank = b.rank;
  if (sigma)
    for (int i = 0; i < std::min<int>(cap, b.rank); ++i) sigma[i] = b.sigma[i];
  return HSF_OK;
}

int64_t hsf_plan_describe(const hsf_plan *p, char *buf, int64_t cap) {
  if (!p) return -1;
  std::string out;
  char line[512];
  for (int s = 0; s < 2; ++s) {
    const SideH &sd = p->side[s];
    std::snprintf(line, sizeof line, "side %c: h=%d store=[", s == 0 ? 'a' : 'b', sd.h);
    out += line;
    for (int q = 0; q < sd.h; ++q) {
      std::snprintf(line, sizeof line, "%s%d", q ? "," : "", sd.store[q]);
      out += line;
    }
    out += "]\n";
    for (size_t k = 0; k < sd.levels.size(); ++k) {
      const LevelH &lv = sd.levels[k];
      std::snprintf(line, sizeof line, " level %zu: radix %llu, %zu ops, %s\n", k,
                    (unsigned long long)p->radix[k], lv.ops.size(),
                    ((lv.mma ? std::string("tensor-core product (") + (lv.post.empty() ? "FP16x3" : "TF32x3") +
                                   ") on the 6 lowest storage bits" +
                                   (lv.post.empty() ? std::string()
                                                    : " + " + std::to_string(lv.post.size()) + " ops in its epilogue") +
                                   ", then "
                             : std::string()) +
                     std::to_string(lv.passes.size()) + " passes")
                        .c_str());
      out += line;
      if (!lv.post.empty()) {
        out += "  epilogue ops:";
        for (const OpH &op : lv.post) {
          std::snprintf(line, sizeof line, " %s%d(%d%s%s)", op.type == OP_DENSE ? "D" : "d", op.nq, op.q[0],
                        op.nq > 1 ? "," : "", op.nq > 1 ? std::to_string(op.q[1]).c_str() : "");
          out += line;
        }
        out += "\n";
      }
      for (size_t pi = 0; pi < lv.passes.size(); ++pi) {
        const PassH &ps = lv.passes[pi];
        std::snprintf(line, sizeof line, "  pass %zu: active=0x%llx t=%d ops=%zu groups=%zu\n", pi,
                      (unsigned long long)ps.active, ps.t, ps.ops.size(), ps.groups.size());
        out += line;
        for (size_t g = 0; g < ps.groups.size(); ++g) {
          const GroupH &G = ps.groups[g];
          std::snprintf(line, sizeof line, "   group %zu: slots=%d,%d,%d,%d,%d ops[%d..%d):", g, G.slots[0], G.slots[1],
                        G.slots[2], G.slots[3], G.slots[4], G.first_op, G.first_op + G.num_ops);
          out += line;
          for (int o = G.first_op; o < G.first_op + G.num_ops; ++o) {
            const OpH &op = ps.ops[o];
            std::snprintf(line, sizeof line, " %s%d(%d%s%s%s%s)", op.type == OP_DENSE ? "D" : "d", op.nq, op.q[0],
                          op.nq > 1 ? "," : "", op.nq > 1 ? std::to_string(op.q[1]).c_str() : "",
                          op.nq > 2 ? "," : "", op.nq > 2 ? std::to_string(op.q[2]).c_str() : "");
            out += line;
          }
          out += "\n";
        }
      }
    }
  }
  for (size_t b = 0; b < p->blocks.size(); ++b) {
    const BlockH &bk = p->blocks[b];
    if (bk.closed >= 0)
      std::snprintf(line, sizeof line, "block %zu: qubits %zu|%zu rank %d closed-form cascade (hub on side %c)\n", b,
                    bk.qa.size(), bk.qb.size(), bk.rank, bk.closed == 0 ? 'a' : 'b');
    else
      std::snprintf(line, sizeof line, "block %zu: qubits %zu|%zu rank %d SVD sweeps %d residual %.3e\n", b,
                    bk.qa.size(), bk.qb.size(), bk.rank, bk.sweeps, bk.residual);
    out += line;
  }
  std::snprintf(line, sizeof line, "leaf_bits=%d paths=%llu%s\n", p->leaf_c, (unsigned long long)p->num_paths,
                p->leaf_pf >= 0 ? " leaf=factored" : "");
  out += line;
  if (buf && cap > 0) {
    const int64_t n = std::min<int64_t>(cap - 1, (int64_t)out.size());
    std::memcpy(buf, out.data(), (size_t)n);
    buf[n] = 0;
  }
  return (int64_t)out.size() + 1;
}

hsf_status hsf_sync(hsf_plan *p, void *stream) {
  if (!p) return set_error(HSF_EINVAL, "NULL plan");
  CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
  int32_t status[2] = {0, 0};
  CUDA_TRY(cudaMemcpyAsync(status, p->dev_status, sizeof status, cudaMemcpyDeviceToHost, plan_stream()));
  CUDA_TRY(cudaStreamSynchronize(plan_stream()));
  if (status[kStatusWait] != 0 || status[kStatusNumeric] != 0) {
    CUDA_TRY(cudaMemsetAsync(p->dev_status, 0, sizeof status, plan_stream()));
    CUDA_TRY(cudaStreamSynchronize(plan_stream()));
  }
  if (status[kStatusWait] != 0)
    return set_error(HSF_ETIMEOUT, "a bounded device-side wait expired (code %d); results of the "
                                   "affected run are invalid", status[kStatusWait]);
  if (status[kStatusNumeric] != 0)
    return set_error(HSF_ENUMERIC, "an amplitude of an earlier run is NaN or infinite");
  return HSF_OK;
}

void hsf_plan_destroy(hsf_plan *p) { delete p; }

hsf_status hsf_workspace_size(const hsf_plan *p, size_t num_bits, uint64_t window, size_t budget, size_t *bytes) {
  if (!p || !bytes) return set_error(HSF_EINVAL, "NULL argument");
  if (p->schrodinger) {
    const size_t need = align256(((size_t)1 << p->n) * (p->precision == HSF_PREC_C64 ? 8 : 16));
    if (num_bits == 0 && window == 0 && p->n > 34) return set_error(HSF_EINVAL, "full output of 2^%d amplitudes", p->n);
    if (budget && need > budget)
      return set_error(HSF_ENOMEM, "the 2^%d-amplitude state needs %zu bytes, more than the %zu-byte budget", p->n, need,
                       budget);
    *bytes = need;
    return HSF_OK;
  }
  if (num_bits == 0 && window == 0 && p->n > 34) return set_error(HSF_EINVAL, "full output of 2^%d amplitudes", p->n);
  RunLayout L;
  if (!choose_layout(*p, num_bits, window, budget, L))
    return set_error(HSF_ENOMEM, "no path chunk fits a %zu-byte budget", budget);
  *bytes = L.total;
  return HSF_OK;
}

hsf_status hsf_run(hsf_plan *p, const uint64_t *bits, size_t num, uint64_t window, uint64_t path_begin,
                   uint64_t path_end, void *out, void *workspace, size_t ws_bytes, void *stream) {
  if (!p || !out) return set_error(HSF_EINVAL, "NULL plan or output");
  if (!workspace) {
    // plan-owned workspace, sized for 60% of the free device memory (paths in flight
    // shrink to fit), made once and grown only when a request needs more
    if (num == 0 && window == 0 && p->n > 34) return set_error(HSF_EINVAL, "full output of 2^%d amplitudes", p->n);
    size_t free_b = 0, total_b = 0;
    CUDA_TRY(cudaMemGetInfo(&free_b, &total_b));
    size_t need = 0;
    hsf_status ws_st = hsf_workspace_size(p, num, window, (size_t)((double)(free_b + p->own_ws_bytes) * 0.6), &need);
    if (ws_st != HSF_OK) return ws_st;
    if (need > p->own_ws_bytes) {
      if (p->own_ws) {
        CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
        if (p->own_release) p->own_release(p->own_ctx, p->own_ws, stream);
        else CUDA_TRY(cudaFree(p->own_ws));
        p->own_ws = nullptr;
        p->own_ws_bytes = 0;
      }
      void *mem = nullptr;
      {
        std::lock_guard<std::mutex> lock(g_alloc_mu);
        if (g_alloc) {
          mem = g_alloc(g_alloc_ctx, need, stream);
          p->own_release = g_release;
          p->own_ctx = g_alloc_ctx;
        } else {
          if (cudaMalloc(&mem, need) != cudaSuccess) mem = nullptr;
          p->own_release = nullptr;
          p->own_ctx = nullptr;
        }
      }
      if (!mem) return set_error(HSF_ENOMEM, "allocating a %zu-byte plan workspace failed", need);
      if ((uintptr_t)mem % 256) {
        if (p->own_release) p->own_release(p->own_ctx, mem, stream);
        else cudaFree(mem);
        return set_error(HSF_ENOMEM, "the registered allocator returned memory that is not 256-byte aligned");
      }
      p->own_ws = mem;
      p->own_ws_bytes = need;
    }
    workspace = p->own_ws;
    ws_bytes = p->own_ws_bytes;
  }
  if (num > 0 && !bits) return set_error(HSF_EINVAL, "num > 0 but bitstrings is NULL");
  if ((uintptr_t)workspace % 256) return set_error(HSF_EINVAL, "workspace must be 256-byte aligned");
  if (path_begin == 0 && path_end == 0) path_end = p->num_paths;
  if (path_begin > path_end || path_end > p->num_paths)
    return set_error(HSF_EINVAL, "path range [%llu, %llu) outside [0, %llu)", (unsigned long long)path_begin,
                     (unsigned long long)path_end, (unsigned long long)p->num_paths);
  if (num == 0) {
    if (p->n > 34 && window == 0) return set_error(HSF_EINVAL, "full output of 2^%d amplitudes", p->n);
    if (window > (1ull << std::min(p->n, 62))) return set_error(HSF_EINVAL, "window larger than 2^n");
  }
  if (p->schrodinger) return run_schrodinger(*p, bits, num, window, (double *)out, workspace, ws_bytes,
                                             (cudaStream_t)stream);
  RunLayout L;
  if (!choose_layout(*p, num, window, ws_bytes, L))
    return set_error(HSF_ENOMEM, "workspace of %zu bytes is too small for one path chunk", ws_bytes);
  cudaStream_t st = (cudaStream_t)stream;
  unsigned char *ws = (unsigned char *)workspace;
  double *outd = (double *)out;
  double *comp = (double *)(ws + L.off_comp);
  const uint64_t count = num > 0 ? num : (window ? window : (1ull << p->n));
  const double csz = p->precision == HSF_PREC_C64 ? 8.0 : 16.0;
  LAUNCH(HSF_KERNEL_OTHER, 16.0 * count, 0.0, launch_zero(outd, (int64_t)(2 * count), st));
  LAUNCH(HSF_KERNEL_OTHER, 16.0 * count, 0.0, launch_zero(comp, (int64_t)(2 * count), st));
  // storage index of every requested amplitude on each side
  uint64_t *ia = nullptr, *ib = nullptr;
  bool sorted = false;                         // streaming leaf: bitstrings sorted once per run
  const uint64_t nbw = 1ull << p->nb;
  const int64_t M = (int64_t)((count + nbw - 1) / nbw), N = (int64_t)std::min<uint64_t>(count, nbw);
  if (num > 0) {
    ia = (uint64_t *)(ws + L.off_index);
    ib = ia + num;
    IndexArgs ix{};
    ix.bits = bits;
    ix.S = (int64_t)num;
    ix.nb = p->nb;
    ix.ha = p->na;
    ix.hb = p->nb;
    for (int q = 0; q < p->na; ++q) ix.store_a[q] = p->side[0].store[q];
    for (int q = 0; q < p->nb; ++q) ix.store_b[q] = p->side[1].store[q];
    ix.ia = ia;
    ix.ib = ib;
    LAUNCH(HSF_KERNEL_OTHER, 24.0 * num, 0.0, launch_index_prep(ix, st));
    if (L.off_mask[0])
      LAUNCH(HSF_KERNEL_OTHER, 16.0 * num, 0.0,
             launch_chunk_mask(ia, ib, (int64_t)num, p->leaf_c, p->na, p->nb, (uint32_t *)(ws + L.off_mask[0]),
                               (uint32_t *)(ws + L.off_mask[1]), st));
    if (L.dots)
      LAUNCH(HSF_KERNEL_OTHER, 40.0 * num, 0.0,
             launch_dot_sort(ia, ib, (int64_t)num, p->na, p->nb, (unsigned char *)p->dev_table + p->side[0].leaf_s_off,
                             (unsigned char *)p->dev_table + p->side[1].leaf_s_off,
                             dot_sort_layout(ws + L.off_dsort, (int64_t)num, p->na, p->nb), st));
  } else {
    ia = (uint64_t *)(ws + L.off_index);
    ib = ia + M;
    LAUNCH(HSF_KERNEL_OTHER, 8.0 * M, 0.0, launch_range_index(ia, M, perm_of(p->side[0]), st));
    LAUNCH(HSF_KERNEL_OTHER, 8.0 * N, 0.0, launch_range_index(ib, N, perm_of(p->side[1]), st));
  }
  const int B = (int)p->blocks.size();
  const int top = L.leaf ? B - 1 : B;
  const uint64_t C = L.chunk;
  // The two halves are independent until they are combined: side b runs on a second
  // stream forked from and joined back into the caller's (events; also under capture).
  // With profiling on, side b stays on the caller's stream, so that every launch's event
  // pair times that launch alone.
  const cudaStream_t st_main = st, st_b = g_profiling.load() ? st : side_stream();
  cudaEvent_t fork_ev = nullptr, join_ev = nullptr;
  CUDA_TRY(cudaEventCreateWithFlags(&fork_ev, cudaEventDisableTiming));
  CUDA_TRY(cudaEventCreateWithFlags(&join_ev, cudaEventDisableTiming));
  std::unique_ptr<CUevent_st, void (*)(cudaEvent_t)> fork_guard(fork_ev, [](cudaEvent_t e) { cudaEventDestroy(e); });
  std::unique_ptr<CUevent_st, void (*)(cudaEvent_t)> join_guard(join_ev, [](cudaEvent_t e) { cudaEventDestroy(e); });
  for (uint64_t a0 = (path_begin / C) * C; a0 < path_end; a0 += C) {
    const uint64_t c0 = std::max(a0, path_begin), c1 = std::min(a0 + C, path_end);
    if (c0 >= c1) continue;
    const void *last[2] = {nullptr, nullptr};
    int64_t last_lo = 0, last_hi = 0;
    CUDA_TRY(cudaEventRecord(fork_ev, st_main));
    CUDA_TRY(cudaStreamWaitEvent(st_b, fork_ev, 0));
    for (int s = 0; s < 2; ++s) {
      const cudaStream_t st = s == 0 ? st_main : st_b;   // the launches below use `st`
      const SideH &sd = p->side[s];
      int64_t prev_lo = 0;
      for (int k = 0; k <= top; ++k) {
        const int64_t lo = (int64_t)(c0 / p->below[k]);
        const int64_t hi = (int64_t)((c1 - 1) / p->below[k]) + 1;
        void *dst = ws + L.off_buf[s][k & 1];
        const void *par = ws + L.off_buf[s][(k + 1) & 1];
        const LevelH &lv = sd.levels[k];
        if (lv.mma) {
          LevelMmaArgs g{};
          g.parent = (const float *)par;
          g.child = (float *)dst;
          g.w = (unsigned char *)p->dev_table + lv.w_off;
          g.h = sd.h;
          g.radix = (int32_t)p->radix[k];
          g.node_lo = lo;
          g.num_nodes = hi - lo;
          g.parent_lo = prev_lo;
          g.err = p->dev_status;
          g.post = (unsigned char *)p->dev_table + lv.post_off;
          g.num_post = (int32_t)lv.post.size();
          // the level the leaf contraction reads: store only the segments bitstrings read
          if (L.leaf && k == top && L.off_mask[s] && lv.post.empty())
            g.store_mask = (const uint32_t *)(ws + L.off_mask[s]);
          const double amps = (double)(hi - lo) * (double)(1ull << sd.h);
          const double parents = (double)((hi - 1) / g.radix - lo / g.radix + 1) * (double)(1ull << sd.h);
          // three 128 x 128 x 128 real products (FP16 or TF32 parts) per 128 64-amplitude rows
          double bytes = (amps + parents) * csz, flops = 3.0 * 2.0 * 128.0 * 128.0 * (amps / 64.0);
          if (L.dots && k == top) {
            // dot form: the parents read, 32 bytes of dots written per (child, bitstring);
            // four dots of 8 complex terms (8 x 32 FLOP) per (child, bitstring)
            const DotSort ds = dot_sort_layout(ws + L.off_dsort, (int64_t)num, p->na, p->nb);
            g.dots = (float4 *)(ws + L.off_dots[s]);
            g.dot_off = ds.off[s];
            g.dot_list = ds.list[s];
            g.dot_T = ds.T[s];
            g.dot_count = (int64_t)num;
            g.dot_pf = p->leaf_pf;
            bytes = parents * csz + 32.0 * (double)(hi - lo) * (double)num;
            flops += 8.0 * 32.0 * (double)(hi - lo) * (double)num;
          }
          LAUNCH(lv.post.empty() ? HSF_KERNEL_LEVEL_F16 : HSF_KERNEL_LEVEL_MMA, bytes, flops, launch_level_mma(g, st));
        }
        for (size_t pi = 0; pi < lv.passes.size(); ++pi) {
          const PassH &ps = lv.passes[pi];
          SweepArgs a{};
          a.ops = (const DevOp *)((unsigned char *)p->dev_table + ps.ops_off);
          a.num_ops = ps.num_ops;
          a.h = sd.h;
          a.mats = (unsigned char *)p->dev_table + ps.mats_off;
          a.read_parent = (pi == 0 && k > 0 && !lv.mma) ? 1 : 0;   // after a product: in place
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
          a.groups = ps.groups.empty() ? nullptr : (const DevGroup *)((unsigned char *)p->dev_table + ps.groups_off);
          a.num_groups = (int32_t)ps.groups.size();
          a.rbits = p->rbits;
          const size_t blk = ps.table_end - ps.ops_off;
          if (!ps.groups.empty() && blk <= (size_t)kMaxStageBytes) {
            a.stage_src = (unsigned char *)p->dev_table + ps.ops_off;
            a.stage_bytes = (int32_t)((blk + 15) / 16 * 16);
            a.stage_mats_off = (int32_t)(ps.mats_off - ps.ops_off);
            a.stage_groups_off = (int32_t)(ps.groups_off - ps.ops_off);
          }
          const double amps = (double)a.num_nodes * (double)(1ull << sd.h);
          double fl = 0.0;
          for (const OpH &op : ps.ops) fl += amps * (op.type == OP_DENSE ? 8.0 * (1 << op.nq) : 6.0);
          LAUNCH(HSF_KERNEL_SWEEP, 2.0 * amps * csz, fl, launch_sweep(a, p->precision, st));
        }
        prev_lo = lo;
        if (k == top) {
          last[s] = dst;
          last_lo = lo;
          last_hi = hi;
        }
      }
    }
    CUDA_TRY(cudaEventRecord(join_ev, st_b));
    CUDA_TRY(cudaStreamWaitEvent(st_main, join_ev, 0));
    if (L.leaf) {
      LeafArgs la{};
      la.Pa = last[0];
      la.Pb = last[1];
      la.ha = p->na;
      la.hb = p->nb;
      la.num_parents = last_hi - last_lo;
      la.La = (unsigned char *)p->dev_table + p->side[0].leaf_off;
      la.Lb = (unsigned char *)p->dev_table + p->side[1].leaf_off;
      la.c = p->leaf_c;
      la.r = (int32_t)p->radix[B];
      la.m_first = (int32_t)(c0 % p->radix[B]);
      la.m_last = (int32_t)((c1 - 1) % p->radix[B]) + 1;
      la.ia = ia;
      la.ib = ib;
      la.S = (int64_t)num;
      la.parents_per_group = L.ppg;
      la.num_groups = (int32_t)((la.num_parents + L.ppg - 1) / L.ppg);
      la.partial = (double *)(ws + L.off_partial);
      la.sync = (uint32_t *)(ws + L.off_sync);
      la.err = p->dev_status;
      la.pf = p->leaf_pf;
      la.H = p->leaf_H.empty() ? nullptr : (unsigned char *)p->dev_table + p->leaf_h_off;
      if (p->leaf_pf >= 0) {
        la.Sa = (unsigned char *)p->dev_table + p->side[0].leaf_s_off;
        la.Sb = (unsigned char *)p->dev_table + p->side[1].leaf_s_off;
        la.G = (unsigned char *)p->dev_table + p->leaf_g_off;
      }
      if (L.dots) {
        // dot form: the dots the deepest level wrote, read once (64 bytes per (parent,
        // bitstring)), the 4 x 4 bilinear form (20 complex products) on each
        const DotSort ds = dot_sort_layout(ws + L.off_dsort, (int64_t)num, p->na, p->nb);
        la.Da = ws + L.off_dots[0];
        la.Db = ws + L.off_dots[1];
        la.dida = ds.ida;
        la.dposb = ds.posb;
        const double units = (double)la.num_parents * (double)num;
        LAUNCH(HSF_KERNEL_LEAF, 64.0 * units + 16.0 * la.num_groups * num, 8.0 * 20.0 * units,
               launch_leaf_dots(la, st));
        LAUNCH(HSF_KERNEL_REDUCE, 16.0 * la.num_groups * num + 64.0 * num, 0.0,
               launch_reduce_partials(la.partial, la.num_groups, la.S, outd, comp, st));
        continue;
      }
      const bool streams = leaf_streams(la, p->precision);
      if (streams) {
        la.parents_per_group = (int32_t)la.num_parents;
        la.num_groups = 1;
        if (L.off_sort) {
          // once per run: the bitstrings sorted by their side-a storage index
          int64_t *perm = (int64_t *)(ws + L.off_sort);
          uint64_t *ia_s = (uint64_t *)(perm + num), *ib_s = ia_s + num;
          uint32_t *counts = (uint32_t *)(ws + L.off_sort + align256(num * 24));
          if (!sorted) {
            LAUNCH(HSF_KERNEL_OTHER, 64.0 * num, 0.0,
                   launch_bitstring_sort(ia, ib, (int64_t)num, p->na, counts, ia_s, ib_s, perm, st));
            sorted = true;
          }
          la.ia = ia_s;
          la.ib = ib_s;
          la.perm = perm;
        }
      }
      const double units = (double)la.num_parents * (double)num;
      // algorithmic DRAM bytes: every parent state read once (at most: the gathered
      // chunks, when the bitstrings touch few of them) plus the FP64 partials
      const double gathered = units * 2.0 * (1 << la.c) * csz;
      const double states = (double)la.num_parents * (double)((1ull << la.ha) + (1ull << la.hb)) * csz;
      // FLOP per (bitstring, parent): r digits x (two dots of 2^c terms + the product), or
      // factored: four dots of 2^(c-1) terms per side + the 4 x 4 bilinear form
      // or, streaming with the pair form, the D x D bilinear form
      const double fl = leaf_factored(la, p->precision) ? 8.0 * (4.0 * (1 << la.c) + 20.0)
                        : (streams && la.H) ? 8.0 * ((1 << (2 * la.c)) + (1 << la.c))
                                            : la.r * (8.0 * 2.0 * (1 << la.c) + 8.0);
      LAUNCH(HSF_KERNEL_LEAF, std::min(gathered, states) + 16.0 * la.num_groups * num, units * fl,
             launch_leaf_contract(la, p->precision, st));
      LAUNCH(HSF_KERNEL_REDUCE, 16.0 * la.num_groups * num + 64.0 * num, 0.0,
             launch_reduce_partials(la.partial, la.num_groups, la.S, outd, comp, st));
    } else if (num > 0) {
      const int64_t np = (int64_t)(c1 - c0);
      GatherArgs g{};
      g.A = last[0];
      g.B = last[1];
      g.num_paths = np;
      g.ha = p->na;
      g.hb = p->nb;
      g.ia = ia;
      g.ib = ib;
      g.S = (int64_t)num;
      g.paths_per_group = L.ppg;
      g.num_groups = (int32_t)((np + L.ppg - 1) / L.ppg);
      g.partial = (double *)(ws + L.off_partial);
      LAUNCH(HSF_KERNEL_GATHER, (double)np * g.S * 2.0 * csz + 16.0 * g.num_groups * g.S,
             8.0 * (double)np * g.S, launch_gather_dot(g, p->precision, st));
      LAUNCH(HSF_KERNEL_REDUCE, 16.0 * g.num_groups * g.S + 64.0 * g.S, 0.0,
             launch_reduce_partials(g.partial, g.num_groups, g.S, outd, comp, st));
    } else {
      const int64_t np = (int64_t)(c1 - c0);
      WindowArgs w{};
      w.A = last[0];
      w.B = last[1];
      w.num_paths = np;
      w.ha = p->na;
      w.hb = p->nb;
      w.window = count;
      w.M = M;
      w.N = N;
      w.out = outd;
      w.comp = comp;
      w.row_index = ia;
      w.col_index = ib;
      if (L.tc) {
        PathGemmArgs g{};
        g.A = last[0];
        g.B = last[1];
        g.paths = np;
        g.ha = p->na;
        g.hb = p->nb;
        g.perm_a = perm_of(p->side[0]);
        g.perm_b = perm_of(p->side[1]);
        g.M = M;
        g.N = N;
        g.window = count;
        g.out = outd;
        g.comp = comp;
        g.scratch = ws + L.off_gemm;
        g.mode = p->gemm_mode;
        g.err = p->dev_status;
        const double terms = p->gemm_mode == HSF_GEMM_TF32 ? 1.0 : 3.0;
        const double esz = p->gemm_mode == HSF_GEMM_BF16X3 ? 2.0 : 4.0;
        const double kcols = terms * 2.0 * (double)np;
        // packing: the leaf rows read once, the split operands written once
        LAUNCH(HSF_KERNEL_PACK, (double)np * (w.M + w.N) * csz + (2.0 * w.M + w.N) * kcols * esz, 0.0,
               launch_path_pack(g, st));
        // the GEMM: its operands read once, the FP64 output and compensation updated
        LAUNCH(HSF_KERNEL_WINDOW, (2.0 * w.M + w.N) * kcols * esz + 64.0 * w.M * w.N,
               8.0 * terms * (double)np * w.M * w.N, launch_path_gemm(g, st));
      } else {
        LAUNCH(HSF_KERNEL_WINDOW, (double)np * (w.M + w.N) * csz + 64.0 * w.M * w.N,
               8.0 * (double)np * w.M * w.N, launch_window(w, p->precision, st));
      }
    }
  }
  LAUNCH(HSF_KERNEL_OTHER, 48.0 * count, 0.0, launch_finalize(outd, comp, (int64_t)(2 * count), p->dev_status + kStatusNumeric, st));
  return HSF_OK;
}

}  // extern "C"
