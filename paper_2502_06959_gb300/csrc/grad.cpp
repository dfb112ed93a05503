// Adjoint gradients (hsf_grad): dL/dtheta_j for a real loss of the amplitudes at the
// requested bitstrings, given the upstream gradient g_s = dL/dRe amp_s + i dL/dIm amp_s.
//
//   * rotations inside one half (Sec. II-B: every path simulates both halves): the
//     path tree is simulated forward, the leaf cotangents are formed from the other
//     half's leaf states, and the tree is walked back level by level (adjoint.cu):
//     unitary ops are undone on the recomputed states, cotangents are pulled back
//     through G^T, and at every level the children's cotangents reach their parent
//     through the transposed Schmidt factors.  Only levels 0..k0 are kept for every
//     node; the deeper levels are recomputed per chunk (the subtree of one level-k0
//     node) and walked back before the next chunk, with k0 the smallest level whose
//     layout fits the caller's workspace, so memory follows the workspace, not the tree;
//   * rotations inside a jointly cut block: the amplitude is linear in the block
//     matrix A (Sec. IV-A, eq. equ-schmidt-decompostion-res), so d amp / d theta_j is the
//     HSF sum with A replaced by dA/dtheta_j (product rule over the block's gates tied
//     to theta_j).  That matrix is Schmidt-decomposed like any block (the SVD exists
//     for every matrix, Sec. III-B) and run through the ordinary forward path.  A
//     cascade block's derivative keeps its closed-form terms (Sec. IV-D): the hub
//     projectors stay, only the other side's factors are differentiated.
#include <algorithm>
#include <cstring>
#include <memory>
#include <vector>

#include "plan.h"

using namespace hsf;

namespace {

#define CUDA_TRY(expr)                                                                   \
  do {                                                                                   \
    cudaError_t e_ = (expr);                                                             \
    if (e_ != cudaSuccess)                                                               \
      return set_error(HSF_ECUDA, "%s failed: %s", #expr, cudaGetErrorString(e_));       \
  } while (0)

size_t a256(size_t x) { return (x + 255) / 256 * 256; }

// Gradient workspace: levels 0..k0 of the path tree are held for every node (the "upper"
// tree); each level-k0 node's subtree (levels k0+1..B, a chunk of below[k0] paths) is
// recomputed forward, contracted with the leaf cotangents and walked back on its own, so
// only one chunk's deeper levels are held at a time.  k0 = 0 holds the whole tree once.
struct GradLayout {
  int k0 = 0;
  std::vector<size_t> psi[2], mu[2];   // per level
  size_t off_index = 0, off_grad = 0, off_amp = 0, off_run = 0, total = 0;
};

// nodes of level k held in the workspace for chunk root level k0
uint64_t held_nodes(const hsf_plan &p, int k0, int k) {
  return k <= k0 ? p.num_paths / p.below[k] : p.below[k0] / p.below[k];
}

GradLayout grad_layout(const hsf_plan &p, size_t num, int k0) {
  GradLayout L;
  L.k0 = k0;
  const size_t csz = p.precision == HSF_PREC_C64 ? 8 : 16;
  const int B = (int)p.blocks.size();
  size_t off = 0;
  for (int s = 0; s < 2; ++s) {
    L.psi[s].resize(B + 1);
    L.mu[s].resize(B + 1);
    const size_t sb = ((size_t)1 << p.gside[s].h) * csz;
    for (int k = 0; k <= B; ++k) {
      const size_t nodes = (size_t)held_nodes(p, k0, k);
      L.psi[s][k] = off;
      off += a256(nodes * sb);
      L.mu[s][k] = off;
      off += a256(nodes * sb);
    }
  }
  L.off_index = off;
  off += a256(num * 16);
  L.off_grad = off;
  off += a256((size_t)std::max(1, p.num_params) * 8);
  L.off_amp = off;
  off += a256(num * 16);
  L.off_run = off;
  L.total = off;
  return L;
}

hsf_status ensure_grad(hsf_plan &p) {
  if (p.grad_ready) return HSF_OK;
  for (size_t b = 0; b < p.blocks.size(); ++b)
    if (!p.blocks[b].fops[0].empty() || !p.blocks[b].fops[1].empty())
      return set_error(HSF_ENOTSUP, "gradients of block %zu (more than 3 qubits on a side) are not supported", b);
  hsf_status st = build_programs(p, true);
  if (st != HSF_OK) return st;
  st = upload_programs(p, true);
  if (st != HSF_OK) return st;
  // Schmidt factors of every level (both sides) for the cotangent pullback
  const int B = (int)p.blocks.size();
  std::vector<unsigned char> host;
  for (int s = 0; s < 2; ++s) {
    p.factor_off[s].assign(B + 1, 0);
    for (int k = 1; k <= B; ++k) {
      const OpH &f = p.gside[s].levels[k].ops[0];
      while (host.size() % 256) host.push_back(0);
      p.factor_off[s][k] = host.size();
      for (const cd &z : f.m) {
        if (p.precision == HSF_PREC_C64) {
          float2 c = make_float2((float)z.real(), (float)z.imag());
          host.insert(host.end(), (unsigned char *)&c, (unsigned char *)&c + sizeof c);
        } else {
          double2 c = make_double2(z.real(), z.imag());
          host.insert(host.end(), (unsigned char *)&c, (unsigned char *)&c + sizeof c);
        }
      }
    }
  }
  if (host.empty()) host.resize(256);
  p.dev_factors = table_alloc(host.size());
  if (!p.dev_factors) return set_error(HSF_ENOMEM, "gradient factor tables of %zu bytes", host.size());
  CUDA_TRY(cudaMemcpyAsync(p.dev_factors, host.data(), host.size(), cudaMemcpyHostToDevice, plan_stream()));
  CUDA_TRY(cudaStreamSynchronize(plan_stream()));
  // derivative blocks: one SVD job per (block, angle) pair
  std::vector<SvdJob> jobs;
  std::vector<std::pair<int, int>> keys;
  for (int b = 0; b < B; ++b) {
    std::vector<int> params;
    for (int gi : p.blocks[b].gates)
      if (p.gates[gi].param_id >= 0 && !p.gates[gi].dm.empty() &&
          std::find(params.begin(), params.end(), p.gates[gi].param_id) == params.end())
        params.push_back(p.gates[gi].param_id);
    for (int j : params) {
      SvdJob job;
      job.block = b;
      for (int gi : p.blocks[b].gates) {
        if (p.gates[gi].param_id != j || p.gates[gi].dm.empty()) continue;
        std::vector<int> term = p.blocks[b].gates;
        for (auto &x : term)
          if (x == gi) x = -1 - gi;
        job.terms.push_back(term);
      }
      jobs.push_back(job);
      keys.push_back({b, j});
    }
  }
  // blocks with closed-form terms get their derivative's terms in closed form too (the
  // derivative of a gate that is diagonal on the hub is diagonal on it): no SVD
  std::vector<BlockH> res(jobs.size());
  std::vector<SvdJob> svd_jobs;
  std::vector<size_t> svd_of;
  for (size_t i = 0; i < jobs.size(); ++i) {
    if (p.blocks[jobs[i].block].closed >= 0 && closed_form_job(p, jobs[i], false, res[i])) continue;
    svd_jobs.push_back(jobs[i]);
    svd_of.push_back(i);
  }
  std::vector<BlockH> sres;
  st = run_svd_jobs(p, svd_jobs, sres);
  if (st != HSF_OK) return st;
  for (size_t j = 0; j < svd_jobs.size(); ++j) res[svd_of[j]] = sres[j];
  for (size_t i = 0; i < jobs.size(); ++i) {
    if (res[i].rank <= 0) continue;                 // the derivative vanishes
    std::unique_ptr<hsf_plan> d(new hsf_plan());
    d->n = p.n;
    d->cut = p.cut;
    d->na = p.na;
    d->nb = p.nb;
    d->precision = p.precision;
    d->gemm_mode = HSF_GEMM_FP32;
    d->flags = p.flags;
    d->tile_max = p.tile_max;
    d->rank_tol = p.rank_tol;
    d->max_paths = 1ull << 62;
    d->gates = p.gates;
    d->blocks = p.blocks;
    d->blocks[keys[i].first] = res[i];
    st = finish_plan(*d);
    if (st != HSF_OK) return st;
    p.dplans.push_back({keys[i].first, keys[i].second, d.release()});
  }
  p.grad_ready = true;
  return HSF_OK;
}

// The layout for a workspace budget (0: the whole tree at once) and the bytes it needs,
// including the forward-run workspace of the derivative plans of cut-block angles.
hsf_status grad_plan_layout(hsf_plan &p, size_t num, size_t budget, GradLayout *out, size_t *bytes) {
  hsf_status st = ensure_grad(p);
  if (st != HSF_OK) return st;
  const int B = (int)p.blocks.size();
  const int kmax = std::max(0, B - 1);
  for (int k0 = 0; k0 <= kmax; ++k0) {
    GradLayout L = grad_layout(p, num, k0);
    if (budget && L.total > budget) continue;
    size_t run = 0;
    bool fits = true;
    for (auto &d : p.dplans) {
      size_t b = 0;
      st = hsf_workspace_size(d.plan, num, 0, budget ? budget - L.total : 0, &b);
      if (st == HSF_ENOMEM) { fits = false; break; }
      if (st != HSF_OK) return st;
      run = std::max(run, b);
    }
    if (!fits || (budget && L.total + run > budget)) continue;
    *out = L;
    *bytes = L.total + run;
    return HSF_OK;
  }
  return set_error(HSF_ENOMEM, "no gradient layout fits a %zu-byte workspace", budget);
}

}  // namespace

extern "C" {

hsf_status hsf_grad_workspace_size(hsf_plan *p, size_t num, size_t budget, size_t *bytes) {
  if (!p || !bytes) return set_error(HSF_EINVAL, "NULL argument");
  if (num == 0) return set_error(HSF_EINVAL, "gradients need at least one bitstring");
  GradLayout L;
  return grad_plan_layout(*p, num, budget, &L, bytes);
}

hsf_status hsf_grad(hsf_plan *p, const uint64_t *bits, size_t num, const void *gout, double *grad,
                    int32_t num_params, void *workspace, size_t ws_bytes, void *stream) {
  if (!p || !bits || !gout || !grad || !workspace) return set_error(HSF_EINVAL, "NULL argument");
  if (num == 0) return set_error(HSF_EINVAL, "gradients need at least one bitstring");
  if ((uintptr_t)workspace % 256) return set_error(HSF_EINVAL, "workspace must be 256-byte aligned");
  if (num_params < p->num_params)
    return set_error(HSF_EINVAL, "num_params %d < %d angles used by the circuit", num_params, p->num_params);
  size_t need = 0;
  GradLayout L;
  hsf_status st = grad_plan_layout(*p, num, ws_bytes, &L, &need);
  if (st != HSF_OK) return st;
  if (ws_bytes < need) return set_error(HSF_ENOMEM, "gradient workspace needs %zu bytes, got %zu", need, ws_bytes);
  cudaStream_t stm = (cudaStream_t)stream;
  unsigned char *ws = (unsigned char *)workspace;
  const int B = (int)p->blocks.size();
  const int k0 = L.k0;
  const size_t csz = p->precision == HSF_PREC_C64 ? 8 : 16;
  double *gacc = (double *)(ws + L.off_grad);
  CUDA_TRY(launch_zero_bytes(gacc, a256((size_t)std::max(1, p->num_params) * 8), stm));
  // storage indices of the bitstrings under the gradient programs' storage order
  uint64_t *ia = (uint64_t *)(ws + L.off_index), *ib = ia + num;
  {
    IndexArgs ix{};
    ix.bits = bits;
    ix.S = (int64_t)num;
    ix.nb = p->nb;
    ix.ha = p->na;
    ix.hb = p->nb;
    for (int q = 0; q < p->na; ++q) ix.store_a[q] = p->gside[0].store[q];
    for (int q = 0; q < p->nb; ++q) ix.store_b[q] = p->gside[1].store[q];
    ix.ia = ia;
    ix.ib = ib;
    CUDA_TRY(launch_index_prep(ix, stm));
  }
  // forward sweep of level k of side s over `nodes` nodes starting at level-global node_lo,
  // from the parent buffer par whose first node is level-global parent_lo
  auto forward = [&](int s, int k, void *dst, const void *par, int64_t node_lo, int64_t parent_lo,
                     int64_t nodes) -> hsf_status {
    const SideH &sd = p->gside[s];
    const LevelH &lv = sd.levels[k];
    for (size_t pi = 0; pi < lv.passes.size(); ++pi) {
      const PassH &ps = lv.passes[pi];
      SweepArgs a{};
      a.ops = (const DevOp *)((unsigned char *)p->dev_gtable + ps.ops_off);
      a.num_ops = ps.num_ops;
      a.h = sd.h;
      a.mats = (unsigned char *)p->dev_gtable + ps.mats_off;
      a.read_parent = (pi == 0 && k > 0) ? 1 : 0;
      a.init_zero = (pi == 0 && k == 0) ? 1 : 0;
      a.src = a.read_parent ? par : dst;
      a.dst = dst;
      a.active_mask = ps.active;
      a.t = ps.t;
      a.radix = (int32_t)p->radix[k];
      a.node_lo = node_lo;
      a.parent_lo = parent_lo;
      a.num_nodes = nodes;
      a.tiles_per_node = 1 << (sd.h - ps.t);
      a.groups = ps.groups.empty() ? nullptr : (const DevGroup *)((unsigned char *)p->dev_gtable + ps.groups_off);
      a.num_groups = (int32_t)ps.groups.size();
      a.rbits = p->rbits;
      const size_t blk = ps.table_end - ps.ops_off;
      if (!ps.groups.empty() && blk <= (size_t)kMaxStageBytes) {
        a.stage_src = (unsigned char *)p->dev_gtable + ps.ops_off;
        a.stage_bytes = (int32_t)((blk + 15) / 16 * 16);
        a.stage_mats_off = (int32_t)(ps.mats_off - ps.ops_off);
        a.stage_groups_off = (int32_t)(ps.groups_off - ps.ops_off);
      }
      CUDA_TRY(launch_sweep(a, p->precision, stm));
      g_launches++;
    }
    return HSF_OK;
  };
  // reverse sweep of level k (rotation gradients, uncomputing the unitary ops in place)
  auto backward = [&](int s, int k, void *psi, void *mu, int64_t nodes) -> hsf_status {
    const SideH &sd = p->gside[s];
    const LevelH &lv = sd.levels[k];
    for (int pi = (int)lv.passes.size() - 1; pi >= 0; --pi) {
      const PassH &ps = lv.passes[pi];
      AdjointArgs a{};
      a.ops = (const DevOp *)((unsigned char *)p->dev_gtable + ps.ops_off);
      a.num_ops = ps.num_ops;
      a.first_op = (pi == 0 && k > 0) ? 1 : 0;
      a.mats = (unsigned char *)p->dev_gtable + ps.mats_off;
      a.psi = psi;
      a.mu = mu;
      a.h = sd.h;
      a.t = ps.t;
      a.active_mask = ps.active;
      a.num_nodes = nodes;
      a.tiles_per_node = 1 << (sd.h - ps.t);
      a.grad = gacc;
      CUDA_TRY(launch_adjoint(a, p->precision, stm));
      g_launches++;
    }
    return HSF_OK;
  };
  // children (level k, first level-global child_lo) to parents (level k-1)
  auto pullback = [&](int s, int k, const void *mu_child, void *mu_parent, int64_t parent_lo, int64_t parents,
                      int64_t child_lo, int64_t children) -> hsf_status {
    const SideH &sd = p->gside[s];
    const OpH &f = sd.levels[k].ops[0];
    PullbackArgs pb{};
    pb.mu_child = mu_child;
    pb.mu_parent = mu_parent;
    pb.factor = (unsigned char *)p->dev_factors + p->factor_off[s][k];
    pb.h = sd.h;
    pb.nf = f.nq;
    for (int x = 0; x < f.nq; ++x) pb.fq[x] = f.q[x];
    pb.radix = (int32_t)p->radix[k];
    pb.parent_lo = parent_lo;
    pb.child_lo = child_lo;
    pb.num_parents = parents;
    pb.num_children = children;
    CUDA_TRY(launch_factor_pullback(pb, p->precision, stm));
    g_launches++;
    return HSF_OK;
  };
#define GTRY(x)                              \
  do {                                       \
    hsf_status s_ = (x);                     \
    if (s_ != HSF_OK) return s_;             \
  } while (0)
  // upper tree, every node: levels 0..k0 (all of it when there is no block)
  const int top = B == 0 ? 0 : k0;
  for (int s = 0; s < 2; ++s)
    for (int k = 0; k <= top; ++k)
      GTRY(forward(s, k, ws + L.psi[s][k], k > 0 ? ws + L.psi[s][k - 1] : nullptr, 0, 0,
                   (int64_t)held_nodes(*p, k0, k)));
  auto leaf_cot = [&](const void *pa, const void *pb_, void *ma, void *mb, int64_t paths) -> hsf_status {
    for (int s = 0; s < 2; ++s)
      CUDA_TRY(launch_zero_bytes(s == 0 ? ma : mb, (size_t)paths * ((size_t)1 << p->gside[s].h) * csz, stm));
    LeafCotArgs lc{};
    lc.psi_a = pa;
    lc.psi_b = pb_;
    lc.mu_a = ma;
    lc.mu_b = mb;
    lc.ha = p->na;
    lc.hb = p->nb;
    lc.paths = paths;
    lc.ia = ia;
    lc.ib = ib;
    lc.gout = (const double *)gout;
    lc.S = (int64_t)num;
    CUDA_TRY(launch_leaf_cot(lc, p->precision, stm));
    g_launches++;
    return HSF_OK;
  };
  if (B == 0) {
    GTRY(leaf_cot(ws + L.psi[0][0], ws + L.psi[1][0], ws + L.mu[0][0], ws + L.mu[1][0], 1));
  } else {
    // chunks: the subtree of every level-k0 node, levels k0+1..B recomputed from it
    const int64_t chunks = (int64_t)held_nodes(*p, k0, k0);
    const size_t sbytes[2] = {((size_t)1 << p->gside[0].h) * csz, ((size_t)1 << p->gside[1].h) * csz};
    for (int64_t c = 0; c < chunks; ++c) {
      for (int s = 0; s < 2; ++s)
        for (int k = k0 + 1; k <= B; ++k) {
          const int64_t nk = (int64_t)held_nodes(*p, k0, k);
          const bool from_upper = k == k0 + 1;
          const int64_t plo = from_upper ? 0 : c * (int64_t)held_nodes(*p, k0, k - 1);
          GTRY(forward(s, k, ws + L.psi[s][k], ws + L.psi[s][k - 1], c * nk, plo, nk));
        }
      GTRY(leaf_cot(ws + L.psi[0][B], ws + L.psi[1][B], ws + L.mu[0][B], ws + L.mu[1][B],
                    (int64_t)held_nodes(*p, k0, B)));
      for (int k = B; k > k0; --k)
        for (int s = 0; s < 2; ++s) {
          const int64_t nk = (int64_t)held_nodes(*p, k0, k);
          GTRY(backward(s, k, ws + L.psi[s][k], ws + L.mu[s][k], nk));
          if (k - 1 > k0) {
            const int64_t np = (int64_t)held_nodes(*p, k0, k - 1);
            GTRY(pullback(s, k, ws + L.mu[s][k], ws + L.mu[s][k - 1], c * np, np, c * nk, nk));
          } else {
            // into the chunk root's cotangent, held with the upper tree
            GTRY(pullback(s, k, ws + L.mu[s][k], ws + L.mu[s][k0] + (size_t)c * sbytes[s], c, 1, c * nk, nk));
          }
        }
    }
  }
  // upper tree, backwards
  for (int k = top; k >= 0; --k)
    for (int s = 0; s < 2; ++s) {
      const int64_t nk = (int64_t)held_nodes(*p, k0, k);
      GTRY(backward(s, k, ws + L.psi[s][k], ws + L.mu[s][k], nk));
      if (k > 0) {
        const int64_t np = (int64_t)held_nodes(*p, k0, k - 1);
        GTRY(pullback(s, k, ws + L.mu[s][k], ws + L.mu[s][k - 1], 0, np, 0, nk));
      }
    }
#undef GTRY
  // angles inside cut blocks: HSF sums with the block replaced by its derivative
  for (auto &d : p->dplans) {
    double *ampd = (double *)(ws + L.off_amp);
    st = hsf_run(d.plan, bits, num, 0, 0, 0, ampd, ws + L.off_run, ws_bytes - L.off_run, stream);
    if (st != HSF_OK) return st;
    CUDA_TRY(launch_grad_dot((const double *)gout, ampd, (int64_t)num, gacc + d.param, stm));
    g_launches++;
  }
  CUDA_TRY(cudaMemsetAsync(grad, 0, (size_t)num_params * 8, stm));
  if (p->num_params > 0)
    CUDA_TRY(cudaMemcpyAsync(grad, gacc, (size_t)p->num_params * 8, cudaMemcpyDeviceToDevice, stm));
  return HSF_OK;
}

}  // extern "C"
