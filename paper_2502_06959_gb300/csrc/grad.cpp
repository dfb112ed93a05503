// Adjoint gradients (hsf_grad): dL/dtheta_j for a real loss of the amplitudes at the
// requested bitstrings, given the upstream gradient g_s = dL/dRe amp_s + i dL/dIm amp_s.
//
//   * rotations inside one half (Sec. II-B: every path simulates both halves): the
//     whole path tree is simulated forward with every node state kept, the leaf
//     cotangents are formed from the other half's leaf states, and the tree is walked
//     back level by level (adjoint.cu): unitary ops are undone on the stored states,
//     cotangents are pulled back through G^T, and at every level the children's
//     cotangents reach their parent through the transposed Schmidt factors;
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

struct GradLayout {
  std::vector<size_t> psi[2], mu[2];   // per level
  size_t off_index = 0, off_grad = 0, off_amp = 0, off_run = 0, total = 0;
};

GradLayout grad_layout(const hsf_plan &p, size_t num) {
  GradLayout L;
  const size_t csz = p.precision == HSF_PREC_C64 ? 8 : 16;
  const int B = (int)p.blocks.size();
  size_t off = 0;
  for (int s = 0; s < 2; ++s) {
    L.psi[s].resize(B + 1);
    L.mu[s].resize(B + 1);
    const size_t sb = ((size_t)1 << p.gside[s].h) * csz;
    for (int k = 0; k <= B; ++k) {
      const size_t nodes = (size_t)(p.num_paths / p.below[k]);
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
  CUDA_TRY(cudaMalloc(&p.dev_factors, host.size()));
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

hsf_status grad_need(hsf_plan &p, size_t num, size_t *bytes) {
  hsf_status st = ensure_grad(p);
  if (st != HSF_OK) return st;
  GradLayout L = grad_layout(p, num);
  size_t run = 0;
  for (auto &d : p.dplans) {
    size_t b = 0;
    st = hsf_workspace_size(d.plan, num, 0, 0, &b);
    if (st != HSF_OK) return st;
    run = std::max(run, b);
  }
  *bytes = L.total + run;
  return HSF_OK;
}

}  // namespace

extern "C" {

hsf_status hsf_grad_workspace_size(hsf_plan *p, size_t num, size_t *bytes) {
  if (!p || !bytes) return set_error(HSF_EINVAL, "NULL argument");
  if (num == 0) return set_error(HSF_EINVAL, "gradients need at least one bitstring");
  return grad_need(*p, num, bytes);
}

hsf_status hsf_grad(hsf_plan *p, const uint64_t *bits, size_t num, const void *gout, double *grad,
                    int32_t num_params, void *workspace, size_t ws_bytes, void *stream) {
  if (!p || !bits || !gout || !grad || !workspace) return set_error(HSF_EINVAL, "NULL argument");
  if (num == 0) return set_error(HSF_EINVAL, "gradients need at least one bitstring");
  if ((uintptr_t)workspace % 256) return set_error(HSF_EINVAL, "workspace must be 256-byte aligned");
  if (num_params < p->num_params)
    return set_error(HSF_EINVAL, "num_params %d < %d angles used by the circuit", num_params, p->num_params);
  size_t need = 0;
  hsf_status st = grad_need(*p, num, &need);
  if (st != HSF_OK) return st;
  if (ws_bytes < need) return set_error(HSF_ENOMEM, "gradient workspace needs %zu bytes, got %zu", need, ws_bytes);
  const GradLayout L = grad_layout(*p, num);
  cudaStream_t stm = (cudaStream_t)stream;
  unsigned char *ws = (unsigned char *)workspace;
  const int B = (int)p->blocks.size();
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
  // forward over the whole tree, every level kept
  for (int s = 0; s < 2; ++s) {
    const SideH &sd = p->gside[s];
    for (int k = 0; k <= B; ++k) {
      const int64_t nodes = (int64_t)(p->num_paths / p->below[k]);
      void *dst = ws + L.psi[s][k];
      const void *par = k > 0 ? (const void *)(ws + L.psi[s][k - 1]) : nullptr;
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
        a.node_lo = 0;
        a.parent_lo = 0;
        a.num_nodes = nodes;
        a.tiles_per_node = 1 << (sd.h - ps.t);
        CUDA_TRY(launch_sweep(a, p->precision, stm));
        g_launches++;
      }
    }
  }
  // leaf cotangents
  const size_t csz = p->precision == HSF_PREC_C64 ? 8 : 16;
  for (int s = 0; s < 2; ++s) {
    const size_t bytes = (size_t)p->num_paths * ((size_t)1 << p->gside[s].h) * csz;
    CUDA_TRY(launch_zero_bytes(ws + L.mu[s][B], bytes, stm));
  }
  {
    LeafCotArgs lc{};
    lc.psi_a = ws + L.psi[0][B];
    lc.psi_b = ws + L.psi[1][B];
    lc.mu_a = ws + L.mu[0][B];
    lc.mu_b = ws + L.mu[1][B];
    lc.ha = p->na;
    lc.hb = p->nb;
    lc.paths = (int64_t)p->num_paths;
    lc.ia = ia;
    lc.ib = ib;
    lc.gout = (const double *)gout;
    lc.S = (int64_t)num;
    CUDA_TRY(launch_leaf_cot(lc, p->precision, stm));
    g_launches++;
  }
  // backward over the tree
  for (int k = B; k >= 0; --k) {
    for (int s = 0; s < 2; ++s) {
      const SideH &sd = p->gside[s];
      const int64_t nodes = (int64_t)(p->num_paths / p->below[k]);
      const LevelH &lv = sd.levels[k];
      for (int pi = (int)lv.passes.size() - 1; pi >= 0; --pi) {
        const PassH &ps = lv.passes[pi];
        AdjointArgs a{};
        a.ops = (const DevOp *)((unsigned char *)p->dev_gtable + ps.ops_off);
        a.num_ops = ps.num_ops;
        a.first_op = (pi == 0 && k > 0) ? 1 : 0;
        a.mats = (unsigned char *)p->dev_gtable + ps.mats_off;
        a.psi = ws + L.psi[s][k];
        a.mu = ws + L.mu[s][k];
        a.h = sd.h;
        a.t = ps.t;
        a.active_mask = ps.active;
        a.num_nodes = nodes;
        a.tiles_per_node = 1 << (sd.h - ps.t);
        a.grad = gacc;
        CUDA_TRY(launch_adjoint(a, p->precision, stm));
        g_launches++;
      }
      if (k > 0) {
        const OpH &f = lv.ops[0];
        PullbackArgs pb{};
        pb.mu_child = ws + L.mu[s][k];
        pb.mu_parent = ws + L.mu[s][k - 1];
        pb.factor = (unsigned char *)p->dev_factors + p->factor_off[s][k];
        pb.h = sd.h;
        pb.nf = f.nq;
        for (int x = 0; x < f.nq; ++x) pb.fq[x] = f.q[x];
        pb.radix = (int32_t)p->radix[k];
        pb.parent_lo = 0;
        pb.child_lo = 0;
        pb.num_parents = (int64_t)(p->num_paths / p->below[k - 1]);
        pb.num_children = nodes;
        CUDA_TRY(launch_factor_pullback(pb, p->precision, stm));
        g_launches++;
      }
    }
  }
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
