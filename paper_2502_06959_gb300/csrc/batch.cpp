// Batches of circuits in one CUDA graph, and the launch-parameter autotuner.
//
// hsf_batch_create records hsf_run for every item (uneven n, path counts and outputs)
// on a capturing stream, instantiates the graph once, and hsf_batch_launch replays it:
// the many small launches of a batch of modest circuits become one graph launch.  The
// items run one after another inside the graph and share one workspace, sized for the
// largest item.
//
// hsf_tune picks, for one circuit shape, the shared-memory tile width of the half-state
// sweeps and whether ops are fused into register groups, by planning and timing every
// candidate on the current device; results are kept in a small text cache keyed by the
// circuit shape and request, so repeated shapes cost nothing.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "plan.h"

using namespace hsf;

struct hsf_batch {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  size_t nodes = 0;
  ~hsf_batch() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
  }
};

namespace {

#define CUDA_TRY(expr)                                                                   \
  do {                                                                                   \
    cudaError_t e_ = (expr);                                                             \
    if (e_ != cudaSuccess)                                                               \
      return set_error(HSF_ECUDA, "%s failed: %s", #expr, cudaGetErrorString(e_));       \
  } while (0)

std::mutex g_tune_mu;

uint64_t shape_key(const hsf_circuit *c, int cut, const hsf_blocks *b, const hsf_plan_opts *o, size_t num,
                   uint64_t window) {
  // FNV-1a over the circuit's structure (kinds, qubits, block membership) and request
  uint64_t h = 1469598103934665603ull;
  auto mix = [&](uint64_t v) {
    for (int i = 0; i < 8; ++i) {
      h ^= (v >> (8 * i)) & 0xff;
      h *= 1099511628211ull;
    }
  };
  mix((uint64_t)c->n);
  mix((uint64_t)cut);
  mix((uint64_t)c->num_gates);
  for (int i = 0; i < c->num_gates; ++i) {
    mix((uint64_t)c->gates[i].kind);
    for (int j = 0; j < c->gates[i].nq && j < 4; ++j) mix((uint64_t)c->gates[i].q[j]);
  }
  mix((uint64_t)b->num_blocks);
  for (int k = 0; k < b->num_blocks; ++k) mix((uint64_t)(b->offsets[k + 1] - b->offsets[k]));
  mix((uint64_t)(o ? o->precision : 0));
  mix((uint64_t)(o ? o->gemm_mode : 0));
  mix((uint64_t)num);
  mix(window);
  return h;
}

// One tuned configuration: plan options and the workspace budget (path batch).
struct TuneCfg {
  int tile = 0, flags = 0, gemm = 0;
  size_t budget = 0;
};

bool cache_lookup(const char *path, uint64_t key, TuneCfg *c) {
  if (!path || !*path) return false;
  FILE *f = std::fopen(path, "r");
  if (!f) return false;
  char line[256];
  bool found = false;
  while (std::fgets(line, sizeof line, f)) {
    unsigned long long k, b = 0;
    int t, fl, g = 0;
    if (std::sscanf(line, "%llx %d %d %d %llu", &k, &t, &fl, &g, &b) != 5) continue;
    if (k == key) {
      *c = TuneCfg{t, fl, g, (size_t)b};
      found = true;
    }
  }
  std::fclose(f);
  return found;
}

void cache_store(const char *path, uint64_t key, const TuneCfg &c) {
  if (!path || !*path) return;
  FILE *f = std::fopen(path, "a");
  if (!f) return;
  std::fprintf(f, "%016llx %d %d %d %llu\n", (unsigned long long)key, c.tile, c.flags, c.gemm,
               (unsigned long long)c.budget);
  std::fclose(f);
}

constexpr int kTunedFlags = HSF_FLAG_NO_REGISTER_SWEEP | HSF_FLAG_REG3 | HSF_FLAG_REG5 | HSF_FLAG_NO_TC_LEVEL;

}  // namespace

extern "C" {

hsf_status hsf_tune(const hsf_circuit *circuit, int32_t cut_l, const hsf_blocks *blocks, hsf_plan_opts *opts,
                    size_t num_bitstrings, const uint64_t *bitstrings, uint64_t window, const char *cache_path,
                    void *workspace, size_t workspace_bytes, size_t *best_budget) {
  if (!circuit || !blocks || !opts || !workspace) return set_error(HSF_EINVAL, "NULL argument");
  std::lock_guard<std::mutex> lock(g_tune_mu);
  const uint64_t key = shape_key(circuit, cut_l, blocks, opts, num_bitstrings, window);
  TuneCfg best_cfg;
  auto apply = [&](const TuneCfg &c) {
    opts->tile_bits = c.tile;
    opts->flags = (opts->flags & ~kTunedFlags) | c.flags;
    opts->gemm_mode = c.gemm;
    if (best_budget) *best_budget = c.budget;
  };
  if (cache_lookup(cache_path, key, &best_cfg)) {
    apply(best_cfg);
    return HSF_OK;
  }
  const int tmax = opts->precision == HSF_PREC_C64 ? kRegTileC64 : kRegTileC128;
  const int half = std::max(circuit->n - cut_l - 1, cut_l + 1);
  cudaStream_t st = nullptr;
  CUDA_TRY(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
  std::unique_ptr<CUstream_st, void (*)(cudaStream_t)> sguard(st, [](cudaStream_t s) { cudaStreamDestroy(s); });
  cudaEvent_t e0, e1;
  CUDA_TRY(cudaEventCreate(&e0));
  CUDA_TRY(cudaEventCreate(&e1));
  const uint64_t count = num_bitstrings ? num_bitstrings : (window ? window : (1ull << circuit->n));
  void *out = nullptr;
  if (cudaMalloc(&out, count * 16) != cudaSuccess) {
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return set_error(HSF_ENOMEM, "hsf_tune: output buffer");
  }
  // time one configuration: plan, one warm run, best of two timed runs (ms; 1e30 if it
  // does not run)
  auto time_cfg = [&](const TuneCfg &c) -> float {
    hsf_plan_opts o = *opts;
    o.tile_bits = c.tile;
    o.flags = (opts->flags & ~kTunedFlags) | c.flags;
    o.gemm_mode = c.gemm;
    hsf_plan *p = nullptr;
    if (hsf_plan_create(circuit, cut_l, blocks, &o, &p) != HSF_OK) return 1e30f;
    size_t need = 0;
    const size_t budget = c.budget ? std::min(c.budget, workspace_bytes) : workspace_bytes;
    if (hsf_workspace_size(p, num_bitstrings, window, budget, &need) != HSF_OK) {
      hsf_plan_destroy(p);
      return 1e30f;
    }
    float ms = 1e30f;
    bool ok = hsf_run(p, bitstrings, num_bitstrings, window, 0, 0, out, workspace, need, st) == HSF_OK;
    for (int rep = 0; rep < 2 && ok; ++rep) {
      cudaEventRecord(e0, st);
      ok = hsf_run(p, bitstrings, num_bitstrings, window, 0, 0, out, workspace, need, st) == HSF_OK;
      cudaEventRecord(e1, st);
      if (cudaEventSynchronize(e1) != cudaSuccess) ok = false;
      float m = 0.f;
      cudaEventElapsedTime(&m, e0, e1);
      ms = std::min(ms, m);
    }
    if (hsf_sync(p, st) != HSF_OK) ok = false;
    hsf_plan_destroy(p);
    return ok ? ms : 1e30f;
  };
  // coordinate search: each dimension in turn, the others held at the best so far
  best_cfg = TuneCfg{std::min(tmax, half), opts->flags & kTunedFlags, opts->gemm_mode, 0};
  float best = time_cfg(best_cfg);
  auto try_cfg = [&](TuneCfg c) {
    const float ms = time_cfg(c);
    if (ms < best) {
      best = ms;
      best_cfg = c;
    }
  };
  {  // shared-memory tile width
    const TuneCfg base = best_cfg;
    for (int t = std::min(tmax, half) - 1; t >= std::max(3, std::min(tmax, half) - 3); --t) try_cfg({t, base.flags, base.gemm, base.budget});
  }
  {  // register-group fusion off, and the register block width (8 / 16 / 32 amplitudes)
    const TuneCfg base = best_cfg;
    const int keep = base.flags & ~(HSF_FLAG_NO_REGISTER_SWEEP | HSF_FLAG_REG3 | HSF_FLAG_REG5);
    try_cfg({base.tile, keep | HSF_FLAG_NO_REGISTER_SWEEP, base.gemm, base.budget});
    if (opts->precision == HSF_PREC_C64) {
      try_cfg({base.tile, keep | HSF_FLAG_REG3, base.gemm, base.budget});
      try_cfg({base.tile, keep | HSF_FLAG_REG5, base.gemm, base.budget});
    }
  }
  if (opts->precision == HSF_PREC_C64) {  // tensor-core tree levels off
    const TuneCfg base = best_cfg;
    try_cfg({base.tile, base.flags ^ HSF_FLAG_NO_TC_LEVEL, base.gemm, base.budget});
  }
  if (num_bitstrings == 0 && opts->precision == HSF_PREC_C64) {  // path-GEMM form (the accurate ones)
    const TuneCfg base = best_cfg;
    for (int g : {HSF_GEMM_BF16X3, HSF_GEMM_TF32X3, HSF_GEMM_FP32})
      if (g != base.gemm) try_cfg({base.tile, base.flags, g, base.budget});
  }
  {  // path batch: the workspace budget (smaller budgets = smaller path chunks)
    const TuneCfg base = best_cfg;
    for (size_t div : {4, 16}) try_cfg({base.tile, base.flags, base.gemm, workspace_bytes / div});
  }
  cudaFree(out);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (best >= 1e29f) return set_error(HSF_ENOTSUP, "hsf_tune: no candidate configuration ran");
  apply(best_cfg);
  cache_store(cache_path, key, best_cfg);
  return HSF_OK;
}

hsf_status hsf_batch_workspace_size(const hsf_batch_item *items, int32_t count, size_t *bytes) {
  if (!items || count <= 0 || !bytes) return set_error(HSF_EINVAL, "bad batch");
  size_t need = 256;
  for (int i = 0; i < count; ++i) {
    size_t b = 0;
    hsf_status st = hsf_workspace_size(items[i].plan, items[i].num, items[i].window, 0, &b);
    if (st != HSF_OK) return st;
    need = std::max(need, b);
  }
  *bytes = need;
  return HSF_OK;
}

hsf_status hsf_batch_create(const hsf_batch_item *items, int32_t count, void *workspace, size_t workspace_bytes,
                            void *stream, hsf_batch **out) {
  if (!items || count <= 0 || !workspace || !out) return set_error(HSF_EINVAL, "bad batch");
  *out = nullptr;
  std::unique_ptr<hsf_batch> b(new hsf_batch());
  cudaStream_t cs = (cudaStream_t)stream;
  CUDA_TRY(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
  hsf_status st = HSF_OK;
  for (int i = 0; i < count && st == HSF_OK; ++i)
    st = hsf_run(items[i].plan, items[i].bitstrings, items[i].num, items[i].window, 0, 0, items[i].out, workspace,
                 workspace_bytes, stream);
  cudaGraph_t g = nullptr;
  const cudaError_t ce = cudaStreamEndCapture(cs, &g);
  if (st != HSF_OK) {
    if (g) cudaGraphDestroy(g);
    return st;
  }
  if (ce != cudaSuccess) return set_error(HSF_ECUDA, "stream capture: %s", cudaGetErrorString(ce));
  b->graph = g;
  size_t n = 0;
  CUDA_TRY(cudaGraphGetNodes(g, nullptr, &n));
  std::vector<cudaGraphNode_t> nodes(n);
  if (n) CUDA_TRY(cudaGraphGetNodes(g, nodes.data(), &n));
  for (auto nd : nodes) {
    cudaGraphNodeType t;
    CUDA_TRY(cudaGraphNodeGetType(nd, &t));
    if (t == cudaGraphNodeTypeKernel) b->nodes++;     // kernels launched per replay
  }
  CUDA_TRY(cudaGraphInstantiate(&b->exec, g, 0));
  *out = b.release();
  return HSF_OK;
}

hsf_status hsf_batch_launch(hsf_batch *b, void *stream) {
  if (!b || !b->exec) return set_error(HSF_EINVAL, "bad batch");
  CUDA_TRY(cudaGraphLaunch(b->exec, (cudaStream_t)stream));
  g_launches += b->nodes;
  return HSF_OK;
}

int64_t hsf_batch_nodes(const hsf_batch *b) { return b ? (int64_t)b->nodes : 0; }

void hsf_batch_destroy(hsf_batch *b) { delete b; }

}  // extern "C"
