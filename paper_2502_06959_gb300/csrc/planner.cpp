// Host planner of the joint-cut HSF library (Sec. II-B, III-A, IV-A, IV-D).
//
//   * validate the circuit, the cut and the blocks; classify gates by side
//     (a: qubits l+1..n-1, b: qubits 0..l);
//   * check that every crossing gate is in exactly one block, that every block is
//     convex in the gate DAG and that the listed block order is compatible with it;
//   * multiply and Schmidt-decompose every block on the GPU (svd.cu), read back ranks,
//     singular values and factors;
//   * give every in-half gate a tree level: the number of the last block whose factor
//     it depends on, so gates that commute with a later Schmidt factor run before the
//     branching and the children of a path-tree node share that work (prefix reuse);
//   * per side, store the qubits touched at deeper levels in lower storage bits;
//   * per level: Schmidt factor first, then gates; merge runs of one-qubit gates;
//     split into tile passes (a tile holds 2^t amplitudes in shared memory) and
//     register groups (ops whose dense operands fit the per-thread register block);
//   * when the leaf level only touches a few low storage bits, precompute its whole
//     program as one small operator per Schmidt digit, so the leaf level is contracted
//     directly at the requested bitstrings instead of being simulated.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <condition_variable>
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
#include <thread>
#include <vector>

#include "plan.h"

namespace hsf {

thread_local std::string g_err;
std::atomic<uint64_t> g_launches{0};

hsf_status set_error(hsf_status code, const char *fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

const char *last_error() { return g_err.c_str(); }

// Plan-time device work (block SVDs, table uploads) runs on a private non-blocking stream
// of the calling thread, so planning the next circuit on the host overlaps with work the
// caller has queued on its own streams.  Each thread keeps one such stream per device it
// has used (created on first use on that device, kept until the thread exits).
namespace {
struct ThreadStreams {
  bool high = false;          // create at the device's highest stream priority
  std::map<int, cudaStream_t> by_dev;
  cudaStream_t get() {
    int cur = 0;
    cudaGetDevice(&cur);
    auto it = by_dev.find(cur);
    if (it != by_dev.end()) return it->second;
    cudaStream_t st = nullptr;
    int least = 0, greatest = 0;
    if (high && cudaDeviceGetStreamPriorityRange(&least, &greatest) == cudaSuccess)
      cudaStreamCreateWithPriority(&st, cudaStreamNonBlocking, greatest);
    else
      cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    by_dev[cur] = st;
    return st;
  }
};
}  // namespace

// The plan stream has the highest priority: the block SVD a plan waits for is scheduled
// as soon as CTAs of the runs already queued on other streams retire, so planning the next
// circuit overlaps the current run instead of waiting for it to drain.
cudaStream_t plan_stream() {
  thread_local ThreadStreams s{true, {}};
  return s.get();
}

// Second stream of the calling thread on which hsf_run sweeps side b (non-blocking).
cudaStream_t side_stream() {
  thread_local ThreadStreams s;
  return s.get();
}

// Device memory of plan tables.  cudaMalloc implicitly synchronises the streams of the
// device, so a plan created while another circuit runs must not call it: its tables
// (and the SVD scratch) are carved first-fit from slabs kept per device, and a slab is
// allocated only when none has room.  Freed blocks merge with their free neighbours.
namespace {
struct Arena {
  std::vector<std::pair<char *, size_t>> slabs;
  std::map<char *, size_t> free_blocks;   // address -> bytes
  std::map<char *, size_t> used;
};
std::mutex g_arena_mu;
std::map<int, Arena> g_arenas;
constexpr size_t kSlabBytes = (size_t)64 << 20;
}  // namespace

void *table_alloc(size_t bytes) {
  bytes = (bytes + 255) / 256 * 256;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
  std::lock_guard<std::mutex> lock(g_arena_mu);
  Arena &A = g_arenas[dev];
  for (auto it = A.free_blocks.begin(); it != A.free_blocks.end(); ++it) {
    if (it->second < bytes) continue;
    char *ptr = it->first;
    const size_t rest = it->second - bytes;
    A.free_blocks.erase(it);
    if (rest) A.free_blocks[ptr + bytes] = rest;
    A.used[ptr] = bytes;
    return ptr;
  }
  const size_t slab = std::max(kSlabBytes, bytes);
  char *mem = nullptr;
  if (cudaMalloc((void **)&mem, slab) != cudaSuccess) return nullptr;
  A.slabs.push_back({mem, slab});
  if (slab > bytes) A.free_blocks[mem + bytes] = slab - bytes;
  A.used[mem] = bytes;
  return mem;
}

void table_free(void *p) {
  if (!p) return;
  std::lock_guard<std::mutex> lock(g_arena_mu);
  for (auto &kv : g_arenas) {
    Arena &A = kv.second;
    auto u = A.used.find((char *)p);
    if (u == A.used.end()) continue;
    char *ptr = u->first;
    size_t bytes = u->second;
    A.used.erase(u);
    // merge with the free neighbours inside the same slab
    auto next = A.free_blocks.lower_bound(ptr);
    if (next != A.free_blocks.end() && next->first == ptr + bytes) {
      bool same = false;
      for (auto &sl : A.slabs) same |= ptr >= sl.first && next->first < sl.first + sl.second;
      if (same) {
        bytes += next->second;
        next = A.free_blocks.erase(next);
      }
    }
    if (next != A.free_blocks.begin()) {
      auto prev = std::prev(next);
      bool same = false;
      for (auto &sl : A.slabs) same |= prev->first >= sl.first && ptr < sl.first + sl.second && prev->first < ptr;
      if (same && prev->first + prev->second == ptr) {
        prev->second += bytes;
        return;
      }
    }
    A.free_blocks[ptr] = bytes;
    return;
  }
}

// Page-locked host staging for the table uploads: a few buffers reused across plans (one
// is taken for an upload and given back once its copy has completed), so the copy runs
// at DMA speed and nothing is allocated once the buffers have grown.
namespace {
std::mutex g_stage_mu;
std::vector<StagingBuf> g_stage_free;
}  // namespace

StagingBuf staging_take() {
  std::lock_guard<std::mutex> lock(g_stage_mu);
  if (g_stage_free.empty()) return StagingBuf{};
  StagingBuf s = g_stage_free.back();
  g_stage_free.pop_back();
  s.size = 0;
  return s;
}

void staging_give(StagingBuf s) {
  if (!s.p) return;
  std::lock_guard<std::mutex> lock(g_stage_mu);
  g_stage_free.push_back(s);
}

bool staging_reserve(StagingBuf &s, size_t need) {
  if (need <= s.cap) return true;
  const size_t cap = std::max(need, std::max(2 * s.cap, (size_t)1 << 20));
  unsigned char *q = nullptr;
  if (cudaHostAlloc((void **)&q, cap, cudaHostAllocPortable) != cudaSuccess) return false;
  if (s.size) std::memcpy(q, s.p, s.size);
  if (s.p) cudaFreeHost(s.p);
  s.p = q;
  s.cap = cap;
  return true;
}

// A persistent pool of host threads for the plan's independent composition tasks (no
// thread start per plan).  run(n, fn) calls fn(0..n-1) on the pool and the caller and
// returns when all are done; a call made while the pool is busy (another host thread
// planning) runs its tasks on the caller alone.
namespace {
class HostPool {
 public:
  explicit HostPool(int workers) {
    for (int i = 0; i < workers; ++i) th_.emplace_back([this] { loop(); });
    for (auto &t : th_) t.detach();       // the pool lives until the process exits
  }
  void run(size_t n, const std::function<void(size_t)> &fn) {
    std::unique_lock<std::mutex> busy(run_mu_, std::try_to_lock);
    if (!busy.owns_lock() || th_.empty() || n <= 1) {
      for (size_t i = 0; i < n; ++i) fn(i);
      return;
    }
    {
      std::lock_guard<std::mutex> lk(mu_);
      fn_ = &fn;
      n_ = n;
      next_ = 0;
      active_ = (int)th_.size();
      ++gen_;
    }
    cv_.notify_all();
    work(fn, n);
    std::unique_lock<std::mutex> lk(mu_);
    done_cv_.wait(lk, [&] { return active_ == 0; });
    fn_ = nullptr;
  }

 private:
  void work(const std::function<void(size_t)> &fn, size_t n) {
    for (size_t i = next_++; i < n; i = next_++) fn(i);
  }
  void loop() {
    uint64_t seen = 0;
    for (;;) {
      const std::function<void(size_t)> *fn;
      size_t n;
      {
        std::unique_lock<std::mutex> lk(mu_);
        cv_.wait(lk, [&] { return gen_ != seen; });
        seen = gen_;
        fn = fn_;
        n = n_;
      }
      work(*fn, n);
      std::lock_guard<std::mutex> lk(mu_);
      if (--active_ == 0) done_cv_.notify_all();
    }
  }
  std::vector<std::thread> th_;
  std::mutex run_mu_, mu_;
  std::condition_variable cv_, done_cv_;
  const std::function<void(size_t)> *fn_ = nullptr;
  size_t n_ = 0;
  std::atomic<size_t> next_{0};
  int active_ = 0;
  uint64_t gen_ = 0;
};
}  // namespace

void host_parallel_for(size_t n, const std::function<void(size_t)> &fn) {
  static HostPool *pool = [] {
    const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
    return new HostPool((int)std::min(15u, hw > 1 ? hw - 1 : 0u));
  }();
  pool->run(n, fn);
}

int device_sm_count() {
  static std::mutex mu;
  static std::map<int, int> cache;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  std::lock_guard<std::mutex> lock(mu);
  auto it = cache.find(dev);
  if (it != cache.end()) return it->second;
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) return 0;
  cache[dev] = sms;
  return sms;
}

#define CUDA_TRY(expr)                                                                   \
  do {                                                                                   \
    cudaError_t e_ = (expr);                                                             \
    if (e_ != cudaSuccess)                                                               \
      return set_error(HSF_ECUDA, "%s failed: %s", #expr, cudaGetErrorString(e_));       \
  } while (0)

namespace {

// ---------------------------------------------------------------------------
// Gate matrices (FP64).  R_P(t) = exp(-i t P / 2).
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
      return set_error(HSF_EINVAL, "unknown gate kind %d", kind);
  }
  return HSF_OK;
}

// acc += a * b, written out (std::complex's operator* takes a slow path that handles
// infinities; the planner's matrices are finite)
inline void cmac(cd &acc, const cd &a, const cd &b) {
  acc = cd(acc.real() + a.real() * b.real() - a.imag() * b.imag(),
           acc.imag() + a.real() * b.imag() + a.imag() * b.real());
}

std::vector<cd> matmul(const std::vector<cd> &a, const std::vector<cd> &b, int d) {
  std::vector<cd> r((size_t)d * d, 0.0);
  for (int i = 0; i < d; ++i)
    for (int k = 0; k < d; ++k) {
      const cd aik = a[(size_t)i * d + k];
      if (aik == 0.0) continue;
      for (int j = 0; j < d; ++j) cmac(r[(size_t)i * d + j], aik, b[(size_t)k * d + j]);
    }
  return r;
}

bool is_diagonal(const std::vector<cd> &m, int d) {
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j)
      if (i != j && m[(size_t)i * d + j] != 0.0) return false;
  return true;
}

int popcount64(uint64_t x) { return __builtin_popcountll(x); }

// ---------------------------------------------------------------------------
// DAG with blocks contracted to single nodes; Kahn's algorithm with the smallest
// gate index first.  The listed block order is enforced as extra edges.
// ---------------------------------------------------------------------------
hsf_status execution_order(const hsf_plan &p, std::vector<std::pair<bool, int>> &order) {
  if (!p.order.empty()) {                      // computed once when the plan was checked
    order = p.order;
    return HSF_OK;
  }
  // Kahn's algorithm over the gate DAG with every block contracted to one node; among the
  // ready nodes the one with the smallest first gate index goes first
  const int G = (int)p.gates.size();
  const int B = (int)p.blocks.size();
  const int V = B + G;
  std::vector<int> owner(G, -1);
  for (int b = 0; b < B; ++b)
    for (int gi : p.blocks[b].gates) owner[gi] = b;
  std::vector<int> key(V, 0);
  std::vector<char> used(V, 0);
  for (int b = 0; b < B; ++b) {
    key[b] = *std::min_element(p.blocks[b].gates.begin(), p.blocks[b].gates.end());
    used[b] = 1;
  }
  for (int gi = 0; gi < G; ++gi)
    if (owner[gi] < 0) {
      key[B + gi] = gi;
      used[B + gi] = 1;
    }
  auto nid = [&](int gi) { return owner[gi] >= 0 ? owner[gi] : B + gi; };
  std::vector<uint64_t> edges;                 // (u << 32) | v, deduplicated below
  edges.reserve((size_t)2 * G + B);
  std::vector<int> last(p.n, -1);
  for (int gi = 0; gi < G; ++gi) {
    const int v = nid(gi);
    for (int j = 0; j < p.gates[gi].nq; ++j) {
      const int q = p.gates[gi].q[j];
      if (last[q] >= 0) {
        const int u = nid(last[q]);
        if (u != v) edges.push_back(((uint64_t)u << 32) | (uint32_t)v);
      }
      last[q] = gi;
    }
  }
  for (int b = 0; b + 1 < B; ++b) edges.push_back(((uint64_t)b << 32) | (uint32_t)(b + 1));
  std::sort(edges.begin(), edges.end());
  edges.erase(std::unique(edges.begin(), edges.end()), edges.end());
  // successor lists in CSR form (edges are sorted by source)
  std::vector<int> start(V + 1, 0), succ(edges.size()), indeg(V, 0);
  for (size_t e = 0; e < edges.size(); ++e) {
    const int u = (int)(edges[e] >> 32), v = (int)(uint32_t)edges[e];
    start[u + 1]++;
    succ[e] = v;
    indeg[v]++;
  }
  for (int v = 0; v < V; ++v) start[v + 1] += start[v];
  using QE = std::pair<int, int>;
  std::priority_queue<QE, std::vector<QE>, std::greater<QE>> pq;
  int total = 0;
  for (int v = 0; v < V; ++v) {
    total += used[v];
    if (used[v] && indeg[v] == 0) pq.push({key[v], v});
  }
  order.clear();
  order.reserve(total);
  while (!pq.empty()) {
    const int v = pq.top().second;
    pq.pop();
    order.push_back({v < B, v < B ? v : v - B});
    for (int e = start[v]; e < start[v + 1]; ++e)
      if (--indeg[succ[e]] == 0) pq.push({key[succ[e]], succ[e]});
  }
  if ((int)order.size() != total)
    return set_error(HSF_EBLOCK, "a block is not convex in the circuit DAG, or the blocks are not "
                                 "listed in an order compatible with the circuit");
  return HSF_OK;
}

// ---------------------------------------------------------------------------
// Ops.
// ---------------------------------------------------------------------------
void merge_one_qubit_runs(std::vector<OpH> &ops) {
  std::vector<OpH> out;
  std::map<int, int> last;   // qubit -> index in out of the last op touching it
  for (auto &op : ops) {
    if (op.nq == 1 && op.digits == 1 && op.param < 0 && op.block < 0) {
      auto it = last.find(op.q[0]);
      if (it != last.end()) {
        OpH &prev = out[it->second];
        if (prev.nq == 1 && prev.digits == 1 && prev.param < 0 && prev.block < 0) {
          // prev then op (the ops in between do not touch this qubit): op * prev
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

// Matrix of op for Schmidt digit d (ops without digits have one matrix), as a dense
// 2^nq x 2^nq matrix.
std::vector<cd> dense_of(const OpH &op, int d) {
  const int dim = 1 << op.nq;
  const size_t per = op.type == OP_DENSE ? (size_t)dim * dim : (size_t)dim;
  const cd *m = op.m.data() + (op.digits > 1 ? (size_t)d * per : 0);
  if (op.type == OP_DENSE) return std::vector<cd>(m, m + per);
  std::vector<cd> full((size_t)dim * dim, 0.0);
  for (int i = 0; i < dim; ++i) full[(size_t)i * (dim + 1)] = m[i];
  return full;
}

// A one-qubit matrix u on operand x (x = 0 is the matrix MSB) of a two-qubit op, as 4x4.
std::vector<cd> embed_operand(const std::vector<cd> &u, int x) {
  std::vector<cd> e(16, 0.0);
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) {
      const int ix = x == 0 ? i >> 1 : i & 1, jx = x == 0 ? j >> 1 : j & 1;
      const int io = x == 0 ? i & 1 : i >> 1, jo = x == 0 ? j & 1 : j >> 1;
      if (io == jo) e[i * 4 + j] = u[ix * 2 + jx];
    }
  return e;
}

// op <- (u on operand x) applied before (after = false) or after (after = true) op, for
// every digit of either; both stay diagonal when both are.
void fold_one_qubit(OpH &op, const OpH &u, int x, bool after) {
  const int D = std::max(op.digits, u.digits);
  const bool diag = op.type == OP_DIAG && u.type == OP_DIAG;
  std::vector<cd> out;
  for (int d = 0; d < D; ++d) {
    const std::vector<cd> e = op.nq == 2 ? embed_operand(dense_of(u, d), x) : dense_of(u, d);
    const std::vector<cd> prod =
        after ? matmul(e, dense_of(op, d), 1 << op.nq) : matmul(dense_of(op, d), e, 1 << op.nq);
    if (diag) {
      for (int i = 0; i < (1 << op.nq); ++i) out.push_back(prod[(size_t)i * ((1 << op.nq) + 1)]);
    } else {
      out.insert(out.end(), prod.begin(), prod.end());
    }
  }
  op.type = diag ? OP_DIAG : OP_DENSE;
  op.m.swap(out);
  op.digits = D;
  if (u.block >= 0) op.block = u.block;
}

// Fold one-qubit ops into two-qubit ops (forward-only programs):
//  * into the next two-qubit op on the qubit (nothing touches the qubit in between, so
//    applying the one-qubit op right before it is the same): U then CZ / RZZ / CX on
//    (a, b) becomes one 4x4 op, which costs what the one-qubit op costs and makes the
//    diagonal gate free.  A Schmidt factor on one qubit folds the same way; the 4x4 op
//    then carries one matrix per digit.
//  * a one-qubit op with no later two-qubit op on its qubit folds into the previous op
//    on the qubit (applied after it), when that op is a two-qubit op or a factor.
void absorb_into_two_qubit(std::vector<OpH> &ops) {
  std::vector<char> dead(ops.size(), 0);
  std::map<int, int> pending;   // qubit -> index of its unabsorbed one-qubit op
  for (size_t o = 0; o < ops.size(); ++o) {
    OpH &op = ops[o];
    if (op.nq == 1 && op.param < 0) {
      auto it = pending.find(op.q[0]);
      if (it != pending.end() && op.digits == 1 && op.block < 0) {
        // a one-qubit op right after another one (e.g. after a Schmidt factor): one op
        fold_one_qubit(ops[it->second], op, 0, true);
        dead[o] = 1;
        continue;
      }
      pending[op.q[0]] = (int)o;
      continue;
    }
    if (op.nq == 2 && op.digits == 1 && op.block < 0 && op.param < 0) {
      for (int x = 0; x < 2; ++x) {
        auto it = pending.find(op.q[x]);
        if (it == pending.end()) continue;
        const OpH &u = ops[it->second];
        if (u.digits > 1 && op.digits > 1) {            // two factors: keep apart
          pending.erase(it);
          continue;
        }
        fold_one_qubit(op, u, x, false);
        dead[it->second] = 1;
        pending.erase(it);
      }
      continue;
    }
    for (int x = 0; x < op.nq; ++x) pending.erase(op.q[x]);
  }
  // what is left pending has no later op on its qubit: fold it into the previous one
  for (auto &kv : pending) {
    const int o = kv.second;
    const OpH &u = ops[o];
    if (u.digits > 1 || u.block >= 0) continue;
    int prev = -1;
    for (int j = o - 1; j >= 0 && prev < 0; --j) {
      if (dead[j]) continue;
      for (int x = 0; x < ops[j].nq; ++x)
        if (ops[j].q[x] == u.q[0]) prev = j;
    }
    if (prev < 0 || ops[prev].param >= 0) continue;
    OpH &tgt = ops[prev];
    if (tgt.nq == 2) {
      fold_one_qubit(tgt, u, tgt.q[0] == u.q[0] ? 0 : 1, true);
    } else if (tgt.nq == 1 && tgt.digits > 1) {
      fold_one_qubit(tgt, u, 0, true);
    } else {
      continue;
    }
    dead[o] = 1;
  }
  std::vector<OpH> out;
  for (size_t o = 0; o < ops.size(); ++o)
    if (!dead[o]) out.push_back(ops[o]);
  ops.swap(out);
}

// Reorder the operands of an op (new operand x = old operand perm[x]) and permute
// its matrices (every digit) to match: new index bit (nq-1-x) = old bit (nq-1-perm[x]).
void permute_operands(OpH &op, const int *perm) {
  const int nq = op.nq;
  const int d = 1 << nq;
  auto sigma = [&](int a) {
    int r = 0;
    for (int x = 0; x < nq; ++x)
      if ((a >> (nq - 1 - x)) & 1) r |= 1 << (nq - 1 - perm[x]);
    return r;
  };
  const int per = op.type == OP_DENSE ? d * d : d;
  std::vector<cd> out(op.m.size());
  for (int dg = 0; dg < op.digits; ++dg) {
    const cd *src = op.m.data() + (size_t)dg * per;
    cd *dst = out.data() + (size_t)dg * per;
    if (op.type == OP_DENSE) {
      for (int a = 0; a < d; ++a)
        for (int b = 0; b < d; ++b) dst[a * d + b] = src[sigma(a) * d + sigma(b)];
    } else {
      for (int a = 0; a < d; ++a) dst[a] = src[sigma(a)];
    }
  }
  op.m.swap(out);
  int q[3] = {op.q[0], op.q[1], op.q[2]};
  for (int x = 0; x < nq; ++x) op.q[x] = q[perm[x]];
}

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
      if (qm & blocked) {
        later.push_back(op);
        blocked |= qm;
        continue;
      }
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
    for (int q = 0; q < tmax; ++q) ps.active |= 1ull << q;
    ps.t = tmax;
    lv.passes.push_back(ps);
  }
}

// Register groups: consecutive ops whose dense operands fit `rb` tile bits.
void build_groups(PassH &ps, int rb) {
  ps.groups.clear();
  if (ps.t < rb) return;                     // the plain shared-memory kernel runs it
  int tile_bit[64];
  int tb = 0;
  for (int q = 0; q < 64; ++q) tile_bit[q] = (ps.active >> q) & 1ull ? tb++ : -1;
  uint32_t cur = 0;
  int first = 0;
  auto close = [&](int end) {
    if (end == first && !ps.groups.empty()) return;
    GroupH g;
    g.first_op = first;
    g.num_ops = end - first;
    int k = 0;
    for (int b = 0; b < ps.t && k < rb; ++b)
      if (cur & (1u << b)) g.slots[k++] = b;
    for (int b = 0; b < ps.t && k < rb; ++b)     // fill with the lowest free tile bits
      if (!(cur & (1u << b))) { cur |= 1u << b; g.slots[k++] = b; }
    std::sort(g.slots, g.slots + k);
    ps.groups.push_back(g);
    first = end;
    cur = 0;
  };
  for (int o = 0; o < (int)ps.ops.size(); ++o) {
    const OpH &op = ps.ops[o];
    if (op.type == OP_DIAG) continue;
    uint32_t need = 0;
    for (int j = 0; j < op.nq; ++j) need |= 1u << tile_bit[op.q[j]];
    if (__builtin_popcount(cur | need) <= rb) {
      cur |= need;
    } else {
      close(o);
      cur = need;
    }
  }
  if (first < (int)ps.ops.size() || ps.groups.empty()) close((int)ps.ops.size());
}

// Apply one op to a vector over the 2^c lowest storage bits (host, FP64).
void host_apply(std::vector<cd> &v, int c, const OpH &op, int digit) {
  const int nq = op.nq, d = 1 << nq;
  const int per = op.type == OP_DENSE ? d * d : d;
  const cd *m = op.m.data() + (op.digits > 1 ? (size_t)digit * per : 0);
  const int dim = 1 << c;
  if (op.type == OP_DIAG) {
    for (int i = 0; i < dim; ++i) {
      int idx = 0;
      for (int x = 0; x < nq; ++x) idx |= ((i >> op.q[x]) & 1) << (nq - 1 - x);
      cd z = 0.0;
      cmac(z, v[i], m[idx]);
      v[i] = z;
    }
    return;
  }
  int mask = 0;
  for (int x = 0; x < nq; ++x) mask |= 1 << op.q[x];
  for (int i = 0; i < dim; ++i) {
    if (i & mask) continue;
    cd in[8], out[8];
    int addr[8];
    for (int k = 0; k < d; ++k) {
      int a = i;
      for (int x = 0; x < nq; ++x)
        if ((k >> (nq - 1 - x)) & 1) a |= 1 << op.q[x];
      addr[k] = a;
      in[k] = v[a];
    }
    for (int r = 0; r < d; ++r) {
      out[r] = 0.0;
      for (int k = 0; k < d; ++k) cmac(out[r], m[r * d + k], in[k]);
    }
    for (int k = 0; k < d; ++k) v[addr[k]] = out[k];
  }
}

// M <- op M for a 2^c x 2^c matrix stored row-major as separate real and imaginary
// parts: the op acts on the row index and every column gets the same op, so the inner
// loop runs over contiguous columns (the product of a level's shared ops, composed
// once for all digits).
void host_apply_rows(std::vector<double> &re, std::vector<double> &im, int c, const OpH &op) {
  const int dim = 1 << c, nq = op.nq, d = 1 << nq;
  const cd *m = op.m.data();
  if (op.type == OP_DIAG) {
    for (int i = 0; i < dim; ++i) {
      int idx = 0;
      for (int x = 0; x < nq; ++x) idx |= ((i >> op.q[x]) & 1) << (nq - 1 - x);
      const double mr = m[idx].real(), mi = m[idx].imag();
      double *r = re.data() + (size_t)i * dim, *q = im.data() + (size_t)i * dim;
      for (int col = 0; col < dim; ++col) {
        const double a = r[col], b = q[col];
        r[col] = mr * a - mi * b;
        q[col] = mr * b + mi * a;
      }
    }
    return;
  }
  int mask = 0;
  for (int x = 0; x < nq; ++x) mask |= 1 << op.q[x];
  std::vector<double> tr((size_t)d * dim), ti((size_t)d * dim);
  for (int i = 0; i < dim; ++i) {
    if (i & mask) continue;
    int addr[8];
    for (int k = 0; k < d; ++k) {
      int a = i;
      for (int x = 0; x < nq; ++x)
        if ((k >> (nq - 1 - x)) & 1) a |= 1 << op.q[x];
      addr[k] = a;
    }
    for (int r = 0; r < d; ++r) {
      double *orr = tr.data() + (size_t)r * dim, *oi = ti.data() + (size_t)r * dim;
      std::fill(orr, orr + dim, 0.0);
      std::fill(oi, oi + dim, 0.0);
      for (int k = 0; k < d; ++k) {
        const double mr = m[r * d + k].real(), mi = m[r * d + k].imag();
        if (mr == 0.0 && mi == 0.0) continue;
        const double *xr = re.data() + (size_t)addr[k] * dim, *xi = im.data() + (size_t)addr[k] * dim;
        for (int col = 0; col < dim; ++col) {
          orr[col] += mr * xr[col] - mi * xi[col];
          oi[col] += mr * xi[col] + mi * xr[col];
        }
      }
    }
    for (int r = 0; r < d; ++r) {
      std::copy(tr.data() + (size_t)r * dim, tr.data() + (size_t)(r + 1) * dim, re.data() + (size_t)addr[r] * dim);
      std::copy(ti.data() + (size_t)r * dim, ti.data() + (size_t)(r + 1) * dim, im.data() + (size_t)addr[r] * dim);
    }
  }
}

template <typename C>
void pack_pass(const PassH &ps, std::vector<DevOp> &dops, std::vector<C> &mats, std::vector<DevGroup> &dgroups) {
  int tile_bit[64];
  int tb = 0;
  for (int q = 0; q < 64; ++q) tile_bit[q] = (ps.active >> q) & 1ull ? tb++ : -1;
  std::vector<int> group_of(ps.ops.size(), -1);
  for (int g = 0; g < (int)ps.groups.size(); ++g)
    for (int o = ps.groups[g].first_op; o < ps.groups[g].first_op + ps.groups[g].num_ops; ++o) group_of[o] = g;
  for (size_t o = 0; o < ps.ops.size(); ++o) {
    OpH op = ps.ops[o];
    int slot[3] = {-1, -1, -1};
    const GroupH *G = group_of[o] >= 0 ? &ps.groups[group_of[o]] : nullptr;
    auto slot_of = [&](int storage_bit) {
      if (!G) return -1;
      const int tbit = tile_bit[storage_bit];
      for (int j = 0; j < kMaxSlots && G->slots[j] >= 0; ++j)
        if (G->slots[j] == tbit && tbit >= 0) return j;
      return -1;
    };
    int kcase = 0;
    if (G) {
      int perm[3] = {0, 1, 2};
      int sl[3];
      for (int x = 0; x < op.nq; ++x) sl[x] = slot_of(op.q[x]);
      // dense: slots descending; diag: slot operands first, descending
      std::sort(perm, perm + op.nq, [&](int a, int b) {
        const int ka = sl[a], kb = sl[b];
        if ((ka >= 0) != (kb >= 0)) return ka >= 0;
        return ka > kb;
      });
      permute_operands(op, perm);
      int ns = 0;
      for (int x = 0; x < op.nq; ++x) {
        slot[x] = slot_of(op.q[x]);
        if (slot[x] >= 0) ++ns;
      }
      if (op.type == OP_DENSE) {
        kcase = op.nq == 1 ? slot[0]
              : op.nq == 2 ? 16 + (slot[0] << 3) + slot[1]
                           : 128 + (slot[0] << 6) + (slot[1] << 3) + slot[2];
      } else {
        kcase = ns;
      }
    }
    DevOp d{};
    d.type = op.type;
    d.nq = op.nq;
    for (int x = 0; x < 3; ++x) {
      d.pos[x] = 0;
      d.slot[x] = slot[x];
    }
    for (int x = 0; x < op.nq; ++x) {
      const int q = op.q[x];
      d.pos[x] = tile_bit[q] >= 0 ? tile_bit[q] : kFixedBit + q;
    }
    d.kcase = kcase;
    d.kidx = -1;
    if (G && op.type == OP_DENSE) {
      // dense index of the slot pattern: 1q J -> J; 2q (J>K) -> 5 + pair; 3q -> 15 + triple
      static const int pair_idx[5][5] = {{-1, -1, -1, -1, -1}, {0, -1, -1, -1, -1}, {1, 2, -1, -1, -1},
                                         {3, 4, 5, -1, -1}, {6, 7, 8, 9, -1}};
      if (op.nq == 1) d.kidx = slot[0];
      else if (op.nq == 2) d.kidx = 5 + pair_idx[slot[0]][slot[1]];
      else {
        int t = 0, found = -1;
        for (int J = 2; J < 5 && found < 0; ++J)
          for (int K = 1; K < J && found < 0; ++K)
            for (int L = 0; L < K && found < 0; ++L, ++t)
              if (J == slot[0] && K == slot[1] && L == slot[2]) found = t;
        d.kidx = 15 + found;
      }
    }
    if (sizeof(C) == 8 && (mats.size() & 1)) mats.push_back(C{});   // 16-byte aligned rows
    d.mat = (int32_t)mats.size();
    const int per = op.type == OP_DENSE ? (1 << (2 * op.nq)) : (1 << op.nq);
    d.digit_stride = op.digits > 1 ? per : 0;
    for (auto &z : op.m) {
      C c;
      c.x = (decltype(c.x))z.real();
      c.y = (decltype(c.y))z.imag();
      mats.push_back(c);
    }
    d.param = op.param;
    d.kmat = -1;
    if (op.param >= 0) {
      if (sizeof(C) == 8 && (mats.size() & 1)) mats.push_back(C{});
      d.kmat = (int32_t)mats.size();
      for (auto &z : op.k) {
        C c;
        c.x = (decltype(c.x))z.real();
        c.y = (decltype(c.y))z.imag();
        mats.push_back(c);
      }
    }
    dops.push_back(d);
  }
  for (auto &g : ps.groups) {
    DevGroup dg{};
    for (int j = 0; j < kMaxSlots; ++j) dg.slots[j] = g.slots[j];
    dg.first_op = g.first_op;
    dg.num_ops = g.num_ops;
    dgroups.push_back(dg);
  }
}

}  // namespace

// W images of the tensor-core levels: per digit m, the level's program U_m (64 x 64,
// column by column) in real form W[2i + a][2j + b] (a, b: re / im), split into TF32 hi
// and lo parts (levels with ops after the product) or scaled by a power of two and split
// into FP16 hi and lo parts (levels without).  The leaf level is left out when it will be contracted at the bitstrings
// (leaf_c > 0): it is never swept then.
void compose_mma_levels(hsf_plan &p, int leaf_c) {
  const int B = (int)p.blocks.size();
  const int dim = 1 << kMmaBits, K = 2 * dim;
  // One composition task per (level, digit); the levels' shared parts (the ops after the
  // last digit-dependent one, composed once as S) are prepared first, one task per level.
  struct LevelJob {
    LevelH *lv;
    std::vector<OpH> prefix;
    size_t split;
    std::vector<cd> S;       // column-major dim x dim
    bool f16;
    int r;
  };
  std::vector<LevelJob> jobs;
  for (int s = 0; s < 2; ++s)
    for (int k = 1; k <= B; ++k) {
      LevelH &lv = p.side[s].levels[k];
      if (lv.mma_prefix == 0 || (k == B && leaf_c > 0)) continue;
      // the prefix becomes the product; the rest stays as in-place passes
      std::vector<OpH> prefix(lv.ops.begin(), lv.ops.begin() + lv.mma_prefix);
      lv.ops.erase(lv.ops.begin(), lv.ops.begin() + lv.mma_prefix);
      lv.passes.clear();
      // the rest goes into the epilogue when every op is a 1- or 2-qubit op on storage
      // bits < kMmaPostBits (and the tiles have at least 32 rows of 64 amplitudes)
      bool post_ok = !lv.ops.empty() && lv.ops.size() <= (size_t)kMmaMaxPost && p.side[s].h >= kMmaPostBits;
      for (auto &op : lv.ops) {
        post_ok = post_ok && op.nq <= 2 && op.digits == 1;
        for (int j = 0; j < op.nq; ++j) post_ok = post_ok && op.q[j] < kMmaPostBits;
      }
      if (post_ok) {
        lv.post.swap(lv.ops);
        lv.ops.clear();
      }
      if (!lv.ops.empty()) {
        split_passes(lv, p.side[s].h, p.tile_max);
        if (!(p.flags & HSF_FLAG_NO_REGISTER_SWEEP))
          for (auto &ps : lv.passes) build_groups(ps, p.rbits);
      }
      lv.mma = true;
      LevelJob job;
      job.lv = &lv;
      job.prefix = prefix;
      job.r = (int)p.radix[k];
      // a level with ops after the product runs the TF32 kernel, one without the FP16 one
      job.f16 = lv.post.empty();
      lv.wimg.clear();        // every entry is written below, so no zero fill
      lv.wimg.resize(job.f16 ? (size_t)job.r * (kMmaWDigitBytes / 4) + (size_t)job.r
                             : (size_t)job.r * 2 * (kMmaWPartBytes / 4));
      // the ops after the last digit-dependent one are shared by every digit: compose
      // them once (S, column-major), then U_m e_col = S (prefix_m e_col), where the
      // prefix image of a basis vector has few nonzeros
      job.split = 0;
      for (size_t o = 0; o < prefix.size(); ++o)
        if (prefix[o].digits > 1) job.split = o + 1;
      jobs.push_back(std::move(job));
    }
  // the shared parts S, one task per level
  host_parallel_for(jobs.size(), [&](size_t j) {
    LevelJob &job = jobs[j];
    std::vector<double> re((size_t)dim * dim, 0.0), im((size_t)dim * dim, 0.0);
    for (int i = 0; i < dim; ++i) re[(size_t)i * dim + i] = 1.0;
    for (size_t o = job.split; o < job.prefix.size(); ++o) host_apply_rows(re, im, kMmaBits, job.prefix[o]);
    job.S.assign((size_t)dim * dim, cd(0.0));              // column-major
    for (int row = 0; row < dim; ++row)
      for (int col = 0; col < dim; ++col)
        job.S[(size_t)col * dim + row] = cd(re[(size_t)row * dim + col], im[(size_t)row * dim + col]);
  });
  std::vector<std::pair<int, int>> tasks;     // (job, digit)
  for (int j = 0; j < (int)jobs.size(); ++j)
    for (int m = 0; m < jobs[j].r; ++m) tasks.push_back({j, m});
  auto run_task = [&](const std::pair<int, int> &t, std::vector<double> &w, std::vector<cd> &u, std::vector<cd> &v) {
    const LevelJob &job = jobs[t.first];
    const int m = t.second;
    for (int col = 0; col < dim; ++col) {
      std::fill(u.begin(), u.end(), cd(0.0));
      u[col] = 1.0;
      for (size_t o = 0; o < job.split; ++o) host_apply(u, kMmaBits, job.prefix[o], m);
      std::fill(v.begin(), v.end(), cd(0.0));
      for (int j = 0; j < dim; ++j) {
        if (u[j] == cd(0.0)) continue;
        const cd *sj = job.S.data() + (size_t)j * dim;
        for (int row = 0; row < dim; ++row) cmac(v[row], sj[row], u[j]);
      }
      for (int row = 0; row < dim; ++row) {
        w[(size_t)(2 * row) * K + 2 * col] = v[row].real();
        w[(size_t)(2 * row) * K + 2 * col + 1] = -v[row].imag();
        w[(size_t)(2 * row + 1) * K + 2 * col] = v[row].imag();
        w[(size_t)(2 * row + 1) * K + 2 * col + 1] = v[row].real();
      }
    }
    LevelH &lv = *job.lv;
    if (job.f16) {
      level_mma_image_f16(w.data(), lv.wimg.data() + (size_t)m * (kMmaWDigitBytes / 4),
                          lv.wimg.data() + (size_t)job.r * (kMmaWDigitBytes / 4) + m);
    } else {
      float *hi = lv.wimg.data() + (size_t)m * 2 * (kMmaWPartBytes / 4);
      level_mma_image(w.data(), hi, hi + kMmaWPartBytes / 4);
    }
  };
  // the digits' compositions write disjoint parts of their level's image: the host pool
  // takes them in turn
  host_parallel_for(tasks.size(), [&](size_t i) {
    thread_local std::vector<double> w;
    thread_local std::vector<cd> u, v;
    w.resize((size_t)K * K);
    u.resize(dim);
    v.resize(dim);
    run_task(tasks[i], w, u, v);
  });
}

// Factored leaf operators.  The leaf level opens with the last block's Schmidt factor
// (Sec. IV-A: the factors X_m, Y_m start the branch of digit m), so before fusion its
// program is [F_m, rest]; when F_m is a one-qubit operator on the same storage bit of
// the chunk on both sides and the rest is digit-independent, L_m = S (F_m (x) I) with S
// the rest's matrix.  Then, with w = row x of S and d[(i, j)] = sum_k w[(i, k)] x[(j, k)]
// (i, j: the factor bit of the output and of the input),
//   sum_m (L^a_m x_a)(L^b_m x_b) = sum_{al, be} G[al][be] d_a[al] d_b[be],
//   G[(i, j)][(i', j')] = sum_m F^a_m[i][j] F^b_m[i'][j'],
// which is what the factored leaf kernel evaluates; the digit sum is done here once (for
// every digit range [m0, m1), so that partial path ranges need no other operator).  Only
// worth it for 3 or 4 digits on chunks of 4..16 amplitudes.
void factor_leaf(hsf_plan &p) {
  p.leaf_pf = -1;
  const int B = (int)p.blocks.size(), r = (int)p.radix[B], c = p.leaf_c, dim = 1 << c;
  if (p.precision != HSF_PREC_C64 || r < 3 || r > 4 || c < 2 || c > 4) return;
  int pf = -1;
  std::vector<cd> F[2];
  for (int s = 0; s < 2; ++s) {
    const std::vector<OpH> &pre = p.side[s].leaf_pre;
    if (pre.empty() || pre[0].type != OP_DENSE || pre[0].nq != 1 || pre[0].digits != r ||
        pre[0].block != B - 1 || pre[0].m.size() != (size_t)4 * r)
      return;
    if (s == 1 && pre[0].q[0] != pf) return;
    pf = pre[0].q[0];
    if (pf >= c) return;
    for (size_t o = 1; o < pre.size(); ++o)
      if (pre[o].digits != 1) return;
    F[s] = pre[0].m;
    std::vector<cd> S((size_t)dim * dim, 0.0);
    for (int col = 0; col < dim; ++col) {
      std::vector<cd> v(dim, 0.0);
      v[col] = 1.0;
      for (size_t o = 1; o < pre.size(); ++o) host_apply(v, c, pre[o], 0);
      for (int row = 0; row < dim; ++row) S[(size_t)row * dim + col] = v[row];
    }
    // check S (F_m (x) I) against the fused operators
    double err = 0.0, mx = 0.0;
    for (int m = 0; m < r; ++m)
      for (int row = 0; row < dim; ++row)
        for (int col = 0; col < dim; ++col) {
          const int jf = (col >> pf) & 1;
          cd z = 0.0;
          for (int kf = 0; kf < 2; ++kf)
            z += S[(size_t)row * dim + ((col & ~(1 << pf)) | (kf << pf))] * F[s][(size_t)m * 4 + kf * 2 + jf];
          const cd L = p.side[s].leaf_ops[((size_t)m * dim + row) * dim + col];
          err = std::max(err, std::abs(z - L));
          mx = std::max(mx, std::abs(L));
        }
    if (!(err <= 1e-10 * std::max(1.0, mx))) return;
    p.side[s].leaf_S = S;
  }
  p.leaf_G.assign((size_t)(r + 1) * (r + 1) * 16, 0.0);
  for (int m0 = 0; m0 < r; ++m0)
    for (int m1 = m0 + 1; m1 <= r; ++m1) {
      cd *G = p.leaf_G.data() + ((size_t)m0 * (r + 1) + m1) * 16;
      for (int m = m0; m < m1; ++m)
        for (int al = 0; al < 4; ++al)
          for (int be = 0; be < 4; ++be) G[al * 4 + be] += F[0][(size_t)m * 4 + al] * F[1][(size_t)m * 4 + be];
    }
  p.leaf_pf = pf;
}

// Leaf digit sums for short chunks.  For a bitstring whose chunk rows are i on side a and
// i' on side b, the parent's contribution sum_m (L^a_m x_a)[i] (L^b_m x_b)[i'] is the
// bilinear form x_a^T H[i][i'] x_b with H[i][i'][j][j'] = sum_m L^a_m[i][j] L^b_m[i'][j']:
// D^2 + D complex products per (bitstring, parent) instead of r (2D + 1), whatever the
// operators.  Built for chunks of 2 and 4 amplitudes (complex64) and every digit range
// [m0, m1), for the streaming leaf kernel.
void pair_leaf(hsf_plan &p) {
  p.leaf_H.clear();
  const int B = (int)p.blocks.size(), r = (int)p.radix[B], c = p.leaf_c, D = 1 << c;
  if (p.precision != HSF_PREC_C64 || c < 1 || c > 2) return;
  const size_t per = (size_t)D * D * D * D;
  p.leaf_H.assign((size_t)(r + 1) * (r + 1) * per, 0.0);
  const std::vector<cd> &La = p.side[0].leaf_ops, &Lb = p.side[1].leaf_ops;
  for (int m0 = 0; m0 < r; ++m0)
    for (int m1 = m0 + 1; m1 <= r; ++m1) {
      cd *H = p.leaf_H.data() + ((size_t)m0 * (r + 1) + m1) * per;
      for (int m = m0; m < m1; ++m)
        for (int i = 0; i < D; ++i)
          for (int i2 = 0; i2 < D; ++i2)
            for (int j = 0; j < D; ++j)
              for (int j2 = 0; j2 < D; ++j2)
                H[((size_t)(i * D + i2) * D + j) * D + j2] +=
                    La[((size_t)m * D + i) * D + j] * Lb[((size_t)m * D + i2) * D + j2];
    }
}

hsf_status build_programs(hsf_plan &p, bool grad) {
  const int B = (int)p.blocks.size();
  std::vector<std::pair<bool, int>> order;
  hsf_status st = execution_order(p, order);
  if (st != HSF_OK) return st;
  p.rbits = p.precision == HSF_PREC_C64
                ? ((p.flags & HSF_FLAG_REG5) ? 5 : (p.flags & HSF_FLAG_REG3) ? 3 : kRegBitsC64)
                : kRegBitsC128;
  int leaf_c = !grad && B > 0 && p.radix[B] <= 8 ? 0 : -1;
  for (int s = 0; s < 2; ++s) {
    SideH &sd = grad ? p.gside[s] : p.side[s];
    sd.h = s == 0 ? p.na : p.nb;
    sd.offset = s == 0 ? p.cut + 1 : 0;
    sd.levels.assign(B + 1, LevelH{});
    for (int b = 0; b < B; ++b) {           // Schmidt factors open levels 1..B
      const BlockH &bk = p.blocks[b];
      if (!bk.fops[s].empty()) {              // a closed-form factor as a list of ops
        for (OpH op : bk.fops[s]) {
          for (int j = 0; j < op.nq; ++j) op.q[j] -= sd.offset;
          sd.levels[b + 1].ops.push_back(op);
        }
        continue;
      }
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
      if (grad && g.param_id >= 0 && !g.k.empty()) {
        op.param = g.param_id;
        if (g.diag) {
          op.k.resize(d);
          for (int i = 0; i < d; ++i) op.k[i] = g.k[(size_t)i * d + i];
        } else {
          op.k = g.k;
        }
      }
      sd.levels[lvl].ops.push_back(op);
    }
    // storage order: qubits touched at deeper levels get lower storage bits
    std::vector<int> deep(sd.h, -1);
    for (int k = 0; k <= B; ++k)
      for (auto &op : sd.levels[k].ops)
        for (int j = 0; j < op.nq; ++j) deep[op.q[j]] = std::max(deep[op.q[j]], k);
    std::vector<int> qs(sd.h);
    for (int q = 0; q < sd.h; ++q) qs[q] = q;
    if (!(p.flags & HSF_FLAG_IDENTITY_STORAGE))
      std::stable_sort(qs.begin(), qs.end(), [&](int x, int y) {
        if (deep[x] != deep[y]) return deep[x] > deep[y];
        return s == 0 ? x < y : x > y;          // nearest to the cut first
      });
    sd.store.assign(sd.h, 0);
    for (int i = 0; i < sd.h; ++i) sd.store[qs[i]] = i;
    for (auto &lv : sd.levels)
      for (auto &op : lv.ops)
        for (int j = 0; j < op.nq; ++j) op.q[j] = sd.store[op.q[j]];
    if (!grad) sd.leaf_pre = sd.levels[B].ops;
    for (auto &lv : sd.levels) {
      merge_one_qubit_runs(lv.ops);
      if (!grad && !(p.flags & HSF_FLAG_NO_REGISTER_SWEEP)) absorb_into_two_qubit(lv.ops);
    }
    if (leaf_c >= 0) {
      int c = 0;
      for (auto &op : sd.levels[B].ops)
        for (int j = 0; j < op.nq; ++j) c = std::max(c, op.q[j] + 1);
      leaf_c = c <= 5 ? std::max(leaf_c, c) : -1;
    }
    // levels whose program, or a leading run of at least kMmaMinPrefix of its ops holding
    // every digit-dependent op, sits on the kMmaBits lowest storage bits run that part as
    // one tensor-core product per digit (complex64 forward programs); W is composed below,
    // once the leaf is known
    for (int k = 1; k <= B && !grad; ++k) {
      LevelH &lv = sd.levels[k];
      if (p.precision != HSF_PREC_C64 || sd.h < kMmaMinH || (p.flags & HSF_FLAG_NO_TC_LEVEL)) break;
      // a partial product whose rest needs a pass is only worth it on large levels; one
      // whose rest fits the product's epilogue already on medium ones
      const long double amps = (long double)(p.num_paths / p.below[k]) * (long double)(1ull << sd.h);
      const bool large = amps >= (long double)(1ull << 26), medium = amps >= (long double)(1ull << 24);
      size_t q = 0;
      for (; q < lv.ops.size(); ++q) {
        bool low = true;
        for (int j = 0; j < lv.ops[q].nq; ++j) low = low && lv.ops[q].q[j] < kMmaBits;
        if (!low) break;
      }
      bool digits_in_prefix = true, post_fit = lv.ops.size() - q <= (size_t)kMmaMaxPost && sd.h >= kMmaPostBits;
      for (size_t o = q; o < lv.ops.size(); ++o) {
        digits_in_prefix = digits_in_prefix && lv.ops[o].digits == 1;
        post_fit = post_fit && lv.ops[o].nq <= 2;
        for (int j = 0; j < lv.ops[o].nq; ++j) post_fit = post_fit && lv.ops[o].q[j] < kMmaPostBits;
      }
      if (q > 0 && digits_in_prefix &&
          (q == lv.ops.size() || (q >= (size_t)kMmaMinPrefix && (large || (medium && post_fit)))))
        lv.mma_prefix = q;
    }
    for (auto &lv : sd.levels) {
      split_passes(lv, sd.h, p.tile_max);
      // gradient programs too: the groups only say how the forward sweep holds the ops in
      // registers; the op list (every rotation its own op) is what the adjoint undoes
      if (!(p.flags & HSF_FLAG_NO_REGISTER_SWEEP))
        for (auto &ps : lv.passes) build_groups(ps, p.rbits);
    }
  }
  if (grad) return HSF_OK;
  // leaf operators L_m: the leaf program with digit m applied to every basis vector
  p.leaf_c = 0;
  const size_t csz = p.precision == HSF_PREC_C64 ? 8 : 16;
  if (leaf_c > 0 && leaf_c <= std::min(p.side[0].h, p.side[1].h) &&
      2 * p.radix[B] * (size_t)(1 << leaf_c) * ((1 << leaf_c) + 1) * csz <= 96 * 1024) {
    p.leaf_c = leaf_c;
    const int dim = 1 << leaf_c;
    const int r = (int)p.radix[B];
    for (int s = 0; s < 2; ++s) {
      SideH &sd = p.side[s];
      sd.leaf_ops.assign((size_t)r * dim * dim, 0.0);
      for (int m = 0; m < r; ++m)
        for (int col = 0; col < dim; ++col) {
          std::vector<cd> v(dim, 0.0);
          v[col] = 1.0;
          for (auto &op : sd.levels[B].ops) host_apply(v, leaf_c, op, m);
          for (int row = 0; row < dim; ++row) sd.leaf_ops[((size_t)m * dim + row) * dim + col] = v[row];
        }
    }
    factor_leaf(p);
    pair_leaf(p);
  }
  compose_mma_levels(p, p.leaf_c);
  return HSF_OK;
}

// Schroedinger plan (Sec. II-A, Example 1; Table I column S): the whole circuit as one
// program on one "side" of h = n qubits with the identity storage order, one tree level,
// no blocks and a single path.  The same fusion, tile-pass and register-group building as
// the HSF half states; the passes sweep the full 2^n state in place.
hsf_status build_schrodinger(hsf_plan &p, const hsf_circuit *c, const hsf_plan_opts *o) {
  if (!c) return set_error(HSF_EINVAL, "circuit must not be NULL");
  if (c->num_gates < 0 || (c->num_gates > 0 && !c->gates)) return set_error(HSF_EINVAL, "bad gate array");
  p.precision = o ? o->precision : HSF_PREC_C64;
  p.flags = o ? o->flags : 0;
  if (p.precision != HSF_PREC_C64 && p.precision != HSF_PREC_C128)
    return set_error(HSF_EINVAL, "precision %d", p.precision);
  const int nmax = p.precision == HSF_PREC_C64 ? 34 : 33;      // a state of at most 128 GB
  if (c->n < 1 || c->n > nmax) return set_error(HSF_EINVAL, "n = %d outside 1..%d for a full state", c->n, nmax);
  p.n = c->n;
  p.cut = c->n - 1;            // every gate on "side a" below (load_gates' side is unused)
  p.na = c->n;
  p.nb = 0;
  p.schrodinger = true;
  const int tcap = p.precision == HSF_PREC_C64 ? kRegTileC64 : kRegTileC128;
  p.tile_max = (o && o->tile_bits) ? o->tile_bits : tcap;
  if (p.tile_max < 3 || p.tile_max > tcap) return set_error(HSF_EINVAL, "tile_bits %d outside 3..%d", p.tile_max, tcap);
  p.tile_max = std::min(p.tile_max, p.n);
  hsf_status st = load_gates(p, c, o);
  if (st != HSF_OK) return st;
  p.rbits = p.precision == HSF_PREC_C64
                ? ((p.flags & HSF_FLAG_REG5) ? 5 : (p.flags & HSF_FLAG_REG3) ? 3 : kRegBitsC64)
                : kRegBitsC128;
  p.radix.assign(1, 1);
  p.below.assign(1, 1);
  p.num_paths = 1;
  p.tree_nodes = 1;
  SideH &sd = p.side[0];
  sd.h = p.n;
  sd.offset = 0;
  sd.store.resize(p.n);
  for (int q = 0; q < p.n; ++q) sd.store[q] = q;
  sd.levels.assign(1, LevelH{});
  LevelH &lv = sd.levels[0];
  for (const GateH &g : p.gates) {
    OpH op;
    op.type = g.diag ? OP_DIAG : OP_DENSE;
    op.nq = g.nq;
    for (int j = 0; j < g.nq; ++j) op.q[j] = g.q[j];
    const int d = 1 << g.nq;
    if (g.diag) {
      op.m.resize(d);
      for (int i = 0; i < d; ++i) op.m[i] = g.m[(size_t)i * d + i];
    } else {
      op.m = g.m;
    }
    lv.ops.push_back(op);
  }
  merge_one_qubit_runs(lv.ops);
  if (!(p.flags & HSF_FLAG_NO_REGISTER_SWEEP)) absorb_into_two_qubit(lv.ops);
  split_passes(lv, sd.h, p.tile_max);
  if (!(p.flags & HSF_FLAG_NO_REGISTER_SWEEP))
    for (auto &ps : lv.passes) build_groups(ps, p.rbits);
  p.side[1] = SideH{};
  st = upload_programs(p);
  if (st != HSF_OK) return st;
  p.launches = (int64_t)lv.passes.size();
  p.dev_status = (int32_t *)table_alloc(256);
  if (!p.dev_status) return set_error(HSF_ENOMEM, "device status words");
  CUDA_TRY(cudaMemsetAsync(p.dev_status, 0, 256, plan_stream()));
  CUDA_TRY(cudaStreamSynchronize(plan_stream()));
  return HSF_OK;
}

hsf_status upload_programs(hsf_plan &p, bool grad) {
  // the table is assembled in page-locked staging and copied with one DMA
  struct HostTable {
    StagingBuf s = staging_take();
    bool ok = true;
    ~HostTable() { staging_give(s); }
    size_t size() const { return s.size; }
    bool empty() const { return s.size == 0; }
    const unsigned char *data() const { return s.p; }
    void put(const void *ptr, size_t bytes, bool zero) {
      if (!bytes || !ok) return;
      if (!staging_reserve(s, s.size + bytes)) {
        ok = false;
        return;
      }
      if (zero) std::memset(s.p + s.size, 0, bytes);
      else std::memcpy(s.p + s.size, ptr, bytes);
      s.size += bytes;
    }
  } host;
  auto align = [&](size_t a) { host.put(nullptr, (a - host.size() % a) % a, true); };
  auto append = [&](const void *ptr, size_t bytes) { host.put(ptr, bytes, false); };
  int64_t launches = 0;
  for (int s = 0; s < 2; ++s) {
    for (auto &lv : (grad ? p.gside[s] : p.side[s]).levels)
      for (auto &ps : lv.passes) {
        std::vector<DevOp> dops;
        std::vector<DevGroup> dgroups;
        ps.num_ops = (int)ps.ops.size();
        if (p.precision == HSF_PREC_C64) {
          std::vector<float2> mats;
          pack_pass(ps, dops, mats, dgroups);
          align(256); ps.ops_off = host.size(); append(dops.data(), dops.size() * sizeof(DevOp));
          align(256); ps.mats_off = host.size(); append(mats.data(), mats.size() * sizeof(float2));
        } else {
          std::vector<double2> mats;
          pack_pass(ps, dops, mats, dgroups);
          align(256); ps.ops_off = host.size(); append(dops.data(), dops.size() * sizeof(DevOp));
          align(256); ps.mats_off = host.size(); append(mats.data(), mats.size() * sizeof(double2));
        }
        align(256); ps.groups_off = host.size(); append(dgroups.data(), dgroups.size() * sizeof(DevGroup));
        ps.table_end = host.size();
        ++launches;
      }
    SideH &sd = grad ? p.gside[s] : p.side[s];
    for (auto &lv : sd.levels)
      if (lv.mma) {
        align(1024);
        lv.w_off = host.size();
        append(lv.wimg.data(), lv.wimg.size() * sizeof(float));
        align(256);
        lv.post_off = host.size();
        for (const OpH &op : lv.post) {
          MmaPostOp d{};
          d.nq = op.nq;
          d.q0 = op.q[0];
          d.q1 = op.nq > 1 ? op.q[1] : 0;
          d.diag = op.type == OP_DIAG ? 1 : 0;
          const size_t cnt = op.type == OP_DIAG ? (size_t)(1 << op.nq) : (size_t)(1 << (2 * op.nq));
          for (size_t i = 0; i < cnt && i < 16; ++i) d.m[i] = make_float2((float)op.m[i].real(), (float)op.m[i].imag());
          append(&d, sizeof d);
        }
      }
    align(256);
    sd.leaf_off = host.size();
    for (auto &z : sd.leaf_ops) {
      if (p.precision == HSF_PREC_C64) {
        float2 c = make_float2((float)z.real(), (float)z.imag());
        append(&c, sizeof c);
      } else {
        double2 c = make_double2(z.real(), z.imag());
        append(&c, sizeof c);
      }
    }
    if (!grad && p.leaf_pf >= 0) {
      align(256);
      sd.leaf_s_off = host.size();
      for (auto &z : sd.leaf_S) {
        float2 c = make_float2((float)z.real(), (float)z.imag());
        append(&c, sizeof c);
      }
    }
  }
  if (!grad && !p.leaf_H.empty()) {
    align(256);
    p.leaf_h_off = host.size();
    for (auto &z : p.leaf_H) {
      float2 c = make_float2((float)z.real(), (float)z.imag());
      append(&c, sizeof c);
    }
  }
  if (!grad && p.leaf_pf >= 0) {
    align(256);
    p.leaf_g_off = host.size();
    for (auto &z : p.leaf_G) {
      float2 c = make_float2((float)z.real(), (float)z.imag());
      append(&c, sizeof c);
    }
  }
  align(256);
  if (host.empty()) host.put(nullptr, 256, true);
  if (!host.ok) return set_error(HSF_ENOMEM, "page-locked staging of %zu bytes", host.size());
  void *&table = grad ? p.dev_gtable : p.dev_table;
  // from the table arena (no implicit stream synchronisation); hsf_plan_destroy waits
  // for the device before returning the block, so no queued kernel can still read it
  table = table_alloc(host.size());
  if (!table) return set_error(HSF_ENOMEM, "device table of %zu bytes", host.size());
  if (!grad) p.dev_table_bytes = host.size();
  CUDA_TRY(cudaMemcpyAsync(table, host.data(), host.size(), cudaMemcpyHostToDevice, plan_stream()));
  CUDA_TRY(cudaStreamSynchronize(plan_stream()));
  if (!grad) p.launches = launches / 2;
  return HSF_OK;
}

hsf_status finish_plan(hsf_plan &p) {
  const int B = (int)p.blocks.size();
  p.radix.assign(B + 1, 1);
  p.below.assign(B + 1, 1);
  long double paths = 1;
  for (int b = 0; b < B; ++b) {
    p.radix[b + 1] = (uint64_t)p.blocks[b].rank;
    paths *= p.blocks[b].rank;
  }
  if (paths > (long double)p.max_paths || paths > (long double)(1ull << 62))
    return set_error(HSF_ERANK, "%.0Lf paths exceed max_paths %llu", paths, (unsigned long long)p.max_paths);
  p.num_paths = (uint64_t)paths;
  for (int k = B - 1; k >= 0; --k) p.below[k] = p.below[k + 1] * p.radix[k + 1];
  int64_t nodes = 0;
  for (int k = 0; k <= B; ++k) nodes += (int64_t)(p.num_paths / p.below[k]);
  p.tree_nodes = nodes;
  hsf_status st = build_programs(p);
  if (st != HSF_OK) return st;
  st = upload_programs(p);
  if (st != HSF_OK) return st;
  p.dev_status = (int32_t *)table_alloc(256);
  if (!p.dev_status) return set_error(HSF_ENOMEM, "device status words");
  CUDA_TRY(cudaMemsetAsync(p.dev_status, 0, 256, plan_stream()));
  CUDA_TRY(cudaStreamSynchronize(plan_stream()));
  return HSF_OK;
}

hsf_status check_order(hsf_plan &p) {
  std::vector<std::pair<bool, int>> order;
  p.order.clear();
  hsf_status st = execution_order(p, order);
  if (st == HSF_OK) p.order = order;
  return st;
}

// Multiply and decompose blocks on the device (svd.cu); read back ranks and factors.
hsf_status run_svd_jobs(const hsf_plan &p, const std::vector<SvdJob> &jobs, std::vector<BlockH> &out) {
  const int J = (int)jobs.size();
  out.assign(J, BlockH{});
  if (J == 0) return HSF_OK;
  std::vector<int32_t> bk(3 * J), tbeg(J + 1, 0), gbeg(1, 0), gdesc;
  std::vector<double> gm;
  for (int j = 0; j < J; ++j) {
    const BlockH &blk = p.blocks[jobs[j].block];
    const int k = (int)blk.qubits.size();
    bk[3 * j] = k;
    bk[3 * j + 1] = (int)blk.qa.size();
    bk[3 * j + 2] = (int)blk.qb.size();
    for (const auto &term : jobs[j].terms) {
      for (int code : term) {
        const bool deriv = code < 0;
        const GateH &g = p.gates[deriv ? -1 - code : code];
        gdesc.push_back(g.nq);
        for (int x = 0; x < 3; ++x) {
          int pos = 0;
          if (x < g.nq) {
            const int idx = (int)(std::find(blk.qubits.begin(), blk.qubits.end(), g.q[x]) - blk.qubits.begin());
            pos = k - 1 - idx;      // block qubits are listed most significant first
          }
          gdesc.push_back(pos);
        }
        gdesc.push_back((int32_t)(gm.size() / 2));
        for (auto &z : (deriv ? g.dm : g.m)) {
          gm.push_back(z.real());
          gm.push_back(z.imag());
        }
      }
      gbeg.push_back((int32_t)(gdesc.size() / 5));
    }
    tbeg[j + 1] = (int32_t)(gbeg.size() - 1);
  }
  const size_t nf = (size_t)J * 64 * 64 * 2;
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t o = off; off += (bytes + 255) / 256 * 256; return o; };
  const size_t o_bk = take(bk.size() * 4), o_tb = take(tbeg.size() * 4), o_gb = take(gbeg.size() * 4),
               o_gd = take(gdesc.size() * 4 + 4), o_gm = take(gm.size() * 8 + 8), o_sig = take((size_t)J * 64 * 8),
               o_rank = take((size_t)J * 4), o_x = take(nf * 8), o_y = take(nf * 8), o_sw = take((size_t)J * 4),
               o_res = take((size_t)J * 8);
  cudaStream_t pst = plan_stream();
  unsigned char *d = nullptr;
  // scratch from the table arena; it is returned only after the stream sync below (or,
  // on an early error, after waiting for the plan stream)
  d = (unsigned char *)table_alloc(off);
  if (!d) return set_error(HSF_ENOMEM, "SVD scratch of %zu bytes", off);
  std::unique_ptr<unsigned char, void (*)(unsigned char *)> guard(d, [](unsigned char *q) {
    cudaStreamSynchronize(plan_stream());
    table_free(q);
  });
  CUDA_TRY(cudaMemcpyAsync(d + o_bk, bk.data(), bk.size() * 4, cudaMemcpyHostToDevice, pst));
  CUDA_TRY(cudaMemcpyAsync(d + o_tb, tbeg.data(), tbeg.size() * 4, cudaMemcpyHostToDevice, pst));
  CUDA_TRY(cudaMemcpyAsync(d + o_gb, gbeg.data(), gbeg.size() * 4, cudaMemcpyHostToDevice, pst));
  if (!gdesc.empty()) CUDA_TRY(cudaMemcpyAsync(d + o_gd, gdesc.data(), gdesc.size() * 4, cudaMemcpyHostToDevice, pst));
  if (!gm.empty()) CUDA_TRY(cudaMemcpyAsync(d + o_gm, gm.data(), gm.size() * 8, cudaMemcpyHostToDevice, pst));
  BlockSvdArgs a{};
  a.num_blocks = J;
  a.block_k = (const int32_t *)(d + o_bk);
  a.term_begin = (const int32_t *)(d + o_tb);
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
  a.residual = (double *)(d + o_res);
  {
    int dmax = 1, wmax = 1, nwmax = 1;
    for (int j = 0; j < J; ++j) {
      const int k = bk[3 * j], ka = bk[3 * j + 1], kb = bk[3 * j + 2];
      const int Mw = std::max(1 << (2 * ka), 1 << (2 * kb)), Nw = std::min(1 << (2 * ka), 1 << (2 * kb));
      dmax = std::max(dmax, 1 << k);
      wmax = std::max(wmax, Mw * Nw);
      nwmax = std::max(nwmax, Nw);
    }
    a.off_w = dmax * dmax;
    a.off_v = a.off_w + wmax;
    a.max_nw = nwmax;
  }
  CUDA_TRY(launch_block_svd(a, pst));
  g_launches++;
  std::vector<double> sig((size_t)J * 64);
  std::vector<int32_t> rank(J), sweeps(J);
  std::vector<double> resid(J);
  // the factors are read back only up to the widest factor row (4^|q_a| or 4^|q_b|
  // entries of the 64 the device layout reserves per term)
  int wx = 1, wy = 1;
  for (int j = 0; j < J; ++j) {
    wx = std::max(wx, 1 << (2 * bk[3 * j + 1]));
    wy = std::max(wy, 1 << (2 * bk[3 * j + 2]));
  }
  std::vector<double> xf((size_t)J * 64 * wx * 2), yf((size_t)J * 64 * wy * 2);
  CUDA_TRY(cudaMemcpyAsync(sweeps.data(), d + o_sw, sweeps.size() * 4, cudaMemcpyDeviceToHost, pst));
  CUDA_TRY(cudaMemcpyAsync(resid.data(), d + o_res, resid.size() * 8, cudaMemcpyDeviceToHost, pst));
  CUDA_TRY(cudaMemcpyAsync(sig.data(), d + o_sig, sig.size() * 8, cudaMemcpyDeviceToHost, pst));
  CUDA_TRY(cudaMemcpyAsync(rank.data(), d + o_rank, rank.size() * 4, cudaMemcpyDeviceToHost, pst));
  CUDA_TRY(cudaMemcpy2DAsync(xf.data(), (size_t)wx * 16, d + o_x, 64 * 16, (size_t)wx * 16, (size_t)J * 64,
                             cudaMemcpyDeviceToHost, pst));
  CUDA_TRY(cudaMemcpy2DAsync(yf.data(), (size_t)wy * 16, d + o_y, 64 * 16, (size_t)wy * 16, (size_t)J * 64,
                             cudaMemcpyDeviceToHost, pst));
  CUDA_TRY(cudaStreamSynchronize(pst));
  for (int j = 0; j < J; ++j) {
    BlockH &r = out[j];
    const BlockH &src = p.blocks[jobs[j].block];
    r.gates = src.gates;
    r.qubits = src.qubits;
    r.qa = src.qa;
    r.qb = src.qb;
    r.rank = rank[j];
    r.sigma.assign(sig.begin() + (size_t)j * 64, sig.begin() + (size_t)j * 64 + std::max(0, r.rank));
    for (double sv : r.sigma)
      if (!std::isfinite(sv)) return set_error(HSF_ENUMERIC, "block %d: non-finite singular value", jobs[j].block);
    // The Jacobi sweeps must have converged, and the kept terms must rebuild the block
    // matrix (eq. equ-schmidt-decompostion-res) up to FP64 round-off plus what the rank
    // threshold dropped (each dropped term has unit-norm factors, so it moves an entry by
    // at most its sigma).
    if (sweeps[j] >= a.max_sweeps)
      return set_error(HSF_ENUMERIC, "block %d: Jacobi SVD did not converge in %d sweeps", jobs[j].block,
                       a.max_sweeps);
    double dropped = 0.0;
    for (int m = std::max(0, r.rank); m < 64; ++m) dropped += sig[(size_t)j * 64 + m];
    const double s0 = r.rank > 0 ? r.sigma[0] : 0.0;
    const double res_tol = 1e-12 * std::max(1.0, s0) + dropped;
    if (!(resid[j] <= res_tol))
      return set_error(HSF_ENUMERIC, "block %d: Schmidt terms rebuild the block matrix only to %.3g (limit %.3g)",
                       jobs[j].block, resid[j], res_tol);
    r.residual = resid[j];
    r.sweeps = sweeps[j];
    const int ea = 1 << (2 * (int)r.qa.size()), eb = 1 << (2 * (int)r.qb.size());
    for (int m = 0; m < r.rank; ++m) {
      for (int e = 0; e < ea; ++e) {
        const size_t i = (((size_t)j * 64 + m) * wx + e) * 2;
        r.x.push_back(cd(xf[i], xf[i + 1]));
      }
      for (int e = 0; e < eb; ++e) {
        const size_t i = (((size_t)j * 64 + m) * wy + e) * 2;
        r.y.push_back(cd(yf[i], yf[i + 1]));
      }
    }
  }
  return HSF_OK;
}

// Closed-form Schmidt terms of cascade blocks (Sec. IV-D, Example 4: a cascade of gates
// that share one control-like qubit keeps rank 2, C_CNOT,3 = P0 (x) I + P1 (x) X X X).
// Generalised to a hub H = all block qubits of one side: when every gate that touches H
// is diagonal on H (block-diagonal in the H basis: CNOT with its control in H, CZ, RZZ,
// diagonal one-qubit gates), then for every hub basis state z the block acts on the
// other side as Y_z = prod_g <z|G_g|z>_H (circuit order, later gates on the left), so
// A = sum_z P_z (x) Y_z with P_z = |z><z| on H.  The P_z are orthogonal; when the Y_z are
// linearly independent there are exactly 2^{k_H} terms, the Schmidt rank.  A job with
// several terms (a derivative by the product rule) sums its terms' Y_z.
static cd m_entry(const GateH &g, int r, int c) { return g.m[(size_t)r * (1 << g.nq) + c]; }

bool closed_form_job(const hsf_plan &p, const SvdJob &job, bool need_independent, BlockH &out) {
  const BlockH &blk = p.blocks[job.block];
  for (int hub = 0; hub < 2; ++hub) {
    const std::vector<int> &H = hub == 0 ? blk.qa : blk.qb;     // descending: H[0] is the MSB of z
    const std::vector<int> &O = hub == 0 ? blk.qb : blk.qa;
    const int kh = (int)H.size(), ko = (int)O.size();
    if (kh == 0 || kh > 3 || ko == 0 || ko > kMaxCascadeLeaves) continue;
    auto hub_pos = [&](int q) {
      for (int i = 0; i < kh; ++i)
        if (H[i] == q) return kh - 1 - i;
      return -1;
    };
    auto other_pos = [&](int q) {
      for (int i = 0; i < ko; ++i)
        if (O[i] == q) return ko - 1 - i;
      return -1;
    };
    bool ok = true;
    for (const auto &term : job.terms) {
      for (int code : term) {
        const GateH &g = p.gates[code < 0 ? -1 - code : code];
        const std::vector<cd> &m = code < 0 ? g.dm : g.m;
        int hmask = 0;                         // matrix-index bits that are hub qubits
        for (int x = 0; x < g.nq; ++x)
          if (hub_pos(g.q[x]) >= 0) hmask |= 1 << (g.nq - 1 - x);
        if (!hmask) continue;
        const int d = 1 << g.nq;
        for (int r = 0; r < d && ok; ++r)
          for (int c = 0; c < d; ++c)
            if (((r ^ c) & hmask) && m[(size_t)r * d + c] != cd(0.0)) {
              ok = false;
              break;
            }
      }
      if (!ok) break;
    }
    if (!ok) continue;
    const int dz = 1 << kh, dob = 1 << ko;
    std::vector<std::vector<cd>> Y(dz, std::vector<cd>((size_t)dob * dob, 0.0));
    std::vector<cd> T((size_t)dob * dob), col(dob);
    for (int z = 0; z < dz; ++z) {
      for (const auto &term : job.terms) {
        std::fill(T.begin(), T.end(), cd(0.0));
        for (int i = 0; i < dob; ++i) T[(size_t)i * dob + i] = 1.0;
        for (int code : term) {
          const GateH &g = p.gates[code < 0 ? -1 - code : code];
          const std::vector<cd> &m = code < 0 ? g.dm : g.m;
          const int d = 1 << g.nq;
          // the gate's matrix restricted to hub state z: its other operands vary
          int fixed = 0, nv = 0, vbit[3] = {0, 0, 0};
          OpH op;
          op.type = OP_DENSE;
          for (int x = 0; x < g.nq; ++x) {
            const int hp = hub_pos(g.q[x]);
            if (hp >= 0) {
              if ((z >> hp) & 1) fixed |= 1 << (g.nq - 1 - x);
            } else {
              vbit[nv] = g.nq - 1 - x;
              op.q[nv] = other_pos(g.q[x]);
              ++nv;
            }
          }
          op.nq = nv;
          const int dv = 1 << nv;
          auto full_index = [&](int v) {
            int i = fixed;
            for (int j = 0; j < nv; ++j)
              if ((v >> (nv - 1 - j)) & 1) i |= 1 << vbit[j];
            return i;
          };
          if (nv == 0) {
            const cd sc = m[(size_t)fixed * d + fixed];
            for (auto &e : T) e *= sc;
            continue;
          }
          op.m.resize((size_t)dv * dv);
          for (int r = 0; r < dv; ++r)
            for (int c = 0; c < dv; ++c) op.m[(size_t)r * dv + c] = m[(size_t)full_index(r) * d + full_index(c)];
          for (int c = 0; c < dob; ++c) {
            for (int r = 0; r < dob; ++r) col[r] = T[(size_t)r * dob + c];
            host_apply(col, ko, op, 0);
            for (int r = 0; r < dob; ++r) T[(size_t)r * dob + c] = col[r];
          }
        }
        for (size_t e = 0; e < T.size(); ++e) Y[z][e] += T[e];
      }
    }
    // norms, and linear independence by Gram-Schmidt on the vectorised Y_z
    std::vector<double> nrm(dz, 0.0);
    for (int z = 0; z < dz; ++z) {
      for (const cd &e : Y[z]) nrm[z] += std::norm(e);
      nrm[z] = std::sqrt(nrm[z]);
    }
    double nmax = 0.0;
    for (double v : nrm) nmax = std::max(nmax, v);
    if (need_independent) {
      if (!(nmax > 0.0)) continue;
      std::vector<std::vector<cd>> basis;
      bool indep = true;
      for (int z = 0; z < dz && indep; ++z) {
        std::vector<cd> v = Y[z];
        for (const auto &u : basis) {
          cd dot = 0.0;
          for (size_t e = 0; e < v.size(); ++e) dot += std::conj(u[e]) * v[e];
          for (size_t e = 0; e < v.size(); ++e) v[e] -= dot * u[e];
        }
        double r = 0.0;
        for (const cd &e : v) r += std::norm(e);
        r = std::sqrt(r);
        if (!(r > 1e-10 * std::max(nrm[z], 1e-300)) || !(nrm[z] > 1e-12 * nmax)) indep = false;
        for (auto &e : v) e /= r;
        basis.push_back(v);
      }
      if (!indep) continue;
    }
    out = BlockH{};
    out.gates = blk.gates;
    out.qubits = blk.qubits;
    out.qa = blk.qa;
    out.qb = blk.qb;
    out.closed = hub;
    const int ka = (int)blk.qa.size(), kb = (int)blk.qb.size();
    if (ko > 3) {
      // more than 3 qubits on the other side: no dense factor; the factor of side O is the
      // block's gates restricted to the hub state (one small op per gate, a matrix per
      // digit), and the hub side's factor is the projector (with the hub-only phases and
      // the balancing scale folded in)
      if (job.terms.size() != 1 || !need_independent) return false;
      std::vector<cd> hub_scale(dz, 1.0);
      for (int z = 0; z < dz; ++z) hub_scale[z] = std::sqrt(nrm[z]);
      bool first_o = true;
      for (int code : job.terms[0]) {
        const GateH &g = p.gates[code];
        const int d = 1 << g.nq;
        int nv = 0, vbit[3] = {0, 0, 0}, vq[3] = {0, 0, 0};
        for (int x = 0; x < g.nq; ++x)
          if (hub_pos(g.q[x]) < 0) {
            vbit[nv] = g.nq - 1 - x;
            vq[nv] = g.q[x];
            ++nv;
          }
        const int dv = 1 << nv;
        OpH op;
        op.nq = nv;
        for (int j = 0; j < nv; ++j) op.q[j] = vq[j];
        op.digits = dz;
        op.block = job.block;
        std::vector<cd> mats;
        bool diag = true;
        for (int z = 0; z < dz; ++z) {
          int fixed = 0;
          for (int x = 0; x < g.nq; ++x) {
            const int hp = hub_pos(g.q[x]);
            if (hp >= 0 && ((z >> hp) & 1)) fixed |= 1 << (g.nq - 1 - x);
          }
          auto full_index = [&](int v) {
            int i = fixed;
            for (int j = 0; j < nv; ++j)
              if ((v >> (nv - 1 - j)) & 1) i |= 1 << vbit[j];
            return i;
          };
          if (nv == 0) {
            hub_scale[z] *= m_entry(g, fixed, fixed);
            continue;
          }
          const double inv = first_o ? 1.0 / std::sqrt(nrm[z]) : 1.0;
          for (int r = 0; r < dv; ++r)
            for (int c = 0; c < dv; ++c) {
              const cd v = g.m[(size_t)full_index(r) * d + full_index(c)] * inv;
              if (r != c && v != cd(0.0)) diag = false;
              mats.push_back(v);
            }
        }
        if (nv == 0) continue;
        first_o = false;
        if (diag) {
          op.type = OP_DIAG;
          for (int z = 0; z < dz; ++z)
            for (int r = 0; r < dv; ++r) op.m.push_back(mats[(size_t)z * dv * dv + (size_t)r * dv + r]);
        } else {
          op.type = OP_DENSE;
          op.m = mats;
        }
        out.fops[1 - hub].push_back(op);
      }
      OpH hop;
      hop.type = OP_DIAG;
      hop.nq = kh;
      for (int j = 0; j < kh; ++j) hop.q[j] = H[j];
      hop.digits = dz;
      hop.block = job.block;
      for (int z = 0; z < dz; ++z)
        for (int e = 0; e < dz; ++e) hop.m.push_back(e == z ? hub_scale[z] : cd(0.0));
      out.fops[hub].push_back(hop);
      for (int z = 0; z < dz; ++z) out.sigma.push_back(nrm[z]);
      out.rank = dz;
      return true;
    }
    const int ea = 1 << (2 * ka), eb = 1 << (2 * kb);
    for (int z = 0; z < dz; ++z) {
      if (!(nrm[z] > 1e-300) || (!need_independent && !(nrm[z] > 1e-14 * nmax))) continue;   // a zero term
      // balanced magnitudes, as the SVD's sqrt(sigma) folding: |X'|_F = |Y'|_F
      const double c = std::sqrt(nrm[z]);
      std::vector<cd> proj((size_t)dz * dz, 0.0);
      proj[(size_t)z * dz + z] = c;
      std::vector<cd> oth(Y[z]);
      for (auto &e : oth) e /= c;
      const std::vector<cd> &xa = hub == 0 ? proj : oth, &yb = hub == 0 ? oth : proj;
      if ((int)xa.size() != ea || (int)yb.size() != eb) return false;
      out.x.insert(out.x.end(), xa.begin(), xa.end());
      out.y.insert(out.y.end(), yb.begin(), yb.end());
      out.sigma.push_back(nrm[z]);      // |P_z|_F |Y_z|_F
      ++out.rank;
    }
    return true;
  }
  return false;
}

hsf_status decompose_blocks(hsf_plan &p) {
  const int B = (int)p.blocks.size();
  std::vector<SvdJob> jobs;
  std::vector<int> svd_of;
  std::vector<BlockH> res(B);
  std::vector<char> done(B, 0);
  for (int b = 0; b < B; ++b) {
    SvdJob job;
    job.block = b;
    job.terms = {p.blocks[b].gates};
    if (!(p.flags & HSF_FLAG_SVD_BLOCKS) && closed_form_job(p, job, true, res[b])) {
      done[b] = 1;
      continue;
    }
    if (p.blocks[b].qa.size() > 3 || p.blocks[b].qb.size() > 3)
      return set_error(HSF_ERANK, "block %d spans %zu|%zu qubits: the SVD takes at most 3 per side (only a cascade, "
                                  "diagonal on one side's block qubits, may have more)", b, p.blocks[b].qa.size(),
                       p.blocks[b].qb.size());
    jobs.push_back(job);
    svd_of.push_back(b);
  }
  std::vector<BlockH> sres;
  hsf_status st = run_svd_jobs(p, jobs, sres);
  if (st != HSF_OK) return st;
  for (size_t j = 0; j < jobs.size(); ++j) res[svd_of[j]] = sres[j];
  for (int b = 0; b < B; ++b) {
    if (res[b].rank <= 0) return set_error(HSF_ENUMERIC, "block %d decomposed to rank 0", b);
    p.blocks[b] = res[b];
  }
  return HSF_OK;
}

// Gate list of the circuit: matrices (named kinds from their definitions, explicit ones
// copied and checked finite), rotation derivatives, qubit checks and the side of every
// gate for the cut p.cut (set by the caller).
hsf_status load_gates(hsf_plan &p, const hsf_circuit *c, const hsf_plan_opts *o) {
  p.gates.resize(c->num_gates);
  for (int i = 0; i < c->num_gates; ++i) {
    const hsf_gate &g = c->gates[i];
    GateH &h = p.gates[i];
    h.kind = g.kind;
    h.param = g.param;
    h.param_id = g.param_id;
    if (g.param_id >= 0 && o && o->angles) {
      if (g.param_id >= o->num_angles) return set_error(HSF_EINVAL, "gate %d: param_id %d >= num_angles", i, g.param_id);
      h.param = o->angles[g.param_id];
    }
    int nq = 0;
    if (g.kind == HSF_GATE_MATRIX) {
      nq = g.nq;
      if (nq < 1 || nq > 3) return set_error(HSF_EINVAL, "gate %d: matrix gates take 1..3 qubits", i);
      if (!g.mat) return set_error(HSF_EINVAL, "gate %d: matrix pointer is NULL", i);
      const int d = 1 << nq;
      h.m.resize((size_t)d * d);
      for (int e = 0; e < d * d; ++e) h.m[e] = cd(g.mat[2 * e], g.mat[2 * e + 1]);
      for (auto &z : h.m)
        if (!std::isfinite(z.real()) || !std::isfinite(z.imag()))
          return set_error(HSF_EINVAL, "gate %d: non-finite matrix", i);
    } else {
      hsf_status st = named_matrix(g.kind, h.param, h.m, nq);
      if (st != HSF_OK) return st;
      if (g.nq != nq) return set_error(HSF_EINVAL, "gate %d: kind %d takes %d qubits, got %d", i, g.kind, nq, g.nq);
    }
    h.nq = nq;
    if (g.kind == HSF_GATE_RX || g.kind == HSF_GATE_RY || g.kind == HSF_GATE_RZ || g.kind == HSF_GATE_RZZ) {
      // G = exp(-i t P / 2): K = dG/dt G^-1 = -i/2 P and dG/dt = K G
      const int d = 1 << nq;
      std::vector<cd> P((size_t)d * d, 0.0);
      const cd I(0.0, 1.0);
      if (g.kind == HSF_GATE_RX) P = {0.0, 1.0, 1.0, 0.0};
      if (g.kind == HSF_GATE_RY) P = {0.0, -I, I, 0.0};
      if (g.kind == HSF_GATE_RZ) P = {1.0, 0.0, 0.0, -1.0};
      if (g.kind == HSF_GATE_RZZ) { P[0] = 1.0; P[5] = -1.0; P[10] = -1.0; P[15] = 1.0; }
      h.k.resize(P.size());
      for (size_t e = 0; e < P.size(); ++e) h.k[e] = cd(0.0, -0.5) * P[e];
      h.dm = matmul(h.k, h.m, d);
      if (g.param_id >= 0) p.num_params = std::max(p.num_params, g.param_id + 1);
    }
    for (int j = 0; j < nq; ++j) {
      h.q[j] = g.q[j];
      if (g.q[j] < 0 || g.q[j] >= c->n) return set_error(HSF_EINVAL, "gate %d: qubit %d out of range", i, g.q[j]);
      for (int k = 0; k < j; ++k)
        if (g.q[k] == g.q[j]) return set_error(HSF_EINVAL, "gate %d: repeated qubit %d", i, g.q[j]);
    }
    h.diag = is_diagonal(h.m, 1 << nq);
    bool hi = false, lo = false;
    for (int j = 0; j < nq; ++j) (h.q[j] > p.cut ? hi : lo) = true;
    h.side = (hi && lo) ? 2 : (hi ? 0 : 1);
  }
  return HSF_OK;
}

hsf_status validate_and_load(hsf_plan &p, const hsf_circuit *c, int cut, const hsf_blocks *bl,
                             const hsf_plan_opts *o) {
  if (!c || !bl) return set_error(HSF_EINVAL, "circuit and blocks must not be NULL");
  if (c->n < 2 || c->n > 62) return set_error(HSF_EINVAL, "n = %d outside 2..62", c->n);
  if (cut < 0 || cut > c->n - 2) return set_error(HSF_EINVAL, "cut %d outside 0..n-2", cut);
  if (c->num_gates < 0 || (c->num_gates > 0 && !c->gates)) return set_error(HSF_EINVAL, "bad gate array");
  p.n = c->n;
  p.cut = cut;
  p.nb = cut + 1;
  p.na = c->n - cut - 1;
  p.max_paths = 1ull << 40;
  if (o) {
    p.precision = o->precision;
    p.gemm_mode = o->gemm_mode;
    p.rank_tol = o->rank_tol > 0 ? o->rank_tol : 1e-12;
    if (o->max_paths) p.max_paths = o->max_paths;
    p.flags = o->flags;
  }
  if (p.precision != HSF_PREC_C64 && p.precision != HSF_PREC_C128)
    return set_error(HSF_EINVAL, "precision %d", p.precision);
  if (p.gemm_mode < 0 || p.gemm_mode > 3) return set_error(HSF_EINVAL, "gemm_mode %d", p.gemm_mode);
  if (p.gemm_mode != HSF_GEMM_FP32 && p.precision != HSF_PREC_C64)
    return set_error(HSF_EINVAL, "tensor-core path GEMM modes take complex64 half states");
  // a shared-memory tile holds at most 2^13 (complex64) or 2^12 (complex128) amplitudes
  const int tcap = p.precision == HSF_PREC_C64 ? kRegTileC64 : kRegTileC128;
  p.tile_max = (o && o->tile_bits) ? o->tile_bits : tcap;
  if (p.tile_max < 3 || p.tile_max > tcap) return set_error(HSF_EINVAL, "tile_bits %d outside 3..%d", p.tile_max, tcap);
  if (p.na > 40 || p.nb > 40) return set_error(HSF_EINVAL, "half of %d/%d qubits is too large", p.na, p.nb);
  hsf_status gst = load_gates(p, c, o);
  if (gst != HSF_OK) return gst;
  if (bl->num_blocks < 0 || bl->num_blocks > 64)
    return set_error(HSF_EINVAL, "num_blocks %d outside 0..64", bl->num_blocks);
  if (bl->num_blocks > 0 && (!bl->offsets || !bl->gate_idx)) return set_error(HSF_EINVAL, "bad block arrays");
  std::vector<int> owner(c->num_gates, -1);
  p.blocks.resize(bl->num_blocks);
  for (int b = 0; b < bl->num_blocks; ++b) {
    const int lo = bl->offsets[b], hi = bl->offsets[b + 1];
    if (lo < 0 || hi < lo) return set_error(HSF_EINVAL, "block %d: bad offsets", b);
    if (hi == lo) return set_error(HSF_EBLOCK, "block %d is empty", b);
    BlockH &blk = p.blocks[b];
    std::set<int> qs;
    bool crossing = false;
    for (int e = lo; e < hi; ++e) {
      const int gi = bl->gate_idx[e];
      if (gi < 0 || gi >= c->num_gates) return set_error(HSF_EINVAL, "block %d: gate index %d out of range", b, gi);
      if (owner[gi] >= 0) return set_error(HSF_EBLOCK, "gate %d is in blocks %d and %d", gi, owner[gi], b);
      owner[gi] = b;
      blk.gates.push_back(gi);
      for (int j = 0; j < p.gates[gi].nq; ++j) qs.insert(p.gates[gi].q[j]);
      crossing |= p.gates[gi].side == 2;
    }
    if (!crossing) return set_error(HSF_EBLOCK, "block %d holds no gate crossing the cut", b);
    std::sort(blk.gates.begin(), blk.gates.end());
    blk.qubits.assign(qs.rbegin(), qs.rend());
    for (int q : blk.qubits) (q > cut ? blk.qa : blk.qb).push_back(q);
    if (std::min(blk.qa.size(), blk.qb.size()) > 3 || std::max(blk.qa.size(), blk.qb.size()) > (size_t)kMaxCascadeLeaves)
      return set_error(HSF_ERANK, "block %d spans %zu|%zu qubits; at most 3 on one side and %d on the other", b,
                       blk.qa.size(), blk.qb.size(), kMaxCascadeLeaves);
  }
  for (int i = 0; i < c->num_gates; ++i)
    if (p.gates[i].side == 2 && owner[i] < 0)
      return set_error(HSF_EBLOCK, "gate %d crosses the cut but is in no block", i);
  return HSF_OK;
}

}  // namespace hsf
