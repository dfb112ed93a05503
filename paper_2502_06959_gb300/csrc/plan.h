// Host-side plan of a joint-cut HSF simulation (internal).
#pragma once

#include <atomic>
#include <complex>
#include <memory>
#include <utility>
#include <cstdint>
#include <string>
#include <functional>
#include <vector>

#include "../../include/hsf.h"
#include "common.h"

namespace hsf {

using cd = std::complex<double>;

// A cascade block (closed-form terms) may hold up to this many qubits on its non-hub side.
constexpr int kMaxCascadeLeaves = 8;

// Allocator whose default construction leaves trivial elements uninitialised (a vector
// resized with it is not zero-filled first: for buffers that are written in full).
template <typename T>
struct NoInitAlloc : std::allocator<T> {
  template <typename U>
  struct rebind {
    using other = NoInitAlloc<U>;
  };
  NoInitAlloc() = default;
  template <typename U>
  NoInitAlloc(const NoInitAlloc<U> &) noexcept {}
  template <typename U>
  void construct(U *p) noexcept {
    ::new (static_cast<void *>(p)) U;
  }
  template <typename U, typename... Args>
  void construct(U *p, Args &&...args) {
    ::new (static_cast<void *>(p)) U(std::forward<Args>(args)...);
  }
};

struct GateH {
  int kind = 0;
  int nq = 0;
  int q[4] = {0, 0, 0, 0};
  double param = 0.0;
  int param_id = -1;
  std::vector<cd> m;       // 2^nq x 2^nq, row-major
  std::vector<cd> dm;      // rotations: dG/dtheta, 2^nq x 2^nq
  std::vector<cd> k;       // rotations: K = (dG/dtheta) G^-1 = -i/2 P, 2^nq x 2^nq
  bool diag = false;
  int side = 0;            // 0 = a (all qubits > l), 1 = b (all <= l), 2 = crossing
};

// One op of a side program, on side-local logical qubits (q[0] = matrix MSB).
struct OpH {
  int type = OP_DENSE;
  int nq = 0;
  int q[3] = {0, 0, 0};
  std::vector<cd> m;       // dense: 4^nq per digit; diag: 2^nq per digit
  int digits = 1;          // > 1: Schmidt factor, matrices for every digit
  int block = -1;
  int param = -1;          // gradient programs: angle index of an unfused rotation
  std::vector<cd> k;       // its K = (dG/dtheta) G^-1 (same form as m: dense or diagonal)
};

struct BlockH {
  std::vector<int> gates;  // circuit order
  std::vector<int> qubits; // descending: a-qubits first
  std::vector<int> qa, qb; // descending
  int rank = 0;
  std::vector<double> sigma;
  std::vector<cd> x, y;    // rank x 4^ka and rank x 4^kb, sqrt(sigma) folded in
  double residual = 0.0;   // max entry of |U_B - sum_m X_m (x) Y_m| (device FP64)
  int sweeps = 0;          // Jacobi sweeps used
  int closed = -1;         // >= 0: closed-form cascade terms with the hub on side 0 (a)
                           // or 1 (b): X_m / Y_m = projector on hub state m (no SVD)
  // closed-form blocks with more than 3 qubits on a side: each side's factor as a list of
  // small ops (global qubits, `rank` digits each) instead of one dense op in x / y
  std::vector<OpH> fops[2];
};

struct GroupH {
  int slots[kMaxSlots] = {-1, -1, -1, -1, -1};   // tile bits held in registers, ascending; -1 unused
  int first_op = 0, num_ops = 0;
};

struct PassH {
  uint64_t active = 0;     // storage bits in the tile
  int t = 0;
  std::vector<OpH> ops;    // storage-bit operands, in application order
  std::vector<GroupH> groups;   // register groups (register-resident kernel), may be empty
  // device
  size_t ops_off = 0, mats_off = 0, groups_off = 0;   // byte offsets in the device table
  size_t table_end = 0;                                // end of this pass's block
  int num_ops = 0;
};

struct LevelH {
  std::vector<OpH> ops;
  std::vector<PassH> passes;
  // Tensor-core level (complex64, whole program on the kMmaBits lowest storage bits):
  // per digit, the program as a real 2^(kMmaBits+1)-square matrix W, stored as the
  // image the kernel loads (per digit TF32 hi then lo part when ops follow the product,
  // else per digit FP16 hi then lo part, then the inverse scales).
  bool mma = false;
  std::vector<float, NoInitAlloc<float>> wimg;   // every entry is written by the composition
  size_t w_off = 0;
  // candidate: the first mma_prefix ops act on the kMmaBits lowest storage bits (the
  // whole program when mma_prefix == ops.size()); once chosen, those ops are composed
  // into W and removed from ops, and the rest run as in-place passes after the product
  size_t mma_prefix = 0;
  // ops after the product that stay on storage bits < kMmaPostBits: applied by the
  // product's epilogue instead of as a pass
  std::vector<OpH> post;
  size_t post_off = 0;
};

struct SideH {
  int h = 0;
  int offset = 0;          // global qubit of local qubit 0
  std::vector<int> store;  // storage bit of every local qubit
  std::vector<LevelH> levels;   // 0 .. B
  // leaf contraction: the last level's program as r operators on the 2^leaf_c lowest
  // storage bits (padded to the plan-wide leaf_c)
  std::vector<cd> leaf_ops;     // r x 2^c x 2^c
  size_t leaf_off = 0;
  std::vector<OpH> leaf_pre;    // the leaf level's ops before fusion (storage bits)
  std::vector<cd> leaf_S;       // factored leaf: L_m = S (F_m (x) I), S as 2^c x 2^c
  size_t leaf_s_off = 0;
};

}  // namespace hsf

namespace hsf {
// planner.cpp
cudaStream_t plan_stream();   // the calling thread's private non-blocking stream for plan work
cudaStream_t side_stream();   // the calling thread's second stream for side b of hsf_run
hsf_status set_error(hsf_status code, const char *fmt, ...);
// Plan-table device memory from a per-device arena (no cudaMalloc on the common path).
// table_free returns a block at once: the caller makes sure no kernel still reads it.
// Page-locked host staging buffer (planner.cpp): taken for one upload, given back after
// its copy has completed.
struct StagingBuf {
  unsigned char *p = nullptr;
  size_t size = 0, cap = 0;
};
StagingBuf staging_take();
void staging_give(StagingBuf s);
bool staging_reserve(StagingBuf &s, size_t need);
// fn(0..n-1) on a persistent pool of host threads and the caller (planner.cpp).
void host_parallel_for(size_t n, const std::function<void(size_t)> &fn);
void *table_alloc(size_t bytes);
void table_free(void *p);
const char *last_error();
hsf_status validate_and_load(hsf_plan &p, const hsf_circuit *c, int cut, const hsf_blocks *bl,
                             const hsf_plan_opts *o);
hsf_status check_order(hsf_plan &p);
hsf_status load_gates(hsf_plan &p, const hsf_circuit *c, const hsf_plan_opts *o);
// Full-state (Schroedinger) plan: one program of all gates on h = n qubits.
hsf_status build_schrodinger(hsf_plan &p, const hsf_circuit *c, const hsf_plan_opts *o);
hsf_status decompose_blocks(hsf_plan &p);
hsf_status build_programs(hsf_plan &p, bool grad = false);
hsf_status upload_programs(hsf_plan &p, bool grad = false);
// One Schmidt decomposition job: the matrix is the sum over `terms` of the product of
// each term's gates (gate indices of the plan; a negative index -1-g uses gate g's
// derivative dG/dtheta instead of G).  Results go to `out` (rank, sigma, x, y).
struct SvdJob {
  int block;
  std::vector<std::vector<int>> terms;
};
hsf_status run_svd_jobs(const hsf_plan &p, const std::vector<SvdJob> &jobs, std::vector<BlockH> &out);
// Closed-form decomposition of a job whose gates, where they touch one side's block qubits
// (the hub), are all diagonal on them: A = sum_z P_z (x) Y_z.  With need_independent the
// Y_z must be linearly independent (then 2^{k_hub} is the Schmidt rank); otherwise zero
// terms are dropped.  Returns false when the block has no such structure.
bool closed_form_job(const hsf_plan &p, const SvdJob &job, bool need_independent, BlockH &out);
// Path counts, gate programs, device tables and the status word of a decomposed plan.
hsf_status finish_plan(hsf_plan &p);
extern std::atomic<uint64_t> g_launches;
}  // namespace hsf

struct hsf_plan {
  int n = 0, cut = 0, na = 0, nb = 0;
  int precision = 0, gemm_mode = 0, flags = 0, tile_max = 14;
  bool schrodinger = false;         // full-state plan (hsf_plan_create_schrodinger)
  double rank_tol = 1e-12;
  uint64_t max_paths = 0;
  std::vector<hsf::GateH> gates;
  std::vector<hsf::BlockH> blocks;
  std::vector<uint64_t> radix;      // radix[k] = rank of level k (radix[0] = 1), k = 0..B
  std::vector<uint64_t> below;      // below[k] = product of radix[k+1..B] (subtree leaves)
  uint64_t num_paths = 1;
  hsf::SideH side[2];               // 0 = a, 1 = b
  hsf::SideH gside[2];              // gradient programs (rotations kept unfused)
  bool grad_ready = false;
  int num_params = 0;               // 1 + largest param_id of the circuit
  void *dev_table = nullptr;        // ops + matrices of every pass
  int32_t *dev_status = nullptr;    // set by kernels whose bounded waits expired
  void *dev_gtable = nullptr;       // gradient programs (built on first hsf_grad)
  size_t dev_table_bytes = 0;
  int64_t tree_nodes = 0;
  int64_t launches = 0;
  int leaf_c = 0;                   // > 0: the leaf level can be contracted at bitstrings
  std::vector<std::pair<bool, int>> order;   // execution order (block?, index), set by check_order
  int leaf_pf = -1;                 // >= 0: factored leaf, the factor's storage bit in the chunk
  std::vector<hsf::cd> leaf_G;      // [(r+1)][(r+1)][4][4]: sum over digits [m0, m1) of F^a (x) F^b
  std::vector<hsf::cd> leaf_H;      // leaf chunks of 2 or 4 amplitudes: [(r+1)][(r+1)][D^2][D][D], H over digits [m0, m1)
  size_t leaf_h_off = 0;
  size_t leaf_g_off = 0;
  int rbits = 4;                    // register slots of the register-resident sweep
  struct ProfRec { int kind; cudaEvent_t e0, e1; double bytes, flops; };
  std::vector<ProfRec> prof;
  // gradients: derivative plans of blocks whose gates carry angles
  struct DerivPlan { int block, param; hsf_plan *plan; };
  std::vector<DerivPlan> dplans;
  void *dev_factors = nullptr;      // Schmidt factors of every level (gradient pullback)
  std::vector<size_t> factor_off[2];// byte offset of level k's factors (k >= 1)
  // workspace owned by the plan (hsf_run with workspace == NULL) and the allocator that
  // made it (release == NULL: cudaMalloc / cudaFree)
  void *own_ws = nullptr;
  size_t own_ws_bytes = 0;
  hsf_free_fn own_release = nullptr;
  void *own_ctx = nullptr;

  hsf_plan() = default;
  hsf_plan(const hsf_plan &) = delete;
  hsf_plan &operator=(const hsf_plan &) = delete;
  ~hsf_plan() {
    for (auto &r : prof) { cudaEventDestroy(r.e0); cudaEventDestroy(r.e1); }
    for (auto &d : dplans) delete d.plan;
    // every kernel that may read the plan's tables has finished before they are reused
    if (dev_table || dev_gtable || dev_status || dev_factors) cudaDeviceSynchronize();
    hsf::table_free(dev_table);
    hsf::table_free(dev_gtable);
    hsf::table_free(dev_status);
    hsf::table_free(dev_factors);
    if (own_ws) {
      cudaDeviceSynchronize();          // no queued run may still use it
      if (own_release) own_release(own_ctx, own_ws, nullptr);
      else cudaFree(own_ws);
    }
  }
};
