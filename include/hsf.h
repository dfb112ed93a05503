/*
 * hsf.h -- C ABI of a GB300 (sm_103a) library for joint-cutting Hybrid
 * Schroedinger-Feynman (HSF) simulation of quantum circuits.
 *
 * Method (Herzog, Burgholzer, Ufrecht, Scherer, Wille, "Joint Cutting for Hybrid
 * Schroedinger-Feynman Simulation of Quantum Circuits"):
 *   - Sec. II-B: the qubits are split horizontally after qubit l; half a holds
 *     qubits l+1..n-1 (the left / most significant Kronecker factor), half b holds
 *     qubits 0..l.
 *   - Sec. III-A / IV-A: the gates crossing the cut are grouped into blocks; each
 *     block unitary A is multiplied out and Schmidt-decomposed,
 *     A = sum_m sigma_m X_m (x) Y_m (eq. equ-schmidt-decompostion-res), via the SVD
 *     of the relabelled matrix A~_{(i^b j^b),(i^a j^a)} (eq. eq-svd).
 *   - Sec. II-B: a path chooses one Schmidt term per block; for each path both
 *     half circuits are simulated from |0...0> and the amplitudes are the sum over
 *     paths of the products psi_a^p(x_a) psi_b^p(x_b) ("Kronecker product ... and
 *     adding up all contributions").
 *
 * Conventions (Sec. II-A): bit q of a basis index / bitstring is qubit q; the
 * amplitude index is x = x_a * 2^{n_b} + x_b.  A gate on the ordered qubits
 * (q[0], q[1], ...) has its matrix index in Kronecker order with q[0] the most
 * significant factor (CNOT with the control listed first is P0 (x) I + P1 (x) X,
 * Example 2).  Rotations: RX/RY/RZ(t) = exp(-i t P/2), RZZ(t) = exp(-i t Z(x)Z/2).
 *
 * Paths are numbered in mixed radix over the blocks in the order they are listed
 * (block 0 is the most significant digit).  The listed order must be compatible with
 * the circuit's dependencies (a block that depends on another is listed after it).
 *
 * Errors: every entry point returns an hsf_status; nothing is thrown across the
 * ABI.  hsf_last_error() returns a human-readable message for the calling thread's
 * last failure.  All device work is ordered on the caller's stream; only hsf_plan
 * synchronises (it reads back the Schmidt ranks).
 */
#ifndef HSF_H
#define HSF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum hsf_status {
  HSF_OK = 0,
  HSF_EINVAL = 1,    /* bad argument: gate, qubit, cut, size, pointer, mode      */
  HSF_EBLOCK = 2,    /* crossing gate not in exactly one block, non-convex block,
                        block without a crossing gate, or blocks listed out of
                        dependency order                                          */
  HSF_ERANK = 3,     /* path count above max_paths / 2^62, block too large         */
  HSF_ENOMEM = 4,    /* workspace too small or host allocation failed            */
  HSF_ECUDA = 5,     /* a CUDA runtime call failed (message has the CUDA error)   */
  HSF_ETIMEOUT = 6,  /* a bounded device-side wait expired                       */
  HSF_ENUMERIC = 7,  /* NaN / Inf detected                                       */
  HSF_ENOTSUP = 8    /* combination not supported by this build                  */
} hsf_status;

typedef enum hsf_gate_kind {
  HSF_GATE_MATRIX = 0, /* explicit 2^nq x 2^nq unitary in `mat`, nq in 1..3        */
  HSF_GATE_H = 1, HSF_GATE_X = 2, HSF_GATE_Y = 3, HSF_GATE_Z = 4,
  HSF_GATE_S = 5, HSF_GATE_T = 6,
  HSF_GATE_RX = 7, HSF_GATE_RY = 8, HSF_GATE_RZ = 9,
  HSF_GATE_CX = 10, HSF_GATE_CZ = 11, HSF_GATE_SWAP = 12, HSF_GATE_ISWAP = 13,
  HSF_GATE_RZZ = 14
} hsf_gate_kind;

/* One gate.  `mat` (HSF_GATE_MATRIX only) points to host memory holding the
 * 2^nq x 2^nq complex128 matrix, row-major, re/im interleaved; it is copied by
 * hsf_plan.  `param_id` >= 0 ties the angle to entry param_id of a shared angle
 * vector (gradients, angle overrides); -1 keeps `param`. */
typedef struct hsf_gate {
  int32_t kind;
  int32_t nq;
  int32_t q[4];
  double param;
  int32_t param_id;
  int32_t reserved;
  const double *mat;
} hsf_gate;

typedef struct hsf_circuit {
  int32_t n;              /* qubits, 2..62                                        */
  int32_t num_gates;
  const hsf_gate *gates;  /* host array of num_gates gates, in circuit order       */
} hsf_circuit;

/* Blocks in CSR form: block k holds gate indices gate_idx[offsets[k] .. offsets[k+1]).
 * Every gate crossing the cut must be in exactly one block; a block may also hold
 * gates of one side (they are multiplied into the block).  Singleton blocks give
 * the standard per-gate cut. */
typedef struct hsf_blocks {
  int32_t num_blocks;
  const int32_t *offsets;   /* num_blocks + 1 entries, host memory */
  const int32_t *gate_idx;  /* host memory                         */
} hsf_blocks;

typedef enum hsf_precision { HSF_PREC_C64 = 0, HSF_PREC_C128 = 1 } hsf_precision;

/* Path-GEMM arithmetic for full / window output. */
typedef enum hsf_gemm_mode {
  HSF_GEMM_FP32 = 0,     /* CUDA-core FP32 products, FP32 accumulate            */
  HSF_GEMM_BF16X3 = 1,   /* tensor cores: split-BF16 (hi*hi + hi*lo + lo*hi)    */
  HSF_GEMM_TF32X3 = 2,   /* tensor cores: split-TF32 (3 products)               */
  HSF_GEMM_TF32 = 3      /* tensor cores: one TF32 product (reported only)      */
} hsf_gemm_mode;

typedef struct hsf_plan_opts {
  int32_t precision;       /* hsf_precision of the half states                      */
  int32_t gemm_mode;       /* hsf_gemm_mode for full / window output                */
  double rank_tol;         /* keep sigma_m > rank_tol * sigma_0; <= 0 means 1e-12   */
  uint64_t max_paths;      /* 0 means 2^40                                          */
  int32_t tile_bits;       /* 0 = automatic                                         */
  int32_t flags;           /* HSF_FLAG_* below                                       */
  const double *angles;    /* optional host array: angle of param_id j is angles[j] */
  int32_t num_angles;
  int32_t reserved;
} hsf_plan_opts;

#define HSF_FLAG_NO_LIGHTCONE 1   /* keep circuit order: no hoisting of gates that
                                     commute with later Schmidt factors             */
#define HSF_FLAG_NO_LEAF_CONTRACT 2 /* always materialise leaf half states         */
#define HSF_FLAG_NO_REGISTER_SWEEP 4 /* sweep with one shared-memory pass per op     */
#define HSF_FLAG_IDENTITY_STORAGE 8  /* store local qubit q at storage bit q          */
#define HSF_FLAG_REG5 16             /* complex64: 32 amplitudes per thread in the
                                        register-resident sweep (default 16)          */
#define HSF_FLAG_REG3 32             /* complex64: 8 amplitudes per thread             */
#define HSF_FLAG_NO_TC_LEVEL 64      /* complex64: sweep every tree level on the CUDA
                                        cores; by default a level whose program acts
                                        only on the 6 lowest storage bits runs as a
                                        TF32x3 tensor-core product per Schmidt digit */
#define HSF_FLAG_SVD_BLOCKS 128      /* decompose every block by the SVD; by default a
                                        cascade block (every gate touching the block's
                                        qubits on one side is diagonal on them: CNOT
                                        controls, CZ, RZZ, phases; Sec. IV-D, Example 4)
                                        gets its terms P_z (x) Y_z in closed form */
#define HSF_FLAG_LEAF_DOTS 256       /* complex64, bitstring output, opt-in: where the
                                        leaf's operators factor (L_m = S (F_m (x) I) on
                                        16-amplitude chunks) and the deepest tree level
                                        runs on the FP16 tensor-core kernel, that level
                                        writes the leaf's four chunk dots per
                                        (bitstring, child) instead of its children, and
                                        the leaf sums their bilinear form (Sec. IV-A;
                                        the same bits as the default path).  Fewer
                                        bytes move, but on GB300 the level's epilogue
                                        is then bound by the dots' shared-memory
                                        latency and the run is slower              */

typedef struct hsf_plan hsf_plan;

typedef struct hsf_plan_info {
  int32_t n, n_a, n_b;
  int32_t num_blocks;
  uint64_t num_paths;       /* product of the Schmidt ranks                         */
  int32_t precision;
  int32_t max_rank;
  int64_t tree_nodes;       /* half-state simulations per side with prefix reuse    */
  int64_t num_launches;     /* sweep launches per side for one full run             */
  int32_t leaf_bits;        /* > 0: bitstring runs contract the leaf level directly,
                               its program spans this many low storage bits          */
  int32_t num_params;       /* 1 + the largest param_id of a rotation gate          */
} hsf_plan_info;

/* Plan a circuit (Sec. II-B: horizontal cut after qubit l; Sec. III-A: gates crossing
 * the cut grouped into jointly cut blocks; Sec. IV-A, eq. eq-svd: Schmidt decomposition
 * of each block unitary through the SVD of its relabelled matrix; Sec. IV-C: the block
 * product is a chain of matrix multiplications).  Validates the circuit, cut and blocks,
 * multiplies every block and Schmidt-decomposes it on the current CUDA device in FP64
 * (one-sided Jacobi SVD), reads back the ranks (synchronous), and builds the per-level
 * gate programs.  Blocks whose SVD does not converge, or whose kept terms rebuild the
 * block matrix only to more than 1e-12 * max(1, sigma_0) plus the dropped singular
 * values, are rejected with HSF_ENUMERIC.
 * cut_l: the cut lies between qubit cut_l and cut_l+1 (Table II "cut pos."),
 * 0 <= cut_l <= n-2.  opts may be NULL (defaults).  On success *out owns all
 * plan-time device tables; release it with hsf_plan_destroy. */
hsf_status hsf_plan_create(const hsf_circuit *circuit, int32_t cut_l,
                           const hsf_blocks *blocks, const hsf_plan_opts *opts,
                           hsf_plan **out);

/* Sizes of a plan: num_paths is the number of paths n_p, the product of the blocks'
 * Schmidt ranks (Sec. II-B, Sec. IV-B: n_p^j for joint cuts; Table I "# Paths");
 * tree_nodes and num_launches describe this library's prefix-sharing schedule, which
 * the paper does not have.  info is written by the call (host memory). */
hsf_status hsf_plan_get_info(const hsf_plan *plan, hsf_plan_info *info);

/* Plan a plain Schroedinger simulation of the same circuit (Sec. II-A, Example 1: the
 * gates applied one after another to the full 2^n statevector from |0...0>; Table I
 * column S is the method it is compared with).  There is no cut and no block: the
 * returned plan holds one program of all gates on all n qubits (the same fusion and
 * tile-pass sweep kernels as the half states) and one path.  hsf_run on it sweeps the
 * full state in place inside the workspace (hsf_workspace_size: 2^n amplitudes of the
 * plan's precision, 256-byte rounded) and writes the requested amplitudes (bitstrings,
 * window or all) as complex128; the path range is ignored.  n <= 34 in complex64 and
 * n <= 33 in complex128 (a state of at most 128 GB).  HSF_EINVAL for a bad circuit. */
hsf_status hsf_plan_create_schrodinger(const hsf_circuit *circuit, const hsf_plan_opts *opts,
                                       hsf_plan **out);

/* Human-readable description of the plan's programs (storage order, tree levels,
 * tile passes, register groups, ops, and per block its rank, Jacobi sweeps and
 * reconstruction residual) written to buf (NUL-terminated, at most cap bytes).
 * Returns the size needed including the NUL, or -1 for a NULL plan.  Diagnostic only;
 * the paper has no counterpart. */
int64_t hsf_plan_describe(const hsf_plan *plan, char *buf, int64_t cap);

/* Singular values sigma_m of block k (eq. eq-svd, Sec. IV-A; descending, only the kept
 * ones) and its Schmidt rank r; copies at most cap values into sigma (host memory).
 * HSF_EINVAL for a NULL plan or a block index out of range. */
hsf_status hsf_plan_get_sigma(const hsf_plan *plan, int32_t block, double *sigma,
                              int32_t cap, int32_t *rank);

/* Automatic joint-cut blocks (Sec. V: cascades of commuting RZZ gates regrouped so that
 * they can be cut jointly; Sec. IV-D, Example 4: a cascade sharing one qubit has rank 2).
 * In every maximal run of consecutive diagonal gates (which commute), the crossing
 * two-qubit gates form a bipartite graph between the qubits of the two halves; a
 * minimum vertex cover of it (Koenig's theorem, from a maximum matching) gives the hub
 * qubits, and each hub's gates become one block (at most max_leaves, 1..8, gates per
 * block; a larger star is split).  Other crossing gates become singleton blocks.  The
 * run is reordered: in-half gates first, then the blocks.  Host-only, no device work.
 *   order:    out, num_gates entries: order[i] is the input index of the i-th gate of
 *             the reordered circuit (the same circuit: only commuting gates move).
 *   offsets, gate_idx: out, CSR blocks over the REORDERED circuit's gate indices, in
 *             dependency order; offsets needs cap_blocks + 1 entries, gate_idx
 *             num_gates entries.
 *   num_blocks: out; num_hubs: out (may be NULL), the vertex-cover size summed over
 *             runs (joint paths = 2^num_blocks when every block has rank 2).
 * HSF_EINVAL for a bad circuit, cut or max_leaves; HSF_ENOMEM if more than cap_blocks
 * blocks are found. */
hsf_status hsf_find_blocks(const hsf_circuit *circuit, int32_t cut_l, int32_t max_leaves,
                           int32_t *order, int32_t *offsets, int32_t *gate_idx, int32_t cap_blocks,
                           int32_t *num_blocks, int32_t *num_hubs);

/* Qubit-reordering search for a better cut (Sec. VI: reordering the qubits to find
 * better blocks is named as future work; no method is given there).  Searches the
 * bipartitions of the qubits with n_b = cut_l + 1 qubits on side b for the one whose
 * hsf_find_blocks blocks give the fewest joint paths: cost = log2 of the path count,
 * with rank 2 for a cascade of two or more gates (Sec. IV-D, Example 4) and the
 * operator-Schmidt rank of the relabeled matrix for a single crossing gate (Sec. IV-A).
 * Local search: Kernighan-Lin passes of swaps of one a-qubit with one b-qubit (the
 * best swap among qubits not yet moved in the pass, kept only up to the pass's best
 * point), repeated while a pass improves, from the input bipartition and from
 * `restarts` random ones drawn with splitmix64(seed).  Deterministic for a given seed.  Host-only, no device work.
 *   perm:   out, n entries: new label of qubit q (side-b qubits get 0..cut_l, side-a
 *           qubits cut_l+1..n-1, each side in ascending old label).  Relabeling every
 *           gate's qubits by perm (and bit q of a bitstring to bit perm[q]) gives the
 *           same circuit with the better cut after qubit cut_l.
 *   log2_paths_before / _after: out (may be NULL), the cost of the input and of the
 *           returned bipartition.
 * HSF_EINVAL for a bad circuit, cut, max_leaves (1..8) or restarts < 0. */
hsf_status hsf_search_cut(const hsf_circuit *circuit, int32_t cut_l, int32_t max_leaves,
                          int32_t restarts, uint64_t seed, int32_t *perm,
                          double *log2_paths_before, double *log2_paths_after);

/* Release a plan and every device buffer it owns (its tables, and the workspace of
 * hsf_run calls made with workspace == NULL).  Waits for device work that may still
 * read them.  NULL is ignored.  The paper has no counterpart. */
void hsf_plan_destroy(hsf_plan *plan);

/* Device workspace (bytes) that hsf_run needs for the given output request:
 * num_bitstrings > 0 selects bitstring output, else window > 0 selects the first
 * `window` amplitudes, else all 2^n amplitudes.  The library sizes its breadth
 * (paths in flight, Sec. II-B: the paths are independent and can be simulated in any
 * grouping) to fit `budget_bytes` when it is nonzero.  HSF_ENOMEM if no path chunk
 * fits the budget; HSF_EINVAL for a full output of more than 2^34 amplitudes. */
hsf_status hsf_workspace_size(const hsf_plan *plan, size_t num_bitstrings,
                              uint64_t window, size_t budget_bytes, size_t *bytes);

/* Amplitudes by HSF path sum over paths [path_begin, path_end) (both 0 = all):
 * amp(x) = sum_p psi_a^p(x_a) psi_b^p(x_b) with x = x_a 2^{n_b} + x_b (Sec. II-B, the
 * Kronecker products of the two halves' states added over all paths; Sec. V computes
 * a leading window of amplitudes, "the first 10^6").
 *   bitstrings: device array of num uint64 (bit q = qubit q), or NULL.
 *   window:     with bitstrings == NULL: the first `window` amplitudes (0 = all 2^n).
 *   out:        device array of complex128 (re, im interleaved), one per amplitude,
 *               caller-owned.
 *   workspace:  device buffer of at least hsf_workspace_size(...) bytes, 256-byte
 *               aligned, caller-owned; or NULL: the plan then owns a workspace sized
 *               for 60% of the device's free memory, allocated on first use (and grown
 *               when a larger request needs it) through the allocator registered with
 *               hsf_set_allocator, freed by hsf_plan_destroy.  Do not pass NULL under
 *               stream capture.  stream: cudaStream_t (NULL = legacy default).
 * The per-path products are formed in the plan's state precision and summed across
 * path chunks in FP64 with Neumaier compensation.  Asynchronous: errors found on the
 * device (an expired bounded wait, a NaN / Inf amplitude) are reported by hsf_sync.
 * Argument errors return HSF_EINVAL before any device work; a workspace that holds no
 * path chunk returns HSF_ENOMEM. */
hsf_status hsf_run(hsf_plan *plan, const uint64_t *bitstrings, size_t num,
                   uint64_t window, uint64_t path_begin, uint64_t path_end,
                   void *out, void *workspace, size_t workspace_bytes, void *stream);

/* Device memory for plan-owned workspaces (hsf_run with workspace == NULL):
 * alloc(ctx, bytes, stream) returns a 256-byte aligned device pointer or NULL, and
 * release(ctx, ptr, stream) takes it back (a binding can route both to its framework's
 * caching allocator).  Passing NULL functions restores the default, cudaMalloc and
 * cudaFree.  Process-wide; a plan releases its workspace with the functions that
 * allocated it.  The paper has no counterpart. */
typedef void *(*hsf_alloc_fn)(void *ctx, size_t bytes, void *stream);
typedef void (*hsf_free_fn)(void *ctx, void *ptr, void *stream);
void hsf_set_allocator(hsf_alloc_fn alloc, hsf_free_fn release, void *ctx);

/* Same as hsf_run, but for callers that cannot allocate device memory (for example
 * code that runs while another runtime owns all device allocations, or a loop that
 * must not block on an allocator).  There is no workspace argument: the library uses a
 * 32 MiB scratch array compiled into it (kept by every GPU that loads the library
 * until the process exits) and allocates nothing.  The paper has no counterpart; this
 * is a deployment convenience.
 * Requests whose smallest path chunk needs more than 32 MiB fail with HSF_ENOMEM and
 * a message naming the limit.  All calls share the array and its contents persist
 * between calls (each run zeroes what it accumulates into); calls that overlap on the
 * GPU race on it, so order them.  The first call on each device looks the array's
 * address up (with that device current); make that first call before any stream
 * capture.  That cached address does not survive a device reset (cudaDeviceReset or a
 * re-created primary context): do not call this again in the process after one.
 * Requests that are invalid for hsf_run (bad plan, output size, window) return the same
 * status as hsf_workspace_size would, not HSF_ENOMEM. */
hsf_status hsf_run_static(hsf_plan *plan, const uint64_t *bitstrings, size_t num,
                          uint64_t window, uint64_t path_begin, uint64_t path_end,
                          void *out, void *stream);

/* Adjoint gradient of a real loss L of the amplitudes at `bitstrings` with respect
 * to the shared angles (gate param_id): grad[j] = dL/dtheta_j, j < num_params.  The
 * paper computes no gradients; this builds on two of its facts: every path's
 * contribution is a product of the two halves' states (Sec. II-B), and the amplitude
 * is linear in each block matrix, whose derivative has a Schmidt decomposition like any
 * matrix (Sec. III-B: an SVD exists for every matrix; Sec. IV-A).
 *   gout: device complex128 per bitstring, the upstream gradient
 *         g_s = dL/dRe(amp_s) + i dL/dIm(amp_s) (PyTorch's convention; for
 *         L = sum_s |amp_s|^2 it is 2 amp_s).
 *   grad: device double[num_params]; num_params must cover every param_id.
 * Rotations inside one half are differentiated by walking the path tree backwards
 * (uncomputing unitary gates, never the Schmidt factors, which are taken from the
 * forward's stored node states); rotations inside a cut block by the HSF sum with
 * the block replaced by its derivative, Schmidt-decomposed on the device (the
 * amplitude is linear in the block matrix, Sec. IV-A; cascade blocks keep their
 * closed-form terms, Sec. IV-D).  Supported rotation kinds: RX, RY, RZ, RZZ.  Forward
 * states are recomputed rather than stored for the whole tree: levels 0..k0 of the path
 * tree are held for every node, and each level-k0 node's subtree is recomputed, walked
 * back and released in turn, k0 being the smallest level whose layout fits the
 * workspace.  hsf_grad_workspace_size(plan, num, budget, &bytes): bytes needed for the
 * layout chosen under `budget` (0: the whole tree at once, the fastest); HSF_ENOMEM if
 * no layout fits.  hsf_grad picks its layout from workspace_bytes the same way.  The
 * first call builds the gradient programs and derivative plans (synchronous).  Blocks
 * with more than 3 qubits on a side return HSF_ENOTSUP. */
hsf_status hsf_grad_workspace_size(hsf_plan *plan, size_t num_bitstrings, size_t budget_bytes, size_t *bytes);
hsf_status hsf_grad(hsf_plan *plan, const uint64_t *bitstrings, size_t num, const void *gout,
                    double *grad, int32_t num_params, void *workspace, size_t workspace_bytes,
                    void *stream);

/* Batches: many circuits (uneven n, path counts, outputs) recorded once into a CUDA
 * graph and replayed with one launch.  The paper has no counterpart (each circuit's
 * run is hsf_run, Sec. II-B).  Items run one after another inside the graph
 * and share `workspace` (hsf_batch_workspace_size: the largest item's need); every
 * plan, bitstring array and output must stay alive and at the same address while
 * the batch exists.  Recording happens on `stream` (stream capture); profiling must be
 * off while recording. */
typedef struct hsf_batch hsf_batch;
typedef struct hsf_batch_item {
  hsf_plan *plan;
  const uint64_t *bitstrings;   /* device, or NULL                          */
  size_t num;
  uint64_t window;              /* with bitstrings == NULL: leading amplitudes */
  void *out;                    /* device complex128                        */
} hsf_batch_item;
hsf_status hsf_batch_workspace_size(const hsf_batch_item *items, int32_t count, size_t *bytes);
hsf_status hsf_batch_create(const hsf_batch_item *items, int32_t count, void *workspace,
                            size_t workspace_bytes, void *stream, hsf_batch **out);
hsf_status hsf_batch_launch(hsf_batch *batch, void *stream);
/* Kernel launches in one replay of the batch graph. */
int64_t hsf_batch_nodes(const hsf_batch *batch);
void hsf_batch_destroy(hsf_batch *batch);

/* Autotuner (the paper has no counterpart; its preprocessing mentions gate fusion,
 * Table I caption): for this circuit shape and request, plan and time candidate
 * configurations on the current device by a coordinate search (each dimension in turn,
 * the others held at the best so far): shared-memory tile width 2^tile_bits, register-
 * group fusion on or off and its width (8 / 16 / 32 amplitudes per thread), tensor-core
 * tree levels on or off, the path-GEMM form for window output (split-BF16, split-TF32 or
 * FP32; never the inexact plain TF32) and the path batch (workspace budget: the full
 * workspace, a quarter or a sixteenth, which sets the path-chunk size).  The fastest is
 * written into opts->tile_bits, opts->flags (HSF_FLAG_NO_REGISTER_SWEEP, _REG3, _REG5,
 * _NO_TC_LEVEL) and opts->gemm_mode, and its workspace budget into *best_budget (may be
 * NULL; pass it to hsf_workspace_size).  Results are appended to the text file
 * cache_path (may be NULL) keyed by a hash of the circuit structure and request, and
 * reused on later calls.  Timing runs use `workspace` (hsf_workspace_size bytes for the
 * request) and synchronise. */
hsf_status hsf_tune(const hsf_circuit *circuit, int32_t cut_l, const hsf_blocks *blocks,
                    hsf_plan_opts *opts, size_t num_bitstrings, const uint64_t *bitstrings,
                    uint64_t window, const char *cache_path, void *workspace,
                    size_t workspace_bytes, size_t *best_budget);

/* Wait for the stream and report device-side failures of earlier runs of this plan:
 * returns HSF_ETIMEOUT (and clears the flag) if a bounded wait inside a kernel expired,
 * or HSF_ENUMERIC (and clears it) if an output amplitude was NaN or infinite; the
 * affected outputs are then invalid.  The paper has no counterpart. */
hsf_status hsf_sync(hsf_plan *plan, void *stream);

/* Message of the calling thread's last failed call (thread-local, valid until that
 * thread's next failing call).  The paper has no counterpart. */
const char *hsf_last_error(void);

/* Per-kernel timing for roofline reporting (the paper has no counterpart).  With profiling on, every kernel that
 * hsf_run launches is bracketed by CUDA events on the caller's stream and tagged
 * with its algorithmic bytes and flops; hsf_profile_collect waits for the events,
 * adds them up per kernel kind (HSF_KERNEL_*) into stats[0..cap) and clears the
 * plan's record.  Profiling is off by default; it is a process-wide switch. */
typedef enum hsf_kernel_kind {
  HSF_KERNEL_SWEEP = 0,      /* half-state gate sweeps                       */
  HSF_KERNEL_GATHER = 1,     /* bitstring gather-dot over paths              */
  HSF_KERNEL_REDUCE = 2,     /* FP64 compensated cross-chunk sums            */
  HSF_KERNEL_WINDOW = 3,     /* window / full path GEMM                      */
  HSF_KERNEL_OTHER = 4,      /* zero-fill, index maps, finalize              */
  HSF_KERNEL_LEAF = 5,       /* leaf level contracted at the bitstrings      */
  HSF_KERNEL_LEVEL_MMA = 6,  /* tree level as a tensor-core product per digit,
                                TF32 parts (levels with ops after the product) */
  HSF_KERNEL_LEVEL_F16 = 7,  /* the same with FP16 parts (levels without)    */
  HSF_KERNEL_PACK = 8,       /* split-operand packing of the tensor-core path GEMM */
  HSF_NUM_KERNEL_KINDS = 9
} hsf_kernel_kind;

typedef struct hsf_kernel_stat {
  int64_t launches;
  double ms;                 /* summed event-timed duration                  */
  double bytes;              /* algorithmic DRAM bytes (read + write)        */
  double flops;              /* algorithmic floating-point operations        */
} hsf_kernel_stat;

void hsf_set_profiling(int32_t on);
hsf_status hsf_profile_collect(hsf_plan *plan, hsf_kernel_stat *stats, int32_t cap);

/* Number of CUDA kernels this library has launched in the process so far. */
uint64_t hsf_launch_count(void);

/* Library version string. */
const char *hsf_version(void);

#ifdef __cplusplus
}
#endif
#endif /* HSF_H */
