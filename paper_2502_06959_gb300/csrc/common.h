// Internal declarations shared by the host planner (C++) and the CUDA kernels.
// Nothing here is part of the public C ABI (include/hsf.h).
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

namespace hsf {

// ---------------------------------------------------------------------------
// Gate programs of the half-state sweep kernel.
// A program is a list of ops applied in order to one tile of a half state.  A tile
// holds 2^t amplitudes: the storage bits in `active_mask` vary inside the tile, the
// other storage bits are fixed per tile.
// ---------------------------------------------------------------------------
enum : int32_t { OP_DENSE = 0, OP_DIAG = 1 };
constexpr int32_t kFixedBit = 64;   // pos >= kFixedBit: storage bit (pos - 64) outside the tile

struct DevOp {
  // the first 16 bytes are all a dense op needs in the register kernel
  int32_t type;          // OP_DENSE: 2^nq x 2^nq matrix; OP_DIAG: 2^nq phases
  int32_t kidx;          // dense ops: index 0..24 of the slot pattern (jump-table dispatch)
  int32_t mat;           // offset (complex elements) into the program's matrix pool
  int32_t digit_stride;  // > 0: matrix = pool[mat + digit * digit_stride] (Schmidt factor)
  int32_t nq;            // 1..3
  int32_t kcase;         // dense ops: which unrolled slot pattern applies (see sweep.cu)
  int32_t param;         // gradient programs: angle index of this rotation, else -1
  int32_t kmat;          // gradient programs: offset of K = (dG/dtheta) G^-1 in the pool
  int32_t pos[3];        // tile bit of each operand qubit, pos[0] = matrix MSB
  int32_t slot[3];       // register slot of each operand, -1 if none; dense ops have
                         // slot[0] > slot[1] > slot[2] (matrix MSB on the highest slot)
  int32_t pad[2];        // 64 bytes: read as int4 words
};
static_assert(sizeof(DevOp) == 64, "DevOp is read as four int4");

// A register group: consecutive ops whose dense operands lie in `nslots` tile bits;
// every thread holds the 2^RB amplitudes spanned by slots[0..RB) (filled with other
// tile bits when fewer are needed) for one assignment of the remaining tile bits.
constexpr int kMaxSlots = 5;
// register-resident sweep: amplitudes per thread = 2^kRegBits, CTA tile = 2^kRegTile
constexpr int kRegBitsC64 = 4, kRegTileC64 = 12;
constexpr int kRegBitsC128 = 3, kRegTileC128 = 11;
constexpr int kSweepThreads = 256;       // 2^(tile - reg bits); two CTAs per SM
struct DevGroup {
  int32_t slots[kMaxSlots];   // tile bits, ascending
  int32_t first_op;
  int32_t num_ops;
  int32_t pad;
};

// One launch of the sweep kernel: all tiles of all nodes of one tree level, one pass.
struct SweepArgs {
  const DevOp *ops;
  int32_t num_ops;
  int32_t h;             // half-state qubits
  const void *mats;      // float2 / double2 pool
  const void *src;       // parent level buffer (read_parent) or == dst
  void *dst;             // this level's buffer, node-major, 2^h amplitudes per node
  uint64_t active_mask;  // storage bits inside a tile
  int32_t t;             // popcount(active_mask)
  int32_t radix;         // Schmidt rank of this level's block (1 at the root)
  int64_t node_lo;       // level-global index of the first node held in dst
  int64_t parent_lo;     // level-global index of the first node held in src
  int64_t num_nodes;
  int32_t tiles_per_node;
  int32_t read_parent;   // 1: tile is loaded from node/radix in src
  int32_t init_zero;     // 1: tile starts from |0...0>
  const DevGroup *groups;// register groups of the pass (register-resident kernel)
  int32_t num_groups;
  int32_t rbits;         // register slots per thread
  // The pass's ops, matrices and groups lie in one contiguous table block; when
  // stage_bytes > 0 the kernel copies it to shared memory first.
  const void *stage_src;
  int32_t stage_bytes;
  int32_t stage_mats_off, stage_groups_off;   // byte offsets within the block
  int32_t pad2;
  // Register kernel with a tile of 2^T elements and 2^L threads (t >= L): element
  // tid + k * 2^L of a CTA's tile buffer belongs to item item_of[k] and sits at storage
  // offset deposit(tid, active_mask) | elem_off[k] from that item's tile origin.
  uint64_t elem_off[32];
  uint8_t item_of[32];
};
constexpr int kMaxStageBytes = 24 * 1024;   // keeps two sweep CTAs resident per SM

// Leaf level contracted at the requested amplitudes: for every parent node (level
// B-1) and bitstring s, amp(s) += sum_m (L^a_m phi_a)(x_a) * (L^b_m phi_b)(x_b), where
// L_m is the leaf level's whole program (Schmidt factor m, then gates) acting on the
// 2^c lowest storage bits.
struct LeafArgs {
  const void *Pa, *Pb;   // parent states, node-major
  int32_t ha, hb;
  int64_t num_parents;
  const void *La, *Lb;   // [r][2^c][2^c] row-major, both sides padded to the same c
  int32_t c, r;
  int32_t m_first;       // digits [m_first, r) of the first parent are in the path range
  int32_t m_last;        // digits [0, m_last) of the last parent are in the path range
  const uint64_t *ia, *ib;   // storage index of every bitstring on each side
  int64_t S;
  int32_t parents_per_group, num_groups;
  int32_t pf;            // >= 0: factored leaf operators (L_m = S (F_m (x) I), factor on chunk bit pf)
  const void *Sa, *Sb;   // factored: S of each side, [2^c][2^c] row-major
  const void *G;         // factored: [(r+1)][(r+1)][4][4], G over digits [m0, m1)
  const void *H;         // chunks of <= 4 amplitudes: [(r+1)][(r+1)][D^2][D][D] or NULL
  const int64_t *perm;   // streaming kernels: bitstring i of ia / ib is output perm[i] (NULL: i)
  // dot form (launch_leaf_dots): the deepest level wrote, per (parent, bitstring, side),
  // the four dots d[2 i + j] of the factored leaf instead of the parent states
  const void *Da, *Db;   // [num_parents][S] x 2 float4, each side in its own bitstring order
  const uint32_t *dida;  // [S] the bitstring at each position of side a's order
  const uint32_t *dposb; // [S] position of each bitstring in side b's order
  double *partial;       // [num_groups][S][2]
  uint32_t *sync;        // 2 words of device scratch (grid barrier of the streaming kernel)
  int32_t *err;          // device status word
};

// Storage index of every bitstring on both sides (bit permutation of x_a, x_b).
struct IndexArgs {
  const uint64_t *bits;
  int64_t S;
  int32_t nb, ha, hb;
  int32_t store_a[64], store_b[64];   // storage bit of each local qubit
  uint64_t *ia, *ib;
};

// Path accumulation over leaf half states (bitstring output).
struct GatherArgs {
  const void *A;         // a-side leaves [paths][2^ha]
  const void *B;         // b-side leaves [paths][2^hb]
  int64_t num_paths;
  int32_t ha, hb;
  const uint64_t *ia, *ib;   // storage index of every bitstring on each side
  int64_t S;
  int32_t paths_per_group;
  int32_t num_groups;
  double *partial;       // [num_groups][S][2]
};

// Window / full output: C[i][j] = sum_p A[p][i] * B[p][j], i < M, j < N.
struct WindowArgs {
  const void *A;
  const void *B;
  int64_t num_paths;
  int32_t ha, hb;
  int64_t M, N;          // rows (x_a) and columns (x_b) of the window rectangle
  uint64_t window;       // amplitudes kept: index x_a * 2^hb + x_b < window
  double *out;           // complex128 accumulator (re, im)
  double *comp;          // Neumaier compensation (re, im)
  const uint64_t *row_index;  // storage index of x_a = 0..M-1 (a side)
  const uint64_t *col_index;  // storage index of x_b = 0..N-1 (b side)
};

struct BlockSvdArgs {
  // inputs
  int32_t num_blocks;
  const int32_t *block_k;        // [num_blocks] total qubits k, k_a, k_b packed as 3 ints
  const int32_t *term_begin;     // [num_blocks + 1] into terms: the block matrix is the
                                 // sum over its terms of the product of the term's gates
  const int32_t *gate_begin;     // [num_terms + 1] into gate descriptors
  const int32_t *gate_desc;      // per gate: nq, pos0, pos1, pos2, mat offset (5 ints)
  const double *gate_mats;       // complex128 pool (re, im)
  double rank_tol;
  int32_t max_sweeps;
  // outputs
  double *sigma;                 // [num_blocks][64]
  int32_t *rank;                 // [num_blocks]
  double *xf;                    // [num_blocks][64][64][2]  X'_m (scaled by sqrt sigma)
  double *yf;                    // [num_blocks][64][64][2]  Y'_m
  int32_t *sweeps_used;          // [num_blocks]; == max_sweeps: not converged
  double *residual;              // [num_blocks] max_e |U_B - sum_m X'_m (x) Y'_m| (kept terms)
  // shared-memory layout for the launch's largest block (complex elements): U at 0, the
  // working matrix at off_w, V at off_v; max_nw = the largest min(4^k_a, 4^k_b)
  int32_t off_w, off_v, max_nw;
};

// Window / full output on the tensor cores (gemm_tc.cu): complex rank-P product as one
// real GEMM with split-BF16 (mode 1), split-TF32 (mode 2) or TF32 (mode 3) operands.
struct PermArgs {
  int32_t h;
  int32_t store[64];     // storage bit of each local qubit
};
struct PathGemmArgs {
  const void *A, *B;               // complex64 leaf states [paths][2^ha] / [paths][2^hb]
  int64_t paths;
  int32_t ha, hb;
  PermArgs perm_a, perm_b;         // storage bit of each local qubit of x_a / x_b
  int64_t M, N;
  uint64_t window;
  double *out, *comp;              // FP64 output and Neumaier compensation
  void *scratch;                   // path_gemm_operand_bytes(...) bytes, 256-B aligned
  int32_t mode;
  int32_t *err;                    // device status word (bounded waits)
};
size_t path_gemm_operand_bytes(int mode, int64_t M, int64_t N, int64_t paths);
// The path GEMM in two launches: the operand packing (zeroing of the padding and the
// pack kernels), then the tcgen05 GEMM that reads the packed operands.
cudaError_t launch_path_pack(const PathGemmArgs &g, cudaStream_t st);

// Tensor-core tree level (gemm_tc.cu): child node g (digit m = g % radix) =
// U_m (x) I applied to its parent, where U_m acts on the kMmaBits lowest storage bits.
// Each parent is a row-major [2^(h - kMmaBits)][2^kMmaBits] complex matrix whose rows
// ("columns" of U_m) are contiguous, so the level is a real GEMM with K = 2^(kMmaBits+1).
constexpr int kMmaBits = 6;
constexpr int kMmaMinH = kMmaBits + 7;           // at least one 128-row tile per node
constexpr int kMmaMinPrefix = 4;                  // ops a partial product must replace
constexpr size_t kMmaWPartBytes = 128 * 128 * 4;       // one TF32 part of W_m (64 KB)
constexpr size_t kMmaWDigitBytes = 128 * 128 * 2 * 2;  // W_m as FP16 hi then lo, 128 x 128 each
struct LevelMmaArgs {
  const float *parent;     // previous level buffer, complex64 as float pairs
  float *child;            // this level's buffer
  const void *w;           // num_post > 0: per digit, TF32 hi then lo (kMmaWPartBytes each);
                           // num_post = 0: per digit, the FP16 image (kMmaWDigitBytes), then
                           // radix inverse scales
  int32_t h;
  int32_t radix;
  int64_t node_lo;         // level-global index of the first node held in child
  int64_t num_nodes;
  int64_t parent_lo;       // level-global index of the first node held in parent
  int32_t *err;            // device status word (bounded waits)
  const void *post;        // ops applied in the epilogue after the product (MmaPostOp[])
  int32_t num_post;
  int32_t pad;
  // FP16 kernel, deepest level before a leaf contraction: bit 4 R + s set when 16-amplitude
  // segment s of row R is read by some bitstring; other segments are not stored (NULL:
  // every segment is stored)
  const uint32_t *store_mask;
  // FP16 kernel, deepest level before a factored leaf on 16-amplitude chunks (dot form):
  // instead of the child rows, the four leaf dots d[2 i + j] = sum_k S[rr][e_i(k)]
  // x[e_j(k)] of every bitstring's chunk x are written, 32 bytes per (child, bitstring)
  // (NULL: store the rows)
  float4 *dots;            // [num_nodes][dot_count] x 2, bitstrings in dot_list order
  // the bitstrings ordered by key (segment within the row s) << (h - 6) | row R of their
  // chunk (storage index 64 R + 16 s + rr): dot_off[key] is the first position of a key,
  // dot_list[pos] = R << 4 | rr
  const uint32_t *dot_off; // [2^(h-4) + 1]
  const uint32_t *dot_list;    // [dot_count]
  const float2 *dot_T;     // [16 e][16 rr] S[rr][e]
  int64_t dot_count;
  int32_t dot_pf;          // the factor's chunk bit
  int32_t pad2;
};
// A one- or two-qubit op on storage bits < kMmaPostBits, applied by the tensor-core
// level's epilogue to each staged 32-row quarter (amplitude bits 0..5, row bits 0..4).
constexpr int kMmaPostBits = kMmaBits + 5;
constexpr int kMmaMaxPost = 8;
struct MmaPostOp {
  int32_t nq;              // 1 or 2
  int32_t q0, q1;          // storage bits; q0 is the matrix MSB
  int32_t diag;            // 1: m holds the 2^nq diagonal phases
  float2 m[16];            // dense 2^nq x 2^nq, row-major (or the diagonal)
};
static_assert(sizeof(MmaPostOp) == 144, "MmaPostOp layout");
cudaError_t launch_level_mma(const LevelMmaArgs &a, cudaStream_t st);
// host: the kernels' images of W_m (128 x 128 real, row-major [n][k]): TF32 hi and lo
// parts (levels with ops after the product), or power-of-two scaled FP16 hi and lo parts
// (kMmaWDigitBytes) with the inverse of the scale (levels without)
void level_mma_image(const double *w, float *hi, float *lo);
void level_mma_image_f16(const double *w, void *digit_image, float *inv_scale);

// Adjoint sweep over one pass of one tree level, in reverse op order (adjoint.cu).
struct AdjointArgs {
  const DevOp *ops;
  int32_t num_ops;
  int32_t first_op;        // ops [first_op, num_ops) are undone; 1 skips the Schmidt factor
  const void *mats;
  void *psi, *mu;          // this level's states and cotangents, node-major
  int32_t h, t;
  uint64_t active_mask;
  int64_t num_nodes;
  int32_t tiles_per_node;
  int32_t pad;
  double *grad;            // per-angle accumulators
};
struct LeafCotArgs {
  const void *psi_a, *psi_b;
  void *mu_a, *mu_b;
  int32_t ha, hb;
  int64_t paths;
  const uint64_t *ia, *ib;
  const double *gout;      // upstream gradient g_s (complex128)
  int64_t S;
};
struct PullbackArgs {
  const void *mu_child;    // children cotangents (level k), node-major
  void *mu_parent;         // parent cotangents (level k-1), overwritten
  const void *factor;      // [radix][2^nf][2^nf] factor matrices of this side
  int32_t h, nf;
  int32_t fq[3];           // storage bits of the factor's operands (fq[0] = matrix MSB)
  int32_t radix;
  int64_t parent_lo, child_lo, num_parents, num_children;
};
cudaError_t launch_adjoint(const AdjointArgs &a, int precision, cudaStream_t st);
cudaError_t launch_leaf_cot(const LeafCotArgs &a, int precision, cudaStream_t st);
cudaError_t launch_factor_pullback(const PullbackArgs &a, int precision, cudaStream_t st);
cudaError_t launch_grad_dot(const double *gout, const double *ampd, int64_t S, double *grad, cudaStream_t st);
cudaError_t launch_zero_bytes(void *p, size_t bytes, cudaStream_t st);
cudaError_t launch_path_gemm(const PathGemmArgs &g, cudaStream_t st);

// Streaming multiprocessors of the current device, looked up once per device (thread-safe);
// 0 if the query fails.
int device_sm_count();

cudaError_t launch_sweep(const SweepArgs &a, int precision, cudaStream_t st);
cudaError_t launch_gather_dot(const GatherArgs &a, int precision, cudaStream_t st);
cudaError_t launch_reduce_partials(const double *partial, int32_t num_groups, int64_t S,
                                   double *out, double *comp, cudaStream_t st);
cudaError_t launch_window(const WindowArgs &a, int precision, cudaStream_t st);
// out += comp over count doubles; sets *numeric (if not NULL) when a result is not finite.
cudaError_t launch_finalize(double *out, const double *comp, int64_t count, int32_t *numeric, cudaStream_t st);
// Words of a plan's device status block (256 bytes): the code of an expired bounded wait,
// and the output canary (non-finite amplitude) of the runs since the last hsf_sync.
constexpr int kStatusWait = 0, kStatusNumeric = 1;
cudaError_t launch_zero(double *p, int64_t count, cudaStream_t st);
// out[i] (complex128) = state[bits ? bits[i] : i] for i < count, state complex64
// (precision 0) or complex128; sets *numeric (if not NULL) on a non-finite amplitude.
cudaError_t launch_state_gather(const void *state, int precision, const uint64_t *bits, int64_t count, double *out,
                                int32_t *numeric, cudaStream_t st);
cudaError_t launch_block_svd(const BlockSvdArgs &a, cudaStream_t st);
cudaError_t launch_leaf_contract(const LeafArgs &a, int precision, cudaStream_t st);
// true when launch_leaf_contract uses the one-wave streaming kernel (large bitstring
// counts); it then writes a single partial per bitstring (num_groups = 1)
bool leaf_streams(const LeafArgs &a, int precision);
// counting sort of S bitstrings by the high bits of ia (2^kSortBits buckets at most):
// ia_s, ib_s in sorted order, perm[i] = the input position of sorted bitstring i
constexpr int kSortBits = 12;
// bit (ia >> 4) of mask_a (and of mask_b for ib) for every 16-amplitude segment that a
// bitstring's 2^c-amplitude chunk covers; the masks hold 2^(ha-4) and 2^(hb-4) bits
cudaError_t launch_chunk_mask(const uint64_t *ia, const uint64_t *ib, int64_t S, int c, int ha, int hb,
                              uint32_t *mask_a, uint32_t *mask_b, cudaStream_t st);
cudaError_t launch_bitstring_sort(const uint64_t *ia, const uint64_t *ib, int64_t S, int ha, uint32_t *counts,
                                  uint64_t *ia_s, uint64_t *ib_s, int64_t *perm, cudaStream_t st);
// the factored leaf kernel runs for this launch (FP32, factored operators, 3-4 digits)
bool leaf_factored(const LeafArgs &a, int precision);
// Dot form of the factored leaf.  launch_dot_sort, once per run: on each side the
// bitstrings ordered by key (segment s within the 64-amplitude row) << (h - 6) | row R
// of their chunk, so that the bitstrings of 16 consecutive rows in one segment are one
// range (off[side] holds the 2^(h-4) + 1 first positions, list[side] R << 4 | rr per
// position, ida the bitstring at each side-a position, posb the side-b position of each
// bitstring; cur[side] is scratch of 2^(h-4) words), and S of each side transposed to
// [e][rr], the table the level epilogue reads.  launch_leaf_dots: the bilinear form
// summed over the parents from the dots the level wrote.
struct DotSort {
  uint32_t *off[2], *cur[2], *list[2], *ida, *posb;
  float2 *T[2];
};
size_t dot_sort_bytes(int64_t S, int ha, int hb);
DotSort dot_sort_layout(unsigned char *base, int64_t S, int ha, int hb);
cudaError_t launch_dot_sort(const uint64_t *ia, const uint64_t *ib, int64_t S, int ha, int hb, const void *Sa,
                            const void *Sb, const DotSort &d, cudaStream_t st);
cudaError_t launch_leaf_dots(const LeafArgs &a, cudaStream_t st);
cudaError_t launch_index_prep(const IndexArgs &a, cudaStream_t st);
// dst[i] = storage index of local index i, i < count.
cudaError_t launch_range_index(uint64_t *dst, int64_t count, const PermArgs &perm, cudaStream_t st);

}  // namespace hsf
