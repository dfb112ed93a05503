// Half-state sweep kernel (tile version): applies one level's gate program to the
// half states of a batch of path-tree nodes (Sec. II-B: per path, the half circuits
// are simulated by consecutive matrix-vector products, Sec. II-A).
//
// Work item = (node, tile).  A CTA stages the tile (2^t amplitudes) in shared memory,
// applies every op of the pass to it and writes it to the node's buffer.  The first
// pass of a level reads the parent node's state (prefix reuse: the r children of a
// node share everything simulated before their Schmidt factor); the root level starts
// from |0...0>.
#include <cstdint>

#include "common.h"

namespace hsf {
namespace {

template <typename R> struct CT;
template <> struct CT<float> { using T = float2; };
template <> struct CT<double> { using T = double2; };

template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
  C r;
  r.x = a.x * b.x - a.y * b.y;
  r.y = a.x * b.y + a.y * b.x;
  return r;
}
template <typename C> __device__ __forceinline__ C cfma(C a, C b, C acc) {
  acc.x = fma(a.x, b.x, fma(-a.y, b.y, acc.x));
  acc.y = fma(a.x, b.y, fma(a.y, b.x, acc.y));
  return acc;
}

// Scatter the low bits of `v` into the set bits of `mask` (software PDEP).
__device__ __forceinline__ uint64_t deposit(uint64_t v, uint64_t mask) {
  uint64_t r = 0;
  while (mask) {
    uint64_t low = mask & (~mask + 1);
    if (v & 1) r |= low;
    v >>= 1;
    mask &= mask - 1;
  }
  return r;
}

__device__ __forceinline__ uint32_t insert_zero(uint32_t v, int b) {
  uint32_t lo = v & ((1u << b) - 1u);
  return ((v >> b) << (b + 1)) | lo;
}

template <typename R>
__global__ void __launch_bounds__(256) sweep_kernel(SweepArgs a) {
  using C = typename CT<R>::T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C *s = reinterpret_cast<C *>(smem_raw);
  __shared__ DevOp ops_sh[64];

  const int t = a.t;
  const uint32_t tile_elems = 1u << t;
  const uint64_t full = (a.h >= 64) ? ~0ull : ((1ull << a.h) - 1ull);
  const uint64_t inactive = full & ~a.active_mask;
  const bool contiguous = a.active_mask == ((1ull << t) - 1ull);
  const C *mats = reinterpret_cast<const C *>(a.mats);
  const int64_t items = a.num_nodes * (int64_t)a.tiles_per_node;
  const uint64_t state = 1ull << a.h;

  for (int64_t item = blockIdx.x; item < items; item += gridDim.x) {
    const int64_t nl = item / a.tiles_per_node;
    const uint64_t tile = (uint64_t)(item % a.tiles_per_node);
    const uint64_t base = deposit(tile, inactive);
    const int64_t node = a.node_lo + nl;
    const int digit = a.radix > 1 ? (int)(node % a.radix) : 0;
    const C *src = a.read_parent
                       ? reinterpret_cast<const C *>(a.src) + (uint64_t)(node / a.radix - a.parent_lo) * state
                       : reinterpret_cast<const C *>(a.dst) + (uint64_t)nl * state;
    C *dst = reinterpret_cast<C *>(a.dst) + (uint64_t)nl * state;

    for (uint32_t u = threadIdx.x; u < tile_elems; u += blockDim.x) {
      const uint64_t off = contiguous ? (base | u) : (base | deposit(u, a.active_mask));
      C v;
      if (a.init_zero) {
        v.x = (off == 0) ? R(1) : R(0);
        v.y = R(0);
      } else {
        v = src[off];
      }
      s[u] = v;
    }
    __syncthreads();

    for (int o0 = 0; o0 < a.num_ops; o0 += 64) {
      const int chunk = min(64, a.num_ops - o0);
      if ((int)threadIdx.x < chunk) ops_sh[threadIdx.x] = a.ops[o0 + threadIdx.x];
      __syncthreads();
      for (int oi = 0; oi < chunk; ++oi) {
        const DevOp op = ops_sh[oi];
        const C *m = mats + op.mat + (op.digit_stride > 0 ? digit * op.digit_stride : 0);
        if (op.type == OP_DIAG) {
          for (uint32_t u = threadIdx.x; u < tile_elems; u += blockDim.x) {
            int idx = 0;
            for (int j = 0; j < op.nq; ++j) {
              const int p = op.pos[j];
              const int bit = p >= kFixedBit ? (int)((base >> (p - kFixedBit)) & 1ull) : (int)((u >> p) & 1u);
              idx = (idx << 1) | bit;
            }
            s[u] = cmul(m[idx], s[u]);
          }
        } else if (op.nq == 1) {
          const int b = op.pos[0];
          const C m00 = m[0], m01 = m[1], m10 = m[2], m11 = m[3];
          for (uint32_t j = threadIdx.x; j < (tile_elems >> 1); j += blockDim.x) {
            const uint32_t i0 = insert_zero(j, b), i1 = i0 | (1u << b);
            const C x0 = s[i0], x1 = s[i1];
            C y0 = cmul(m00, x0), y1 = cmul(m10, x0);
            y0 = cfma(m01, x1, y0);
            y1 = cfma(m11, x1, y1);
            s[i0] = y0;
            s[i1] = y1;
          }
        } else {
          const int nq = op.nq;
          const int dim = 1 << nq;
          int sorted[3] = {op.pos[0], op.pos[1], op.pos[2]};
          for (int x = 0; x < nq; ++x)
            for (int y = x + 1; y < nq; ++y)
              if (sorted[y] < sorted[x]) { int tmp = sorted[x]; sorted[x] = sorted[y]; sorted[y] = tmp; }
          for (uint32_t j = threadIdx.x; j < (tile_elems >> nq); j += blockDim.x) {
            uint32_t i = j;
            for (int x = 0; x < nq; ++x) i = insert_zero(i, sorted[x]);
            C v[8];
            uint32_t addr[8];
            for (int k = 0; k < dim; ++k) {
              uint32_t ad = i;
              for (int x = 0; x < nq; ++x)
                if ((k >> (nq - 1 - x)) & 1) ad |= 1u << op.pos[x];
              addr[k] = ad;
              v[k] = s[ad];
            }
            for (int r = 0; r < dim; ++r) {
              C acc;
              acc.x = R(0);
              acc.y = R(0);
              for (int c = 0; c < dim; ++c) acc = cfma(m[r * dim + c], v[c], acc);
              s[addr[r]] = acc;
            }
          }
        }
        __syncthreads();
      }
    }

    for (uint32_t u = threadIdx.x; u < tile_elems; u += blockDim.x) {
      const uint64_t off = contiguous ? (base | u) : (base | deposit(u, a.active_mask));
      dst[off] = s[u];
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Register-resident variant.  The CTA stages 2^T amplitudes (T = 14 for complex64,
// 13 for complex128) of one or more tiles in shared memory, padded by one element
// every 32 (bank-conflict-free strided access).  The pass's ops come in register
// groups: every thread loads the 2^RB amplitudes spanned by the group's slots for its
// assignment of the other tile bits, applies all ops of the group in registers, and
// writes them back; dense ops are fully unrolled per slot pattern (kcase).
// ---------------------------------------------------------------------------
// Shared-memory position of tile element u: bits 4..7 and 8..11 are folded into bits
// 0..3 (XOR), so the 16 lanes of a half-warp land in 16 different 8-byte bank pairs
// whenever their four lowest varying tile bits have distinct residues mod 4.
__device__ __forceinline__ uint32_t pad32(uint32_t u) { return u ^ (((u >> 4) ^ (u >> 8)) & 15u); }

// Two consecutive complex entries (16-byte aligned for complex64).
template <typename C>
__device__ __forceinline__ void ld2(const C *p, C &a, C &b) {
  if constexpr (sizeof(C) == 8) {
    const float4 q = *reinterpret_cast<const float4 *>(p);
    a.x = q.x; a.y = q.y; b.x = q.z; b.y = q.w;
  } else {
    a = p[0];
    b = p[1];
  }
}

template <int J, int NR, typename C>
__device__ __forceinline__ void ap1(C (&v)[NR], const C *__restrict__ m) {
  C m0, m1, m2, m3;
  ld2(m, m0, m1);
  ld2(m + 2, m2, m3);
#pragma unroll
  for (int i = 0; i < NR; ++i) {
    if (i & (1 << J)) continue;
    const int k = i | (1 << J);
    const C x0 = v[i], x1 = v[k];
    v[i] = cfma(m1, x1, cmul(m0, x0));
    v[k] = cfma(m3, x1, cmul(m2, x0));
  }
}

// Packed FP32 pair FMA (two lanes per instruction): d = a * b + c elementwise.
__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) {
  float2 d;
  asm("{\n .reg .b64 ra, rb, rc, rd;\n"
      " mov.b64 ra, {%2, %3};\n mov.b64 rb, {%4, %5};\n mov.b64 rc, {%6, %7};\n"
      " fma.rn.f32x2 rd, ra, rb, rc;\n mov.b64 {%0, %1}, rd;\n}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
  return d;
}

template <int J, int K, int NR, typename C>
__device__ __forceinline__ void ap2(C (&v)[NR], const C *m0) {
  if constexpr (sizeof(C) == 8 && NR >= 16) {
    // complex64: the 4x4 matrix is loaded once as broadcast pairs (Re m, Re m) and
    // (Im m, Im m) and stays in registers for every quad; with x = (Re x, Im x) as it
    // sits in registers, P = sum mr x and Q = sum mi x are packed FMAs and
    // (m x)_r = (P.x - Q.y, P.y + Q.x)
    C mr[16], mi[16];
#pragma unroll
    for (int e = 0; e < 16; e += 2) {
      C a0, a1;
      ld2(m0 + e, a0, a1);
      mr[e] = make_float2(a0.x, a0.x);
      mi[e] = make_float2(a0.y, a0.y);
      mr[e + 1] = make_float2(a1.x, a1.x);
      mi[e + 1] = make_float2(a1.y, a1.y);
    }
#pragma unroll
    for (int i = 0; i < NR; ++i) {
      if (i & ((1 << J) | (1 << K))) continue;
      const int id[4] = {i, i | (1 << K), i | (1 << J), i | (1 << J) | (1 << K)};
      C x[4];
#pragma unroll
      for (int c = 0; c < 4; ++c) x[c] = v[id[c]];
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        C P = make_float2(0.f, 0.f), Q = P;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          P = ffma2(mr[4 * r + c], x[c], P);
          Q = ffma2(mi[4 * r + c], x[c], Q);
        }
        v[id[r]] = make_float2(P.x - Q.y, P.y + Q.x);
      }
    }
    return;
  } else if constexpr (sizeof(C) == 8) {
    // complex64 with 8-amplitude register blocks (64 registers a thread): the matrix as
    // plain complex values, to stay in registers
    C mm[16];
#pragma unroll
    for (int e = 0; e < 16; e += 2) ld2(m0 + e, mm[e], mm[e + 1]);
#pragma unroll
    for (int i = 0; i < NR; ++i) {
      if (i & ((1 << J) | (1 << K))) continue;
      const int id[4] = {i, i | (1 << K), i | (1 << J), i | (1 << J) | (1 << K)};
      C x[4];
#pragma unroll
      for (int c = 0; c < 4; ++c) x[c] = v[id[c]];
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        C acc = cmul(mm[4 * r], x[0]);
        acc = cfma(mm[4 * r + 1], x[1], acc);
        acc = cfma(mm[4 * r + 2], x[2], acc);
        acc = cfma(mm[4 * r + 3], x[3], acc);
        v[id[r]] = acc;
      }
    }
    return;
  }
#pragma unroll
  for (int i = 0; i < NR; ++i) {
    if (i & ((1 << J) | (1 << K))) continue;
    // complex128: matrix rows are re-read per quad (L1 broadcast) to keep register use low
    const C *m = m0;
    asm volatile("" : "+l"(m));
    const int id[4] = {i, i | (1 << K), i | (1 << J), i | (1 << J) | (1 << K)};
    C x[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) x[c] = v[id[c]];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      C r0, r1, r2, r3;
      ld2(m + 4 * r, r0, r1);
      ld2(m + 4 * r + 2, r2, r3);
      C acc = cmul(r0, x[0]);
      acc = cfma(r1, x[1], acc);
      acc = cfma(r2, x[2], acc);
      acc = cfma(r3, x[3], acc);
      v[id[r]] = acc;
    }
  }
}

template <int J, int K, int L, int NR, typename C>
__device__ __forceinline__ void ap3(C (&v)[NR], const C *m0) {
#pragma unroll
  for (int i = 0; i < NR; ++i) {
    if (i & ((1 << J) | (1 << K) | (1 << L))) continue;
    // reload the 8x8 matrix per octet rather than keeping 64 entries live
    const C *m = m0;
    asm volatile("" : "+l"(m));
    int id[8];
#pragma unroll
    for (int c = 0; c < 8; ++c)
      id[c] = i | ((c & 4) ? (1 << J) : 0) | ((c & 2) ? (1 << K) : 0) | ((c & 1) ? (1 << L) : 0);
    C x[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) x[c] = v[id[c]];
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      C acc = cmul(m[8 * r], x[0]);
#pragma unroll
      for (int c = 1; c < 8; ++c) acc = cfma(m[8 * r + c], x[c], acc);
      v[id[r]] = acc;
    }
  }
}

#define KC1(J) (J)
#define KC2(J, K) (16 + ((J) << 3) + (K))
#define KC3(J, K, L) (128 + ((J) << 6) + ((K) << 3) + (L))

template <int NR, typename C>
__device__ __forceinline__ void apply_dense(C (&v)[NR], int kidx, const C *__restrict__ m) {
  // kidx enumerates the slot patterns densely (1q: J; 2q: 5 + pair; 3q: 15 + triple), so the
  // switch compiles to a jump table; patterns outside the 2^RB register block are empty
#define HSF_C1(I, J) case I: if constexpr ((1 << (J)) < NR) ap1<J>(v, m); break;
#define HSF_C2(I, J, K) case I: if constexpr ((1 << (J)) < NR) ap2<J, K>(v, m); break;
#define HSF_C3(I, J, K, L) case I: if constexpr ((1 << (J)) < NR) ap3<J, K, L>(v, m); break;
  switch (kidx) {
    HSF_C1(0, 0) HSF_C1(1, 1) HSF_C1(2, 2) HSF_C1(3, 3) HSF_C1(4, 4)
    HSF_C2(5, 1, 0) HSF_C2(6, 2, 0) HSF_C2(7, 2, 1) HSF_C2(8, 3, 0) HSF_C2(9, 3, 1) HSF_C2(10, 3, 2)
    HSF_C2(11, 4, 0) HSF_C2(12, 4, 1) HSF_C2(13, 4, 2) HSF_C2(14, 4, 3)
    HSF_C3(15, 2, 1, 0) HSF_C3(16, 3, 1, 0) HSF_C3(17, 3, 2, 0) HSF_C3(18, 3, 2, 1)
    HSF_C3(19, 4, 1, 0) HSF_C3(20, 4, 2, 0) HSF_C3(21, 4, 2, 1) HSF_C3(22, 4, 3, 0) HSF_C3(23, 4, 3, 1)
    HSF_C3(24, 4, 3, 2)
    default: break;
  }
#undef HSF_C1
#undef HSF_C2
#undef HSF_C3
}

// Asynchronous global -> shared copy of one amplitude (8 or 16 bytes).
template <int BYTES>
__device__ __forceinline__ void cp_async_elem(void *smem, const void *gmem) {
  const uint32_t sa = (uint32_t)__cvta_generic_to_shared(smem);
  if constexpr (BYTES == 8)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem) : "memory");
  else
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// Per-batch addressing of the items (tiles) a CTA holds.
template <int MAXI>
struct ItemInfo {
  int64_t src[MAXI], dst[MAXI];   // element offsets of each item's tile origin
  uint64_t base[MAXI];            // fixed storage bits of each item's tile
  int digit[MAXI];
  int nvalid;
};

template <typename R, int RB, int T>
__global__ void __launch_bounds__(1 << (T - RB), 2) sweep_reg_kernel(SweepArgs a) {
  using C = typename CT<R>::T;
  constexpr int NR = 1 << RB;
  constexpr int MAXI = 64;                   // most items a CTA holds (t >= T - 6)
  constexpr uint32_t BUF = 1u << T;                       // tile elements (swizzled)
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C *sbuf = reinterpret_cast<C *>(smem_raw);   // two tile buffers (double buffering)
  __shared__ ItemInfo<MAXI> info[2];
  const int t = a.t;
  const int tb = t - RB;                     // thread bits per item
  const int ipc = 1 << (T - t);              // items per CTA
  const uint32_t tmask = (1u << t) - 1u;
  const uint64_t full = (1ull << a.h) - 1ull;
  const uint64_t inactive = full & ~a.active_mask;
  const bool contiguous = a.active_mask == ((1ull << t) - 1ull);
  const C *mats = reinterpret_cast<const C *>(a.mats);
  const int64_t items = a.num_nodes * (int64_t)a.tiles_per_node;
  const int tpn_bits = a.h - t;              // tiles per node = 2^(h - t)
  const int tid = threadIdx.x;
  const int il = tid >> tb;                  // my item within the CTA
  const uint32_t inst = (uint32_t)tid & ((1u << tb) - 1u);
  const C *src = reinterpret_cast<const C *>(a.read_parent ? a.src : a.dst);
  C *dst = reinterpret_cast<C *>(a.dst);
  const int64_t stride = (int64_t)gridDim.x * ipc;
  // op tables: staged in shared memory after the two tile buffers when they fit
  const DevOp *ops = a.ops;
  const DevGroup *groups = a.groups;
  if (a.stage_bytes > 0) {
    unsigned char *st = reinterpret_cast<unsigned char *>(sbuf + 2 * BUF);
    const int4 *gs = reinterpret_cast<const int4 *>(a.stage_src);
    for (int e = tid; e < a.stage_bytes / 16; e += blockDim.x) reinterpret_cast<int4 *>(st)[e] = gs[e];
    ops = reinterpret_cast<const DevOp *>(st);
    mats = reinterpret_cast<const C *>(st + a.stage_mats_off);
    groups = reinterpret_cast<const DevGroup *>(st + a.stage_groups_off);
    __syncthreads();
  }

  // Fast copy path (t >= LNT, no |0> start): thread tid moves elements tid + k * NT,
  // k < NR, whose swizzled position is closed-form (the swizzle folds tile bits 4..11
  // into bits 0..3: bits 4..7 come from tid, bits 8..11 from tid and k).
  constexpr int LNT = T - RB;
  constexpr int NT = 1 << LNT;
  const bool fast = t >= LNT && !a.init_zero;
  const uint64_t dep_tid = contiguous ? (uint64_t)tid : deposit((uint64_t)tid, a.active_mask);
  const uint32_t tsw = (uint32_t)tid ^ ((((uint32_t)tid >> 4) ^ ((uint32_t)tid >> 8)) & 15u);
  auto fast_pos = [&](int k) -> uint32_t {
    if constexpr (LNT >= 8)
      return (tsw ^ (((uint32_t)k << (LNT - 8)) & 15u)) + ((uint32_t)k << LNT);
    else
      return pad32((uint32_t)tid + ((uint32_t)k << LNT));
  };

  // Start the copies of the batch beginning at item0 into buffer `slot`.
  auto prefetch = [&](int64_t item0, int slot) {
    ItemInfo<MAXI> &in = info[slot];
    const int nvalid = (int)min((int64_t)ipc, items - item0);
    for (int j = tid; j < nvalid; j += blockDim.x) {
      const int64_t item = item0 + j;
      const int64_t nl = item >> tpn_bits;
      const uint64_t tile = (uint64_t)item & ((1ull << tpn_bits) - 1ull);
      const uint64_t base = contiguous ? (tile << t) : deposit(tile, inactive);
      const int64_t node = a.node_lo + nl;
      const int64_t srcnode = a.read_parent ? node / a.radix - a.parent_lo : nl;
      in.src[j] = (srcnode << a.h) + (int64_t)base;
      in.dst[j] = (nl << a.h) + (int64_t)base;
      in.base[j] = base;
      in.digit[j] = a.radix > 1 ? (int)(node % a.radix) : 0;
    }
    if (tid == 0) in.nvalid = nvalid;
    __syncthreads();
    C *sb = sbuf + slot * BUF;
    if (fast) {
#pragma unroll
      for (int k = 0; k < NR; ++k) {
        const int j = a.item_of[k];
        if (j < nvalid)
          cp_async_elem<(int)sizeof(C)>(sb + fast_pos(k), src + in.src[j] + (int64_t)(dep_tid | a.elem_off[k]));
      }
      cp_async_commit();
      return;
    }
    const uint32_t total = (uint32_t)nvalid << t;
    for (uint32_t e = tid; e < total; e += blockDim.x) {
      const int j = (int)(e >> t);
      const uint32_t u = e & tmask;
      if (a.init_zero) {
        C v;
        v.x = (in.base[j] == 0 && u == 0) ? R(1) : R(0);
        v.y = R(0);
        sb[pad32(e)] = v;
      } else {
        cp_async_elem<(int)sizeof(C)>(sb + pad32(e), src + in.src[j] + (int64_t)(contiguous ? u : deposit(u, a.active_mask)));
      }
    }
    cp_async_commit();
  };

  int64_t item0 = (int64_t)blockIdx.x * ipc;
  if (item0 < items) prefetch(item0, 0);
  for (int k = 0; item0 < items; item0 += stride, ++k) {
    const int slot = k & 1;
    const int64_t next = item0 + stride;
    if (next < items) {
      prefetch(next, slot ^ 1);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    C *s = sbuf + slot * BUF;
    const ItemInfo<MAXI> &in = info[slot];
    const int nvalid = in.nvalid;
    const bool valid = il < nvalid;
    const int digit = valid ? in.digit[il] : 0;
    const uint64_t my_base = valid ? in.base[il] : 0ull;

    for (int g = 0; g < a.num_groups; ++g) {
      const DevGroup G = groups[g];
      uint32_t smask = 0;
      uint32_t w[RB];
#pragma unroll
      for (int j = 0; j < RB; ++j) {
        w[j] = 1u << G.slots[j];
        smask |= w[j];
      }
      // this thread's instance bits fill the tile bits that are not slots (ascending)
      uint32_t dep = inst;
#pragma unroll
      for (int j = 0; j < RB; ++j) dep = insert_zero(dep, G.slots[j]);
      const uint32_t ubase = ((uint32_t)il << t) | dep;
      // the swizzle is linear over the tile bits and ubase has no slot bits, so the
      // position of element i is swz(ubase) ^ (XOR of swz(w_j) over the bits j of i)
      const uint32_t sbase = pad32(ubase);
      uint32_t sw[RB];
#pragma unroll
      for (int j = 0; j < RB; ++j) sw[j] = pad32(w[j]);
      C v[NR];
#pragma unroll
      for (int i = 0; i < NR; ++i) {
        uint32_t u = sbase;
#pragma unroll
        for (int j = 0; j < RB; ++j)
          if (i & (1 << j)) u ^= sw[j];
        v[i] = s[u];
      }
      for (int o = G.first_op; o < G.first_op + G.num_ops; ++o) {
        // the op record is read as int4 words into scalars (no local-memory copy); a
        // dense op needs only the first
        const int4 *o4 = reinterpret_cast<const int4 *>(ops + o);
        const int4 w0 = o4[0];
        const int op_type = w0.x, op_kidx = w0.y, op_mat = w0.z, op_dstride = w0.w;
        const C *m = mats + op_mat + (op_dstride > 0 ? digit * op_dstride : 0);
        if (op_type == OP_DIAG) {
          const int4 w1 = o4[1], w2 = o4[2], w3 = o4[3];
          const int op_nq = w1.x, op_kcase = w1.y;
          const int pos_[3] = {w2.x, w2.y, w2.z};
          const int slot_[3] = {w2.w, w3.x, w3.y};
          // operands are ordered slot operands first (kcase = their count); the
          // others are bits of this thread's instance or of the tile's fixed bits
          const int ns = op_kcase;
          int tpart = 0;
#pragma unroll
          for (int x = 0; x < 3; ++x) {
            if (x < ns || x >= op_nq) continue;
            const int p = pos_[x];
            const int bit = p >= kFixedBit ? (int)((my_base >> (p - kFixedBit)) & 1ull) : (int)((ubase >> p) & 1u);
            tpart |= bit << (op_nq - 1 - x);
          }
          const int sh = op_nq - ns;            // slot bits sit above the fixed part
          if (ns == 0) {
            const C d = m[tpart];
#pragma unroll
            for (int i = 0; i < NR; ++i) v[i] = cmul(d, v[i]);
          } else if (ns == 1) {
            const C d0 = m[tpart], d1 = m[tpart | (1 << sh)];
            const int s0 = slot_[0];
#pragma unroll
            for (int i = 0; i < NR; ++i) v[i] = cmul(((i >> s0) & 1) ? d1 : d0, v[i]);
          } else if (ns == 2) {
            const C d0 = m[tpart], d1 = m[tpart | (1 << sh)], d2 = m[tpart | (2 << sh)], d3 = m[tpart | (3 << sh)];
            const int s0 = slot_[0], s1 = slot_[1];
#pragma unroll
            for (int i = 0; i < NR; ++i) {
              const int b0 = (i >> s0) & 1, b1 = (i >> s1) & 1;
              const C d = b0 ? (b1 ? d3 : d2) : (b1 ? d1 : d0);
              v[i] = cmul(d, v[i]);
            }
          } else {
            const int s0 = slot_[0], s1 = slot_[1], s2 = slot_[2];
#pragma unroll
            for (int i = 0; i < NR; ++i) {
              const int idx = (((i >> s0) & 1) << 2) | (((i >> s1) & 1) << 1) | ((i >> s2) & 1);
              v[i] = cmul(m[idx], v[i]);
            }
          }
        } else {
          apply_dense<NR>(v, op_kidx, m);
        }
      }
      // recompute the addresses instead of keeping 2^RB of them live across the ops
      uint32_t sb2 = sbase;
      asm volatile("" : "+r"(sb2));
#pragma unroll
      for (int j = 0; j < RB; ++j) asm volatile("" : "+r"(sw[j]));
#pragma unroll
      for (int i = 0; i < NR; ++i) {
        uint32_t u = sb2;
#pragma unroll
        for (int j = 0; j < RB; ++j)
          if (i & (1 << j)) u ^= sw[j];
        s[u] = v[i];
      }
      __syncthreads();
    }

    // ---- store ----
    const uint32_t total = (uint32_t)nvalid << t;
    if (fast) {
#pragma unroll
      for (int k = 0; k < NR; ++k) {
        const int j = a.item_of[k];
        if (j < nvalid) dst[in.dst[j] + (int64_t)(dep_tid | a.elem_off[k])] = s[fast_pos(k)];
      }
    } else if (contiguous && t >= 1) {
      for (uint32_t e = 2 * tid; e < total; e += 2 * blockDim.x) {
        const int j = (int)(e >> t);
        const uint32_t u = e & tmask;
        const C v0 = s[pad32(e)], v1 = s[pad32(e + 1)];
        C *gp = dst + in.dst[j] + u;
        if constexpr (sizeof(C) == 8) {
          float4 q;
          q.x = v0.x; q.y = v0.y; q.z = v1.x; q.w = v1.y;
          *reinterpret_cast<float4 *>(gp) = q;
        } else {
          gp[0] = v0;
          gp[1] = v1;
        }
      }
    } else {
      for (uint32_t e = tid; e < total; e += blockDim.x) {
        const int j = (int)(e >> t);
        const uint32_t u = e & tmask;
        dst[in.dst[j] + (int64_t)(contiguous ? u : deposit(u, a.active_mask))] = s[pad32(e)];
      }
    }
    __syncthreads();
  }
}

}  // namespace

cudaError_t launch_sweep(const SweepArgs &args, int precision, cudaStream_t st) {
  if (args.num_nodes <= 0) return cudaSuccess;
  const int64_t items = args.num_nodes * (int64_t)args.tiles_per_node;
  const int T = precision == 0 ? kRegTileC64 : kRegTileC128;
  if (args.groups && args.t >= args.rbits && args.t >= T - 6) {
    // element k of a thread (element tid + k * 2^L of the tile buffer, L = T - rbits)
    SweepArgs a = args;
    const int L = T - a.rbits, nk = 1 << a.rbits;
    for (int k = 0; k < 32; ++k) {
      a.elem_off[k] = 0;
      a.item_of[k] = 255;
    }
    if (a.t >= L)
      for (int k = 0; k < nk && k < 32; ++k) {
        const uint64_t within = (uint64_t)(k & ((1 << (a.t - L)) - 1)) << L;   // tile-local bits >= L
        uint64_t dep = 0, m = a.active_mask;
        for (int b = 0; m; ++b, m &= m - 1)
          if ((within >> b) & 1ull) dep |= m & (~m + 1);
        a.elem_off[k] = dep;
        a.item_of[k] = (uint8_t)(k >> (a.t - L));
      }
    const int64_t ipc = 1ll << (T - a.t);
    const int64_t ctas = (items + ipc - 1) / ipc;
    const int grid = (int)(ctas < (1 << 20) ? ctas : (1 << 20));
    const size_t smem = 2 * (size_t)(1u << T) * (precision == 0 ? 8 : 16) + (size_t)a.stage_bytes;
    if (precision == 0) {
      auto k = a.rbits == 5   ? sweep_reg_kernel<float, 5, kRegTileC64>
               : a.rbits == 3 ? sweep_reg_kernel<float, 3, kRegTileC64>
                              : sweep_reg_kernel<float, kRegBitsC64, kRegTileC64>;
      const int threads = 1 << (kRegTileC64 - a.rbits);
      cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      k<<<grid, threads, smem, st>>>(a);
    } else {
      auto k = sweep_reg_kernel<double, kRegBitsC128, kRegTileC128>;
      cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      k<<<grid, kSweepThreads, smem, st>>>(a);
    }
    return cudaGetLastError();
  }
  const SweepArgs &a = args;
  const int grid = (int)(items < (1 << 20) ? items : (1 << 20));
  if (precision == 0) {
    const size_t smem = (size_t)8 << a.t;
    cudaError_t e = cudaFuncSetAttribute(sweep_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    sweep_kernel<float><<<grid, 256, smem, st>>>(a);
  } else {
    const size_t smem = (size_t)16 << a.t;
    cudaError_t e = cudaFuncSetAttribute(sweep_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    sweep_kernel<double><<<grid, 256, smem, st>>>(a);
  }
  return cudaGetLastError();
}

}  // namespace hsf
