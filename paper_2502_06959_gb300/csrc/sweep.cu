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

}  // namespace

cudaError_t launch_sweep(const SweepArgs &a, int precision, cudaStream_t st) {
  if (a.num_nodes <= 0) return cudaSuccess;
  const int64_t items = a.num_nodes * (int64_t)a.tiles_per_node;
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
