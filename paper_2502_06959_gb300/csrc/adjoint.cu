// Adjoint (reverse-mode) gradients of a real loss of the amplitudes with respect to
// shared rotation angles, through every path of the HSF sum (Sec. II-B).
//
// With c_s = conj(dL/d amp_s) (the upstream gradient g_s = dL/dRe + i dL/dIm, conjugated
// here), dL/dtheta = Re sum_s c_s d amp_s / dtheta.  Because amp_s = sum_p psi_a^p(x_a)
// psi_b^p(x_b), the a side of path p receives the cotangent
//   mu_a^p(y) = sum_{s : x_a(s) = y} c_s psi_b^p(x_b(s))          (leaf_cot_kernel)
// and symmetrically for b.  Cotangents are pulled back through each half circuit:
// for an op G applied to state psi_k (after the op), mu_{k-1} = G^T mu_k, psi_{k-1} =
// G^dagger psi_k (unitary ops only: the Schmidt factors are never inverted -- the
// walk stops there and resumes from the parent's stored state), and a rotation
// G = exp(-i t P/2) adds Re <mu_k, K psi_k> with K = dG/dt G^-1 = -i P/2
// (adjoint_kernel).  At a tree level the children's cotangents reach the parent through
// the transposed factors, summed over the digits (factor_pullback_kernel), which
// reuses the parent state like the forward prefix sharing.
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
template <typename C> __device__ __forceinline__ C cconj(C a) {
  a.y = -a.y;
  return a;
}

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
  return ((v >> b) << (b + 1)) | (v & ((1u << b) - 1u));
}

// Entry (r, c) of G (mode 0), G^dagger (mode 1) or G^T (mode 2) for a dense op.
template <typename C>
__device__ __forceinline__ C mat_entry(const C *m, int dim, int r, int c, int mode) {
  if (mode == 0) return m[r * dim + c];
  if (mode == 1) return cconj(m[c * dim + r]);
  return m[c * dim + r];
}

// Apply one op (or its dagger / transpose) to a shared-memory tile.
template <typename R>
__device__ void apply_tile(typename CT<R>::T *s, uint32_t tile_elems, const DevOp &op,
                           const typename CT<R>::T *m, int mode, uint64_t base) {
  using C = typename CT<R>::T;
  if (op.type == OP_DIAG) {
    for (uint32_t u = threadIdx.x; u < tile_elems; u += blockDim.x) {
      int idx = 0;
      for (int j = 0; j < op.nq; ++j) {
        const int p = op.pos[j];
        const int bit = p >= kFixedBit ? (int)((base >> (p - kFixedBit)) & 1ull) : (int)((u >> p) & 1u);
        idx = (idx << 1) | bit;
      }
      const C d = mode == 1 ? cconj(m[idx]) : m[idx];
      s[u] = cmul(d, s[u]);
    }
  } else {
    const int nq = op.nq, dim = 1 << nq;
    int sorted[3] = {op.pos[0], op.pos[1], op.pos[2]};
    for (int x = 0; x < nq; ++x)
      for (int y = x + 1; y < nq; ++y)
        if (sorted[y] < sorted[x]) { int t = sorted[x]; sorted[x] = sorted[y]; sorted[y] = t; }
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
        for (int c = 0; c < dim; ++c) {
          const C e = mat_entry(m, dim, r, c, mode);
          acc.x += e.x * v[c].x - e.y * v[c].y;
          acc.y += e.x * v[c].y + e.y * v[c].x;
        }
        s[addr[r]] = acc;
      }
    }
  }
  __syncthreads();
}

// Re sum_u mu(u) (K psi)(u) over the tile, K dense or diagonal on the op's qubits.
template <typename R>
__device__ double kdot_tile(const typename CT<R>::T *psi, const typename CT<R>::T *mu, uint32_t tile_elems,
                            const DevOp &op, const typename CT<R>::T *k, uint64_t base, double *red) {
  using C = typename CT<R>::T;
  double acc = 0.0;
  const int nq = op.nq, dim = 1 << nq;
  for (uint32_t u = threadIdx.x; u < tile_elems; u += blockDim.x) {
    int row = 0;
    for (int j = 0; j < nq; ++j) {
      const int p = op.pos[j];
      const int bit = p >= kFixedBit ? (int)((base >> (p - kFixedBit)) & 1ull) : (int)((u >> p) & 1u);
      row = (row << 1) | bit;
    }
    C kp;
    if (op.type == OP_DIAG) {
      kp = cmul(k[row], psi[u]);
    } else {
      kp.x = R(0);
      kp.y = R(0);
      uint32_t b0 = u;
      for (int j = 0; j < nq; ++j) b0 &= ~(1u << op.pos[j]);
      for (int c = 0; c < dim; ++c) {
        uint32_t ad = b0;
        for (int j = 0; j < nq; ++j)
          if ((c >> (nq - 1 - j)) & 1) ad |= 1u << op.pos[j];
        const C t = cmul(k[row * dim + c], psi[ad]);
        kp.x += t.x;
        kp.y += t.y;
      }
    }
    const C w = cmul(mu[u], kp);
    acc += (double)w.x;
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  double tot = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += red[w];
  __syncthreads();
  return tot;
}

// One op of at most two qubits undone on both tiles in a single pass, with the
// gradient term first: g += Re sum_u mu(u) (K psi)(u), then psi <- G^dagger psi and
// mu <- G^T mu (the same three steps as kdot_tile + two apply_tile, one sweep over the
// tile and one barrier).  The op's G^dagger, G^T and K are staged in shared memory
// first.  Dense ops act on tile bits; a diagonal op's bits may be fixed bits of the tile.
template <typename R, int NQ, bool DIAG>
__device__ double fused_op(typename CT<R>::T *psi, typename CT<R>::T *mu, uint32_t tile_elems, const DevOp &op,
                           const typename CT<R>::T *mats, uint64_t base, double *red, typename CT<R>::T *sm) {
  using C = typename CT<R>::T;
  constexpr int DIM = 1 << NQ;
  constexpr int E = DIAG ? DIM : DIM * DIM;
  const bool grad = op.param >= 0;
  const C *m = mats + op.mat;
  C *gd = sm, *gt = sm + 16, *kk = sm + 32;
  if (threadIdx.x < E) {
    const int e = threadIdx.x;
    const int src = DIAG ? e : (e % DIM) * DIM + e / DIM;     // (r, c) <- (c, r)
    gd[e] = cconj(m[src]);
    gt[e] = m[src];
    if (grad) kk[e] = mats[op.kmat + e];
  }
  __syncthreads();
  double acc = 0.0;
  if constexpr (DIAG) {
    for (uint32_t u = threadIdx.x; u < tile_elems; u += blockDim.x) {
      int idx = 0;
#pragma unroll
      for (int j = 0; j < NQ; ++j) {
        const int p = op.pos[j];
        const int bit = p >= kFixedBit ? (int)((base >> (p - kFixedBit)) & 1ull) : (int)((u >> p) & 1u);
        idx = (idx << 1) | bit;
      }
      const C x = psi[u], y = mu[u];
      if (grad) acc += (double)cmul(y, cmul(kk[idx], x)).x;
      psi[u] = cmul(gd[idx], x);
      mu[u] = cmul(gt[idx], y);
    }
  } else {
    int lo = op.pos[0], hi = NQ == 2 ? op.pos[1] : 0;
    if (NQ == 2 && lo > hi) {
      const int t = lo;
      lo = hi;
      hi = t;
    }
    for (uint32_t j = threadIdx.x; j < (tile_elems >> NQ); j += blockDim.x) {
      uint32_t i = insert_zero(j, lo);
      if (NQ == 2) i = insert_zero(i, hi);
      uint32_t addr[DIM];
      C x[DIM], y[DIM];
#pragma unroll
      for (int k = 0; k < DIM; ++k) {
        uint32_t ad = i;
#pragma unroll
        for (int q = 0; q < NQ; ++q)
          if ((k >> (NQ - 1 - q)) & 1) ad |= 1u << op.pos[q];
        addr[k] = ad;
        x[k] = psi[ad];
        y[k] = mu[ad];
      }
      if (grad) {
#pragma unroll
        for (int r = 0; r < DIM; ++r) {
          C kp;
          kp.x = R(0);
          kp.y = R(0);
#pragma unroll
          for (int c = 0; c < DIM; ++c) {
            const C t = cmul(kk[r * DIM + c], x[c]);
            kp.x += t.x;
            kp.y += t.y;
          }
          acc += (double)cmul(y[r], kp).x;
        }
      }
#pragma unroll
      for (int r = 0; r < DIM; ++r) {
        C np, nm;
        np.x = np.y = nm.x = nm.y = R(0);
#pragma unroll
        for (int c = 0; c < DIM; ++c) {
          const C a = cmul(gd[r * DIM + c], x[c]), b = cmul(gt[r * DIM + c], y[c]);
          np.x += a.x;
          np.y += a.y;
          nm.x += b.x;
          nm.y += b.y;
        }
        psi[addr[r]] = np;
        mu[addr[r]] = nm;
      }
    }
  }
  double tot = 0.0;
  if (grad) {
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  }
  __syncthreads();
  if (grad && threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += red[w];
  return tot;
}

template <typename R>
__global__ void __launch_bounds__(256, sizeof(R) == 4 ? 2 : 1) adjoint_kernel(AdjointArgs a) {
  using C = typename CT<R>::T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const uint32_t tile_elems = 1u << a.t;
  C *psi = reinterpret_cast<C *>(smem_raw);
  C *mu = psi + tile_elems;
  __shared__ double red[8];
  __shared__ C sm[48];                         // the current op's G^dagger, G^T and K
  const bool contiguous = a.active_mask == ((1ull << a.t) - 1ull);
  const uint64_t full = (1ull << a.h) - 1ull;
  const uint64_t inactive = full & ~a.active_mask;
  const C *mats = reinterpret_cast<const C *>(a.mats);
  const uint64_t state = 1ull << a.h;
  const int64_t items = a.num_nodes * (int64_t)a.tiles_per_node;
  for (int64_t item = blockIdx.x; item < items; item += gridDim.x) {
    const int64_t nl = item / a.tiles_per_node;
    const uint64_t base = deposit((uint64_t)(item % a.tiles_per_node), inactive);
    C *gpsi = reinterpret_cast<C *>(a.psi) + (uint64_t)nl * state;
    C *gmu = reinterpret_cast<C *>(a.mu) + (uint64_t)nl * state;
    for (uint32_t u = threadIdx.x; u < tile_elems; u += blockDim.x) {
      const uint64_t off = base | (contiguous ? (uint64_t)u : deposit(u, a.active_mask));
      psi[u] = gpsi[off];
      mu[u] = gmu[off];
    }
    __syncthreads();
    for (int o = a.num_ops - 1; o >= a.first_op; --o) {
      const DevOp op = a.ops[o];
      const C *m = mats + op.mat;
      double g = 0.0;
      if (op.nq == 1) {
        g = op.type == OP_DIAG ? fused_op<R, 1, true>(psi, mu, tile_elems, op, mats, base, red, sm)
                               : fused_op<R, 1, false>(psi, mu, tile_elems, op, mats, base, red, sm);
      } else if (op.nq == 2) {
        g = op.type == OP_DIAG ? fused_op<R, 2, true>(psi, mu, tile_elems, op, mats, base, red, sm)
                               : fused_op<R, 2, false>(psi, mu, tile_elems, op, mats, base, red, sm);
      } else {
        if (op.param >= 0) g = kdot_tile<R>(psi, mu, tile_elems, op, mats + op.kmat, base, red);
        apply_tile<R>(psi, tile_elems, op, m, 1, base);   // psi <- G^dagger psi
        apply_tile<R>(mu, tile_elems, op, m, 2, base);    // mu  <- G^T mu
      }
      if (op.param >= 0 && threadIdx.x == 0) atomicAdd(a.grad + op.param, g);
    }
    for (uint32_t u = threadIdx.x; u < tile_elems; u += blockDim.x) {
      const uint64_t off = base | (contiguous ? (uint64_t)u : deposit(u, a.active_mask));
      gpsi[off] = psi[u];
      gmu[off] = mu[u];
    }
    __syncthreads();
  }
}

// mu_a^p(x_a(s)) += c_s psi_b^p(x_b(s)) and mu_b^p(x_b(s)) += c_s psi_a^p(x_a(s)).
template <typename R>
__global__ void leaf_cot_kernel(LeafCotArgs a) {
  using C = typename CT<R>::T;
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t p = blockIdx.y + (int64_t)gridDim.y * blockIdx.z;
  if (s >= a.S || p >= a.paths) return;
  const double2 g = reinterpret_cast<const double2 *>(a.gout)[s];
  C c;
  c.x = (R)g.x;
  c.y = (R)-g.y;                       // c_s = conj(g_s)
  const uint64_t ia = a.ia[s], ib = a.ib[s];
  const C *A = reinterpret_cast<const C *>(a.psi_a) + ((uint64_t)p << a.ha);
  const C *B = reinterpret_cast<const C *>(a.psi_b) + ((uint64_t)p << a.hb);
  C *MA = reinterpret_cast<C *>(a.mu_a) + ((uint64_t)p << a.ha);
  C *MB = reinterpret_cast<C *>(a.mu_b) + ((uint64_t)p << a.hb);
  const C ta = cmul(c, B[ib]), tb = cmul(c, A[ia]);
  atomicAdd(&MA[ia].x, ta.x);
  atomicAdd(&MA[ia].y, ta.y);
  atomicAdd(&MB[ib].x, tb.x);
  atomicAdd(&MB[ib].y, tb.y);
}

// mu_parent(y) = sum_m sum_y' X_m[y'_F, y_F] mu_child_m(y with F <- y')  (X_m^T mu).
template <typename R>
__global__ void factor_pullback_kernel(PullbackArgs a) {
  using C = typename CT<R>::T;
  const uint64_t state = 1ull << a.h;
  const uint64_t y = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t j = blockIdx.y + (int64_t)gridDim.y * blockIdx.z;   // parent within the level
  if (y >= state || j >= a.num_parents) return;
  const int dim = 1 << a.nf;
  uint64_t fmask = 0;
  int row = 0;
  for (int x = 0; x < a.nf; ++x) {
    fmask |= 1ull << a.fq[x];
    row = (row << 1) | (int)((y >> a.fq[x]) & 1ull);
  }
  const C *X = reinterpret_cast<const C *>(a.factor);
  const C *mc = reinterpret_cast<const C *>(a.mu_child);
  C acc;
  acc.x = R(0);
  acc.y = R(0);
  const int64_t first_child = (a.parent_lo + j) * a.radix - a.child_lo;
  for (int m = 0; m < a.radix; ++m) {
    const int64_t ch = first_child + m;
    if (ch < 0 || ch >= a.num_children) continue;
    const C *Xm = X + (size_t)m * dim * dim;
    const C *mu = mc + (uint64_t)ch * state;
    for (int yp = 0; yp < dim; ++yp) {
      uint64_t src = y & ~fmask;
      for (int x = 0; x < a.nf; ++x)
        if ((yp >> (a.nf - 1 - x)) & 1) src |= 1ull << a.fq[x];
      const C t = cmul(Xm[yp * dim + row], mu[src]);
      acc.x += t.x;
      acc.y += t.y;
    }
  }
  reinterpret_cast<C *>(a.mu_parent)[(uint64_t)j * state + y] = acc;
}

// grad[j] += Re sum_s conj(g_s) amp'_s
__global__ void grad_dot_kernel(const double *gout, const double *ampd, int64_t S, double *grad) {
  __shared__ double red[8];
  double acc = 0.0;
  for (int64_t s = threadIdx.x; s < S; s += blockDim.x)
    acc += gout[2 * s] * ampd[2 * s] + gout[2 * s + 1] * ampd[2 * s + 1];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    *grad += t;
  }
}

__global__ void zero_bytes_kernel(uint32_t *p, int64_t words) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < words) p[i] = 0u;
}

}  // namespace

cudaError_t launch_adjoint(const AdjointArgs &a, int precision, cudaStream_t st) {
  if (a.num_nodes <= 0) return cudaSuccess;
  const int64_t items = a.num_nodes * (int64_t)a.tiles_per_node;
  const int grid = (int)(items < (1 << 20) ? items : (1 << 20));
  const size_t smem = (size_t)2 * (precision == 0 ? 8 : 16) << a.t;
  if (precision == 0) {
    cudaError_t e = cudaFuncSetAttribute(adjoint_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    adjoint_kernel<float><<<grid, 256, smem, st>>>(a);
  } else {
    cudaError_t e = cudaFuncSetAttribute(adjoint_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    adjoint_kernel<double><<<grid, 256, smem, st>>>(a);
  }
  return cudaGetLastError();
}

cudaError_t launch_leaf_cot(const LeafCotArgs &a, int precision, cudaStream_t st) {
  if (a.S <= 0 || a.paths <= 0) return cudaSuccess;
  const unsigned gy = (unsigned)(a.paths < 65535 ? a.paths : 65535);
  dim3 grid((unsigned)((a.S + 255) / 256), gy, (unsigned)((a.paths + gy - 1) / gy));
  if (precision == 0)
    leaf_cot_kernel<float><<<grid, 256, 0, st>>>(a);
  else
    leaf_cot_kernel<double><<<grid, 256, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_factor_pullback(const PullbackArgs &a, int precision, cudaStream_t st) {
  if (a.num_parents <= 0) return cudaSuccess;
  const uint64_t state = 1ull << a.h;
  const unsigned gy = (unsigned)(a.num_parents < 65535 ? a.num_parents : 65535);
  dim3 grid((unsigned)((state + 255) / 256), gy, (unsigned)((a.num_parents + gy - 1) / gy));
  if (precision == 0)
    factor_pullback_kernel<float><<<grid, 256, 0, st>>>(a);
  else
    factor_pullback_kernel<double><<<grid, 256, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_grad_dot(const double *gout, const double *ampd, int64_t S, double *grad, cudaStream_t st) {
  grad_dot_kernel<<<1, 256, 0, st>>>(gout, ampd, S, grad);
  return cudaGetLastError();
}

cudaError_t launch_zero_bytes(void *p, size_t bytes, cudaStream_t st) {
  const int64_t words = (int64_t)(bytes / 4);
  if (words <= 0) return cudaSuccess;
  zero_bytes_kernel<<<(unsigned)((words + 255) / 256), 256, 0, st>>>(reinterpret_cast<uint32_t *>(p), words);
  return cudaGetLastError();
}

}  // namespace hsf
