// Block product and Schmidt decomposition of jointly cut blocks, FP64 on device
// (Sec. IV-A and IV-C: "merging a block of gates into one requires consecutive matrix
// multiplications first and afterwards a Schmidt Decomposition").
//
// One CTA per block:
//   1. U_B = G_T ... G_1 on the block's k <= 6 qubits (columns updated in parallel).
//   2. Relabel A~_{(i^b j^b),(i^a j^a)} = U_B[(i^a i^b),(j^a j^b)]  (eq. for A~).
//   3. SVD of A~ by the one-sided (Hestenes) Jacobi method: pairs of columns are
//      rotated by 2x2 unitaries until all columns are mutually orthogonal; the
//      column norms are the singular values and the accumulated rotations give V
//      (eq. eq-svd: A~ = U Sigma V^H).  Pairs are scheduled with the round-robin
//      (circle) ordering so that the Nw/2 pairs of one round are disjoint; one warp
//      handles one pair.  The working matrix is A~ or A~^H, whichever has fewer
//      columns.
//   4. Keep sigma_m > rank_tol * sigma_0 and emit the Schmidt factors with sqrt(sigma_m)
//      folded into both sides: X'_m = sqrt(s) X_m, Y'_m = sqrt(s) Y_m where
//      X_m[i^a, j^a] = conj(V[(i^a j^a), m]) and Y_m[i^b, j^b] = U[(i^b j^b), m].
//   5. Reconstruction check: the largest entry of |U_B - sum_m X'_m (x) Y'_m| over the
//      kept terms (eq. equ-schmidt-decompostion-res), for the host to accept or reject.
// The sweep count is bounded (max_sweeps); the kernel never waits on anything.
#include <algorithm>
#include <cstdint>

#include "common.h"

namespace hsf {
namespace {

constexpr int kMaxDim = 64;        // 2^k for k <= 6; also 4^k_a, 4^k_b for k_side <= 3
constexpr int kThreads = 1024;

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__global__ void __launch_bounds__(kThreads) block_svd_kernel(BlockSvdArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  // sized by the launch for its largest block (a small block needs a few hundred bytes,
  // so the CTA fits beside other kernels' CTAs on a busy SM)
  double2 *U = reinterpret_cast<double2 *>(smem_raw);          // D x D, row-major
  double2 *W = U + a.off_w;                                     // Mw x Nw, column-major
  double2 *V = U + a.off_v;                                     // Nw x Nw, column-major
  __shared__ double sig[kMaxDim];
  __shared__ int order[kMaxDim];
  __shared__ int rotated;
  __shared__ double fro2;

  const int b = blockIdx.x;
  const int k = a.block_k[3 * b], ka = a.block_k[3 * b + 1], kb = a.block_k[3 * b + 2];
  const int D = 1 << k;
  const int tid = threadIdx.x;

  // 1. block product (a sum of products when the block has several terms, e.g. the
  //    product rule of a derivative); the running sum is kept in W
  const int t0 = a.term_begin[b], t1 = a.term_begin[b + 1];
  for (int term = t0; term < t1; ++term) {
  for (int e = tid; e < D * D; e += blockDim.x)
    U[e] = make_double2((e / D) == (e % D) ? 1.0 : 0.0, 0.0);
  __syncthreads();
  for (int gi = a.gate_begin[term]; gi < a.gate_begin[term + 1]; ++gi) {
    const int *gd = a.gate_desc + 5 * gi;
    const int nq = gd[0];
    const int pos[3] = {gd[1], gd[2], gd[3]};
    const double2 *m = reinterpret_cast<const double2 *>(a.gate_mats) + gd[4];
    const int dim = 1 << nq;
    int mask = 0;
    for (int x = 0; x < nq; ++x) mask |= 1 << pos[x];
    const int groups = D >> nq;
    for (int w = tid; w < D * groups; w += blockDim.x) {
      const int col = w / groups;
      int g = w % groups;
      // base row index: the bits outside the gate taken from g in order
      int base = 0, src = 0;
      for (int bit = 0; bit < k; ++bit) {
        if (mask & (1 << bit)) continue;
        if (g & (1 << src)) base |= 1 << bit;
        ++src;
      }
      double2 v[8];
      int rows[8];
      for (int s = 0; s < dim; ++s) {
        int r = base;
        for (int x = 0; x < nq; ++x)
          if ((s >> (nq - 1 - x)) & 1) r |= 1 << pos[x];
        rows[s] = r;
        v[s] = U[r * D + col];
      }
      for (int s = 0; s < dim; ++s) {
        double2 acc = make_double2(0.0, 0.0);
        for (int c = 0; c < dim; ++c) {
          const double2 p = cmul(m[s * dim + c], v[c]);
          acc.x += p.x;
          acc.y += p.y;
        }
        U[rows[s] * D + col] = acc;
      }
    }
    __syncthreads();
  }
  if (t1 - t0 > 1) {
    for (int e = tid; e < D * D; e += blockDim.x) {
      const double2 prev = term == t0 ? make_double2(0.0, 0.0) : W[e];
      W[e] = make_double2(prev.x + U[e].x, prev.y + U[e].y);
    }
    __syncthreads();
  }
  }
  if (t1 - t0 > 1) {
    for (int e = tid; e < D * D; e += blockDim.x) U[e] = W[e];
    __syncthreads();
  }

  // 2. relabel: A~ has M = 4^kb rows (i^b, j^b) and N = 4^ka columns (i^a, j^a)
  const int M = 1 << (2 * kb), N = 1 << (2 * ka);
  const bool swapped = N > M;
  const int Mw = swapped ? N : M, Nw = swapped ? M : N;
  const int db = 1 << kb, da = 1 << ka;
  for (int e = tid; e < M * N; e += blockDim.x) {
    const int row = e / N, col = e % N;           // row = ib*db + jb, col = ia*da + ja
    const int ib = row / db, jb = row % db, ia = col / da, ja = col % da;
    const double2 val = U[((ia << kb) | ib) * D + ((ja << kb) | jb)];
    if (!swapped)
      W[col * Mw + row] = val;
    else
      W[row * Mw + col] = cconj(val);             // W = A~^H: W[r'=col][c'=row]
  }
  for (int e = tid; e < Nw * Nw; e += blockDim.x)
    V[e] = make_double2((e / Nw) == (e % Nw) ? 1.0 : 0.0, 0.0);
  if (tid == 0) {
    double f = 0.0;
    for (int e = 0; e < Mw * Nw; ++e) f += W[e].x * W[e].x + W[e].y * W[e].y;
    fro2 = f;
  }
  __syncthreads();

  // 3. one-sided Jacobi
  const int warp = tid >> 5, lane = tid & 31;
  int sweep = 0;
  for (; sweep < a.max_sweeps; ++sweep) {
    if (tid == 0) rotated = 0;
    __syncthreads();
    for (int round = 0; round < Nw - 1; ++round) {
      if (warp < Nw / 2) {
        int p, q;
        if (warp == 0) {
          p = 0;
          q = 1 + (round % (Nw - 1));
        } else {
          p = 1 + ((warp + round) % (Nw - 1));
          q = 1 + ((Nw - 1 - warp + round) % (Nw - 1));
        }
        double2 *wp = W + p * Mw, *wq = W + q * Mw;
        double al = 0.0, be = 0.0, gr = 0.0, gi = 0.0;
        for (int r = lane; r < Mw; r += 32) {
          const double2 x = wp[r], y = wq[r];
          al += x.x * x.x + x.y * x.y;
          be += y.x * y.x + y.y * y.y;
          gr += x.x * y.x + x.y * y.y;               // conj(x) * y
          gi += x.x * y.y - x.y * y.x;
        }
        al = warp_sum(al);
        be = warp_sum(be);
        gr = warp_sum(gr);
        gi = warp_sum(gi);
        const double ag = sqrt(gr * gr + gi * gi);
        // rotate while the columns' cosine is above 1e-14 (the rounding of a 64-term
        // complex dot product sits near 1e-15, so a lower threshold never stops) and both
        // columns are above round-off of the whole matrix: a column of norm below
        // 1e-14 |A~|_F is numerically zero (its sigma is dropped by any rank threshold
        // above 1e-14), and its noise would otherwise keep rotating
        if (ag > 1e-14 * sqrt(al * be) && fmin(al, be) > 1e-28 * fro2 && ag > 1e-300) {
          const double zeta = (be - al) / (2.0 * ag);
          const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
          const double c = 1.0 / sqrt(1.0 + t * t), s = c * t;
          const double2 ph = make_double2(gr / ag, gi / ag);      // e^{i phi}
          const double2 sph = make_double2(s * ph.x, s * ph.y);    // s e^{i phi}
          const double2 sphc = cconj(sph);                         // s e^{-i phi}
          for (int r = lane; r < Mw; r += 32) {
            const double2 x = wp[r], y = wq[r];
            const double2 a1 = cmul(sphc, y), a2 = cmul(sph, x);
            wp[r] = make_double2(c * x.x - a1.x, c * x.y - a1.y);
            wq[r] = make_double2(a2.x + c * y.x, a2.y + c * y.y);
          }
          double2 *vp = V + p * Nw, *vq = V + q * Nw;
          for (int r = lane; r < Nw; r += 32) {
            const double2 x = vp[r], y = vq[r];
            const double2 a1 = cmul(sphc, y), a2 = cmul(sph, x);
            vp[r] = make_double2(c * x.x - a1.x, c * x.y - a1.y);
            vq[r] = make_double2(a2.x + c * y.x, a2.y + c * y.y);
          }
          if (lane == 0) rotated = 1;
        }
      }
      __syncthreads();
    }
    if (!rotated) break;
    __syncthreads();
  }

  // 4. singular values, ordering, rank, factors
  for (int j = warp; j < Nw; j += blockDim.x / 32) {
    double acc = 0.0;
    for (int r = lane; r < Mw; r += 32) {
      const double2 x = W[j * Mw + r];
      acc += x.x * x.x + x.y * x.y;
    }
    acc = warp_sum(acc);
    if (lane == 0) sig[j] = sqrt(acc);
  }
  __syncthreads();
  if (tid == 0) {
    for (int j = 0; j < Nw; ++j) order[j] = j;
    for (int x = 0; x < Nw; ++x)
      for (int y = x + 1; y < Nw; ++y)
        if (sig[order[y]] > sig[order[x]]) { int tmp = order[x]; order[x] = order[y]; order[y] = tmp; }
    const double s0 = sig[order[0]];
    int r = 0;
    for (int j = 0; j < Nw; ++j)
      if (s0 > 0.0 && sig[order[j]] > a.rank_tol * s0) ++r;
    a.rank[b] = r;
    a.sweeps_used[b] = sweep;
    for (int m = 0; m < kMaxDim; ++m) a.sigma[b * kMaxDim + m] = m < Nw ? sig[order[m]] : 0.0;
  }
  __syncthreads();
  const int rank = a.rank[b];
  double2 *xf = reinterpret_cast<double2 *>(a.xf) + (size_t)b * kMaxDim * kMaxDim;
  double2 *yf = reinterpret_cast<double2 *>(a.yf) + (size_t)b * kMaxDim * kMaxDim;
  for (int e = tid; e < rank * kMaxDim; e += blockDim.x) {
    const int m = e / kMaxDim, idx = e % kMaxDim;
    const int j = order[m];
    const double s = sig[j], rs = sqrt(s);
    if (!swapped) {
      // Y'_m = W_j / sqrt(s)   (index (i^b, j^b), M entries)
      // X'_m = sqrt(s) conj(V_j) (index (i^a, j^a), N entries)
      if (idx < M) {
        const double2 w = W[j * Mw + idx];
        yf[m * kMaxDim + idx] = make_double2(w.x / rs, w.y / rs);
      }
      if (idx < N) {
        const double2 v = V[j * Nw + idx];
        xf[m * kMaxDim + idx] = make_double2(rs * v.x, -rs * v.y);
      }
    } else {
      // A~ = V_w Sigma U_w^H: Y'_m = sqrt(s) V_j, X'_m = conj(W_j) / sqrt(s)
      if (idx < M) {
        const double2 v = V[j * Nw + idx];
        yf[m * kMaxDim + idx] = make_double2(rs * v.x, rs * v.y);
      }
      if (idx < N) {
        const double2 w = W[j * Mw + idx];
        xf[m * kMaxDim + idx] = make_double2(w.x / rs, -w.y / rs);
      }
    }
  }
  // 5. reconstruction residual against the block matrix (U is untouched since step 1)
  __shared__ unsigned long long res_bits;
  if (tid == 0) res_bits = 0ull;
  __syncthreads();
  const int rda = 1 << ka, rdb = 1 << kb;
  double worst = 0.0;
  for (int e = tid; e < D * D; e += blockDim.x) {
    const int row = e / D, col = e % D;
    const int ia = row >> kb, ib = row & (rdb - 1), ja = col >> kb, jb = col & (rdb - 1);
    double2 acc = make_double2(0.0, 0.0);
    for (int m = 0; m < rank; ++m) {
      const double2 x = xf[m * kMaxDim + ia * rda + ja], y = yf[m * kMaxDim + ib * rdb + jb];
      const double2 xy = cmul(x, y);
      acc.x += xy.x;
      acc.y += xy.y;
    }
    const double2 u = U[e];
    worst = fmax(worst, hypot(u.x - acc.x, u.y - acc.y));
  }
  atomicMax(&res_bits, (unsigned long long)__double_as_longlong(worst));   // non-negative: bit order
  __syncthreads();
  if (tid == 0) a.residual[b] = __longlong_as_double((long long)res_bits);
}

}  // namespace

cudaError_t launch_block_svd(const BlockSvdArgs &a, cudaStream_t st) {
  if (a.num_blocks <= 0) return cudaSuccess;
  // shared memory and threads for the largest block of the launch: U is D x D, the
  // working matrix Mw x Nw, V Nw x Nw; a Jacobi round uses Nw / 2 warps
  const size_t elems = (size_t)a.off_v + (size_t)a.max_nw * a.max_nw;
  const size_t smem = elems * sizeof(double2);
  const int threads = std::min(kThreads, std::max(128, 32 * (a.max_nw / 2)));
  cudaError_t e = cudaFuncSetAttribute(block_svd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  block_svd_kernel<<<a.num_blocks, threads, smem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace hsf
