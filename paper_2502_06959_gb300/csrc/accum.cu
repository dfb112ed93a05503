// Path accumulation (Sec. II-B: "applying the Kronecker product between the
// subcircuits per simulation and adding up all contributions"):
//   amp(x) = sum_p psi_a^p(x_a) * psi_b^p(x_b),   x = x_a * 2^{n_b} + x_b.
//
// * gather_dot: bitstring output.  One thread per bitstring walks a group of paths,
//   accumulating the products in the state precision; the per-group partial sums are
//   written in FP64 and folded into the output with Neumaier-compensated FP64
//   additions (reduce_partials), so cancellation across many path groups keeps
//   FP64 accuracy.
// * window: full / leading-window output as the rank-P complex product
//   Out[x_a, x_b] = sum_p L[p, x_a] R[p, x_b] on CUDA cores (FP32 or FP64), folded
//   into the FP64 output with the same compensation.
#include <algorithm>
#include <cstdint>

#include "common.h"

namespace hsf {
namespace {

template <typename R> struct CT;
template <> struct CT<float> { using T = float2; };
template <> struct CT<double> { using T = double2; };

__device__ __forceinline__ void neumaier_add(double &sum, double &c, double x) {
  const double t = sum + x;
  if (fabs(sum) >= fabs(x))
    c += (sum - t) + x;
  else
    c += (x - t) + sum;
  sum = t;
}

template <typename R>
__global__ void gather_dot_kernel(GatherArgs a) {
  using C = typename CT<R>::T;
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int g = blockIdx.y;
  if (s >= a.S) return;
  const uint64_t xa = a.ia[s], xb = a.ib[s];
  const C *A = reinterpret_cast<const C *>(a.A);
  const C *B = reinterpret_cast<const C *>(a.B);
  const int64_t p0 = (int64_t)g * a.paths_per_group;
  const int64_t p1 = min(a.num_paths, p0 + a.paths_per_group);
  R re = R(0), im = R(0);
  for (int64_t p = p0; p < p1; ++p) {
    const C u = A[((uint64_t)p << a.ha) | xa];
    const C v = B[((uint64_t)p << a.hb) | xb];
    re = fma(u.x, v.x, fma(-u.y, v.y, re));
    im = fma(u.x, v.y, fma(u.y, v.x, im));
  }
  double *dst = a.partial + 2 * ((int64_t)g * a.S + s);
  dst[0] = (double)re;
  dst[1] = (double)im;
}

// out[s] += sum_g partial[g][s] (compensated).  A CTA takes 32 bitstrings; its 8 rows of
// threads sum every 8th group each (Neumaier), and row 0 folds the 8 compensated pairs
// into the running output.
constexpr int kReduceRows = 8;
__global__ void __launch_bounds__(32 * kReduceRows) reduce_partials_kernel(const double *partial, int32_t num_groups,
                                                                           int64_t S, double *out, double *comp) {
  __shared__ double sh[kReduceRows][32][4];
  const int64_t s = (int64_t)blockIdx.x * 32 + threadIdx.x;
  const int y = threadIdx.y;
  double sr = 0.0, si = 0.0, cr = 0.0, ci = 0.0;
  if (s < S)
    for (int g = y; g < num_groups; g += kReduceRows) {
      const double2 v = reinterpret_cast<const double2 *>(partial)[(int64_t)g * S + s];
      neumaier_add(sr, cr, v.x);
      neumaier_add(si, ci, v.y);
    }
  sh[y][threadIdx.x][0] = sr;
  sh[y][threadIdx.x][1] = si;
  sh[y][threadIdx.x][2] = cr;
  sh[y][threadIdx.x][3] = ci;
  __syncthreads();
  if (y != 0 || s >= S) return;
  double tr = out[2 * s], ti = out[2 * s + 1];
  double kr = comp[2 * s], ki = comp[2 * s + 1];
  for (int r = 0; r < kReduceRows; ++r) {
    neumaier_add(tr, kr, sh[r][threadIdx.x][0]);
    neumaier_add(ti, ki, sh[r][threadIdx.x][1]);
    kr += sh[r][threadIdx.x][2];
    ki += sh[r][threadIdx.x][3];
  }
  out[2 * s] = tr;
  out[2 * s + 1] = ti;
  comp[2 * s] = kr;
  comp[2 * s + 1] = ki;
}

// 32x32 output tile per CTA, 256 threads, 4 outputs per thread, K staged by 16.
template <typename R>
__global__ void __launch_bounds__(256) window_kernel(WindowArgs a) {
  using C = typename CT<R>::T;
  __shared__ C As[16][32];
  __shared__ C Bs[16][32];
  const C *A = reinterpret_cast<const C *>(a.A);
  const C *B = reinterpret_cast<const C *>(a.B);
  const int64_t i0 = (int64_t)blockIdx.y * 32;
  const int64_t j0 = (int64_t)blockIdx.x * 32;
  const int tx = threadIdx.x & 31;        // column in tile
  const int ty = threadIdx.x >> 5;        // rows ty, ty+8, ty+16, ty+24
  R accr[4] = {0, 0, 0, 0}, acci[4] = {0, 0, 0, 0};
  for (int64_t p0 = 0; p0 < a.num_paths; p0 += 16) {
    for (int e = threadIdx.x; e < 16 * 32; e += 256) {
      const int kk = e >> 5, cc = e & 31;
      const int64_t p = p0 + kk;
      C va, vb;
      va.x = va.y = vb.x = vb.y = R(0);
      if (p < a.num_paths) {
        if (i0 + cc < a.M) va = A[((uint64_t)p << a.ha) + a.row_index[i0 + cc]];
        if (j0 + cc < a.N) vb = B[((uint64_t)p << a.hb) + a.col_index[j0 + cc]];
      }
      As[kk][cc] = va;
      Bs[kk][cc] = vb;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      const C vb = Bs[kk][tx];
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const C va = As[kk][ty + 8 * r];
        accr[r] = fma(va.x, vb.x, fma(-va.y, vb.y, accr[r]));
        acci[r] = fma(va.x, vb.y, fma(va.y, vb.x, acci[r]));
      }
    }
    __syncthreads();
  }
  for (int r = 0; r < 4; ++r) {
    const int64_t i = i0 + ty + 8 * r, j = j0 + tx;
    if (i >= a.M || j >= a.N) continue;
    const uint64_t idx = ((uint64_t)i << a.hb) + (uint64_t)j;
    if (idx >= a.window) continue;
    double sr = a.out[2 * idx], si = a.out[2 * idx + 1];
    double cr = a.comp[2 * idx], ci = a.comp[2 * idx + 1];
    neumaier_add(sr, cr, (double)accr[r]);
    neumaier_add(si, ci, (double)acci[r]);
    a.out[2 * idx] = sr;
    a.out[2 * idx + 1] = si;
    a.comp[2 * idx] = cr;
    a.comp[2 * idx + 1] = ci;
  }
}

// Leaf contraction.  Thread = bitstring s; it walks a group of parent nodes and, for
// each, reads the 2^C amplitudes of both parents around x_a(s) / x_b(s) (contiguous:
// the leaf level only touches the C lowest storage bits), applies row x(s) of every
// leaf operator L_m and accumulates sum_m (L^a_m phi_a)(x_a) (L^b_m phi_b)(x_b).
template <typename R, int CB>
__global__ void __launch_bounds__(128) leaf_contract_kernel(LeafArgs a) {
  using C = typename CT<R>::T;
  constexpr int D = 1 << CB;
  constexpr int LD = D + 1;                    // padded row stride (bank spread)
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C *La = reinterpret_cast<C *>(smem_raw);
  C *Lb = La + a.r * D * LD;
  const C *gLa = reinterpret_cast<const C *>(a.La), *gLb = reinterpret_cast<const C *>(a.Lb);
  for (int e = threadIdx.x; e < a.r * D * D; e += blockDim.x) {
    const int row = e / D, col = e % D;        // row runs over (m, row)
    La[row * LD + col] = gLa[e];
    Lb[row * LD + col] = gLb[e];
  }
  __syncthreads();
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= a.S) return;
  const int g = blockIdx.y;
  const uint64_t ia = a.ia[s], ib = a.ib[s];
  const int ra = (int)(ia & (D - 1)), rb = (int)(ib & (D - 1));
  const uint64_t ba = ia - ra, bb = ib - rb;
  const int64_t j0 = (int64_t)g * a.parents_per_group;
  const int64_t j1 = min(a.num_parents, j0 + a.parents_per_group);
  R accr = R(0), acci = R(0);
  for (int64_t j = j0; j < j1; ++j) {
    const int mlo = j == 0 ? a.m_first : 0;
    const int mhi = j == a.num_parents - 1 ? a.m_last : a.r;
    C x[D];
    const C *pa = reinterpret_cast<const C *>(a.Pa) + ((uint64_t)j << a.ha) + ba;
#pragma unroll
    for (int k = 0; k < D; ++k) x[k] = pa[k];
    C va[8];
#pragma unroll
    for (int m = 0; m < 8; ++m) {
      va[m].x = va[m].y = R(0);
      if (m < a.r) {
        const C *row = La + (m * D + ra) * LD;
#pragma unroll
        for (int k = 0; k < D; ++k) {
          const C l = row[k];
          va[m].x = fma(l.x, x[k].x, fma(-l.y, x[k].y, va[m].x));
          va[m].y = fma(l.x, x[k].y, fma(l.y, x[k].x, va[m].y));
        }
      }
    }
    const C *pb = reinterpret_cast<const C *>(a.Pb) + ((uint64_t)j << a.hb) + bb;
#pragma unroll
    for (int k = 0; k < D; ++k) x[k] = pb[k];
#pragma unroll
    for (int m = 0; m < 8; ++m) {
      if (m < mlo || m >= mhi) continue;
      const C *row = Lb + (m * D + rb) * LD;
      R vr = R(0), vi = R(0);
#pragma unroll
      for (int k = 0; k < D; ++k) {
        const C l = row[k];
        vr = fma(l.x, x[k].x, fma(-l.y, x[k].y, vr));
        vi = fma(l.x, x[k].y, fma(l.y, x[k].x, vi));
      }
      accr = fma(va[m].x, vr, fma(-va[m].y, vi, accr));
      acci = fma(va[m].x, vi, fma(va[m].y, vr, acci));
    }
  }
  double *dst = a.partial + 2 * ((int64_t)g * a.S + s);
  dst[0] = (double)accr;
  dst[1] = (double)acci;
}

// Leaf contraction, register variant (2^C <= 16 and r <= 8).  RM consecutive threads
// serve one bitstring, one Schmidt digit m each: the thread keeps row x_a(s) of L^a_m and
// row x_b(s) of L^b_m in registers for all parents of its group, reads the two chunks
// (shared by the RM threads, so one coalesced request), and the RM per-digit sums are
// added with shuffles at the end.
template <typename R, int CB, int RM>
__global__ void __launch_bounds__(128) leaf_contract_reg_kernel(LeafArgs a) {
  using C = typename CT<R>::T;
  constexpr int D = 1 << CB;
  constexpr int SPB = 128 / RM;                // bitstrings per CTA
  const int m = threadIdx.x % RM;
  const int64_t s = (int64_t)blockIdx.x * SPB + threadIdx.x / RM;
  const int g = blockIdx.y;
  const bool on = s < a.S && m < a.r;
  uint64_t ia = 0, ib = 0;
  if (s < a.S) {
    ia = a.ia[s];
    ib = a.ib[s];
  }
  const int ra = (int)(ia & (D - 1)), rb = (int)(ib & (D - 1));
  const uint64_t ba = ia - ra, bb = ib - rb;
  C la[D], lb[D];
  {
    const C *gLa = reinterpret_cast<const C *>(a.La) + ((size_t)(on ? m : 0) * D + ra) * D;
    const C *gLb = reinterpret_cast<const C *>(a.Lb) + ((size_t)(on ? m : 0) * D + rb) * D;
#pragma unroll
    for (int k = 0; k < D; ++k) {
      la[k] = gLa[k];
      lb[k] = gLb[k];
    }
  }
  const int64_t j0 = (int64_t)g * a.parents_per_group;
  const int64_t j1 = min(a.num_parents, j0 + a.parents_per_group);
  R accr = R(0), acci = R(0);
  if (on) {
    for (int64_t j = j0; j < j1; ++j) {
      if ((j == 0 && m < a.m_first) || (j == a.num_parents - 1 && m >= a.m_last)) continue;
      const C *pa = reinterpret_cast<const C *>(a.Pa) + ((uint64_t)j << a.ha) + ba;
      const C *pb = reinterpret_cast<const C *>(a.Pb) + ((uint64_t)j << a.hb) + bb;
      // both chunks are requested before any arithmetic (16-byte loads: the chunks
      // start at multiples of 2^C amplitudes)
      C xa[D], xb[D];
      if constexpr (sizeof(C) == 8 && D >= 2) {
#pragma unroll
        for (int k = 0; k < D; k += 2) {
          const float4 qa = *reinterpret_cast<const float4 *>(pa + k);
          const float4 qb = *reinterpret_cast<const float4 *>(pb + k);
          xa[k].x = qa.x; xa[k].y = qa.y; xa[k + 1].x = qa.z; xa[k + 1].y = qa.w;
          xb[k].x = qb.x; xb[k].y = qb.y; xb[k + 1].x = qb.z; xb[k + 1].y = qb.w;
        }
      } else {
#pragma unroll
        for (int k = 0; k < D; ++k) {
          xa[k] = pa[k];
          xb[k] = pb[k];
        }
      }
      R var = R(0), vai = R(0), vbr = R(0), vbi = R(0);
#pragma unroll
      for (int k = 0; k < D; ++k) {
        var = fma(la[k].x, xa[k].x, fma(-la[k].y, xa[k].y, var));
        vai = fma(la[k].x, xa[k].y, fma(la[k].y, xa[k].x, vai));
        vbr = fma(lb[k].x, xb[k].x, fma(-lb[k].y, xb[k].y, vbr));
        vbi = fma(lb[k].x, xb[k].y, fma(lb[k].y, xb[k].x, vbi));
      }
      accr = fma(var, vbr, fma(-vai, vbi, accr));
      acci = fma(var, vbi, fma(vai, vbr, acci));
    }
  }
#pragma unroll
  for (int o = RM / 2; o > 0; o >>= 1) {
    accr += __shfl_xor_sync(0xffffffffu, accr, o);
    acci += __shfl_xor_sync(0xffffffffu, acci, o);
  }
  if (m == 0 && s < a.S) {
    double *dst = a.partial + 2 * ((int64_t)g * a.S + s);
    dst[0] = (double)accr;
    dst[1] = (double)acci;
  }
}

// Leaf contraction with the parents' chunks streamed through shared memory: the CTA's
// bitstrings need 2 x 2^C amplitudes of every parent; they are copied with cp.async a
// few parents ahead (kDepth stages), so the DRAM / L2 latency of the next parents hides
// behind the arithmetic on the current one.  Thread roles as in the register variant.
constexpr int kDepth = 4;

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
  const uint32_t sa = (uint32_t)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// bytes of the cp.async stage ring of leaf_contract_async_kernel<CB, RM>
constexpr size_t leaf_ring_bytes(int cb, int rm) { return (size_t)kDepth * (128 / rm) * ((2u << cb) + 2) * 8; }

// Four CTAs per SM: with up to 128 registers a thread keeps a parent's chunk loads ahead
// of its FMAs (six CTAs per SM at 80 registers measured 5 % slower at n = 30).
template <int CB, int RM>
__global__ void __launch_bounds__(128, 4) leaf_contract_async_kernel(LeafArgs a) {
  using C = float2;
  constexpr int D = 1 << CB;
  constexpr int SPB = 128 / RM;                // bitstrings per CTA
  // Stage row of one bitstring: its a chunk then its b chunk, padded by one 16-byte
  // piece so that consecutive bitstrings start 4 banks apart and the 16-byte reads of
  // the (up to 8) bitstrings of a warp fall in distinct banks.
  constexpr int SB = 2 * D + 2;
  constexpr int STAGE = SPB * SB;
  constexpr int PIECES = D;                    // 16-byte pieces per bitstring and parent
  constexpr int HALF = D / 2;                  // pieces per side
  extern __shared__ __align__(16) unsigned char leaf_smem[];   // kDepth stages of STAGE
  C(*buf)[STAGE] = reinterpret_cast<C(*)[STAGE]>(leaf_smem);
  const int m = threadIdx.x % RM;
  const int sl = threadIdx.x / RM;
  const int64_t s = (int64_t)blockIdx.x * SPB + sl;
  const int g = blockIdx.y;
  const bool on = s < a.S && m < a.r;
  uint64_t ia = 0, ib = 0;
  if (s < a.S) {
    ia = a.ia[s];
    ib = a.ib[s];
  }
  const int ra = (int)(ia & (D - 1)), rb = (int)(ib & (D - 1));
  C la[D], lb[D];
  {
    const C *gLa = reinterpret_cast<const C *>(a.La) + ((size_t)(on ? m : 0) * D + ra) * D;
    const C *gLb = reinterpret_cast<const C *>(a.Lb) + ((size_t)(on ? m : 0) * D + rb) * D;
#pragma unroll
    for (int k = 0; k < D; ++k) {
      la[k] = gLa[k];
      lb[k] = gLb[k];
    }
  }
  const int64_t j0 = (int64_t)g * a.parents_per_group;
  const int64_t j1 = min(a.num_parents, j0 + a.parents_per_group);
  const int64_t np = j1 - j0;
  // the RM threads of a bitstring (adjacent lanes of one warp) copy its pieces:
  // piece q = m + i*RM; pieces [0, HALF) are the a chunk, [HALF, D) the b chunk
  const C *pa = reinterpret_cast<const C *>(a.Pa) + (ia - ra);
  const C *pb = reinterpret_cast<const C *>(a.Pb) + (ib - rb);
  auto issue = [&](int64_t jj, int stage) {
    if (jj < j1 && s < a.S) {
      C *row = buf[stage] + sl * SB;
      const C *sa = pa + ((uint64_t)jj << a.ha);
      const C *sb = pb + ((uint64_t)jj << a.hb);
#pragma unroll
      for (int i = 0; i < (PIECES + RM - 1) / RM; ++i) {
        const int q = m + i * RM;
        if (q < PIECES) {
          if (q < HALF)
            cp_async16(row + 2 * q, sa + 2 * q);
          else
            cp_async16(row + 2 * q, sb + 2 * (q - HALF));
        }
      }
    }
    cp_commit();
  };
#pragma unroll
  for (int d = 0; d < kDepth - 1; ++d) issue(j0 + d, d);
  float accr = 0.f, acci = 0.f;
  for (int64_t t = 0; t < np; ++t) {
    // parent t has landed for this thread; the warp barrier publishes the other lanes'
    // pieces and orders every lane's reads of parent t-1 before its stage is refilled
    cp_wait<kDepth - 2>();
    __syncwarp();
    issue(j0 + t + kDepth - 1, (int)((t + kDepth - 1) % kDepth));
    const int64_t j = j0 + t;
    const bool use = on && !((j == 0 && m < a.m_first) || (j == a.num_parents - 1 && m >= a.m_last));
    if (use) {
      const float4 *x = reinterpret_cast<const float4 *>(buf[t % kDepth] + sl * SB);
      float var = 0.f, vai = 0.f, vbr = 0.f, vbi = 0.f;
#pragma unroll
      for (int k2 = 0; k2 < HALF; ++k2) {
        const float4 xa = x[k2], xb = x[HALF + k2];
        const C a0 = la[2 * k2], a1 = la[2 * k2 + 1], b0 = lb[2 * k2], b1 = lb[2 * k2 + 1];
        var = fmaf(a0.x, xa.x, fmaf(-a0.y, xa.y, var));
        vai = fmaf(a0.x, xa.y, fmaf(a0.y, xa.x, vai));
        var = fmaf(a1.x, xa.z, fmaf(-a1.y, xa.w, var));
        vai = fmaf(a1.x, xa.w, fmaf(a1.y, xa.z, vai));
        vbr = fmaf(b0.x, xb.x, fmaf(-b0.y, xb.y, vbr));
        vbi = fmaf(b0.x, xb.y, fmaf(b0.y, xb.x, vbi));
        vbr = fmaf(b1.x, xb.z, fmaf(-b1.y, xb.w, vbr));
        vbi = fmaf(b1.x, xb.w, fmaf(b1.y, xb.z, vbi));
      }
      accr = fmaf(var, vbr, fmaf(-vai, vbi, accr));
      acci = fmaf(var, vbi, fmaf(vai, vbr, acci));
    }
  }
  cp_wait<0>();
#pragma unroll
  for (int o = RM / 2; o > 0; o >>= 1) {
    accr += __shfl_xor_sync(0xffffffffu, accr, o);
    acci += __shfl_xor_sync(0xffffffffu, acci, o);
  }
  if (m == 0 && s < a.S) {
    double *dst = a.partial + 2 * ((int64_t)g * a.S + s);
    dst[0] = (double)accr;
    dst[1] = (double)acci;
  }
}

// Leaf contraction with one thread per (bitstring, digit, side): the thread keeps only its
// side's row of L_m (half the registers of one thread per digit), copies and reads only
// its side's chunk, and the two sides' dot products meet with one shuffle.  Lanes of a
// warp: bitstring (t / 2RM), side ((t / RM) & 1), digit (t % RM).  Stage row of a
// bitstring: a chunk, two complex of padding, b chunk, two more: with the row stride of
// 2^(C+1) + 4 complex the 16-byte reads of a warp's four bitstrings and two sides fall
// in eight distinct bank groups.
constexpr int kPairDepth = 4;
constexpr size_t leaf_pair_ring_bytes(int cb, int rm) {
  return (size_t)kPairDepth * (128 / (2 * rm)) * ((2u << cb) + 4) * 8;
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

template <int CB, int RM>
__global__ void __launch_bounds__(128, 6) leaf_contract_pair_kernel(LeafArgs a) {
  using C = float2;
  constexpr int D = 1 << CB;
  constexpr int SPB = 128 / (2 * RM);          // bitstrings per CTA
  constexpr int SB = 2 * D + 4;
  constexpr int BOFF = D + 2;                  // offset (complex) of the b chunk in a row
  constexpr int STAGE = SPB * SB;
  constexpr int HALF = D / 2 > 0 ? D / 2 : 1;  // 16-byte pieces per side
  extern __shared__ __align__(16) unsigned char leaf_smem[];
  C(*buf)[STAGE] = reinterpret_cast<C(*)[STAGE]>(leaf_smem);
  const int m = threadIdx.x % RM;
  const int side = (threadIdx.x / RM) & 1;
  const int sl = threadIdx.x / (2 * RM);
  const int64_t s = (int64_t)blockIdx.x * SPB + sl;
  const int g = blockIdx.y;
  const bool on = s < a.S && m < a.r;
  uint64_t idx = 0;
  if (s < a.S) idx = side == 0 ? a.ia[s] : a.ib[s];
  const int rr = (int)(idx & (D - 1));
  // the row of L_m as broadcast pairs: lr[k] = (Re l_k, Re l_k), li[k] = (Im l_k, Im l_k),
  // so that with x_k = (Re x_k, Im x_k) as it sits in memory,
  //   P = sum_k lr[k] * x_k = (sum Re l Re x, sum Re l Im x)
  //   Q = sum_k li[k] * x_k = (sum Im l Re x, sum Im l Im x)
  // and l . x = (P.x - Q.y, P.y + Q.x): two packed FMAs per complex term, no shuffling
  C lr[D], li[D];
  {
    const C *gL = reinterpret_cast<const C *>(side == 0 ? a.La : a.Lb) + ((size_t)(on ? m : 0) * D + rr) * D;
#pragma unroll
    for (int k = 0; k < D; ++k) {
      const C v = gL[k];
      lr[k] = make_float2(v.x, v.x);
      li[k] = make_float2(v.y, v.y);
    }
  }
  const int64_t j0 = (int64_t)g * a.parents_per_group;
  const int64_t j1 = min(a.num_parents, j0 + a.parents_per_group);
  const int64_t np = j1 - j0;
  const int hbits = side == 0 ? a.ha : a.hb;
  const C *src = reinterpret_cast<const C *>(side == 0 ? a.Pa : a.Pb) + (idx - rr);
  const int roff = sl * SB + side * BOFF;
  auto issue = [&](int64_t jj, int stage) {
    if (jj < j1 && s < a.S) {
      C *row = buf[stage] + roff;
      const C *sp = src + ((uint64_t)jj << hbits);
#pragma unroll
      for (int i = 0; i < (HALF + RM - 1) / RM; ++i) {
        const int q = m + i * RM;
        if (q < HALF) cp_async16(row + 2 * q, sp + 2 * q);
      }
    }
    cp_commit();
  };
#pragma unroll
  for (int d = 0; d < kPairDepth - 1; ++d) issue(j0 + d, d);
  float accr = 0.f, acci = 0.f;
  for (int64_t t = 0; t < np; ++t) {
    cp_wait<kPairDepth - 2>();
    __syncwarp();
    issue(j0 + t + kPairDepth - 1, (int)((t + kPairDepth - 1) % kPairDepth));
    const int64_t j = j0 + t;
    const bool use = on && !((j == 0 && m < a.m_first) || (j == a.num_parents - 1 && m >= a.m_last));
    float vr = 0.f, vi = 0.f;
    if (use) {
      const float4 *x = reinterpret_cast<const float4 *>(buf[t % kPairDepth] + roff);
      // two independent accumulator pairs (even and odd k) halve the dependent chains
      C P0 = make_float2(0.f, 0.f), Q0 = P0, P1 = P0, Q1 = P0;
#pragma unroll
      for (int k2 = 0; k2 < D / 2; ++k2) {
        const float4 xv = x[k2];
        const C x0 = make_float2(xv.x, xv.y), x1 = make_float2(xv.z, xv.w);
        P0 = ffma2(lr[2 * k2], x0, P0);
        Q0 = ffma2(li[2 * k2], x0, Q0);
        P1 = ffma2(lr[2 * k2 + 1], x1, P1);
        Q1 = ffma2(li[2 * k2 + 1], x1, Q1);
      }
      vr = (P0.x + P1.x) - (Q0.y + Q1.y);
      vi = (P0.y + P1.y) + (Q0.x + Q1.x);
    }
    // the other side's value for the same bitstring and digit (all lanes take part)
    const float wr = __shfl_xor_sync(0xffffffffu, vr, RM);
    const float wi = __shfl_xor_sync(0xffffffffu, vi, RM);
    accr = fmaf(vr, wr, fmaf(-vi, wi, accr));
    acci = fmaf(vr, wi, fmaf(vi, wr, acci));
  }
  cp_wait<0>();
#pragma unroll
  for (int o = RM / 2; o > 0; o >>= 1) {
    accr += __shfl_xor_sync(0xffffffffu, accr, o);
    acci += __shfl_xor_sync(0xffffffffu, acci, o);
  }
  if (m == 0 && side == 0 && s < a.S) {
    double *dst = a.partial + 2 * ((int64_t)g * a.S + s);
    dst[0] = (double)accr;
    dst[1] = (double)acci;
  }
}

// Leaf contraction with the chunk split over the digit lanes: the RM lanes of one
// (bitstring, side) each read only their D / RM entries of the chunk and form the partial
// products of ALL RM digits over them; a reduce-scatter across the RM lanes (log2 RM
// shuffle rounds, halving the digits each round) leaves lane q with digit q summed over
// the whole chunk.  The same FMAs as one lane per digit over the whole chunk, but each
// chunk entry is read from shared memory once instead of RM times (broadcast).  Lane
// layout and stage rows as in leaf_contract_pair_kernel.
template <int CB, int RM>
__global__ void __launch_bounds__(128, 5) leaf_contract_split_kernel(LeafArgs a) {
  using C = float2;
  constexpr int D = 1 << CB;
  constexpr int KQ = D / RM;                   // complex chunk entries per lane
  static_assert(KQ >= 2 && KQ % 2 == 0, "a lane reads whole 16-byte pieces");
  constexpr int SPB = 128 / (2 * RM);
  constexpr int SB = 2 * D + 4;
  constexpr int BOFF = D + 2;
  constexpr int STAGE = SPB * SB;
  constexpr int HALF = D / 2;
  extern __shared__ __align__(16) unsigned char leaf_smem[];
  C(*buf)[STAGE] = reinterpret_cast<C(*)[STAGE]>(leaf_smem);
  const int q = threadIdx.x % RM;              // chunk part; after the reduce-scatter, the digit
  const int side = (threadIdx.x / RM) & 1;
  const int sl = threadIdx.x / (2 * RM);
  const int64_t s = (int64_t)blockIdx.x * SPB + sl;
  const int g = blockIdx.y;
  uint64_t idx = 0;
  if (s < a.S) idx = side == 0 ? a.ia[s] : a.ib[s];
  const int rr = (int)(idx & (D - 1));
  // entries k = q KQ + i of row rr of every L_m, as broadcast pairs (see the pair kernel);
  // slot j holds digit j ^ q, so that in every reduce-scatter round the values a lane
  // keeps and the ones it sends sit at fixed slots (no selects)
  C lr[RM][KQ], li[RM][KQ];
  {
    const C *gL = reinterpret_cast<const C *>(side == 0 ? a.La : a.Lb);
#pragma unroll
    for (int jm = 0; jm < RM; ++jm) {
      const int m = jm ^ q;
      const bool mv = s < a.S && m < a.r;
      const C *row = gL + ((size_t)(mv ? m : 0) * D + rr) * D + q * KQ;
#pragma unroll
      for (int i = 0; i < KQ; ++i) {
        const C v = mv ? row[i] : make_float2(0.f, 0.f);
        lr[jm][i] = make_float2(v.x, v.x);
        li[jm][i] = make_float2(v.y, v.y);
      }
    }
  }
  const bool on = s < a.S && q < a.r;
  const int64_t j0 = (int64_t)g * a.parents_per_group;
  const int64_t j1 = min(a.num_parents, j0 + a.parents_per_group);
  const int64_t np = j1 - j0;
  const int hbits = side == 0 ? a.ha : a.hb;
  const C *src = reinterpret_cast<const C *>(side == 0 ? a.Pa : a.Pb) + (idx - rr);
  const int roff = sl * SB + side * BOFF;
  auto issue = [&](int64_t jj, int stage) {
    if (jj < j1 && s < a.S) {
      C *row = buf[stage] + roff;
      const C *sp = src + ((uint64_t)jj << hbits);
#pragma unroll
      for (int i = 0; i < (HALF + RM - 1) / RM; ++i) {
        const int p = q + i * RM;
        if (p < HALF) cp_async16(row + 2 * p, sp + 2 * p);
      }
    }
    cp_commit();
  };
#pragma unroll
  for (int d = 0; d < kPairDepth - 1; ++d) issue(j0 + d, d);
  float accr = 0.f, acci = 0.f;
  for (int64_t t = 0; t < np; ++t) {
    cp_wait<kPairDepth - 2>();
    __syncwarp();
    issue(j0 + t + kPairDepth - 1, (int)((t + kPairDepth - 1) % kPairDepth));
    const int64_t j = j0 + t;
    const float4 *x = reinterpret_cast<const float4 *>(buf[t % kPairDepth] + roff + q * KQ);
    C xk[KQ];
#pragma unroll
    for (int i = 0; i < KQ / 2; ++i) {
      const float4 v = x[i];
      xk[2 * i] = make_float2(v.x, v.y);
      xk[2 * i + 1] = make_float2(v.z, v.w);
    }
    float vr[RM], vi[RM];
#pragma unroll
    for (int m = 0; m < RM; ++m) {
      C P = make_float2(0.f, 0.f), Q = P;
#pragma unroll
      for (int i = 0; i < KQ; ++i) {
        P = ffma2(lr[m][i], xk[i], P);
        Q = ffma2(li[m][i], xk[i], Q);
      }
      vr[m] = P.x - Q.y;
      vi[m] = P.y + Q.x;
    }
    // reduce-scatter: in the round over lane bit o a lane keeps slots [0, o) and sends
    // slots [o, 2o); slot i + o of lane q ^ o holds the digit of slot i of lane q, since
    // (i + o) ^ (q ^ o) = i ^ q for i < o.  Slot 0 ends with digit q summed over the RM lanes.
#pragma unroll
    for (int o = RM / 2; o > 0; o >>= 1) {
#pragma unroll
      for (int i = 0; i < o; ++i) {
        vr[i] += __shfl_xor_sync(0xffffffffu, vr[i + o], o);
        vi[i] += __shfl_xor_sync(0xffffffffu, vi[i + o], o);
      }
    }
    const bool use = on && !((j == 0 && q < a.m_first) || (j == a.num_parents - 1 && q >= a.m_last));
    const float ur = use ? vr[0] : 0.f, ui = use ? vi[0] : 0.f;
    // the other side's value for the same bitstring and digit
    const float wr = __shfl_xor_sync(0xffffffffu, ur, RM);
    const float wi = __shfl_xor_sync(0xffffffffu, ui, RM);
    accr = fmaf(ur, wr, fmaf(-ui, wi, accr));
    acci = fmaf(ur, wi, fmaf(ui, wr, acci));
  }
  cp_wait<0>();
#pragma unroll
  for (int o = RM / 2; o > 0; o >>= 1) {
    accr += __shfl_xor_sync(0xffffffffu, accr, o);
    acci += __shfl_xor_sync(0xffffffffu, acci, o);
  }
  if (q == 0 && side == 0 && s < a.S) {
    double *dst = a.partial + 2 * ((int64_t)g * a.S + s);
    dst[0] = (double)accr;
    dst[1] = (double)acci;
  }
}

// Factored leaf contraction.  When every leaf operator is L_m = S (F_m (x) I) with F_m a
// one-qubit factor on chunk bit PF (both sides), a parent's contribution at a bitstring
// is the bilinear form sum_{al, be} G[al][be] d_a[al] d_b[be] (see factor_leaf): d holds
// the four dots d[(i, j)] = sum_k w[(i, k)] x[(j, k)] of the row w = S[rr] with the
// bitstring's chunk x (i, j the factor bit, k the other chunk bits), and G the digit sum
// of F^a (x) F^b.  One thread per (bitstring, side): lanes t (side a) and t ^ 1 (side b)
// swap their d with one shuffle per value, and each adds half of the form (rows al of
// its own side's pair).  Stage rows as in leaf_contract_pair_kernel.
constexpr int kFactDepth = 4;
constexpr int kFactSpb = 64;                   // bitstrings per 128-thread CTA
constexpr size_t leaf_fact_ring_bytes(int cb) { return (size_t)kFactDepth * kFactSpb * ((2u << cb) + 4) * 8; }

template <int CB, int PF>
__global__ void __launch_bounds__(128, 3) leaf_contract_fact_kernel(LeafArgs a) {
  using C = float2;
  constexpr int D = 1 << CB;
  constexpr int H = D / 2;
  constexpr int SB = 2 * D + 4;
  constexpr int BOFF = D + 2;
  constexpr int STAGE = kFactSpb * SB;
  static_assert(PF < CB, "the factor bit lies in the chunk");
  extern __shared__ __align__(16) unsigned char leaf_smem[];
  C(*buf)[STAGE] = reinterpret_cast<C(*)[STAGE]>(leaf_smem);
  const int side = threadIdx.x & 1;
  const int sl = threadIdx.x >> 1;
  const int64_t s = (int64_t)blockIdx.x * kFactSpb + sl;
  const int g = blockIdx.y;
  uint64_t idx = 0;
  if (s < a.S) idx = side == 0 ? a.ia[s] : a.ib[s];
  const int rr = (int)(idx & (D - 1));
  // w = S[rr] as broadcast pairs (see the pair kernel)
  C wr[D], wi[D];
  {
    const C *row = reinterpret_cast<const C *>(side == 0 ? a.Sa : a.Sb) + (size_t)rr * D;
#pragma unroll
    for (int k = 0; k < D; ++k) {
      const C v = row[k];
      wr[k] = make_float2(v.x, v.x);
      wi[k] = make_float2(v.y, v.y);
    }
  }
  // rows al = 2 side, 2 side + 1 of G over all digits
  const C *Gt = reinterpret_cast<const C *>(a.G);
  const int r1 = a.r + 1;
  C g0[4], g1[4];
  {
    const C *G = Gt + (size_t)a.r * 16;        // [m0 = 0][m1 = r]
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      g0[b] = G[(2 * side) * 4 + b];
      g1[b] = G[(2 * side + 1) * 4 + b];
    }
  }
  const int64_t j0 = (int64_t)g * a.parents_per_group;
  const int64_t j1 = min(a.num_parents, j0 + a.parents_per_group);
  const int64_t np = j1 - j0;
  const int roff = sl * SB + side * BOFF;
  // The warp's 32 chunks (16 bitstrings x 2 sides) are copied with whole chunks per
  // instruction: in copy q lane l moves 16-byte piece l % H of chunk (32 / H) q + l / H,
  // so one instruction covers 32 / H chunks of contiguous bytes instead of 32 scattered
  // pieces.  Chunk c of the warp is bitstring c / 2, side c % 2; cof[q] is its origin.
  // CPI is even, so the side of every chunk a lane copies is (lane / H) & 1: the lane's
  // source base, shift and destination column are fixed, and copy q only adds its
  // chunk's origin and row.
  constexpr int CPI = 32 / H;                  // chunks per copy instruction
  static_assert(CPI % 2 == 0, "a lane copies chunks of one side");
  const int lane = threadIdx.x & 31, wbase = threadIdx.x & ~31;
  const int csd = (lane / H) & 1, piece = lane % H;
  const C *cbase = reinterpret_cast<const C *>(csd == 0 ? a.Pa : a.Pb) + 2 * piece;
  const int chb = csd == 0 ? a.ha : a.hb;
  uint32_t cof[H];
  int crow[H];                                 // destination offset (complex) of copy q
#pragma unroll
  for (int q = 0; q < H; ++q) {
    const int c = CPI * q + lane / H;
    const int64_t sc = (int64_t)blockIdx.x * kFactSpb + (wbase >> 1) + (c >> 1);
    const bool ok = sc < a.S;
    const uint64_t ic = ok ? (csd == 0 ? a.ia[sc] : a.ib[sc]) : 0;
    cof[q] = (uint32_t)(ic & ~(uint64_t)(D - 1));
    crow[q] = ok ? ((wbase >> 1) + (c >> 1)) * SB + csd * BOFF + 2 * piece : -1;
  }
  auto issue = [&](int64_t jj, int stage) {
    if (jj < j1) {
      const C *pj = cbase + ((uint64_t)jj << chb);
#pragma unroll
      for (int q = 0; q < H; ++q)
        if (crow[q] >= 0) cp_async16(buf[stage] + crow[q], pj + cof[q]);
    }
    cp_commit();
  };
#pragma unroll
  for (int d = 0; d < kFactDepth - 1; ++d) issue(j0 + d, d);
  float accr = 0.f, acci = 0.f;
  for (int64_t t = 0; t < np; ++t) {
    cp_wait<kFactDepth - 2>();
    __syncwarp();
    issue(j0 + t + kFactDepth - 1, (int)((t + kFactDepth - 1) % kFactDepth));
    const int64_t j = j0 + t;
    const float4 *x4 = reinterpret_cast<const float4 *>(buf[t % kFactDepth] + roff);
    C x[D];
#pragma unroll
    for (int q = 0; q < H; ++q) {
      const float4 v = x4[q];
      x[2 * q] = make_float2(v.x, v.y);
      x[2 * q + 1] = make_float2(v.z, v.w);
    }
    // the four dots, al = 2 i + j
    C P[4], Q[4];
#pragma unroll
    for (int al = 0; al < 4; ++al) P[al] = Q[al] = make_float2(0.f, 0.f);
#pragma unroll
    for (int k = 0; k < H; ++k) {
      constexpr int lo = (1 << PF) - 1;
      const int e0 = ((k & ~lo) << 1) | (k & lo), e1 = e0 | (1 << PF);   // factor bit 0 / 1
      P[0] = ffma2(wr[e0], x[e0], P[0]);
      Q[0] = ffma2(wi[e0], x[e0], Q[0]);
      P[1] = ffma2(wr[e0], x[e1], P[1]);
      Q[1] = ffma2(wi[e0], x[e1], Q[1]);
      P[2] = ffma2(wr[e1], x[e0], P[2]);
      Q[2] = ffma2(wi[e1], x[e0], Q[2]);
      P[3] = ffma2(wr[e1], x[e1], P[3]);
      Q[3] = ffma2(wi[e1], x[e1], Q[3]);
    }
    float dr[4], di[4], er[4], ei[4];
#pragma unroll
    for (int al = 0; al < 4; ++al) {
      dr[al] = P[al].x - Q[al].y;
      di[al] = P[al].y + Q[al].x;
      er[al] = __shfl_xor_sync(0xffffffffu, dr[al], 1);
      ei[al] = __shfl_xor_sync(0xffffffffu, di[al], 1);
    }
    // d_a and d_b of this bitstring
    float ar[4], ai[4], br[4], bi[4];
#pragma unroll
    for (int al = 0; al < 4; ++al) {
      ar[al] = side == 0 ? dr[al] : er[al];
      ai[al] = side == 0 ? di[al] : ei[al];
      br[al] = side == 0 ? er[al] : dr[al];
      bi[al] = side == 0 ? ei[al] : di[al];
    }
    C h0[4], h1[4];
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      h0[b] = g0[b];
      h1[b] = g1[b];
    }
    if ((j == 0 && a.m_first > 0) || (j == a.num_parents - 1 && a.m_last < a.r)) {
      // a parent with only part of its digits in the path range
      const int m0 = j == 0 ? a.m_first : 0, m1 = j == a.num_parents - 1 ? a.m_last : a.r;
      const C *G = Gt + ((size_t)m0 * r1 + m1) * 16;
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        h0[b] = G[(2 * side) * 4 + b];
        h1[b] = G[(2 * side + 1) * 4 + b];
      }
    }
    // this lane's half: sum over al = 2 side + {0, 1} of d_a[al] (G[al] . d_b)
    float u0r = 0.f, u0i = 0.f, u1r = 0.f, u1i = 0.f;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      u0r = fmaf(h0[b].x, br[b], fmaf(-h0[b].y, bi[b], u0r));
      u0i = fmaf(h0[b].x, bi[b], fmaf(h0[b].y, br[b], u0i));
      u1r = fmaf(h1[b].x, br[b], fmaf(-h1[b].y, bi[b], u1r));
      u1i = fmaf(h1[b].x, bi[b], fmaf(h1[b].y, br[b], u1i));
    }
    const float a0r = side == 0 ? ar[0] : ar[2], a0i = side == 0 ? ai[0] : ai[2];
    const float a1r = side == 0 ? ar[1] : ar[3], a1i = side == 0 ? ai[1] : ai[3];
    accr = fmaf(a0r, u0r, fmaf(-a0i, u0i, accr));
    acci = fmaf(a0r, u0i, fmaf(a0i, u0r, acci));
    accr = fmaf(a1r, u1r, fmaf(-a1i, u1i, accr));
    acci = fmaf(a1r, u1i, fmaf(a1i, u1r, acci));
  }
  cp_wait<0>();
  accr += __shfl_xor_sync(0xffffffffu, accr, 1);
  acci += __shfl_xor_sync(0xffffffffu, acci, 1);
  if (side == 0 && s < a.S) {
    double *dst = a.partial + 2 * ((int64_t)g * a.S + s);
    dst[0] = (double)accr;
    dst[1] = (double)acci;
  }
}

// Leaf contraction for large bitstring counts.  One co-resident wave of CTAs; CTA b
// owns bitstrings [b * per_cta, (b + 1) * per_cta), and every CTA walks all parents in
// the same order, so the parents being read at any time are few and stay in L2 however
// many bitstrings gather from them.  A bitstring's chunk origins, leaf rows and FP32
// running sum live in shared memory; every kStreamBatch parents the FP32 sums are added
// into the FP64 partial (one per bitstring: num_groups = 1).
constexpr int kStreamThreads = 256;
constexpr int kStreamBatch = 64;
constexpr int kStreamPerSm = 8;                // CTAs per SM the wave aims for
constexpr int kStreamSync = 8;                 // parents between grid barriers
constexpr uint32_t kStreamSpin = 1u << 20;     // bounded barrier wait (polls of ~100 ns)

// Grid barrier for a cooperative launch (all CTAs resident).  It only keeps the CTAs
// within kStreamSync parents of one another, for L2 locality; results do not depend on
// it, so on expiry it records an error code and lets the CTA go on.
__device__ __forceinline__ void stream_barrier(uint32_t *count, volatile uint32_t *gen, uint32_t nblocks,
                                               int32_t *err) {
  __syncthreads();
  if (threadIdx.x == 0) {
    const uint32_t g = *gen;
    __threadfence();
    if (atomicAdd(count, 1u) == nblocks - 1) {
      *count = 0;
      __threadfence();
      atomicAdd((uint32_t *)gen, 1u);
    } else {
      uint32_t it = 0;
      while (*gen == g && ++it < kStreamSpin) __nanosleep(100);
      if (it >= kStreamSpin) atomicExch(err, 11);
    }
  }
  __syncthreads();
}
struct StreamBits {
  uint32_t oa, ob;                             // chunk origin (storage index) on each side
  uint32_t rr;                                 // ra | rb << 8
  uint32_t pad;
  float2 acc;
};

template <int CB>
__global__ void __launch_bounds__(kStreamThreads) leaf_stream_kernel(LeafArgs a, int64_t per_cta) {
  using C = float2;
  constexpr int D = 1 << CB;
  constexpr int LD = D + 2;                    // row stride (complex): 16-byte aligned rows
  extern __shared__ __align__(16) unsigned char leaf_smem[];
  C *sLa = reinterpret_cast<C *>(leaf_smem);
  C *sLb = sLa + a.r * D * LD;
  StreamBits *bs = reinterpret_cast<StreamBits *>(sLb + a.r * D * LD);
  const int64_t s0 = (int64_t)blockIdx.x * per_cta;
  const int ns = (int)(min(a.S, s0 + per_cta) - s0);
  for (int e = threadIdx.x; e < a.r * D * D; e += blockDim.x) {
    const int row = e / D, k = e % D;          // row = m * D + output index
    sLa[row * LD + k] = reinterpret_cast<const C *>(a.La)[e];
    sLb[row * LD + k] = reinterpret_cast<const C *>(a.Lb)[e];
  }
  for (int i = threadIdx.x; i < ns; i += blockDim.x) {
    const uint64_t ia = a.ia[s0 + i], ib = a.ib[s0 + i];
    const uint32_t ra = (uint32_t)(ia & (D - 1)), rb = (uint32_t)(ib & (D - 1));
    bs[i].oa = (uint32_t)(ia - ra);
    bs[i].ob = (uint32_t)(ib - rb);
    bs[i].rr = ra | (rb << 8);
    bs[i].acc = make_float2(0.f, 0.f);
    const int64_t o = a.perm ? a.perm[s0 + i] : s0 + i;
    a.partial[2 * o] = 0.0;
    a.partial[2 * o + 1] = 0.0;
  }
  __syncthreads();
  for (int64_t j0 = 0; j0 < a.num_parents; j0 += kStreamBatch) {
    const int64_t j1 = min(a.num_parents, j0 + kStreamBatch);
    for (int64_t j = j0; j < j1; ++j) {
      if (j % kStreamSync == 0 && j > 0) stream_barrier(a.sync, a.sync + 1, gridDim.x, a.err);
      const int mlo = j == 0 ? a.m_first : 0;
      const int mhi = j == a.num_parents - 1 ? a.m_last : a.r;
      const C *Pa = reinterpret_cast<const C *>(a.Pa) + ((uint64_t)j << a.ha);
      const C *Pb = reinterpret_cast<const C *>(a.Pb) + ((uint64_t)j << a.hb);
      for (int i = threadIdx.x; i < ns; i += blockDim.x) {
        const StreamBits st = bs[i];
        float4 xa[D / 2], xb[D / 2];
#pragma unroll
        for (int k2 = 0; k2 < D / 2; ++k2) {
          xa[k2] = __ldg(reinterpret_cast<const float4 *>(Pa + st.oa) + k2);
          xb[k2] = __ldg(reinterpret_cast<const float4 *>(Pb + st.ob) + k2);
        }
        const int ra = (int)(st.rr & 255u), rb = (int)(st.rr >> 8);
        float sr = 0.f, si = 0.f;
        for (int m = mlo; m < mhi; ++m) {
          const float4 *la = reinterpret_cast<const float4 *>(sLa + (m * D + ra) * LD);
          const float4 *lb = reinterpret_cast<const float4 *>(sLb + (m * D + rb) * LD);
          float var = 0.f, vai = 0.f, vbr = 0.f, vbi = 0.f;
#pragma unroll
          for (int k2 = 0; k2 < D / 2; ++k2) {
            const float4 p = la[k2], x = xa[k2], u = lb[k2], y = xb[k2];
            var = fmaf(p.x, x.x, fmaf(-p.y, x.y, var));
            vai = fmaf(p.x, x.y, fmaf(p.y, x.x, vai));
            var = fmaf(p.z, x.z, fmaf(-p.w, x.w, var));
            vai = fmaf(p.z, x.w, fmaf(p.w, x.z, vai));
            vbr = fmaf(u.x, y.x, fmaf(-u.y, y.y, vbr));
            vbi = fmaf(u.x, y.y, fmaf(u.y, y.x, vbi));
            vbr = fmaf(u.z, y.z, fmaf(-u.w, y.w, vbr));
            vbi = fmaf(u.z, y.w, fmaf(u.w, y.z, vbi));
          }
          sr = fmaf(var, vbr, fmaf(-vai, vbi, sr));
          si = fmaf(var, vbi, fmaf(vai, vbr, si));
        }
        bs[i].acc = make_float2(st.acc.x + sr, st.acc.y + si);
      }
    }
    // every thread only ever touches its own bitstrings i = tid + k * blockDim.x
    for (int i = threadIdx.x; i < ns; i += blockDim.x) {
      const float2 c = bs[i].acc;
      const int64_t o = a.perm ? a.perm[s0 + i] : s0 + i;
      a.partial[2 * o] += (double)c.x;
      a.partial[2 * o + 1] += (double)c.y;
      bs[i].acc = make_float2(0.f, 0.f);
    }
  }
}

// The streaming kernel with the digit sum folded into the pair form: each (bitstring,
// parent) adds x_a^T H[i][i'] x_b (see pair_leaf), H[i][i'] of the full digit range
// from shared memory, of a partial range (the first or last parent of a path range)
// from the table in global memory.
template <int CB>
__global__ void __launch_bounds__(kStreamThreads) leaf_stream_pair_kernel(LeafArgs a, int64_t per_cta) {
  using C = float2;
  constexpr int D = 1 << CB;
  constexpr int PER = D * D * D * D;
  extern __shared__ __align__(16) unsigned char leaf_smem[];
  C *sH = reinterpret_cast<C *>(leaf_smem);
  StreamBits *bs = reinterpret_cast<StreamBits *>(sH + PER);
  const C *gH = reinterpret_cast<const C *>(a.H);
  const int r1 = a.r + 1;
  const int64_t s0 = (int64_t)blockIdx.x * per_cta;
  const int ns = (int)(min(a.S, s0 + per_cta) - s0);
  for (int e = threadIdx.x; e < PER; e += blockDim.x) sH[e] = gH[(size_t)a.r * PER + e];   // [0][r]
  for (int i = threadIdx.x; i < ns; i += blockDim.x) {
    const uint64_t ia = a.ia[s0 + i], ib = a.ib[s0 + i];
    const uint32_t ra = (uint32_t)(ia & (D - 1)), rb = (uint32_t)(ib & (D - 1));
    bs[i].oa = (uint32_t)(ia - ra);
    bs[i].ob = (uint32_t)(ib - rb);
    bs[i].rr = ra | (rb << 8);
    bs[i].acc = make_float2(0.f, 0.f);
    const int64_t o = a.perm ? a.perm[s0 + i] : s0 + i;
    a.partial[2 * o] = 0.0;
    a.partial[2 * o + 1] = 0.0;
  }
  __syncthreads();
  for (int64_t j0 = 0; j0 < a.num_parents; j0 += kStreamBatch) {
    const int64_t j1 = min(a.num_parents, j0 + kStreamBatch);
    for (int64_t j = j0; j < j1; ++j) {
      if (j % kStreamSync == 0 && j > 0) stream_barrier(a.sync, a.sync + 1, gridDim.x, a.err);
      const int mlo = j == 0 ? a.m_first : 0;
      const int mhi = j == a.num_parents - 1 ? a.m_last : a.r;
      const bool full = mlo == 0 && mhi == a.r;
      const C *Ht = full ? sH : gH + ((size_t)mlo * r1 + mhi) * PER;
      const C *Pa = reinterpret_cast<const C *>(a.Pa) + ((uint64_t)j << a.ha);
      const C *Pb = reinterpret_cast<const C *>(a.Pb) + ((uint64_t)j << a.hb);
      for (int i = threadIdx.x; i < ns; i += blockDim.x) {
        const StreamBits st = bs[i];
        C xa[D], xb[D];
#pragma unroll
        for (int k2 = 0; k2 < D / 2; ++k2) {
          const float4 u = __ldg(reinterpret_cast<const float4 *>(Pa + st.oa) + k2);
          const float4 v = __ldg(reinterpret_cast<const float4 *>(Pb + st.ob) + k2);
          xa[2 * k2] = make_float2(u.x, u.y);
          xa[2 * k2 + 1] = make_float2(u.z, u.w);
          xb[2 * k2] = make_float2(v.x, v.y);
          xb[2 * k2 + 1] = make_float2(v.z, v.w);
        }
        const int ra = (int)(st.rr & 255u), rb = (int)(st.rr >> 8);
        const C *h = Ht + (size_t)(ra * D + rb) * D * D;
        float sr = 0.f, si = 0.f;
#pragma unroll
        for (int jj = 0; jj < D; ++jj) {
          float ur = 0.f, ui = 0.f;       // (H[i][i'] x_b)[jj]
#pragma unroll
          for (int j2 = 0; j2 < D; ++j2) {
            const C hv = h[jj * D + j2];
            ur = fmaf(hv.x, xb[j2].x, fmaf(-hv.y, xb[j2].y, ur));
            ui = fmaf(hv.x, xb[j2].y, fmaf(hv.y, xb[j2].x, ui));
          }
          sr = fmaf(xa[jj].x, ur, fmaf(-xa[jj].y, ui, sr));
          si = fmaf(xa[jj].x, ui, fmaf(xa[jj].y, ur, si));
        }
        bs[i].acc = make_float2(st.acc.x + sr, st.acc.y + si);
      }
    }
    for (int i = threadIdx.x; i < ns; i += blockDim.x) {
      const float2 c = bs[i].acc;
      const int64_t o = a.perm ? a.perm[s0 + i] : s0 + i;
      a.partial[2 * o] += (double)c.x;
      a.partial[2 * o + 1] += (double)c.y;
      bs[i].acc = make_float2(0.f, 0.f);
    }
  }
}

template <int CB, bool PAIR>
size_t leaf_stream_smem(int r, int64_t per_cta) {
  const size_t ops = PAIR ? (size_t)(1 << (4 * CB)) * sizeof(float2)
                          : (size_t)2 * r * (1 << CB) * ((1 << CB) + 2) * sizeof(float2);
  return ops + (size_t)per_cta * sizeof(StreamBits);
}
template <int CB, bool PAIR>
constexpr auto stream_kernel() {
  if constexpr (PAIR) return leaf_stream_pair_kernel<CB>;
  else return leaf_stream_kernel<CB>;
}

// Launch shape of the one-wave kernel for S bitstrings: CTAs (all co-resident) and
// bitstrings per CTA; false if S does not fit one wave.
template <int CB, bool PAIR>
bool leaf_stream_shape(int r, int64_t S, int *grid, int64_t *per_cta) {
  const int sms = device_sm_count();
  if (sms <= 0) return false;
  const auto kernel = stream_kernel<CB, PAIR>();
  for (int per_sm = kStreamPerSm; per_sm >= 1; --per_sm) {
    const int64_t pc = (S + (int64_t)sms * per_sm - 1) / ((int64_t)sms * per_sm);
    const size_t smem = leaf_stream_smem<CB, PAIR>(r, pc);
    if (smem > 200 * 1024) continue;
    int occ = 0;
    if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, kStreamThreads, smem) != cudaSuccess)
      return false;
    if (occ >= per_sm) {
      *per_cta = pc;
      *grid = (int)((S + pc - 1) / pc);
      return true;
    }
  }
  return false;
}

template <int CB, bool PAIR>
cudaError_t leaf_stream_launch(const LeafArgs &a, cudaStream_t st) {
  int grid = 0;
  int64_t per_cta = 0;
  if (!leaf_stream_shape<CB, PAIR>(a.r, a.S, &grid, &per_cta)) return cudaErrorInvalidConfiguration;
  // the barrier words start at zero (and return there after every barrier)
  cudaError_t e = cudaMemsetAsync(a.sync, 0, 2 * sizeof(uint32_t), st);
  if (e != cudaSuccess) return e;
  LeafArgs args = a;
  void *params[] = {&args, &per_cta};
  return cudaLaunchCooperativeKernel((const void *)stream_kernel<CB, PAIR>(), dim3(grid), dim3(kStreamThreads),
                                     params, leaf_stream_smem<CB, PAIR>(a.r, per_cta), st);
}

__global__ void index_prep_kernel(IndexArgs a) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= a.S) return;
  const uint64_t x = a.bits[s];
  uint64_t ia = 0, ib = 0;
  for (int q = 0; q < a.hb; ++q)
    if ((x >> q) & 1ull) ib |= 1ull << a.store_b[q];
  for (int q = 0; q < a.ha; ++q)
    if ((x >> (a.nb + q)) & 1ull) ia |= 1ull << a.store_a[q];
  a.ia[s] = ia;
  a.ib[s] = ib;
}

__global__ void range_index_kernel(uint64_t *dst, int64_t count, PermArgs perm) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  uint64_t r = 0;
  for (int q = 0; q < perm.h; ++q)
    if (((uint64_t)i >> q) & 1ull) r |= 1ull << perm.store[q];
  dst[i] = r;
}

// out += comp; a non-finite result sets *numeric (the output canary read by hsf_sync).
__global__ void finalize_kernel(double *out, const double *comp, int64_t count, int32_t *numeric) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  bool bad = false;
  if (i < count) {
    const double v = out[i] + comp[i];
    out[i] = v;
    bad = !isfinite(v);
  }
  if (__ballot_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0 && numeric) atomicOr(numeric, 1);
}

// Full-state output: out[i] = state[idx_i] in complex128, idx_i = bits[i] (bitstrings)
// or i (leading window); a non-finite amplitude sets *numeric.
template <typename R>
__global__ void state_gather_kernel(const R *state, const uint64_t *bits, int64_t count, double *out,
                                    int32_t *numeric) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  bool bad = false;
  if (i < count) {
    const uint64_t j = bits ? bits[i] : (uint64_t)i;
    const double re = (double)state[2 * j], im = (double)state[2 * j + 1];
    out[2 * i] = re;
    out[2 * i + 1] = im;
    bad = !isfinite(re) || !isfinite(im);
  }
  if (__ballot_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0 && numeric) atomicOr(numeric, 1);
}

__global__ void zero_kernel(double *p, int64_t count) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) p[i] = 0.0;
}

}  // namespace

cudaError_t launch_gather_dot(const GatherArgs &a, int precision, cudaStream_t st) {
  if (a.S <= 0 || a.num_paths <= 0) return cudaSuccess;
  dim3 grid((unsigned)((a.S + 255) / 256), (unsigned)a.num_groups);
  if (precision == 0)
    gather_dot_kernel<float><<<grid, 256, 0, st>>>(a);
  else
    gather_dot_kernel<double><<<grid, 256, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_reduce_partials(const double *partial, int32_t num_groups, int64_t S,
                                   double *out, double *comp, cudaStream_t st) {
  if (S <= 0) return cudaSuccess;
  reduce_partials_kernel<<<(unsigned)((S + 31) / 32), dim3(32, kReduceRows), 0, st>>>(partial, num_groups, S, out,
                                                                                      comp);
  return cudaGetLastError();
}

cudaError_t launch_window(const WindowArgs &a, int precision, cudaStream_t st) {
  if (a.M <= 0 || a.N <= 0 || a.num_paths <= 0) return cudaSuccess;
  dim3 grid((unsigned)((a.N + 31) / 32), (unsigned)((a.M + 31) / 32));
  if (precision == 0)
    window_kernel<float><<<grid, 256, 0, st>>>(a);
  else
    window_kernel<double><<<grid, 256, 0, st>>>(a);
  return cudaGetLastError();
}

template <typename R, int CB>
cudaError_t leaf_reg_dispatch(const LeafArgs &a, cudaStream_t st) {
  const int rm = a.r <= 1 ? 1 : a.r <= 2 ? 2 : a.r <= 4 ? 4 : 8;
  if constexpr (sizeof(R) == 4 && CB >= 1) {
    // the stage ring (kDepth x 128/rm bitstrings x (2^(CB+1)+2) complex) is dynamic
    // shared memory: up to 139 KB for one operator per thread at CB = 4
    dim3 grid((unsigned)((a.S * rm + 127) / 128), (unsigned)a.num_groups);
    auto go = [&](auto kernel, int rmv) -> cudaError_t {
      const size_t smem = leaf_ring_bytes(CB, rmv);
      cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      kernel<<<grid, 128, smem, st>>>(a);
      return cudaGetLastError();
    };
    auto go_pair = [&](auto kernel, int rmv) -> cudaError_t {
      dim3 gp((unsigned)((a.S * 2 * rmv + 127) / 128), (unsigned)a.num_groups);
      const size_t smem = leaf_pair_ring_bytes(CB, rmv);
      cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      kernel<<<gp, 128, smem, st>>>(a);
      return cudaGetLastError();
    };
    if constexpr (CB >= 2) {
      // chunk split over the digit lanes where every lane gets whole 16-byte pieces
      if (rm >= 2 && (1 << CB) >= 2 * rm) {
        switch (rm) {
          case 2: return go_pair(leaf_contract_split_kernel<CB, (CB >= 2 ? 2 : 1)>, 2);
          case 4: return go_pair(leaf_contract_split_kernel<CB, (CB >= 3 ? 4 : 1)>, 4);
          default: return go_pair(leaf_contract_split_kernel<CB, (CB >= 4 ? 8 : 1)>, 8);
        }
      }
      switch (rm) {
        case 1: return go_pair(leaf_contract_pair_kernel<CB, 1>, 1);
        case 2: return go_pair(leaf_contract_pair_kernel<CB, 2>, 2);
        case 4: return go_pair(leaf_contract_pair_kernel<CB, 4>, 4);
        default: return go_pair(leaf_contract_pair_kernel<CB, 8>, 8);
      }
    }
    switch (rm) {
      case 1: return go(leaf_contract_async_kernel<CB, 1>, 1);
      case 2: return go(leaf_contract_async_kernel<CB, 2>, 2);
      case 4: return go(leaf_contract_async_kernel<CB, 4>, 4);
      default: return go(leaf_contract_async_kernel<CB, 8>, 8);
    }
  }
  dim3 grid((unsigned)((a.S * rm + 127) / 128), (unsigned)a.num_groups);
  switch (rm) {
    case 1: leaf_contract_reg_kernel<R, CB, 1><<<grid, 128, 0, st>>>(a); break;
    case 2: leaf_contract_reg_kernel<R, CB, 2><<<grid, 128, 0, st>>>(a); break;
    case 4: leaf_contract_reg_kernel<R, CB, 4><<<grid, 128, 0, st>>>(a); break;
    default: leaf_contract_reg_kernel<R, CB, 8><<<grid, 128, 0, st>>>(a); break;
  }
  return cudaGetLastError();
}

template <typename R>
cudaError_t leaf_dispatch(const LeafArgs &a, cudaStream_t st) {
  using C = typename CT<R>::T;
  switch (a.c) {
    case 1: return leaf_reg_dispatch<R, 1>(a, st);
    case 2: return leaf_reg_dispatch<R, 2>(a, st);
    case 3: return leaf_reg_dispatch<R, 3>(a, st);
    case 4: return leaf_reg_dispatch<R, 4>(a, st);
    default: break;
  }
  dim3 grid((unsigned)((a.S + 127) / 128), (unsigned)a.num_groups);
  const int D = 1 << a.c;
  const size_t smem = (size_t)2 * a.r * D * (D + 1) * sizeof(C);
  switch (a.c) {
#define HSF_LEAF(CBV)                                                                         \
  case CBV: {                                                                                \
    auto k = leaf_contract_kernel<R, CBV>;                                                   \
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
    if (e != cudaSuccess) return e;                                                          \
    k<<<grid, 128, smem, st>>>(a);                                                           \
    break;                                                                                   \
  }
    HSF_LEAF(1) HSF_LEAF(2) HSF_LEAF(3) HSF_LEAF(4) HSF_LEAF(5)
#undef HSF_LEAF
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

bool leaf_streams(const LeafArgs &a, int precision) {
  // worth it once the bitstrings far outnumber the threads of one wave; the chunk
  // origins must fit 32 bits
  if (precision != 0 || a.c < 1 || a.c > 3 || a.S < 65536 || a.r > 8 || a.ha > 32 || a.hb > 32) return false;
  int grid = 0;
  int64_t pc = 0;
  switch (a.c) {
    case 1: return a.H ? leaf_stream_shape<1, true>(a.r, a.S, &grid, &pc) : leaf_stream_shape<1, false>(a.r, a.S, &grid, &pc);
    case 2: return a.H ? leaf_stream_shape<2, true>(a.r, a.S, &grid, &pc) : leaf_stream_shape<2, false>(a.r, a.S, &grid, &pc);
    default: return leaf_stream_shape<3, false>(a.r, a.S, &grid, &pc);
  }
}

bool leaf_factored(const LeafArgs &a, int precision) {
  return precision == 0 && a.pf >= 0 && a.pf < a.c && a.c >= 2 && a.c <= 4 && a.r >= 3 && a.r <= 4 &&
         a.ha <= 32 && a.hb <= 32 && !leaf_streams(a, precision);
}

template <int CB>
cudaError_t leaf_fact_launch(const LeafArgs &a, cudaStream_t st) {
  auto go = [&](auto kernel) -> cudaError_t {
    const size_t smem = leaf_fact_ring_bytes(CB);
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)((a.S + kFactSpb - 1) / kFactSpb), (unsigned)a.num_groups);
    kernel<<<grid, 128, smem, st>>>(a);
    return cudaGetLastError();
  };
  switch (a.pf) {
    case 0: return go(leaf_contract_fact_kernel<CB, 0>);
    case 1: return go(leaf_contract_fact_kernel<CB, (CB > 1 ? 1 : 0)>);
    case 2: return go(leaf_contract_fact_kernel<CB, (CB > 2 ? 2 : 0)>);
    default: return go(leaf_contract_fact_kernel<CB, (CB > 3 ? 3 : 0)>);
  }
}

cudaError_t launch_leaf_contract(const LeafArgs &a, int precision, cudaStream_t st) {
  if (a.S <= 0 || a.num_parents <= 0) return cudaSuccess;
  if (leaf_factored(a, precision)) {
    switch (a.c) {
      case 2: return leaf_fact_launch<2>(a, st);
      case 3: return leaf_fact_launch<3>(a, st);
      default: return leaf_fact_launch<4>(a, st);
    }
  }
  if (leaf_streams(a, precision)) {
    switch (a.c) {
      case 1: return a.H ? leaf_stream_launch<1, true>(a, st) : leaf_stream_launch<1, false>(a, st);
      case 2: return a.H ? leaf_stream_launch<2, true>(a, st) : leaf_stream_launch<2, false>(a, st);
      default: return leaf_stream_launch<3, false>(a, st);
    }
  }
  return precision == 0 ? leaf_dispatch<float>(a, st) : leaf_dispatch<double>(a, st);
}

// Counting sort of the bitstrings by the high bits of their side-a storage index (the
// streaming leaf kernel then gives each CTA bitstrings whose side-a chunks lie close
// together, so those gathers hit in L1).  Buckets are filled with atomics: the order
// inside a bucket varies, the results do not (every bitstring's sum is formed alone).
__global__ void sort_count_kernel(const uint64_t *ia, int64_t S, int shift, uint32_t *counts) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s < S) atomicAdd(&counts[ia[s] >> shift], 1u);
}
__global__ void __launch_bounds__(1024) sort_scan_kernel(uint32_t *counts, int nb) {
  // exclusive prefix sum of nb <= 4096 counters by one CTA (each thread a run of 4)
  __shared__ uint32_t part[1024];
  const int t = threadIdx.x;
  uint32_t v[4], sum = 0;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int i = 4 * t + k;
    v[k] = i < nb ? counts[i] : 0u;
    sum += v[k];
  }
  part[t] = sum;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {
    const uint32_t x = t >= o ? part[t - o] : 0u;
    __syncthreads();
    part[t] += x;
    __syncthreads();
  }
  uint32_t run = part[t] - sum;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int i = 4 * t + k;
    if (i < nb) counts[i] = run;
    run += v[k];
  }
}
__global__ void sort_scatter_kernel(const uint64_t *ia, const uint64_t *ib, int64_t S, int shift,
                                    uint32_t *offsets, uint64_t *ia_s, uint64_t *ib_s, int64_t *perm) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= S) return;
  const uint64_t a = ia[s];
  const uint32_t pos = atomicAdd(&offsets[a >> shift], 1u);
  ia_s[pos] = a;
  ib_s[pos] = ib[s];
  perm[pos] = s;
}

cudaError_t launch_bitstring_sort(const uint64_t *ia, const uint64_t *ib, int64_t S, int ha, uint32_t *counts,
                                  uint64_t *ia_s, uint64_t *ib_s, int64_t *perm, cudaStream_t st) {
  if (S <= 0) return cudaSuccess;
  const int bits = ha < kSortBits ? ha : kSortBits, shift = ha - bits, nb = 1 << bits;
  cudaError_t e = cudaMemsetAsync(counts, 0, (size_t)nb * sizeof(uint32_t), st);
  if (e != cudaSuccess) return e;
  const unsigned grid = (unsigned)((S + 255) / 256);
  sort_count_kernel<<<grid, 256, 0, st>>>(ia, S, shift, counts);
  sort_scan_kernel<<<1, 1024, 0, st>>>(counts, nb);
  sort_scatter_kernel<<<grid, 256, 0, st>>>(ia, ib, S, shift, counts, ia_s, ib_s, perm);
  return cudaGetLastError();
}

// Which 16-amplitude segments of the deepest stored level the leaf contraction reads:
// the segments covered by each bitstring's chunk on either side.
__global__ void chunk_mask_kernel(const uint64_t *ia, const uint64_t *ib, int64_t S, int c, uint32_t *mask_a,
                                  uint32_t *mask_b) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= S) return;
  const uint64_t D = 1ull << c;
  for (int side = 0; side < 2; ++side) {
    const uint64_t first = (side == 0 ? ia[s] : ib[s]) & ~(D - 1);
    uint32_t *mask = side == 0 ? mask_a : mask_b;
    for (uint64_t seg = first >> 4; seg <= (first + D - 1) >> 4; ++seg)
      atomicOr(&mask[seg >> 5], 1u << (seg & 31));
  }
}

cudaError_t launch_chunk_mask(const uint64_t *ia, const uint64_t *ib, int64_t S, int c, int ha, int hb,
                              uint32_t *mask_a, uint32_t *mask_b, cudaStream_t st) {
  if (S <= 0) return cudaSuccess;
  // at least one word per mask (a half state below 2^9 amplitudes has fewer than 32 bits)
  const size_t ba = ((((size_t)1 << (ha - 4)) + 31) / 32) * 4, bb = ((((size_t)1 << (hb - 4)) + 31) / 32) * 4;
  cudaError_t e = cudaMemsetAsync(mask_a, 0, ba, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(mask_b, 0, bb, st);
  if (e != cudaSuccess) return e;
  chunk_mask_kernel<<<(unsigned)((S + 255) / 256), 256, 0, st>>>(ia, ib, S, c, mask_a, mask_b);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Dot form of the factored leaf (Sec. IV-A, the leaf digits' sum folded into
// sum_{al,be} G[al][be] d_a[al] d_b[be]).  The deepest tree level's epilogue forms the
// four dots d[2 i + j] = sum_k S[rr][e_i(k)] x[e_j(k)] of every bitstring's chunk x
// (e_j(k) puts bit j at the factor's chunk bit) while the child rows are still in
// registers, so the children never reach memory; the leaf kernel below sums the
// bilinear form over the parents from those dots.  To find its bitstrings a level
// epilogue needs them grouped by segment, which the kernels here do once per run.
// ---------------------------------------------------------------------------
size_t dot_sort_bytes(int64_t S, int ha, int hb) {
  auto a256 = [](size_t x) { return (x + 255) / 256 * 256; };
  size_t t = 0;
  for (int s = 0; s < 2; ++s) {
    const size_t nb = (size_t)1 << ((s == 0 ? ha : hb) - 4);
    t += a256((nb + 1) * 4) + a256(nb * 4) + a256((size_t)S * 4);
  }
  return t + 2 * a256((size_t)S * 4) + 2 * a256(256 * 8);
}

DotSort dot_sort_layout(unsigned char *base, int64_t S, int ha, int hb) {
  auto a256 = [](size_t x) { return (x + 255) / 256 * 256; };
  DotSort d{};
  size_t o = 0;
  for (int s = 0; s < 2; ++s) {
    const size_t nb = (size_t)1 << ((s == 0 ? ha : hb) - 4);
    d.off[s] = reinterpret_cast<uint32_t *>(base + o);
    o += a256((nb + 1) * 4);
    d.cur[s] = reinterpret_cast<uint32_t *>(base + o);
    o += a256(nb * 4);
    d.list[s] = reinterpret_cast<uint32_t *>(base + o);
    o += a256((size_t)S * 4);
  }
  d.ida = reinterpret_cast<uint32_t *>(base + o);
  o += a256((size_t)S * 4);
  d.posb = reinterpret_cast<uint32_t *>(base + o);
  o += a256((size_t)S * 4);
  d.T[0] = reinterpret_cast<float2 *>(base + o);
  o += a256(256 * 8);
  d.T[1] = reinterpret_cast<float2 *>(base + o);
  return d;
}

struct DotSortArgs {
  const uint64_t *idx[2];
  int64_t S;
  int32_t nb[2];
  int32_t h[2];
  const float2 *Sm[2];
  DotSort d;
};
// key of storage index ix on a side of 2^h amplitudes: segment within the row, then row
__device__ __forceinline__ uint32_t dot_key(uint64_t ix, int h) {
  return (uint32_t)((((ix >> 4) & 3u) << (h - 6)) | (ix >> 6));
}

// blockIdx.y = side: count the bitstrings of each key into off[key + 1] (off zeroed);
// the first 256 threads also write the side's S transposed to [e][rr]
__global__ void dot_count_kernel(DotSortArgs a) {
  const int side = blockIdx.y;
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s < a.S) atomicAdd(&a.d.off[side][dot_key(a.idx[side][s], a.h[side]) + 1], 1u);
  if (s < 256) {
    const int e = (int)(s >> 4), rr = (int)(s & 15);
    a.d.T[side][s] = a.Sm[side][rr * 16 + e];
  }
}

// blockIdx.x = side: inclusive scan of off[1..nb] in place (off[0] = 0), so off[key] is
// the first position of a key; cur = off[0..nb) as the scatter's cursors
__global__ void __launch_bounds__(1024) dot_scan_kernel(DotSortArgs a) {
  __shared__ uint32_t part[1024];
  const int side = blockIdx.x, t = threadIdx.x;
  const int nb = a.nb[side];
  uint32_t *off = a.d.off[side] + 1;
  const int per = (nb + 1023) / 1024, i0 = min(nb, t * per), i1 = min(nb, i0 + per);
  uint32_t sum = 0;
  for (int i = i0; i < i1; ++i) sum += off[i];
  part[t] = sum;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {
    const uint32_t x = t >= o ? part[t - o] : 0u;
    __syncthreads();
    part[t] += x;
    __syncthreads();
  }
  uint32_t run = part[t] - sum;
  for (int i = i0; i < i1; ++i) {
    run += off[i];
    off[i] = run;
  }
  __syncthreads();
  for (int i = t; i < nb; i += 1024) a.d.cur[side][i] = a.d.off[side][i];
}

// blockIdx.y = side: each bitstring takes the next position of its key (the order
// inside a key varies from run to run; every bitstring's dots and sum do not)
__global__ void dot_scatter_kernel(DotSortArgs a) {
  const int side = blockIdx.y;
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= a.S) return;
  const uint64_t ix = a.idx[side][s];
  const uint32_t pos = atomicAdd(&a.d.cur[side][dot_key(ix, a.h[side])], 1u);
  a.d.list[side][pos] = (uint32_t)((ix >> 6) << 4) | (uint32_t)(ix & 15);
  if (side == 0)
    a.d.ida[pos] = (uint32_t)s;
  else
    a.d.posb[s] = pos;
}

cudaError_t launch_dot_sort(const uint64_t *ia, const uint64_t *ib, int64_t S, int ha, int hb, const void *Sa,
                            const void *Sb, const DotSort &d, cudaStream_t st) {
  if (S <= 0) return cudaSuccess;
  if (ha < 6 || hb < 6 || ha > 24 || hb > 24 || S > ((int64_t)1 << 30)) return cudaErrorInvalidValue;
  DotSortArgs a{};
  a.idx[0] = ia;
  a.idx[1] = ib;
  a.S = S;
  a.nb[0] = 1 << (ha - 4);
  a.nb[1] = 1 << (hb - 4);
  a.h[0] = ha;
  a.h[1] = hb;
  a.Sm[0] = static_cast<const float2 *>(Sa);
  a.Sm[1] = static_cast<const float2 *>(Sb);
  a.d = d;
  for (int s = 0; s < 2; ++s) {
    cudaError_t e = cudaMemsetAsync(d.off[s], 0, ((size_t)a.nb[s] + 1) * 4, st);
    if (e != cudaSuccess) return e;
  }
  const unsigned gx = (unsigned)((std::max<int64_t>(S, 256) + 255) / 256);
  dot_count_kernel<<<dim3(gx, 2), 256, 0, st>>>(a);
  dot_scan_kernel<<<2, 1024, 0, st>>>(a);
  dot_scatter_kernel<<<dim3((unsigned)((S + 255) / 256), 2), 256, 0, st>>>(a);
  return cudaGetLastError();
}

// One thread per bitstring, taken in side-a order (its side-a dots are read
// contiguously, its side-b dots gathered), parents [g ppg, (g + 1) ppg) of the chunk.
// The arithmetic, and its order, is that of leaf_contract_fact_kernel's two lanes: lane
// `side` adds d_a[2 side + {0, 1}] (G[2 side + {0, 1}] . d_b) into its own FP32 sum,
// and the two sums are added at the end.
__global__ void __launch_bounds__(256) leaf_dots_kernel(LeafArgs a) {
  using C = float2;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= a.S) return;
  const int g = blockIdx.y;
  const uint32_t id = a.dida[t];
  const int64_t tb = a.dposb[id];
  const C *Gt = reinterpret_cast<const C *>(a.G);
  const int r1 = a.r + 1;
  C gf[4][4];
  {
    const C *G = Gt + (size_t)a.r * 16;        // [m0 = 0][m1 = r]
#pragma unroll
    for (int al = 0; al < 4; ++al)
#pragma unroll
      for (int b = 0; b < 4; ++b) gf[al][b] = G[al * 4 + b];
  }
  const float4 *Da = static_cast<const float4 *>(a.Da), *Db = static_cast<const float4 *>(a.Db);
  const int64_t j0 = (int64_t)g * a.parents_per_group;
  const int64_t j1 = min(a.num_parents, j0 + a.parents_per_group);
  float accr[2] = {0.f, 0.f}, acci[2] = {0.f, 0.f};
#pragma unroll 2
  for (int64_t j = j0; j < j1; ++j) {
    const float4 a01 = __ldcs(Da + 2 * (j * a.S + t)), a23 = __ldcs(Da + 2 * (j * a.S + t) + 1);
    const float4 b01 = __ldcs(Db + 2 * (j * a.S + tb)), b23 = __ldcs(Db + 2 * (j * a.S + tb) + 1);
    const float ar[4] = {a01.x, a01.z, a23.x, a23.z}, ai[4] = {a01.y, a01.w, a23.y, a23.w};
    const float br[4] = {b01.x, b01.z, b23.x, b23.z}, bi[4] = {b01.y, b01.w, b23.y, b23.w};
    C h[4][4];
#pragma unroll
    for (int al = 0; al < 4; ++al)
#pragma unroll
      for (int b = 0; b < 4; ++b) h[al][b] = gf[al][b];
    if ((j == 0 && a.m_first > 0) || (j == a.num_parents - 1 && a.m_last < a.r)) {
      // a parent with only part of its digits in the path range
      const int m0 = j == 0 ? a.m_first : 0, m1 = j == a.num_parents - 1 ? a.m_last : a.r;
      const C *G = Gt + ((size_t)m0 * r1 + m1) * 16;
#pragma unroll
      for (int al = 0; al < 4; ++al)
#pragma unroll
        for (int b = 0; b < 4; ++b) h[al][b] = G[al * 4 + b];
    }
#pragma unroll
    for (int side = 0; side < 2; ++side) {
      float u0r = 0.f, u0i = 0.f, u1r = 0.f, u1i = 0.f;
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const C h0 = h[2 * side][b], h1 = h[2 * side + 1][b];
        u0r = fmaf(h0.x, br[b], fmaf(-h0.y, bi[b], u0r));
        u0i = fmaf(h0.x, bi[b], fmaf(h0.y, br[b], u0i));
        u1r = fmaf(h1.x, br[b], fmaf(-h1.y, bi[b], u1r));
        u1i = fmaf(h1.x, bi[b], fmaf(h1.y, br[b], u1i));
      }
      const float a0r = ar[2 * side], a0i = ai[2 * side], a1r = ar[2 * side + 1], a1i = ai[2 * side + 1];
      accr[side] = fmaf(a0r, u0r, fmaf(-a0i, u0i, accr[side]));
      acci[side] = fmaf(a0r, u0i, fmaf(a0i, u0r, acci[side]));
      accr[side] = fmaf(a1r, u1r, fmaf(-a1i, u1i, accr[side]));
      acci[side] = fmaf(a1r, u1i, fmaf(a1i, u1r, acci[side]));
    }
  }
  double *dst = a.partial + 2 * ((int64_t)g * a.S + id);
  dst[0] = (double)(accr[0] + accr[1]);
  dst[1] = (double)(acci[0] + acci[1]);
}

cudaError_t launch_leaf_dots(const LeafArgs &a, cudaStream_t st) {
  if (a.S <= 0 || a.num_parents <= 0) return cudaSuccess;
  if (!a.Da || !a.Db || !a.dida || !a.dposb || !a.G || a.r < 1) return cudaErrorInvalidValue;
  leaf_dots_kernel<<<dim3((unsigned)((a.S + 255) / 256), (unsigned)a.num_groups), 256, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_index_prep(const IndexArgs &a, cudaStream_t st) {
  if (a.S <= 0) return cudaSuccess;
  index_prep_kernel<<<(unsigned)((a.S + 255) / 256), 256, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_range_index(uint64_t *dst, int64_t count, const PermArgs &perm, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  range_index_kernel<<<(unsigned)((count + 255) / 256), 256, 0, st>>>(dst, count, perm);
  return cudaGetLastError();
}

cudaError_t launch_finalize(double *out, const double *comp, int64_t count, int32_t *numeric, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  finalize_kernel<<<(unsigned)((count + 255) / 256), 256, 0, st>>>(out, comp, count, numeric);
  return cudaGetLastError();
}

cudaError_t launch_state_gather(const void *state, int precision, const uint64_t *bits, int64_t count, double *out,
                                int32_t *numeric, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  const unsigned grid = (unsigned)((count + 255) / 256);
  if (precision == 0)
    state_gather_kernel<float><<<grid, 256, 0, st>>>(static_cast<const float *>(state), bits, count, out, numeric);
  else
    state_gather_kernel<double><<<grid, 256, 0, st>>>(static_cast<const double *>(state), bits, count, out, numeric);
  return cudaGetLastError();
}

cudaError_t launch_zero(double *p, int64_t count, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  zero_kernel<<<(unsigned)((count + 255) / 256), 256, 0, st>>>(p, count);
  return cudaGetLastError();
}

}  // namespace hsf
