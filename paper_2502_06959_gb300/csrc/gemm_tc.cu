// Path GEMM on the 5th-generation tensor cores (tcgen05) for full / window output.
//
// The path sum of Sec. II-B over the requested amplitude rectangle,
//   Out[x_a, x_b] = sum_p psi_a^p(x_a) psi_b^p(x_b),
// is a complex rank-P product.  It is written as one real GEMM C = A'' B''^T:
//   rows [0, Mp) of A'' give Re(Out), rows [Mp, 2Mp) give Im(Out);
//   K' = 2P columns hold (Re, -Im | Im, Re) of psi_a against (Re | Im) of psi_b;
//   the K' columns are repeated per split term: with x = hi + lo (hi = round(x), lo =
//   round(x - hi)) the product is hi*hi + hi*lo + lo*hi (split-BF16 or split-TF32,
//   3 terms) or a single TF32 term.
// pack_kernel gathers the leaf states at the window's storage indices and writes these
// operands (zero padded to the tile sizes); the a operand's real rows are interleaved
// (row 2i: Re of x_a = i, row 2i+1: Im).  gemm_kernel is persistent (one CTA per SM) and
// computes 128 x 256 tiles of C^T: the MMA's M dimension runs over 128 columns x_b (the
// b operand), its N dimension over 256 interleaved real rows (128 values of x_a).  One
// thread issues TMA tile loads (128-byte swizzle) into a 4-stage shared-memory ring, one
// thread issues tcgen05.mma into one of two TMEM accumulators (2 x 256 FP32 columns), and
// four epilogue warps drain the other: TMEM lane = x_b, columns = (Re, Im) pairs, so each
// thread adds complex values into the FP64 output (Neumaier compensation) and a warp's
// 16-byte stores cover 512 contiguous bytes.  Every wait on an mbarrier is bounded: on
// expiry the kernel records an error code, drains its MMAs and loads, frees its TMEM and
// returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <type_traits>

#include "common.h"

namespace hsf {
namespace {

constexpr int kBM = 128, kBN = 128, kStages = 4;   // padding: 128 x_b, 128 x_a (256 real rows)
constexpr int kGM = 128, kGN = 256;                 // MMA tile: M = x_b columns, N = real rows
constexpr int kTileA = kGM * 128, kTileB = kGN * 128;   // bytes: rows x 128 bytes of K
constexpr int kGemmThreads = 192;                   // TMA, MMA, 4 epilogue warps
constexpr uint32_t kWaitLimit = 1u << 22;           // bounded mbarrier polls (about a second)

// ---------------------------------------------------------------------------
// operand packing
// ---------------------------------------------------------------------------
__device__ __forceinline__ float tf32_round(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

template <int MODE>   // 1 = split bf16, 2 = split tf32, 3 = tf32
__device__ __forceinline__ void split(float x, float &hi, float &lo) {
  if (MODE == 1) {
    hi = __bfloat162float(__float2bfloat16_rn(x));
    lo = x - hi;
  } else {
    hi = tf32_round(x);
    lo = tf32_round(x - hi);
  }
}

struct PackArgs {
  const float2 *src;            // leaf states [paths][2^h]
  int32_t h;
  int64_t paths;
  int64_t rows;                 // M (a side) or N (b side)
  int64_t rows_pad;             // padded row count of one part
  int32_t side;                 // 0: a operand (2 x rows_pad rows), 1: b operand
  int64_t kpad;                 // padded K'' (row length of the operand)
  void *dst;                    // bf16 or fp32 operand, row-major [rows][kpad]
  // Rows are enumerated in storage order: enumeration index j has storage index
  // sum_k bit_k(j) << upos[k] and row (local index) sum_k bit_k(j) << ibit[k], with
  // upos ascending, so consecutive j read consecutive amplitudes.
  int32_t w;                    // enumerated bits: rows <= 2^w
  int8_t upos[64], ibit[64];
};

constexpr int kPackRows = 32, kPackPaths = 64;

// One CTA moves a tile of 32 rows x 64 paths: the reads run along the storage index of
// each path's leaf state, the tile is transposed in shared memory, and the writes run
// along K (paths) of each operand row.  Each path contributes K' = 2P columns per row;
// each split term is a further block of 2P columns.
template <int MODE>
__global__ void __launch_bounds__(256) pack_kernel(PackArgs a) {
  __shared__ float2 tile[kPackRows][kPackPaths + 1];
  const int lane = threadIdx.x & 31, wy = threadIdx.x >> 5;
  const int64_t j = (int64_t)blockIdx.x * kPackRows + lane;
  const int64_t p0 = ((int64_t)blockIdx.z * gridDim.y + blockIdx.y) * kPackPaths;
  uint64_t u = 0;
  int64_t i = 0;
  for (int k = 0; k < a.w; ++k)
    if ((j >> k) & 1) {
      u |= 1ull << a.upos[k];
      i |= 1ll << a.ibit[k];
    }
  const int rv = (j >> a.w) == 0 && i < a.rows;
#pragma unroll
  for (int t = 0; t < kPackPaths / 8; ++t) {
    const int pl = wy + 8 * t;
    const int64_t p = p0 + pl;
    float2 v = make_float2(0.f, 0.f);
    if (rv && p < a.paths) v = a.src[((uint64_t)p << a.h) + u];
    tile[lane][pl] = v;
  }
  __syncthreads();
  const int64_t P = a.paths, kp = 2 * P;
  constexpr int nterms = MODE == 3 ? 1 : 3;
#pragma unroll 1
  for (int t = 0; t < kPackRows / 8; ++t) {
    const int rl = wy + 8 * t;
    const int64_t ir = __shfl_sync(0xffffffffu, i, rl);
    if (!__shfl_sync(0xffffffffu, rv, rl)) continue;        // padding rows stay zero
#pragma unroll
    for (int hp = 0; hp < 2; ++hp) {
      const int pl = lane + 32 * hp;
      const int64_t p = p0 + pl;
      if (p >= P) continue;
      const float2 v = tile[rl][pl];
#pragma unroll
      for (int part = 0; part < 2; ++part) {
        if (a.side == 1 && part == 1) break;
        // the two K' entries of this path: columns p and P + p
        //   a Re row: ( Re a, -Im a );  a Im row: ( Im a, Re a );  b column: ( Re b, Im b )
        float x0, x1;
        if (a.side == 0) {
          x0 = part == 0 ? v.x : v.y;
          x1 = part == 0 ? -v.y : v.x;
        } else {
          x0 = v.x;
          x1 = v.y;
        }
        float h0, l0, h1, l1;
        split<MODE == 3 ? 2 : MODE>(x0, h0, l0);
        split<MODE == 3 ? 2 : MODE>(x1, h1, l1);
        // term order: a = [hi, hi, lo], b = [hi, lo, hi]  (hi*hi + hi*lo + lo*hi)
        float t0[3], t1[3];
        if (MODE == 3) {
          t0[0] = h0; t1[0] = h1;
        } else if (a.side == 0) {
          t0[0] = h0; t0[1] = h0; t0[2] = l0;
          t1[0] = h1; t1[1] = h1; t1[2] = l1;
        } else {
          t0[0] = h0; t0[1] = l0; t0[2] = h0;
          t1[0] = h1; t1[1] = l1; t1[2] = h1;
        }
        const int64_t r = a.side == 0 ? 2 * ir + part : ir;   // a: (Re, Im) rows interleaved
#pragma unroll
        for (int tt = 0; tt < nterms; ++tt) {
          const int64_t c0 = tt * kp + p, c1 = tt * kp + P + p;
          if (MODE == 1) {
            __nv_bfloat16 *d = reinterpret_cast<__nv_bfloat16 *>(a.dst) + r * a.kpad;
            d[c0] = __float2bfloat16_rn(t0[tt]);
            d[c1] = __float2bfloat16_rn(t1[tt]);
          } else {
            float *d = reinterpret_cast<float *>(a.dst) + r * a.kpad;
            d[c0] = t0[tt];
            d[c1] = t1[tt];
          }
        }
      }
    }
  }
}

// ---------------------------------------------------------------------------
// tcgen05 GEMM
// ---------------------------------------------------------------------------
struct EpiArgs {
  double *out, *comp;
  int64_t M, N;          // complex rows (x_a) and columns (x_b)
  int64_t Mp;            // padded complex rows (multiple of 128)
  int32_t hb;            // out index = x_a * 2^hb + x_b
  uint64_t window;
  int32_t k_tiles;
  int32_t kind;          // 0: kind::f16 (bf16 operands), 1: kind::tf32
  int32_t *err;          // device error word (0 = ok)
  int32_t num_m, num_n;  // tiles along the real rows (256 each) and along x_b (128 each)
  int32_t pad;
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
// Bounded wait for the phase with the given parity to complete; false on expiry.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
  const uint32_t a = smem_u32(bar);
  for (uint32_t it = 0; it < kWaitLimit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
      ::"r"(smem_u32(dst)), "l"((uint64_t)map), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

// Shared-memory matrix descriptor: K-major tile, 128-byte swizzle, 8-row atoms 1024 B apart.
__device__ __forceinline__ uint64_t make_desc(const void *tile) {
  const uint64_t addr = smem_u32(tile);
  uint64_t d = 0;
  d |= (addr & 0x3FFFFull) >> 4;               // start address
  d |= (uint64_t)1 << 16;                       // leading byte offset (unused with swizzle)
  d |= (uint64_t)(1024 >> 4) << 32;             // stride byte offset: 8 rows x 128 B
  d |= (uint64_t)1 << 46;                       // descriptor version
  d |= (uint64_t)2 << 61;                       // 128-byte swizzle
  return d;
}

__device__ __forceinline__ void neumaier(double &sum, double &c, double x) {
  const double t = sum + x;
  if (fabs(sum) >= fabs(x))
    c += (sum - t) + x;
  else
    c += (x - t) + sum;
  sum = t;
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t *bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__global__ void __launch_bounds__(kGemmThreads, 1) gemm_kernel(const __grid_constant__ CUtensorMap tmA,
                                                                const __grid_constant__ CUtensorMap tmB, EpiArgs ep) {
  // tmA: a operand (2 Mp interleaved real rows), tmB: b operand (Np rows of x_b)
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  uint8_t *sX = smem;                                   // b tiles (MMA A): kStages x 16 KB
  uint8_t *sY = smem + kStages * kTileA;                // a tiles (MMA B): kStages x 32 KB
  __shared__ __align__(8) uint64_t full_bar[kStages], empty_bar[kStages], tfull[2], tempty[2], drain;
  __shared__ uint32_t tmem_base_sh;
  __shared__ volatile int abort_sh;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // tiles: x_b tile major, real-row tile minor, so the CTAs in flight share x_b tiles
  // (read from DRAM once) while the small a operand stays in L2
  const int64_t tiles = (int64_t)ep.num_m * ep.num_n;
  const int ktiles = ep.k_tiles;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], 128);
    }
    mbar_init(&drain, 1);
    abort_sh = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {   // the whole warp allocates both accumulators
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_sh)),
                 "r"(2 * kGN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base_sh;

  if (warp == 0) {
    if (lane == 0) {
      // TMA producer: k-tiles of every tile this CTA owns, one ring across tiles
      int64_t it = 0, issued = 0;
      for (int64_t t = blockIdx.x; t < tiles && !abort_sh; t += gridDim.x) {
        const int x0 = (int)(t / ep.num_m) * kGM, y0 = (int)(t % ep.num_m) * kGN;
        for (int kt = 0; kt < ktiles; ++kt, ++it) {
          const int s = (int)(it % kStages);
          const uint32_t ph = (uint32_t)(it / kStages) & 1u;
          if (!mbar_wait(&empty_bar[s], ph ^ 1u)) { atomicExch(ep.err, 1); abort_sh = 1; break; }
          mbar_expect_tx(&full_bar[s], kTileA + kTileB);
          const int kx = kt * (ep.kind == 0 ? 64 : 32);   // K elements per 128-byte row
          tma_load_2d(sX + s * kTileA, &tmB, kx, x0, &full_bar[s]);
          tma_load_2d(sY + s * kTileB, &tmA, kx, y0, &full_bar[s]);
          issued = it + 1;
        }
      }
      // every load issued has landed before the CTA can exit (matters only on abort)
      for (int64_t i = issued > kStages ? issued - kStages : 0; i < issued; ++i)
        if (!mbar_wait(&full_bar[i % kStages], (uint32_t)(i / kStages) & 1u)) atomicExch(ep.err, 10);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // MMA issuer: D[x_b][real row] += B-tile rows x a-tile rows, accumulator t % 2
      const uint32_t fmt = ep.kind == 0 ? 1u : 2u;        // BF16 (kind::f16) or TF32
      const uint32_t idesc = (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(kGN >> 3) << 17) |
                             ((uint32_t)(kGM >> 4) << 24);
      int64_t it = 0, tl = 0;
      bool ok = true;
      for (int64_t t = blockIdx.x; t < tiles && ok && !abort_sh; t += gridDim.x, ++tl) {
        const int b = (int)(tl & 1);
        if (!mbar_wait(&tempty[b], ((uint32_t)(tl >> 1) & 1u) ^ 1u)) { atomicExch(ep.err, 5); abort_sh = 1; break; }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t d = tmem + (uint32_t)(b * kGN);
        for (int kt = 0; kt < ktiles; ++kt, ++it) {
          const int s = (int)(it % kStages);
          const uint32_t ph = (uint32_t)(it / kStages) & 1u;
          if (!mbar_wait(&full_bar[s], ph)) { atomicExch(ep.err, 2); abort_sh = 1; ok = false; break; }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint64_t da = make_desc(sX + s * kTileA), db = make_desc(sY + s * kTileB);
#pragma unroll
          for (int k = 0; k < 4; ++k) {                    // 4 MMAs of 32 bytes of K per k-tile
            const uint64_t adv = (uint64_t)((k * 32) >> 4);
            const uint32_t acc = (kt > 0 || k > 0) ? 1u : 0u;
            if (ep.kind == 0) {
              asm volatile(
                  "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
                  " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
                  ::"r"(d), "l"(da + adv), "l"(db + adv), "r"(idesc), "r"(acc)
                  : "memory");
            } else {
              asm volatile(
                  "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
                  " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n"
                  ::"r"(d), "l"(da + adv), "l"(db + adv), "r"(idesc), "r"(acc)
                  : "memory");
            }
          }
          mma_commit(&empty_bar[s]);                        // the stage is free once these finish
        }
        if (!ok) break;
        mma_commit(&tfull[b]);                              // accumulator b is complete
      }
      // every MMA issued above has finished before TMEM is released
      mma_commit(&drain);
      if (!mbar_wait(&drain, 0)) atomicExch(ep.err, 7);
    }
  } else {
    // ---- epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31, i.e. x_b = x0 + that
    // lane; the accumulator's columns are 128 (Re, Im) pairs of x_a = y0 / 2 + c ----
    const int q4 = warp & 3;
    int64_t tl = 0;
    for (int64_t t = blockIdx.x; t < tiles; t += gridDim.x, ++tl) {
      const int b = (int)(tl & 1);
      const bool ok = mbar_wait(&tfull[b], (uint32_t)(tl >> 1) & 1u);
      if (!__all_sync(0xffffffffu, ok)) {
        if (lane == 0) atomicExch(ep.err, 3);
        abort_sh = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const int64_t j = (t / ep.num_m) * kGM + q4 * 32 + lane;          // x_b
      const int64_t i0 = (t % ep.num_m) * (kGN / 2);                     // first x_a
#pragma unroll 1
      for (int c0 = 0; c0 < kGN; c0 += 32) {
        uint32_t v[32];
        const uint32_t taddr = tmem + ((uint32_t)(q4 * 32) << 16) + (uint32_t)(b * kGN + c0);
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
            "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
              "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
              "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
              "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
            : "r"(taddr));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (j < ep.N) {
          // 8 pairs at a time: load their running sums first (independent requests), then fold
#pragma unroll
          for (int h8 = 0; h8 < 16; h8 += 8) {
            double2 sum[8], cmp[8];
            uint64_t idx[8];
            bool in[8];
#pragma unroll
            for (int c = 0; c < 8; ++c) {
              const int64_t i = i0 + c0 / 2 + h8 + c;
              idx[c] = ((uint64_t)i << ep.hb) + (uint64_t)j;
              in[c] = i < ep.M && idx[c] < ep.window;
              if (in[c]) {
                sum[c] = reinterpret_cast<const double2 *>(ep.out)[idx[c]];
                cmp[c] = reinterpret_cast<const double2 *>(ep.comp)[idx[c]];
              }
            }
#pragma unroll
            for (int c = 0; c < 8; ++c) {
              if (!in[c]) continue;
              neumaier(sum[c].x, cmp[c].x, (double)__uint_as_float(v[2 * (h8 + c)]));
              neumaier(sum[c].y, cmp[c].y, (double)__uint_as_float(v[2 * (h8 + c) + 1]));
              reinterpret_cast<double2 *>(ep.out)[idx[c]] = sum[c];
              reinterpret_cast<double2 *>(ep.comp)[idx[c]] = cmp[c];
            }
          }
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      mbar_arrive(&tempty[b]);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 1) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * kGN) : "memory");
  }
}

// ---------------------------------------------------------------------------
// Tensor-core tree level
// ---------------------------------------------------------------------------
// Child g of a level whose program (or its leading ops) sits on the 6 lowest storage bits
// is U_m applied to every 64-amplitude row of its parent (m = g % radix).  Real form,
// k = 2 r + (re, im): child[row][n] = sum_k W_m[n][k] parent[row][k], W_m 128 x 128.
// A CTA serves one digit.  W_m's TF32 hi and lo parts sit in tensor memory as the MMA's
// A operand (lanes = output component n, columns = k), so shared memory holds only the
// streamed parent rows: 128-row tiles (MMA N = 128) in 32-float K-chunks.  One thread
// issues TMA loads (128-byte swizzle) into a 4-stage ring; four warps compute each
// chunk's TF32 low part; one thread issues W_hi P_hi + W_hi P_lo + W_lo P_hi
// (tcgen05.mma kind::tf32, A from TMEM) into one of two TMEM accumulators; two groups of
// four warps read the other back, stage 32-row quarters in shared memory for the ops that
// follow the product and write the child rows with bulk copies.  This kernel serves the
// levels with ops after the product; level_mma_f16_kernel the others.  Every wait is
// bounded; on expiry the CTA records an error, drains its MMAs and loads, frees TMEM and
// returns.
constexpr int kLvlRaw = 4;                      // TMA stages (raw FP32 chunks = the hi parts)
constexpr int kLvlLo = 3;                       // low-part buffers
constexpr int kLvlOut = 6;                      // 32-row output staging buffers (16 KB each)
constexpr int kLvlChunk = 128 * 128;            // bytes: 128 rows x 32 floats
constexpr int kLvlThreads = 576;                // 4 low-part, 3 x 4 epilogue, 1 MMA, 1 TMA warp
constexpr uint32_t kLvlTmemCols = 512;          // W hi [0,128), W lo [128,256), D 2 x 128
constexpr size_t kLvlSmem = (size_t)(kLvlRaw + kLvlLo + kLvlOut) * kLvlChunk + 1024;

// D (TMEM) += A (TMEM) x B (shared-memory descriptor)
__device__ __forceinline__ void mma_tf32_ts(uint32_t d, uint32_t a, uint64_t db, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n}\n"
      ::"r"(d), "r"(a), "l"(db), "r"(idesc), "r"(acc)
      : "memory");
}

// One post-product op on a staged quarter: element i (i < 2^11) of the quarter is
// amplitude i & 63 of row i >> 6, at stage[(i >> 6) * 128 + 2 * (i & 63)] (re, im); its
// index bits are the storage bits 0..10.  The 128 epilogue threads (t) split the work.
__device__ __forceinline__ uint32_t ins0(uint32_t v, int b) { return ((v >> b) << (b + 1)) | (v & ((1u << b) - 1u)); }
__device__ __forceinline__ float2 *post_elem(float *stage, uint32_t i) {
  return reinterpret_cast<float2 *>(stage + (i >> 6) * 128 + 2 * (i & 63));
}
__device__ __forceinline__ float2 cmulf(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
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

__device__ __forceinline__ void apply_post_op(float *stage, const MmaPostOp *op, int t) {
  // the op (staged in shared memory) is read into registers once, not per element
  const int nq = op->nq, q0 = op->q0, q1 = op->q1, diag = op->diag;
  if (diag) {
    const float2 d0 = op->m[0], d1 = op->m[1];
    const float2 d2 = nq == 2 ? op->m[2] : d0, d3 = nq == 2 ? op->m[3] : d1;
    for (uint32_t i = t; i < 2048; i += 128) {
      const uint32_t b0 = (i >> q0) & 1u;
      float2 m;
      if (nq == 2) {
        const uint32_t b1 = (i >> q1) & 1u;
        m = b0 ? (b1 ? d3 : d2) : (b1 ? d1 : d0);
      } else {
        m = b0 ? d1 : d0;
      }
      float2 *e = post_elem(stage, i);
      *e = cmulf(m, *e);
    }
  } else if (nq == 1) {
    const float2 m0 = op->m[0], m1 = op->m[1], m2 = op->m[2], m3 = op->m[3];
    for (uint32_t j = t; j < 1024; j += 128) {
      const uint32_t i0 = ins0(j, q0), i1 = i0 | (1u << q0);
      float2 *e0 = post_elem(stage, i0), *e1 = post_elem(stage, i1);
      const float2 x0 = *e0, x1 = *e1;
      const float2 a = cmulf(m0, x0), b = cmulf(m1, x1), c = cmulf(m2, x0), d = cmulf(m3, x1);
      *e0 = make_float2(a.x + b.x, a.y + b.y);
      *e1 = make_float2(c.x + d.x, c.y + d.y);
    }
  } else {
    // two-qubit dense op: the matrix as broadcast pairs (Re m, Re m) and (Im m, Im m), so
    // that with x_k = (Re x_k, Im x_k) as it sits in the stage, P = sum mr * x and
    // Q = sum mi * x are packed FMAs and (m x)_r = (P.x - Q.y, P.y + Q.x)
    float2 mr[16], mi[16];
#pragma unroll
    for (int e = 0; e < 16; ++e) {
      const float2 v = op->m[e];
      mr[e] = make_float2(v.x, v.x);
      mi[e] = make_float2(v.y, v.y);
    }
    const int lo = min(q0, q1), hi = max(q0, q1);
    for (uint32_t j = t; j < 512; j += 128) {
      const uint32_t base = ins0(ins0(j, lo), hi);
      float2 *e[4];
      float2 x[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        e[k] = post_elem(stage, base | ((uint32_t)(k >> 1) << q0) | ((uint32_t)(k & 1) << q1));
        x[k] = *e[k];
      }
      float2 y[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        float2 P = make_float2(0.f, 0.f), Q = P;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          P = ffma2(mr[r * 4 + k], x[k], P);
          Q = ffma2(mi[r * 4 + k], x[k], Q);
        }
        y[r] = make_float2(P.x - Q.y, P.y + Q.x);
      }
#pragma unroll
      for (int k = 0; k < 4; ++k) *e[k] = y[k];
    }
  }
}

__global__ void __launch_bounds__(kLvlThreads, 1) level_mma_kernel(const __grid_constant__ CUtensorMap tmP,
                                                                  LevelMmaArgs a) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  uint8_t *sR = smem;                                   // raw stage r (hi part): sR + r * kLvlChunk
  uint8_t *sL = sR + kLvlRaw * kLvlChunk;               // low-part buffer l: sL + l * kLvlChunk
  float *sO = reinterpret_cast<float *>(sL + kLvlLo * kLvlChunk);   // output staging: [6][32 rows][128]
  __shared__ __align__(8) uint64_t loaded[kLvlRaw], raw_empty[kLvlRaw], full_bar[kLvlLo], lo_empty[kLvlLo], tfull[2],
      tempty[2], drain;
  __shared__ uint32_t tmem_sh;
  __shared__ volatile int abort_sh, epi_abort[3];
  __shared__ __align__(16) MmaPostOp post_sh[kMmaMaxPost];   // the epilogue's ops, staged once
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t radix = a.radix;
  const int m = blockIdx.y;
  {
    constexpr int kWords = (int)(sizeof(MmaPostOp) / 16);
    const int n = min(a.num_post, kMmaMaxPost) * kWords;
    for (int e = threadIdx.x; e < n; e += blockDim.x)
      reinterpret_cast<int4 *>(post_sh)[e] = reinterpret_cast<const int4 *>(a.post)[e];
  }
  const int64_t g_first = a.node_lo + ((m - a.node_lo % radix) % radix + radix) % radix;
  const int64_t g_end = a.node_lo + a.num_nodes;
  const int64_t nchild = g_first < g_end ? (g_end - g_first + radix - 1) / radix : 0;
  const int tb = a.h - kMmaMinH;                        // 2^tb row tiles per node
  const int64_t units = nchild << tb;
  const int64_t nchunks = units > blockIdx.x ? ((units - 1 - blockIdx.x) / gridDim.x + 1) * 4 : 0;

  if (threadIdx.x == 0) {
    epi_abort[0] = epi_abort[1] = epi_abort[2] = 0;
    for (int s = 0; s < kLvlRaw; ++s) {
      mbar_init(&loaded[s], 1);
      mbar_init(&raw_empty[s], 1);
    }
    for (int s = 0; s < kLvlLo; ++s) {
      mbar_init(&full_bar[s], 128);
      mbar_init(&lo_empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], 384);
    }
    mbar_init(&drain, 1);
    abort_sh = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 8) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_sh)),
                 "r"(kLvlTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_sh;
  if (warp >= 4 && warp < 8) {
    // W_m into TMEM: lane n holds row n; columns [0,128) the hi part, [128,256) the lo part
    const int q4 = warp & 3;
    const float *wrow = reinterpret_cast<const float *>(a.w) + (size_t)m * 2 * 128 * 128 + (size_t)(q4 * 32 + lane) * 128;
#pragma unroll 1
    for (int c = 0; c < 8; ++c) {
      const float *src = wrow + (size_t)(c >> 2) * 128 * 128 + (c & 3) * 32;
      uint32_t v[32];
#pragma unroll
      for (int j = 0; j < 32; j += 4) {
        const float4 x = *reinterpret_cast<const float4 *>(src + j);
        v[j] = __float_as_uint(x.x);
        v[j + 1] = __float_as_uint(x.y);
        v[j + 2] = __float_as_uint(x.z);
        v[j + 3] = __float_as_uint(x.w);
      }
      const uint32_t taddr = tmem + ((uint32_t)(q4 * 32) << 16) + (uint32_t)(c * 32);
      asm volatile(
          "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,"
          "%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};" ::"r"(taddr),
          "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]), "r"(v[8]),
          "r"(v[9]), "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15]), "r"(v[16]),
          "r"(v[17]), "r"(v[18]), "r"(v[19]), "r"(v[20]), "r"(v[21]), "r"(v[22]), "r"(v[23]), "r"(v[24]),
          "r"(v[25]), "r"(v[26]), "r"(v[27]), "r"(v[28]), "r"(v[29]), "r"(v[30]), "r"(v[31])
          : "memory");
    }
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

  if (warp < 4) {
    // ---- low parts: lo = x - (x with its 13 low mantissa bits cleared) ----
    // The TMA lands the raw FP32 chunk in a raw stage; kind::tf32 reads only the top 19
    // bits of each operand, so the hi part is that truncation and lo is exact.
    const int t = threadIdx.x;
    for (int64_t it = 0; it < nchunks && !abort_sh; ++it) {
      const int r = (int)(it % kLvlRaw), l = (int)(it % kLvlLo);
      if (!mbar_wait(&loaded[r], (uint32_t)(it / kLvlRaw) & 1u) ||
          !mbar_wait(&lo_empty[l], ((uint32_t)(it / kLvlLo) & 1u) ^ 1u)) {
        atomicExch(a.err, 4);
        abort_sh = 1;
        break;
      }
      const uint8_t *hi = sR + r * kLvlChunk;
      uint8_t *lo = sL + l * kLvlChunk;
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const uint32_t off = (uint32_t)(t + 128 * i) * 16;    // same swizzled place in both
        const float4 x = *reinterpret_cast<const float4 *>(hi + off);
        float4 v;
        v.x = x.x - __uint_as_float(__float_as_uint(x.x) & 0xffffe000u);
        v.y = x.y - __uint_as_float(__float_as_uint(x.y) & 0xffffe000u);
        v.z = x.z - __uint_as_float(__float_as_uint(x.z) & 0xffffe000u);
        v.w = x.w - __uint_as_float(__float_as_uint(x.w) & 0xffffe000u);
        *reinterpret_cast<float4 *>(lo + off) = v;
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mbar_arrive(&full_bar[l]);
    }
  } else if (warp == 9) {
    // ---- TMA: chunk c = chunk c % 4 of unit blockIdx.x + (c / 4) * gridDim.x ----
    if (lane == 0) {
      auto row_of = [&](int64_t c) {
        const int64_t u = blockIdx.x + (c >> 2) * gridDim.x;
        const int64_t g = g_first + (u >> tb) * radix;
        return ((g / radix - a.parent_lo) << (a.h - kMmaBits)) + ((u & ((1 << tb) - 1)) << 7);
      };
      int64_t issued = 0;
      for (int64_t it = 0; it < nchunks && !abort_sh; ++it) {
        const int s = (int)(it % kLvlRaw);
        const uint32_t ph = (uint32_t)(it / kLvlRaw) & 1u;

        if (!mbar_wait(&raw_empty[s], ph ^ 1)) {
          atomicExch(a.err, 9);
          abort_sh = 1;
          break;
        }
        mbar_expect_tx(&loaded[s], kLvlChunk);
        tma_load_2d(sR + s * kLvlChunk, &tmP, (int)(it & 3) * 32, (int)row_of(it), &loaded[s]);
        issued = it + 1;
      }
      // every load issued has landed before the CTA can exit (matters only on abort)
      for (int64_t it = issued > kLvlRaw ? issued - kLvlRaw : 0; it < issued; ++it)
        if (!mbar_wait(&loaded[it % kLvlRaw], (uint32_t)(it / kLvlRaw) & 1u)) atomicExch(a.err, 10);
    }
    __syncwarp();
  } else if (warp == 8) {
    // ---- MMA issuer ----
    if (lane == 0) {
      const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(128 >> 3) << 17) |
                             ((uint32_t)(128 >> 4) << 24);
      int64_t it = 0, tu = 0;
      for (int64_t u = blockIdx.x; u < units && !abort_sh; u += gridDim.x, ++tu) {
        const int b = (int)(tu & 1);
        if (!mbar_wait(&tempty[b], ((uint32_t)(tu >> 1) & 1u) ^ 1u)) {
          atomicExch(a.err, 5);
          abort_sh = 1;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t d = tmem + 256u + (uint32_t)(b * 128);
        bool ok = true;
        for (int kc = 0; kc < 4; ++kc, ++it) {
          const int r = (int)(it % kLvlRaw), l = (int)(it % kLvlLo);
          if (!mbar_wait(&full_bar[l], (uint32_t)(it / kLvlLo) & 1u)) {
            atomicExch(a.err, 6);
            abort_sh = 1;
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint64_t phi = make_desc(sR + r * kLvlChunk), plo = make_desc(sL + l * kLvlChunk);
          // D[n][row] = sum_k W[n][k] parent[row][k]: W (TMEM) is the MMA's A operand
          // (M = 128 output components), the parent rows its B operand (N = 128 rows)
#pragma unroll
          for (int term = 0; term < 3; ++term) {
            const uint64_t dp = term == 1 ? plo : phi;
            const uint32_t wcol = (term == 2 ? 128u : 0u) + (uint32_t)(kc * 32);
#pragma unroll
            for (int k = 0; k < 4; ++k)      // 8 TF32 of K per MMA (32 bytes, 8 columns)
              mma_tf32_ts(d, tmem + wcol + 8u * k, dp + 2 * k, idesc, (kc | term | k) ? 1u : 0u);
          }
          mma_commit(&raw_empty[r]);          // both buffers are free once these MMAs finish
          mma_commit(&lo_empty[l]);
        }
        if (!ok) break;
        mma_commit(&tfull[b]);                // the accumulator is complete
      }
      // every MMA issued above has finished before TMEM is released
      mma_commit(&drain);
      if (!mbar_wait(&drain, 0)) atomicExch(a.err, 7);
    }
    __syncwarp();
  } else {
    // ---- epilogue: three groups of four warps (4..7, 10..13 and 14..17) take the 32-row
    // quarters of the accumulators round-robin (quarter q of unit tu goes to group
    // (4 tu + q) mod 3), so up to three quarters get their ops at once.  TMEM lane quarter (warp & 3) holds output
    // components 32 (warp & 3) .. + 31; TMEM column j of the accumulator is row j of the
    // tile.  A quarter is staged in shared memory row-major (the global layout), gets the
    // rest of the level's program, and goes out as one bulk copy (its 32 rows are 16 KB
    // contiguous in the child state). ----
    const int grp = warp >= 14 ? 2 : (warp >= 10 ? 1 : 0);
    const uint32_t bar_id = 1 + grp;                     // named barrier of the group
    const int q4 = warp & 3;
    const int comp = q4 * 32 + lane;
    const bool leader = q4 == 0 && lane == 0;
    constexpr int kOutPerGroup = kLvlOut / 3;
    int64_t tu = 0, nq = 0;                              // units done, quarters stored
    // The four warps of a group meet at named barriers, so they decide to stop together:
    // only they write their epi_abort word, before a barrier, and all read it after.
    for (int64_t u = blockIdx.x; u < units; u += gridDim.x, ++tu) {
      const int b = (int)(tu & 1);
      const bool ok = mbar_wait(&tfull[b], (uint32_t)(tu >> 1) & 1u);
      if (!ok) epi_abort[grp] = 1;
      asm volatile("bar.sync %0, 128;" ::"r"(bar_id) : "memory");
      if (epi_abort[grp]) {
        if (!ok) atomicExch(a.err, 8);
        abort_sh = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const int64_t g = g_first + (u >> tb) * radix;
      float *dst = a.child + (((uint64_t)(g - a.node_lo) << a.h) + ((uint64_t)(u & ((1 << tb) - 1)) << 13)) * 2;
#pragma unroll 1
      for (int qr = 0; qr < 4; ++qr) {
        if ((int)((tu * 4 + qr) % 3) != grp) continue;
        uint32_t v[32];
        const uint32_t taddr = tmem + ((uint32_t)(q4 * 32) << 16) + 256u + (uint32_t)(b * 128 + qr * 32);
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
            "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
              "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
              "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
              "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
            : "r"(taddr));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        // this group's staging buffer was last read by its bulk copy kOutPerGroup quarters ago
        if (leader && nq >= kOutPerGroup)
          asm volatile("cp.async.bulk.wait_group.read %0;" ::"n"(kOutPerGroup - 1) : "memory");
        asm volatile("bar.sync %0, 128;" ::"r"(bar_id) : "memory");
        float *stage = sO + (size_t)(grp * kOutPerGroup + nq % kOutPerGroup) * 32 * 128;
#pragma unroll
        for (int j = 0; j < 32; ++j) stage[j * 128 + comp] = __uint_as_float(v[j]);
        // the rest of the level's program, on storage bits 0..10 of this quarter
        for (int o = 0; o < a.num_post; ++o) {
          asm volatile("bar.sync %0, 128;" ::"r"(bar_id) : "memory");
          apply_post_op(stage, post_sh + o, comp);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("bar.sync %0, 128;" ::"r"(bar_id) : "memory");
        if (leader) {
          asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst + (size_t)qr * 32 * 128),
                       "r"(smem_u32(stage)), "r"(32 * 128 * 4)
                       : "memory");
          asm volatile("cp.async.bulk.commit_group;" ::: "memory");
        }
        ++nq;
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      mbar_arrive(&tempty[b]);
    }
    // the CTA exits only once its output copies are complete
    if (leader) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 8) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kLvlTmemCols) : "memory");
  }
}

// ---------------------------------------------------------------------------
// Tensor-core tree level, FP16 split (levels with no ops after the product)
// ---------------------------------------------------------------------------
// Same product as level_mma_kernel, with both operands split into FP16 hi and lo parts:
// W_hi P_hi + W_hi P_lo + W_lo P_hi (tcgen05.mma kind::f16, FP32 accumulate), twice the
// tensor rate of TF32.  FP16's exponent range is handled by powers of two: W_m is scaled
// on the host so that its largest entry lies in [2^14, 2^15), and every 64-amplitude
// parent row by its own power of two (largest component in [2^14, 2^15)); hi is the
// scaled value rounded to a multiple of 16 (exact in FP16) and lo the FP16 rounding of
// the exact rest (|lo| <= 8), so each operand is split within 2^-23 of its row's (or
// W_m's) largest entry.  The epilogue multiplies each output row by both inverse scales,
// which is exact.  W_m's parts sit in tensor memory as the MMA's A operand (lanes =
// output component n, columns = k, two FP16 per column).  Eight split warps stream the raw
// FP32 parent rows through a shared-memory ring with cp.async (each warp copies the rows
// it converts) and write the FP16 hi and lo B operands of a 128-row unit (K-major,
// 128-byte swizzle, two buffers).  A CTA serves two Schmidt digits (both W_m in tensor
// memory), so each parent unit is streamed and split once for two children; one thread
// issues each digit's 24 MMAs into one of two TMEM accumulators in turn; two groups of
// four warps read the other back, unscale it and store the child rows from registers.
// With one digit per CTA the split's input latency bounded the kernel; with two, the
// level runs close to its read/write pattern's DRAM rate.  A level with ops after the
// product uses the TF32 kernel, whose epilogue stages rows in the shared memory this one
// spends on the split's operand buffers.  Every wait is bounded; on expiry the CTA
// records an error, drains its MMAs and copies, frees TMEM and returns.
constexpr int kHQuarter = 32 * 512;             // bytes: 32 parent rows x 128 floats
constexpr int kHRaw = 5;                        // raw quarters in the ring
constexpr int kHOps = 2;                        // FP16 operand buffers (one 128-row unit each)
constexpr int kHAtom = 128 * 128;               // bytes: 128 rows x 64 FP16 (one swizzle atom column)
constexpr int kHOpBytes = 4 * kHAtom;           // hi (K 0..63, 64..127) then lo (same)
constexpr int kHDigits = 2;                     // Schmidt digits per CTA (W_m of each in TMEM)
constexpr int kHSplit = 8;                      // split warps: 0..3 and 13..16
constexpr int kHSplitThreads = kHSplit * 32;
constexpr int kHThreads = (9 + kHSplit) * 32;   // + 2 x 4 epilogue warps and the MMA warp
constexpr uint32_t kHTmemCols = 512;            // W_i hi 128 i + [0,64), lo + [64,128); D 2 x 128 at 256
constexpr size_t kHSmem = (size_t)kHOps * kHOpBytes + (size_t)kHRaw * kHQuarter + 1024;
static_assert(kHSmem <= 227 * 1024 - 4096, "FP16 level kernel shared memory");
// Dot form: each epilogue warp stages 16 rows of its 16-amplitude segment (2 KB) for the
// lanes that form the leaf dots, and keeps the bitstring entries of its unit's rows
// (kDotMeta, 1 KB); the CTA keeps S as the [e][rr] table (2 KB).  For that room the raw
// ring has four stages, the row scales are kept as exponent bytes and the store mask is
// not used.
constexpr int kDotRows = 16;
constexpr int kHRawDots = 4;
constexpr int kDotMeta = 256;                   // entries per warp held in shared memory
constexpr size_t kHSmemDots = (size_t)kHOps * kHOpBytes + (size_t)kHRawDots * kHQuarter + 1024;
static_assert(kHSmemDots + 8 * kDotRows * 128 + 2048 + 8 * kDotMeta * 4 + 4 * 128 + 256 <= 227 * 1024,
              "FP16 level kernel shared memory (dot form)");

__device__ __forceinline__ void lvl_cp_async16(uint32_t dst, const void *src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void lvl_cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void lvl_cp_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }
// D (TMEM) += A (TMEM) x B (shared-memory descriptor), FP16 operands
__device__ __forceinline__ void mma_f16_ts(uint32_t d, uint32_t a, uint64_t db, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}\n"
      ::"r"(d), "r"(a), "l"(db), "r"(idesc), "r"(acc)
      : "memory");
}
// explicit shared-space accesses (the buffers are reached through an aligned generic
// pointer, which the compiler cannot place in shared memory by itself)
__device__ __forceinline__ float4 lds128(uint32_t addr) {
  float4 v;
  asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(addr));
  return v;
}
__device__ __forceinline__ void sts128(uint32_t addr, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
  asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(a), "r"(b), "r"(c), "r"(d) : "memory");
}
__device__ __forceinline__ uint32_t h2_bits(__half2 h) {
  uint32_t u;
  memcpy(&u, &h, 4);
  return u;
}

constexpr int kHMaskWords = (1 << (17 - 4)) / 32;   // store mask of a half state of up to 2^17 amplitudes

template <int PF>
__global__ void __launch_bounds__(kHThreads, 1) level_mma_f16_kernel(LevelMmaArgs a) {
  constexpr bool DOTS = PF >= 0;
  constexpr int RAW = DOTS ? kHRawDots : kHRaw;   // raw quarters in the ring
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  uint8_t *sOp = smem;                                  // operand buffer o: sOp + o * kHOpBytes
  uint8_t *sR = sOp + kHOps * kHOpBytes;            // raw quarter r: sR + r * kHQuarter
  __shared__ __align__(8) uint64_t ops_full[kHOps], ops_empty[kHOps],
      sc_full[4], tfull[2], tempty[2], drain;
  // per unit (4 in flight): 1 / row scale (dot form: the scale's exponent byte)
  __shared__ typename std::conditional<DOTS, uint8_t, float>::type row_inv[4][128];
  __shared__ uint32_t tmem_sh;
  __shared__ volatile int abort_sh, epi_abort[2];
  __shared__ uint32_t mask_sh[DOTS ? 1 : kHMaskWords];  // the store mask, when it fits
  // dot form: per epilogue warp a row tile and an entry buffer; S as [e][rr]
  __shared__ __align__(16) float dot_tile[DOTS ? 8 * kDotRows * 32 : 4];
  __shared__ __align__(16) float2 dot_S[DOTS ? 256 : 1];   // S[rr][e] at [e][rr]
  __shared__ uint32_t dot_meta[DOTS ? 8 * kDotMeta : 1];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t radix = a.radix;
  // 2^(h-4) mask bits; staged in shared memory for h <= 17 (visible after the first
  // __syncthreads below)
  const bool mask_in_smem = !DOTS && a.store_mask && a.h <= 17;
  if (mask_in_smem)
    for (int e = threadIdx.x; e < (1 << (a.h - 4)) / 32; e += blockDim.x) mask_sh[e] = a.store_mask[e];
  const uint32_t *smask = DOTS ? nullptr : mask_in_smem ? mask_sh : a.store_mask;
  if constexpr (DOTS)
    for (int e = threadIdx.x; e < 256; e += blockDim.x) dot_S[e] = a.dot_T[e];
  // A CTA serves kHDigits consecutive digits (one when the radix is odd): each parent unit
  // is split once and multiplied by every digit's W.  Units run over the parents with a
  // child in [node_lo, node_lo + num_nodes); children outside are computed, not stored.
  const int dpc = radix % kHDigits == 0 ? kHDigits : 1;
  const int m0 = blockIdx.y * dpc;
  const int64_t p_first = a.node_lo / radix;
  const int64_t p_last = (a.node_lo + a.num_nodes - 1) / radix;
  const int tb = a.h - kMmaMinH;                        // 2^tb row units per node
  const int64_t units = (p_last - p_first + 1) << tb;
  const int64_t my_units = units > blockIdx.x ? (units - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  const int64_t nquarters = my_units * 4;
  const uint8_t *wimg = static_cast<const uint8_t *>(a.w);

  if (threadIdx.x == 0) {
    epi_abort[0] = epi_abort[1] = 0;
    for (int s = 0; s < kHOps; ++s) {
      mbar_init(&ops_full[s], kHSplitThreads);
      mbar_init(&ops_empty[s], 1);
    }
    for (int s = 0; s < 4; ++s) mbar_init(&sc_full[s], kHSplitThreads);
    for (int b = 0; b < 2; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], 256);
    }
    mbar_init(&drain, 1);
    abort_sh = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 8) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_sh)),
                 "r"(kHTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_sh;
  if (warp >= 4 && warp < 8) {
    // W_m into TMEM for each digit i served: lane n holds row n, two FP16 per column;
    // columns 128 i + [0,64) the hi part, 128 i + [64,128) the lo part (the image holds
    // 128 rows x 64 words per part)
    const int q4 = warp & 3;
#pragma unroll 1
    for (int c = 0; c < 4 * dpc; ++c) {
      const uint32_t *wrow = reinterpret_cast<const uint32_t *>(wimg + (size_t)(m0 + (c >> 2)) * kMmaWDigitBytes) +
                             (size_t)(q4 * 32 + lane) * 64;
      const uint32_t *src = wrow + (size_t)((c >> 1) & 1) * 128 * 64 + (c & 1) * 32;
      uint32_t v[32];
#pragma unroll
      for (int j = 0; j < 32; j += 4) {
        const uint4 x = *reinterpret_cast<const uint4 *>(src + j);
        v[j] = x.x;
        v[j + 1] = x.y;
        v[j + 2] = x.z;
        v[j + 3] = x.w;
      }
      const uint32_t taddr = tmem + ((uint32_t)(q4 * 32) << 16) + (uint32_t)(c * 32);
      asm volatile(
          "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,"
          "%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};" ::"r"(taddr),
          "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]), "r"(v[8]),
          "r"(v[9]), "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15]), "r"(v[16]),
          "r"(v[17]), "r"(v[18]), "r"(v[19]), "r"(v[20]), "r"(v[21]), "r"(v[22]), "r"(v[23]), "r"(v[24]),
          "r"(v[25]), "r"(v[26]), "r"(v[27]), "r"(v[28]), "r"(v[29]), "r"(v[30]), "r"(v[31])
          : "memory");
    }
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

  if (warp < 4 || warp >= 13) {
    // ---- split: each 64-amplitude row (128 floats) is scaled by 2^e (largest component
    // in [2^14, 2^15); exact) and split into hi = fp16(x) and lo = fp16(x - hi).  Thread
    // t converts 8 consecutive floats (K 8 pc .. 8 pc + 7) of rows t / 16 + R i (R rows
    // per pass); the 16 threads of a row find its maximum with shuffles.
    // The parent quarters (quarter c = rows 32 (c % 4) .. + 31 of unit blockIdx.x +
    // (c / 4) gridDim.x) stream through a kHRaw-stage ring with cp.async: each warp
    // copies exactly the two rows per pass that it converts (1 KB, coalesced), so a
    // warp-level sync is all a stage needs. ----
    const int t = warp < 4 ? (int)threadIdx.x : (int)threadIdx.x - 13 * 32 + 128;
    constexpr int R = kHSplitThreads / 16;
    constexpr int kItems = 32 / R;
    const int pc = t & 15;
    const int sw = t >> 5;                               // split warp: rows i R + 2 sw, + 1
    const int64_t pbase = p_first - a.parent_lo;        // unit u's parent, in the parent buffer
    auto src_of = [&](int64_t c) {
      const int64_t u = blockIdx.x + (c >> 2) * gridDim.x;
      const int64_t row = ((pbase + (u >> tb)) << (a.h - kMmaBits)) + ((u & ((1 << tb) - 1)) << 7) + (c & 3) * 32;
      return reinterpret_cast<const uint8_t *>(a.parent) + row * 512;
    };
    auto issue = [&](int64_t c) {
      if (c < nquarters) {
        const uint8_t *src = src_of(c);
        const uint32_t dst = smem_u32(sR + (int)(c % RAW) * kHQuarter);
#pragma unroll
        for (int i = 0; i < kItems; ++i)
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int off = (i * R + 2 * sw + h) * 512 + lane * 16;
            lvl_cp_async16(dst + off, src + off);
          }
      }
      lvl_cp_commit();                                   // (empty groups keep the count uniform)
    };
#pragma unroll
    for (int c = 0; c < RAW - 1; ++c) issue(c);
    int64_t it = 0;
    // A split warp stops as a whole: its lanes meet at __syncwarp and full-mask shuffles
    // below, so the abort flag and the result of the bounded wait are combined across
    // the warp before anyone leaves the loop.
    for (int64_t tu = 0; tu < my_units; ++tu) {
      if (__any_sync(0xffffffffu, abort_sh != 0)) break;
      const int o = (int)(tu & 1);
      const bool ok = mbar_wait(&ops_empty[o], ((uint32_t)(tu >> 1) & 1u) ^ 1u);
      if (!__all_sync(0xffffffffu, ok)) {
        if (lane == 0) atomicExch(a.err, 4);
        abort_sh = 1;
        break;
      }
      const uint32_t op = smem_u32(sOp + o * kHOpBytes);
      auto *inv = row_inv[tu & 3];
      for (int q = 0; q < 4; ++q, ++it) {
        issue(it + RAW - 1);                           // into the stage read last iteration
        lvl_cp_wait<RAW - 1>();                        // this thread's copies of quarter it
        __syncwarp();                                    // ... and the rest of its warp's
        const uint32_t raw = smem_u32(sR + (int)(it % RAW) * kHQuarter);
        float4 xr[kItems][2];
#pragma unroll
        for (int i = 0; i < kItems; ++i) {
          const int rr = i * R + (t >> 4);
          xr[i][0] = lds128(raw + rr * 512 + pc * 32);
          xr[i][1] = lds128(raw + rr * 512 + pc * 32 + 16);
        }
        __syncwarp();                                    // read before the stage is refilled
#pragma unroll
        for (int i = 0; i < kItems; ++i) {
          const int rr = i * R + (t >> 4);                 // row within the quarter
          const int n = q * 32 + rr;                       // row within the unit (MMA N)
          const float4 x0 = xr[i][0], x1 = xr[i][1];
          float mx = fmaxf(fmaxf(fmaxf(fabsf(x0.x), fabsf(x0.y)), fmaxf(fabsf(x0.z), fabsf(x0.w))),
                           fmaxf(fmaxf(fabsf(x1.x), fabsf(x1.y)), fmaxf(fabsf(x1.z), fabsf(x1.w))));
#pragma unroll
          for (int sh = 8; sh > 0; sh >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, sh));
          // scale 2^(141 - eb) for biased exponent eb of the maximum (largest scaled
          // component in [2^14, 2^15)), capped at 2^126 so that its inverse stays a normal
          // float (zero rows keep zero).  hi = x s rounded to a multiple of 16 (adding and
          // removing 1.5 2^27), exact in FP16; lo = x s - hi, exact, |lo| <= 8, rounded to
          // FP16: the split is within 2^-23 of the row's largest component.
          const uint32_t eb = __float_as_uint(mx) >> 23;
          const uint32_t sb = min(268u - min(eb, 254u), 253u);
          const float sc = __uint_as_float(sb << 23);
          constexpr float kRound = 201326592.0f;           // 1.5 x 2^27: ulp 16
          const float xv[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
          uint32_t hb[4], lb[4];
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const float h0 = __fsub_rn(__fmaf_rn(xv[2 * j], sc, kRound), kRound);
            const float h1 = __fsub_rn(__fmaf_rn(xv[2 * j + 1], sc, kRound), kRound);
            hb[j] = h2_bits(__floats2half2_rn(h0, h1));
            lb[j] = h2_bits(__floats2half2_rn(__fmaf_rn(xv[2 * j], sc, -h0), __fmaf_rn(xv[2 * j + 1], sc, -h1)));
          }
          // K-major, 128-byte swizzle: atom pc / 8, 16-byte piece (pc % 8) ^ (n % 8) of row n
          const uint32_t off = (uint32_t)(pc >> 3) * kHAtom + (uint32_t)n * 128 + ((uint32_t)((pc & 7) ^ (n & 7)) << 4);
          sts128(op + off, hb[0], hb[1], hb[2], hb[3]);
          sts128(op + 2 * kHAtom + off, lb[0], lb[1], lb[2], lb[3]);
          if (pc == 0) {
            if constexpr (DOTS)
              inv[n] = (uint8_t)sb;
            else
              inv[n] = __uint_as_float((254u - sb) << 23);
          }
        }
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mbar_arrive(&ops_full[o]);
      mbar_arrive(&sc_full[tu & 3]);
    }
    lvl_cp_wait<0>();                                    // no copy is in flight at exit
  } else if (warp == 8) {
    // ---- MMA issuer ----
    if (lane == 0) {
      // FP32 accumulate, FP16 A and B, both K-major, N = 128, M = 128
      const uint32_t idesc = (1u << 4) | ((uint32_t)(128 >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
      for (int64_t tu = 0; tu < my_units && !abort_sh; ++tu) {
        const int o = (int)(tu & 1);
        if (!mbar_wait(&ops_full[o], (uint32_t)(tu >> 1) & 1u)) {
          atomicExch(a.err, 6);
          abort_sh = 1;
          break;
        }
        const uint8_t *op = sOp + o * kHOpBytes;
        bool ok = true;
        for (int i = 0; i < dpc; ++i) {
          // output tu dpc + i goes to accumulator b once the epilogue has drained it
          const int64_t oi = tu * dpc + i;
          const int b = (int)(oi & 1);
          if (!mbar_wait(&tempty[b], ((uint32_t)(oi >> 1) & 1u) ^ 1u)) {
            atomicExch(a.err, 5);
            abort_sh = 1;
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t d = tmem + 256u + (uint32_t)(b * 128);
          // D[n][row] = sum_k W[n][k] parent[row][k]: W (TMEM) is the MMA's A operand
          // (M = 128 output components), the parent rows its B operand (N = 128 rows)
#pragma unroll
          for (int kc = 0; kc < 2; ++kc) {
            const uint64_t phi = make_desc(op + kc * kHAtom), plo = make_desc(op + (2 + kc) * kHAtom);
#pragma unroll
            for (int term = 0; term < 3; ++term) {
              const uint64_t dp = term == 1 ? plo : phi;
              const uint32_t wcol = (uint32_t)(i * 128) + (term == 2 ? 64u : 0u) + (uint32_t)(kc * 32);
#pragma unroll
              for (int kk = 0; kk < 4; ++kk)   // 16 FP16 of K per MMA (32 bytes, 8 columns)
                mma_f16_ts(d, tmem + wcol + 8u * kk, dp + 2 * kk, idesc, (kc | term | kk) ? 1u : 0u);
            }
          }
          mma_commit(&tfull[b]);              // the accumulator is complete
        }
        if (!ok) break;
        mma_commit(&ops_empty[o]);            // the operand buffer is free once these finish
      }
      // every MMA issued above has finished before TMEM is released
      mma_commit(&drain);
      if (!mbar_wait(&drain, 0)) atomicExch(a.err, 7);
    }
    __syncwarp();
  } else {
    // ---- epilogue: two groups of four warps (4..7 and 9..12) take alternate 32-row
    // quarters of each accumulator.  TMEM lane quarter (warp & 3) holds output
    // components 32 (warp & 3) .. + 31; TMEM column j of the accumulator is row j of the
    // unit; a quarter is unscaled and stored straight from registers. ----
    const int grp = warp >= 9 ? 1 : 0;
    const uint32_t bar_id = 1 + grp;                     // named barrier of the group
    const int q4 = warp & 3;
    const int comp = q4 * 32 + lane;
    const float *inv_ws = reinterpret_cast<const float *>(wimg + (size_t)radix * kMmaWDigitBytes) + m0;
    // dot form: this warp's row tile and entry buffer
    const int ew = grp * 4 + q4;
    float *tile = dot_tile + (DOTS ? ew * kDotRows * 32 : 0);
    uint32_t *meta = dot_meta + (DOTS ? ew * kDotMeta : 0);
    // dot form: lane 3 qi + b (< 6) loads boundary b (row 32 qr + 16 b, qr = grp + 2 qi)
    // of the bitstring ranges of unit uu's rows in segment q4, one unit ahead
    auto load_bnd = [&](int64_t uu) -> uint32_t {
      if (!DOTS || uu >= units || lane >= 6) return 0u;
      const uint32_t kq = ((uint32_t)q4 << (a.h - 6)) + ((uint32_t)(uu & ((1 << tb) - 1)) << 7);
      return a.dot_off[kq + 32u * (uint32_t)(grp + 2 * (lane / 3)) + 16u * (uint32_t)(lane % 3)];
    };
    uint32_t bnd_next = load_bnd(blockIdx.x);
    int64_t tu = 0;
    // The four warps of a group meet at named barriers, so they decide to stop together:
    // only they write their epi_abort word, before a barrier, and all read it after.
    for (int64_t u = blockIdx.x; u < units; u += gridDim.x, ++tu) {
      const auto *inv = row_inv[tu & 3];
      const int64_t pu = p_first + (u >> tb);           // the unit's parent
      bool stop = false;
      // dot form: the bitstring entries of this unit's rows in segment q4 for the group's
      // two quarters (qr = grp, grp + 2), shared by every digit of the unit.  Sorted by
      // (segment in row, row), those of 16 consecutive rows are one range of dot_list;
      // lane 3 qi + b holds boundary b (row 32 qr + 16 b) of quarter qi, and the entries
      // of quarter 0 then 1 go to meta (up to kDotMeta; the rest are read from dot_list).
      uint32_t bnd = 0, n0 = 0;
      if constexpr (DOTS) {
        bnd = bnd_next;
        bnd_next = load_bnd(u + gridDim.x);
        const uint32_t s0 = __shfl_sync(0xffffffffu, bnd, 0), e0 = __shfl_sync(0xffffffffu, bnd, 2);
        const uint32_t s1 = __shfl_sync(0xffffffffu, bnd, 3), e1 = __shfl_sync(0xffffffffu, bnd, 5);
        n0 = e0 - s0;
        const uint32_t n = min(n0 + (e1 - s1), (uint32_t)kDotMeta);
        for (uint32_t m = (uint32_t)lane; m < n; m += 32) meta[m] = __ldg(a.dot_list + (m < n0 ? s0 + m : s1 + (m - n0)));
        __syncwarp();
      }
      for (int i = 0; i < dpc; ++i) {
        const int64_t oi = tu * dpc + i;
        const int b = (int)(oi & 1);
        const bool ok = mbar_wait(&tfull[b], (uint32_t)(oi >> 1) & 1u) &&
                        mbar_wait(&sc_full[tu & 3], (uint32_t)(tu >> 2) & 1u);
        if (!ok) epi_abort[grp] = 1;
        asm volatile("bar.sync %0, 128;" ::"r"(bar_id) : "memory");
        if (epi_abort[grp]) {
          if (!ok) atomicExch(a.err, 8);
          abort_sh = 1;
          stop = true;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const int64_t g = pu * radix + m0 + i;
        const bool store = g >= a.node_lo && g < a.node_lo + a.num_nodes;
        const uint64_t dst_off = store ? (((uint64_t)(g - a.node_lo) << a.h) + ((uint64_t)(u & ((1 << tb) - 1)) << 13)) * 2 : 0;
        const float inv_w = inv_ws[i];
        if constexpr (DOTS) {
          if (store) {
            // Dot form.  Per half quarter (16 rows), this warp's segment q4 of each row is
            // staged in its tile (row jj, 16-byte piece p at p ^ (jj % 8)), and each lane
            // takes one bitstring whose chunk is one of those segments (the range
            // [hs, he) of dot_list), forms its four dots and writes them at its position.
            const uint64_t row0 = (uint64_t)(u & ((1 << tb) - 1)) << 7;
            float4 *dout = a.dots + (uint64_t)(g - a.node_lo) * (uint64_t)a.dot_count * 2u;
#pragma unroll 1
            for (int qr = grp; qr < 4; qr += 2) {
              const int qi = qr >> 1;
              const uint32_t qs = __shfl_sync(0xffffffffu, bnd, 3 * qi);
#pragma unroll
              for (int hh = 0; hh < 2; ++hh) {
                const uint32_t hs = __shfl_sync(0xffffffffu, bnd, 3 * qi + hh);
                const uint32_t he = __shfl_sync(0xffffffffu, bnd, 3 * qi + hh + 1);
                const uint32_t rbase = (uint32_t)row0 + (uint32_t)(qr * 32 + hh * kDotRows);
                const uint32_t mbase = (qi ? n0 : 0u) + (hs - qs);
                uint32_t v[kDotRows];
                const uint32_t taddr =
                    tmem + ((uint32_t)(q4 * 32) << 16) + 256u + (uint32_t)(b * 128 + qr * 32 + hh * kDotRows);
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
                    "[%16];"
                    : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                      "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
                      "=r"(v[15])
                    : "r"(taddr));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                // the 16 values first, then the 16 stores (interleaving the two ran three
                // times slower)
                float xs[kDotRows];
#pragma unroll
                for (int jj = 0; jj < kDotRows; ++jj) {
                  const float sc = __uint_as_float((254u - (uint32_t)inv[qr * 32 + hh * kDotRows + jj]) << 23);
                  xs[jj] = __uint_as_float(v[jj]) * sc * inv_w;
                }
#pragma unroll
                for (int jj = 0; jj < kDotRows; ++jj) tile[jj * 32 + ((((lane >> 2) ^ (jj & 7)) << 2) | (lane & 3))] = xs[jj];
                __syncwarp();
                for (uint32_t t0 = hs; t0 < he; t0 += 32) {
                  const uint32_t pos = t0 + (uint32_t)lane;
                  if (pos < he) {
                    const uint32_t m = mbase + (pos - hs);
                    const uint32_t ent = m < (uint32_t)kDotMeta ? meta[m] : __ldg(a.dot_list + pos);
                    const uint32_t j = (ent >> 4) - rbase, rr = ent & 15u;
                    // the chunk x and the row w = S[rr] into registers first: 16-byte
                    // piece p (amplitudes 2p, 2p+1) of row j sits at piece p ^ (j % 8);
                    // w[e] = S[rr][e] is dot_S[16 e + rr] (16 lanes read one 128-byte
                    // row of the table: no bank conflicts)
                    const float4 *xq = reinterpret_cast<const float4 *>(tile) + j * 8;
                    float2 x[16], w[16];
#pragma unroll
                    for (int pc = 0; pc < 8; ++pc) {
                      const float4 q = xq[pc ^ (j & 7u)];
                      x[2 * pc] = make_float2(q.x, q.y);
                      x[2 * pc + 1] = make_float2(q.z, q.w);
                    }
#pragma unroll
                    for (int e = 0; e < 16; ++e) w[e] = dot_S[e * 16 + rr];
                    // the four dots as in the factored leaf kernel: P = sum Re w . x,
                    // Q = sum Im w . x over (re, im) pairs, w x = (P.x - Q.y, P.y + Q.x);
                    // scalar FMAs give the bits of its packed pair FMAs (the broadcast
                    // pairs those need cost 16-byte table reads, which conflict: 2.5 ms
                    // per level-7 launch against 2.0)
                    float2 P[4], Q[4];
#pragma unroll
                    for (int al = 0; al < 4; ++al) P[al] = Q[al] = make_float2(0.f, 0.f);
#pragma unroll
                    for (int k = 0; k < 8; ++k) {
                      // the k-th term's amplitudes e_0(k), e_1(k): factor bit 0 / 1 put at
                      // chunk bit PF
                      constexpr int lo = (1 << (DOTS ? PF : 0)) - 1;
                      const int e0 = ((k & ~lo) << 1) | (k & lo), e1 = e0 | (lo + 1);
                      const float2 x0 = x[e0], x1 = x[e1], w0 = w[e0], w1 = w[e1];
                      P[0].x = fmaf(w0.x, x0.x, P[0].x);
                      P[0].y = fmaf(w0.x, x0.y, P[0].y);
                      Q[0].x = fmaf(w0.y, x0.x, Q[0].x);
                      Q[0].y = fmaf(w0.y, x0.y, Q[0].y);
                      P[1].x = fmaf(w0.x, x1.x, P[1].x);
                      P[1].y = fmaf(w0.x, x1.y, P[1].y);
                      Q[1].x = fmaf(w0.y, x1.x, Q[1].x);
                      Q[1].y = fmaf(w0.y, x1.y, Q[1].y);
                      P[2].x = fmaf(w1.x, x0.x, P[2].x);
                      P[2].y = fmaf(w1.x, x0.y, P[2].y);
                      Q[2].x = fmaf(w1.y, x0.x, Q[2].x);
                      Q[2].y = fmaf(w1.y, x0.y, Q[2].y);
                      P[3].x = fmaf(w1.x, x1.x, P[3].x);
                      P[3].y = fmaf(w1.x, x1.y, P[3].y);
                      Q[3].x = fmaf(w1.y, x1.x, Q[3].x);
                      Q[3].y = fmaf(w1.y, x1.y, Q[3].y);
                    }
                    float4 *dp = dout + 2 * (uint64_t)pos;
                    dp[0] = make_float4(P[0].x - Q[0].y, P[0].y + Q[0].x, P[1].x - Q[1].y, P[1].y + Q[1].x);
                    dp[1] = make_float4(P[2].x - Q[2].y, P[2].y + Q[2].x, P[3].x - Q[3].y, P[3].y + Q[3].x);
                  }
                }
                __syncwarp();                                // the tile is read before the next half
              }
            }
          }
        } else {
  #pragma unroll 1
          for (int qr = grp; qr < 4; qr += 2) {
            uint32_t v[32];
            const uint32_t taddr = tmem + ((uint32_t)(q4 * 32) << 16) + 256u + (uint32_t)(b * 128 + qr * 32);
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                  "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
                  "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
                  "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
                : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (store) {
              // row j of the quarter goes out from registers, a warp writing its 32
              // components (128 contiguous bytes: segment q4 of the row) per row; with a
              // store mask, segments no bitstring reads are skipped (the bit is the same
              // for the whole warp)
              float *out = a.child + dst_off + (size_t)qr * 32 * 128 + comp;
              uint32_t keep = 0xffffffffu;
              if (smask) {
                const uint64_t r0 = ((uint64_t)(u & ((1 << tb) - 1)) << 7) + (uint64_t)qr * 32;   // first row
                const uint32_t *mw = smask + (r0 >> 3);                  // 8 rows (4 bits each) per word
                keep = 0;
  #pragma unroll
                for (int w4 = 0; w4 < 4; ++w4) {
                  const uint32_t word = mw[w4];
  #pragma unroll
                  for (int jj = 0; jj < 8; ++jj) keep |= ((word >> (4 * jj + q4)) & 1u) << (8 * w4 + jj);
                }
              }
  #pragma unroll
              for (int j = 0; j < 32; ++j)
                if ((keep >> j) & 1u) out[(size_t)j * 128] = __uint_as_float(v[j]) * inv[qr * 32 + j] * inv_w;
            }
          }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        mbar_arrive(&tempty[b]);
      }
      if (stop) break;
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 8) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kHTmemCols) : "memory");
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, []() {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &p, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

bool make_map(CUtensorMap *m, void *base, bool bf16, uint64_t kpad, uint64_t rows, uint32_t box_rows) {
  auto enc = get_encode();
  if (!enc) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)kpad, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)(kpad * (bf16 ? 2 : 4))};
  const cuuint32_t box[2] = {(cuuint32_t)(bf16 ? 64 : 32), (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = enc(m, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, base, dims,
                         strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

}  // namespace

size_t path_gemm_operand_bytes(int mode, int64_t M, int64_t N, int64_t paths) {
  const int64_t Mp = (M + kBM - 1) / kBM * kBM, Np = (N + kBN - 1) / kBN * kBN;
  const int nterms = mode == 3 ? 1 : 3;
  const int kalign = mode == 1 ? 64 : 32;
  const int64_t kpad = (nterms * 2 * paths + kalign - 1) / kalign * kalign;
  const int esz = mode == 1 ? 2 : 4;
  return (size_t)(2 * Mp + Np) * (size_t)kpad * esz + 256;
}

cudaError_t launch_path_pack(const PathGemmArgs &g, cudaStream_t st) {
  const int64_t Mp = (g.M + kBM - 1) / kBM * kBM, Np = (g.N + kBN - 1) / kBN * kBN;
  const int nterms = g.mode == 3 ? 1 : 3;
  const bool bf16 = g.mode == 1;
  const int kalign = bf16 ? 64 : 32;
  const int64_t kcols = (int64_t)nterms * 2 * g.paths;
  const int64_t kpad = (kcols + kalign - 1) / kalign * kalign;
  const int esz = bf16 ? 2 : 4;
  uint8_t *opA = reinterpret_cast<uint8_t *>(g.scratch);
  uint8_t *opB = opA + (size_t)2 * Mp * kpad * esz;
  // zero only the padding (rows past M or N, columns past the K'' used), which must
  // contribute nothing; the pack kernels write every other entry
  cudaError_t e = cudaSuccess;
  if (Mp > g.M) e = cudaMemsetAsync(opA + (size_t)2 * g.M * kpad * esz, 0, (size_t)2 * (Mp - g.M) * kpad * esz, st);
  if (e == cudaSuccess && Np > g.N) e = cudaMemsetAsync(opB + (size_t)g.N * kpad * esz, 0, (size_t)(Np - g.N) * kpad * esz, st);
  if (e == cudaSuccess && kpad > kcols)
    e = cudaMemset2DAsync(opA + (size_t)kcols * esz, (size_t)kpad * esz, 0, (size_t)(kpad - kcols) * esz,
                          (size_t)(2 * Mp + Np), st);
  if (e != cudaSuccess) return e;
  for (int side = 0; side < 2; ++side) {
    PackArgs pa{};
    pa.src = reinterpret_cast<const float2 *>(side == 0 ? g.A : g.B);
    pa.h = side == 0 ? g.ha : g.hb;
    pa.paths = g.paths;
    pa.rows = side == 0 ? g.M : g.N;
    pa.rows_pad = side == 0 ? Mp : Np;
    pa.side = side;
    pa.kpad = kpad;
    pa.dst = side == 0 ? (void *)opA : (void *)opB;
    // enumerate the rows' local bits in ascending storage-bit order
    const PermArgs &pm = side == 0 ? g.perm_a : g.perm_b;
    int w = 0;
    while (w < pa.h && (1ll << w) < pa.rows) ++w;
    pa.w = w;
    int order[64];
    for (int q = 0; q < w; ++q) order[q] = q;
    std::sort(order, order + w, [&](int x, int y) { return pm.store[x] < pm.store[y]; });
    for (int k = 0; k < w; ++k) {
      pa.upos[k] = (int8_t)pm.store[order[k]];
      pa.ibit[k] = (int8_t)order[k];
    }
    const int64_t ptiles = (g.paths + kPackPaths - 1) / kPackPaths;
    const unsigned gy = (unsigned)(ptiles < 65535 ? ptiles : 65535);
    const unsigned gz = (unsigned)((ptiles + gy - 1) / gy);
    dim3 grid((unsigned)(((1ll << w) + kPackRows - 1) / kPackRows), gy, gz);
    if (g.mode == 1) pack_kernel<1><<<grid, 256, 0, st>>>(pa);
    else if (g.mode == 2) pack_kernel<2><<<grid, 256, 0, st>>>(pa);
    else pack_kernel<3><<<grid, 256, 0, st>>>(pa);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_path_gemm(const PathGemmArgs &g, cudaStream_t st) {
  const int64_t Mp = (g.M + kBM - 1) / kBM * kBM, Np = (g.N + kBN - 1) / kBN * kBN;
  const int nterms = g.mode == 3 ? 1 : 3;
  const bool bf16 = g.mode == 1;
  const int kalign = bf16 ? 64 : 32;
  const int64_t kpad = (nterms * 2 * g.paths + kalign - 1) / kalign * kalign;
  const int esz = bf16 ? 2 : 4;
  uint8_t *opA = reinterpret_cast<uint8_t *>(g.scratch);
  uint8_t *opB = opA + (size_t)2 * Mp * kpad * esz;
  cudaError_t e = cudaSuccess;
  CUtensorMap tmA, tmB;
  if (!make_map(&tmA, opA, bf16, (uint64_t)kpad, (uint64_t)(2 * Mp), (uint32_t)kGN) ||
      !make_map(&tmB, opB, bf16, (uint64_t)kpad, (uint64_t)Np, (uint32_t)kGM))
    return cudaErrorInvalidValue;
  EpiArgs ep{};
  ep.out = g.out;
  ep.comp = g.comp;
  ep.M = g.M;
  ep.N = g.N;
  ep.Mp = Mp;
  ep.hb = g.hb;
  ep.window = g.window;
  ep.k_tiles = (int32_t)(kpad / kalign);
  ep.kind = bf16 ? 0 : 1;
  ep.err = g.err;
  const size_t smem = (size_t)kStages * (kTileA + kTileB) + 1024;
  e = cudaFuncSetAttribute(gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  ep.num_m = (int32_t)(2 * Mp / kGN);
  ep.num_n = (int32_t)(Np / kGM);
  (void)esz;
  const int64_t tiles = (int64_t)ep.num_m * ep.num_n;
  int sms = device_sm_count();
  if (sms <= 0) sms = 148;
  const unsigned grid = (unsigned)std::min<int64_t>(tiles, sms);   // persistent: one CTA per SM
  gemm_kernel<<<grid, kGemmThreads, smem, st>>>(tmA, tmB, ep);
  return cudaGetLastError();
}

void level_mma_image(const double *w, float *hi, float *lo) {
  auto rna = [](float x) {               // round to TF32 (nearest, ties away), as cvt.rna.tf32
    uint32_t u;
    std::memcpy(&u, &x, 4);
    if ((u & 0x7f800000u) != 0x7f800000u) u = (u + 0x1000u) & 0xffffe000u;
    float r;
    std::memcpy(&r, &u, 4);
    return r;
  };
  // row-major [n][k]: the kernel loads row n into TMEM lane n
  for (int i = 0; i < 128 * 128; ++i) {
    const float x = (float)w[i];
    hi[i] = rna(x);
    lo[i] = rna(x - hi[i]);
  }
}

// binary32 -> binary16 bits, round to nearest with ties to even, from the IEEE 754
// encodings (the host library conversion is a slow call per element)
static uint16_t f16_bits_rn(float f) {
  uint32_t x;
  std::memcpy(&x, &f, 4);
  const uint32_t sign = (x >> 16) & 0x8000u, ax = x & 0x7fffffffu;
  if (ax >= 0x7f800000u) return (uint16_t)(sign | (ax > 0x7f800000u ? 0x7e00u : 0x7c00u));   // NaN / Inf
  if (ax >= 0x477ff000u) return (uint16_t)(sign | 0x7c00u);          // >= 65520 rounds to Inf
  const uint32_t e = ax >> 23;                                        // biased binary32 exponent
  if (e >= 113) {                                                     // normal binary16 (>= 2^-14)
    uint32_t r = ((e - 112) << 10) | ((ax & 0x7fffffu) >> 13);
    const uint32_t rem = ax & 0x1fffu;
    r += (rem + (r & 1u)) > 0x1000u;                                 // ties to even; a carry moves to the exponent
    return (uint16_t)(sign | r);
  }
  if (e < 102) return (uint16_t)sign;                                 // below 2^-25: zero
  // subnormal binary16 in units of 2^-24: m 2^(e - 150) = (m >> (126 - e)) units
  const uint32_t m = (ax & 0x7fffffu) | 0x800000u, sh = 126 - e;      // sh in 14..24
  uint32_t r = m >> sh;
  const uint32_t rem = m & ((1u << sh) - 1u), half = 1u << (sh - 1);
  r += (rem + (r & 1u)) > half;                                       // ties to even; may reach 0x400 (2^-14)
  return (uint16_t)(sign | r);
}

void level_mma_image_f16(const double *w, void *digit_image, float *inv_scale) {
  // scale 2^e with the largest |entry| in [2^14, 2^15); hi = entry rounded to a multiple
  // of 16 (exact in FP16), lo = fp16(entry - hi), as the kernel splits the parent rows
  double mx = 0.0;
  for (int i = 0; i < 128 * 128; ++i) mx = std::max(mx, std::fabs(w[i]));
  int ex = 0;
  if (mx > 0.0) std::frexp(mx, &ex);                   // mx = f 2^ex, f in [0.5, 1)
  const int e = mx > 0.0 ? 15 - ex : 0;
  const double sc = std::ldexp(1.0, e);
  constexpr double kRound = 6755399441055744.0;        // 1.5 x 2^52: rounds to an integer, ties to even
  // row-major [n][k]: the kernel loads row n into TMEM lane n, two FP16 per column
  uint16_t *hi = static_cast<uint16_t *>(digit_image), *lo = hi + 128 * 128;
  for (int i = 0; i < 128 * 128; ++i) {
    const double xs = w[i] * sc;                       // exact: a power of two
    const double t = xs * 0.0625;                      // exact; |t| < 2^11
    const double h = 16.0 * std::copysign((t + kRound) - kRound, t);   // 16 nearbyint(t)
    hi[i] = f16_bits_rn((float)h);                     // exact
    lo[i] = f16_bits_rn((float)(xs - h));
  }
  *inv_scale = std::ldexp(1.0f, -e);
}

cudaError_t launch_level_mma(const LevelMmaArgs &a, cudaStream_t st) {
  if (a.num_nodes <= 0) return cudaSuccess;
  int sms = device_sm_count();
  if (sms <= 0) sms = 148;
  const int r = a.radix > 0 ? a.radix : 1;
  if (a.num_post == 0) {
    // FP16 split kernel (W image: FP16 parts per digit, then the inverse scales)
    if (a.h < kMmaMinH || (reinterpret_cast<uintptr_t>(a.parent) & 15) || (reinterpret_cast<uintptr_t>(a.child) & 15))
      return cudaErrorInvalidValue;
    if (a.dots && (!a.dot_off || !a.dot_list || !a.dot_T || a.dot_pf < 0 || a.dot_pf > 3 || a.dot_count <= 0 ||
                   (reinterpret_cast<uintptr_t>(a.dots) & 15) || (reinterpret_cast<uintptr_t>(a.dot_T) & 15)))
      return cudaErrorInvalidValue;
    const size_t smem = a.dots ? kHSmemDots : kHSmem;
    auto kernel = !a.dots ? level_mma_f16_kernel<-1>
                  : a.dot_pf == 0 ? level_mma_f16_kernel<0>
                  : a.dot_pf == 1 ? level_mma_f16_kernel<1>
                  : a.dot_pf == 2 ? level_mma_f16_kernel<2>
                                  : level_mma_f16_kernel<3>;
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int dpc = r % kHDigits == 0 ? kHDigits : 1;
    const int gy = r / dpc;
    const int64_t units = ((a.node_lo + a.num_nodes - 1) / r - a.node_lo / r + 1) << (a.h - kMmaMinH);
    const int64_t gx = std::min<int64_t>(std::max(1, (sms + gy - 1) / gy), std::max<int64_t>(1, units));
    kernel<<<dim3((unsigned)gx, (unsigned)gy), kHThreads, smem, st>>>(a);
    return cudaGetLastError();
  }
  const size_t smem = kLvlSmem;
  cudaError_t e = cudaFuncSetAttribute(level_mma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int64_t per_digit_units = ((a.num_nodes + r - 1) / r) << (a.h - kMmaMinH);
  const int64_t gx = std::min<int64_t>(std::max(1, (sms + r - 1) / r), std::max<int64_t>(1, per_digit_units));
  // the parents as a [rows][128] FP32 matrix (one row = 64 amplitudes); 32 x 128 boxes
  const int64_t parents = (a.node_lo + a.num_nodes - 1) / r - a.parent_lo + 1;
  const int64_t rows = parents << (a.h - kMmaBits);
  auto enc = get_encode();
  if (!enc || rows <= 0 || rows > INT32_MAX) return cudaErrorInvalidValue;
  CUtensorMap tmP;
  const cuuint64_t dims[2] = {128, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {512};
  const cuuint32_t box[2] = {32, 128};
  const cuuint32_t estr[2] = {1, 1};
  if (enc(&tmP, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(a.parent), dims, strides, box, estr,
          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return cudaErrorInvalidValue;
  level_mma_kernel<<<dim3((unsigned)gx, (unsigned)r), kLvlThreads, smem, st>>>(tmP, a);
  return cudaGetLastError();
}

}  // namespace hsf
