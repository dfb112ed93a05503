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
  const uint64_t x = a.bits[s];
  const uint64_t xb = x & ((1ull << a.hb) - 1ull);
  const uint64_t xa = (x >> a.hb) & ((1ull << a.ha) - 1ull);
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

__global__ void reduce_partials_kernel(const double *partial, int32_t num_groups, int64_t S,
                                       double *out, double *comp) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= S) return;
  double sr = out[2 * s], si = out[2 * s + 1];
  double cr = comp[2 * s], ci = comp[2 * s + 1];
  for (int g = 0; g < num_groups; ++g) {
    neumaier_add(sr, cr, partial[2 * ((int64_t)g * S + s)]);
    neumaier_add(si, ci, partial[2 * ((int64_t)g * S + s) + 1]);
  }
  out[2 * s] = sr;
  out[2 * s + 1] = si;
  comp[2 * s] = cr;
  comp[2 * s + 1] = ci;
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
        if (i0 + cc < a.M) va = A[((uint64_t)p << a.ha) + (uint64_t)(i0 + cc)];
        if (j0 + cc < a.N) vb = B[((uint64_t)p << a.hb) + (uint64_t)(j0 + cc)];
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

__global__ void finalize_kernel(double *out, const double *comp, int64_t count) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) out[i] += comp[i];
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
  reduce_partials_kernel<<<(unsigned)((S + 255) / 256), 256, 0, st>>>(partial, num_groups, S, out, comp);
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

cudaError_t launch_finalize(double *out, const double *comp, int64_t count, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  finalize_kernel<<<(unsigned)((count + 255) / 256), 256, 0, st>>>(out, comp, count);
  return cudaGetLastError();
}

cudaError_t launch_zero(double *p, int64_t count, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  zero_kernel<<<(unsigned)((count + 255) / 256), 256, 0, st>>>(p, count);
  return cudaGetLastError();
}

}  // namespace hsf
