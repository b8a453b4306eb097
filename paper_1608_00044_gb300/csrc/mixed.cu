// FP64 residual, norms and correction update for iterative refinement with a
// low-precision factor: x_{k+1} = x_k + P^T L^{-T} L^{-1} P (b - A x_k), the
// residual b - A x_k always computed in FP64 from the original values of A.
#include <cstdint>

#include "kernels.hpp"

namespace spchol {

namespace {

// Non-negative doubles order like their bit patterns as unsigned 64-bit integers.
__device__ __forceinline__ void atomic_max_nonneg(unsigned long long* p, double v) {
  atomicMax(p, (unsigned long long)__double_as_longlong(v));
}

__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// R = B - A X over the full symmetric pattern (CSR gather, one thread per row),
// and the column maxima |R|, |X|, |B| (3 per right-hand side).
__global__ void residual_kernel(int64_t n, int nrhs, const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                const int64_t* __restrict__ vmap, const double* __restrict__ aval,
                                const double* __restrict__ X, int64_t ldx, const double* __restrict__ B, int64_t ldb,
                                double* __restrict__ R, int64_t ldr, unsigned long long* __restrict__ colmax) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const bool active = i < n;
  for (int r = 0; r < nrhs; ++r) {
    double res = 0.0, xa = 0.0, ba = 0.0;
    if (active) {
      const double* x = X + r * ldx;
      double acc = B[i + r * ldb];
      for (int64_t k = rp[i]; k < rp[i + 1]; ++k) acc -= aval[vmap[k]] * x[ci[k]];
      R[i + r * ldr] = acc;
      res = fabs(acc);
      xa = fabs(x[i]);
      ba = fabs(B[i + r * ldb]);
    }
    res = warp_max(res);
    xa = warp_max(xa);
    ba = warp_max(ba);
    if ((threadIdx.x & 31) == 0) {
      atomic_max_nonneg(colmax + 3 * r + 0, res);
      atomic_max_nonneg(colmax + 3 * r + 1, xa);
      atomic_max_nonneg(colmax + 3 * r + 2, ba);
    }
  }
}

// max_i sum_j |a_ij| over the full symmetric matrix.
__global__ void anorm_kernel(int64_t n, const int64_t* __restrict__ rp, const int64_t* __restrict__ vmap,
                             const double* __restrict__ aval, unsigned long long* __restrict__ out) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  double s = 0.0;
  if (i < n)
    for (int64_t k = rp[i]; k < rp[i + 1]; ++k) s += fabs(aval[vmap[k]]);
  s = warp_max(s);
  if ((threadIdx.x & 31) == 0) atomic_max_nonneg(out, s);
}

// X[perm[i], r] += Y[i, r]
__global__ void correct_kernel(const double* __restrict__ Y, int64_t ldy, double* __restrict__ X, int64_t ldx,
                               const int32_t* __restrict__ perm, int64_t n, int nrhs) {
  const int64_t total = n * nrhs;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e % n, r = e / n;
    X[perm[i] + r * ldx] += Y[i + r * ldy];
  }
}

int blocks_for(int64_t n, int threads) {
  int64_t g = (n + threads - 1) / threads;
  return g < 1 ? 1 : (int)g;
}

// ---- GMRES-IR vector kernels (FP64; every reduction in one fixed order, so
// the refinement stays bitwise reproducible in deterministic mode)

// y = A x over the full symmetric pattern, one thread per row.
__global__ void spmv_kernel(int64_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                            const int64_t* __restrict__ vmap, const double* __restrict__ aval,
                            const double* __restrict__ x, double* __restrict__ y) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  double acc = 0.0;
  for (int64_t k = rp[i]; k < rp[i + 1]; ++k) acc += aval[vmap[k]] * x[ci[k]];
  y[i] = acc;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// partial[b * k + j] = block b's share of V_j . z for j < k (V_j at V + j ldv).
__global__ void dots_kernel(int64_t n, int k, const double* __restrict__ V, int64_t ldv, const double* __restrict__ z,
                            double* __restrict__ partial) {
  __shared__ double red[kGmresThreads / 32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int j = 0; j < k; ++j) {
    const double* v = V + j * ldv;
    double acc = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
      acc += v[i] * z[i];
    acc = warp_sum(acc);
    if (lane == 0) red[warp] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
      double s = 0.0;
      for (int w = 0; w < kGmresThreads / 32; ++w) s += red[w];
      partial[blockIdx.x * k + j] = s;
    }
    __syncthreads();
  }
}

// out[j] = sum over blocks b (in order) of partial[b * k + j].
__global__ void dots_finish_kernel(int nb, int k, const double* __restrict__ partial, double* __restrict__ out) {
  for (int j = threadIdx.x; j < k; j += blockDim.x) {
    double s = 0.0;
    for (int b = 0; b < nb; ++b) s += partial[b * k + j];
    out[j] = s;
  }
}

// z += alpha * sum_j V_j h_j, j < k.
__global__ void axpy_multi_kernel(int64_t n, int k, const double* __restrict__ V, int64_t ldv,
                                  const double* __restrict__ h, double alpha, double* __restrict__ z) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int j = 0; j < k; ++j) acc += V[j * ldv + i] * h[j];
    z[i] += alpha * acc;
  }
}

// y = alpha x
__global__ void scale_kernel(int64_t n, double alpha, const double* __restrict__ x, double* __restrict__ y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = alpha * x[i];
}

int grid_stride_blocks(int64_t n) {
  int64_t g = (n + kGmresThreads - 1) / kGmresThreads;
  if (g > kGmresBlocks) g = kGmresBlocks;
  return g < 1 ? 1 : (int)g;
}

}  // namespace

cudaError_t launch_residual(int64_t n, int nrhs, const int64_t* rp, const int32_t* ci, const int64_t* vmap,
                            const double* aval, const double* X, int64_t ldx, const double* B, int64_t ldb, double* R,
                            int64_t ldr, unsigned long long* colmax, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(colmax, 0, 3 * (size_t)nrhs * sizeof(unsigned long long), st);
  if (e != cudaSuccess) return e;
  if (n == 0) return cudaSuccess;
  residual_kernel<<<blocks_for(n, 256), 256, 0, st>>>(n, nrhs, rp, ci, vmap, aval, X, ldx, B, ldb, R, ldr, colmax);
  return cudaGetLastError();
}

cudaError_t launch_anorm(int64_t n, const int64_t* rp, const int64_t* vmap, const double* aval,
                         unsigned long long* out, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(out, 0, sizeof(unsigned long long), st);
  if (e != cudaSuccess) return e;
  if (n == 0) return cudaSuccess;
  anorm_kernel<<<blocks_for(n, 256), 256, 0, st>>>(n, rp, vmap, aval, out);
  return cudaGetLastError();
}

cudaError_t launch_spmv(int64_t n, const int64_t* rp, const int32_t* ci, const int64_t* vmap, const double* aval,
                        const double* x, double* y, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  spmv_kernel<<<blocks_for(n, 256), 256, 0, st>>>(n, rp, ci, vmap, aval, x, y);
  return cudaGetLastError();
}

cudaError_t launch_dots(int64_t n, int k, const double* V, int64_t ldv, const double* z, double* partial,
                        double* out, cudaStream_t st) {
  if (k == 0) return cudaSuccess;
  const int nb = grid_stride_blocks(n);
  dots_kernel<<<nb, kGmresThreads, 0, st>>>(n, k, V, ldv, z, partial);
  dots_finish_kernel<<<1, 64, 0, st>>>(nb, k, partial, out);
  return cudaGetLastError();
}

cudaError_t launch_axpy_multi(int64_t n, int k, const double* V, int64_t ldv, const double* h, double alpha, double* z,
                              cudaStream_t st) {
  if (n == 0 || k == 0) return cudaSuccess;
  axpy_multi_kernel<<<grid_stride_blocks(n), kGmresThreads, 0, st>>>(n, k, V, ldv, h, alpha, z);
  return cudaGetLastError();
}

cudaError_t launch_scale(int64_t n, double alpha, const double* x, double* y, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  scale_kernel<<<grid_stride_blocks(n), kGmresThreads, 0, st>>>(n, alpha, x, y);
  return cudaGetLastError();
}

cudaError_t launch_correct(const double* Y, int64_t ldy, double* X, int64_t ldx, const int32_t* perm, int64_t n,
                           int nrhs, cudaStream_t st) {
  if (n * nrhs == 0) return cudaSuccess;
  int64_t g = (n * nrhs + 255) / 256;
  if (g > 152 * 8) g = 152 * 8;
  correct_kernel<<<(int)g, 256, 0, st>>>(Y, ldy, X, ldx, perm, n, nrhs);
  return cudaGetLastError();
}

}  // namespace spchol
