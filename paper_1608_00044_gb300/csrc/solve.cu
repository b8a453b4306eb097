// Supernodal triangular solves L y = P b and L^T z = y (Section II-A), as one
// persistent launch over a task graph derived from the panel elimination tree.
//
// Task ids:
//   [0, ns)                      FWD_D(s): y_s <- L11^{-1} y_s
//   [ns, ns + nst)               FWD_T(s, k): y[rows of tile k] -= L21[k] y_s
//   [ns + nst, ns + 2 nst)       BWD_T(s, k): y_s -= L21[k]^T x[rows of tile k]
//   [ns + 2 nst, 2 ns + 2 nst)   BWD_D(s): x_s <- L11^{-T} y_s
// Dependencies are exact, per panel and per tile.  Forward: FWD_D(t) runs once
// every FWD_T tile whose rows fall in t's columns has subtracted its part.
// Backward: BWD_T(s, k) runs once every panel its rows fall in has finished
// BWD_D (those x are final) and every forward tile of s is done (so y_s is no
// longer read by them); BWD_D(s) runs after all tiles of s.  A root has no
// rows below its diagonal block, so its FWD_D is followed directly by its
// BWD_D.
#include <climits>
#include <cstdint>
#include <map>
#include <mutex>

#include "device_common.cuh"
#include "kernels.hpp"
#include "sched.cuh"

namespace spchol {

namespace {

struct SolveShared {
  int task;
  int flag;
  int base;
};

template <typename T>
__device__ __forceinline__ const T* spanel(const SolveArgs& a, int s) {
  return reinterpret_cast<const T*>(a.pool) + a.pv.valoff[s];
}

// y_s <- L11^{-1} y_s with the inverse formed by the diagonal factor task:
// every entry is an independent dot product, no sequential substitution.
__device__ void fwd_diag(const SolveArgs& a, int s, double* sm) {
  const int f = a.pv.fcol[s], w = a.pv.fcol[s + 1] - f;
  const double* X = a.inv + a.invoff[s];
  double* Xs = sm;          // [w][w] column-major, lower part
  double* Ys = sm + w * w;  // [nrc][w]
  stage_lower<false>(X, w, w, Xs);
  for (int r0 = 0; r0 < a.nrhs; r0 += kSolveNRC) {
    const int nrc = min(kSolveNRC, a.nrhs - r0);
    __syncthreads();
    for (int idx = threadIdx.x; idx < w * nrc; idx += blockDim.x) {
      const int j = idx % w, r = idx / w;
      Ys[idx] = ldcg(a.Y + f + j + (size_t)(r0 + r) * a.ldy);
    }
    __syncthreads();
    for (int p = threadIdx.x; p < w * nrc; p += blockDim.x) {
      const int i = p % w, r = p / w;
      const double* y = Ys + r * w;
      double a0 = 0.0, a1 = 0.0;
      int k = 0;
      for (; k + 1 <= i; k += 2) {
        a0 += Xs[i + k * w] * y[k];
        a1 += Xs[i + (k + 1) * w] * y[k + 1];
      }
      if (k <= i) a0 += Xs[i + k * w] * y[k];
      a.Y[f + i + (size_t)(r0 + r) * a.ldy] = a0 + a1;
    }
  }
}

// x_s <- L11^{-T} y_s with the stored inverse.
__device__ void bwd_diag(const SolveArgs& a, int s, double* sm) {
  const int f = a.pv.fcol[s], w = a.pv.fcol[s + 1] - f;
  const double* X = a.inv + a.invoff[s];
  double* Xs = sm;
  double* Ys = sm + w * w;
  stage_lower<false>(X, w, w, Xs);
  for (int r0 = 0; r0 < a.nrhs; r0 += kSolveNRC) {
    const int nrc = min(kSolveNRC, a.nrhs - r0);
    __syncthreads();
    for (int idx = threadIdx.x; idx < w * nrc; idx += blockDim.x) {
      const int j = idx % w, r = idx / w;
      Ys[idx] = ldcg(a.Y + f + j + (size_t)(r0 + r) * a.ldy);
    }
    __syncthreads();
    for (int p = threadIdx.x; p < w * nrc; p += blockDim.x) {
      const int kcol = p % w, r = p / w;
      const double* y = Ys + r * w;
      const double* xc = Xs + kcol * w;  // column kcol of L11^{-1}: rows kcol..w-1
      double a0 = 0.0, a1 = 0.0;
      int i = kcol;
      for (; i + 1 < w; i += 2) {
        a0 += xc[i] * y[i];
        a1 += xc[i + 1] * y[i + 1];
      }
      if (i < w) a0 += xc[i] * y[i];
      a.Y[f + kcol + (size_t)(r0 + r) * a.ldy] = a0 + a1;
    }
  }
}

// y[rows of tile] -= L21[tile] y_s, one row per thread.
template <typename T>
__device__ void fwd_tile(const SolveArgs& a, int s, int k, double* sm) {
  const int f = a.pv.fcol[s], w = a.pv.fcol[s + 1] - f, ld = a.pv.ld[s], r = a.pv.nrows[s];
  const int row0 = w + k * a.solve_rows, cnt = min(a.solve_rows, r - row0);
  const T* P = spanel<T>(a, s);
  const int32_t* R = a.pv.rows + a.pv.rowoff[s];
  double* Ys = sm;  // [nrc][w]
  for (int r0 = 0; r0 < a.nrhs; r0 += kSolveNRC) {
    const int nrc = min(kSolveNRC, a.nrhs - r0);
    __syncthreads();
    for (int idx = threadIdx.x; idx < w * nrc; idx += blockDim.x) {
      const int j = idx % w, rr = idx / w;
      Ys[idx] = ldcg(a.Y + f + j + (size_t)(r0 + rr) * a.ldy);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
      const T* Pi = P + row0 + i;
      double acc[kSolveNRC];
#pragma unroll
      for (int rr = 0; rr < kSolveNRC; ++rr) acc[rr] = 0.0;
      for (int j = 0; j < w; ++j) {
        const double l = (double)Pi[(size_t)j * ld];
#pragma unroll
        for (int rr = 0; rr < kSolveNRC; ++rr) acc[rr] += l * Ys[j + rr * w];
      }
      const int g = R[row0 + i];
#pragma unroll
      for (int rr = 0; rr < kSolveNRC; ++rr)
        if (rr < nrc) red_add(a.Y + g + (size_t)(r0 + rr) * a.ldy, -acc[rr]);
    }
  }
}

// y_s -= L21[tile]^T x[rows of tile]: rows staged 32 at a time in shared memory.
template <typename T>
__device__ void bwd_tile(const SolveArgs& a, int s, int k, double* sm) {
  const int f = a.pv.fcol[s], w = a.pv.fcol[s + 1] - f, ld = a.pv.ld[s], r = a.pv.nrows[s];
  const int row0 = w + k * a.solve_rows, cnt = min(a.solve_rows, r - row0);
  const T* P = spanel<T>(a, s);
  const int32_t* R = a.pv.rows + a.pv.rowoff[s];
  constexpr int CH = 32;
  double* Lc = sm;                  // [w][CH + 1]
  double* Xc = Lc + w * (CH + 1);   // [nrc][CH]
  for (int r0 = 0; r0 < a.nrhs; r0 += kSolveNRC) {
    const int nrc = min(kSolveNRC, a.nrhs - r0);
    // each thread owns (j, rr) pairs p = tid + q * blockDim
    double part[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) part[q] = 0.0;
    for (int c0 = 0; c0 < cnt; c0 += CH) {
      const int nc = min(CH, cnt - c0);
      __syncthreads();
      for (int idx = threadIdx.x; idx < CH * w; idx += blockDim.x) {
        const int i = idx % CH, j = idx / CH;
        Lc[j * (CH + 1) + i] = (i < nc) ? (double)P[row0 + c0 + i + (size_t)j * ld] : 0.0;
      }
      for (int idx = threadIdx.x; idx < CH * nrc; idx += blockDim.x) {
        const int i = idx % CH, rr = idx / CH;
        Xc[rr * CH + i] = (i < nc) ? ldcg(a.Y + R[row0 + c0 + i] + (size_t)(r0 + rr) * a.ldy) : 0.0;
      }
      __syncthreads();
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int p = threadIdx.x + q * blockDim.x;
        if (p < w * nrc) {
          const int j = p % w, rr = p / w;
          double acc = part[q];
#pragma unroll 8
          for (int i = 0; i < CH; ++i) acc += Lc[j * (CH + 1) + i] * Xc[rr * CH + i];
          part[q] = acc;
        }
      }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int p = threadIdx.x + q * blockDim.x;
      if (p < w * nrc) {
        const int j = p % w, rr = p / w;
        red_add(a.Y + f + j + (size_t)(r0 + rr) * a.ldy, -part[q]);
      }
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(kSolveThreads) solve_kernel(SolveArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ SolveShared sh;
  double* sm = reinterpret_cast<double*>(smem_raw);
  const Ring q{a.ring, a.ctrl, a.ntask, a.budget_ns};
  const int ns = a.pv.ns, nst = a.n_st;
  unsigned long long busy[4] = {0, 0, 0, 0}, wait = 0;
  for (;;) {
    uint64_t t1 = 0;
    if (threadIdx.x == 0) {
      const uint64_t t0 = a.prof ? global_ns() : 0;
      sh.task = ring_claim(q);
      if (a.prof) {
        t1 = global_ns();
        wait += t1 - t0;
      }
    }
    __syncthreads();
    const int task = sh.task;
    if (task < 0) break;
    const int type = task < ns ? 0 : task < ns + nst ? 1 : task < ns + 2 * nst ? 2 : 3;
    if (task < ns) {
      const int s = task;
      fwd_diag(a, s, sm);
      publish_cta_writes();
      if (a.nst[s] > 0) {
        ring_push_range(q, ns + a.st_first[s], a.nst[s], &sh.base);
      } else if (threadIdx.x == 0) {
        ring_push_one(q, ns + 2 * nst + s);
      }
    } else if (task < ns + nst) {
      const int kt = task - ns, s = a.st_sn[kt];
      fwd_tile<T>(a, s, kt - a.st_first[s], sm);
      publish_cta_writes();
      // Counter updates are spread over the CTA's threads: a panel near the
      // root has thousands of dependent tiles, and they sit on the critical path.
      for (int e = a.st_tptr[kt] + threadIdx.x; e < a.st_tptr[kt + 1]; e += blockDim.x) {
        const int t = a.st_tgt[e];
        if (atom_add_acqrel(&a.fdep[t], -1) == 1) ring_push_one(q, t);
      }
      if (threadIdx.x == 0) sh.flag = (atom_add_acqrel(&a.ftiles[s], -1) == 1);
      __syncthreads();
      if (sh.flag) {
        for (int k = threadIdx.x; k < a.nst[s]; k += blockDim.x) {
          const int tile = a.st_first[s] + k;
          if (atom_add_acqrel(&a.bdep[tile], -1) == 1) ring_push_one(q, ns + nst + tile);
        }
      }
    } else if (task < ns + 2 * nst) {
      const int kt = task - ns - nst, s = a.st_sn[kt];
      bwd_tile<T>(a, s, kt - a.st_first[s], sm);
      publish_cta_writes();
      if (threadIdx.x == 0 && atom_add_acqrel(&a.btiles[s], -1) == 1) ring_push_one(q, ns + 2 * nst + s);
    } else {
      const int s = task - ns - 2 * nst;
      bwd_diag(a, s, sm);
      publish_cta_writes();
      for (int e = a.rt_ptr[s] + threadIdx.x; e < a.rt_ptr[s + 1]; e += blockDim.x) {
        const int tile = a.rt_tile[e];
        if (atom_add_acqrel(&a.bdep[tile], -1) == 1) ring_push_one(q, ns + nst + tile);
      }
    }
    if (threadIdx.x == 0) {
      atomicAdd(&a.ctrl[kDone], 1);
      if (a.trace) {
        a.trace[2 * (size_t)task] = t1;
        a.trace[2 * (size_t)task + 1] = global_ns();
      }
      if (a.prof) busy[type] += global_ns() - t1;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0 && a.prof) {
    for (int k = 0; k < 4; ++k) atomicAdd(&a.prof[k], busy[k]);
    atomicAdd(&a.prof[4], wait);
  }
}

__global__ void permute_in_kernel(const double* __restrict__ B, int64_t ldb, double* __restrict__ Y, int64_t ldy,
                                  const int32_t* __restrict__ perm, int64_t n, int nrhs) {
  const int64_t total = n * nrhs;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e % n, r = e / n;
    Y[i + r * ldy] = B[perm[i] + r * ldb];
  }
}

__global__ void permute_out_kernel(const double* __restrict__ Y, int64_t ldy, double* __restrict__ B, int64_t ldb,
                                   const int32_t* __restrict__ perm, int64_t n, int nrhs) {
  const int64_t total = n * nrhs;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e % n, r = e / n;
    B[perm[i] + r * ldb] = Y[i + r * ldy];
  }
}

}  // namespace

size_t solve_smem_bytes(int max_w) {
  const size_t diag = ((size_t)max_w * max_w + (size_t)max_w * kSolveNRC) * sizeof(double);
  const size_t tile = ((size_t)max_w * 33 + 32 * kSolveNRC) * sizeof(double);
  return diag > tile ? diag : tile;
}

cudaError_t solve_configure(bool fp32, size_t smem, int* blocks_per_sm) {
  const void* fn = fp32 ? (const void*)solve_kernel<float> : (const void*)solve_kernel<double>;
  cudaError_t e = ensure_smem_limit(fn, smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, fn, kSolveThreads, smem);
}

cudaError_t launch_solve(bool fp32, const SolveArgs& a, int grid, size_t smem, cudaStream_t st) {
  if (fp32)
    solve_kernel<float><<<grid, kSolveThreads, smem, st>>>(a);
  else
    solve_kernel<double><<<grid, kSolveThreads, smem, st>>>(a);
  return cudaGetLastError();
}

cudaError_t ensure_smem_limit(const void* fn, size_t need) {
  static std::mutex mu;
  static std::map<const void*, size_t> current;
  std::lock_guard<std::mutex> lock(mu);
  size_t& cur = current[fn];
  if (need <= cur) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)need);
  if (e == cudaSuccess) cur = need;
  return e;
}

static int grid_for(int64_t total) {
  int64_t g = (total + 255) / 256;
  if (g > 152 * 8) g = 152 * 8;
  return g < 1 ? 1 : (int)g;
}

cudaError_t launch_permute_in(const double* B, int64_t ldb, double* Y, int64_t ldy, const int32_t* perm,
                              int64_t n, int nrhs, cudaStream_t st) {
  if (n * nrhs == 0) return cudaSuccess;
  permute_in_kernel<<<grid_for(n * nrhs), 256, 0, st>>>(B, ldb, Y, ldy, perm, n, nrhs);
  return cudaGetLastError();
}

cudaError_t launch_permute_out(const double* Y, int64_t ldy, double* B, int64_t ldb, const int32_t* perm,
                               int64_t n, int nrhs, cudaStream_t st) {
  if (n * nrhs == 0) return cudaSuccess;
  permute_out_kernel<<<grid_for(n * nrhs), 256, 0, st>>>(Y, ldy, B, ldb, perm, n, nrhs);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- ring reset
__global__ void ring_reset_kernel(int* slots, int ntask, const int* seeds, int nseed, int seeds_hi, int* ctrl,
                                  int* c0, const int* c0_init, int n0, int* c1, const int* c1_init, int n1, int* c2,
                                  const int* c2_init, int n2, int* c3, const int* c3_init, int n3) {
  const int stride = gridDim.x * blockDim.x;
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  for (int i = tid; i < ntask; i += stride) slots[i] = (i < nseed) ? seeds[i] : -1;
  for (int i = tid; i < n0; i += stride) c0[i] = c0_init[i];
  for (int i = tid; i < n1; i += stride) c1[i] = c1_init[i];
  for (int i = tid; i < n2; i += stride) c2[i] = c2_init[i];
  for (int i = tid; i < n3; i += stride) c3[i] = c3_init[i];
  if (tid < kCtrlWords) {  // one thread per control word
    int v = 0;
    if (tid == kTail) v = seeds_hi ? 0 : nseed;
    if (tid == kHiTail) v = seeds_hi ? nseed : 0;
    if (tid == kInfo) v = INT_MAX;
    if (tid == kWhere) v = -1;
    ctrl[tid] = v;
  }
}

// ---------------------------------------------------------------- fixed scratch for spchol_solve_noalloc
// Callers that must not allocate device memory during a solve (a process whose
// device memory is fully reserved up front, or code running where allocation
// calls are not permitted) use spchol_solve_noalloc, whose workspace lives in
// this file-scope array instead of memory from cudaMalloc.  Every GPU that
// loads the library holds it until the process exits.  All calls share it, so
// calls whose work overlaps on the GPU race on it.
__device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

cudaError_t noalloc_scratch(int device, void** ptr) {
  // One address per device, looked up once with that device current: in host
  // code the array's name is only a host-side stand-in, never a device address.
  constexpr int kMaxDevices = 64;
  static std::mutex mu;
  static void* addr[kMaxDevices] = {};
  if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(mu);
  if (addr[device]) {
    *ptr = addr[device];
    return cudaSuccess;
  }
  int prev = -1;
  cudaError_t e = cudaGetDevice(&prev);
  if (e != cudaSuccess) return e;
  if (prev != device && (e = cudaSetDevice(device)) != cudaSuccess) return e;
  void* p = nullptr;
  e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (prev != device) cudaSetDevice(prev);
  if (e != cudaSuccess) return e;
  addr[device] = p;
  *ptr = p;
  return cudaSuccess;
}

cudaError_t launch_ring_reset(int* slots, int ntask, const int* seeds, int nseed, int* ctrl, int* c0,
                              const int* c0_init, int n0, int* c1, const int* c1_init, int n1, int* c2,
                              const int* c2_init, int n2, cudaStream_t st, int* c3, const int* c3_init, int n3,
                              int seeds_hi) {
  int m = ntask > kCtrlWords ? ntask : kCtrlWords;
  if (n0 > m) m = n0;
  if (n1 > m) m = n1;
  if (n2 > m) m = n2;
  if (n3 > m) m = n3;
  ring_reset_kernel<<<grid_for(m), 256, 0, st>>>(slots, ntask, seeds, nseed, seeds_hi, ctrl, c0, c0_init, n0, c1,
                                                 c1_init, n1, c2, c2_init, n2, c3, c3_init, n3);
  return cudaGetLastError();
}

}  // namespace spchol
