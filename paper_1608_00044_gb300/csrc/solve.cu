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
  int next;  // continuation: a task this CTA made ready and runs next (-1: none)
};

template <typename T>
__device__ __forceinline__ const T* spanel(const SolveArgs& a, int s) {
  return reinterpret_cast<const T*>(a.pool) + a.pv.valoff[s];
}

// L11^{-1} (w x w, column-major, read-only here) into shared memory with
// leading dimension lx, the lower triangle only; loads in batches of 8.
__device__ __forceinline__ void stage_inverse(const double* __restrict__ X, int w, double* __restrict__ Xs, int lx) {
  const int total = w * w, nt = blockDim.x;
  for (int base = threadIdx.x; base < total; base += 8 * nt) {
    double v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int idx = base + u * nt, i = idx % w, j = idx / w;
      v[u] = (idx < total && i >= j) ? X[idx] : 0.0;
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int idx = base + u * nt, i = idx % w, j = idx / w;
      if (idx < total) Xs[i + j * lx] = v[u];
    }
  }
}

// y_s <- L11^{-1} y_s with the inverse formed by the diagonal factor task:
// every entry is an independent dot product, no sequential substitution.
// Thread (r, c) computes rows c and w - 1 - c for right-hand side r: i + 1
// and w - i terms, w + 1 in all, so every thread and warp does the same work.
__device__ void fwd_diag(const SolveArgs& a, int s, double* sm) {
  const int f = a.pv.fcol[s], w = a.pv.fcol[s + 1] - f;
  const double* X = a.inv + a.invoff[s];
  const int lx = w + 1;           // padded: lanes that walk a row or a column both avoid bank conflicts
  double* Xs = sm;                // [w][lx] column-major, lower part
  double* Ys = sm + w * lx;       // [nrc][w]
  stage_inverse(X, w, Xs, lx);
  const int half = (w + 1) >> 1;
  for (int r0 = 0; r0 < a.nrhs; r0 += kSolveNRC) {
    const int nrc = min(kSolveNRC, a.nrhs - r0);
    __syncthreads();
    for (int idx = threadIdx.x; idx < w * nrc; idx += blockDim.x) {
      const int j = idx % w, r = idx / w;
      Ys[idx] = ldcg(a.Y + f + j + (size_t)(r0 + r) * a.ldy);
    }
    __syncthreads();
    for (int p = threadIdx.x; p < half * nrc; p += blockDim.x) {
      const int c = p % half, r = p / half;
      const double* y = Ys + r * w;
      const int i1 = c, i2 = w - 1 - c;
      double a0 = 0.0, a1 = 0.0, b0 = 0.0, b1 = 0.0;
      int k = 0;
      for (; k + 1 <= i1; k += 2) {
        a0 += Xs[i1 + k * lx] * y[k];
        a1 += Xs[i1 + (k + 1) * lx] * y[k + 1];
      }
      if (k <= i1) a0 += Xs[i1 + k * lx] * y[k];
      if (i2 != i1) {
        for (k = 0; k + 1 <= i2; k += 2) {
          b0 += Xs[i2 + k * lx] * y[k];
          b1 += Xs[i2 + (k + 1) * lx] * y[k + 1];
        }
        if (k <= i2) b0 += Xs[i2 + k * lx] * y[k];
      }
      a.Y[f + i1 + (size_t)(r0 + r) * a.ldy] = a0 + a1;
      if (i2 != i1) a.Y[f + i2 + (size_t)(r0 + r) * a.ldy] = b0 + b1;
    }
  }
}

// x_s <- L11^{-T} y_s with the stored inverse: entry k is the dot product of
// column k of L11^{-1} (rows k .. w-1) with y_s; thread (r, c) takes columns c
// and w - 1 - c.
__device__ void bwd_diag(const SolveArgs& a, int s, double* sm) {
  const int f = a.pv.fcol[s], w = a.pv.fcol[s + 1] - f;
  const double* X = a.inv + a.invoff[s];
  const int lx = w + 1;
  double* Xs = sm;
  double* Ys = sm + w * lx;
  stage_inverse(X, w, Xs, lx);
  const int half = (w + 1) >> 1;
  for (int r0 = 0; r0 < a.nrhs; r0 += kSolveNRC) {
    const int nrc = min(kSolveNRC, a.nrhs - r0);
    __syncthreads();
    for (int idx = threadIdx.x; idx < w * nrc; idx += blockDim.x) {
      const int j = idx % w, r = idx / w;
      Ys[idx] = ldcg(a.Y + f + j + (size_t)(r0 + r) * a.ldy);
    }
    __syncthreads();
    for (int p = threadIdx.x; p < half * nrc; p += blockDim.x) {
      const int c = p % half, r = p / half;
      const double* y = Ys + r * w;
      const int k1 = c, k2 = w - 1 - c;
      double a0 = 0.0, a1 = 0.0, b0 = 0.0, b1 = 0.0;
      const double* x1 = Xs + k1 * lx;
      int i = k1;
      for (; i + 1 < w; i += 2) {
        a0 += x1[i] * y[i];
        a1 += x1[i + 1] * y[i + 1];
      }
      if (i < w) a0 += x1[i] * y[i];
      if (k2 != k1) {
        const double* x2 = Xs + k2 * lx;
        for (i = k2; i + 1 < w; i += 2) {
          b0 += x2[i] * y[i];
          b1 += x2[i + 1] * y[i + 1];
        }
        if (i < w) b0 += x2[i] * y[i];
      }
      a.Y[f + k1 + (size_t)(r0 + r) * a.ldy] = a0 + a1;
      if (k2 != k1) a.Y[f + k2 + (size_t)(r0 + r) * a.ldy] = b0 + b1;
    }
  }
}

// y[rows of tile] -= L21[tile] y_s.  A thread owns one row and NPER of the
// right-hand sides, g + G q (q < NPER) for its group g of G: with 8
// right-hand sides, four groups of 64 threads take two each (every warp busy on
// the 64-row tiles near the root); with one, all threads take rows.  The group
// is uniform in a warp and the right-hand sides a thread owns are fixed at
// compile time, so no FMA is spent on another group's right-hand sides.
template <typename T, int NPER>
__device__ void fwd_tile_rows(const SolveArgs& a, const T* P, int ld, int row0, int cnt, const int32_t* R, int w,
                              const double* Ys, int r0, int nrc, int G) {
  const int rows_per = blockDim.x / G;
  const int g = threadIdx.x / rows_per, il = threadIdx.x - g * rows_per;
  int nv = 0;  // right-hand sides of this thread that exist
#pragma unroll
  for (int q = 0; q < NPER; ++q) nv += (g + G * q < nrc) ? 1 : 0;
  if (nv == 0) return;
  for (int i = il; i < cnt; i += rows_per) {
    const T* Pi = P + row0 + i;
    double acc[NPER];
#pragma unroll
    for (int q = 0; q < NPER; ++q) acc[q] = 0.0;
    // the row's entries in batches of 8 independent loads, so that their
    // latencies overlap instead of following one another
    for (int j0 = 0; j0 < w; j0 += 8) {
      double l[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) l[u] = (j0 + u < w) ? (double)Pi[(size_t)(j0 + u) * ld] : 0.0;
      const int nu = min(8, w - j0);
      for (int u = 0; u < nu; ++u) {
#pragma unroll
        for (int q = 0; q < NPER; ++q) acc[q] += l[u] * Ys[j0 + u + (g + G * q) * w];
      }
    }
    const int gr = R[row0 + i];
#pragma unroll
    for (int q = 0; q < NPER; ++q)
      if (q < nv) red_add(a.Y + gr + (size_t)(r0 + g + G * q) * a.ldy, -acc[q]);
  }
}

template <typename T>
__device__ void fwd_tile(const SolveArgs& a, int s, int k, double* sm) {
  const int f = a.pv.fcol[s], w = a.pv.fcol[s + 1] - f, ld = a.pv.ld[s], r = a.pv.nrows[s];
  const int ts = a.st_rows[s];
  const int row0 = w + k * ts, cnt = min(ts, r - row0);
  const T* P = spanel<T>(a, s);
  const int32_t* R = a.pv.rows + a.pv.rowoff[s];
  double* Ys = sm;  // [kSolveNRC][w], zero past nrc
  for (int r0 = 0; r0 < a.nrhs; r0 += kSolveNRC) {
    const int nrc = min(kSolveNRC, a.nrhs - r0);
    __syncthreads();
    for (int idx = threadIdx.x; idx < w * kSolveNRC; idx += blockDim.x) {
      const int j = idx % w, rr = idx / w;
      Ys[idx] = rr < nrc ? ldcg(a.Y + f + j + (size_t)(r0 + rr) * a.ldy) : 0.0;
    }
    __syncthreads();
    if (nrc >= 5 && cnt <= 32)
      fwd_tile_rows<T, 1>(a, P, ld, row0, cnt, R, w, Ys, r0, nrc, 8);
    else if (nrc >= 5)
      fwd_tile_rows<T, 2>(a, P, ld, row0, cnt, R, w, Ys, r0, nrc, 4);
    else if (nrc >= 3)
      fwd_tile_rows<T, 1>(a, P, ld, row0, cnt, R, w, Ys, r0, nrc, 4);
    else
      fwd_tile_rows<T, 1>(a, P, ld, row0, cnt, R, w, Ys, r0, nrc, nrc);
  }
}

// y_s -= L21[tile]^T x[rows of tile]: rows staged kBwdCH at a time in shared
// memory (one batched pass and one barrier per chunk); thread (j, rr) sums
// column j of the chunk against x with four accumulators.
constexpr int kBwdCH = 64;

template <typename T>
__device__ void bwd_tile(const SolveArgs& a, int s, int k, double* sm) {
  const int f = a.pv.fcol[s], w = a.pv.fcol[s + 1] - f, ld = a.pv.ld[s], r = a.pv.nrows[s];
  const int ts = a.st_rows[s];
  const int row0 = w + k * ts, cnt = min(ts, r - row0);
  const T* P = spanel<T>(a, s);
  const int32_t* R = a.pv.rows + a.pv.rowoff[s];
  constexpr int CH = kBwdCH, LD = CH + 1;
  double* Lc = sm;                 // [w][LD]: Lc[i + j LD] = L21[c0 + i][j]
  double* Xc = Lc + w * LD;        // [nrc][CH]
  for (int r0 = 0; r0 < a.nrhs; r0 += kSolveNRC) {
    const int nrc = min(kSolveNRC, a.nrhs - r0);
    // each thread owns (j, rr) pairs p = tid + q * blockDim
    double part[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) part[q] = 0.0;
    for (int c0 = 0; c0 < cnt; c0 += CH) {
      const int nc = min(CH, cnt - c0);
      __syncthreads();
      for (int base = threadIdx.x; base < CH * w; base += 8 * blockDim.x) {
        double v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int idx = base + u * blockDim.x, i = idx % CH, j = idx / CH;
          v[u] = (idx < CH * w && i < nc) ? (double)P[row0 + c0 + i + (size_t)j * ld] : 0.0;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int idx = base + u * blockDim.x, i = idx % CH, j = idx / CH;
          if (idx < CH * w) Lc[i + j * LD] = v[u];
        }
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
          const double* lj = Lc + j * LD;
          const double* xr = Xc + rr * CH;
          double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
          for (int i = 0; i < nc; i += 4) {  // rows past nc are zero in both
            s0 += lj[i] * xr[i];
            s1 += lj[i + 1] * xr[i + 1];
            s2 += lj[i + 2] * xr[i + 2];
            s3 += lj[i + 3] * xr[i + 3];
          }
          part[q] += (s0 + s1) + (s2 + s3);
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

// Lower the counters cnt[id] of ids list[e] (or e itself when list is null),
// e in [e0, e1), by one, and push task task0 + id for each that reaches zero.
// Whole CTA; each thread issues its decrements in batches of 8 whose round
// trips overlap (a panel near the root releases thousands of tiles).
__device__ __forceinline__ void release_tiles(const Ring2& q, const int32_t* list, int e0, int e1, int32_t* cnt,
                                              int task0, int* next) {
  for (int base = e0 + threadIdx.x; base < e1; base += 8 * blockDim.x) {
    int id[8], old[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int e = base + u * blockDim.x;
      id[u] = e < e1 ? (list ? list[e] : e) : -1;
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) old[u] = id[u] >= 0 ? atom_add_acqrel(&cnt[id[u]], -1) : 0;
#pragma unroll
    for (int u = 0; u < 8; ++u)
      if (id[u] >= 0 && old[u] == 1) keep_or_push(q, next, task0 + id[u]);
  }
}

template <typename T>
__global__ void __launch_bounds__(kSolveThreads, 4) solve_kernel(SolveArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ SolveShared sh;
  double* sm = reinterpret_cast<double*>(smem_raw);
  // Two rings: tasks made ready by a finished task (high priority) ahead of
  // the seeds, so that chains up the tree advance instead of queueing behind
  // every leaf.
  const Ring2 q{a.ring, a.ring + a.n_hi, a.n_hi, a.ntask - a.n_hi, a.ctrl, a.budget_ns};
  __shared__ int pend[2];
  if (threadIdx.x == 0) {
    pend[0] = pend[1] = -1;
    sh.next = -1;
  }
  const int ns = a.pv.ns, nst = a.n_st;
  unsigned long long busy[4] = {0, 0, 0, 0}, wait = 0;
  for (;;) {
    uint64_t t1 = 0;
    if (threadIdx.x == 0) {
      const uint64_t t0 = a.prof ? global_ns() : 0;
      if (sh.next >= 0) {  // continue with a task this CTA made ready
        sh.task = sh.next;
        sh.next = -1;
      } else {
        int lo_ready;
        sh.task = ring2_claim(q, pend, &lo_ready, a.ntask);
      }
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
      // continue with the first forward tile (the rows of the parent) and
      // release the others
      if (a.nst[s] > 0) {
        if (threadIdx.x == 0) sh.next = ns + a.st_first[s];
        ring2_push_range(q, true, ns + a.st_first[s] + 1, a.nst[s] - 1, &sh.base);
      } else if (threadIdx.x == 0) {
        sh.next = ns + 2 * nst + s;
      }
    } else if (task < ns + nst) {
      const int kt = task - ns, s = a.st_sn[kt];
      fwd_tile<T>(a, s, kt - a.st_first[s], sm);
      publish_cta_writes();
      // Counter updates are spread over the CTA's threads: a panel near the
      // root has thousands of dependent tiles, and they sit on the critical path.
      for (int e = a.st_tptr[kt] + threadIdx.x; e < a.st_tptr[kt + 1]; e += blockDim.x) {
        const int t = a.st_tgt[e];
        if (atom_add_acqrel(&a.fdep[t], -1) == 1) keep_or_push(q, &sh.next, t);
      }
      if (threadIdx.x == 0) sh.flag = (atom_add_acqrel(&a.ftiles[s], -1) == 1);
      __syncthreads();
      if (sh.flag) release_tiles(q, nullptr, a.st_first[s], a.st_first[s] + a.nst[s], a.bdep, ns + nst, &sh.next);
    } else if (task < ns + 2 * nst) {
      const int kt = task - ns - nst, s = a.st_sn[kt];
      bwd_tile<T>(a, s, kt - a.st_first[s], sm);
      publish_cta_writes();
      if (threadIdx.x == 0 && atom_add_acqrel(&a.btiles[s], -1) == 1) keep_or_push(q, &sh.next, ns + 2 * nst + s);
    } else {
      const int s = task - ns - 2 * nst;
      bwd_diag(a, s, sm);
      publish_cta_writes();
      release_tiles(q, a.rt_tile, a.rt_ptr[s], a.rt_ptr[s + 1], a.bdep, ns + nst, &sh.next);
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
  const size_t diag = ((size_t)max_w * (max_w + 1) + (size_t)max_w * kSolveNRC) * sizeof(double);
  const size_t tile = ((size_t)max_w * (kBwdCH + 1) + kBwdCH * kSolveNRC) * sizeof(double);
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
__global__ void ring_reset_kernel(int* slots, int ntask, const int* seeds, int nseed, int seed_off, int seeds_hi,
                                  int* ctrl,
                                  int* c0, const int* c0_init, int n0, int* c1, const int* c1_init, int n1, int* c2,
                                  const int* c2_init, int n2, int* c3, const int* c3_init, int n3) {
  const int stride = gridDim.x * blockDim.x;
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  for (int i = tid; i < ntask; i += stride) slots[i] = (i >= seed_off && i < seed_off + nseed) ? seeds[i - seed_off] : -1;
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
                              int seeds_hi, int seed_off) {
  int m = ntask > kCtrlWords ? ntask : kCtrlWords;
  if (n0 > m) m = n0;
  if (n1 > m) m = n1;
  if (n2 > m) m = n2;
  if (n3 > m) m = n3;
  ring_reset_kernel<<<grid_for(m), 256, 0, st>>>(slots, ntask, seeds, nseed, seed_off, seeds_hi, ctrl, c0, c0_init,
                                                 n0, c1, c1_init, n1, c2, c2_init, n2, c3, c3_init, n3);
  return cudaGetLastError();
}

}  // namespace spchol
