// Device-side helpers shared by the factorization and solve kernels:
// memory-model primitives for the task ring and dependency counters, and the
// control block layout.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace spchol {

// Control block (int32 words) of one persistent launch.
enum CtrlWord : int {
  kHead = 0,     // next ring slot to claim (the factorization's normal-priority ring)
  kTail = 1,     // next ring slot to fill
  kErr = 2,      // 0, or an SPCHOL_E* code (timeout, internal check)
  kInfo = 3,     // smallest failing pivot column + 1, INT32_MAX if none
  kWhere = 5,    // diagnostic: task id where a wait gave up
  kWarpNext = 6, // the next warp-level subtree task (FactorArgs::wsub; the solves' forward launch)
  kWarpNextB = 7, // the solves' backward launch's next warp-level subtree
  kHiHead = 32,  // the high-priority ring, in its own 128-byte line
  kHiTail = 33,
  kDone = 64,    // tasks completed: the end test, updated by every task, in a line of its own
  kCtrlWords = 96
};

__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(int* p, int v) {
  asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ int atom_add_acqrel(int* p, int v) {
  int old;
  asm volatile("atom.acq_rel.gpu.global.add.s32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
  return old;
}
__device__ __forceinline__ int ld_relaxed(const int* p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
// Two adjacent words (8-byte aligned) in one load: x = p[0], y = p[1].
__device__ __forceinline__ int2 ld_relaxed_pair(const int* p) {
  int2 v;
  asm volatile("ld.relaxed.gpu.global.v2.b32 {%0, %1}, [%2];" : "=r"(v.x), "=r"(v.y) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Loads of data that other CTAs of the same launch may have written: served
// from L2, never from a possibly stale L1 line.
__device__ __forceinline__ double ldcg(const double* p) { return __ldcg(p); }
__device__ __forceinline__ float ldcg(const float* p) { return __ldcg(p); }
__device__ __forceinline__ int ldcg(const int* p) { return __ldcg(p); }

__device__ __forceinline__ void red_add(double* p, double v) { atomicAdd(p, v); }

// Copy the lower triangle of a w x w column-major block (leading dimension ld)
// into shared memory as double (ld w, zeros above the diagonal).  Each thread
// issues a batch of independent loads before it stores any of them, so the
// copy costs a few memory latencies instead of one per element.
template <bool kL2Only, typename T>
__device__ __forceinline__ void stage_lower(const T* __restrict__ src, int w, int ld, double* __restrict__ dst) {
  constexpr int B = 8;
  const int total = w * w, nt = blockDim.x;
  for (int base = threadIdx.x; base < total; base += B * nt) {
    double v[B];
#pragma unroll
    for (int u = 0; u < B; ++u) {
      const int idx = base + u * nt;
      const int i = idx % w, j = idx / w;
      v[u] = 0.0;
      if (idx < total && i >= j) {
        const T* p = src + i + (size_t)j * ld;
        v[u] = kL2Only ? (double)__ldcg(p) : (double)*p;
      }
    }
#pragma unroll
    for (int u = 0; u < B; ++u) {
      const int idx = base + u * nt;
      if (idx < total) dst[idx] = v[u];
    }
  }
}

// Raise a kernel's dynamic shared-memory limit to at least `need` bytes (host).
// The limit is a per-kernel setting shared by every handle of the process; it
// only ever grows, to the largest size any handle has needed, so a launch
// never finds it lowered by another handle.  (Raising it straight to the
// device maximum would lower the occupancy the runtime reports.)
cudaError_t ensure_smem_limit(const void* fn, size_t need);
__device__ __forceinline__ void red_add(float* p, float v) { atomicAdd(p, v); }

// An update value into its destination: an atomic add into a target panel
// that other tiles update too, or a plain store into a buffer that only this
// tile writes (the fan-in mode of the factorization).
template <typename T>
__device__ __forceinline__ void scatter_put(T* p, T v, bool store) {
  if (store)
    *p = v;
  else
    red_add(p, v);
}

}  // namespace spchol
