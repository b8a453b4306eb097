// Ready-task ring shared by the persistent factorization and solve kernels.
//
// The paper keeps, per process, a queue of statically mapped tasks and a queue
// of ready tasks; a task becomes ready when its incoming-dependency counter
// reaches zero, and the producer of its input notifies it (Section IV, the
// LTQ/RTQ pair and the signal/poll/get protocol of Section IV-A).  On one GPU
// the ready queue is a ring of task ids in global memory: a CTA that finishes a
// task decrements the counters of the dependent tasks with an acq_rel atomic
// (the "signal"), pushes every task whose counter reached zero with a release
// store, and claims the next slot of the ring (the "poll").  Only ready tasks
// are ever pushed, so a CTA never waits on work that has not been started by a
// running CTA -- the ordering argument that keeps the paper's pull variant free
// of deadlock (Section III-D) -- and every wait is bounded in time and in
// iterations.
#pragma once
#include <climits>
#include <cstdint>

#include "device_common.cuh"

namespace spchol {

#define SPCHOL_DEV_ETIMEOUT (-1002)
#define SPCHOL_DEV_EINTERNAL (-1006)

struct Ring {
  int* slots;  // ntask entries, -1 while empty
  int* ctrl;   // CtrlWord layout
  int ntask;
  int64_t budget_ns;
};

// Thread 0 only.  Returns the claimed task id, or -1 when every task has been
// claimed, another CTA reported an error, or the wait ran out of budget.
__device__ __forceinline__ int ring_claim(const Ring& q) {
  const int slot = atomicAdd(&q.ctrl[kHead], 1);
  if (slot >= q.ntask) return -1;
  const uint64_t t0 = global_ns();
  const uint64_t max_iter = (uint64_t)(q.budget_ns / 32) + 100000;
  unsigned backoff = 32;
  for (uint64_t it = 0;; ++it) {
    const int v = ld_acquire(&q.slots[slot]);
    if (v >= 0) {
      __threadfence();
      return v;
    }
    if (ld_relaxed(&q.ctrl[kErr]) != 0) return -1;
    if (it > max_iter || (int64_t)(global_ns() - t0) > q.budget_ns) {
      atomicCAS(&q.ctrl[kErr], 0, SPCHOL_DEV_ETIMEOUT);
      atomicExch(&q.ctrl[kWhere], slot);
      return -1;
    }
    __nanosleep(backoff);
    if (backoff < 1024) backoff <<= 1;
  }
}

// Thread 0 only: push one ready task.  The caller has made the task's inputs
// visible (__threadfence by every writer, then __syncthreads).
__device__ __forceinline__ void ring_push_one(const Ring& q, int task) {
  const int slot = atomicAdd(&q.ctrl[kTail], 1);
  if (slot < q.ntask) {
    st_release(&q.slots[slot], task);
  } else {
    atomicCAS(&q.ctrl[kErr], 0, SPCHOL_DEV_EINTERNAL);
  }
}

// Whole CTA: push the ready tasks first .. first+count-1.  s_base is a shared
// int.  Same visibility precondition as ring_push_one.
__device__ __forceinline__ void ring_push_range(const Ring& q, int first, int count, int* s_base) {
  if (count <= 0) return;
  if (threadIdx.x == 0) *s_base = atomicAdd(&q.ctrl[kTail], count);
  __syncthreads();
  const int base = *s_base;
  for (int i = threadIdx.x; i < count; i += blockDim.x) {
    if (base + i < q.ntask) {
      st_release(&q.slots[base + i], first + i);
    } else {
      atomicCAS(&q.ctrl[kErr], 0, SPCHOL_DEV_EINTERNAL);
    }
  }
  __syncthreads();
}

// Make this CTA's global writes visible before a counter update or a push.
__device__ __forceinline__ void publish_cta_writes() {
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) __threadfence();
}

// Reset kernel: ring slots to -1 with the seed tasks in front, counters from
// their initial copies, control words.
__global__ void ring_reset_kernel(int* slots, int ntask, const int* seeds, int nseed, int* ctrl,
                                  int* c0, const int* c0_init, int n0, int* c1, const int* c1_init,
                                  int n1, int* c2, const int* c2_init, int n2, int* c3,
                                  const int* c3_init, int n3);

}  // namespace spchol
