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

// The factorization's two ready rings.  High priority: diagonal and panel-solve
// tasks and the update tiles that gate the next diagonal task near the root
// (the critical path); normal priority: all other update tiles.  An idle CTA
// takes a visible high-priority task first.  A CTA claims a slot only when the
// ring shows an unclaimed filled or reserved slot, so it holds a claimed slot
// that is still empty only after losing a race for the last one, and a ready
// task never waits behind a busy CTA for longer than such a race.  Every
// claimed slot is filled eventually (a pusher reserves slots in order, so the
// lowest claimed empty slot is the next to be filled).  A CTA holding a
// claimed empty slot below the tail waits for the push that is filling it; one
// holding a slot past the tail keeps serving the other ring, since the push
// that fills it may need that ring's tasks: no CTA blocks the progress of
// another.
struct Ring2 {
  int* hi;  // n_hi slots, -1 while empty
  int* lo;  // n_lo slots
  int n_hi, n_lo;
  int* ctrl;
  int64_t budget_ns;
};

// Thread 0 only.  pend[0]: this CTA's claimed, not yet taken slot of the
// high-priority ring; pend[1], pend[2]: of the normal-priority ring, taken in
// that order (-1 none); all kept across calls.  Returns a task id, or -1 when
// every task has been claimed, another CTA reported an error, or the wait ran
// out.  *lo_ready: unclaimed slots of the normal-priority ring at the last
// look (0 if the task came from the high-priority ring before the other was
// read).  When the task comes from pend[1] and pend[2] is filled as well, and
// stash is given, pend[2]'s task is acquired too and returned in *stash, for
// the caller to run next without a claim.
__device__ __forceinline__ int ring2_claim(const Ring2& q, int* pend, int* lo_ready, int ntask_total,
                                           int* stash = nullptr) {
  *lo_ready = 0;
  const uint64_t t0 = global_ns();
  const uint64_t max_iter = (uint64_t)(q.budget_ns / 32) + 100000;
  unsigned backoff = 32;
  for (uint64_t it = 0;; ++it) {
    // Both rings' (head, tail) and the normal-priority slots this CTA already
    // holds, in one round trip: relaxed loads, none waiting for another (a
    // claim with slots held ahead -- the common case -- used to take three
    // round trips).  A slot value is used only after the fence below: a
    // relaxed load that sees the pusher's release store, then the fence, is
    // an acquire.
    const int2 hi = ld_relaxed_pair(&q.ctrl[kHiHead]);  // (head, tail)
    const int2 lo = ld_relaxed_pair(&q.ctrl[kHead]);
    const int v1 = pend[1] >= 0 ? ld_relaxed(&q.lo[pend[1]]) : -1;
    const int v2 = pend[2] >= 0 ? ld_relaxed(&q.lo[pend[2]]) : -1;
    *lo_ready = lo.y - lo.x;
    if (pend[0] < 0 && hi.x < hi.y && hi.x < q.n_hi) {
      const int s = atomicAdd(&q.ctrl[kHiHead], 1);
      pend[0] = s < q.n_hi ? s : -1;
    }
    if (pend[0] >= 0) {
      const int v = ld_acquire(&q.hi[pend[0]]);
      if (v >= 0) {
        pend[0] = -1;
        __threadfence();
        return v;
      }
    }
    if (pend[0] >= 0 && pend[0] < hi.y) {
      // The slot lies below the tail: a push that reserved it is storing into
      // it now, so wait for it rather than start a normal-priority task,
      // whose continuations could hold this reservation -- and delay its task
      // -- for milliseconds (one such solve tile waited 3.6 ms).  A slot past
      // the tail (a lost race for the last one) is filled only by a future
      // push, which may need the other ring's tasks: keep serving that ring.
    } else if (v1 >= 0) {
      pend[1] = -1;
      if (v2 >= 0 && stash) {
        *stash = v2;
        pend[2] = -1;
      } else if (pend[2] >= 0) {
        pend[1] = pend[2];
        pend[2] = -1;
      }
      __threadfence();
      return v1;
    } else if (pend[1] < 0 && lo.x < lo.y && lo.x < q.n_lo) {
      const int s = atomicAdd(&q.ctrl[kHead], 1);
      pend[1] = s < q.n_lo ? s : -1;
      if (pend[1] >= 0) {
        const int v = ld_acquire(&q.lo[pend[1]]);
        if (v >= 0) {
          pend[1] = -1;
          __threadfence();
          return v;
        }
      }
    }
    if (pend[0] < 0 && pend[1] < 0 && pend[2] < 0 && hi.x >= q.n_hi && lo.x >= q.n_lo) return -1;  // all claimed
    // An idle grid polls these words from every CTA: the error word is read on
    // every 8th round only, and the backoff grows to 2 us, so that the polling
    // does not queue up the claims and pushes on the same L2 lines.
    if ((it & 7) == 7) {
      if (ld_relaxed(&q.ctrl[kErr]) != 0) return -1;
      // a task made ready may run in the CTA that released it without passing
      // through a ring, so the rings' slot counts do not tell the end: the
      // completed-task count does
      if (ld_relaxed(&q.ctrl[kDone]) >= ntask_total) return -1;
    }
    if (it > max_iter || (int64_t)(global_ns() - t0) > q.budget_ns) {
      atomicCAS(&q.ctrl[kErr], 0, SPCHOL_DEV_ETIMEOUT);
      atomicExch(&q.ctrl[kWhere], pend[0] >= 0 ? pend[0] : pend[1]);
      return -1;
    }
    __nanosleep(backoff);
    if (backoff < 2048) backoff <<= 1;
  }
}

// Push ready tasks first .. first+count-1 to one ring of a Ring2 (hi: the
// high-priority one; a Ring2 with n_hi = 0 is a single FIFO ring, and every
// push goes to it).  Whole CTA; s_base is a shared int.  Same visibility
// precondition as ring_push_one.
__device__ __forceinline__ void ring2_push_range(const Ring2& q, bool hi, int first, int count, int* s_base) {
  if (count <= 0) return;
  hi = hi && q.n_hi > 0;  // a launch without a high-priority ring: one FIFO ring
  int* tail = &q.ctrl[hi ? kHiTail : kTail];
  int* slots = hi ? q.hi : q.lo;
  const int n = hi ? q.n_hi : q.n_lo;
  if (threadIdx.x == 0) *s_base = atomicAdd(tail, count);
  __syncthreads();
  const int base = *s_base;
  for (int i = threadIdx.x; i < count; i += blockDim.x) {
    if (base + i < n) {
      st_release(&slots[base + i], first + i);
    } else {
      atomicCAS(&q.ctrl[kErr], 0, SPCHOL_DEV_EINTERNAL);
    }
  }
  __syncthreads();
}

// Any thread: push the ready tasks first .. first+count-1 to one ring of a
// Ring2 with one reservation (a W panel's forward tiles, made ready by one
// counter).
__device__ __forceinline__ void ring2_push_span(const Ring2& q, bool hi, int first, int count) {
  if (count <= 0) return;
  hi = hi && q.n_hi > 0;
  const int base = atomicAdd(&q.ctrl[hi ? kHiTail : kTail], count);
  int* slots = hi ? q.hi : q.lo;
  const int n = hi ? q.n_hi : q.n_lo;
  for (int i = 0; i < count; ++i) {
    if (base + i < n) {
      st_release(&slots[base + i], first + i);
    } else {
      atomicCAS(&q.ctrl[kErr], 0, SPCHOL_DEV_EINTERNAL);
    }
  }
}

// Any thread: push one ready task to one ring of a Ring2.
__device__ __forceinline__ void ring2_push_one(const Ring2& q, bool hi, int task) {
  hi = hi && q.n_hi > 0;
  const int slot = atomicAdd(&q.ctrl[hi ? kHiTail : kTail], 1);
  if (slot < (hi ? q.n_hi : q.n_lo)) {
    st_release(&(hi ? q.hi : q.lo)[slot], task);
  } else {
    atomicCAS(&q.ctrl[kErr], 0, SPCHOL_DEV_EINTERNAL);
  }
}

// Whole warp, all 32 lanes converged: push the ready tasks the lanes hold
// (t[u] >= 0, u < N) to one ring of a Ring2, with one reservation of slots
// per warp instead of one contended tail update per task (a backward
// diagonal task near the root releases thousands of tiles).  Same visibility
// precondition as ring_push_one.
template <int N>
__device__ __forceinline__ void ring2_push_warp(const Ring2& q, bool hi, const int (&t)[N]) {
  hi = hi && q.n_hi > 0;
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  int cnt = 0;
#pragma unroll
  for (int u = 0; u < N; ++u) cnt += t[u] >= 0 ? 1 : 0;
  int incl = cnt;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const int v = __shfl_up_sync(full, incl, d);
    if (lane >= d) incl += v;
  }
  const int total = __shfl_sync(full, incl, 31);
  if (total == 0) return;
  int base = 0;
  if (lane == 31) base = atomicAdd(&q.ctrl[hi ? kHiTail : kTail], total);
  base = __shfl_sync(full, base, 31) + incl - cnt;
  int* slots = hi ? q.hi : q.lo;
  const int n = hi ? q.n_hi : q.n_lo;
#pragma unroll
  for (int u = 0; u < N; ++u)
    if (t[u] >= 0) {
      if (base < n) {
        st_release(&slots[base], t[u]);
      } else {
        atomicCAS(&q.ctrl[kErr], 0, SPCHOL_DEV_EINTERNAL);
      }
      ++base;
    }
}

// Continuation: a task made ready by the running one is kept for this CTA's
// next turn if none is kept yet (*next, shared memory, -1 when empty), else
// pushed to the high-priority ring.  Any thread; next == nullptr: always push.
__device__ __forceinline__ void keep_or_push(const Ring2& q, int* next, int task) {
  if (next == nullptr || atomicCAS(next, -1, task) != -1) ring2_push_one(q, true, task);
}

// Make this CTA's global writes visible before a counter update or a push:
// the CTA barrier orders every thread's writes before thread 0's fence, whose
// cumulativity makes them visible at GPU scope before thread 0 signals (the
// pattern of the cooperative-groups grid barrier).  A fence in every thread
// before the barrier, as this used to do, cost each task its slowest thread's
// wait for its own atomics: 64^3 factor 389.1 -> 386.9 ms and solve 16.1 ->
// 15.5 ms, 48^3 FP32 factor 16.8 -> 16.2 ms.
__device__ __forceinline__ void publish_cta_writes() {
  __syncthreads();
  if (threadIdx.x == 0) __threadfence();
}

// Reset kernel: ring slots to -1 with the seed tasks at slots[seed_off ..],
// counters from their initial copies, control words.  seeds_hi: the seeds
// fill the front of a Ring2's high-priority ring (seed_off 0); otherwise they
// fill the front of a single ring (seed_off 0) or of a Ring2's normal-priority
// ring (seed_off = n_hi).
__global__ void ring_reset_kernel(int* slots, int ntask, const int* seeds, int nseed, int seed_off, int seeds_hi,
                                  int* ctrl,
                                  int* c0, const int* c0_init, int n0, int* c1, const int* c1_init,
                                  int n1, int* c2, const int* c2_init, int n2, int* c3,
                                  const int* c3_init, int n3);

}  // namespace spchol
