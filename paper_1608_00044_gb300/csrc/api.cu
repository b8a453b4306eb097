// C-ABI of the library: handle lifetime, device storage, and the
// analyze -> factorize -> solve sequence (see include/spchol.h).
#include <algorithm>
#include <chrono>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <type_traits>
#include <unordered_map>
#include <vector>

#include <cuda.h>  // CUtensorMap and its encoder's signature (called through the runtime's driver entry point)
#include <cuda_runtime.h>

#include "../../include/spchol.h"
#include "device_common.cuh"
#include "kernels.hpp"
#include "options.hpp"
#include "plan.hpp"

using namespace spchol;

namespace {

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

// One device allocation carved into 256-byte aligned pieces.
struct Arena {
  size_t bytes = 0;
  char* base = nullptr;
  size_t reserve(size_t n) {
    size_t off = bytes;
    bytes += (n + 255) & ~size_t(255);
    return off;
  }
};

}  // namespace

struct spchol_handle_s {
  Plan plan;
  spchol_options opt{};
  spchol_stats stats{};
  int device = 0;
  int num_sms = 0;
  bool fp32 = false;
  bool factored = false;
  bool pending = false;  // a factorization was enqueued without a status read
  std::vector<int32_t> a_row, a_col;  // A's lower entries (original order); dropped after analyze
  int batch_count = 0;                // 0 = single matrix
  std::vector<int64_t> batch_n, batch_col0, batch_nnz0;  // per matrix: order, first column, first value
  // device structures
  Arena arena;
  int32_t *d_fcol = nullptr, *d_nrows = nullptr, *d_ld = nullptr, *d_rows = nullptr, *d_parent = nullptr;
  int64_t *d_rowoff = nullptr, *d_valoff = nullptr, *d_adest = nullptr;
  int32_t *d_trsm_first = nullptr, *d_ntrsm = nullptr, *d_trsm_sn = nullptr, *d_u_first = nullptr, *d_nu = nullptr;
  int32_t* d_nu_hi = nullptr;
  int32_t *d_sub_lo = nullptr, *d_sub_hi = nullptr;  // subtree tasks' panel ranges
  int32_t* d_relpos = nullptr;  // relative row indices of the update tiles
  unsigned char* d_tmaps = nullptr;  // TMA tensor maps, one per panel (null: operands staged by cp.async)
  int32_t* d_trsm_rows = nullptr;
  UTask* d_ut = nullptr;
  int32_t *d_dep_init = nullptr, *d_trsm_init = nullptr, *d_dep = nullptr, *d_trsm_left = nullptr;
  int32_t *d_fseeds = nullptr;
  int nfseeds = 0;
  int32_t* d_wsub = nullptr;  // subtree tasks run by single warps (Plan::wsub), when used
  int n_wsub = 0, grid_wsub = 0;  // the factorization's warp subtrees (0: none)
  int n_wsub_solve = 0;            // the solves' (0: none)
  int solve_done = 0;  // SolveArgs::ntask_done
  int32_t *d_st_first = nullptr, *d_nst = nullptr, *d_st_sn = nullptr, *d_st_rows = nullptr, *d_kid_ptr = nullptr, *d_kids = nullptr;
  int32_t *d_nkids_init = nullptr, *d_fkids = nullptr, *d_ftiles = nullptr, *d_btiles = nullptr;
  int32_t *d_st_tptr = nullptr, *d_st_tgt = nullptr, *d_rt_ptr = nullptr, *d_rt_tile = nullptr;
  int32_t *d_fdep0 = nullptr, *d_bdep0 = nullptr, *d_bdep = nullptr;
  // deterministic order (options.deterministic): the chains of Plan::u_next and
  // Plan::ft_sptr, their initial counters and the live counters
  int32_t *d_u_next = nullptr, *d_u_dep0 = nullptr, *d_u_dep = nullptr;
  int32_t *d_ft_sptr = nullptr, *d_ft_succ = nullptr, *d_ft_dep0 = nullptr, *d_ftdep = nullptr;
  // fan-in mode (options.deterministic = 2): Plan::fan_* and the update
  // tiles' private buffers (a separate allocation, in the panels' type)
  int64_t *d_fan_off = nullptr, *d_fan_ptr = nullptr;
  int32_t* d_fan_task = nullptr;
  FanEnt* d_fan_ent = nullptr;
  FanRec* d_fan_rec = nullptr;  // the gather's records (a separate allocation)
  // fan-in solves: Plan::st_zf and friends, and the tiles' buffers for up to
  // fan_nrhs right-hand sides
  int64_t *d_st_zf = nullptr, *d_st_zb = nullptr;
  // fan-in gather tasks: Plan::gat_first and friends, and the live counters
  int32_t *d_gat_first = nullptr, *d_gat_pc = nullptr, *d_pc_owner = nullptr, *d_gdiag0 = nullptr,
          *d_tdep0 = nullptr, *d_gdiag = nullptr, *d_tdep = nullptr;
  Plan::SolveFanRec* d_rt_rec = nullptr;
  double *d_zf = nullptr, *d_zb = nullptr;
  int fan_nrhs = 0;
  void* d_fan_buf = nullptr;
  size_t fan_buf_bytes = 0;
  int fan_cap = 0;
  int32_t *d_sseeds = nullptr;
  int nsseeds = 0;
  int32_t* d_perm = nullptr;
  int* d_ring = nullptr;
  int* d_ctrl = nullptr;
  double* d_vals = nullptr;  // staging for host values
  // value pool and solve workspace (separate allocations)
  void* d_pool = nullptr;
  size_t pool_bytes = 0;
  double* d_inv = nullptr;  // diagonal-block inverses (FP64)
  void* d_wbuf = nullptr;   // W = L21 L11^{-1} of the W panels (Plan::woff), in the panels' precision
  int64_t* d_woff = nullptr;
  uint16_t* d_slices = nullptr;  // FP64_TC: BF16 digit slices of the rows below each diagonal block
  int32_t* d_rexp = nullptr;     // FP64_TC: row exponents
  int64_t* d_sliceoff = nullptr;
  int64_t* d_invoff = nullptr;
  double* d_Y = nullptr;
  double* d_B = nullptr;
  int64_t y_cap = 0;  // capacity in doubles of d_Y and d_B
  // mixed precision: full symmetric CSR of A (original order) for the FP64 residual
  int64_t* d_csr_rp = nullptr;
  int32_t* d_csr_ci = nullptr;
  int64_t* d_csr_vmap = nullptr;
  unsigned long long* d_norms = nullptr;  // [0] = ||A||_inf, then 3 per right-hand side
  unsigned long long* h_norms = nullptr;  // pinned
  int norms_cap = 0;                      // right-hand sides the norm buffers hold
  double* d_X = nullptr;
  double* d_R = nullptr;
  // GMRES-IR workspace (allocated at its first use): Krylov basis (n x
  // (kGmresRestart + 1)), one work vector, reduction partials, Hessenberg
  // column buffers on the device and in pinned host memory
  double* d_gmV = nullptr;
  double* d_gmW = nullptr;
  double* d_gmPart = nullptr;
  double* d_gmH = nullptr;
  double* h_gmH = nullptr;
  unsigned long long* d_prof = nullptr;  // [0..9] factorization, [16..23] solve
  unsigned long long* d_trace_f = nullptr;  // profile = 2: per factorization task start/end
  unsigned long long* d_trace_s = nullptr;  // profile = 2: per solve task start/end
  bool traced_f = false, traced_s = false;
  unsigned long long* h_prof = nullptr;
  int* h_ctrl = nullptr;  // pinned
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  size_t smem_factor = 0, smem_solve = 0;
  int grid_factor = 0, grid_solve = 0;
  // sizes of the live device allocations (the caller's dev_free takes the size)
  std::unordered_map<void*, size_t> dev_bytes;
  // pinned host blocks (recycled through the process-wide cache) and their sizes
  size_t h_norms_bytes = 0;
};

namespace {

// Text of the last failing CUDA call of this host thread (spchol_last_cuda_error).
thread_local char g_cuda_err[256] = "";

inline int cuda_fail(cudaError_t e, const char* what, int line) {
  snprintf(g_cuda_err, sizeof(g_cuda_err), "%s (%d) at api.cu:%d in %s", cudaGetErrorName(e), (int)e, line, what);
  return e == cudaErrorMemoryAllocation ? SPCHOL_ENOMEM : SPCHOL_ECUDA;
}

#define CU(x)                                                 \
  do {                                                        \
    cudaError_t e_ = (x);                                     \
    if (e_ != cudaSuccess) return cuda_fail(e_, #x, __LINE__); \
  } while (0)

// A non-sticky error left in this thread's CUDA error slot by another library
// must not be reported as the failure of our next launch.
inline void clear_stale_error() { (void)cudaGetLastError(); }

// Structure uploads go through a private non-blocking stream so that analyze
// never orders itself behind work that other threads run on other streams.
thread_local cudaStream_t g_upload_stream = nullptr;

// ---- device memory of a handle
// Through the caller's allocator (spchol_options.dev_alloc / dev_free), else
// stream-ordered from the device's default memory pool.  cudaFree waits for
// the whole device, so one handle's release or workspace growth would stall
// every other stream's persistent kernel; cudaFreeAsync does not.  Every
// release happens when the library has no pending work on the memory (its
// calls synchronise their stream before returning), so the stream a block is
// released on only orders the release itself.
bool pools_supported(int dev) {
  static std::mutex mu;
  static std::map<int, bool> known;
  std::lock_guard<std::mutex> lock(mu);
  auto it = known.find(dev);
  if (it != known.end()) return it->second;
  int v = 0;
  if (cudaDeviceGetAttribute(&v, cudaDevAttrMemoryPoolsSupported, dev) != cudaSuccess) {
    cudaGetLastError();
    v = 0;
  }
  known[dev] = v != 0;
  return v != 0;
}

// One non-blocking stream per device on which spchol_destroy releases memory.
cudaStream_t release_stream(int dev) {
  static std::mutex mu;
  static std::map<int, cudaStream_t> streams;
  std::lock_guard<std::mutex> lock(mu);
  auto it = streams.find(dev);
  if (it != streams.end()) return it->second;
  cudaStream_t st = nullptr;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    st = nullptr;  // the legacy stream, which orders the release after prior work
  }
  streams[dev] = st;
  return st;
}

// stream: where the memory is first used (nullptr: analyze, any stream after it
// returns; the pool path then allocates on the upload stream, synchronised
// before analyze returns).
int dalloc_impl(spchol_handle_t h, void** out, size_t bytes, cudaStream_t stream, const char* what, int line) {
  *out = nullptr;
  bytes = std::max<size_t>((bytes + 255) & ~size_t(255), 256);
  void* p = nullptr;
  if (h->opt.dev_alloc) {
    p = h->opt.dev_alloc(bytes, (void*)stream, h->opt.alloc_ctx);
    if (!p || ((uintptr_t)p & 255) != 0) {
      if (p) h->opt.dev_free(p, bytes, (void*)stream, h->opt.alloc_ctx);
      snprintf(g_cuda_err, sizeof(g_cuda_err), "dev_alloc %s %zu bytes at api.cu:%d for %s",
               p ? "returned memory not 256-byte aligned for" : "returned NULL for", bytes, line, what);
      return SPCHOL_ENOMEM;
    }
  } else if (pools_supported(h->device)) {
    cudaError_t e = cudaMallocAsync(&p, bytes, stream ? stream : g_upload_stream);
    if (e != cudaSuccess) return cuda_fail(e, what, line);
  } else {
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) return cuda_fail(e, what, line);
  }
  h->dev_bytes[p] = bytes;
  *out = p;
  return 0;
}

void dfree(spchol_handle_t h, void* p, cudaStream_t stream) {
  if (!p) return;
  auto it = h->dev_bytes.find(p);
  const size_t bytes = it != h->dev_bytes.end() ? it->second : 0;
  if (it != h->dev_bytes.end()) h->dev_bytes.erase(it);
  if (h->opt.dev_free) {
    h->opt.dev_free(p, bytes, (void*)stream, h->opt.alloc_ctx);
  } else if (pools_supported(h->device)) {
    if (cudaFreeAsync(p, stream ? stream : release_stream(h->device)) != cudaSuccess) cudaGetLastError();
  } else {
    cudaFree(p);
  }
}

#define DALLOC(ptr, bytes, stream)                                                                       \
  do {                                                                                                   \
    void* p_ = nullptr;                                                                                  \
    int rc_ = dalloc_impl(h, &p_, (bytes), (stream), #ptr, __LINE__);                                    \
    if (rc_) return rc_;                                                                                 \
    (ptr) = reinterpret_cast<std::remove_reference<decltype(ptr)>::type>(p_);                            \
  } while (0)

// ---- pinned host blocks (status words, small read-backs), recycled for the
// life of the process: cudaFreeHost may wait for the device, which would stall
// other streams' work whenever a handle is destroyed.  Size classes are powers
// of two from 256 bytes.
std::mutex g_pinned_mu;
std::map<size_t, std::vector<void*>> g_pinned_free;

size_t pinned_class(size_t bytes) {
  size_t c = 256;
  while (c < bytes) c <<= 1;
  return c;
}

int pinned_get(void** out, size_t bytes, int line) {
  const size_t c = pinned_class(bytes);
  {
    std::lock_guard<std::mutex> lock(g_pinned_mu);
    auto& v = g_pinned_free[c];
    if (!v.empty()) {
      *out = v.back();
      v.pop_back();
      return 0;
    }
  }
  cudaError_t e = cudaHostAlloc(out, c, cudaHostAllocPortable);
  if (e != cudaSuccess) return cuda_fail(e, "cudaHostAlloc", line);
  return 0;
}

void pinned_put(void* p, size_t bytes) {
  if (!p) return;
  std::lock_guard<std::mutex> lock(g_pinned_mu);
  g_pinned_free[pinned_class(bytes)].push_back(p);
}

#define PINNED(ptr, bytes)                                            \
  do {                                                                \
    void* p_ = nullptr;                                               \
    int rc_ = pinned_get(&p_, (bytes), __LINE__);                     \
    if (rc_) return rc_;                                              \
    (ptr) = reinterpret_cast<std::remove_reference<decltype(ptr)>::type>(p_); \
  } while (0)

constexpr size_t kProfWords = 24;

template <typename V>
int upload(spchol_handle_t h, V* dst, const std::vector<V>& src) {
  (void)h;
  if (src.empty()) return 0;
  CU(cudaMemcpyAsync(dst, src.data(), src.size() * sizeof(V), cudaMemcpyHostToDevice, g_upload_stream));
  return 0;
}

int mma_mode_of(int precision) {
  return precision == SPCHOL_TF32 ? 1 : precision == SPCHOL_TF32X3 ? 2 : precision == SPCHOL_FP64_TC ? 3 : 0;
}

// One TMA tensor map per panel: the column-major panel as a 2-D tensor of
// ld rows x w columns (row stride ld elements), box kUpdBoxRows x kUpdKC,
// zero fill outside.  The encoder is a driver function, reached through the
// runtime's entry-point query.  Returns false (and the update tiles stage
// their operands with cp.async) if it is unavailable or rejects a panel.
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

bool build_tensor_maps(spchol_handle_t h, std::vector<CUtensorMap>& maps) {
  static EncodeTiledFn encode = [] {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      fn = nullptr;
    cudaGetLastError();
    return reinterpret_cast<EncodeTiledFn>(fn);
  }();
  if (!encode) return false;
  const Plan& P = h->plan;
  const size_t esz = h->fp32 ? sizeof(float) : sizeof(double);
  const CUtensorMapDataType dt = h->fp32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64;
  maps.resize(P.ns);
  for (int32_t s = 0; s < P.ns; ++s) {
    const int w = P.fcol[s + 1] - P.fcol[s];
    const cuuint64_t dims[2] = {(cuuint64_t)P.ld[s], (cuuint64_t)w};
    const cuuint64_t strides[1] = {(cuuint64_t)P.ld[s] * esz};
    const cuuint32_t box[2] = {(cuuint32_t)kUpdBoxRows((int)esz), (cuuint32_t)kUpdKC};
    const cuuint32_t estr[2] = {1, 1};
    void* base = static_cast<unsigned char*>(h->d_pool) + (size_t)P.valoff[s] * esz;
    if (encode(&maps[s], dt, 2, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return false;
  }
  return true;
}

int setup_device(spchol_handle_t h) {
  Plan& P = h->plan;
  const int ns = P.ns;
  Arena& A = h->arena;
  auto r32 = [&](size_t n) { return A.reserve(std::max<size_t>(n, 1) * sizeof(int32_t)); };
  auto r64 = [&](size_t n) { return A.reserve(std::max<size_t>(n, 1) * sizeof(int64_t)); };
  size_t o_fcol = r32(ns + 1), o_nrows = r32(ns), o_ld = r32(ns), o_rows = r32(P.rows.size()), o_parent = r32(ns);
  size_t o_rowoff = r64(ns + 1), o_valoff = r64(ns + 1), o_adest = r64(P.a_dest.size()), o_invoff = r64(ns + 1);
  size_t o_woff = r64(ns);
  const bool oz = h->opt.precision == SPCHOL_FP64_TC;
  size_t o_sliceoff = r64(ns + 1), o_rexp = oz ? r32(P.rows.size()) : 0;
  size_t o_tf = r32(ns), o_nt = r32(ns), o_tsn = r32(P.trsm_sn.size()), o_uf = r32(ns), o_nu = r32(ns);
  size_t o_trows = r32(ns), o_nuhi = r32(ns), o_sublo = r32(P.sub_lo.size()), o_subhi = r32(P.sub_hi.size());
  size_t o_ut = A.reserve(std::max<size_t>(P.ut.size(), 1) * sizeof(UTask));
  size_t o_depi = r32(ns), o_trsi = r32(ns), o_dep = r32(ns), o_trs = r32(ns);
  // seeds: every subtree task, and the panels outside subtrees with no
  // incoming update
  std::vector<int32_t> fseeds;
  // the subtree tasks run by single warps (FP64 DFMA mode) in a launch of
  // their own before the task loop, when every subtree task qualifies and the
  // subtrees hold a good part of the work (a batch of small matrices: 30-47 %;
  // a single large matrix: under 6 %, where the launch ahead of the task loop
  // costs more than the warps gain; with some subtree tasks left to the CTAs
  // the task loop would wait for that launch and then run them)
  const bool warp_sub = mma_mode_of(h->opt.precision) == 0 && !P.params.fanin && P.n_sub > 0 &&
                        (int32_t)P.wsub.size() == P.n_sub && P.sub_work_frac >= 0.2 &&
                        h->opt.fault_inject == 0;
  std::vector<char> by_warp(P.n_sub, 0);
  if (warp_sub)
    for (int32_t k : P.wsub) by_warp[k] = 1;
  // the solves take the same subtrees on single warps under the same
  // condition.  (Whenever the subtrees qualify, whatever their share of the
  // work, was measured too: 48^3 diffusion, one right-hand side, 4.2 -> 3.8
  // ms, but 40^3 with eight 4.5 -> 6.1 ms: a large subtree's solve on one warp
  // then holds the task loop back.)
  const bool warp_solve = warp_sub;
  for (int32_t k = 0; k < P.n_sub; ++k)
    if (!by_warp[k]) fseeds.push_back(ns + P.n_trsm + P.n_u + k);
  for (int s = 0; s < ns; ++s)
    if (P.dep_f[s] == 0 && P.in_sub[s] < 0) fseeds.push_back(s);
  if (h->opt.fault_inject == 1 && ns > 0 && P.in_sub[ns - 1] >= 0) {
    // fault injection when the root belongs to a subtree task: that task is
    // never released (its seed is withheld), so the run must time out
    const int32_t missing = ns + P.n_trsm + P.n_u + P.in_sub[ns - 1];
    fseeds.erase(std::find(fseeds.begin(), fseeds.end(), missing));
  }
  size_t o_fseeds = r32(fseeds.size()), o_wsub = r32(warp_sub || warp_solve ? P.wsub.size() : 0);
  size_t o_stf = r32(ns), o_nst = r32(ns), o_strows = r32(ns), o_stsn = r32(P.st_sn.size()), o_kp = r32(ns + 1), o_k = r32(P.kids.size());
  // the panels of the warp subtrees: solved by the subtree solve launches, so
  // none of their tasks is seeded, and their backward tiles' counters start
  // out of reach of the task loop
  std::vector<char> in_wsub(ns, 0);
  std::vector<int32_t> bdep0 = P.bdep0;
  int64_t sub_tasks = 0;
  if (warp_solve)
    for (int32_t k : P.wsub)
      for (int32_t q = P.sub_lo[k]; q <= P.sub_hi[k]; ++q) {
        in_wsub[q] = 1;
        sub_tasks += 2 + 2 * (int64_t)P.nst[q];
        for (int32_t kt = P.st_first[q]; kt < P.st_first[q] + P.nst[q]; ++kt) bdep0[kt] = 1 << 30;
      }
  h->solve_done = (int)((int64_t)P.n_solve_tasks - P.n_wpan - sub_tasks + (warp_solve ? (int64_t)P.wsub.size() : 0));
  std::vector<int32_t> nkids(ns, 0), sseeds;
  for (int s = 0; s < ns; ++s) {
    nkids[s] = P.kid_ptr[s + 1] - P.kid_ptr[s];
    if (P.fdep0[s] == 0 && !in_wsub[s]) {
      if (P.woff[s] >= 0)  // a W panel starts with its forward tiles
        for (int k = 0; k < P.nst[s]; ++k) sseeds.push_back(ns + P.st_first[s] + k);
      else
        sseeds.push_back(s);
    }
  }
  size_t o_sttp = r32(P.st_tptr.size()), o_sttg = r32(P.st_tgt.size()), o_rtp = r32(P.rt_ptr.size()),
         o_rtt = r32(P.rt_tile.size()), o_fd0 = r32(ns), o_bd0 = r32(P.n_st), o_bd = r32(P.n_st);
  size_t o_nki = r32(ns), o_fk = r32(ns), o_ft = r32(ns), o_bt = r32(ns), o_sseeds = r32(sseeds.size());
  size_t o_perm = r32(P.n);
  const bool det = P.params.deterministic;
  size_t o_unx = det ? r32(P.u_next.size()) : 0, o_ud0 = det ? r32(P.u_dep0.size()) : 0,
         o_ud = det ? r32(P.u_dep0.size()) : 0, o_fsp = det ? r32(P.ft_sptr.size()) : 0,
         o_fsu = det ? r32(P.ft_succ.size()) : 0, o_fd0d = det ? r32(P.ft_dep0.size()) : 0,
         o_fdd = det ? r32(P.ft_dep0.size()) : 0;
  const bool fan = P.params.fanin;
  size_t o_fano = fan ? r64(P.fan_off.size()) : 0, o_fant = fan ? r32(P.fan_task.size()) : 0,
         o_fanp = fan ? r64(P.fan_ptr.size()) : 0,
         o_fane = fan ? A.reserve(std::max<size_t>(P.fan_ent.size(), 1) * sizeof(FanEnt)) : 0,
         o_stzf = fan ? r64(P.st_zf.size()) : 0, o_stzb = fan ? r64(P.st_zb.size()) : 0,
         o_rtrec = fan ? A.reserve(std::max<size_t>(P.rt_rec.size(), 1) * sizeof(Plan::SolveFanRec)) : 0,
         o_gatf = fan ? r32(P.gat_first.size()) : 0, o_gatp = fan ? r32(P.gat_pc.size()) : 0,
         o_pco = fan ? r32(P.pc_owner.size()) : 0, o_gd0 = fan ? r32(P.gdiag0.size()) : 0,
         o_td0 = fan ? r32(P.tdep0.size()) : 0, o_gd = fan ? r32(P.gdiag0.size()) : 0,
         o_td = fan ? r32(P.tdep0.size()) : 0;
  const int ring_n = std::max(P.n_factor_tasks, P.n_solve_tasks);
  size_t o_ring = r32(ring_n), o_ctrl = r32(kCtrlWords);
  size_t o_prof = A.reserve(24 * sizeof(unsigned long long));
  size_t o_vals = A.reserve(std::max<int64_t>(P.nnz_a, 1) * sizeof(double));
  // full symmetric CSR of A for the refinement residual (mixed precision only)
  std::vector<int64_t> crp, cvm;
  std::vector<int32_t> cci;
  size_t o_crp = 0, o_cci = 0, o_cvm = 0;
  if (h->fp32) {
    const int64_t n = P.n;
    crp.assign(n + 1, 0);
    for (int64_t e = 0; e < P.nnz_a; ++e) {
      crp[h->a_row[e] + 1]++;
      if (h->a_row[e] != h->a_col[e]) crp[h->a_col[e] + 1]++;
    }
    for (int64_t i = 0; i < n; ++i) crp[i + 1] += crp[i];
    cci.resize(crp[n]);
    cvm.resize(crp[n]);
    std::vector<int64_t> fill(crp.begin(), crp.end() - 1);
    for (int64_t e = 0; e < P.nnz_a; ++e) {
      const int64_t i = h->a_row[e], j = h->a_col[e];
      cci[fill[i]] = (int32_t)j;
      cvm[fill[i]++] = e;
      if (i != j) {
        cci[fill[j]] = (int32_t)i;
        cvm[fill[j]++] = e;
      }
    }
    o_crp = r64(crp.size());
    o_cci = r32(cci.size());
    o_cvm = r64(cvm.size());
  }
  CU(cudaStreamCreateWithFlags(&g_upload_stream, cudaStreamNonBlocking));
  struct StreamGuard {
    ~StreamGuard() {
      if (g_upload_stream) {
        cudaStreamSynchronize(g_upload_stream);
        cudaStreamDestroy(g_upload_stream);
        g_upload_stream = nullptr;
      }
    }
  } upload_guard;
  DALLOC(A.base, A.bytes, nullptr);
  char* b = A.base;
  h->d_fcol = (int32_t*)(b + o_fcol);
  h->d_nrows = (int32_t*)(b + o_nrows);
  h->d_ld = (int32_t*)(b + o_ld);
  h->d_rows = (int32_t*)(b + o_rows);
  h->d_parent = (int32_t*)(b + o_parent);
  h->d_rowoff = (int64_t*)(b + o_rowoff);
  h->d_valoff = (int64_t*)(b + o_valoff);
  h->d_adest = (int64_t*)(b + o_adest);
  h->d_invoff = (int64_t*)(b + o_invoff);
  h->d_woff = (int64_t*)(b + o_woff);
  h->d_sliceoff = (int64_t*)(b + o_sliceoff);
  if (oz) h->d_rexp = (int32_t*)(b + o_rexp);
  h->d_trsm_first = (int32_t*)(b + o_tf);
  h->d_ntrsm = (int32_t*)(b + o_nt);
  h->d_trsm_sn = (int32_t*)(b + o_tsn);
  h->d_trsm_rows = (int32_t*)(b + o_trows);
  h->d_u_first = (int32_t*)(b + o_uf);
  h->d_nu = (int32_t*)(b + o_nu);
  h->d_nu_hi = (int32_t*)(b + o_nuhi);
  h->d_sub_lo = (int32_t*)(b + o_sublo);
  h->d_sub_hi = (int32_t*)(b + o_subhi);
  h->d_ut = (UTask*)(b + o_ut);
  h->d_dep_init = (int32_t*)(b + o_depi);
  h->d_trsm_init = (int32_t*)(b + o_trsi);
  h->d_dep = (int32_t*)(b + o_dep);
  h->d_trsm_left = (int32_t*)(b + o_trs);
  h->d_fseeds = (int32_t*)(b + o_fseeds);
  h->nfseeds = (int)fseeds.size();
  h->d_wsub = (int32_t*)(b + o_wsub);
  h->n_wsub = warp_sub ? (int)P.wsub.size() : 0;
  h->n_wsub_solve = warp_solve ? (int)P.wsub.size() : 0;
  h->d_st_first = (int32_t*)(b + o_stf);
  h->d_nst = (int32_t*)(b + o_nst);
  h->d_st_sn = (int32_t*)(b + o_stsn);
  h->d_st_rows = (int32_t*)(b + o_strows);
  h->d_kid_ptr = (int32_t*)(b + o_kp);
  h->d_kids = (int32_t*)(b + o_k);
  h->d_nkids_init = (int32_t*)(b + o_nki);
  h->d_fkids = (int32_t*)(b + o_fk);
  h->d_ftiles = (int32_t*)(b + o_ft);
  h->d_btiles = (int32_t*)(b + o_bt);
  h->d_sseeds = (int32_t*)(b + o_sseeds);
  h->d_st_tptr = (int32_t*)(b + o_sttp);
  h->d_st_tgt = (int32_t*)(b + o_sttg);
  h->d_rt_ptr = (int32_t*)(b + o_rtp);
  h->d_rt_tile = (int32_t*)(b + o_rtt);
  h->d_fdep0 = (int32_t*)(b + o_fd0);
  h->d_bdep0 = (int32_t*)(b + o_bd0);
  h->d_bdep = (int32_t*)(b + o_bd);
  h->nsseeds = (int)sseeds.size();
  if (det) {
    h->d_u_next = (int32_t*)(b + o_unx);
    h->d_u_dep0 = (int32_t*)(b + o_ud0);
    h->d_u_dep = (int32_t*)(b + o_ud);
    h->d_ft_sptr = (int32_t*)(b + o_fsp);
    h->d_ft_succ = (int32_t*)(b + o_fsu);
    h->d_ft_dep0 = (int32_t*)(b + o_fd0d);
    h->d_ftdep = (int32_t*)(b + o_fdd);
  }
  if (fan) {
    h->d_fan_off = (int64_t*)(b + o_fano);
    h->d_fan_task = (int32_t*)(b + o_fant);
    h->d_fan_ptr = (int64_t*)(b + o_fanp);
    h->d_fan_ent = (FanEnt*)(b + o_fane);
    h->d_st_zf = (int64_t*)(b + o_stzf);
    h->d_st_zb = (int64_t*)(b + o_stzb);
    h->d_rt_rec = (Plan::SolveFanRec*)(b + o_rtrec);
    h->d_gat_first = (int32_t*)(b + o_gatf);
    h->d_gat_pc = (int32_t*)(b + o_gatp);
    h->d_pc_owner = (int32_t*)(b + o_pco);
    h->d_gdiag0 = (int32_t*)(b + o_gd0);
    h->d_tdep0 = (int32_t*)(b + o_td0);
    h->d_gdiag = (int32_t*)(b + o_gd);
    h->d_tdep = (int32_t*)(b + o_td);
  }
  h->d_perm = (int32_t*)(b + o_perm);
  h->d_ring = (int*)(b + o_ring);
  h->d_ctrl = (int*)(b + o_ctrl);
  h->d_prof = (unsigned long long*)(b + o_prof);
  h->d_vals = (double*)(b + o_vals);
  if (h->fp32) {
    h->d_csr_rp = (int64_t*)(b + o_crp);
    h->d_csr_ci = (int32_t*)(b + o_cci);
    h->d_csr_vmap = (int64_t*)(b + o_cvm);
  }
  int rc = 0;
  if (h->fp32 && ((rc = upload(h, h->d_csr_rp, crp)) || (rc = upload(h, h->d_csr_ci, cci)) ||
                  (rc = upload(h, h->d_csr_vmap, cvm))))
    return rc;
  std::vector<int32_t>().swap(h->a_row);
  std::vector<int32_t>().swap(h->a_col);
  std::vector<int32_t> perm32(P.perm.begin(), P.perm.end());
  if ((rc = upload(h, h->d_fcol, P.fcol)) || (rc = upload(h, h->d_nrows, P.nrows)) ||
      (rc = upload(h, h->d_ld, P.ld)) || (rc = upload(h, h->d_rows, P.rows)) ||
      (rc = upload(h, h->d_parent, P.parent)) || (rc = upload(h, h->d_rowoff, P.rowoff)) ||
      (rc = upload(h, h->d_valoff, P.valoff)) || (rc = upload(h, h->d_adest, P.a_dest)) ||
      (rc = upload(h, h->d_invoff, P.invoff)) || (rc = upload(h, h->d_sliceoff, P.sliceoff)) ||
      (rc = upload(h, h->d_woff, P.woff)) ||
      (rc = upload(h, h->d_trsm_first, P.trsm_first)) || (rc = upload(h, h->d_ntrsm, P.ntrsm)) ||
      (rc = upload(h, h->d_trsm_sn, P.trsm_sn)) || (rc = upload(h, h->d_u_first, P.u_first)) ||
      (rc = upload(h, h->d_trsm_rows, P.trsm_rows)) ||
      (rc = upload(h, h->d_nu, P.nu)) || (rc = upload(h, h->d_nu_hi, P.nu_hi)) ||
      (rc = upload(h, h->d_sub_lo, P.sub_lo)) || (rc = upload(h, h->d_sub_hi, P.sub_hi)) || (rc = upload(h, h->d_ut, P.ut)) ||
      (rc = upload(h, h->d_dep_init, P.dep_f)) || (rc = upload(h, h->d_trsm_init, P.ntrsm)) ||
      (rc = upload(h, h->d_fseeds, fseeds)) || (rc = upload(h, h->d_st_first, P.st_first)) ||
      ((warp_sub || warp_solve) && (rc = upload(h, h->d_wsub, P.wsub))) ||
      (rc = upload(h, h->d_nst, P.nst)) || (rc = upload(h, h->d_st_sn, P.st_sn)) ||
      (rc = upload(h, h->d_st_rows, P.st_rows)) ||
      (rc = upload(h, h->d_kid_ptr, P.kid_ptr)) || (rc = upload(h, h->d_kids, P.kids)) ||
      (rc = upload(h, h->d_nkids_init, nkids)) || (rc = upload(h, h->d_sseeds, sseeds)) ||
      (rc = upload(h, h->d_st_tptr, P.st_tptr)) || (rc = upload(h, h->d_st_tgt, P.st_tgt)) ||
      (rc = upload(h, h->d_rt_ptr, P.rt_ptr)) || (rc = upload(h, h->d_rt_tile, P.rt_tile)) ||
      (rc = upload(h, h->d_fdep0, P.fdep0)) || (rc = upload(h, h->d_bdep0, bdep0)) ||
      (rc = upload(h, h->d_perm, perm32)))
    return rc;
  if (det && ((rc = upload(h, h->d_u_next, P.u_next)) || (rc = upload(h, h->d_u_dep0, P.u_dep0)) ||
              (rc = upload(h, h->d_ft_sptr, P.ft_sptr)) || (rc = upload(h, h->d_ft_succ, P.ft_succ)) ||
              (rc = upload(h, h->d_ft_dep0, P.ft_dep0))))
    return rc;
  if (fan && ((rc = upload(h, h->d_fan_off, P.fan_off)) || (rc = upload(h, h->d_fan_task, P.fan_task)) ||
              (rc = upload(h, h->d_fan_ptr, P.fan_ptr)) || (rc = upload(h, h->d_fan_ent, P.fan_ent)) ||
              (rc = upload(h, h->d_st_zf, P.st_zf)) || (rc = upload(h, h->d_st_zb, P.st_zb)) ||
              (rc = upload(h, h->d_gat_first, P.gat_first)) || (rc = upload(h, h->d_gat_pc, P.gat_pc)) ||
              (rc = upload(h, h->d_pc_owner, P.pc_owner)) || (rc = upload(h, h->d_gdiag0, P.gdiag0)) ||
              (rc = upload(h, h->d_tdep0, P.tdep0)) || (rc = upload(h, h->d_rt_rec, P.rt_rec))))
    return rc;
  const size_t esz = h->fp32 ? sizeof(float) : sizeof(double);
  if (fan) {  // never read before written: no initialisation
    // + 16 bytes: the gather copies whole 16-byte pieces, up to one past the last value
    h->fan_buf_bytes = std::max<size_t>((((size_t)P.fan_off.back() * esz + 15) & ~size_t(15)) + 16, 256);
    DALLOC(h->d_fan_buf, h->fan_buf_bytes, nullptr);
    DALLOC(h->d_fan_rec, std::max<size_t>(P.fan_ent.size(), 1) * sizeof(FanRec), nullptr);
    CU(launch_fanrec(h->d_fan_ent, (int64_t)P.fan_ent.size(), h->d_ut, h->d_fan_off, h->d_rowoff, h->d_fan_rec,
                     g_upload_stream));
  }
  h->pool_bytes = std::max<size_t>((size_t)P.valoff[ns] * esz, 256);
  DALLOC(h->d_pool, h->pool_bytes, nullptr);
  DALLOC(h->d_inv, std::max<size_t>((size_t)P.invoff[ns] * sizeof(double), 256), nullptr);
  if (P.n_w > 0) DALLOC(h->d_wbuf, (size_t)P.n_w * esz, nullptr);
  if (mma_mode_of(h->opt.precision) != 1 && mma_mode_of(h->opt.precision) != 2 && P.ns > 0) {
    std::vector<CUtensorMap> maps;
    if (build_tensor_maps(h, maps)) {
      static_assert(sizeof(CUtensorMap) == 128, "tensor map size");
      DALLOC(h->d_tmaps, maps.size() * sizeof(CUtensorMap), nullptr);
      CU(cudaMemcpyAsync(h->d_tmaps, maps.data(), maps.size() * sizeof(CUtensorMap), cudaMemcpyHostToDevice,
                         g_upload_stream));
      CU(cudaStreamSynchronize(g_upload_stream));  // the host vector goes out of scope
    }
  }
  DALLOC(h->d_relpos, std::max<size_t>((size_t)P.n_rel * sizeof(int32_t), 256), nullptr);
  CU(launch_relpos(h->d_ut, P.n_u, h->d_rows, h->d_rowoff, h->d_nrows, h->d_relpos, g_upload_stream));
  if (oz) DALLOC(h->d_slices, std::max<size_t>((size_t)P.sliceoff[ns] * sizeof(uint16_t), 256), nullptr);
  PINNED(h->h_ctrl, kCtrlWords * sizeof(int));
  PINNED(h->h_prof, kProfWords * sizeof(unsigned long long));
  if (h->opt.profile == 2) {
    DALLOC(h->d_trace_f, 2 * (size_t)std::max(P.n_task_ids, 1) * sizeof(unsigned long long), nullptr);
    DALLOC(h->d_trace_s, 2 * (size_t)std::max(P.n_solve_tasks, 1) * sizeof(unsigned long long), nullptr);
    // tasks that never run on their own (panels inside subtree tasks) keep 0 / 0
    CU(cudaMemsetAsync(h->d_trace_f, 0, 2 * (size_t)std::max(P.n_task_ids, 1) * sizeof(unsigned long long),
                       g_upload_stream));
    CU(cudaMemsetAsync(h->d_trace_s, 0, 2 * (size_t)std::max(P.n_solve_tasks, 1) * sizeof(unsigned long long),
                       g_upload_stream));
  }
  CU(cudaEventCreate(&h->ev0));
  CU(cudaEventCreate(&h->ev1));
  // launch geometry: persistent grids no larger than what can be co-resident
  int dev = h->device;
  CU(cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, dev));
  const int wmax = std::max<int>(P.max_w, 1);
  h->smem_factor = factor_smem_bytes(wmax, mma_mode_of(h->opt.precision));
  if (mma_mode_of(h->opt.precision) == 3) {
    // each CTA of this mode owns a quarter of the SM's 512 TMEM columns:
    // request more than a fifth of the SM's shared memory so that five CTAs can
    // never share one (a fifth CTA's allocation would wait)
    int smem_sm = 0;
    CU(cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, h->device));
    h->smem_factor = std::max<size_t>(h->smem_factor, (size_t)smem_sm / 5 + 1024);
  }
  if (fan) h->smem_factor = std::max(h->smem_factor, fanin_smem_bytes(wmax, h->fp32, &h->fan_cap));
  h->smem_solve = solve_smem_bytes(wmax, h->opt.precision == SPCHOL_FP64_TC, fan);
  int bf = 0, bs = 0;
  CU(factor_configure(h->fp32, mma_mode_of(h->opt.precision), fan, h->smem_factor, &bf));
  if (h->n_wsub > 0 || h->n_wsub_solve > 0) {
    int bw = 0;
    CU(warp_subtree_configure(h->fp32, &bw));
    h->grid_wsub = std::max(1, std::min(std::max(bw, 1) * h->num_sms, ((int)P.wsub.size() + 3) / 4));
  }
  CU(solve_configure(h->fp32, fan, h->opt.precision == SPCHOL_FP64_TC, h->smem_solve, &bs));
  if (bf < 1 || bs < 1) return SPCHOL_ECUDA;
  if (h->opt.ctas_per_sm > 0) {
    bf = std::min(bf, h->opt.ctas_per_sm);
    bs = std::min(bs, h->opt.ctas_per_sm);
  }
  h->grid_factor = std::max(1, std::min(bf * h->num_sms, std::max(P.n_factor_tasks, 1)));
  h->grid_solve = std::max(1, std::min(bs * h->num_sms, std::max(P.n_solve_tasks, 1)));
  h->stats.footprint_bytes = (int64_t)(A.bytes + h->pool_bytes + (size_t)P.invoff[ns] * sizeof(double) +
                                       (size_t)P.n_w * (h->fp32 ? sizeof(float) : sizeof(double)) +
                                       (size_t)P.n_rel * sizeof(int32_t) + (size_t)P.ns * (h->d_tmaps ? 128 : 0) +
                                       (oz ? (size_t)P.sliceoff[ns] * sizeof(uint16_t) : 0) + h->fan_buf_bytes +
                                       (h->d_fan_rec ? P.fan_ent.size() * sizeof(FanRec) : 0));
  h->stats.grid_factor = h->grid_factor;
  h->stats.grid_solve = h->grid_solve;
  h->stats.tma_staging = h->d_tmaps != nullptr ? 1 : 0;
  return 0;
}

// The solve's workspace for n x nrhs right-hand sides, grown on demand.  The old
// buffers' last users (earlier calls) have completed, so they are released at
// once, stream-ordered on st, and the new ones allocated on st.
int ensure_workspace(spchol_handle_t h, int64_t need, int nrhs, cudaStream_t st) {
  if (h->plan.params.fanin && nrhs > h->fan_nrhs) {  // the fan-in solves' tile buffers
    for (double** p : {&h->d_zf, &h->d_zb}) {
      dfree(h, *p, st);
      *p = nullptr;
    }
    h->fan_nrhs = 0;
    DALLOC(h->d_zf, std::max<size_t>((size_t)h->plan.st_zf.back() * nrhs, 1) * sizeof(double), st);
    DALLOC(h->d_zb, std::max<size_t>((size_t)h->plan.st_zb.back() * nrhs, 1) * sizeof(double), st);
    h->fan_nrhs = nrhs;
  }
  if (need > h->y_cap) {
    for (double** p : {&h->d_Y, &h->d_B, &h->d_X, &h->d_R}) {
      dfree(h, *p, st);
      *p = nullptr;
    }
    h->y_cap = 0;
    DALLOC(h->d_Y, need * sizeof(double), st);
    DALLOC(h->d_B, need * sizeof(double), st);
    if (h->fp32) {
      DALLOC(h->d_X, need * sizeof(double), st);
      DALLOC(h->d_R, need * sizeof(double), st);
    }
    h->y_cap = need;
  }
  if (h->fp32 && nrhs > h->norms_cap) {
    dfree(h, h->d_norms, st);
    pinned_put(h->h_norms, h->h_norms_bytes);
    h->d_norms = nullptr;
    h->h_norms = nullptr;
    h->norms_cap = 0;
    DALLOC(h->d_norms, (1 + 3 * (size_t)nrhs) * sizeof(unsigned long long), st);
    h->h_norms_bytes = (1 + 3 * (size_t)nrhs) * sizeof(unsigned long long);
    PINNED(h->h_norms, h->h_norms_bytes);
    h->norms_cap = nrhs;
  }
  return 0;
}

bool is_device_ptr(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

int read_status(spchol_handle_t h, cudaStream_t st, int expect_done) {
  CU(cudaMemcpyAsync(h->h_ctrl, h->d_ctrl, kCtrlWords * sizeof(int), cudaMemcpyDeviceToHost, st));
  CU(cudaStreamSynchronize(st));
  const int* c = h->h_ctrl;
  if (c[kErr] != 0) return c[kErr];
  if (c[kInfo] != INT_MAX) return c[kInfo];
  if (c[kDone] != expect_done) return SPCHOL_EINTERNAL;
  return 0;
}

int finish_analyze(spchol_handle_t h, std::chrono::steady_clock::time_point t0) {
  Plan& P = h->plan;
  int rc = setup_device(h);
  if (rc) return rc;
  spchol_stats& S = h->stats;
  S.n = P.n;
  S.nnz_a = P.nnz_a;
  S.nnz_l = P.nnz_l;
  S.nnz_l_stored = P.nnz_l_stored;
  S.flops = P.flops;
  S.n_supernodes = P.ns;
  S.n_tasks = P.n_factor_tasks;
  S.n_subtrees = P.n_sub;
  S.n_warp_subtrees = h->n_wsub;
  S.max_width = P.max_w;
  S.max_rows = P.max_r;
  S.analyze_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  S.factor_ms = S.solve_ms = 0.0;
  S.ir_iters = 0;
  S.berr = -1.0;
  S.precision = h->opt.precision;
  return 0;
}

// Queue assembly, counter reset, the persistent factorization and the copy
// of its status words to pinned host memory; no host synchronisation and no
// allocation, so the sequence can be captured into a CUDA graph.
int enqueue_factor(spchol_handle_t h, const double* vals, cudaStream_t st, bool profile = false) {
  Plan& P = h->plan;
  CU(cudaMemsetAsync(h->d_pool, 0, h->pool_bytes, st));
  CU(launch_assemble(h->fp32, vals, h->d_adest, P.nnz_a, h->d_pool, st));
  if (P.ns == 0) return 0;
  const bool fifo = P.params.fifo;  // one FIFO ring: no high-priority slots, seeds at the front
  CU(launch_ring_reset(h->d_ring, P.n_factor_tasks, h->d_fseeds, h->nfseeds, h->d_ctrl, h->d_dep, h->d_dep_init,
                       P.ns, h->d_trsm_left, h->d_trsm_init, P.ns, nullptr, nullptr, 0, st, nullptr, nullptr, 0,
                       /*seeds_hi=*/fifo ? 0 : 1));
  FactorArgs a{};
  a.gat0 = INT_MAX;  // no gather tasks outside the fan-in mode
  a.pv = PanelView{P.ns, h->d_fcol, h->d_nrows, h->d_ld, h->d_rowoff, h->d_rows, h->d_valoff, h->d_parent};
  a.trsm_first = h->d_trsm_first;
  a.ntrsm = h->d_ntrsm;
  a.trsm_sn = h->d_trsm_sn;
  a.trsm_rows_of = h->d_trsm_rows;
  a.u_first = h->d_u_first;
  a.nu = h->d_nu;
  a.nu_hi = h->d_nu_hi;
  a.sub_lo = h->d_sub_lo;
  a.sub_hi = h->d_sub_hi;
  a.wsub = h->d_wsub;
  a.n_wsub = h->n_wsub;
  a.relpos = h->d_relpos;
  a.tmaps = h->d_tmaps;
  a.n_hi = fifo ? 0 : P.n_hi_tasks;
  a.ut = h->d_ut;
  a.n_trsm = P.n_trsm;
  a.n_u = P.n_u;
  a.ntask = P.n_factor_tasks;
  a.trsm_rows = P.params.trsm_rows;
  a.mma_mode = mma_mode_of(h->opt.precision);
  a.slices = h->d_slices;
  a.sliceoff = h->d_sliceoff;
  a.rexp = h->d_rexp;
  a.tc_min_width = P.params.tc_min_width;
  a.dep_f = h->d_dep;
  a.trsm_left = h->d_trsm_left;
  if (P.params.deterministic && !P.params.fanin && P.n_u > 0) {
    CU(cudaMemcpyAsync(h->d_u_dep, h->d_u_dep0, (size_t)P.n_u * sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
    a.u_next = h->d_u_next;
    a.u_dep = h->d_u_dep;
  }
  if (P.params.fanin) {
    a.fan_buf = h->d_fan_buf;
    a.fan_off = h->d_fan_off;
    a.fan_task = h->d_fan_task;
    a.fan_ptr = h->d_fan_ptr;
    a.fan_rec = h->d_fan_rec;
    CU(cudaMemcpyAsync(h->d_gdiag, h->d_gdiag0, (size_t)P.ns * sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
    if (P.n_trsm > 0)
      CU(cudaMemcpyAsync(h->d_tdep, h->d_tdep0, (size_t)P.n_trsm * sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
    a.gat0 = P.ns + P.n_trsm + P.n_u + P.n_sub;
    a.gat_first = h->d_gat_first;
    a.gat_pc = h->d_gat_pc;
    a.pc_owner = h->d_pc_owner;
    a.gdiag0 = h->d_gdiag0;
    a.gdiag = h->d_gdiag;
    a.tdep = h->d_tdep;
    a.fan_cap = h->fan_cap;
  }
  a.ring = h->d_ring;
  a.ctrl = h->d_ctrl;
  a.budget_ns = h->opt.wait_budget_ns;
  a.pool = h->d_pool;
  a.inv = h->d_inv;
  a.invoff = h->d_invoff;
  a.wbuf = h->d_wbuf;
  a.woff = P.n_wpan > 0 ? h->d_woff : nullptr;
  a.prof = profile ? h->d_prof : nullptr;
  a.trace = profile ? h->d_trace_f : nullptr;
  if (a.prof) CU(cudaMemsetAsync(h->d_prof, 0, 16 * sizeof(unsigned long long), st));
  CU(launch_warp_subtrees(h->fp32, a, h->grid_wsub, st));  // their tiles' counters release ring tasks
  CU(launch_factor(h->fp32, a, h->grid_factor, h->smem_factor, st));
  CU(cudaMemcpyAsync(h->h_ctrl, h->d_ctrl, kCtrlWords * sizeof(int), cudaMemcpyDeviceToHost, st));
  return 0;
}

int status_of(spchol_handle_t h) {
  const int* c = h->h_ctrl;
  if (c[kErr] != 0) return c[kErr];
  if (c[kInfo] != INT_MAX) return c[kInfo];
  if (c[kDone] != h->plan.n_factor_tasks) return SPCHOL_EINTERNAL;
  return 0;
}

int factorize_impl(spchol_handle_t h, const double* values_dev_or_null, const double* values_host,
                   cudaStream_t st) {
  Plan& P = h->plan;
  h->factored = false;
  if (values_host && P.nnz_a > 0)
    CU(cudaMemcpyAsync(h->d_vals, values_host, P.nnz_a * sizeof(double), cudaMemcpyHostToDevice, st));
  const double* vals = values_host ? h->d_vals : values_dev_or_null;
  if (h->fp32 && !values_host && P.nnz_a > 0 && vals != h->d_vals) {
    // the refinement residual needs A's FP64 values after the caller's buffer is gone
    CU(cudaMemcpyAsync(h->d_vals, vals, P.nnz_a * sizeof(double), cudaMemcpyDeviceToDevice, st));
    vals = h->d_vals;
  }
  CU(cudaEventRecord(h->ev0, st));
  int rc = enqueue_factor(h, vals, st, h->opt.profile != 0);
  if (rc) return rc;
  CU(cudaEventRecord(h->ev1, st));
  CU(cudaStreamSynchronize(st));
  if (P.ns > 0) {
    rc = status_of(h);
    if (h->opt.profile) {
      CU(cudaMemcpy(h->h_prof, h->d_prof, 16 * sizeof(unsigned long long), cudaMemcpyDeviceToHost));
      for (int k = 0; k < 3; ++k) {
        h->stats.factor_task_ms[k] = h->h_prof[k] * 1e-6;
        h->stats.factor_task_count[k] = (int64_t)h->h_prof[4 + k];
      }
      h->stats.factor_wait_ms = h->h_prof[3] * 1e-6;
      h->stats.factor_tc_update_ms = h->h_prof[7] * 1e-6;
      h->stats.factor_subtree_ms = h->h_prof[8] * 1e-6;
      h->stats.factor_subtree_count = (int64_t)h->h_prof[9];
      for (int k = 0; k < 3; ++k) h->stats.factor_gather_ms[k] = h->h_prof[10 + k] * 1e-6;
      h->stats.factor_gather_batches = (int64_t)h->h_prof[13];
      h->stats.factor_gather_tiles = (int64_t)h->h_prof[14];
    }
  }
  float ms = 0.f;
  cudaEventElapsedTime(&ms, h->ev0, h->ev1);
  h->stats.factor_ms = ms;
  if (rc == 0) h->factored = true;
  h->traced_f = h->d_trace_f != nullptr && P.ns > 0;
  return rc;
}

// Forward + backward solve of Y (permuted order, device, ld = n) in place.
int solve_permuted(spchol_handle_t h, double* Y, int nrhs, cudaStream_t st) {
  Plan& P = h->plan;
  if (P.ns == 0 || nrhs == 0) return 0;
  // seeds: the normal-priority ring, after the other (one FIFO ring: no high-priority slots)
  const int n_hi = P.params.fifo ? 0 : P.n_solve_tasks - h->nsseeds;
  CU(launch_ring_reset(h->d_ring, P.n_solve_tasks, h->d_sseeds, h->nsseeds, h->d_ctrl, h->d_fkids, h->d_fdep0,
                       P.ns, h->d_ftiles, h->d_nst, P.ns, h->d_btiles, h->d_nst, P.ns, st, h->d_bdep, h->d_bdep0,
                       P.n_st, /*seeds_hi=*/0, /*seed_off=*/n_hi));
  SolveArgs a{};
  a.pv = PanelView{P.ns, h->d_fcol, h->d_nrows, h->d_ld, h->d_rowoff, h->d_rows, h->d_valoff, h->d_parent};
  a.kid_ptr = h->d_kid_ptr;
  a.kids = h->d_kids;
  a.st_first = h->d_st_first;
  a.nst = h->d_nst;
  a.st_sn = h->d_st_sn;
  a.n_st = P.n_st;
  a.ntask = P.n_solve_tasks;
  a.st_rows = h->d_st_rows;
  a.n_hi = n_hi;
  a.st_tptr = h->d_st_tptr;
  a.st_tgt = h->d_st_tgt;
  a.rt_ptr = h->d_rt_ptr;
  a.rt_tile = h->d_rt_tile;
  a.fdep = h->d_fkids;
  a.bdep = h->d_bdep;
  a.ftiles = h->d_ftiles;
  a.btiles = h->d_btiles;
  if (P.params.deterministic && !P.params.fanin && P.n_st > 0) {
    CU(cudaMemcpyAsync(h->d_ftdep, h->d_ft_dep0, (size_t)P.n_st * sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
    a.ft_sptr = h->d_ft_sptr;
    a.ft_succ = h->d_ft_succ;
    a.ftdep = h->d_ftdep;
  }
  if (P.params.fanin) {
    if (nrhs > h->fan_nrhs) return SPCHOL_EINTERNAL;  // the caller sizes the workspace first
    a.zf = h->d_zf;
    a.zb = h->d_zb;
    a.st_zf = h->d_st_zf;
    a.st_zb = h->d_st_zb;
    a.rt_rec = h->d_rt_rec;
  }
  a.ring = h->d_ring;
  a.ctrl = h->d_ctrl;
  a.budget_ns = h->opt.wait_budget_ns;
  a.pool = h->d_pool;
  a.inv = h->d_inv;
  a.invoff = h->d_invoff;
  a.wbuf = h->d_wbuf;
  a.woff = P.n_wpan > 0 ? h->d_woff : nullptr;
  a.n_wpan = P.n_wpan;
  a.sub_lo = h->d_sub_lo;
  a.sub_hi = h->d_sub_hi;
  a.wsub = h->d_wsub;
  a.n_wsub = h->n_wsub_solve;
  a.ntask_done = h->solve_done;
  a.Y = Y;
  a.ldy = P.n;
  a.nrhs = nrhs;
  a.tc_tiles = h->opt.precision == SPCHOL_FP64_TC ? 1 : 0;
  a.prof = h->opt.profile ? h->d_prof + 16 : nullptr;
  a.trace = h->d_trace_s;
  if (a.prof) CU(cudaMemsetAsync(h->d_prof + 16, 0, 8 * sizeof(unsigned long long), st));
  CU(launch_subtree_solve(h->fp32, true, a, h->grid_wsub, st));
  CU(launch_solve(h->fp32, a, h->grid_solve, h->smem_solve, st));
  CU(launch_subtree_solve(h->fp32, false, a, h->grid_wsub, st));
  int rc = read_status(h, st, h->solve_done + h->n_wsub_solve);
  h->traced_s = h->d_trace_s != nullptr;
  if (h->opt.profile) {
    CU(cudaMemcpy(h->h_prof + 16, h->d_prof + 16, 8 * sizeof(unsigned long long), cudaMemcpyDeviceToHost));
    for (int k = 0; k < 4; ++k) h->stats.solve_task_ms[k] = h->h_prof[16 + k] * 1e-6;
    h->stats.solve_wait_ms = h->h_prof[20] * 1e-6;
  }
  return rc;
}

// dst = M^{-1} src for one vector in the original order: M = P^T L L^T P the
// low-precision factor.
int apply_factor_inverse(spchol_handle_t h, const double* src, double* dst, cudaStream_t st) {
  const int64_t n = h->plan.n;
  CU(launch_permute_in(src, n, h->d_Y, n, h->d_perm, n, 1, st));
  int rc = solve_permuted(h, h->d_Y, 1, st);
  if (rc) return rc;
  CU(launch_permute_out(h->d_Y, n, dst, n, h->d_perm, n, 1, st));
  return 0;
}

int ensure_gmres(spchol_handle_t h, cudaStream_t st) {
  if (h->d_gmV) return 0;
  const int64_t n = h->plan.n;
  DALLOC(h->d_gmV, (size_t)n * (kGmresRestart + 1) * sizeof(double), st);
  DALLOC(h->d_gmW, (size_t)n * sizeof(double), st);
  DALLOC(h->d_gmPart, (size_t)kGmresBlocks * (kGmresRestart + 1) * sizeof(double), st);
  DALLOC(h->d_gmH, 3 * (kGmresRestart + 2) * sizeof(double), st);
  PINNED(h->h_gmH, 3 * (kGmresRestart + 2) * sizeof(double));
  return 0;
}

// One GMRES-IR correction (Carson and Higham, "Accelerating the solution of
// linear systems by iterative refinement in three precisions", SIAM J. Sci.
// Comput. 40, 2018, restated with two precisions): the correction equation
// A d = r of right-hand side c is solved by GMRES in FP64 on M^{-1} A d =
// M^{-1} r, left-preconditioned by the low-precision factor, instead of by one
// application of M^{-1}; it converges where the classic step's contraction
// u_f kappa(A) exceeds one.  Arnoldi by classical Gram-Schmidt applied twice;
// Givens rotations on the host; one cycle of at most kGmresRestart steps, to
// a preconditioned residual reduction of 1e-10.  x_c += d.  *steps: the
// Arnoldi steps taken.
int gmres_correction(spchol_handle_t h, int c, cudaStream_t st, int* steps) {
  const int64_t n = h->plan.n;
  const int m = kGmresRestart;
  double* V = h->d_gmV;
  double* hd = h->d_gmH;  // [0, m+1): first pass, [m+2, 2m+3): second pass, [2m+4]: norm
  double* hh = h->h_gmH;
  int rc = apply_factor_inverse(h, h->d_R + (size_t)c * n, V, st);
  if (rc) return rc;
  CU(launch_dots(n, 1, V, n, V, h->d_gmPart, hd, st));
  CU(cudaMemcpyAsync(hh, hd, sizeof(double), cudaMemcpyDeviceToHost, st));
  CU(cudaStreamSynchronize(st));
  const double beta = std::sqrt(hh[0]);
  *steps = 0;
  if (!(beta > 0.0) || !std::isfinite(beta)) return 0;
  CU(launch_scale(n, 1.0 / beta, V, V, st));
  std::vector<double> H((size_t)(m + 1) * m, 0.0), cs(m), sn(m), g(m + 1, 0.0);
  g[0] = beta;
  int k = 0;
  for (; k < m; ++k) {
    double* vk = V + (size_t)k * n;
    double* z = V + (size_t)(k + 1) * n;
    CU(launch_spmv(n, h->d_csr_rp, h->d_csr_ci, h->d_csr_vmap, h->d_vals, vk, h->d_gmW, st));
    rc = apply_factor_inverse(h, h->d_gmW, z, st);
    if (rc) return rc;
    for (int pass = 0; pass < 2; ++pass) {
      double* hp = hd + pass * (m + 2);
      CU(launch_dots(n, k + 1, V, n, z, h->d_gmPart, hp, st));
      CU(launch_axpy_multi(n, k + 1, V, n, hp, -1.0, z, st));
    }
    CU(launch_dots(n, 1, z, n, z, h->d_gmPart, hd + 2 * (m + 2), st));
    CU(cudaMemcpyAsync(hh, hd, 3 * (m + 2) * sizeof(double), cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
    double* col = H.data() + (size_t)k * (m + 1);
    for (int j = 0; j <= k; ++j) col[j] = hh[j] + hh[(m + 2) + j];
    const double hk1 = std::sqrt(hh[2 * (m + 2)]);
    col[k + 1] = hk1;
    if (hk1 > 0.0) CU(launch_scale(n, 1.0 / hk1, z, z, st));
    for (int j = 0; j < k; ++j) {  // earlier rotations
      const double a = col[j], b = col[j + 1];
      col[j] = cs[j] * a + sn[j] * b;
      col[j + 1] = -sn[j] * a + cs[j] * b;
    }
    const double r = std::hypot(col[k], col[k + 1]);
    cs[k] = r > 0.0 ? col[k] / r : 1.0;
    sn[k] = r > 0.0 ? col[k + 1] / r : 0.0;
    col[k] = r;
    col[k + 1] = 0.0;
    g[k + 1] = -sn[k] * g[k];
    g[k] = cs[k] * g[k];
    if (!(std::fabs(g[k + 1]) > 1e-10 * beta) || !(hk1 > 0.0)) {
      ++k;
      break;
    }
  }
  if (k > m) k = m;
  // y = R^{-1} g (upper triangular), then x_c += V y
  std::vector<double> y(k, 0.0);
  for (int i = k - 1; i >= 0; --i) {
    double s = g[i];
    for (int j = i + 1; j < k; ++j) s -= H[(size_t)j * (m + 1) + i] * y[j];
    const double d = H[(size_t)i * (m + 1) + i];
    y[i] = d != 0.0 ? s / d : 0.0;
  }
  for (int i = 0; i < k; ++i) hh[i] = y[i];
  CU(cudaMemcpyAsync(hd, hh, (size_t)std::max(k, 1) * sizeof(double), cudaMemcpyHostToDevice, st));
  CU(launch_axpy_multi(n, k, V, n, hd, 1.0, h->d_X + (size_t)c * n, st));
  *steps = k;
  return 0;
}

// Mixed precision: X = A^{-1} B by the low-precision factor plus FP64
// refinement.  B0 = d_B (original order, ld n, nrhs columns); X ends in d_B.
// Classic refinement first; if it stops contracting, GMRES-IR continues from
// the current iterate.
int solve_refined(spchol_handle_t h, int nrhs, cudaStream_t st) {
  Plan& P = h->plan;
  const int64_t n = P.n;
  const size_t nb = (1 + 3 * (size_t)nrhs) * sizeof(unsigned long long);
  CU(launch_anorm(n, h->d_csr_rp, h->d_csr_vmap, h->d_vals, h->d_norms, st));
  CU(launch_permute_in(h->d_B, n, h->d_Y, n, h->d_perm, n, nrhs, st));
  int rc = solve_permuted(h, h->d_Y, nrhs, st);
  if (rc) return rc;
  CU(cudaMemsetAsync(h->d_X, 0, n * nrhs * sizeof(double), st));
  CU(launch_correct(h->d_Y, n, h->d_X, n, h->d_perm, n, nrhs, st));
  double prev = INFINITY, berr = INFINITY;
  int iters = 0, gmres_outer = 0, gmres_steps = 0;
  bool gmres = false;
  rc = 0;
  for (;;) {
    CU(launch_residual(n, nrhs, h->d_csr_rp, h->d_csr_ci, h->d_csr_vmap, h->d_vals, h->d_X, n, h->d_B, n, h->d_R, n,
                       h->d_norms + 1, st));
    CU(cudaMemcpyAsync(h->h_norms, h->d_norms, nb, cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
    double anorm;
    std::memcpy(&anorm, &h->h_norms[0], sizeof(double));
    berr = 0.0;
    for (int r = 0; r < nrhs; ++r) {
      double rn, xn, bn;
      std::memcpy(&rn, &h->h_norms[1 + 3 * r], sizeof(double));
      std::memcpy(&xn, &h->h_norms[2 + 3 * r], sizeof(double));
      std::memcpy(&bn, &h->h_norms[3 + 3 * r], sizeof(double));
      const double den = anorm * xn + bn;
      const double e = den > 0.0 ? rn / den : (rn > 0.0 ? INFINITY : 0.0);
      if (!(e <= berr)) berr = e;  // NaN propagates
    }
    if (berr <= h->opt.ir_tol) break;
    if (!gmres && (!(berr == berr) || iters >= h->opt.ir_max_iter || berr > 0.5 * prev)) {
      // classic refinement stopped contracting: GMRES-IR from here (from zero
      // if the iterate is no longer finite)
      gmres = true;
      if (!(berr == berr) || std::isinf(berr)) {
        CU(cudaMemsetAsync(h->d_X, 0, n * nrhs * sizeof(double), st));
        prev = INFINITY;
        continue;
      }
    }
    if (gmres) {
      if (gmres_outer >= h->opt.ir_max_iter || !(berr == berr) || (gmres_outer > 0 && berr > 0.5 * prev)) {
        rc = SPCHOL_ENOCONV;
        break;
      }
      prev = berr;
      if ((rc = ensure_gmres(h, st)) != 0) return rc;
      for (int c = 0; c < nrhs; ++c) {
        int steps = 0;
        int r2 = gmres_correction(h, c, st, &steps);
        if (r2) return r2;
        gmres_steps += steps;
      }
      ++gmres_outer;
      ++iters;
      continue;
    }
    prev = berr;
    CU(launch_permute_in(h->d_R, n, h->d_Y, n, h->d_perm, n, nrhs, st));
    int r2 = solve_permuted(h, h->d_Y, nrhs, st);
    if (r2) return r2;
    CU(launch_correct(h->d_Y, n, h->d_X, n, h->d_perm, n, nrhs, st));
    ++iters;
  }
  h->stats.ir_iters = iters;
  h->stats.ir_gmres_iters = gmres_steps;
  h->stats.berr = berr;
  CU(cudaMemcpyAsync(h->d_B, h->d_X, n * nrhs * sizeof(double), cudaMemcpyDeviceToDevice, st));
  return rc;
}

}  // namespace

extern "C" {

void spchol_default_options(spchol_options* opt) {
  if (opt) spchol::default_options(opt);
}

const char* spchol_last_cuda_error(void) { return g_cuda_err; }

const char* spchol_strerror(int code) {
  if (code == 0) return "success";
  if (code > 0) return "matrix is not positive definite (the code is the failing permuted column, 1-based)";
  switch (code) {
    case SPCHOL_ENOMEM: return "out of memory";
    case SPCHOL_ETIMEOUT: return "a device-side wait exceeded the wait budget";
    case SPCHOL_ESTATE: return "call out of order (no factor for this handle)";
    case SPCHOL_ENOCONV: return "iterative refinement did not reach the target backward error";
    case SPCHOL_ECUDA: return "a CUDA runtime call failed";
    case SPCHOL_EINTERNAL: return "a device-side consistency check failed";
    case SPCHOL_ESCRATCH: return "the problem does not fit the fixed 32 MiB scratch of spchol_solve_noalloc";
    default: break;
  }
  if (code < 0 && code > -100) return "invalid argument (the code is minus the argument's 1-based position)";
  return "unknown error";
}

int spchol_analyze(int64_t n, const int64_t* colptr, const int32_t* rowind, const int64_t* perm,
                   const spchol_options* opt, spchol_handle_t* out) {
  if (!out) return -6;
  *out = nullptr;
  const auto t0 = std::chrono::steady_clock::now();
  spchol_options o;
  if (opt) {
    o = *opt;
    if (!options_valid(o)) return -5;
  } else {
    spchol::default_options(&o);
  }
  spchol_handle_t h = new (std::nothrow) spchol_handle_s();
  if (!h) return SPCHOL_ENOMEM;
  clear_stale_error();
  h->opt = o;
  h->fp32 = (o.precision == SPCHOL_FP32 || o.precision == SPCHOL_TF32 || o.precision == SPCHOL_TF32X3);
  if (cudaGetDevice(&h->device) != cudaSuccess) {
    delete h;
    return SPCHOL_ECUDA;
  }
  PlanError err;
  int rc = build_plan(n, colptr, rowind, perm, params_from(o), h->plan, err);
  if (rc == 0 && h->fp32) {
    h->a_row.resize(h->plan.nnz_a);
    h->a_col.resize(h->plan.nnz_a);
    for (int64_t j = 0; j < n; ++j)
      for (int64_t p = colptr[j]; p < colptr[j + 1]; ++p) {
        h->a_row[p] = rowind[p];
        h->a_col[p] = (int32_t)j;
      }
  }
  if (rc == 0 && o.fault_inject == 1 && h->plan.ns > 0) h->plan.dep_f[h->plan.ns - 1] += 1;
  if (rc == 0) rc = finish_analyze(h, t0);
  if (rc != 0) {
    spchol_destroy(h);
    return rc;
  }
  *out = h;
  return 0;
}

int spchol_factorize(spchol_handle_t h, const double* values, void* stream) {
  if (!h) return -1;
  if (!values && h->plan.nnz_a > 0) return -2;
  DeviceGuard g(h->device);
  clear_stale_error();
  cudaStream_t st = (cudaStream_t)stream;
  const bool dev = values && is_device_ptr(values);
  return factorize_impl(h, dev ? values : nullptr, dev ? nullptr : values, st);
}

int spchol_factorize_enqueue(spchol_handle_t h, const double* values, void* stream) {
  if (!h) return -1;
  if (!values && h->plan.nnz_a > 0) return -2;
  DeviceGuard g(h->device);
  clear_stale_error();
  if (values && !is_device_ptr(values)) return -2;
  h->factored = false;
  h->pending = true;
  cudaStream_t st = (cudaStream_t)stream;
  if (h->fp32 && h->plan.nnz_a > 0) {  // the refinement residual reads A's FP64 values later
    CU(cudaMemcpyAsync(h->d_vals, values, h->plan.nnz_a * sizeof(double), cudaMemcpyDeviceToDevice, st));
    values = h->d_vals;
  }
  return enqueue_factor(h, values, st);
}

int spchol_factorize_status(spchol_handle_t h) {
  if (!h) return -1;
  if (!h->pending) return SPCHOL_ESTATE;
  if (h->plan.ns == 0) {
    h->factored = true;
    return 0;
  }
  const int rc = status_of(h);
  h->factored = (rc == 0);
  return rc;
}

int spchol_solve(spchol_handle_t h, double* B, int64_t ldb, int nrhs, void* stream) {
  if (!h) return -1;
  if (nrhs < 0) return -4;
  if (ldb < std::max<int64_t>(h->plan.n, 1)) return -3;
  if (!B && nrhs > 0 && h->plan.n > 0) return -2;
  if (!h->factored) return SPCHOL_ESTATE;
  if (nrhs == 0 || h->plan.n == 0) return 0;
  DeviceGuard g(h->device);
  clear_stale_error();
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t n = h->plan.n;
  int rc = ensure_workspace(h, n * nrhs, nrhs, st);
  if (rc) return rc;
  const bool dev = is_device_ptr(B);
  CU(cudaEventRecord(h->ev0, st));
  if (dev && !h->fp32) {
    // FP64 fast path: permute straight from and back into the caller's buffer
    CU(launch_permute_in(B, ldb, h->d_Y, n, h->d_perm, n, nrhs, st));
    rc = solve_permuted(h, h->d_Y, nrhs, st);
    if (rc) return rc;
    CU(launch_permute_out(h->d_Y, n, B, ldb, h->d_perm, n, nrhs, st));
  } else {
    CU(cudaMemcpy2DAsync(h->d_B, n * sizeof(double), B, ldb * sizeof(double), n * sizeof(double), nrhs,
                         dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
    int core;
    if (h->fp32) {
      core = solve_refined(h, nrhs, st);
      if (core != 0 && core != SPCHOL_ENOCONV) return core;
    } else {
      CU(launch_permute_in(h->d_B, n, h->d_Y, n, h->d_perm, n, nrhs, st));
      core = solve_permuted(h, h->d_Y, nrhs, st);
      if (core) return core;
      CU(launch_permute_out(h->d_Y, n, h->d_B, n, h->d_perm, n, nrhs, st));
    }
    CU(cudaMemcpy2DAsync(B, ldb * sizeof(double), h->d_B, n * sizeof(double), n * sizeof(double), nrhs,
                         dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
    rc = core;
  }
  CU(cudaEventRecord(h->ev1, st));
  CU(cudaStreamSynchronize(st));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, h->ev0, h->ev1);
  h->stats.solve_ms = ms;
  return rc;
}

int spchol_solve_noalloc(spchol_handle_t h, double* B, int64_t ldb, int nrhs, void* stream) {
  if (!h) return -1;
  if (nrhs < 0) return -4;
  if (ldb < std::max<int64_t>(h->plan.n, 1)) return -3;
  if (!B && nrhs > 0 && h->plan.n > 0) return -2;
  if (h->fp32) return -1;  // FP64 factors only (the refined mixed solve needs more workspace)
  if (!h->factored) return SPCHOL_ESTATE;
  if (nrhs == 0 || h->plan.n == 0) return 0;
  DeviceGuard g(h->device);
  clear_stale_error();
  if (!is_device_ptr(B)) return -2;
  const Plan& P = h->plan;
  const int64_t n = P.n;
  // scratch layout: Y (n x nrhs doubles) | ring | fdep | ftiles | btiles | bdep | control words
  auto up = [](size_t x) { return (x + 255) & ~size_t(255); };
  const size_t y_bytes = up((size_t)n * nrhs * sizeof(double));
  const size_t ring_bytes = up((size_t)P.n_solve_tasks * sizeof(int));
  const size_t cnt_bytes = up((size_t)P.ns * sizeof(int32_t));
  const size_t tile_bytes = up((size_t)P.n_st * sizeof(int32_t));
  const bool fan = P.params.fanin && P.n_st > 0;
  const bool det = P.params.deterministic && !fan && P.n_st > 0;
  // fan-in mode: the tiles' forward and backward buffers follow
  const size_t zf_bytes = fan ? up((size_t)P.st_zf.back() * nrhs * sizeof(double)) : 0;
  const size_t zb_bytes = fan ? up((size_t)P.st_zb.back() * nrhs * sizeof(double)) : 0;
  const size_t need = y_bytes + ring_bytes + 3 * cnt_bytes + (det ? 2 : 1) * tile_bytes +
                      up(kCtrlWords * sizeof(int)) + zf_bytes + zb_bytes;
  if (need > kNoallocScratchBytes) return SPCHOL_ESCRATCH;
  void* base = nullptr;
  CU(noalloc_scratch(h->device, &base));
  char* b = (char*)base;
  double* Y = (double*)b;
  int* ring = (int*)(b + y_bytes);
  int32_t* fdep = (int32_t*)(b + y_bytes + ring_bytes);
  int32_t* ftiles = (int32_t*)((char*)fdep + cnt_bytes);
  int32_t* btiles = (int32_t*)((char*)ftiles + cnt_bytes);
  int32_t* bdep = (int32_t*)((char*)btiles + cnt_bytes);
  int* ctrl = (int*)((char*)bdep + tile_bytes);
  int32_t* ftdep = det ? (int32_t*)((char*)ctrl + up(kCtrlWords * sizeof(int))) : nullptr;
  double* zf = fan ? (double*)((char*)ctrl + up(kCtrlWords * sizeof(int))) : nullptr;
  double* zb = fan ? (double*)((char*)zf + zf_bytes) : nullptr;
  cudaStream_t st = (cudaStream_t)stream;
  // the array keeps the previous call's contents: the reset kernel re-initialises
  // the ring, the counters and the control words before every launch
  const int n_hi = P.params.fifo ? 0 : P.n_solve_tasks - h->nsseeds;
  CU(launch_ring_reset(ring, P.n_solve_tasks, h->d_sseeds, h->nsseeds, ctrl, fdep, h->d_fdep0, P.ns, ftiles,
                       h->d_nst, P.ns, btiles, h->d_nst, P.ns, st, bdep, h->d_bdep0, P.n_st, /*seeds_hi=*/0,
                       /*seed_off=*/n_hi));
  CU(launch_permute_in(B, ldb, Y, n, h->d_perm, n, nrhs, st));
  SolveArgs a{};
  a.pv = PanelView{P.ns, h->d_fcol, h->d_nrows, h->d_ld, h->d_rowoff, h->d_rows, h->d_valoff, h->d_parent};
  a.kid_ptr = h->d_kid_ptr;
  a.kids = h->d_kids;
  a.st_first = h->d_st_first;
  a.nst = h->d_nst;
  a.st_sn = h->d_st_sn;
  a.n_st = P.n_st;
  a.ntask = P.n_solve_tasks;
  a.st_rows = h->d_st_rows;
  a.n_hi = n_hi;
  a.st_tptr = h->d_st_tptr;
  a.st_tgt = h->d_st_tgt;
  a.rt_ptr = h->d_rt_ptr;
  a.rt_tile = h->d_rt_tile;
  a.fdep = fdep;
  a.bdep = bdep;
  a.ftiles = ftiles;
  a.btiles = btiles;
  if (det) {
    CU(cudaMemcpyAsync(ftdep, h->d_ft_dep0, (size_t)P.n_st * sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
    a.ft_sptr = h->d_ft_sptr;
    a.ft_succ = h->d_ft_succ;
    a.ftdep = ftdep;
  }
  if (fan) {
    a.zf = zf;
    a.zb = zb;
    a.st_zf = h->d_st_zf;
    a.st_zb = h->d_st_zb;
    a.rt_rec = h->d_rt_rec;
  }
  a.ring = ring;
  a.ctrl = ctrl;
  a.budget_ns = h->opt.wait_budget_ns;
  a.pool = h->d_pool;
  a.inv = h->d_inv;
  a.invoff = h->d_invoff;
  a.wbuf = h->d_wbuf;
  a.woff = P.n_wpan > 0 ? h->d_woff : nullptr;
  a.n_wpan = P.n_wpan;
  a.sub_lo = h->d_sub_lo;
  a.sub_hi = h->d_sub_hi;
  a.wsub = h->d_wsub;
  a.n_wsub = h->n_wsub_solve;
  a.ntask_done = h->solve_done;
  a.Y = Y;
  a.ldy = n;
  a.nrhs = nrhs;
  a.tc_tiles = h->opt.precision == SPCHOL_FP64_TC ? 1 : 0;
  a.prof = nullptr;
  a.trace = nullptr;
  CU(launch_subtree_solve(false, true, a, h->grid_wsub, st));
  CU(launch_solve(false, a, h->grid_solve, h->smem_solve, st));
  CU(launch_subtree_solve(false, false, a, h->grid_wsub, st));
  CU(launch_permute_out(Y, n, B, ldb, h->d_perm, n, nrhs, st));
  CU(cudaMemcpyAsync(h->h_ctrl, ctrl, kCtrlWords * sizeof(int), cudaMemcpyDeviceToHost, st));
  CU(cudaStreamSynchronize(st));
  const int* c = h->h_ctrl;
  if (c[kErr] != 0) return c[kErr];
  if (c[kDone] != h->solve_done + h->n_wsub_solve) return SPCHOL_EINTERNAL;
  return 0;
}

int spchol_stats_get(spchol_handle_t h, spchol_stats* st) {
  if (!h) return -1;
  if (!st) return -2;
  *st = h->stats;
  return 0;
}

int spchol_export_factor(spchol_handle_t h, int64_t* nnz, int64_t* Lp, int64_t* Li, double* Lx, int64_t* perm_out) {
  if (!h) return -1;
  if (!nnz) return -2;
  const Plan& P = h->plan;
  int64_t total = 0;
  for (int s = 0; s < P.ns; ++s) {
    const int64_t w = P.fcol[s + 1] - P.fcol[s], r = P.nrows[s];
    total += w * r - w * (w - 1) / 2;
  }
  if (perm_out)
    for (int64_t i = 0; i < P.n; ++i) perm_out[i] = P.perm[i];
  if (!Lp && !Li && !Lx) {
    *nnz = total;
    return 0;
  }
  if (*nnz < total) return -2;
  if (!h->factored) return SPCHOL_ESTATE;
  DeviceGuard g(h->device);
  const size_t esz = h->fp32 ? sizeof(float) : sizeof(double);
  std::vector<char> pool(h->pool_bytes);
  CU(cudaMemcpy(pool.data(), h->d_pool, h->pool_bytes, cudaMemcpyDeviceToHost));
  int64_t q = 0;
  for (int s = 0; s < P.ns; ++s) {
    const int w = P.fcol[s + 1] - P.fcol[s], r = P.nrows[s], ld = P.ld[s];
    const int32_t* R = P.rows.data() + P.rowoff[s];
    for (int j = 0; j < w; ++j) {
      if (Lp) Lp[P.fcol[s] + j] = q;
      for (int i = j; i < r; ++i) {
        const size_t idx = (size_t)P.valoff[s] + i + (size_t)j * ld;
        double v = h->fp32 ? (double)((float*)pool.data())[idx] : ((double*)pool.data())[idx];
        if (Li) Li[q] = R[i];
        if (Lx) Lx[q] = v;
        ++q;
      }
    }
  }
  (void)esz;
  if (Lp) Lp[P.n] = q;
  *nnz = q;
  return 0;
}

int spchol_trace_get(spchol_handle_t h, int which, uint64_t* out, int64_t* count) {
  if (!h) return -1;
  if (which != 0 && which != 1) return -2;
  if (!count) return -4;
  const int64_t nt = which == 0 ? h->plan.n_task_ids : h->plan.n_solve_tasks;
  if (!out) {
    *count = nt;
    return 0;
  }
  if (*count < nt) return -4;
  if (!(which == 0 ? h->traced_f : h->traced_s)) return SPCHOL_ESTATE;
  DeviceGuard g(h->device);
  CU(cudaMemcpy(out, which == 0 ? h->d_trace_f : h->d_trace_s, 2 * (size_t)nt * sizeof(uint64_t),
                cudaMemcpyDeviceToHost));
  *count = nt;
  return 0;
}

int spchol_destroy(spchol_handle_t h) {
  if (!h) return 0;
  DeviceGuard g(h->device);
  // Nothing here waits for the device: the memory goes back stream-ordered (or
  // to the caller's allocator), the pinned blocks to the process-wide cache.
  for (void* p : {(void*)h->arena.base, h->d_pool, h->d_fan_buf, (void*)h->d_fan_rec, (void*)h->d_inv, h->d_wbuf,
                  (void*)h->d_relpos, (void*)h->d_tmaps, (void*)h->d_slices, (void*)h->d_trace_f,
                  (void*)h->d_trace_s, (void*)h->d_Y, (void*)h->d_zf, (void*)h->d_zb, (void*)h->d_B,
                  (void*)h->d_X, (void*)h->d_R, (void*)h->d_gmV, (void*)h->d_gmW, (void*)h->d_gmPart,
                  (void*)h->d_gmH, (void*)h->d_norms})
    dfree(h, p, nullptr);
  pinned_put(h->h_ctrl, kCtrlWords * sizeof(int));
  pinned_put(h->h_prof, kProfWords * sizeof(unsigned long long));
  pinned_put(h->h_gmH, 3 * (kGmresRestart + 2) * sizeof(double));
  pinned_put(h->h_norms, h->h_norms_bytes);
  if (h->ev0) cudaEventDestroy(h->ev0);
  if (h->ev1) cudaEventDestroy(h->ev1);
  delete h;
  return 0;
}

// ------------------------------------------------------------------ batch

int spchol_batch_analyze(int count, const int64_t* n, const int64_t* const* colptr, const int32_t* const* rowind,
                         const int64_t* const* perm, const spchol_options* opt, spchol_handle_t* out) {
  if (count < 1) return -1;
  if (!n) return -2;
  if (!colptr) return -3;
  if (!rowind) return -4;
  if (!out) return -7;
  *out = nullptr;
  int64_t N = 0, NNZ = 0;
  for (int i = 0; i < count; ++i) {
    if (n[i] < 0 || (n[i] > 0 && (!colptr[i] || !rowind[i]))) return -2;
    N += n[i];
    NNZ += n[i] > 0 ? colptr[i][n[i]] : 0;
  }
  if (N > INT32_MAX - 1) return -2;
  std::vector<int64_t> cp(N + 1, 0), pm(N);
  std::vector<int32_t> ri(NNZ);
  std::vector<int64_t> col0(count), nnz0(count);
  int64_t c = 0, z = 0;
  for (int i = 0; i < count; ++i) {
    col0[i] = c;
    nnz0[i] = z;
    for (int64_t j = 0; j < n[i]; ++j) {
      for (int64_t p = colptr[i][j]; p < colptr[i][j + 1]; ++p) ri[z + p - colptr[i][0]] = (int32_t)(rowind[i][p] + c);
      cp[c + j + 1] = z + colptr[i][j + 1] - colptr[i][0];
      int64_t pj = (perm && perm[i]) ? perm[i][j] : j;
      if (pj < 0 || pj >= n[i]) return -5;
      pm[c + j] = pj + c;
    }
    z += n[i] > 0 ? colptr[i][n[i]] - colptr[i][0] : 0;
    c += n[i];
  }
  // W panels (solve_w_depth) by default only for single matrices: a batch of
  // small trees would form W for most of its panels
  spchol_options bo;
  if (opt) {
    bo = *opt;
  } else {
    spchol::default_options(&bo);
  }
  if (bo.solve_w_depth == 0) bo.solve_w_depth = -1;
  int rc = spchol_analyze(N, cp.data(), ri.data(), pm.data(), &bo, out);
  if (rc < 0 && rc > -100) {
    // map the combined call's argument positions back to this call's
    const int map[7] = {0, -2, -3, -4, -5, -6, -7};
    return map[-rc];
  }
  if (rc) return rc;
  (*out)->batch_count = count;
  (*out)->batch_n.assign(n, n + count);
  (*out)->batch_col0 = col0;
  (*out)->batch_nnz0 = nnz0;
  return 0;
}

int spchol_batch_factorize(spchol_handle_t h, const double* const* values, void* stream) {
  if (!h || h->batch_count == 0) return -1;
  if (!values) return -2;
  DeviceGuard g(h->device);
  clear_stale_error();
  cudaStream_t st = (cudaStream_t)stream;
  const int cnt = h->batch_count;
  for (int i = 0; i < cnt; ++i) {
    const int64_t len = (i + 1 < cnt ? h->batch_nnz0[i + 1] : h->plan.nnz_a) - h->batch_nnz0[i];
    if (len == 0) continue;
    if (!values[i]) return -2;
    const bool dev = is_device_ptr(values[i]);
    CU(cudaMemcpyAsync(h->d_vals + h->batch_nnz0[i], values[i], len * sizeof(double),
                       dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
  }
  return factorize_impl(h, h->d_vals, nullptr, st);
}

int spchol_batch_solve(spchol_handle_t h, double* const* B, const int64_t* ldb, const int* nrhs, void* stream) {
  if (!h || h->batch_count == 0) return -1;
  if (!B) return -2;
  if (!ldb) return -3;
  if (!nrhs) return -4;
  if (!h->factored) return SPCHOL_ESTATE;
  DeviceGuard g(h->device);
  cudaStream_t st = (cudaStream_t)stream;
  const int cnt = h->batch_count;
  int maxr = 0;
  for (int i = 0; i < cnt; ++i) {
    if (nrhs[i] < 0) return -4;
    if (ldb[i] < std::max<int64_t>(h->batch_n[i], 1)) return -3;
    maxr = std::max(maxr, nrhs[i]);
  }
  if (maxr == 0) return 0;
  const int64_t N = h->plan.n;
  int rc = ensure_workspace(h, N * maxr, maxr, st);
  if (rc) return rc;
  // Gather every matrix's RHS into one N x maxr block (zero columns where a
  // matrix has fewer right-hand sides), solve once, scatter back.
  CU(cudaMemsetAsync(h->d_B, 0, N * maxr * sizeof(double), st));
  for (int i = 0; i < cnt; ++i) {
    if (nrhs[i] == 0 || h->batch_n[i] == 0) continue;
    const bool dev = is_device_ptr(B[i]);
    CU(cudaMemcpy2DAsync(h->d_B + h->batch_col0[i], N * sizeof(double), B[i], ldb[i] * sizeof(double),
                         h->batch_n[i] * sizeof(double), nrhs[i],
                         dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
  }
  CU(cudaEventRecord(h->ev0, st));
  int core = 0;
  if (h->fp32) {
    core = solve_refined(h, maxr, st);
    if (core != 0 && core != SPCHOL_ENOCONV) return core;
  } else {
    CU(launch_permute_in(h->d_B, N, h->d_Y, N, h->d_perm, N, maxr, st));
    rc = solve_permuted(h, h->d_Y, maxr, st);
    if (rc) return rc;
    CU(launch_permute_out(h->d_Y, N, h->d_B, N, h->d_perm, N, maxr, st));
  }
  CU(cudaEventRecord(h->ev1, st));
  for (int i = 0; i < cnt; ++i) {
    if (nrhs[i] == 0 || h->batch_n[i] == 0) continue;
    const bool dev = is_device_ptr(B[i]);
    CU(cudaMemcpy2DAsync(B[i], ldb[i] * sizeof(double), h->d_B + h->batch_col0[i], N * sizeof(double),
                         h->batch_n[i] * sizeof(double), nrhs[i],
                         dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
  }
  CU(cudaStreamSynchronize(st));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, h->ev0, h->ev1);
  h->stats.solve_ms = ms;
  return core;
}

int spchol_batch_info(spchol_handle_t h, int64_t k, int* matrix, int64_t* column) {
  if (!h || h->batch_count == 0) return -1;
  if (k < 1 || k > h->plan.n) return -2;
  // k is a permuted column of the block-diagonal system; the permutation keeps
  // each matrix's columns inside its own block.
  const int64_t orig = h->plan.perm[k - 1];
  int i = (int)(std::upper_bound(h->batch_col0.begin(), h->batch_col0.end(), orig) - h->batch_col0.begin()) - 1;
  // position of column k within matrix i's permuted order: count columns of
  // matrix i that precede k in the permuted order
  int64_t pos = 0;
  for (int64_t c = 0; c < k - 1; ++c) {
    const int64_t o = h->plan.perm[c];
    if (o >= h->batch_col0[i] && o < h->batch_col0[i] + h->batch_n[i]) ++pos;
  }
  if (matrix) *matrix = i;
  if (column) *column = pos + 1;
  return 0;
}

}  // extern "C"
