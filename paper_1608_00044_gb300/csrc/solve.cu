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
  int hold;  // this CTA holds a claimed, still empty ring slot: no continuation
};

template <typename T>
__device__ __forceinline__ const T* spanel(const SolveArgs& a, int s) {
  return reinterpret_cast<const T*>(a.pool) + a.pv.valoff[s];
}

// W panels (Plan::woff) keep W = L21 L11^{-1}, stored like the panel.
__device__ __forceinline__ bool is_wpanel(const SolveArgs& a, int s) { return a.woff != nullptr && a.woff[s] >= 0; }

// The operand of a panel's solve tiles: W for a W panel, else the panel (L21).
template <typename T>
__device__ __forceinline__ const T* tile_operand(const SolveArgs& a, int s) {
  return is_wpanel(a, s) ? reinterpret_cast<const T*>(a.wbuf) + a.woff[s] : spanel<T>(a, s);
}

// ---------------------------------------------------------------- FP64 products on the BF16 tensor cores
// The panel tiles' products C = A B (A: up to 64 x 64 of L21 or its
// transpose, B: up to 64 x 8 right-hand sides) cost w FP64 FMAs per output,
// and the FP64 pipe retires 2 FMAs per clock per SM.  For FP64 panels 16 to 64
// wide they run instead as exact integer products on the BF16 tensor
// cores (the splitting of Ozaki, Ogita, Oishi and Rump, "Error-free
// transformations of matrix multiplication by using fast routines of matrix
// multiplication", Numer. Algorithms 2012): with e_i the smallest integer such
// that every |A_ik| of row i is below 2^e_i, A_ik 2^(56 - e_i) truncated to an
// integer q_ik < 2^56 is cut into kOzSl 8-bit digits; digit p, with the sign of
// A_ik, is an integer in [-255, 255] (exact in BF16) of weight
// 2^(e_i - 8(p + 1)).  B is split the same way per column.  Products of digit
// p of A and digit q of B with p + q = d are summed (mma.sync m16n8k8, FP32
// accumulation) into group d; for K <= 64 a group d <= 3 stays below 2^24 and
// is exact, the others round at most 2^-56 relative to the leading group.
// Products with p + q >= kOzSl weigh below 2^-56 and are dropped.  The seven
// group sums are combined exactly into two integers and converted to FP64 with
// one rounding.  The result differs from the exact product by at most a few
// units of 2^-56 max_k|A_ik| max_k|B_kj| K, the size of an FP64 dot
// product's own rounding bound.
constexpr int kOzSl = 7;     // digits per value
constexpr int kOzLda = 65;   // staged A: row m at As[m * kOzLda] (odd: no bank conflicts down a column)
constexpr int kOzBLd = 72;   // staged B digits: (slice q, column n) row of 64 + 8 BF16 (no bank conflicts)
constexpr int kOzMaxK = 64;  // K and M of one pass (the exactness bound above)
constexpr int kOzMinW = 16;  // narrower panels keep the FP64 FMA path (their products are tiny)

struct OzBuf {
  double* As;   // [64][kOzLda]; its first 14 KB also hold the second K half's group sums
  double* Bs;   // [8][64]: B column n at Bs[n * 64]
  uint16_t* Bd; // [kOzSl][8][kOzBLd]
  int* eA;      // [64] biased exponent bits of each A row's largest entry (0: zero row)
  int* eB;      // [8]
};

__device__ __forceinline__ OzBuf oz_carve(double* sm) {
  OzBuf b;
  b.As = sm;
  b.Bs = b.As + 64 * kOzLda;
  b.Bd = reinterpret_cast<uint16_t*>(b.Bs + 8 * 64);
  b.eA = reinterpret_cast<int*>(b.Bd + kOzSl * 8 * kOzBLd);
  b.eB = b.eA + 64;
  return b;
}

constexpr size_t kOzSmemBytes =
    (64 * kOzLda + 8 * 64) * sizeof(double) + kOzSl * 8 * kOzBLd * sizeof(uint16_t) + 72 * sizeof(int);

__device__ __forceinline__ int exp_bits(double x) { return (int)((__double_as_longlong(x) >> 52) & 0x7FF); }

// |x| 2^(56 - e), e = emax - 1022, truncated to an integer below 2^56, as its
// bits 32..55 (hi) and 0..31 (lo).  emax: the biased exponent bits of the
// largest |x| of the row; subnormal x count as zero.
__device__ __forceinline__ void oz_fix(double x, int emax, uint32_t& hi, uint32_t& lo) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int ex = (int)((b >> 52) & 0x7FF);
  unsigned long long q = 0ull;
  if (ex != 0) {
    const unsigned long long mant = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    const int sh = ex - emax + 3;  // at most 3
    q = sh >= 0 ? (mant << sh) : (sh > -64 ? (mant >> (-sh)) : 0ull);
  }
  hi = (uint32_t)(q >> 32);
  lo = (uint32_t)q;
}

// Digit p (0 most significant) of the 56-bit integer (hi, lo).
template <int P>
__device__ __forceinline__ uint32_t oz_digit(uint32_t hi, uint32_t lo) {
  if constexpr (P < 3)
    return (hi >> (16 - 8 * P)) & 0xFFu;
  else
    return (lo >> (24 - 8 * (P - 3))) & 0xFFu;
}

// Two digits d0, d1 < 256 as a BF16 pair (d0 in the low half), signs from
// sgn (bit 15: d0, bit 31: d1).  2^23 + d is exact in FP32 and subtracting
// 2^23 leaves d, whose FP32 bits have zeros in their low half: the high half is
// d in BF16.
__device__ __forceinline__ uint32_t oz_pair(uint32_t d0, uint32_t d1, uint32_t sgn) {
  const float f0 = __uint_as_float(0x4B000000u | d0) - 8388608.0f;
  const float f1 = __uint_as_float(0x4B000000u | d1) - 8388608.0f;
  return __byte_perm(__float_as_uint(f0), __float_as_uint(f1), 0x7632) ^ sgn;
}

__device__ __forceinline__ uint32_t oz_signs(double x0, double x1) {
  return ((uint32_t)((unsigned long long)__double_as_longlong(x0) >> 63) << 15) |
         ((uint32_t)((unsigned long long)__double_as_longlong(x1) >> 63) << 31);
}

__device__ __forceinline__ void mma_bf16_1688(float (&c)[4], uint32_t a0, uint32_t a1, uint32_t b0) {
  asm volatile("mma.sync.aligned.m16n8k8.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5}, {%6}, {%0,%1,%2,%3};"
               : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
               : "r"(a0), "r"(a1), "r"(b0));
}

// One warp: the group sums of the 16 x 8 block of C whose rows are m0 .. m0+15,
// over the k blocks kb0 <= kb < kb1 of 16, each as two m16n8k8 steps.
// Fragment layout of m16n8k8 (g = lane / 4, t = lane % 4): A elements (g |
// g+8, 2t | 2t+1), B elements (2t | 2t+1, g), C elements acc[d][0..3] at (g,
// 2t), (g, 2t+1), (g+8, 2t), (g+8, 2t+1).
__device__ __forceinline__ void oz_block(const OzBuf& b, int m0, int kb0, int kb1, float (&acc)[kOzSl][4]) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const int e0 = b.eA[m0 + g], e1 = b.eA[m0 + g + 8];
  const double* r0 = b.As + (m0 + g) * kOzLda + 2 * t;
  const double* r1 = b.As + (m0 + g + 8) * kOzLda + 2 * t;
  const uint16_t* bg = b.Bd + g * kOzBLd + 2 * t;
  for (int k8 = 2 * kb0; k8 < 2 * kb1; ++k8) {
    const int c0 = 8 * k8;
    const double x[4] = {r0[c0], r0[c0 + 1], r1[c0], r1[c0 + 1]};
    // hi carries the sign in bit 31 (its digits use bits 0..23)
    uint32_t hi[4], lo[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      oz_fix(x[e], (e & 2) ? e1 : e0, hi[e], lo[e]);
      hi[e] |= (uint32_t)((unsigned long long)__double_as_longlong(x[e]) >> 63) << 31;
    }
    const uint16_t* bk = bg + c0;
#define SPCHOL_OZ_SLICE(P)                                                                               \
  {                                                                                                     \
    uint32_t a0 = oz_pair(oz_digit<P>(hi[0], lo[0]), oz_digit<P>(hi[1], lo[1]),                          \
                          ((hi[0] >> 31) << 15) | (hi[1] & 0x80000000u));                               \
    uint32_t a1 = oz_pair(oz_digit<P>(hi[2], lo[2]), oz_digit<P>(hi[3], lo[3]),                          \
                          ((hi[2] >> 31) << 15) | (hi[3] & 0x80000000u));                               \
    _Pragma("unroll") for (int q = 0; q < kOzSl - P; ++q)                                               \
        mma_bf16_1688(acc[P + q], a0, a1, *reinterpret_cast<const uint32_t*>(bk + q * 8 * kOzBLd));      \
  }
    SPCHOL_OZ_SLICE(0)
    SPCHOL_OZ_SLICE(1)
    SPCHOL_OZ_SLICE(2)
    SPCHOL_OZ_SLICE(3)
    SPCHOL_OZ_SLICE(4)
    SPCHOL_OZ_SLICE(5)
    SPCHOL_OZ_SLICE(6)
#undef SPCHOL_OZ_SLICE
  }
}

// Exact integer x (|x| < 2^51) as a double: x + 2^52 + 2^51 in the mantissa field.
__device__ __forceinline__ double oz_i2d(long long x) {
  return __longlong_as_double(x + 0x4338000000000000LL) - 6755399441055744.0;
}

// The value of output c of this thread: t = sum_d G_d 2^(8 (6 - d)) (G_0..G_2
// and G_3..G_6 combined exactly in two integers below 2^42 and 2^50, one
// rounding in the final FMA), times 2^(ea + eb - 2108) for the biased
// exponent bits ea, eb of the row of A and the column of B.
__device__ __forceinline__ double oz_value(const float (&acc)[kOzSl][4], int c, int ea, int eb) {
  if (ea == 0 || eb == 0) return 0.0;
  long long h = __float2int_rn(acc[0][c]);
  h = h * 256 + __float2int_rn(acc[1][c]);
  h = h * 256 + __float2int_rn(acc[2][c]);
  long long l = __float2int_rn(acc[3][c]);
  l = l * 256 + __float2int_rn(acc[4][c]);
  l = l * 256 + __float2int_rn(acc[5][c]);
  l = l * 256 + __float2int_rn(acc[6][c]);
  const double tv = fma(oz_i2d(h), 4294967296.0, oz_i2d(l));
  const int E = ea + eb - 2108;
  if (E >= -1022 && E <= 1023) return tv * __longlong_as_double((long long)(E + 1023) << 52);
  return ldexp(tv, E);
}

// Digits of the staged B (K x 8, K <= 64, column n at Bs[n * 64]) into Bd,
// with each column's exponent in eB; entries k >= K (up to K rounded up to 16)
// are zero.  All threads; ends with a barrier.
__device__ __forceinline__ void oz_split_b(const OzBuf& b, int K) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int kpad = (K + 15) & ~15;
  for (int n = warp; n < 8; n += kSolveThreads / 32) {
    int e = 0;
    for (int k = lane; k < K; k += 32) e = max(e, exp_bits(b.Bs[n * 64 + k]));
    e = (int)__reduce_max_sync(0xffffffffu, (unsigned)e);
    if (lane == 0) b.eB[n] = e;
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < 8 * (kpad / 2); idx += blockDim.x) {
    const int n = idx / (kpad / 2), k = 2 * (idx - n * (kpad / 2));
    const double x0 = k < K ? b.Bs[n * 64 + k] : 0.0, x1 = k + 1 < K ? b.Bs[n * 64 + k + 1] : 0.0;
    uint32_t h0, l0, h1, l1;
    oz_fix(x0, b.eB[n], h0, l0);
    oz_fix(x1, b.eB[n], h1, l1);
    const uint32_t sg = oz_signs(x0, x1);
    uint32_t* dst = reinterpret_cast<uint32_t*>(b.Bd + n * kOzBLd + k);
    dst[0 * 8 * kOzBLd / 2] = oz_pair(oz_digit<0>(h0, l0), oz_digit<0>(h1, l1), sg);
    dst[1 * 8 * kOzBLd / 2] = oz_pair(oz_digit<1>(h0, l0), oz_digit<1>(h1, l1), sg);
    dst[2 * 8 * kOzBLd / 2] = oz_pair(oz_digit<2>(h0, l0), oz_digit<2>(h1, l1), sg);
    dst[3 * 8 * kOzBLd / 2] = oz_pair(oz_digit<3>(h0, l0), oz_digit<3>(h1, l1), sg);
    dst[4 * 8 * kOzBLd / 2] = oz_pair(oz_digit<4>(h0, l0), oz_digit<4>(h1, l1), sg);
    dst[5 * 8 * kOzBLd / 2] = oz_pair(oz_digit<5>(h0, l0), oz_digit<5>(h1, l1), sg);
    dst[6 * 8 * kOzBLd / 2] = oz_pair(oz_digit<6>(h0, l0), oz_digit<6>(h1, l1), sg);
  }
  __syncthreads();
}

// C = A B for the staged A (M x K, M, K <= 64, zero past M and K up to their
// multiples of 16) and the split B: out(c, m, n, value) for every output m < M,
// n < nrc, called by the thread that owns it (c: its slot 0..3, fixed per
// thread for a given M and K).  Warps w and w + 4 take m block w % 4 and the
// lower and upper halves of the k blocks; the upper half's group sums are
// added exactly to the lower's through shared memory (they are integers with
// an exact sum below 2^24 in the exact groups).  All threads; begins after the
// staging barrier and ends with one; A is overwritten.
template <class Out>
__device__ __forceinline__ void oz_product(const OzBuf& b, int M, int K, int nrc, Out out) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // row exponents: warp w takes rows w, w + 8, ...
  for (int m = warp; m < M; m += kSolveThreads / 32) {
    int e = 0;
    for (int k = lane; k < K; k += 32) e = max(e, exp_bits(b.As[m * kOzLda + k]));
    e = (int)__reduce_max_sync(0xffffffffu, (unsigned)e);
    if (lane == 0) b.eA[m] = e;
  }
  __syncthreads();
  const int mb = warp & 3, half = warp >> 2, m0 = 16 * mb;
  const int nkb = (K + 15) >> 4, split = (nkb + 1) >> 1;
  float acc[kOzSl][4];
#pragma unroll
  for (int d = 0; d < kOzSl; ++d)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[d][c] = 0.0f;
  const bool active = m0 < M;
  if (active) oz_block(b, m0, half ? split : 0, half ? nkb : split, acc);
  __syncthreads();  // A is read; its space takes the upper half's sums
  float* gx = reinterpret_cast<float*>(b.As) + (size_t)mb * (kOzSl * 4 * 32);
  if (active && half && split < nkb) {
#pragma unroll
    for (int d = 0; d < kOzSl; ++d)
#pragma unroll
      for (int c = 0; c < 4; ++c) gx[(d * 4 + c) * 32 + lane] = acc[d][c];
  }
  __syncthreads();
  if (active && !half) {
    if (split < nkb) {
#pragma unroll
      for (int d = 0; d < kOzSl; ++d)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[d][c] += gx[(d * 4 + c) * 32 + lane];
    }
    const int g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int m = m0 + g + ((c & 2) ? 8 : 0), n = 2 * t + (c & 1);
      if (m < M && n < nrc) out(c, m, n, oz_value(acc, c, b.eA[m], b.eB[n]));
    }
  }
  __syncthreads();
}

// Zero the staged A outside its M x K corner, up to 64 rows and K rounded up to 16.
__device__ __forceinline__ void oz_zero_pad(const OzBuf& b, int M, int K) {
  const int kpad = (K + 15) & ~15, mpad = (M + 15) & ~15;
  for (int idx = threadIdx.x; idx < mpad * kpad; idx += blockDim.x) {
    const int m = idx / kpad, k = idx - m * kpad;
    if (m >= M || k >= K) b.As[m * kOzLda + k] = 0.0;
  }
}

// dst(i, src(i)) for i < total, the loads issued in batches of 8 per thread so
// that their latencies overlap (a load followed by its store, one at a time,
// costs a full memory round trip per element).
template <class Src, class Dst>
__device__ __forceinline__ void copy_batched(int total, Src src, Dst dst) {
  for (int base = threadIdx.x; base < total; base += 8 * blockDim.x) {
    double v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int idx = base + u * blockDim.x;
      v[u] = idx < total ? src(idx) : 0.0;
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int idx = base + u * blockDim.x;
      if (idx < total) dst(idx, v[u]);
    }
  }
}

// ---------------------------------------------------------------- asynchronous staging of the factor
// The factor (the panels and the diagonal-block inverses) was written by the
// factorization, an earlier launch, and is only read here, so it may come
// through L1.  Element-sized cp.async copies put every load of a block in
// flight at once (a thread issues them all before waiting), where plain loads
// in batches of eight cost one memory round trip per batch, and they allow an
// odd leading dimension in shared memory, which keeps both a row walk and a
// column walk free of bank conflicts.
__device__ __forceinline__ uint32_t sm_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }


template <typename T>
__device__ __forceinline__ void cp_async_elem(T* dst, const T* src) {
  if constexpr (sizeof(T) == 8)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(sm_u32(dst)), "l"(src) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(sm_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit_group() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait_group() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// L11^{-1} (w x w, column-major) into shared memory with leading dimension lx,
// all copies in flight; the caller commits, waits and synchronises.  Only the
// lower triangle is read later.
__device__ __forceinline__ void stage_inverse(const double* __restrict__ X, int w, double* __restrict__ Xs, int lx) {
  const int total = w * w;
  for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
    const int i = idx % w, j = idx / w;
    if (i >= j) cp_async_elem(Xs + i + j * lx, X + idx);
  }
  cp_async_commit_group();
}

// Rows row0 .. row0 + cnt - 1 of the w columns of a column-major panel into
// Ls[i + j * lds]; the caller commits.
template <typename T>
__device__ __forceinline__ void stage_rows(const T* __restrict__ P, int ld, int row0, int cnt, int w, T* Ls, int lds) {
  for (int idx = threadIdx.x; idx < cnt * w; idx += blockDim.x) {
    const int i = idx % cnt, j = idx / cnt;
    cp_async_elem(Ls + i + j * lds, P + row0 + i + (size_t)j * ld);
  }
}

// Stage y_s (w entries of right-hand sides r0 .. r0+nrc-1) as the B operand.
__device__ __forceinline__ void oz_stage_ys(const SolveArgs& a, const OzBuf& b, int f, int w, int r0, int nrc) {
  const double* Y = a.Y + f + (size_t)r0 * a.ldy;
  const int64_t ldy = a.ldy;
  copy_batched(
      8 * w,
      [&](int idx) {
        const int n = idx / w;
        return n < nrc ? ldcg(Y + (idx - n * w) + n * ldy) : 0.0;
      },
      [&](int idx, double v) {
        const int n = idx / w;
        b.Bs[n * 64 + (idx - n * w)] = v;
      });
}

// ---------------------------------------------------------------- fan-in gathers
// Fan-in mode (the fan-in family of Section II-C, restated for the solves):
// the tiles store their products in private buffers and the diagonal tasks
// add them, in tile order, into the right-hand sides they stage in shared
// memory.  Forward: the tiles with rows in the panel's columns, up to
// kSolveFanBatch list entries at a time: warp 0 cuts the batch where its
// values would overflow the staging area (the entries' records were fetched
// during the previous batch); all threads load the batch's values (eight
// loads in flight each) and map each entry's rows to the panel's columns;
// then each thread adds, for the (column, right-hand side) entries it owns,
// the batch's values in order from shared memory.  Backward: the panel's own
// tiles, each thread summing its entries' values over the tiles in order.
using SolveFanRec = Plan::SolveFanRec;
constexpr int kSolveFanBatch = 32;
constexpr int kSolveFanVals = 2048;  // staged values per batch (an entry has at most 64 x 8)
struct SolveFanMeta {
  long long zo, ro;  // the entry's first value of this pass in the buffer; its first row in the row lists
  int cnt, ni, pre;  // the tile's rows; the entry's rows; its first staged value
  float inv_ni;      // 1 / ni: value index -> (row, right-hand side) without a division
};
constexpr size_t solve_fan_smem_bytes(int max_w) {
  return kSolveFanBatch * sizeof(SolveFanMeta) + 16 + (((size_t)kSolveFanBatch * max_w * sizeof(int16_t) + 15) & ~size_t(15)) +
         kSolveFanVals * sizeof(double);
}

__device__ void fwd_gather(const SolveArgs& a, int s, int f, int w, double* Ys, int r0, int nrc, unsigned char* ex) {
  const int tid = threadIdx.x, nt = blockDim.x;
  SolveFanMeta* meta = reinterpret_cast<SolveFanMeta*>(ex);
  int* scal = reinterpret_cast<int*>(meta + kSolveFanBatch);  // entries and values of the batch
  int16_t* inv = reinterpret_cast<int16_t*>(scal + 4);        // [batch entry][column]: its row, or -1
  double* Bv = reinterpret_cast<double*>(reinterpret_cast<unsigned char*>(inv) +
                                         (((size_t)kSolveFanBatch * w * sizeof(int16_t) + 15) & ~size_t(15)));
  const int e0 = a.rt_ptr[s], e1 = a.rt_ptr[s + 1];
  // ascending tile order: the list from its end; warp 0 holds the next window's records
  SolveFanRec rec{};
  if (tid < 32 && e1 - 1 - tid >= e0) rec = a.rt_rec[e1 - 1 - tid];
  for (int eb = e1; eb > e0;) {
    __syncthreads();  // the right-hand sides are staged, or the previous batch is added
    for (int idx = tid; idx < kSolveFanBatch * w; idx += nt) inv[idx] = -1;
    if (tid < 32) {
      const bool have = eb - 1 - tid >= e0;
      const int n = have ? rec.ni * nrc : 0;
      int in = n;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, in, o);
        if (tid >= o) in += y;
      }
      const int nb = max(1, __popc(__ballot_sync(0xffffffffu, have && in <= kSolveFanVals)));
      if (tid < nb) {
        SolveFanMeta m;
        m.zo = rec.z * a.nrhs + rec.i0 + (long long)r0 * rec.cnt;
        m.ro = rec.ro;
        m.cnt = rec.cnt;
        m.ni = rec.ni;
        m.pre = in - n;
        m.inv_ni = 1.0f / (float)max(1, (int)rec.ni);
        meta[tid] = m;
      }
      if (tid == nb - 1) {
        scal[0] = nb;
        scal[1] = in;
      }
      rec = SolveFanRec{};
      if (eb - nb - 1 - tid >= e0) rec = a.rt_rec[eb - nb - 1 - tid];  // in flight during this batch
    }
    __syncthreads();
    const int nb = scal[0];
    int total = scal[1];
    if (total > kSolveFanVals) {  // cannot happen for a consistent plan
      if (tid == 0) atomicCAS(&a.ctrl[kErr], 0, SPCHOL_DEV_EINTERNAL);
      total = 0;
    }
    // the entries' rows mapped to the panel's columns ...
    for (int idx = tid; idx < nb * w; idx += nt) {
      const int b = idx / w, i = idx - b * w;
      if (i < meta[b].ni) {
        const int c = __ldg(a.pv.rows + meta[b].ro + i) - f;
        if (c >= 0 && c < w)
          inv[b * w + c] = (int16_t)i;
        else
          atomicCAS(&a.ctrl[kErr], 0, SPCHOL_DEV_EINTERNAL);
      }
    }
    // ... and their values, eight loads in flight per thread
    for (int v0 = 0; v0 < total; v0 += 8 * nt) {
      double v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int idx = v0 + u * nt + tid;
        v[u] = 0.0;
        if (idx < total) {
          int b = 0;
#pragma unroll
          for (int h = kSolveFanBatch / 2; h > 0; h >>= 1)
            if (b + h < nb && meta[b + h].pre <= idx) b += h;
          const int lv = idx - meta[b].pre;
          // lv / ni exactly: lv < 2^9 and ni <= 64 leave a margin of 1 / 128 for rounding
          const int r = (int)(((float)lv + 0.5f) * meta[b].inv_ni), i = lv - r * meta[b].ni;
          v[u] = ldcg(a.zf + meta[b].zo + i + (size_t)r * meta[b].cnt);
        }
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int idx = v0 + u * nt + tid;
        if (idx < total) Bv[idx] = v[u];
      }
    }
    __syncthreads();
    for (int p = tid; p < w * nrc; p += nt) {
      const int c = p % w, r = p / w;
      double y = Ys[p];
      for (int b = 0; b < nb; ++b) {
        const int i = inv[b * w + c];
        if (i >= 0) y += Bv[meta[b].pre + r * meta[b].ni + i];
      }
      Ys[p] = y;
    }
    eb -= nb;
  }
  __syncthreads();
}

__device__ void bwd_gather(const SolveArgs& a, int s, int w, double* Ys, int r0, int nrc) {
  const int nk = a.nst[s];
  const double* z0 = a.zb + a.st_zb[a.st_first[s]] * a.nrhs;  // the panel's tiles' buffers, w x nrhs each
  for (int p = threadIdx.x; p < w * nrc; p += blockDim.x) {
    const int j = p % w, r = p / w;
    const double* z = z0 + j + (size_t)(r0 + r) * w;
    double y = Ys[p];
    for (int k0 = 0; k0 < nk; k0 += 8) {
      double v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) v[u] = k0 + u < nk ? ldcg(z + (size_t)(k0 + u) * w * a.nrhs) : 0.0;
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if (k0 + u < nk) y += v[u];
    }
    Ys[p] = y;
  }
  __syncthreads();
}

// Lanes per dot product of the diagonal solves: the 256 threads cover
// (w / 2) row pairs x nrc right-hand sides x P parts.
__device__ __forceinline__ int diag_parts(int nrc) { return nrc == 1 ? 8 : nrc == 2 ? 4 : nrc <= 4 ? 2 : 1; }

// The products of the diagonal solves with the stored inverse X = L11^{-1}
// (staged at Xs, column-major with leading dimension lx, lower part): every
// entry is an independent dot product, no sequential substitution.  TR =
// false: L11^{-1} y, entry i the dot product of row i of X (columns 0 .. i)
// with y; TR = true: L11^{-T} y, entry k that of column k of X (rows k .. w-1).
// y: nrc right-hand sides at Ys [nrc][w].  Lanes (r, c, q) compute entries c
// and w - 1 - c for right-hand side r, terms k = q mod P: w + 1 terms in all,
// so every thread and warp does the same work.  With few right-hand sides each
// dot product is split over P lanes, so that every warp -- and every
// sub-partition's FP64 pipe -- takes a share; the parts meet by shuffles
// within the P lanes.  out(i, r, value) is called by one lane per entry.
template <bool TR, class Out>
__device__ __forceinline__ void diag_product(const double* Xs, int lx, int w, const double* Ys, int nrc, Out out) {
  const int half = (w + 1) >> 1;
  const int P = diag_parts(nrc);
  const int total = (half * nrc * P + 31) & ~31;  // whole warps: every lane takes part in the shuffles
  for (int p = threadIdx.x; p < total; p += blockDim.x) {
    const int q = p % P, cr = p / P, c = cr % half, r = cr / half;
    const bool valid = cr < half * nrc;
    const double* y = Ys + r * w;
    const int i1 = c, i2 = w - 1 - c;
    double a0 = 0.0, b0 = 0.0;
    if (valid) {
      double a1 = 0.0, b1 = 0.0;
      if constexpr (!TR) {
        int k = q;
        for (; k + P <= i1; k += 2 * P) {
          a0 += Xs[i1 + k * lx] * y[k];
          a1 += Xs[i1 + (k + P) * lx] * y[k + P];
        }
        if (k <= i1) a0 += Xs[i1 + k * lx] * y[k];
        if (i2 != i1) {
          for (k = q; k + P <= i2; k += 2 * P) {
            b0 += Xs[i2 + k * lx] * y[k];
            b1 += Xs[i2 + (k + P) * lx] * y[k + P];
          }
          if (k <= i2) b0 += Xs[i2 + k * lx] * y[k];
        }
      } else {
        const double* x1 = Xs + i1 * lx;
        int i = i1 + q;
        for (; i + P < w; i += 2 * P) {
          a0 += x1[i] * y[i];
          a1 += x1[i + P] * y[i + P];
        }
        if (i < w) a0 += x1[i] * y[i];
        if (i2 != i1) {
          const double* x2 = Xs + i2 * lx;
          for (i = i2 + q; i + P < w; i += 2 * P) {
            b0 += x2[i] * y[i];
            b1 += x2[i + P] * y[i + P];
          }
          if (i < w) b0 += x2[i] * y[i];
        }
      }
      a0 += a1;
      b0 += b1;
    }
    for (int d = 1; d < P; d <<= 1) {
      a0 += __shfl_xor_sync(0xffffffffu, a0, d);
      b0 += __shfl_xor_sync(0xffffffffu, b0, d);
    }
    if (valid && q == 0) {
      out(i1, r, a0);
      if (i2 != i1) out(i2, r, b0);
    }
  }
}

// y_s <- L11^{-1} y_s (forward) or L11^{-T} y_s (backward, TR) with the
// inverse formed by the diagonal factor task.
template <bool TR, bool FAN>
__device__ void diag_solve(const SolveArgs& a, int s, double* sm) {
  const int f = a.pv.fcol[s], w = a.pv.fcol[s + 1] - f;
  const double* X = a.inv + a.invoff[s];
  const int lx = w + 1;           // padded: lanes that walk a row or a column both avoid bank conflicts
  double* Xs = sm;                // [w][lx] column-major, lower part
  double* Ys = sm + w * lx;       // [nrc][w]
  stage_inverse(X, w, Xs, lx);
  for (int r0 = 0; r0 < a.nrhs; r0 += kSolveNRC) {
    const int nrc = min(kSolveNRC, a.nrhs - r0);
    __syncthreads();
    for (int idx = threadIdx.x; idx < w * nrc; idx += blockDim.x) {
      const int j = idx % w, r = idx / w;
      Ys[idx] = ldcg(a.Y + f + j + (size_t)(r0 + r) * a.ldy);
    }
    if constexpr (FAN) {
      if constexpr (TR) {
        __syncthreads();
        bwd_gather(a, s, w, Ys, r0, nrc);
      } else {
        fwd_gather(a, s, f, w, Ys, r0, nrc, reinterpret_cast<unsigned char*>(Ys + kSolveNRC * w));
      }
    }
    cp_async_wait_group<0>();  // the inverse (first pass)
    __syncthreads();
    double* Y = a.Y + f + (size_t)r0 * a.ldy;
    const int64_t ldy = a.ldy;
    diag_product<TR>(Xs, lx, w, Ys, nrc, [&](int i, int r, double v) { Y[i + r * ldy] = v; });
  }
}

// The diagonal task of a W panel (Plan::woff): y_s <- L11^{-T} L11^{-1} b_s,
// the product with L11^{-1} kept in shared memory (Ts) for the second.
__device__ void diag_solve_w(const SolveArgs& a, int s, double* sm) {
  const int f = a.pv.fcol[s], w = a.pv.fcol[s + 1] - f;
  const double* X = a.inv + a.invoff[s];
  const int lx = w + 1;
  double* Xs = sm;                      // [w][lx]
  double* Ys = sm + w * lx;             // [nrc][w]
  double* Ts = Ys + kSolveNRC * w;      // [nrc][w]: L11^{-1} b_s
  stage_inverse(X, w, Xs, lx);
  for (int r0 = 0; r0 < a.nrhs; r0 += kSolveNRC) {
    const int nrc = min(kSolveNRC, a.nrhs - r0);
    __syncthreads();
    for (int idx = threadIdx.x; idx < w * nrc; idx += blockDim.x) {
      const int j = idx % w, r = idx / w;
      Ys[idx] = ldcg(a.Y + f + j + (size_t)(r0 + r) * a.ldy);
    }
    cp_async_wait_group<0>();
    __syncthreads();
    diag_product<false>(Xs, lx, w, Ys, nrc, [&](int i, int r, double v) { Ts[i + r * w] = v; });
    __syncthreads();
    double* Y = a.Y + f + (size_t)r0 * a.ldy;
    const int64_t ldy = a.ldy;
    diag_product<true>(Xs, lx, w, Ts, nrc, [&](int i, int r, double v) { Y[i + r * ldy] = v; });
  }
}

// ---------------------------------------------------------------- panel tiles on the FP64 / FP32 pipes
// A tile's rows go through shared memory in chunks of kTileCH rows, double
// buffered: the copies of chunk c + 1 are in flight while chunk c is used.
// The work of a chunk is spread over the eight warps by right-hand side and,
// when there are fewer than eight right-hand sides, by a split of the dot
// products' range (parts = 8 / the right-hand sides rounded up to a power of
// two), whose partial sums meet in shared memory.
constexpr int kTileCH = 32;          // rows per chunk: one per lane
constexpr int kTileLD = kTileCH + 1;  // odd: a lane per row or a lane per column, both conflict free

__device__ __forceinline__ int tile_groups(int nrc) { return nrc > 4 ? 8 : nrc > 2 ? 4 : nrc > 1 ? 2 : 1; }

// y[rows of tile] -= L21[tile] y_s.  Warp wp takes right-hand side wp % G and
// part wp / G of the columns; lane i the chunk's row i.
template <typename T, bool FAN>
__device__ void fwd_tile_fma(const SolveArgs& a, const T* P, int ld, int row0, int cnt, const int32_t* R, int f,
                             int w, double* sm, double* z) {
  double* Ys = sm;                                                   // [kSolveNRC][w]
  double* Red = Ys + kSolveNRC * w;                                  // [8][kTileCH] partial sums
  T* Lb = reinterpret_cast<T*>(Red + 8 * kTileCH);                   // [2][w][kTileLD]
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nchunk = (cnt + kTileCH - 1) / kTileCH;
  for (int r0 = 0; r0 < a.nrhs; r0 += kSolveNRC) {
    const int nrc = min(kSolveNRC, a.nrhs - r0);
    const int G = tile_groups(nrc), parts = 8 / G;
    const int g = warp % G, part = warp / G;
    const int k0 = part * w / parts, k1 = (part + 1) * w / parts;
    __syncthreads();  // the previous pass is done with Ys and the buffers
    stage_rows(P, ld, row0, min(kTileCH, cnt), w, Lb, kTileLD);
    cp_async_commit_group();
    for (int idx = threadIdx.x; idx < w * nrc; idx += blockDim.x) {
      const int j = idx % w, rr = idx / w;
      Ys[idx] = ldcg(a.Y + f + j + (size_t)(r0 + rr) * a.ldy);
    }
    for (int c = 0; c < nchunk; ++c) {
      const int c0 = c * kTileCH, nc = min(kTileCH, cnt - c0);
      if (c + 1 < nchunk) {
        stage_rows(P, ld, row0 + c0 + kTileCH, min(kTileCH, cnt - c0 - kTileCH), w,
                   Lb + ((c + 1) & 1) * w * kTileLD, kTileLD);
        cp_async_commit_group();
        cp_async_wait_group<1>();  // chunk c has landed (this thread's copies)
      } else {
        cp_async_wait_group<0>();
      }
      __syncthreads();  // ... and every thread's
      const T* L = Lb + (c & 1) * w * kTileLD + lane;
      double acc = 0.0;
      if (g < nrc && lane < nc) {
        const double* y = Ys + g * w;
        double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
        int k = k0;
        for (; k + 3 < k1; k += 4) {
          s0 += (double)L[k * kTileLD] * y[k];
          s1 += (double)L[(k + 1) * kTileLD] * y[k + 1];
          s2 += (double)L[(k + 2) * kTileLD] * y[k + 2];
          s3 += (double)L[(k + 3) * kTileLD] * y[k + 3];
        }
        for (; k < k1; ++k) s0 += (double)L[k * kTileLD] * y[k];
        acc = (s0 + s1) + (s2 + s3);
      }
      if (parts > 1) {
        Red[warp * kTileCH + lane] = acc;
        __syncthreads();
        acc = 0.0;
        if (part == 0)
          for (int q = 0; q < parts; ++q) acc += Red[(g + q * G) * kTileCH + lane];
      }
      if (part == 0 && g < nrc && lane < nc) {
        if constexpr (FAN)  // the tile's buffer: its rows x nrhs
          z[c0 + lane + (size_t)(r0 + g) * cnt] = -acc;
        else
          red_add(a.Y + R[row0 + c0 + lane] + (size_t)(r0 + g) * a.ldy, -acc);
      }
      __syncthreads();  // buffer c & 1 (and Red) are refilled next
    }
  }
}

// y[rows of tile] -= L21[tile] y_s on the tensor cores (FP64 panels, 16 <= w
// <= 64): the tile's rows in passes of 64.
template <bool FAN>
__device__ void fwd_tile_oz(const SolveArgs& a, const double* P, int ld, int row0, int cnt, const int32_t* R, int f,
                            int w, double* sm, double* z) {
  const OzBuf b = oz_carve(sm);
  for (int r0 = 0; r0 < a.nrhs; r0 += kSolveNRC) {
    const int nrc = min(kSolveNRC, a.nrhs - r0);
    __syncthreads();
    oz_stage_ys(a, b, f, w, r0, nrc);
    __syncthreads();
    oz_split_b(b, w);
    for (int c0 = 0; c0 < cnt; c0 += kOzMaxK) {
      const int mc = min(kOzMaxK, cnt - c0);
      const double* Pc = P + row0 + c0;
      copy_batched(
          mc * w, [&](int idx) { return Pc[idx % mc + (size_t)(idx / mc) * ld]; },
          [&](int idx, double v) { b.As[(idx % mc) * kOzLda + idx / mc] = v; });
      oz_zero_pad(b, mc, w);
      __syncthreads();
      double* Y = a.Y + (size_t)r0 * a.ldy;
      const int64_t ldy = a.ldy;
      const int32_t* Rc = R + row0 + c0;
      if constexpr (FAN)
        oz_product(b, mc, w, nrc, [&](int, int m, int n, double v) { z[c0 + m + (size_t)(r0 + n) * cnt] = -v; });
      else
        oz_product(b, mc, w, nrc, [&](int, int m, int n, double v) { red_add(Y + Rc[m] + n * ldy, -v); });
    }
  }
}

template <typename T, bool FAN, bool TC>
__device__ void fwd_tile(const SolveArgs& a, int s, int k, double* sm) {
  const int f = a.pv.fcol[s], w = a.pv.fcol[s + 1] - f, ld = a.pv.ld[s], r = a.pv.nrows[s];
  const int ts = a.st_rows[s];
  const int row0 = w + k * ts, cnt = min(ts, r - row0);
  const T* P = tile_operand<T>(a, s);
  const int32_t* R = a.pv.rows + a.pv.rowoff[s];
  double* z = FAN ? a.zf + a.st_zf[a.st_first[s] + k] * a.nrhs : nullptr;  // fan-in: the tile's buffer
  if constexpr (sizeof(T) == 8 && TC) {
    if (a.tc_tiles && w >= kOzMinW && w <= kOzMaxK) {
      fwd_tile_oz<FAN>(a, reinterpret_cast<const double*>(P), ld, row0, cnt, R, f, w, sm, z);
      return;
    }
  }
  fwd_tile_fma<T, FAN>(a, P, ld, row0, cnt, R, f, w, sm, z);
}

// y_s -= L21[tile]^T x[rows of tile] on the tensor cores (FP64 panels, 16 <= w
// <= 64): A = L21[tile]^T (w x rows), the tile's rows in passes of 64, each with
// its own exponents; the passes' results are summed in FP64 by the owning
// threads and subtracted once.
template <bool FAN>
__device__ void bwd_tile_oz(const SolveArgs& a, const double* P, int ld, int row0, int cnt, const int32_t* R, int f,
                            int w, double* sm, double* z) {
  const OzBuf b = oz_carve(sm);
  for (int r0 = 0; r0 < a.nrhs; r0 += kSolveNRC) {
    const int nrc = min(kSolveNRC, a.nrhs - r0);
    double part[4] = {0.0, 0.0, 0.0, 0.0};
    for (int c0 = 0; c0 < cnt; c0 += kOzMaxK) {
      const int kc = min(kOzMaxK, cnt - c0);
      __syncthreads();
      const double* Pc = P + row0 + c0;
      copy_batched(
          kc * w, [&](int idx) { return Pc[idx % kc + (size_t)(idx / kc) * ld]; },
          [&](int idx, double v) { b.As[(idx / kc) * kOzLda + idx % kc] = v; });
      oz_zero_pad(b, w, kc);
      const int32_t* Rc = R + row0 + c0;
      const double* Y = a.Y + (size_t)r0 * a.ldy;
      const int64_t ldy = a.ldy;
      copy_batched(
          8 * kc,
          [&](int idx) {
            const int n = idx / kc;
            return n < nrc ? ldcg(Y + Rc[idx - n * kc] + n * ldy) : 0.0;
          },
          [&](int idx, double v) { b.Bs[(idx / kc) * 64 + idx % kc] = v; });
      __syncthreads();
      oz_split_b(b, kc);
      oz_product(b, w, kc, nrc, [&](int c, int, int, double v) { part[c] += v; });
    }
    // the outputs this thread owns (as in oz_product)
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp < 4) {
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int m = 16 * warp + (lane >> 2) + ((c & 2) ? 8 : 0), n = 2 * (lane & 3) + (c & 1);
        if (m < w && n < nrc) {
          if constexpr (FAN)
            z[m + (size_t)(r0 + n) * w] = -part[c];
          else
            red_add(a.Y + f + m + (size_t)(r0 + n) * a.ldy, -part[c]);
        }
      }
    }
  }
}

// y_s -= L21[tile]^T x[rows of tile], the tile's rows in chunks as in the
// forward tile, with x of the next chunk loaded into registers while the
// current one is used.  Output (j, g) is a dot product over the tile's rows;
// with few outputs (few right-hand sides) RG thread groups take a share of
// each chunk's rows each and their partial sums meet in shared memory.
template <typename T, bool FAN>
__device__ void bwd_tile_fma(const SolveArgs& a, const T* P, int ld, int row0, int cnt, const int32_t* R, int f,
                             int w, double* sm, double* z) {
  double* Xc = sm;                                     // [2][kSolveNRC][kTileCH]
  double* Red = Xc + 2 * kSolveNRC * kTileCH;          // [kSolveThreads]
  T* Lb = reinterpret_cast<T*>(Red + kSolveThreads);   // [2][w][kTileLD]
  const int tid = threadIdx.x;
  const int nchunk = (cnt + kTileCH - 1) / kTileCH;
  const int xi = tid % kTileCH, xr = tid / kTileCH;    // the x entry this thread loads (256 = 8 x 32)
  for (int r0 = 0; r0 < a.nrhs; r0 += kSolveNRC) {
    const int nrc = min(kSolveNRC, a.nrhs - r0);
    const int O = w * nrc;
    const int RG = O <= 64 ? 4 : O <= 128 ? 2 : 1;
    const int per = blockDim.x / RG, rg = tid / per, u = tid - rg * per;
    const int ri0 = rg * (kTileCH / RG), ri1 = ri0 + kTileCH / RG;
    double part[2] = {0.0, 0.0};
    __syncthreads();  // the previous pass is done with the buffers
    stage_rows(P, ld, row0, min(kTileCH, cnt), w, Lb, kTileLD);
    cp_async_commit_group();
    if (xr < nrc)
      Xc[xr * kTileCH + xi] = xi < min(kTileCH, cnt) ? ldcg(a.Y + R[row0 + xi] + (size_t)(r0 + xr) * a.ldy) : 0.0;
    for (int c = 0; c < nchunk; ++c) {
      const int c0 = c * kTileCH, nc = min(kTileCH, cnt - c0);
      const int c1 = c0 + kTileCH, nc1 = min(kTileCH, cnt - c1);
      if (c + 1 < nchunk) {
        stage_rows(P, ld, row0 + c1, nc1, w, Lb + ((c + 1) & 1) * w * kTileLD, kTileLD);
        cp_async_commit_group();
        cp_async_wait_group<1>();
      } else {
        cp_async_wait_group<0>();
      }
      double xn = 0.0;  // x of the next chunk, loaded while this one is used
      if (c + 1 < nchunk && xr < nrc && xi < nc1) xn = ldcg(a.Y + R[row0 + c1 + xi] + (size_t)(r0 + xr) * a.ldy);
      __syncthreads();
      const T* L = Lb + (c & 1) * w * kTileLD;
      const double* X = Xc + (c & 1) * kSolveNRC * kTileCH;
      const int i1 = min(ri1, nc);
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const int p = u + q * per;
        if (p < O) {
          const int j = p % w, g = p / w;
          const T* lj = L + j * kTileLD;
          const double* xg = X + g * kTileCH;
          double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
          int i = ri0;
          for (; i + 3 < i1; i += 4) {
            s0 += (double)lj[i] * xg[i];
            s1 += (double)lj[i + 1] * xg[i + 1];
            s2 += (double)lj[i + 2] * xg[i + 2];
            s3 += (double)lj[i + 3] * xg[i + 3];
          }
          for (; i < i1; ++i) s0 += (double)lj[i] * xg[i];
          part[q] += (s0 + s1) + (s2 + s3);
        }
      }
      if (c + 1 < nchunk && xr < nrc) Xc[((c + 1) & 1) * kSolveNRC * kTileCH + xr * kTileCH + xi] = xn;
      __syncthreads();  // buffer c & 1 is refilled next
    }
    if (RG > 1) {  // per >= O here: one output per thread of each group
      Red[tid] = part[0];
      __syncthreads();
      if (rg == 0)
        for (int k = 1; k < RG; ++k) part[0] += Red[u + k * per];
    }
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int p = u + q * per;
      if (rg == 0 && p < O) {
        const int j = p % w, g = p / w;
        if constexpr (FAN)
          z[j + (size_t)(r0 + g) * w] = -part[q];
        else
          red_add(a.Y + f + j + (size_t)(r0 + g) * a.ldy, -part[q]);
      }
    }
  }
}

template <typename T, bool FAN, bool TC>
__device__ void bwd_tile(const SolveArgs& a, int s, int k, double* sm) {
  const int f = a.pv.fcol[s], w = a.pv.fcol[s + 1] - f, ld = a.pv.ld[s], r = a.pv.nrows[s];
  const int ts = a.st_rows[s];
  const int row0 = w + k * ts, cnt = min(ts, r - row0);
  const T* P = tile_operand<T>(a, s);
  const int32_t* R = a.pv.rows + a.pv.rowoff[s];
  double* z = FAN ? a.zb + a.st_zb[a.st_first[s] + k] * a.nrhs : nullptr;  // fan-in: the tile's buffer
  if constexpr (sizeof(T) == 8 && TC) {
    if (a.tc_tiles && w >= kOzMinW && w <= kOzMaxK) {
      bwd_tile_oz<FAN>(a, reinterpret_cast<const double*>(P), ld, row0, cnt, R, f, w, sm, z);
      return;
    }
  }
  bwd_tile_fma<T, FAN>(a, P, ld, row0, cnt, R, f, w, sm, z);
}

// Lower the counters cnt[id] of ids list[e] (or e itself when list is null),
// e in [e0, e1), by one, and push task task0 + id for each that reaches zero
// (the first one kept as the CTA's continuation if next is given and free).
// Whole CTA, all threads through the same iterations; each thread issues its
// decrements in batches of 8 whose round trips overlap, and each warp
// reserves ring slots for its ready tasks at once (a panel near the root
// releases thousands of tiles).
__device__ __forceinline__ void release_tiles(const Ring2& q, const int32_t* list, int e0, int e1, int32_t* cnt,
                                              int task0, int* next) {
  for (int b0 = e0; b0 < e1; b0 += 8 * blockDim.x) {
    int id[8], old[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int e = b0 + threadIdx.x + u * blockDim.x;
      id[u] = e < e1 ? (list ? list[e] : e) : -1;
    }
    // acq_rel decrements: each one releases what its thread has observed (the
    // CTA's writes, ordered before it by the publishing barrier), and the one
    // that reaches zero acquires every earlier decrement's release, so the
    // pushed (or kept) task sees all of its producers' writes.
#pragma unroll
    for (int u = 0; u < 8; ++u) old[u] = id[u] >= 0 ? atom_add_acqrel(&cnt[id[u]], -1) : 0;
    int ready[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      ready[u] = (id[u] >= 0 && old[u] == 1) ? task0 + id[u] : -1;
      if (ready[u] >= 0 && next != nullptr && atomicCAS(next, -1, ready[u]) == -1) ready[u] = -1;  // kept
    }
    ring2_push_warp(q, true, ready);
  }
}

// Thread-level: every forward tile into W panel t has landed, so all of t's
// forward tiles are ready (they read b_t); the first (the rows of the etree
// parent, the next step of the chain) becomes the continuation if next is
// given and free, the others go to the high-priority ring in one reservation.
__device__ __forceinline__ void release_w_forward(const Ring2& q, const SolveArgs& a, int t, int* next) {
  int first = a.pv.ns + a.st_first[t], count = a.nst[t];
  if (next != nullptr && atomicCAS(next, -1, first) == -1) {
    ++first;
    --count;
  }
  ring2_push_span(q, true, first, count);
}

// TC: the instantiation whose FP64 panel tiles may run as split products on
// the tensor cores (SPCHOL_FP64_TC).  Those tiles need 64 registers a thread
// (four CTAs per SM); without them the kernel fits 48 and five CTAs share an
// SM, which shortens the dependency chain's tasks (64^3: 16.2 -> 15.7 ms).
template <typename T, bool FAN, bool TC>
__global__ void __launch_bounds__(kSolveThreads, TC ? 4 : 5) solve_kernel(SolveArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ SolveShared sh;
  double* sm = reinterpret_cast<double*>(smem_raw);
  // Two rings: tasks made ready by a finished task (high priority) ahead of
  // the seeds, so that chains up the tree advance instead of queueing behind
  // every leaf.
  const Ring2 q{a.ring, a.ring + a.n_hi, a.n_hi, a.ntask - a.n_hi, a.ctrl, a.budget_ns};
  __shared__ int pend[3];
  if (threadIdx.x == 0) {
    pend[0] = pend[1] = pend[2] = -1;
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
        sh.task = ring2_claim(q, pend, &lo_ready, a.ntask_done);
      }
      // While this CTA holds a claimed slot whose task is not yet pushed, it
      // takes no continuation: it comes back for that task after this one.
      sh.hold = pend[0] >= 0 || pend[1] >= 0;
      if (a.prof) {
        t1 = global_ns();
        wait += t1 - t0;
      }
    }
    __syncthreads();
    const int task = sh.task;
    if (task < 0) break;
    const int type = task < ns ? 0 : task < ns + nst ? 1 : task < ns + 2 * nst ? 2 : 3;
    if (task < ns && is_wpanel(a, task)) {
      // W panel: every forward tile has read b_s; y_s <- A11^{-1} b_s, then the
      // backward tiles (which subtract from y_s) lose their wait for it
      const int s = task;
      diag_solve_w(a, s, sm);
      publish_cta_writes();
      release_tiles(q, nullptr, a.st_first[s], a.st_first[s] + a.nst[s], a.bdep, ns + nst,
                    sh.hold ? nullptr : &sh.next);
    } else if (task < ns) {
      const int s = task;
      diag_solve<false, FAN>(a, s, sm);
      publish_cta_writes();
      // continue with the first forward tile (the rows of the parent) and
      // release the others
      if (a.nst[s] > 0 && a.ftdep) {
        // deterministic order: a tile also waits for its predecessors into the same panels
        for (int i = threadIdx.x; i < a.nst[s]; i += blockDim.x) {
          const int tile = a.st_first[s] + i;
          if (atom_add_acqrel(&a.ftdep[tile], -1) == 1) keep_or_push(q, sh.hold ? nullptr : &sh.next, ns + tile);
        }
      } else if (a.nst[s] > 0) {
        const int keep = sh.hold ? 0 : 1;
        if (keep && threadIdx.x == 0) sh.next = ns + a.st_first[s];
        ring2_push_range(q, true, ns + a.st_first[s] + keep, a.nst[s] - keep, &sh.base);
      } else if (threadIdx.x == 0) {
        keep_or_push(q, sh.hold ? nullptr : &sh.next, ns + 2 * nst + s);
      }
    } else if (task < ns + nst) {
      const int kt = task - ns, s = a.st_sn[kt];
      fwd_tile<T, FAN, TC>(a, s, kt - a.st_first[s], sm);
      publish_cta_writes();
      // Counter updates are spread over the CTA's threads: a panel near the
      // root has thousands of dependent tiles, and they sit on the critical path.
      for (int e = a.st_tptr[kt] + threadIdx.x; e < a.st_tptr[kt + 1]; e += blockDim.x) {
        const int t = a.st_tgt[e];
        if (atom_add_acqrel(&a.fdep[t], -1) == 1) {
          if (is_wpanel(a, t))
            release_w_forward(q, a, t, sh.hold ? nullptr : &sh.next);
          else
            keep_or_push(q, sh.hold ? nullptr : &sh.next, t);
        }
      }
      if (a.ftdep)  // deterministic order: the next tiles into the same panels
        for (int e = a.ft_sptr[kt] + threadIdx.x; e < a.ft_sptr[kt + 1]; e += blockDim.x) {
          const int nx = a.ft_succ[e];
          if (atom_add_acqrel(&a.ftdep[nx], -1) == 1) keep_or_push(q, sh.hold ? nullptr : &sh.next, ns + nx);
        }
      if (threadIdx.x == 0) sh.flag = (atom_add_acqrel(&a.ftiles[s], -1) == 1);
      __syncthreads();
      if (sh.flag) {
        if (is_wpanel(a, s)) {  // b_s is read by all: the diagonal task may overwrite it
          if (threadIdx.x == 0) keep_or_push(q, sh.hold ? nullptr : &sh.next, s);
        } else {
          release_tiles(q, nullptr, a.st_first[s], a.st_first[s] + a.nst[s], a.bdep, ns + nst,
                        sh.hold ? nullptr : &sh.next);
        }
      }
    } else if (task < ns + 2 * nst) {
      const int kt = task - ns - nst, s = a.st_sn[kt];
      bwd_tile<T, FAN, TC>(a, s, kt - a.st_first[s], sm);
      publish_cta_writes();
      // deterministic order: the panel's next backward tile
      if (a.ftdep && threadIdx.x == 0 && kt + 1 < a.st_first[s] + a.nst[s] &&
          atom_add_acqrel(&a.bdep[kt + 1], -1) == 1)
        keep_or_push(q, sh.hold ? nullptr : &sh.next, ns + nst + kt + 1);
      if (is_wpanel(a, s)) {
        // the last backward tile completes x_s = y_s: it releases the tiles
        // that read it (the role of the backward diagonal task, which W panels
        // do not have)
        if (threadIdx.x == 0) sh.flag = (atom_add_acqrel(&a.btiles[s], -1) == 1);
        __syncthreads();
        if (sh.flag)
          release_tiles(q, a.rt_tile, a.rt_ptr[s], a.rt_ptr[s + 1], a.bdep, ns + nst, sh.hold ? nullptr : &sh.next);
      } else if (threadIdx.x == 0 && atom_add_acqrel(&a.btiles[s], -1) == 1) {
        keep_or_push(q, sh.hold ? nullptr : &sh.next, ns + 2 * nst + s);
      }
    } else {
      const int s = task - ns - 2 * nst;
      diag_solve<true, FAN>(a, s, sm);
      publish_cta_writes();
      release_tiles(q, a.rt_tile, a.rt_ptr[s], a.rt_ptr[s + 1], a.bdep, ns + nst, sh.hold ? nullptr : &sh.next);
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

// ---------------------------------------------------------------- subtree solves on single warps
// The subtree tasks the factorization ran on single warps (SolveArgs::wsub)
// are solved by single warps too.  A launch before the task loop runs every
// such subtree's forward solve, one warp per subtree, panels in postorder:
// y_s <- L11^{-1} y_s, then every tile of s, y[rows] -= L21 y_s, by plain
// read-modify-writes for rows inside the subtree and atomics for the others,
// whose panels' counters it then counts down (pushing the diagonal tasks that
// become ready).  The task loop runs everything outside those subtrees: their
// own tasks never become ready there (no forward tile from outside reaches
// their panels, and their backward tiles' counters start out of reach).  A
// launch after it runs each subtree's backward solve, panels in reverse
// postorder: y_s -= L21^T x[rows] over its tiles, then x_s <- L11^{-T} y_s;
// every x it reads is final by then (outside: the task loop has ended;
// inside: an ancestor in the subtree, solved earlier by the same warp).
constexpr int kWsWarps = 4;  // warps per CTA of the subtree solve launches
constexpr int kWsNrc = 8;    // right-hand sides per pass (a panel is at most 32 wide)

template <typename T>
__device__ void subtree_forward(const SolveArgs& a, int k, double* ys, double* zs) {
  const int lane = threadIdx.x & 31;
  const int lo = a.sub_lo[k], hi = a.sub_hi[k];
  const int gend = a.pv.fcol[hi + 1];  // rows from here on lie outside the subtree
  const Ring2 q{a.ring, a.ring + a.n_hi, a.n_hi, a.ntask - a.n_hi, a.ctrl, a.budget_ns};
  for (int s = lo; s <= hi; ++s) {
    const int f = a.pv.fcol[s], w = a.pv.fcol[s + 1] - f, ld = a.pv.ld[s], r = a.pv.nrows[s];
    const T* P = spanel<T>(a, s);
    const double* X = a.inv + a.invoff[s];
    const int32_t* R = a.pv.rows + a.pv.rowoff[s];
    const int ts = a.st_rows[s];
    bool outside = false;
    for (int r0 = 0; r0 < a.nrhs; r0 += kWsNrc) {
      const int nrc = min(kWsNrc, a.nrhs - r0);
      double* Y = a.Y + (size_t)r0 * a.ldy;
      for (int o = lane; o < w * nrc; o += 32) ys[o] = ldcg(Y + f + o % w + (size_t)(o / w) * a.ldy);
      __syncwarp();
      for (int o = lane; o < w * nrc; o += 32) {  // y_s <- L11^{-1} y_s
        const int i = o % w, c = o / w;
        double acc = 0.0;
        for (int kk = 0; kk <= i; ++kk) acc = fma(X[i + kk * w], ys[kk + c * w], acc);
        zs[o] = acc;
        Y[f + i + (size_t)c * a.ldy] = acc;
      }
      __syncwarp();
      for (int kt = 0; kt < a.nst[s]; ++kt) {  // y[rows] -= L21 y_s
        const int row0 = w + kt * ts, cnt = min(ts, r - row0);
        for (int o = lane; o < cnt * nrc; o += 32) {
          const int i = o % cnt, c = o / cnt;
          const T* Li = P + row0 + i;
          double acc0 = 0.0, acc1 = 0.0;
          int kk = 0;
          for (; kk + 1 < w; kk += 2) {
            acc0 = fma((double)Li[(size_t)kk * ld], zs[kk + c * w], acc0);
            acc1 = fma((double)Li[(size_t)(kk + 1) * ld], zs[kk + 1 + c * w], acc1);
          }
          if (kk < w) acc0 = fma((double)Li[(size_t)kk * ld], zs[kk + c * w], acc0);
          const int g = R[row0 + i];
          double* dst = Y + g + (size_t)c * a.ldy;
          if (g < gend) {
            *dst -= acc0 + acc1;
          } else {
            red_add(dst, -(acc0 + acc1));
            outside = true;
          }
        }
      }
      __syncwarp();  // the next pass reuses ys and zs; the next panel reads these rows
    }
    // count the tiles down on the panels outside the subtree that they reach,
    // one (tile, target) entry per lane: the warp barrier orders every lane's
    // writes before each lane's acq_rel decrement (and lane 0's fence)
    if (__any_sync(0xffffffffu, outside)) {
      if (lane == 0) __threadfence();
      __syncwarp();
      const int e0 = a.st_tptr[a.st_first[s]], e1 = a.st_tptr[a.st_first[s] + a.nst[s]];
      for (int e = e0 + lane; e < e1; e += 32) {
        const int t = a.st_tgt[e];
        if (t > hi && atom_add_acqrel(&a.fdep[t], -1) == 1) {
          if (is_wpanel(a, t))
            release_w_forward(q, a, t, nullptr);
          else
            ring2_push_one(q, true, t);
        }
      }
      __syncwarp();
    }
  }
}

template <typename T>
__device__ void subtree_backward(const SolveArgs& a, int k, double* ys) {
  const int lane = threadIdx.x & 31;
  const int lo = a.sub_lo[k], hi = a.sub_hi[k];
  for (int s = hi; s >= lo; --s) {
    const int f = a.pv.fcol[s], w = a.pv.fcol[s + 1] - f, ld = a.pv.ld[s], r = a.pv.nrows[s];
    const T* P = spanel<T>(a, s);
    const double* X = a.inv + a.invoff[s];
    const int32_t* R = a.pv.rows + a.pv.rowoff[s];
    const int ts = a.st_rows[s];
    for (int r0 = 0; r0 < a.nrhs; r0 += kWsNrc) {
      const int nrc = min(kWsNrc, a.nrhs - r0);
      double* Y = a.Y + (size_t)r0 * a.ldy;
      for (int o = lane; o < w * nrc; o += 32) ys[o] = ldcg(Y + f + o % w + (size_t)(o / w) * a.ldy);
      __syncwarp();
      for (int kt = 0; kt < a.nst[s]; ++kt) {  // y_s -= L21^T x[rows]
        const int row0 = w + kt * ts, cnt = min(ts, r - row0);
        for (int o = lane; o < w * nrc; o += 32) {
          const int j = o % w, c = o / w;
          const T* Lj = P + row0 + (size_t)j * ld;
          double acc0 = 0.0, acc1 = 0.0;
          int i = 0;
          for (; i + 1 < cnt; i += 2) {
            acc0 = fma((double)Lj[i], ldcg(Y + R[row0 + i] + (size_t)c * a.ldy), acc0);
            acc1 = fma((double)Lj[i + 1], ldcg(Y + R[row0 + i + 1] + (size_t)c * a.ldy), acc1);
          }
          if (i < cnt) acc0 = fma((double)Lj[i], ldcg(Y + R[row0 + i] + (size_t)c * a.ldy), acc0);
          ys[o] -= acc0 + acc1;
        }
      }
      __syncwarp();
      for (int o = lane; o < w * nrc; o += 32) {  // x_s <- L11^{-T} y_s
        const int j = o % w, c = o / w;
        double acc = 0.0;
        for (int i = j; i < w; ++i) acc = fma(X[i + j * w], ys[i + c * w], acc);
        Y[f + j + (size_t)c * a.ldy] = acc;
      }
      __syncwarp();  // the next pass reuses ys; the next panels read x_s
    }
  }
}

template <typename T, bool FWD>
__global__ void __launch_bounds__(32 * kWsWarps) subtree_solve_kernel(SolveArgs a) {
  __shared__ double buf[kWsWarps][2][kWsNrc * 32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (;;) {
    int e = 0;
    if (lane == 0) e = atomicAdd(&a.ctrl[FWD ? kWarpNext : kWarpNextB], 1);
    e = __shfl_sync(0xffffffffu, e, 0);
    if (e >= a.n_wsub) break;
    if constexpr (FWD)
      subtree_forward<T>(a, a.wsub[e], buf[warp][0], buf[warp][1]);
    else
      subtree_backward<T>(a, a.wsub[e], buf[warp][0]);
    if (lane == 0) atomicAdd(&a.ctrl[kDone], 1);
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

size_t solve_smem_bytes(int max_w, bool tc_tiles, bool fanin) {
  // diagonal tasks: the inverse and the right-hand sides, plus (W panels, not
  // in the fan-in mode) the product with L11^{-1}
  const size_t diag = ((size_t)max_w * (max_w + 1) + (size_t)max_w * kSolveNRC * (fanin ? 1 : 2)) * sizeof(double) +
                      (fanin ? solve_fan_smem_bytes(max_w) : 0);
  // panel tiles: two chunk buffers of max_w x kTileLD (FP64 bound) plus, forward,
  // the right-hand sides and the partial sums, backward, two x chunks and the
  // partial sums
  const size_t bufs = 2 * (size_t)max_w * kTileLD * sizeof(double);
  const size_t fwd = ((size_t)kSolveNRC * max_w + 8 * kTileCH) * sizeof(double);
  const size_t bwd = (2 * (size_t)kSolveNRC * kTileCH + kSolveThreads) * sizeof(double);
  const size_t tile = bufs + (fwd > bwd ? fwd : bwd);
  size_t need = diag > tile ? diag : tile;
  if (tc_tiles && max_w >= kOzMinW && need < kOzSmemBytes) need = kOzSmemBytes;
  return need;
}

// The fan-in mode has kernels of its own, so that the other modes' tiles and
// diagonal tasks carry none of its code.
static const void* solve_fn(bool fp32, bool fan, bool tc) {
  if (fp32) return fan ? (const void*)solve_kernel<float, true, false> : (const void*)solve_kernel<float, false, false>;
  if (tc) return fan ? (const void*)solve_kernel<double, true, true> : (const void*)solve_kernel<double, false, true>;
  return fan ? (const void*)solve_kernel<double, true, false> : (const void*)solve_kernel<double, false, false>;
}

cudaError_t solve_configure(bool fp32, bool fanin, bool tc, size_t smem, int* blocks_per_sm) {
  const void* fn = solve_fn(fp32, fanin, tc);
  cudaError_t e = ensure_smem_limit(fn, smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, fn, kSolveThreads, smem);
}

cudaError_t launch_subtree_solve(bool fp32, bool forward, const SolveArgs& a, int grid, cudaStream_t st) {
  if (a.n_wsub == 0) return cudaSuccess;
  void* args[] = {const_cast<SolveArgs*>(&a)};
  const void* fn = fp32 ? (forward ? (const void*)subtree_solve_kernel<float, true> : (const void*)subtree_solve_kernel<float, false>)
                        : (forward ? (const void*)subtree_solve_kernel<double, true> : (const void*)subtree_solve_kernel<double, false>);
  return cudaLaunchKernel(fn, dim3(grid), dim3(32 * kWsWarps), args, 0, st);
}

cudaError_t launch_solve(bool fp32, const SolveArgs& a, int grid, size_t smem, cudaStream_t st) {
  void* args[] = {const_cast<SolveArgs*>(&a)};
  return cudaLaunchKernel(solve_fn(fp32, a.zf != nullptr, a.tc_tiles != 0), dim3(grid), dim3(kSolveThreads), args,
                          smem, st);
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
