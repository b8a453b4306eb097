// Supernodal numeric factorization: assembly and the persistent task kernel.
//
// Tasks (Section III-A; Section IV labels a task by source and target):
//   POTRF(s)     F on the diagonal block of panel s: the dense Cholesky of
//                Algorithm 1 on a w x w block, always in FP64.
//   TRSM(s, k)   F on rows tile k below the diagonal block:
//                L21 = A21 L11^{-T} by forward substitution along each row.
//   UPD(s, t, k) U + A fused: C = L_s[rows k] L_s[rows in t]^T, subtracted
//                from panel t at the relative positions of those rows and
//                columns in t (the aggregate vector of Section III-A is
//                applied immediately, by atomic adds, instead of being kept).
// Dependencies (Section II-C): UPD(s, ., .) needs every TRSM tile of s;
// POTRF(t) needs every update tile targeting t.
#include <algorithm>
#include <climits>
#include <cstdint>

#include <cuda_bf16.h>

#include "device_common.cuh"
#include "kernels.hpp"
#include "sched.cuh"

namespace spchol {

namespace {

constexpr int kTrsmJB = 8;     // wide panels: columns solved together per row (independent FMA chains)
constexpr int kTrsmMaxW = 64;  // panels up to this width take the register-resident panel solve

struct FactorShared {
  int task;
  int skip;
  int flag;
  int base;
};

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ Ring2 rings_of(const FactorArgs& a) {
  return Ring2{a.ring, a.ring + a.n_hi, a.n_hi, a.ntask - a.n_hi, a.ctrl, a.budget_ns};
}

template <typename T>
__device__ __forceinline__ T* panel_ptr(const FactorArgs& a, int s) {
  return reinterpret_cast<T*>(a.pool) + a.pv.valoff[s];
}

// ---------------------------------------------------------------- POTRF(s)
// Cholesky of the w x w diagonal block in shared memory (Algorithm 1), taken
// right-looking in the square-root-free form A = M D M^T, one barrier per
// column, then L = M D^{1/2}.  Step j: warps 0..6 form the multipliers
// m_ij = a_ij / d_j (into a double-buffered vector), write column j - 1 of M
// back in place, and apply the rank-1 update a_ik -= m_ij a_kj of the
// trailing triangle; meanwhile warp 7 already updates d_{j+1} and forms
// 1 / d_{j+1} (look-ahead).  The serial chain from one column to the next is
// a multiply, an FMA and a reciprocal; the square roots come after the loop,
// all columns at once.  The update is enumerated by the pair index p of the
// trailing triangle in column-major order from its bottom-right corner, so
// that p < m (m + 1) / 2 is exactly the triangle of order m and consecutive p
// touch consecutive rows; the pairs are decoded once into a table.
constexpr int kPivotWarp = 7;
constexpr int kUpdWarps = 7;

__device__ __forceinline__ void tri_pair(int p, int& ei, int& ek) {
  int e = (int)((sqrtf((float)(8 * p + 1)) - 1.0f) * 0.5f);
  if ((e + 1) * (e + 2) / 2 <= p) ++e;
  if (e * (e + 1) / 2 > p) --e;
  ek = e;
  ei = p - e * (e + 1) / 2;
}

// 1 / d for the pivot d > 0 by Newton's iteration y <- y (2 - d y) from the
// single-precision approximate reciprocal (relative error below 2^-22; two
// steps take it below the FP64 rounding error); outside the range where the
// seed is representable, the division.
__device__ __forceinline__ double pivot_recip(double d) {
  if (d > 1e-30 && d < 1e30) {
    float y0;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y0) : "f"((float)d));
    double y = (double)y0;
    y = fma(y, fma(-d, y, 1.0), y);
    y = fma(y, fma(-d, y, 1.0), y);
    return y;
  }
  return 1.0 / d;
}

template <typename T, bool FAN>
__device__ void task_potrf(const FactorArgs& a, int s, double* sm, FactorShared& sh, bool skip, bool release = true) {
  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  const int f = a.pv.fcol[s], w = a.pv.fcol[s + 1] - f, ld = a.pv.ld[s];
  T* P = panel_ptr<T>(a, s);
  double* xd = sm + w * w;  // during the loop 1 / d_j; after it r_j = 1 / l_jj (the diagonal of L11^{-1})
  double* cb = xd + w;      // 2 x w: multipliers of the current step, by parity
  // pair table: the column index ek of pair p of the trailing triangle (its
  // row index is p - ek (ek + 1) / 2), decoded once
  uint8_t* pt = reinterpret_cast<uint8_t*>(cb + 2 * w);
  const int npair = w * (w - 1) / 2;  // pairs of the largest trailing triangle (step 0)
  bool ok = true;
  if (!skip) {
    stage_lower<true>(P, w, ld, sm);  // lower triangle; zeros above (used below for L11^{-1})
    for (int p = tid; p < npair; p += blockDim.x) {
      int ei, ek;
      tri_pair(p, ei, ek);
      pt[p] = (uint8_t)ek;
    }
    if (tid == 0) sh.flag = 0;
    __syncthreads();
    if (tid == kPivotWarp * 32) {
      const double d0 = sm[0];
      if (d0 > 0.0) {
        xd[0] = pivot_recip(d0);
      } else {
        atomicMin(&a.ctrl[kInfo], f + 1);
        sh.flag = 1;
      }
    }
    __syncthreads();
    for (int j = 0; j < w && !sh.flag; ++j) {
      const double qj = xd[j];
      if (warp < kUpdWarps) {
        double* cj = cb + (j & 1) * w;
        const double* cprev = cb + ((j + 1) & 1) * w;
        for (int i = j + 1 + tid; i < w; i += kUpdWarps * 32) cj[i] = sm[i + j * w] * qj;
        if (j > 0)
          for (int i = j + tid; i < w; i += kUpdWarps * 32) sm[i + (j - 1) * w] = cprev[i];
        asm volatile("bar.sync 1, %0;" ::"n"(kUpdWarps * 32) : "memory");
        const int m = w - 1 - j;
        const int np = m * (m + 1) / 2 - 1;  // all but (j + 1, j + 1), which warp 7 owns
        const double* aj = sm + j * w;       // column j, not yet divided by d_j
        constexpr int kStep = kUpdWarps * 32;
        // two pairs per round, every load issued before the arithmetic: the
        // pairs are distinct entries, so the rounds' chains overlap
        for (int p = tid; p < np; p += 2 * kStep) {
          const int p2 = p + kStep;
          const int q2 = p2 < np ? p2 : p;
          const int ek1 = pt[p], ek2 = pt[q2];
          const int i1 = w - 1 - (p - ek1 * (ek1 + 1) / 2), k1 = w - 1 - ek1;
          const int i2 = w - 1 - (q2 - ek2 * (ek2 + 1) / 2), k2 = w - 1 - ek2;
          const double a1 = cj[i1], b1 = aj[k1], s1 = sm[i1 + k1 * w];
          const double a2 = cj[i2], b2 = aj[k2], s2 = sm[i2 + k2 * w];
          sm[i1 + k1 * w] = fma(-a1, b1, s1);
          if (p2 < np) sm[i2 + k2 * w] = fma(-a2, b2, s2);
        }
      } else if (lane == 0 && j + 1 < w) {
        const double a1 = sm[(j + 1) + j * w];
        const double d = fma(-(a1 * qj), a1, sm[(j + 1) * (w + 1)]);
        const double q = pivot_recip(d);
        if (d > 0.0) {
          sm[(j + 1) * (w + 1)] = d;
          xd[j + 1] = q;
        } else {
          atomicMin(&a.ctrl[kInfo], f + j + 2);
          sh.flag = 1;
        }
      }
      __syncthreads();
    }
    ok = !sh.flag;
    if (ok) {
      // L = M D^{1/2}: l_jj = sqrt(d_j) (and r_j = 1 / l_jj for the solves),
      // then l_ij = m_ij l_jj below the diagonal
      for (int j = tid; j < w; j += blockDim.x) {
        const double l = sqrt(sm[j * (w + 1)]);
        sm[j * (w + 1)] = l;
        xd[j] = 1.0 / l;
      }
      __syncthreads();
      for (int j = warp; j < w; j += kFactorThreads / 32) {
        const double l = sm[j * (w + 1)];
        for (int i = j + 1 + lane; i < w; i += 32) sm[i + j * w] *= l;
      }
      __syncthreads();
    }
    for (int j = warp; j < w; j += kFactorThreads / 32)
      for (int i = j + lane; i < w; i += 32) P[i + (size_t)j * ld] = (T)sm[i + j * w];
  }
  publish_cta_writes();
  if (FAN && release) {  // fan-in mode: a panel-solve tile also waits for its rows' gathers
    for (int k = tid; k < a.ntrsm[s]; k += blockDim.x) {
      const int kt = a.trsm_first[s] + k;
      if (atom_add_acqrel(&a.tdep[kt], -1) == 1) ring2_push_one(rings_of(a), true, a.pv.ns + kt);
    }
  } else if (release) {
    ring2_push_range(rings_of(a), true, a.pv.ns + a.trsm_first[s], a.ntrsm[s], &sh.base);
  }
  if (!skip && ok) {
    // L11^{-1} for the solves, off the critical path (the panel-solve tiles are
    // already released).  X = L11^{-1} by right-looking forward substitution
    // on all columns at once: after row k of X is final, every row i > k
    // subtracts l_ik X[k][:]; the row k + 1 is finished (scaled by r_{k+1}) by
    // the same thread that applies its last update.  X[i][c], i > c, lives in
    // the zeroed upper triangle at (c, i); the diagonal is xd.
    for (int k = 0; k < w - 1; ++k) {
      for (int i = k + 1 + warp; i < w; i += kFactorThreads / 32) {
        const double lik = sm[i + k * w];
        const double ri = xd[i];
        for (int c = lane; c <= k; c += 32) {
          const double xkc = (c == k) ? xd[k] : sm[c + k * w];
          double v = fma(-lik, xkc, sm[c + i * w]);
          if (i == k + 1) v *= ri;
          sm[c + i * w] = v;
        }
      }
      __syncthreads();
    }
    double* X = a.inv + a.invoff[s];
    for (int j = warp; j < w; j += kFactorThreads / 32)
      for (int i = j + lane; i < w; i += 32) X[i + (size_t)j * w] = (i == j) ? xd[j] : sm[j + i * w];
  }
}

// ---------------------------------------------------------------- FP64 operand slicing
// Error-free splitting of a row of L for the BF16 tensor cores (the splitting
// step of Ozaki, Ogita, Oishi and Rump, "Error-free transformations of matrix
// multiplication by using fast routines of matrix multiplication", Numer.
// Algorithms 2012).  With e the smallest integer such that every |x_k| of the
// row is below 2^e, x_k * 2^(56-e) is written as a 56-bit fixed-point integer
// q_k (truncated below 2^(e-56), a relative perturbation of the row of at most
// 2^-56) and cut into kSlices 8-bit digits; digit p carries weight
// 2^(e - 8(p+1)).  Each digit, with the sign of x_k, is an integer in
// [-255, 255] and is exact in BF16.  Products of two digit matrices summed over
// k <= 64 stay below 2^22 and are exact in the FP32 accumulator.
__device__ __forceinline__ int row_exponent_bits(const double* Pi, int w, int ld) {
  int emax = 0;
  for (int k = 0; k < w; ++k) {
    const int ex = (int)((__double_as_longlong(ldcg(Pi + (size_t)k * ld)) >> 52) & 0x7FF);
    emax = max(emax, ex);
  }
  return emax;  // 0: the row is zero (or denormal)
}

__device__ __forceinline__ unsigned long long fixed56(double x, int e, bool& neg) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
  neg = (bits >> 63) != 0;
  const int ex = (int)((bits >> 52) & 0x7FF);
  if (ex == 0) return 0ull;
  const unsigned long long mant = (bits & 0xFFFFFFFFFFFFFull) | (1ull << 52);
  const int sh = ex - 1019 - e;  // q = mant * 2^sh < 2^56
  if (sh >= 0) return mant << sh;
  return (-sh < 64) ? (mant >> (-sh)) : 0ull;
}

__device__ __forceinline__ uint32_t bf16_digit(unsigned long long q, int p, bool neg) {
  const int d = (int)((q >> (56 - kSliceBits * (p + 1))) & 0xFF);
  return (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn((float)(neg ? -d : d)));
}

// Slice one row (Pi[k * ld], k < w) into the panel's slice block: slice p of
// below-row ib at sl[(p * nb + ib) * kpad + k], zero for k >= w.
__device__ void slice_row(const double* Pi, int w, int ld, int kpad, int nb, int ib, uint16_t* sl, int32_t* rexp) {
  const int emax = row_exponent_bits(Pi, w, ld);
  const int e = emax ? emax - 1022 : 0;
  *rexp = e;
  for (int k0 = 0; k0 < kpad; k0 += 8) {
    uint32_t packed[kSlices][4];
#pragma unroll
    for (int p = 0; p < kSlices; ++p)
#pragma unroll
      for (int c = 0; c < 4; ++c) packed[p][c] = 0u;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const int k = k0 + c;
      bool neg = false;
      const unsigned long long q = (k < w && emax) ? fixed56(ldcg(Pi + (size_t)k * ld), e, neg) : 0ull;
#pragma unroll
      for (int p = 0; p < kSlices; ++p) packed[p][c >> 1] |= bf16_digit(q, p, neg) << (16 * (c & 1));
    }
#pragma unroll
    for (int p = 0; p < kSlices; ++p) {
      uint4 v = make_uint4(packed[p][0], packed[p][1], packed[p][2], packed[p][3]);
      *reinterpret_cast<uint4*>(sl + ((size_t)p * nb + ib) * kpad + k0) = v;
    }
  }
}

// ---------------------------------------------------------------- TRSM(s, k)
// Arithmetic in the panel's type: FP64 panels solve in FP64, FP32 panels (the
// mixed-precision modes) in FP32.
// W = L21 L11^{-1} for rows row0 .. row0 + cnt - 1 of a W panel (Plan::woff):
// each row w solves w L11 = l21 by back substitution, w_c = (l21_c - sum over
// q > c of w_q l_qc) / l_cc for c = w-1 .. 0, from the rows this panel-solve
// tile has just written and L11 (the inverse of the diagonal task is formed
// after the release of these tiles, so it is not read here).  The layout of
// the panel solve: warp q takes 4-row strips, lane (lr, lc) row lr at columns
// lc + 8 cc; L11 is restaged with leading dimension 65, so that the 8 lanes of
// a row read the entries l_c,lc+8cc of row c of L11 from distinct banks.
template <typename T>
__device__ void form_w_rows(const FactorArgs& a, int s, int row0, int cnt, double* smd) {
  using ct = T;
  constexpr int kLd = kTrsmMaxW + 1;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int w = a.pv.fcol[s + 1] - a.pv.fcol[s], ld = a.pv.ld[s];
  const T* P = panel_ptr<T>(a, s);
  T* W = reinterpret_cast<T*>(a.wbuf) + a.woff[s];
  ct* Ls = reinterpret_cast<ct*>(smd);  // Ls[q + kLd c] = l_qc for q > c
  ct* rinv = Ls + kLd * w;              // 1 / l_cc
  __syncthreads();                      // the panel solve is done with shared memory
  for (int idx = tid; idx < kTrsmMaxW * w; idx += nt) {
    const int qq = idx & (kTrsmMaxW - 1), c = idx >> 6;
    Ls[qq + kLd * c] = (qq < w && qq > c) ? (ct)ldcg(P + qq + (size_t)c * ld) : ct(0);
  }
  for (int c = tid; c < w; c += nt) rinv[c] = ct(1) / (ct)ldcg(P + c + (size_t)c * ld);
  __syncthreads();
  const int warp = tid >> 5, lane = tid & 31, lr = lane >> 3, lc = lane & 7;
  const int nstrip = (cnt + 3) >> 2;
  for (int st = warp; st < nstrip; st += nt >> 5) {
    const int rloc = 4 * st + lr;
    const bool rv = rloc < cnt;
    const T* Pi = P + row0 + rloc;
    ct x[8];
#pragma unroll
    for (int cc = 0; cc < 8; ++cc) {
      const int c = lc + 8 * cc;
      x[cc] = (rv && c < w) ? (ct)ldcg(Pi + (size_t)c * ld) : ct(0);
    }
#pragma unroll
    for (int cbk = 7; cbk >= 0; --cbk) {
      if (8 * cbk >= w) continue;
      for (int c8 = 7; c8 >= 0; --c8) {
        const int c = 8 * cbk + c8;
        if (c >= w) continue;
        if (lc == c8) x[cbk] *= rinv[c];
        const ct xc = __shfl_sync(0xffffffffu, x[cbk], (lr << 3) | c8);
        const ct* Lr = Ls + c;  // l_c,c' at Lr[kLd c'] for c' < c
        if (lc < c8) x[cbk] -= xc * Lr[kLd * (lc + 8 * cbk)];
#pragma unroll
        for (int cc = 0; cc < cbk; ++cc) x[cc] -= xc * Lr[kLd * (lc + 8 * cc)];
      }
    }
    T* Wi = W + row0 + rloc;
#pragma unroll
    for (int cc = 0; cc < 8; ++cc) {
      const int c = lc + 8 * cc;
      if (rv && c < w) Wi[(size_t)c * ld] = (T)x[cc];
    }
  }
}

template <typename T, int MODE>
__device__ void task_trsm(const FactorArgs& a, int s, int k, double* smd, FactorShared& sh, bool skip,
                          bool release = true) {
  using ct = T;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int f = a.pv.fcol[s], w = a.pv.fcol[s + 1] - f, ld = a.pv.ld[s], r = a.pv.nrows[s];
  const int tr = a.trsm_rows_of[s];
  const int row0 = w + k * tr;
  const int cnt = min(tr, r - row0);
  T* P = panel_ptr<T>(a, s);
  ct* sm = reinterpret_cast<ct*>(smd);
  (void)f;
  if (!skip && w <= kTrsmMaxW) {
    // L21 = A21 L11^{-T}, row by row: forward substitution along each row with
    // the columns in registers.  Warp q takes 4-row strips 4 (q + 8 v); lane
    // (lr, lc) holds row lr of the strip at columns lc + 8 cc.  Step c: the lane
    // holding column c scales it by 1 / l_cc, the value is broadcast within the
    // 8 lanes of the row, and every later column subtracts it times l_qc.
    const int warp = tid >> 5, lane = tid & 31, lr = lane >> 3, lc = lane & 7;
    ct* Ls = sm;                        // Ls[q + 64 c] = l_qc for q > c, else 0
    ct* rinv = sm + kTrsmMaxW * w;      // 1 / l_cc
    for (int idx = tid; idx < kTrsmMaxW * w; idx += nt) {
      const int qq = idx & (kTrsmMaxW - 1), c = idx >> 6;
      Ls[idx] = (qq < w && qq > c) ? (ct)ldcg(P + qq + (size_t)c * ld) : ct(0);
    }
    for (int c = tid; c < w; c += nt) rinv[c] = ct(1) / (ct)ldcg(P + c + (size_t)c * ld);
    __syncthreads();
    const int nstrip = (cnt + 3) >> 2;
    for (int st = warp; st < nstrip; st += nt >> 5) {
      const int rloc = 4 * st + lr;
      const bool rv = rloc < cnt;
      T* Pi = P + row0 + rloc;
      ct x[8];
#pragma unroll
      for (int cc = 0; cc < 8; ++cc) {
        const int c = lc + 8 * cc;
        x[cc] = (rv && c < w) ? (ct)ldcg(Pi + (size_t)c * ld) : ct(0);
      }
#pragma unroll
      for (int cbk = 0; cbk < 8; ++cbk) {
        if (8 * cbk >= w) break;
        for (int c8 = 0; c8 < 8; ++c8) {
          const int c = 8 * cbk + c8;
          if (c >= w) break;
          if (lc == c8) x[cbk] *= rinv[c];
          const ct xc = __shfl_sync(0xffffffffu, x[cbk], (lr << 3) | c8);
          const ct* Lc = Ls + kTrsmMaxW * c;
          if (lc > c8) x[cbk] -= xc * Lc[lc + 8 * cbk];
#pragma unroll
          for (int cc = cbk + 1; cc < 8; ++cc) {
            if (8 * cc >= w) break;
            x[cc] -= xc * Lc[lc + 8 * cc];
          }
        }
      }
#pragma unroll
      for (int cc = 0; cc < 8; ++cc) {
        const int c = lc + 8 * cc;
        if (rv && c < w) Pi[(size_t)c * ld] = (T)x[cc];
      }
    }
    if constexpr (sizeof(T) == 8 && MODE == 3) {
      if (w >= a.tc_min_width) {
        __syncthreads();  // the tile's rows are written (visible to this CTA through L2)
        const int kpad = (w + 15) & ~15, nbel = r - w;
        for (int rr = tid; rr < cnt; rr += nt)
          slice_row(reinterpret_cast<const double*>(P + row0 + rr), w, ld, kpad, nbel, row0 + rr - w,
                    a.slices + a.sliceoff[s], a.rexp + a.pv.rowoff[s] + row0 + rr);
      }
    }
  } else if (!skip) {
    // Panels wider than kTrsmMaxW: one thread per row, columns in blocks.
    if constexpr (sizeof(ct) == 8) {
      stage_lower<true>(P, w, ld, reinterpret_cast<double*>(sm));
    } else {
      for (int idx = tid; idx < w * w; idx += nt) {
        const int i = idx % w, j = idx / w;
        sm[idx] = (i >= j) ? (ct)ldcg(P + i + (size_t)j * ld) : ct(0);
      }
    }
    __syncthreads();
    for (int rr = tid; rr < cnt; rr += nt) {
      T* Pi = P + row0 + rr;
      for (int jb = 0; jb < w; jb += kTrsmJB) {
        const int nb = min(kTrsmJB, w - jb);
        ct x[kTrsmJB];
#pragma unroll
        for (int c = 0; c < kTrsmJB; ++c) x[c] = (c < nb) ? (ct)ldcg(Pi + (size_t)(jb + c) * ld) : ct(0);
        for (int kk = 0; kk < jb; ++kk) {
          const ct xk = (ct)ldcg(Pi + (size_t)kk * ld);
          const ct* Lk = sm + kk * w + jb;  // L[jb + c][kk]
#pragma unroll
          for (int c = 0; c < kTrsmJB; ++c)
            if (c < nb) x[c] -= xk * Lk[c];
        }
#pragma unroll
        for (int c = 0; c < kTrsmJB; ++c) {
          if (c < nb) {
#pragma unroll
            for (int c2 = 0; c2 < c; ++c2) x[c] -= x[c2] * sm[(jb + c) + (jb + c2) * w];
            x[c] = x[c] / sm[(jb + c) + (jb + c) * w];
            Pi[(size_t)(jb + c) * ld] = (T)x[c];
          }
        }
      }
      if constexpr (sizeof(T) == 8 && MODE == 3) {
        if (w >= a.tc_min_width) {
          const int kpad = (w + 15) & ~15, nbel = r - w, ib = row0 + rr - w;
          slice_row(reinterpret_cast<const double*>(Pi), w, ld, kpad, nbel, ib, a.slices + a.sliceoff[s],
                    a.rexp + a.pv.rowoff[s] + row0 + rr);
        }
      }
    }
  }
  publish_cta_writes();
  if (!release) return;  // inside a subtree task: no counters, the same CTA goes on
  if (tid == 0) sh.flag = (atom_add_acqrel(&a.trsm_left[s], -1) == 1);
  __syncthreads();
  if (sh.flag) {
    const Ring2 q = rings_of(a);
    const int first = a.pv.ns + a.n_trsm + a.u_first[s], nhi = a.nu_hi[s];
    if (a.u_dep) {  // deterministic order: a tile also waits for its predecessor into the same target
      for (int i = threadIdx.x; i < a.nu[s]; i += blockDim.x)
        if (atom_add_acqrel(&a.u_dep[a.u_first[s] + i], -1) == 1) ring2_push_one(q, i < nhi, first + i);
    } else {
      ring2_push_range(q, true, first, nhi, &sh.base);
      ring2_push_range(q, false, first + nhi, a.nu[s] - nhi, &sh.base);
    }
  }
  // W rows after the release: the updates of this panel do not wait for them
  // (the solves, a later launch, read them)
  if (!skip && a.woff != nullptr && a.woff[s] >= 0) form_w_rows<T>(a, s, row0, cnt, smd);
}

// ---------------------------------------------------------------- an update has landed
// Count down the updates still to land in target panel t; the last one makes
// the panel's diagonal task ready -- in the fan-in mode its gather tasks, and
// the diagonal task too when none of them holds rows of its diagonal block.
// Whole CTA (the fan-in mode pushes its gathers together).
template <bool FAN>
__device__ __forceinline__ void target_update_done(const FactorArgs& a, int t, FactorShared& sh, bool release) {
  if constexpr (!FAN) {
    if (release && threadIdx.x == 0 && atom_add_acqrel(&a.dep_f[t], -1) == 1) ring2_push_one(rings_of(a), true, t);
  } else {
    if (threadIdx.x == 0) sh.flag = release && atom_add_acqrel(&a.dep_f[t], -1) == 1;
    __syncthreads();
    if (sh.flag) {
      const int g0 = a.gat_first[t], g1 = a.gat_first[t + 1];
      ring2_push_range(rings_of(a), true, a.gat0 + g0, g1 - g0, &sh.base);
      if (threadIdx.x == 0 && a.gdiag0[t] == 0) ring2_push_one(rings_of(a), true, t);
    }
  }
}

// ---------------------------------------------------------------- relative indices
// The relative index of row g of panel s in a target panel t is the position
// of g in t's sorted row list (the relative-index maps of the supernodal
// update, Section III-A).  They are fixed by the structure, so one kernel at
// analysis time finds them for every row of every update tile (a binary search
// each), and an update tile only loads its rowlen of them.
// In the fan-in mode the tile writes its own buffer instead, addressed as a
// panel whose rows are the tile's rows and whose columns are the segment's:
// position i for row i, and the source's own row numbers for the lower-
// triangle test (the row lists are increasing, so it gives the same answer).
__device__ __forceinline__ void load_relpos(const FactorArgs& a, const UTask& u, int* pos, int* grow,
                                            const int32_t* Rs, bool fan) {
  for (int i = threadIdx.x; i < u.rowlen; i += blockDim.x) {
    if (fan) {
      pos[i] = i;
      grow[i] = u.row0 + i;
      continue;
    }
    const int p = __ldg(a.relpos + u.rel + i);
    if (p < 0) atomicCAS(&a.ctrl[kErr], 0, SPCHOL_DEV_EINTERNAL);  // cannot happen for a consistent plan
    pos[i] = p;
    grow[i] = __ldg(Rs + u.row0 + i);
  }
}

__global__ void relpos_kernel(const UTask* __restrict__ ut, int n_u, const int32_t* __restrict__ rows,
                              const int64_t* __restrict__ rowoff, const int32_t* __restrict__ nrows,
                              int32_t* __restrict__ relpos) {
  for (int k = blockIdx.x; k < n_u; k += gridDim.x) {
    const UTask u = ut[k];
    const int32_t* Rs = rows + rowoff[u.s];
    const int32_t* Rt = rows + rowoff[u.t];
    const int rt = nrows[u.t];
    for (int i = threadIdx.x; i < u.rowlen; i += blockDim.x) {
      const int g = Rs[u.row0 + i];
      int lo = 0, hi = rt;
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (Rt[mid] < g) lo = mid + 1; else hi = mid;
      }
      relpos[u.rel + i] = (lo < rt && Rt[lo] == g) ? lo : -1;
    }
  }
}

// ---------------------------------------------------------------- UPD(s, t, k)
// C = A B^T for one tile, A = L_s[row tile] (rowlen x ws), B = L_s[segment]
// (ncol x ws), staged through shared memory in k-chunks.  Warp q owns the
// 8-row strip [8q, 8q + 8) of C; lane (lr, lc) = (lane / 8, lane % 8) holds
// rows 8q + lr + 4 rr (rr < NR) and columns lc + 8 cc (cc < NC).  Strips past
// rowlen, the second half of a strip with at most 4 valid rows, column blocks
// past ncol and, where the row tile overlaps the segment (the diagonal tiles),
// column blocks entirely above the diagonal are never computed: the FP64 pipe
// only runs on entries of the lower triangle, padded to 4 x 8 blocks.
// Operand staging.  A k-column of the tile (rows row0 .. row0 + len - 1 of one
// column of panel s) is copied in 16-byte pieces by cp.async (L2 only, no
// register round trip), starting at the 16-byte boundary at or below row0:
// the rows sit at offset row0 % E (E = 16 / sizeof(T)) of a shared-memory row
// of kStageStr elements.  A piece that would reach past the column's padded
// length ld is shortened to the elements inside it (the rest zero-filled), so
// no copy leaves the panel's storage.
template <typename T>
struct Stage {
  static constexpr int E = 16 / (int)sizeof(T);
  static constexpr int kStr = kUpdBoxRows((int)sizeof(T));  // row stride: 64 + E, a multiple of E
  static constexpr int kPieces = (kUpdTileM + E - 1) / E + 1;  // pieces per k-column, worst alignment
};

template <typename T>
__device__ __forceinline__ void cp_async16(T* dst, const T* src, int valid_elems) {
  const int bytes = valid_elems * (int)sizeof(T);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_addr(dst)), "l"(src), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// TMA staging.  When the handle has a tensor map per panel (a 2-D view of
// the column-major panel: ld rows x w columns, box kStr rows x kUpdKC
// columns), one thread loads a k-chunk of an operand with one
// cp.async.bulk.tensor whose x coordinate (the first row) is rounded down to
// a 16-byte boundary; rows past ld and columns past w arrive as zeros.  The
// copies complete on an mbarrier per buffer.
struct UpdTma {
  uint32_t mbar[2];  // shared addresses of the two buffers' mbarriers
  uint32_t* phase;   // shared: parity bits of the next completion of each
};

__device__ __forceinline__ void tma_load_2d(void* dst, const void* tmap, int x, int y, uint32_t mbar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
          "r"(smem_addr(dst)),
      "l"(tmap), "r"(x), "r"(y), "r"(mbar)
      : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t mbar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_wait_parity(uint32_t mbar, uint32_t phase) {
  for (int it = 0; it < (1 << 24); ++it) {
    uint32_t done;
    asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}"
                 : "=r"(done)
                 : "r"(mbar), "r"(phase)
                 : "memory");
    if (done) return true;
  }
  return false;
}

// Issue the copies of k-columns k0 .. k0 + kc - 1 of rows r0 .. r0 + len - 1 of
// a panel (column-major, leading dimension ld) into dst[kk][...].
template <typename T>
__device__ __forceinline__ void stage_cols(const T* __restrict__ P, int ld, int r0, int len, int k0, int kc,
                                           T* __restrict__ dst) {
  constexpr int E = Stage<T>::E, NP = Stage<T>::kPieces, STR = Stage<T>::kStr;
  const int base = r0 - (r0 % E);
  const int np = (r0 % E + len + E - 1) / E;  // pieces that cover the rows
  for (int idx = threadIdx.x; idx < kc * NP; idx += blockDim.x) {
    const int kk = idx / NP, pc = idx - kk * NP;
    if (pc < np) {
      const int row = base + pc * E;
      const int valid = min(E, ld - row);
      cp_async16(dst + kk * STR + pc * E, P + row + (size_t)(k0 + kk) * ld, valid);
    }
  }
}

// C = A B^T for one tile, A = L_s[row tile] (rowlen x ws), B = L_s[segment]
// (ncol x ws), staged through shared memory in k-chunks, double-buffered (the
// copies of chunk c + 1 are in flight while chunk c is multiplied).  Warp q owns
// the 8-row strip [8q, 8q + 8) of C; lane (lr, lc) = (lane / 8, lane % 8) holds
// rows 8q + lr + 4 rr (rr < NR) and columns lc + 8 cc (cc < NC).  Strips past
// rowlen, the second half of a strip with at most 4 valid rows, column blocks
// past ncol and, where the row tile overlaps the segment (the diagonal tiles),
// column blocks entirely above the diagonal are never computed: the FP64 pipe
// only runs on entries of the lower triangle, padded to 4 x 8 blocks.
template <typename acc_t, int NR, int NC>
__device__ __forceinline__ void upd_strip(const acc_t* __restrict__ As, const acc_t* __restrict__ Bs, int kc, int r0,
                                          int lc, acc_t (&acc)[2][8]) {
  constexpr int STR = Stage<acc_t>::kStr;
#pragma unroll 1
  for (int kk = 0; kk < kc; ++kk) {
    acc_t av[NR];
#pragma unroll
    for (int rr = 0; rr < NR; ++rr) av[rr] = As[kk * STR + r0 + 4 * rr];
#pragma unroll
    for (int cc = 0; cc < NC; ++cc) {
      const acc_t bv = Bs[kk * STR + lc + 8 * cc];
#pragma unroll
      for (int rr = 0; rr < NR; ++rr) acc[rr][cc] += av[rr] * bv;
    }
  }
}

template <typename acc_t, int NR>
__device__ __forceinline__ void upd_strip_nc(int nc, const acc_t* As, const acc_t* Bs, int kc, int r0, int lc,
                                             acc_t (&acc)[2][8]) {
  switch (nc) {
    case 1: upd_strip<acc_t, NR, 1>(As, Bs, kc, r0, lc, acc); break;
    case 2: upd_strip<acc_t, NR, 2>(As, Bs, kc, r0, lc, acc); break;
    case 3: upd_strip<acc_t, NR, 3>(As, Bs, kc, r0, lc, acc); break;
    case 4: upd_strip<acc_t, NR, 4>(As, Bs, kc, r0, lc, acc); break;
    case 5: upd_strip<acc_t, NR, 5>(As, Bs, kc, r0, lc, acc); break;
    case 6: upd_strip<acc_t, NR, 6>(As, Bs, kc, r0, lc, acc); break;
    case 7: upd_strip<acc_t, NR, 7>(As, Bs, kc, r0, lc, acc); break;
    default: upd_strip<acc_t, NR, 8>(As, Bs, kc, r0, lc, acc); break;
  }
}

template <typename T, bool FAN>
__device__ void task_update(const FactorArgs& a, const UTask u, unsigned char* smraw, FactorShared& sh,
                            bool skip, int rot, const UpdTma& tma, long long fo, bool release = true) {
  using acc_t = T;
  constexpr int STR = Stage<T>::kStr, E = Stage<T>::E;
  constexpr uint32_t kBoxBytes = (uint32_t)(kUpdKC * STR * sizeof(T));
  const int tid = threadIdx.x;
  const int s = u.s, t = u.t;
  if (!skip) {
    const int fs = a.pv.fcol[s], ws = a.pv.fcol[s + 1] - fs, lds = a.pv.ld[s];
    constexpr bool fan = FAN;  // fan-in mode: the tile's buffer at fo (see load_relpos)
    const int ft = fan ? u.seg0 : a.pv.fcol[t], ldt = fan ? u.rowlen : a.pv.ld[t];
    const T* Ps = panel_ptr<T>(a, s);
    T* Pt = fan ? reinterpret_cast<T*>(a.fan_buf) + fo : panel_ptr<T>(a, t);
    const int32_t* Rs = a.pv.rows + a.pv.rowoff[s];

    // [2][A, B][kUpdKC][STR], 128-byte aligned (each chunk is a multiple of 128 bytes)
    T* buf = reinterpret_cast<T*>(smraw + ((128u - (smem_addr(smraw) & 127u)) & 127u));
    const void* tmap = a.tmaps ? (const void*)(a.tmaps + 128 * (size_t)s) : nullptr;
    uint32_t ph = tmap ? *tma.phase : 0u;
    constexpr int kBuf = 2 * kUpdKC * STR;                // one buffer: A and B chunks
    // FP32 panels: the shared memory sized for two FP64 buffers holds four FP32
    // ones, so a tile of K <= 64 stages its whole K at once and waits once
    constexpr int kSlots = sizeof(T) == 4 ? 4 : 2;
    int* pos = reinterpret_cast<int*>(buf + kSlots * kBuf);  // [kUpdTileM] row position in t
    int* grow = pos + kUpdTileM;                          // [kUpdTileM] global row
    int* gcol = grow + kUpdTileM;                         // [kUpdTileN] global column (pass-local)

    // Relative row indices (computed once per analysis): position of each
    // row of the tile in t's sorted row list.
    load_relpos(a, u, pos, grow, Rs, fan);
    // Warp slot q' = (warp - rot) % 8 (tiles of few strips load the four SM
    // sub-partitions, warp % 4, evenly over many tasks).  A tile of S strips
    // gives each strip C = 8 / S (rounded down to a power of two) warps, which
    // split its column blocks: short tiles near the root keep every warp busy.
    const int lane = tid & 31, qs = ((tid >> 5) - rot) & 7;
    const int nstrip = (u.rowlen + 7) >> 3;
    const int C = nstrip >= 5 ? 1 : nstrip >= 3 ? 2 : nstrip == 2 ? 4 : 8;
    const int q = qs / C, cg = qs - q * C;              // strip and column group of this warp
    const int lr = lane >> 3, lc = lane & 7;
    const int srows = min(8, u.rowlen - 8 * q);        // valid rows of this warp's strip
    const int nr = srows > 4 ? 2 : 1;
    const int off = u.row0 - u.seg0;                   // >= 0: tile row i >= segment column j iff off + i >= j
    const int oa = u.row0 % E;                         // row offset of the A rows in shared memory
    const int r0 = oa + 8 * q + lr;                    // this lane's first A row in shared memory
    const int nchunk = (ws + kUpdKC - 1) / kUpdKC;
    for (int cb = 0; cb < u.seglen; cb += kUpdTileN) {
      const int ncol = min(kUpdTileN, u.seglen - cb);
      const int c0 = u.seg0 + cb;
      const int ob = c0 % E;
      const int dd = off - cb + 8 * q + 7;  // last column any row of the strip needs
      const int nall = (ncol + 7) >> 3;
      const int nper = (nall + C - 1) / C;
      const int b0 = cg * nper;             // this warp's column blocks b0 .. b0 + ncb - 1
      const int ncb = dd < 0 ? 0 : max(0, min(min(nall, b0 + nper), dd / 8 + 1) - b0);
      const bool active = srows > 0 && ncb > 0;
      __syncthreads();  // the previous pass is done with the buffers and gcol
      for (int j = tid; j < ncol; j += blockDim.x) gcol[j] = fan ? c0 + j : Rs[c0 + j];
      acc_t acc[2][8];
#pragma unroll
      for (int rr = 0; rr < 2; ++rr)
#pragma unroll
        for (int cc = 0; cc < 8; ++cc) acc[rr][cc] = acc_t(0);
      if (sizeof(T) == 4 && nchunk <= kSlots) {
        // every k-chunk in flight at once, one wait, then the arithmetic in
        // the same chunk order as below (the same sums)
        if (tmap) {
          if (tid == 0) {
            asm volatile("fence.proxy.async.global;" ::: "memory");
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_expect_tx(tma.mbar[0], 2 * kBoxBytes * (uint32_t)nchunk);
            for (int c = 0; c < nchunk; ++c) {
              tma_load_2d(buf + c * kBuf, tmap, u.row0 - oa, c * kUpdKC, tma.mbar[0]);
              tma_load_2d(buf + c * kBuf + kUpdKC * STR, tmap, c0 - ob, c * kUpdKC, tma.mbar[0]);
            }
          }
          if (!mbar_wait_parity(tma.mbar[0], ph & 1u) && tid == 0) atomicCAS(&a.ctrl[kErr], 0, SPCHOL_DEV_ETIMEOUT);
          ph ^= 1u;
        } else {
          for (int c = 0; c < nchunk; ++c) {
            const int k0 = c * kUpdKC, kc = min(kUpdKC, ws - k0);
            stage_cols(Ps, lds, u.row0, u.rowlen, k0, kc, buf + c * kBuf);
            stage_cols(Ps, lds, c0, ncol, k0, kc, buf + c * kBuf + kUpdKC * STR);
          }
          cp_async_commit();
          cp_async_wait<0>();
        }
        __syncthreads();
        if (active)
          for (int c = 0; c < nchunk; ++c) {
            const int kc = min(kUpdKC, ws - c * kUpdKC);
            const T* As = buf + c * kBuf;
            const T* Bs = As + kUpdKC * STR + ob + 8 * b0;
            if (nr == 2)
              upd_strip_nc<acc_t, 2>(ncb, As, Bs, kc, r0, lc, acc);
            else
              upd_strip_nc<acc_t, 1>(ncb, As, Bs, kc, r0, lc, acc);
          }
        __syncthreads();  // the buffers are refilled by the next pass or tile
      } else {
      // chunk 0 into buffer 0
      if (tmap) {
        if (tid == 0) {
          // the panel was written through the generic proxy (by other CTAs, or
          // by this one inside a subtree task); order that before the TMA reads
          asm volatile("fence.proxy.async.global;" ::: "memory");
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          mbar_expect_tx(tma.mbar[0], 2 * kBoxBytes);
          tma_load_2d(buf, tmap, u.row0 - oa, 0, tma.mbar[0]);
          tma_load_2d(buf + kUpdKC * STR, tmap, c0 - ob, 0, tma.mbar[0]);
        }
      } else {
        stage_cols(Ps, lds, u.row0, u.rowlen, 0, min(kUpdKC, ws), buf);
        stage_cols(Ps, lds, c0, ncol, 0, min(kUpdKC, ws), buf + kUpdKC * STR);
        cp_async_commit();
      }
      for (int c = 0; c < nchunk; ++c) {
        const int k0 = c * kUpdKC, kc = min(kUpdKC, ws - k0);
        if (tmap) {
          if (c + 1 < nchunk && tid == 0) {
            const int b1 = (c + 1) & 1;
            T* nb = buf + b1 * kBuf;
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_expect_tx(tma.mbar[b1], 2 * kBoxBytes);
            tma_load_2d(nb, tmap, u.row0 - oa, k0 + kUpdKC, tma.mbar[b1]);
            tma_load_2d(nb + kUpdKC * STR, tmap, c0 - ob, k0 + kUpdKC, tma.mbar[b1]);
          }
          const int b = c & 1;
          if (!mbar_wait_parity(tma.mbar[b], (ph >> b) & 1u) && tid == 0)
            atomicCAS(&a.ctrl[kErr], 0, SPCHOL_DEV_ETIMEOUT);
          ph ^= 1u << b;
        } else if (c + 1 < nchunk) {
          T* nb = buf + ((c + 1) & 1) * kBuf;
          const int k1 = k0 + kUpdKC, kc1 = min(kUpdKC, ws - k1);
          stage_cols(Ps, lds, u.row0, u.rowlen, k1, kc1, nb);
          stage_cols(Ps, lds, c0, ncol, k1, kc1, nb + kUpdKC * STR);
          cp_async_commit();
          cp_async_wait<1>();  // chunk c has landed (this thread's copies)
        } else {
          cp_async_wait<0>();
        }
        __syncthreads();       // ... and every thread's
        if (active) {
          const T* As = buf + (c & 1) * kBuf;
          const T* Bs = As + kUpdKC * STR + ob + 8 * b0;
          if (nr == 2)
            upd_strip_nc<acc_t, 2>(ncb, As, Bs, kc, r0, lc, acc);
          else
            upd_strip_nc<acc_t, 1>(ncb, As, Bs, kc, r0, lc, acc);
        }
        __syncthreads();  // buffer c & 1 is refilled by the next iteration's copies
      }
      }
      if (tmap && tid == 0) *tma.phase = ph;  // every thread has waited on the last chunk
      // Scatter-subtract into panel t: only the lower triangle (row >= column).
      if (active) {
#pragma unroll
        for (int rr = 0; rr < 2; ++rr) {
          const int i = 8 * q + lr + 4 * rr;
          if (rr >= nr || i >= u.rowlen || pos[i] < 0) continue;
          T* dst = Pt + pos[i];
          const int gi = grow[i];
#pragma unroll
          for (int cc = 0; cc < 8; ++cc) {
            const int j = lc + 8 * (b0 + cc);
            if (cc < ncb && j < ncol && gi >= gcol[j])
              scatter_put(dst + (size_t)(gcol[j] - ft) * ldt, (T)(-acc[rr][cc]), fan);
          }
        }
      }
    }
  }
  publish_cta_writes();
  target_update_done<FAN>(a, t, sh, release);  // not for a target inside the running subtree task
}

// ---------------------------------------------------------------- UPD on tensor cores (FP32 panels)
// The same update tile computed with tcgen05.mma kind::tf32: A (tile rows, up
// to 128) and B (segment rows, up to 64 per pass) are staged K-major in shared
// memory (8-row x 16-byte core matrices, no swizzle), one elected thread issues
// the MMAs into a TMEM accumulator (128 lanes x 64 columns, allocated once per
// CTA), the commit arrives on an mbarrier, and the epilogue reads TMEM by warp
// quadrant and scatter-adds into the target panel.  With split = 1 each operand
// is also split into a TF32 high part and a TF32 remainder, and three products
// (hi*hi + hi*lo + lo*hi) recover FP32-level accuracy.
struct TcState {
  uint32_t tmem;   // TMEM base address of this CTA's accumulator
  uint32_t mbar;   // shared address of the MMA-completion mbarrier
  uint32_t phase;  // parity of the next completion
};


// Shared-memory matrix descriptor: K-major, no swizzle; LBO = byte distance of
// K-adjacent core matrices, SBO = byte distance of row-adjacent core matrices.
__device__ __forceinline__ uint64_t kmajor_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

// Instruction descriptor: FP32 accumulator, TF32 A and B, both K-major, M x N.
__device__ __forceinline__ uint32_t tf32_idesc(int m, int n) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ float to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// Byte offset of element (r, k) in a K-major tile whose rows hold kpad fp32 values.
__device__ __forceinline__ uint32_t kmaj_off(int r, int k, int kpad) {
  return (uint32_t)((r >> 3) * (kpad * 32) + (k >> 2) * 128 + (r & 7) * 16 + (k & 3) * 4);
}

constexpr int kTcM = 128;      // MMA rows (tile rows are padded up to it)
constexpr int kTcN = 64;       // accumulator columns per pass
constexpr int kTcKmax = 64;    // panel width bound for the tensor-core path

__device__ __forceinline__ bool mbar_wait_bounded(uint32_t mbar, uint32_t phase) {
  for (int it = 0; it < (1 << 24); ++it) {
    uint32_t done;
    asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}"
                 : "=r"(done)
                 : "r"(mbar), "r"(phase)
                 : "memory");
    if (done) return true;
  }
  return false;
}

template <bool FAN>
__device__ void task_update_tc(const FactorArgs& a, const UTask u, unsigned char* smraw, FactorShared& sh, bool skip,
                               TcState& tc, long long fo, bool release = true) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int s = u.s, t = u.t;
  if (!skip) {
    const int fs = a.pv.fcol[s], ws = a.pv.fcol[s + 1] - fs, lds = a.pv.ld[s];
    constexpr bool fan = FAN;  // fan-in mode: the tile's buffer at fo (see load_relpos)
    const int ft = fan ? u.seg0 : a.pv.fcol[t], ldt = fan ? u.rowlen : a.pv.ld[t];
    const float* Ps = reinterpret_cast<const float*>(a.pool) + a.pv.valoff[s];
    float* Pt = fan ? reinterpret_cast<float*>(a.fan_buf) + fo : reinterpret_cast<float*>(a.pool) + a.pv.valoff[t];
    const int32_t* Rs = a.pv.rows + a.pv.rowoff[s];
    const int split = a.mma_mode == 2 ? 1 : 0;
    const int kpad = (ws + 7) & ~7;
    const int abytes = kTcM * kpad * 4, bbytes = kTcN * kpad * 4;
    // operand tiles start on a 128-byte boundary of shared memory
    unsigned char* Ah = smraw + ((128u - (smem_addr(smraw) & 127u)) & 127u);
    unsigned char* Bh = Ah + abytes;
    unsigned char* Al = Bh + bbytes;           // remainders (split only)
    unsigned char* Bl = Al + abytes;
    int* pos = reinterpret_cast<int*>(Ah + 2 * (abytes + bbytes));
    int* grow = pos + kTcM;
    int* gcol = grow + kTcM;

    load_relpos(a, u, pos, grow, Rs, fan);
    // A: tile rows x k (rows >= rowlen and k >= ws are zero)
    for (int idx = tid; idx < kTcM * kpad; idx += blockDim.x) {
      const int i = idx % kTcM, k = idx / kTcM;
      const float v = (i < u.rowlen && k < ws) ? ldcg(Ps + (u.row0 + i) + (size_t)k * lds) : 0.f;
      const float h = to_tf32(v);
      *reinterpret_cast<float*>(Ah + kmaj_off(i, k, kpad)) = h;
      if (split) *reinterpret_cast<float*>(Al + kmaj_off(i, k, kpad)) = to_tf32(v - h);
    }
    for (int cb = 0; cb < u.seglen; cb += kTcN) {
      const int ncol = min(kTcN, u.seglen - cb);
      const int npad = kTcN;  // the MMA always spans the full accumulator width; unused B rows are zero
      for (int j = tid; j < ncol; j += blockDim.x) gcol[j] = fan ? u.seg0 + cb + j : Rs[u.seg0 + cb + j];
      for (int idx = tid; idx < npad * kpad; idx += blockDim.x) {
        const int j = idx % npad, k = idx / npad;
        const float v = (j < ncol && k < ws) ? ldcg(Ps + (u.seg0 + cb + j) + (size_t)k * lds) : 0.f;
        const float h = to_tf32(v);
        *reinterpret_cast<float*>(Bh + kmaj_off(j, k, kpad)) = h;
        if (split) *reinterpret_cast<float*>(Bl + kmaj_off(j, k, kpad)) = to_tf32(v - h);
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncthreads();
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      if (tid == 0) {
        const uint32_t idesc = tf32_idesc(kTcM, npad);
        const uint32_t sbo = (uint32_t)kpad * 32;
        const uint32_t ah = smem_addr(Ah), bh = smem_addr(Bh), al = smem_addr(Al), bl = smem_addr(Bl);
        int first = 1;
        for (int k0 = 0; k0 < kpad; k0 += 8) {
          const uint32_t off = (uint32_t)(k0 >> 2) * 128;  // two K-adjacent core matrices per MMA
          const int nprod = split ? 3 : 1;
          for (int pr = 0; pr < nprod; ++pr) {
            const uint32_t aa = (pr == 2) ? al : ah;
            const uint32_t bb = (pr == 1) ? bl : bh;
            const uint64_t ad = kmajor_desc(aa + off, 128, sbo);
            const uint64_t bd = kmajor_desc(bb + off, 128, sbo);
            const uint32_t acc = first ? 0u : 1u;
            asm volatile("{\n.reg .pred p;\nsetp.ne.u32 p, %4, 0;\n"
                         "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(tc.tmem),
                         "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
                         : "memory");
            first = 0;
          }
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(tc.mbar)
                     : "memory");
      }
      const bool ok = mbar_wait_bounded(tc.mbar, tc.phase);
      tc.phase ^= 1u;
      if (!ok && tid == 0) atomicCAS(&a.ctrl[kErr], 0, SPCHOL_DEV_ETIMEOUT);
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      // epilogue: warp w reads TMEM lanes 32*(w%4).. (tile rows), columns half (w/4)
      const int quad = warp & 3, half = warp >> 2;
      const int row = 32 * quad + lane;
      for (int c0 = half * 32; c0 < half * 32 + 32; c0 += 16) {
        uint32_t v[16];
        const uint32_t taddr = tc.tmem + ((uint32_t)(32 * quad) << 16) + (uint32_t)c0;
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
              "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
            : "r"(taddr));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (ok && row < u.rowlen && pos[row] >= 0) {
#pragma unroll
          for (int q = 0; q < 16; ++q) {
            const int j = c0 + q;
            if (j < ncol && grow[row] >= gcol[j])
              scatter_put(Pt + pos[row] + (size_t)(gcol[j] - ft) * ldt, -__uint_as_float(v[q]), fan);
          }
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncthreads();  // TMEM and the B tile are reused by the next pass / task
    }
  }
  publish_cta_writes();
  target_update_done<FAN>(a, t, sh, release);  // not for a target inside the running subtree task
}

// ---------------------------------------------------------------- UPD, FP64 on BF16 tensor cores
// C = A B^T with A, B given by their kSlices digit matrices (see slice_row):
// C_ij = 2^(e_i + e_j) sum_{p,q} 2^(-8(p+q+2)) (A_p B_q^T)_ij.  The products
// with p + q <= kSlices - 1 are kept (the dropped ones weigh below 2^-64 of
// the leading one); products of equal p + q share one TMEM accumulator
// (group d = p + q, kOzN columns each), in which the integer sums stay exact
// for d <= 3 and round at most at 2^-56 relative beyond.  The epilogue
// combines the seven group values per entry exactly in two 64-bit integers,
// converts once to FP64 and scales by 2^(e_i + e_j).
// The double nearest to t * 2^k for a 64-bit integer t, with integer
// operations only (round to nearest, ties to even).
__device__ __forceinline__ double fixed64_to_double(long long t, int k) {
  if (t == 0) return 0.0;
  const bool neg = t < 0;
  const unsigned long long u = neg ? (unsigned long long)(-t) : (unsigned long long)t;
  int msb = 63 - __clzll((long long)u);
  unsigned long long m;
  if (msb <= 52) {
    m = u << (52 - msb);
  } else {
    const int sh = msb - 52;
    m = u >> sh;
    const unsigned long long rem = u & ((1ull << sh) - 1), halfw = 1ull << (sh - 1);
    if (rem > halfw || (rem == halfw && (m & 1ull))) {
      ++m;
      if (m >> 53) {
        m >>= 1;
        ++msb;
      }
    }
  }
  const int be = msb + k + 1023;
  if (be <= 0 || be >= 2047) {
    const double r = ldexp((double)m, msb - 52 + k);  // outside the range of this path's data
    return neg ? -r : r;
  }
  return __longlong_as_double(
      (long long)(((unsigned long long)neg << 63) | ((unsigned long long)be << 52) | (m & ((1ull << 52) - 1))));
}

// The MMAs have M = 64 (the tile's at most kOzRows = 64 rows) and cover one
// 16-column block of the segment: the accumulator of group d is TMEM columns
// 16 d .. 16 d + 15.  With M = 64 the accumulator's row 16 q + i (i < 16) sits
// in TMEM lane 32 q + i, columns as N.  7 groups x 16 columns fit 128 TMEM
// columns, a quarter of the SM's, and a CTA needs 73 KB of shared memory, so
// three CTAs share an SM.  A tcgen05.mma costs about the same to issue whatever
// its M and N (~48 clocks from one thread, ~28 SM-wide when several issue), so
// the MMA phase is bound by the instruction count: each A digit p is issued
// once per K step against the stacked B digits 0 .. 6 - p (N up to 112),
// 28 MMAs per block instead of 112 single products.
constexpr int kOzM = 64, kOzN = 16, kOzRows = 64;
constexpr int kOzCols = 128;  // TMEM columns: kSlices groups x kOzN, rounded to a power of two

__device__ __forceinline__ uint32_t bf16_idesc(int m, int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

template <bool FAN>
__device__ void task_update_oz(const FactorArgs& a, const UTask u, unsigned char* smraw, FactorShared& sh, bool skip,
                               TcState& tc, long long fo, bool release = true) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int s = u.s, t = u.t;
  if (!skip) {
    const int fs = a.pv.fcol[s], ws = a.pv.fcol[s + 1] - fs, rs = a.pv.nrows[s];
    constexpr bool fan = FAN;  // fan-in mode: the tile's buffer at fo (see load_relpos)
    const int ft = fan ? u.seg0 : a.pv.fcol[t], ldt = fan ? u.rowlen : a.pv.ld[t];
    double* Pt = fan ? reinterpret_cast<double*>(a.fan_buf) + fo : reinterpret_cast<double*>(a.pool) + a.pv.valoff[t];
    const int32_t* Rs = a.pv.rows + a.pv.rowoff[s];
    const int32_t* ex = a.rexp + a.pv.rowoff[s];
    const int kpad = (ws + 15) & ~15, nb = rs - ws;
    const uint16_t* sl = a.slices + a.sliceoff[s];
    const int arow = kOzRows * kpad * 2, brow = kOzN * kpad * 2;  // bytes of one slice tile
    unsigned char* A0 = smraw + ((128u - (smem_addr(smraw) & 127u)) & 127u);
    unsigned char* B0 = A0 + kSlices * arow;
    int* pos = reinterpret_cast<int*>(B0 + kSlices * brow);
    int* grow = pos + kOzRows;
    int* gcol = grow + kOzRows;
    int* ea = gcol + kOzN;
    int* eb = ea + kOzRows;
    const uint32_t sbo = (uint32_t)kpad * 16;  // 8 rows x (kpad bf16) bytes
    const int chunks = kpad / 8;               // 16-byte chunks per row

    load_relpos(a, u, pos, grow, Rs, fan);
    for (int i = tid; i < u.rowlen; i += blockDim.x) ea[i] = ldcg(ex + u.row0 + i);
    // A digits: kSlices x rowlen rows x kpad, K-major core matrices (8 rows x
    // 16 bytes).  Rows past rowlen are left as they are: they only feed rows
    // of the product that are never scattered.  Columns past ws are zero in
    // the slices themselves.
    // 16-byte pieces by cp.async (L2 only): every piece of the tile is in
    // flight at once instead of one load's latency per piece
    for (int idx = tid; idx < kSlices * u.rowlen * chunks; idx += blockDim.x) {
      const int c = idx % chunks, pr = idx / chunks;
      const int p = pr / u.rowlen, r = pr - p * u.rowlen;
      const uint16_t* src = sl + ((size_t)p * nb + (u.row0 - ws + r)) * kpad + 8 * c;
      unsigned char* dst = A0 + p * arow + (r >> 3) * sbo + (r & 7) * 16 + c * 128;
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
    }
    cp_async_commit();
    for (int cb = 0; cb < u.seglen; cb += kOzN) {
      const int ncol = min(kOzN, u.seglen - cb);
      for (int j = tid; j < ncol; j += blockDim.x) {
        gcol[j] = fan ? u.seg0 + cb + j : Rs[u.seg0 + cb + j];
        eb[j] = ldcg(ex + u.seg0 + cb + j);
      }
      for (int idx = tid; idx < kSlices * ncol * chunks; idx += blockDim.x) {
        const int c = idx % chunks, pr = idx / chunks;
        const int p = pr / ncol, r = pr - p * ncol;
        const uint16_t* src = sl + ((size_t)p * nb + (u.seg0 + cb - ws + r)) * kpad + 8 * c;
        unsigned char* dst = B0 + p * brow + (r >> 3) * sbo + (r & 7) * 16 + c * 128;
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
      }
      cp_async_commit();
      cp_async_wait<0>();  // this thread's A (first pass) and B pieces have landed
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncthreads();
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      if (tid == 0) {
        // One MMA per A digit p and K step: its B operand is the run of B
        // digits 0 .. 6 - p (N = (7 - p) x 16 rows, contiguous in shared
        // memory), its accumulator starts at group p's columns, so the product
        // with B digit q lands in group p + q.  28 MMAs per block instead of
        // one per (p, q) pair (112); the first (p = 0, all groups) initialises.
        const uint32_t a0 = smem_addr(A0), b0 = smem_addr(B0);
        for (int p = 0; p < kSlices; ++p) {
          const uint32_t idesc = bf16_idesc(kOzM, (kSlices - p) * kOzN);
          const uint32_t dcol = tc.tmem + (uint32_t)(p * kOzN);
          for (int k0 = 0; k0 < kpad; k0 += 16) {
            const uint32_t off = (uint32_t)(k0 >> 3) * 128;  // 16 bf16 = two K-adjacent core matrices
            const uint64_t ad = kmajor_desc(a0 + p * arow + off, 128, sbo);
            const uint64_t bd = kmajor_desc(b0 + off, 128, sbo);
            const uint32_t acc = (p == 0 && k0 == 0) ? 0u : 1u;
            asm volatile("{\n.reg .pred pp;\nsetp.ne.u32 pp, %4, 0;\n"
                         "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, pp;\n}" ::"r"(dcol),
                         "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
                         : "memory");
          }
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(tc.mbar)
                     : "memory");
      }
      const bool ok = mbar_wait_bounded(tc.mbar, tc.phase);
      tc.phase ^= 1u;
      if (!ok && tid == 0) atomicCAS(&a.ctrl[kErr], 0, SPCHOL_DEV_ETIMEOUT);
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      // Epilogue: warp w reads TMEM lanes 32*(w%4).. (lanes 0..15 of them hold
      // tile rows 16*(w%4)..) and a column half; warps whose rows or columns
      // are all unused skip (tcgen05.ld is warp-collective, so the condition
      // is warp-uniform).
      const int quad = warp & 3, half = warp >> 2;
      const int row = 16 * quad + lane;
      constexpr int kHalf = kOzN / 2;
      if (16 * quad < u.rowlen) {
        for (int c0 = half * kHalf; c0 < half * kHalf + kHalf && c0 < ncol; c0 += 8) {
          uint32_t v[kSlices][8];
#pragma unroll
          for (int d = 0; d < kSlices; ++d) {
            const uint32_t taddr = tc.tmem + ((uint32_t)(32 * quad) << 16) + (uint32_t)(d * kOzN + c0);
            asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                         : "=r"(v[d][0]), "=r"(v[d][1]), "=r"(v[d][2]), "=r"(v[d][3]), "=r"(v[d][4]),
                           "=r"(v[d][5]), "=r"(v[d][6]), "=r"(v[d][7])
                         : "r"(taddr));
          }
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
          if (ok && lane < 16 && row < u.rowlen && pos[row] >= 0) {
#pragma unroll
            for (int q = 0; q < 8; ++q) {
              const int j = c0 + q;
              if (j < ncol && grow[row] >= gcol[j]) {
                // t = sum_d v_d 2^(8 (6 - d)), C = t 2^(e_i + e_j - 64).  The group
                // sums are integers below 2^25 in magnitude; t (< 2^75) is formed
                // as hi 2^32 + lo and kept to 2^12 units in one int64, a
                // truncation of at most 2^(e_i + e_j - 52), below the rounding
                // bound of an FP64 dot product of these rows.
                long long hi = 0, lo = 0;
#pragma unroll
                for (int d = 0; d < 3; ++d) hi = hi * 256 + __float2int_rn(__uint_as_float(v[d][q]));
#pragma unroll
                for (int d = 3; d < kSlices; ++d) lo = lo * 256 + __float2int_rn(__uint_as_float(v[d][q]));
                const long long t12 = hi * (1ll << 20) + (lo >> 12);  // floor((hi 2^32 + lo) / 2^12)
                const double c = fixed64_to_double(t12, ea[row] + eb[j] - 52);
                scatter_put(Pt + pos[row] + (size_t)(gcol[j] - ft) * ldt, -c, fan);
              }
            }
          }
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncthreads();
    }
  }
  publish_cta_writes();
  target_update_done<FAN>(a, t, sh, release);  // not for a target inside the running subtree task
}

// ---------------------------------------------------------------- fan-in gather
// Deterministic fan-in mode (the fan-in family of Section II-C, restated for
// one GPU): update tiles store their products in private buffers, and a
// gather task per piece of a target panel's rows (at most kFanPieceRows rows,
// all columns) adds them in, tile after tile in the piece's list order, before
// the task that owns those rows factors or solves them; every entry of L thus
// receives its updates in one fixed order whatever the schedule, and the
// pieces of one panel are gathered in parallel.  The piece sits in shared
// memory and the list is consumed in batches of up to kFanBatch tiles:
//   1. warp 0 cuts the batch where its staged values would overflow the
//      staging area (the records were fetched during the previous batch);
//   2. all threads copy, for each column of each tile, the 16-byte pieces that
//      hold its rows in the piece (cp.async, L2 only: the buffers were written
//      by other CTAs; every copy of the batch in flight at once) and load the
//      rows' positions in the piece and the columns' positions in the panel;
//   3. the values are added tile by tile (a barrier between tiles).
// The piece and the buffers are read around L1; the records were written at
// analysis.
struct FanMeta {
  long long fo, rp, rs;  // FanRec: buffer offset of the first listed row, relative rows, segment rows
  int pre_b, pre_v;      // the tile's first staged 16-byte piece and first staged position
  int rowlen, cps;       // buffer rows; staged pieces per column
  short ni, seglen;
  float inv_ni;  // 1 / ni: value index -> (row, column) without a division
  float inv_cps;
};
constexpr int kFanBatch = 32;
constexpr int kFanVcap = 1024;  // staged positions per batch (a tile has at most 32 + 128)
constexpr size_t kFanMetaBytes = ((kFanBatch * sizeof(FanMeta) + 16) + 15) & ~size_t(15);

// 16-byte pieces that can hold ni consecutive values starting anywhere.
template <typename T>
__host__ __device__ constexpr int fan_pieces(int ni) {
  return (ni + 16 / (int)sizeof(T) - 2) / (16 / (int)sizeof(T)) + 1;
}

// The batch tile that staged piece (pieces) or position (!pieces) idx belongs to.
__device__ __forceinline__ int fan_tile_of(const FanMeta* meta, int nb, int idx, bool pieces) {
  int k = 0;
#pragma unroll
  for (int b = kFanBatch / 2; b > 0; b >>= 1)
    if (k + b < nb && (pieces ? meta[k + b].pre_b : meta[k + b].pre_v) <= idx) k += b;
  return k;
}

template <typename T>
__device__ void fanin_gather(const FactorArgs& a, int t, int pc, int p0, int np, unsigned char* smraw) {
  constexpr int E = 16 / (int)sizeof(T);  // values per 16-byte piece
  const int tid = threadIdx.x, nt = blockDim.x;
  long long e = a.fan_ptr[pc];
  const long long e1 = a.fan_ptr[pc + 1];
  if (e == e1) return;  // nothing lands in these rows
  const int ft = a.pv.fcol[t], wt = a.pv.fcol[t + 1] - ft, ldt = a.pv.ld[t];
  T* Pt = panel_ptr<T>(a, t);
  const T* F = reinterpret_cast<const T*>(a.fan_buf);
  const int cap = a.fan_cap;  // 16-byte pieces per batch; one tile's always fit
  unsigned char* base = smraw + ((16u - (smem_addr(smraw) & 15u)) & 15u);
  FanMeta* meta = reinterpret_cast<FanMeta*>(base);
  int* scal = reinterpret_cast<int*>(meta + kFanBatch);  // tiles, pieces and positions of the batch
  int16_t* pv = reinterpret_cast<int16_t*>(base + kFanMetaBytes);  // positions: rows in the piece, then columns
  T* Bs = reinterpret_cast<T*>(pv + kFanVcap);                     // the staged pieces
  T* S = Bs + (size_t)cap * E;  // the piece: np rows x wt columns, leading dimension kFanPieceRows
  for (int idx = tid; idx < np * wt; idx += nt) {
    const int p = idx % np, c = idx / np;
    S[p + kFanPieceRows * c] = ldcg(Pt + p0 + p + (size_t)c * ldt);
  }
  FanRec r{};  // warp 0: the records of the next batch window
  if (tid < 32 && e + tid < e1) r = a.fan_rec[e + tid];
  const bool prof = a.prof != nullptr && tid == 0;
  uint64_t tp[3] = {0, 0, 0}, tq = prof ? global_ns() : 0;
  long long nbat = 0, ntile = 0;
  while (e < e1) {
    __syncthreads();  // the piece is loaded, or the previous batch is added
    int nb = 0;
    if (tid < 32) {
      const bool have = e + tid < e1;
      const int cps = have ? fan_pieces<T>(r.ni) : 0;
      const int n = have ? r.seglen * cps : 0, v = have ? r.ni + r.seglen : 0;
      int in = n, iv = v;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, in, o), z = __shfl_up_sync(0xffffffffu, iv, o);
        if (tid >= o) {
          in += y;
          iv += z;
        }
      }
      // the tiles that fit form a prefix; the first one always fits
      nb = max(1, __popc(__ballot_sync(0xffffffffu, have && in <= cap && iv <= kFanVcap)));
      if (tid < nb) {
        FanMeta mm;
        mm.fo = r.fo;
        mm.rp = r.rp;
        mm.rs = r.rs;
        mm.pre_b = in - n;
        mm.pre_v = iv - v;
        mm.rowlen = r.rowlen;
        mm.cps = cps;
        mm.ni = r.ni;
        mm.seglen = r.seglen;
        mm.inv_ni = 1.0f / (float)max(1, (int)r.ni);
        mm.inv_cps = 1.0f / (float)max(1, cps);
        meta[tid] = mm;
      }
      if (tid == nb - 1) {
        scal[0] = nb;
        scal[1] = in;
        scal[2] = iv;
      }
      r = FanRec{};
      if (e + nb + tid < e1) r = a.fan_rec[e + nb + tid];  // in flight during this batch
    }
    __syncthreads();
    if (prof) {
      const uint64_t tn = global_ns();
      tp[0] += tn - tq;
      tq = tn;
    }
    nb = scal[0];
    int npc = scal[1], npos = scal[2];
    if (npc > cap || npos > kFanVcap) {  // cannot happen for a consistent plan
      if (tid == 0) atomicCAS(&a.ctrl[kErr], 0, SPCHOL_DEV_EINTERNAL);
      npc = npos = 0;
    }
    // 2. the pieces that hold each column's rows (the 16-byte piece at or below
    // its first value, and on), and the positions
    for (int idx = tid; idx < npc; idx += nt) {
      const FanMeta& mk = meta[fan_tile_of(meta, nb, idx, true)];
      const int lp = idx - mk.pre_b;
      // lp / cps exactly: lp < 2^12 and cps <= 17 leave a margin of 1 / 34 for rounding
      const int j = (int)(((float)lp + 0.5f) * mk.inv_cps), q = lp - j * mk.cps;
      const long long g0 = mk.fo + (long long)j * mk.rowlen;  // the column's first value
      const long long a0 = (g0 & ~(long long)(E - 1)) + (long long)q * E;
      if (a0 < g0 + mk.ni)  // a piece past the column's last value holds nothing it needs
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(Bs + (size_t)idx * E)),
                     "l"(F + a0)
                     : "memory");
    }
    cp_async_commit();
    for (int idx = tid; idx < npos; idx += nt) {
      const FanMeta& mk = meta[fan_tile_of(meta, nb, idx, false)];
      const int lv = idx - mk.pre_v;
      int q;
      bool ok;
      if (lv < mk.ni) {
        q = __ldg(a.relpos + mk.rp + lv) - p0;
        ok = q >= 0 && q < np;
      } else {
        q = __ldg(a.pv.rows + mk.rs + (lv - mk.ni)) - ft;
        ok = q >= 0 && q < wt;
      }
      if (!ok) atomicCAS(&a.ctrl[kErr], 0, SPCHOL_DEV_EINTERNAL);  // outside the piece: an inconsistent plan
      pv[idx] = ok ? (int16_t)q : (int16_t)-1;
    }
    cp_async_wait<0>();
    __syncthreads();
    if (prof) {
      const uint64_t tn = global_ns();
      tp[1] += tn - tq;
      tq = tn;
    }
    // 3. tile by tile: an entry's updates land in list order
    for (int k = 0; k < nb; ++k) {
      const FanMeta& mk = meta[k];
      const int ni = mk.ni, n = ni * mk.seglen;
      for (int idx = tid; idx < n; idx += nt) {
        // idx / ni exactly: idx < 2^12 and ni <= 32 leave a margin of 1 / 64 for rounding
        const int j = (int)(((float)idx + 0.5f) * mk.inv_ni), ii = idx - j * ni;
        const int p = pv[mk.pre_v + ii], c = pv[mk.pre_v + ni + j];
        // lower triangle of the target (rows below its diagonal block always are)
        if (p >= 0 && c >= 0 && (p0 + p >= wt || p0 + p >= c)) {
          const int sub = (int)((mk.fo + (long long)j * mk.rowlen) & (E - 1));
          S[p + kFanPieceRows * c] += Bs[(size_t)(mk.pre_b + j * mk.cps) * E + sub + ii];
        }
      }
      __syncthreads();
    }
    if (prof) {
      const uint64_t tn = global_ns();
      tp[2] += tn - tq;
      tq = tn;
      ++nbat;
      ntile += nb;
    }
    e += nb;
  }
  for (int idx = tid; idx < np * wt; idx += nt) {
    const int p = idx % np, c = idx / np;
    Pt[p0 + p + (size_t)c * ldt] = S[p + kFanPieceRows * c];
  }
  if (prof) {
    for (int k = 0; k < 3; ++k) atomicAdd(&a.prof[10 + k], (unsigned long long)tp[k]);
    atomicAdd(&a.prof[13], (unsigned long long)nbat);
    atomicAdd(&a.prof[14], (unsigned long long)ntile);
  }
  __syncthreads();  // the task reads these rows next, and reuses the shared memory
}

// ---------------------------------------------------------------- warp-level subtree tasks
// A subtree task whose panels are all at most kWarpSubW columns wide
// (FactorArgs::wsub) runs on one warp, before the warps of its CTA join the
// task loop: the many small subtrees of a batch of small matrices, or the
// leaves of a large one, then advance kWarpExec per CTA side by side with warp
// barriers only, where a CTA subtree task runs one of them with CTA barriers
// at every column and step.  A warp-wide FP64 instruction holds the SM's FP64
// pipe as long whatever its active lanes (the pipe bounds these warps), so
// each step spreads its entries over the lanes.  Per panel, in postorder:
//   * the diagonal block in shared memory (leading dimension kWarpLd): each
//     multiplier, update and pivot is the diagonal task's operation on the
//     same operands in the same order, so L11 is the same; the lane of row i
//     forms its multiplier, then the trailing triangle's updates take one
//     entry per lane and pass, as does the scaling L = M D^{1/2};
//   * its inverse by the diagonal task's substitution (the same operations
//     per entry), each step's entries one per lane and pass;
//   * the panel solve by that inverse, l_rc = sum_{k <= c} a_rk X_ck, one
//     output per lane and pass (the panel-solve tiles of the task loop solve
//     by substitution instead: they run before the inverse exists);
//   * the update tiles, one output per lane at a time (a dot product over the
//     panel's columns in two chains): into panels inside the subtree by plain
//     read-modify-write (no other task touches them), into the others by
//     atomics, each tile then counted down on its target as a CTA subtree task
//     does.
// After a failed pivot (here or anywhere) the rest of the subtree skips its
// arithmetic but still counts its outside targets down.
// Entry p of a lower triangle numbered row by row (p = a (a + 1) / 2 + b,
// 0 <= b <= a): row a, column b.  The float square root is exact at the
// triangular numbers; the two corrections absorb its rounding elsewhere.
__device__ __forceinline__ void tri_decode(int p, int& ra, int& cb) {
  int t = (int)((sqrtf(8.0f * (float)p + 1.0f) - 1.0f) * 0.5f);
  if ((t + 1) * (t + 2) / 2 <= p) ++t;
  if (t * (t + 1) / 2 > p) --t;
  ra = t;
  cb = p - t * (t + 1) / 2;
}

constexpr int kWarpLd = kWarpSubW + 1;
constexpr int kWarpExec = 4;                                   // warps of a CTA that run them
constexpr int kWarpSmem = kWarpSubW * kWarpLd + kWarpSubW;     // doubles per warp: the block, 1 / l_jj

template <typename T>
__device__ void warp_subtree(const FactorArgs& a, int k, double* ws) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int lo = a.sub_lo[k], hi = a.sub_hi[k];
  double* xd = ws + kWarpSubW * kWarpLd;
  bool skip = ld_relaxed(&a.ctrl[kInfo]) != INT_MAX;
  const Ring2 q = rings_of(a);
  for (int s = lo; s <= hi; ++s) {
    const int f = a.pv.fcol[s], w = a.pv.fcol[s + 1] - f, ld = a.pv.ld[s], r = a.pv.nrows[s];
    T* P = panel_ptr<T>(a, s);
    if (!skip) {
      for (int idx = lane; idx < w * w; idx += 32) {
        const int i = idx % w, j = idx / w;
        ws[i + j * kWarpLd] = i >= j ? (double)ldcg(P + i + (size_t)j * ld) : 0.0;  // zeros above: the inverse goes there
      }
      __syncwarp();
      double qj = 0.0;  // lane j: 1 / d_j
      int bad = 0;
      if (lane == 0) {
        const double d0 = ws[0];
        if (d0 > 0.0)
          qj = pivot_recip(d0);
        else
          bad = 1;
      }
      if (__any_sync(full, bad)) {
        if (lane == 0) atomicMin(&a.ctrl[kInfo], f + 1);
        skip = true;
      }
      for (int j = 0; j < w && !skip; ++j) {
        const double qv = __shfl_sync(full, qj, j);
        const bool mine = lane > j && lane < w;
        const double ci = mine ? ws[lane + j * kWarpLd] * qv : 0.0;  // the multiplier of row lane
        // the trailing triangle a_ik -= c_i a_kj (j < k <= i < w), one entry
        // per lane and pass; column j is read here and rewritten only below
        const int m = w - j - 1, ntri = m * (m + 1) / 2;
        for (int p0 = 0; p0 < ntri; p0 += 32) {
          const int p = p0 + lane;
          int ta, tb;
          tri_decode(p < ntri ? p : 0, ta, tb);
          const int i = j + 1 + ta, kk = j + 1 + tb;
          const double c = __shfl_sync(full, ci, i);
          if (p < ntri) ws[i + kk * kWarpLd] = fma(-c, ws[kk + j * kWarpLd], ws[i + kk * kWarpLd]);
        }
        __syncwarp();
        if (lane == j + 1 && lane < w) {
          const double d = ws[lane * (kWarpLd + 1)];
          if (d > 0.0)
            qj = pivot_recip(d);
          else
            bad = 1;
        }
        if (mine) ws[lane + j * kWarpLd] = ci;  // column j now holds the multipliers
        if (__any_sync(full, bad)) {
          if (lane == 0) atomicMin(&a.ctrl[kInfo], f + j + 2);
          skip = true;
        }
        __syncwarp();
      }
      if (!skip) {
        // L = M D^{1/2}: l_jj = sqrt(d_j), r_j = 1 / l_jj, l_ij = m_ij l_jj (one
        // entry of the strictly lower triangle per lane and pass)
        if (lane < w) {
          const double l = sqrt(ws[lane * (kWarpLd + 1)]);
          ws[lane * (kWarpLd + 1)] = l;
          xd[lane] = 1.0 / l;
        }
        __syncwarp();
        for (int p = lane; p < w * (w - 1) / 2; p += 32) {
          int ta, tb;
          tri_decode(p, ta, tb);
          ws[ta + 1 + tb * kWarpLd] *= ws[tb * (kWarpLd + 1)];
        }
        __syncwarp();
        for (int idx = lane; idx < w * w; idx += 32) {
          const int i = idx % w, j = idx / w;
          if (i >= j) P[i + (size_t)j * ld] = (T)ws[i + j * kWarpLd];
        }
        // L11^{-1}: X_ic (i > c) in the upper triangle at (c, i); step kk adds
        // -l_ik X_kc to every X_ic with c <= kk < i (one per lane and pass) and
        // completes X_{kk+1,c} by 1 / l_{kk+1,kk+1}
        for (int kk = 0; kk < w - 1; ++kk) {
          const int nc = kk + 1, n = nc * (w - kk - 1);
          for (int p = lane; p < n; p += 32) {
            const int c = p % nc, i = kk + 1 + p / nc;
            const double xkc = c == kk ? xd[kk] : ws[c + kk * kWarpLd];
            double v = fma(-ws[i + kk * kWarpLd], xkc, ws[c + i * kWarpLd]);
            if (i == kk + 1) v *= xd[i];
            ws[c + i * kWarpLd] = v;
          }
          __syncwarp();
        }
        double* X = a.inv + a.invoff[s];
        for (int idx = lane; idx < w * w; idx += 32) {
          const int i = idx % w, j = idx / w;
          if (i >= j) X[idx] = i == j ? xd[j] : ws[j + i * kWarpLd];
        }
        // L21 = A21 L11^{-T} by the inverse, in the panels' precision:
        // l_rc = sum_{k <= c} a_rk X_ck, one output per lane and pass, columns
        // in decreasing order, so that a_rc is overwritten only after every
        // output that reads it (its row's higher columns: an earlier pass, or
        // this one, whose reads all precede its writes)
        using ct = T;
        const int rb = r - w, nout = rb * w;
        for (int o0 = 0; o0 < nout; o0 += 32) {
          const int o = o0 + lane;
          const bool ov = o < nout;
          const int c = ov ? w - 1 - o / rb : 0, rr = ov ? o % rb : 0;
          T* Pr = P + w + rr;
          ct acc = ct(0);
          if (ov)
            for (int k = 0; k <= c; ++k)
              acc = fma((ct)ldcg(Pr + (size_t)k * ld), k == c ? (ct)xd[c] : (ct)ws[k + c * kWarpLd], acc);
          __syncwarp();
          if (ov) Pr[(size_t)c * ld] = (T)acc;
        }
        __syncwarp();  // the rows below are written before the update tiles read them
      }
    }
    // update tiles of panel s
    const int32_t* Rs = a.pv.rows + a.pv.rowoff[s];
    for (int ui = a.u_first[s]; ui < a.u_first[s] + a.nu[s]; ++ui) {
      const UTask u = a.ut[ui];
      const bool outside = u.t > hi;
      if (!skip) {
        const int ft = a.pv.fcol[u.t], ldt = a.pv.ld[u.t];
        T* Pt = panel_ptr<T>(a, u.t);
        const int nout = u.rowlen * u.seglen;
        for (int o = lane; o < nout; o += 32) {
          const int i = o % u.rowlen, j = o / u.rowlen;
          const int gi = Rs[u.row0 + i], gj = Rs[u.seg0 + j];
          if (gi < gj) continue;  // the upper part of a target's diagonal block
          const T* ai = P + u.row0 + i;
          const T* bj = P + u.seg0 + j;
          T c0 = T(0), c1 = T(0);
          int kk = 0;
          for (; kk + 1 < w; kk += 2) {
            c0 = fma(ai[(size_t)kk * ld], bj[(size_t)kk * ld], c0);
            c1 = fma(ai[(size_t)(kk + 1) * ld], bj[(size_t)(kk + 1) * ld], c1);
          }
          if (kk < w) c0 = fma(ai[(size_t)kk * ld], bj[(size_t)kk * ld], c0);
          const int p = __ldg(a.relpos + u.rel + i);
          if (p < 0) {  // cannot happen for a consistent plan
            atomicCAS(&a.ctrl[kErr], 0, SPCHOL_DEV_EINTERNAL);
            continue;
          }
          T* dst = Pt + p + (size_t)(gj - ft) * ldt;
          if (outside)
            red_add(dst, -(c0 + c1));
          else
            *dst -= c0 + c1;
        }
      }
      if (outside) {  // publish the warp's atomics, then count the tile down on its target
        __syncwarp();
        if (lane == 0) {
          __threadfence();
          if (atom_add_acqrel(&a.dep_f[u.t], -1) == 1) ring2_push_one(q, true, u.t);
        }
      }
    }
    __syncwarp();  // the next panel reads what this one's tiles wrote into it
  }
}

// MODE: 0 = CUDA-core update tiles (DFMA / FFMA), 1 = TF32 tensor cores (FP32
// panels, split or not), 3 = BF16 tensor cores on split FP64 operands.
// Five CTAs per SM (48 registers a thread; a few live values of the update
// tile's epilogue spill to L1) for the DFMA mode, six (40 registers) for FP32
// panels on FFMA, whose tasks are shortest: more resident CTAs hide each
// other's latencies (measured: FP32 factor -12 %, FP64 -0.8 % for five against
// four).  The TF32 mode runs two CTAs per SM and the BF16-split mode three, as
// their operand tiles' shared memory allows (a BF16-split CTA holds 128 of the
// SM's 512 TMEM columns).  The fan-in mode's CUDA-core kernels run four: the
// gather's staging area takes a quarter of the SM's shared memory.
template <typename T, int MODE, bool FAN>
__global__ void __launch_bounds__(kFactorThreads, MODE == 3 ? 3 : MODE != 0 ? 2 : FAN ? 4 : sizeof(T) == 4 ? 6 : 5)
    factor_kernel(FactorArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ FactorShared sh;
  double* smd = reinterpret_cast<double*>(smem_raw);
  const Ring2 q = rings_of(a);
  __shared__ int pend[3];  // claimed, not yet taken ring slots (thread 0)
  if (threadIdx.x == 0) pend[0] = pend[1] = pend[2] = -1;
  // per-CTA task timing (thread 0 only, in shared memory so that no register
  // stays live across the tasks), flushed once at exit: [0..4] busy ns per task
  // type ([3]: tensor-core update tiles, [4]: subtree tasks), [5..9] counts,
  // [10] wait ns, [11] start of the current task
  __shared__ unsigned long long tprof[12];
  if (threadIdx.x == 0)
    for (int k = 0; k < 12; ++k) tprof[k] = 0ull;
  // TMA staging of the CUDA-core update tiles: one mbarrier per operand buffer
  __shared__ __align__(8) uint64_t upd_mbar[2];
  __shared__ uint32_t upd_phase;
  UpdTma utma{{smem_addr(&upd_mbar[0]), smem_addr(&upd_mbar[1])}, &upd_phase};
  if (a.tmaps && threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(utma.mbar[0]), "r"(1) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(utma.mbar[1]), "r"(1) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    upd_phase = 0u;
  }
  __syncthreads();
  // tensor-core state (FP32 panels with mma_mode 1 / 2): TMEM accumulator + mbarrier
  __shared__ __align__(8) uint64_t tc_mbar;
  __shared__ uint32_t tc_tmem;
  TcState tc{0u, 0u, 0u};
  constexpr bool use_tc = MODE != 0;
  constexpr uint32_t tmem_cols = MODE == 3 ? kOzCols : kTcN;
  if (use_tc) {
    if (threadIdx.x < 32) {
      asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tc_tmem)),
                   "r"(tmem_cols)
                   : "memory");
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (threadIdx.x == 0) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(&tc_mbar)), "r"(1) : "memory");
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    tc.tmem = tc_tmem;
    tc.mbar = smem_addr(&tc_mbar);
  }
  // Thread 0: a normal-priority slot claimed ahead while the ring is deep, so
  // that the claim's round trip overlaps the current task; it joins pend[1] at
  // the next claim (a deep ring fills it long before).  Two adjacent slots are
  // claimed ahead at a time: the next claim reads both in one round trip and
  // the second task (the stash) then runs without a claim of its own.
  int ahead = -1, stash = -1;
  bool deep = false;
  // Subtree task cursor (thread 0): a claimed subtree task is run as a
  // sequence of panel-level steps through the same dispatch as the ring's
  // tasks -- diagonal, panel-solve tiles, update tiles of each panel in
  // postorder -- with counters only for targets outside the subtree.
  __shared__ int cur_task, cur_lo, cur_hi, cur_s, cur_ph, cur_i, cur_skip;
  __shared__ int step_kind, step_s, step_i, step_release, step_last;
  if (threadIdx.x == 0) cur_task = -1;
  const int sub0 = a.pv.ns + a.n_trsm + a.n_u;  // first subtree task id
  for (;;) {
    if (threadIdx.x == 0) {
      const bool timed = a.prof || a.trace;
      if (cur_task < 0) {
        const uint64_t t0 = timed ? global_ns() : 0;
        const bool idle = pend[1] < 0 && pend[2] < 0;
        if (stash >= 0) {  // acquired by the previous claim
          sh.task = stash;
          stash = -1;
          if (deep && idle) ahead = atomicAdd(&q.ctrl[kHead], 2);
        } else {
          if (ahead >= 0) {
            pend[1] = ahead < q.n_lo ? ahead : -1;
            pend[2] = ahead + 1 < q.n_lo ? ahead + 1 : -1;
            ahead = -1;
          }
          int lo_ready;
          sh.task = ring2_claim(q, pend, &lo_ready, a.ntask, &stash);
          deep = lo_ready > 4 * (int)gridDim.x;
          if (sh.task >= 0 && pend[1] < 0 && pend[2] < 0 && stash < 0 && deep) ahead = atomicAdd(&q.ctrl[kHead], 2);
        }
        // The failure word is read after the claim's acquire: a task whose
        // inputs were skipped by tasks that saw a failed pivot (their release
        // precedes this claim) then sees it too and skips as well.  Read
        // before the claim, a diagonal task could factor a panel missing
        // skipped updates and report a pivot failure that is not there.
        sh.skip = (ld_relaxed(&a.ctrl[kInfo]) != INT_MAX);
        if (timed) {
          const uint64_t t1 = global_ns();
          tprof[10] += t1 - t0;
          tprof[11] = t1;
        }
        if (sh.task >= sub0 && (!FAN || sh.task < a.gat0)) {
          const int k = sh.task - sub0;
          cur_task = sh.task;
          cur_lo = a.sub_lo[k];
          cur_hi = a.sub_hi[k];
          cur_s = cur_lo;
          cur_ph = 0;
          cur_i = 0;
          cur_skip = sh.skip;
        }
      }
      if (cur_task >= 0) {  // the next step of the subtree, then advance the cursor
        const int s = cur_s;
        step_kind = cur_ph;
        step_s = s;
        step_i = cur_i;
        step_release = cur_ph == 2 ? (a.ut[a.u_first[s] + cur_i].t > cur_hi) : 0;
        sh.skip = cur_skip;
        sh.task = cur_task;
        int ph = cur_ph, i = cur_i + 1;
        if (ph == 0) {
          ph = 1;
          i = 0;
        }
        if (ph == 1 && i >= a.ntrsm[s]) {
          ph = 2;
          i = 0;
        }
        step_last = 0;
        if (ph == 2 && i >= a.nu[s]) {
          if (s < cur_hi) {
            cur_s = s + 1;
            ph = 0;
            i = 0;
          } else {
            step_last = 1;
          }
        }
        cur_ph = ph;
        cur_i = i;
      } else if (sh.task >= 0) {  // a task of the rings
        const int task = sh.task;
        step_release = 1;
        step_last = 1;
        if (task < a.pv.ns) {
          step_kind = 0;
          step_s = task;
          step_i = 0;
        } else if (task < a.pv.ns + a.n_trsm) {
          const int kt = task - a.pv.ns;
          step_kind = 1;
          step_s = a.trsm_sn[kt];
          step_i = kt - a.trsm_first[step_s];
        } else if (FAN && task >= a.gat0) {
          step_kind = 4;  // a gather task (fan-in mode)
          step_s = -1;
          step_i = task - a.gat0;
        } else {
          step_kind = 3;  // an update tile by its global index
          step_s = -1;
          step_i = task - a.pv.ns - a.n_trsm;
        }
      }
    }
    __syncthreads();
    const int task = sh.task;
    if (task < 0) break;
    const bool skip = sh.skip != 0;
    const int kind = step_kind, s = step_s, si = step_i;
    const bool release = step_release != 0;
    int type;
    if (FAN && kind == 4) {
      // fan-in mode: a gather task adds the buffered updates of one row piece
      // of a panel, then counts down the task that owns those rows
      type = 0;
      const int pc = a.gat_pc[si], o = a.pc_owner[pc];
      const int t = o < a.pv.ns ? o : a.trsm_sn[o - a.pv.ns];
      const int w = a.pv.fcol[t + 1] - a.pv.fcol[t];
      int p0, p1;
      if (o < a.pv.ns) {
        p0 = (pc - a.fan_task[t]) * kFanPieceRows;
        p1 = min(w, p0 + kFanPieceRows);
      } else {
        const int tr = a.trsm_rows_of[t], r0 = w + (o - a.pv.ns - a.trsm_first[t]) * tr;
        p0 = r0 + (pc - a.fan_task[o]) * kFanPieceRows;
        p1 = min(min(a.pv.nrows[t], r0 + tr), p0 + kFanPieceRows);
      }
      if (!skip) fanin_gather<T>(a, t, pc, p0, p1 - p0, smem_raw);
      publish_cta_writes();
      if (threadIdx.x == 0) {
        if (o < a.pv.ns) {
          if (atom_add_acqrel(&a.gdiag[t], -1) == 1) ring2_push_one(rings_of(a), true, t);
        } else if (atom_add_acqrel(&a.tdep[o - a.pv.ns], -1) == 1) {
          ring2_push_one(rings_of(a), true, o);
        }
      }
    } else if (kind == 0) {
      type = 0;
      task_potrf<T, FAN>(a, s, smd, sh, skip, release);
    } else if (kind == 1) {
      type = 1;
      task_trsm<T, MODE>(a, s, si, smd, sh, skip, release);
    } else {
      type = 2;
      const int ui = kind == 2 ? a.u_first[s] + si : si;
      const UTask u = a.ut[ui];
      const long long fo = FAN ? (long long)a.fan_off[ui] : -1ll;  // fan-in: the tile's buffer
      if constexpr (MODE == 3) {
        if (a.pv.fcol[u.s + 1] - a.pv.fcol[u.s] >= a.tc_min_width) {
          type = 3;
          task_update_oz<FAN>(a, u, smem_raw, sh, skip, tc, fo, release);
        } else {
          task_update<T, FAN>(a, u, smem_raw, sh, skip, ui & 7, utma, fo, release);
        }
      } else if constexpr (MODE == 1) {
        task_update_tc<FAN>(a, u, smem_raw, sh, skip, tc, fo, release);
      } else {
        task_update<T, FAN>(a, u, smem_raw, sh, skip, ui & 7, utma, fo, release);
      }
      // deterministic order: the next tile into the same target may start
      // (the tile's scatter-adds were published before its own release)
      if (a.u_next && release && threadIdx.x == 0) {
        const int nx = a.u_next[ui];
        if (nx >= 0 && atom_add_acqrel(&a.u_dep[nx], -1) == 1) {
          const int sx = a.ut[nx].s;
          ring2_push_one(rings_of(a), nx - a.u_first[sx] < a.nu_hi[sx], a.pv.ns + a.n_trsm + nx);
        }
      }
    }
    if (threadIdx.x == 0) {
      const bool in_sub = cur_task >= 0;
      if (in_sub) {
        type = 4;
        // after a failed pivot the rest of the subtree skips its arithmetic
        if (kind == 0 && ld_relaxed(&a.ctrl[kInfo]) != INT_MAX) cur_skip = 1;
      }
      if (step_last) {
        atomicAdd(&a.ctrl[kDone], 1);
        if (a.trace) {
          a.trace[2 * (size_t)task] = tprof[11];
          a.trace[2 * (size_t)task + 1] = global_ns();
        }
        if (a.prof) {
          tprof[type] += global_ns() - tprof[11];
          tprof[5 + type] += 1;
        }
        if (in_sub) cur_task = -1;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0 && a.prof) {
    for (int k = 0; k < 3; ++k) {
      atomicAdd(&a.prof[k], tprof[k] + (k == 2 ? tprof[3] : 0ull));
      atomicAdd(&a.prof[4 + k], tprof[5 + k] + (k == 2 ? tprof[8] : 0ull));
    }
    atomicAdd(&a.prof[3], tprof[10]);
    atomicAdd(&a.prof[7], tprof[3]);   // tensor-core share of the update tiles
    atomicAdd(&a.prof[8], tprof[4]);   // subtree tasks
    atomicAdd(&a.prof[9], tprof[9]);
  }
  if (use_tc) {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (threadIdx.x < 32)
      asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tc.tmem), "r"(tmem_cols) : "memory");
  }
}

// The warp-level subtree tasks, launched before the task loop's kernel (on the
// same stream, after the ring reset): kWarpExec warps per CTA, each taking
// the next subtree from a counter until none is left.  The tiles they count
// down push ready tasks into the rings, which the task loop's kernel then
// finds there; every subtree adds one to the completed-task count.
template <typename T>
__global__ void __launch_bounds__(32 * kWarpExec) warp_subtree_kernel(FactorArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  double* ws = reinterpret_cast<double*>(smem_raw) + warp * kWarpSmem;
  const int sub0 = a.pv.ns + a.n_trsm + a.n_u;  // first subtree task id
  for (;;) {
    int e = 0;
    if (lane == 0) e = atomicAdd(&a.ctrl[kWarpNext], 1);
    e = __shfl_sync(0xffffffffu, e, 0);
    if (e >= a.n_wsub) break;
    const int k = a.wsub[e];
    const unsigned long long t0 = a.trace && lane == 0 ? global_ns() : 0ull;
    warp_subtree<T>(a, k, ws);
    if (lane == 0) {
      atomicAdd(&a.ctrl[kDone], 1);
      if (a.trace) {
        a.trace[2 * (size_t)(sub0 + k)] = t0;
        a.trace[2 * (size_t)(sub0 + k) + 1] = global_ns();
      }
    }
  }
}

template <typename T>
__global__ void assemble_kernel(const double* __restrict__ values, const int64_t* __restrict__ dest,
                                int64_t nnz, T* __restrict__ pool) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x)
    pool[dest[e]] = (T)values[e];
}

}  // namespace

size_t warp_subtree_smem_bytes() { return (size_t)kWarpExec * kWarpSmem * sizeof(double); }

static const void* warp_subtree_fn(bool fp32) {
  return fp32 ? (const void*)warp_subtree_kernel<float> : (const void*)warp_subtree_kernel<double>;
}

cudaError_t warp_subtree_configure(bool fp32, int* blocks_per_sm) {
  const size_t smem = warp_subtree_smem_bytes();
  cudaError_t e = ensure_smem_limit(warp_subtree_fn(fp32), smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, warp_subtree_fn(fp32), 32 * kWarpExec, smem);
}

cudaError_t launch_warp_subtrees(bool fp32, const FactorArgs& a, int grid, cudaStream_t st) {
  if (a.n_wsub == 0) return cudaSuccess;
  void* args[] = {const_cast<FactorArgs*>(&a)};
  return cudaLaunchKernel(warp_subtree_fn(fp32), dim3(grid), dim3(32 * kWarpExec), args, warp_subtree_smem_bytes(),
                          st);
}

size_t factor_smem_bytes(int max_w, int mma_mode) {
  // POTRF: the block, 1 / l_jj, two scaled columns and the 8-bit pair table;
  // TRSM: L11 with 64-row columns and 1 / l_cc.
  size_t tri = ((size_t)max_w * max_w + 3 * (size_t)max_w) * sizeof(double) +
               (((size_t)max_w * (max_w - 1) / 2 + 15) & ~size_t(15));
  // (+ 1: the W rows of W panels restage L11 with leading dimension 65)
  if (max_w <= kTrsmMaxW) tri = std::max(tri, (size_t)(kTrsmMaxW + 2) * max_w * sizeof(double));
  if (mma_mode == 3) {
    const size_t kpad = ((size_t)max_w + 15) & ~size_t(15);
    const size_t oz = (size_t)kSlices * (kOzRows + kOzN) * kpad * 2 + (3 * kOzRows + 2 * kOzN) * sizeof(int) + 1024;
    if (oz > tri) tri = oz;
  } else if (mma_mode != 0) {
    const size_t kpad = ((size_t)max_w + 7) & ~size_t(7);
    const size_t tcb = 2 * (kTcM + kTcN) * kpad * 4 + (2 * kTcM + kTcN) * sizeof(int) + 1024;
    if (tcb > tri) tri = tcb;
  }
  // update tiles: two FP64 chunk buffers, or four FP32 ones (A and B each),
  // then the row positions, rows and columns
  const size_t bufs = std::max((size_t)2 * 2 * kUpdKC * Stage<double>::kStr * sizeof(double),
                               (size_t)4 * 2 * kUpdKC * Stage<float>::kStr * sizeof(float));
  size_t upd = bufs + 128 + (size_t)(2 * kUpdTileM + kUpdTileN) * sizeof(int);
  return tri > upd ? tri : upd;
}

size_t fanin_smem_bytes(int max_w, bool fp32, int* cap) {
  const size_t es = fp32 ? sizeof(float) : sizeof(double);
  const int per_col = fp32 ? fan_pieces<float>(kFanPieceRows) : fan_pieces<double>(kFanPieceRows);
  const int c = std::max(2048, per_col * max_w);  // 32 KB of pieces, and never less than one tile
  if (cap) *cap = c;
  return 16 + kFanMetaBytes + kFanVcap * sizeof(int16_t) + (size_t)c * 16 + (size_t)kFanPieceRows * max_w * es;
}

// The fan-in mode has kernels of its own, so that the other modes' update
// tiles and dispatch carry none of its code.
template <bool FAN>
static const void* factor_fn_of(bool fp32, int mma_mode) {
  if (fp32)
    return mma_mode == 0 ? (const void*)factor_kernel<float, 0, FAN> : (const void*)factor_kernel<float, 1, FAN>;
  return mma_mode == 3 ? (const void*)factor_kernel<double, 3, FAN> : (const void*)factor_kernel<double, 0, FAN>;
}

static const void* factor_fn(bool fp32, int mma_mode, bool fan) {
  return fan ? factor_fn_of<true>(fp32, mma_mode) : factor_fn_of<false>(fp32, mma_mode);
}

cudaError_t factor_configure(bool fp32, int mma_mode, bool fan, size_t smem, int* blocks_per_sm) {
  const void* fn = factor_fn(fp32, mma_mode, fan);
  cudaError_t e = ensure_smem_limit(fn, smem);
  if (e != cudaSuccess) return e;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, fn, kFactorThreads, smem);
  if (e != cudaSuccess || mma_mode == 0) return e;
  // The runtime's occupancy query reports one block per SM for the kernels
  // that allocate TMEM, while their registers and shared memory allow more
  // (the profiler's launch statistics agree).  Count those limits directly,
  // capped by the TMEM columns a CTA holds (512 per SM; the BF16-split mode's
  // shared-memory request, over a third of the SM, also keeps a third CTA out).
  cudaFuncAttributes fa{};
  int dev = 0, regs_sm = 0, smem_sm = 0;
  if ((e = cudaFuncGetAttributes(&fa, fn)) != cudaSuccess || (e = cudaGetDevice(&dev)) != cudaSuccess ||
      (e = cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev)) != cudaSuccess ||
      (e = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev)) != cudaSuccess)
    return e;
  const int regs_cta = ((fa.numRegs + 7) / 8) * 8 * kFactorThreads;
  const size_t smem_cta = smem + fa.sharedSizeBytes + 1024;  // + the driver's per-block reserve
  const int by_regs = regs_cta > 0 ? regs_sm / regs_cta : 0;
  const int by_smem = (int)((size_t)smem_sm / smem_cta);
  const int by_tmem = 512 / (mma_mode == 3 ? kOzCols : kTcN);
  const int direct = std::min(by_tmem, std::min(by_regs, by_smem));
  if (direct > *blocks_per_sm) *blocks_per_sm = direct;
  return cudaSuccess;
}

cudaError_t launch_relpos(const UTask* ut, int n_u, const int32_t* rows, const int64_t* rowoff,
                          const int32_t* nrows, int32_t* relpos, cudaStream_t st) {
  if (n_u <= 0) return cudaSuccess;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int grid = std::max(1, std::min(n_u, 32 * std::max(sms, 1)));
  relpos_kernel<<<grid, 64, 0, st>>>(ut, n_u, rows, rowoff, nrows, relpos);
  return cudaGetLastError();
}

cudaError_t launch_assemble(bool fp32, const double* values, const int64_t* dest, int64_t nnz, void* pool,
                            cudaStream_t st) {
  if (nnz <= 0) return cudaSuccess;
  int grid = (int)((nnz + 255) / 256);
  if (grid > 152 * 16) grid = 152 * 16;
  if (fp32)
    assemble_kernel<float><<<grid, 256, 0, st>>>(values, dest, nnz, (float*)pool);
  else
    assemble_kernel<double><<<grid, 256, 0, st>>>(values, dest, nnz, (double*)pool);
  return cudaGetLastError();
}

__global__ void fanrec_kernel(const FanEnt* __restrict__ ent, int64_t n, const UTask* __restrict__ ut,
                              const int64_t* __restrict__ fan_off, const int64_t* __restrict__ rowoff,
                              FanRec* __restrict__ rec) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    const FanEnt fe = ent[k];
    const UTask u = ut[fe.u];
    FanRec r;
    r.fo = fan_off[fe.u] + fe.i0;
    r.rp = u.rel + fe.i0;
    r.rs = rowoff[u.s] + u.seg0;
    r.rowlen = u.rowlen;
    r.ni = (int16_t)(fe.i1 - fe.i0);
    r.seglen = (int16_t)u.seglen;
    rec[k] = r;
  }
}

cudaError_t launch_fanrec(const FanEnt* ent, int64_t n, const UTask* ut, const int64_t* fan_off,
                          const int64_t* rowoff, FanRec* rec, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const int grid = (int)std::min<int64_t>((n + 255) / 256, 152 * 16);
  fanrec_kernel<<<grid, 256, 0, st>>>(ent, n, ut, fan_off, rowoff, rec);
  return cudaGetLastError();
}

cudaError_t launch_factor(bool fp32, const FactorArgs& a, int grid, size_t smem, cudaStream_t st) {
  void* args[] = {const_cast<FactorArgs*>(&a)};
  return cudaLaunchKernel(factor_fn(fp32, a.mma_mode, a.fan_ptr != nullptr), dim3(grid), dim3(kFactorThreads), args,
                          smem, st);
}

}  // namespace spchol
