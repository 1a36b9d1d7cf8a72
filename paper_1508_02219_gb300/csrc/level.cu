// Steps 2-4 of VBARMS for one level on the GPU (Section 3, Eq. 4-8, and the
// two-sweep implementation of Section 3.1).
//
//   A5  Step 2: row max-abs scaling, then column max-abs scaling of the row
//       scaled matrix (column maxima by atomicMax on the IEEE bit patterns of
//       non-negative doubles, which order like the values)
//   A6  Step 3: weights w(Y) = ||A_YY||_F / sum_Z ||A_YZ||_F in a fixed order
//       (one thread per supernode, no contraction), then the greedy independent
//       set in (w desc, index asc) order as the lexicographically first MIS,
//       decided in deterministic rounds; P_I puts D ascending, then C ascending
//   A7  gather of D (pivot blocks), F, E, C and batched GEPP of the pivot
//       blocks (one thread per block, the oracle's operation order)
//   A8  W = L^{-1} P F, A9 G = E U^{-1}, each block tested against the drop
//       rule and trimmed to lfil per block row
//   A10 S = C - G W as a row-wise block SpGEMM: hashed symbolic union of the
//       patterns of C and of the W rows reached from G, then the numeric
//       accumulation in the order C, then G blocks ascending, then k
//
// FP64 kernels evaluate every product and sum as separate IEEE operations in
// the oracle's order (the library is built without FMA contraction), so FP64
// results match the CPU oracle bit for bit.  FP32 kernels use fused
// multiply-adds.
#include <algorithm>
#include <map>
#include <mutex>

#include "internal.h"
#include "blockops.cuh"
#include "level.cuh"
#include "vbsr_ops.cuh"

namespace vb {
namespace {

constexpr int LW = 8;           // warps per block
constexpr int PAT_CAP = 1024;   // per-warp shared hash capacity
constexpr int PAT_LIMIT = 640;


// ---- A5: Step 2 scaling ----------------------------------------------------
// |x| maxima: exact in any precision and any order.  FP64 values are
// compared by their bit patterns (integer maxima, no FP64 pipe); FP32 ones by
// fmaxf.
__device__ __forceinline__ double absmax_acc(double m, double x) {
  const long long a = __double_as_longlong(m), b = __double_as_longlong(x) & 0x7fffffffffffffffLL;
  return __longlong_as_double(a > b ? a : b);
}
__device__ __forceinline__ float absmax_acc(float m, float x) { return fmaxf(m, fabsf(x)); }

// Row maxima, one warp per block row: lane (a, g) takes scalar row a of the
// blocks g, g + G, ... of the block row (G = 32 / m groups), then the groups
// combine by shuffles.  Rows of more than 16 scalars use lanes over rows.
template <typename TA>
__global__ void k_rowmax(VBView<TA> A, double* __restrict__ r) {
  const int lane = threadIdx.x & 31;
  const int64_t wpb = blockDim.x >> 5;
  for (int64_t I = blockIdx.x * wpb + (threadIdx.x >> 5); I < A.nbr; I += (int64_t)gridDim.x * wpb) {
    const int m = A.rsz[I];
    const int64_t b0 = A.bptr[I], b1 = A.bptr[I + 1];
    if (m <= 16) {
      const int G = 32 / m, a = lane % m, g = lane / m;
      TA mx = (TA)0;
      if (g < G)
        for (int64_t b = b0 + g; b < b1; b += G) {
          const int nc = A.csz[A.bcol[b]];
          const TA* v = A.val + A.voff[b] + (int64_t)a * nc;
          for (int j = 0; j < nc; ++j) mx = absmax_acc(mx, v[j]);
        }
      for (int k = 1; k < G; ++k) {
        const TA o = __shfl_sync(0xffffffffu, mx, (a + k * m) & 31);
        if (lane < m) mx = absmax_acc(mx, o);
      }
      if (lane < m) {
        const double d = (double)mx;
        r[A.roff[I] + a] = d > 0.0 ? __ddiv_rn(1.0, d) : 1.0;
      }
    } else {
      for (int a = lane; a < m; a += 32) {
        TA mx = (TA)0;
        for (int64_t b = b0; b < b1; ++b) {
          const int nc = A.csz[A.bcol[b]];
          const TA* v = A.val + A.voff[b] + (int64_t)a * nc;
          for (int j = 0; j < nc; ++j) mx = absmax_acc(mx, v[j]);
        }
        const double d = (double)mx;
        r[A.roff[I] + a] = d > 0.0 ? __ddiv_rn(1.0, d) : 1.0;
      }
    }
  }
}

// Products r_a * a_aj in the value type's arithmetic: FP64 (exact IEEE
// products, the oracle's) for FP64 values, FP32 for the FP32 levels of the
// mixed factor.
__device__ __forceinline__ double rprod(double r, double v) { return __dmul_rn(r, v); }
__device__ __forceinline__ float rprod(double r, float v) { return __fmul_rn((float)r, v); }

// Column maxima of the row-scaled matrix, one warp per block row: lane
// (g, j) takes column j (then j + 8, ...) of the blocks g, g + 4, ...; one
// atomicMax per block column on the bit pattern of the non-negative maximum.
template <typename TA>
__global__ void k_colmax(VBView<TA> A, const double* __restrict__ r, unsigned long long* __restrict__ cmax) {
  const int lane = threadIdx.x & 31;
  const int64_t wpb = blockDim.x >> 5;
  const int g = lane >> 3, j0 = lane & 7;
  for (int64_t I = blockIdx.x * wpb + (threadIdx.x >> 5); I < A.nbr; I += (int64_t)gridDim.x * wpb) {
    const int m = A.rsz[I];
    const int64_t r0 = A.roff[I];
    for (int64_t b = A.bptr[I] + g; b < A.bptr[I + 1]; b += 4) {
      const int J = A.bcol[b];
      const int nc = A.csz[J];
      const int64_t c0 = A.coff[J];
      const TA* v = A.val + A.voff[b];
      for (int j = j0; j < nc; j += 8) {
        TA mx = (TA)0;
        for (int a = 0; a < m; ++a) mx = absmax_acc(mx, rprod(r[r0 + a], v[a * nc + j]));
        atomicMax(&cmax[c0 + j], (unsigned long long)__double_as_longlong((double)mx));
      }
    }
  }
}

__global__ void k_colinv(int64_t n, const unsigned long long* __restrict__ cmax, double* __restrict__ c) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
    const double x = __longlong_as_double((long long)cmax[j]);
    c[j] = x > 0.0 ? __ddiv_rn(1.0, x) : 1.0;
  }
}

__device__ __forceinline__ double rcprod(double r, double v, double c) { return __dmul_rn(__dmul_rn(r, v), c); }
__device__ __forceinline__ float rcprod(double r, float v, double c) {
  return __fmul_rn(__fmul_rn((float)r, v), (float)c);
}

// a_ij <- r_i a_ij c_j, one warp per block row, lanes (g, j) as in k_colmax.
template <typename TA>
__global__ void k_apply_scale(VBView<TA> A, const double* __restrict__ r, const double* __restrict__ c) {
  const int lane = threadIdx.x & 31;
  const int64_t wpb = blockDim.x >> 5;
  const int g = lane >> 3, j0 = lane & 7;
  for (int64_t I = blockIdx.x * wpb + (threadIdx.x >> 5); I < A.nbr; I += (int64_t)gridDim.x * wpb) {
    const int m = A.rsz[I];
    const int64_t r0 = A.roff[I];
    for (int64_t b = A.bptr[I] + g; b < A.bptr[I + 1]; b += 4) {
      const int J = A.bcol[b];
      const int nc = A.csz[J];
      const int64_t c0 = A.coff[J];
      TA* v = A.val + A.voff[b];
      for (int j = j0; j < nc; j += 8) {
        const double cj = c[c0 + j];
        for (int a = 0; a < m; ++a) v[a * nc + j] = (TA)rcprod(r[r0 + a], v[a * nc + j], cj);
      }
    }
  }
}

// ---- A6: Step 3 ----------------------------------------------------------
// Weights, one warp per block row: lane k forms ||A_Yb||_F of the row's
// blocks k, k + 32, ... (row-major sum of squares, the oracle's order for
// FP64 values), then lane 0 adds the norms in block order.
__device__ __forceinline__ double sq_acc(double s, double x) { return __dadd_rn(s, __dmul_rn(x, x)); }
__device__ __forceinline__ float sq_acc(float s, float x) { return __fmaf_rn(x, x, s); }
__device__ __forceinline__ double sqrt_rn(double x) { return __dsqrt_rn(x); }
__device__ __forceinline__ float sqrt_rn(float x) { return __fsqrt_rn(x); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }

template <typename TA>
__global__ void k_weights(VBView<TA> A, double* __restrict__ w) {
  const int lane = threadIdx.x & 31;
  const int64_t wpb = blockDim.x >> 5;
  for (int64_t Y = blockIdx.x * wpb + (threadIdx.x >> 5); Y < A.nbr; Y += (int64_t)gridDim.x * wpb) {
    const int m = A.rsz[Y];
    const int64_t b0 = A.bptr[Y], b1 = A.bptr[Y + 1];
    TA dsum = (TA)0, diag = (TA)0;
    for (int64_t c0 = b0; c0 < b1; c0 += 32) {
      const int64_t b = c0 + lane;
      TA f = (TA)0;
      bool isdiag = false;
      if (b < b1) {
        const int J = A.bcol[b];
        const int nc = A.csz[J];
        const TA* v = A.val + A.voff[b];
        TA s = (TA)0;
        for (int e = 0; e < m * nc; ++e) s = sq_acc(s, v[e]);
        f = sqrt_rn(s);
        isdiag = J == Y;
      }
      const int cnt = b1 - c0 < 32 ? (int)(b1 - c0) : 32;
      for (int k = 0; k < cnt; ++k) {
        const TA fk = __shfl_sync(0xffffffffu, f, k);
        dsum = add_rn(dsum, fk);
      }
      const unsigned dm = __ballot_sync(0xffffffffu, isdiag);
      if (dm) diag = __shfl_sync(0xffffffffu, f, __ffs(dm) - 1);
    }
    if (lane == 0) {
      const double ds = (double)dsum, dg = (double)diag;
      w[Y] = ds > 0.0 ? __ddiv_rn(dg, ds) : 0.0;
    }
  }
}

__global__ void k_tcount(int64_t nbr, const int64_t* __restrict__ bptr, const int32_t* __restrict__ bcol,
                         int32_t* __restrict__ tcnt) {
  const int lane = threadIdx.x & 31;
  const int64_t wpb = blockDim.x >> 5;
  for (int64_t I = blockIdx.x * wpb + (threadIdx.x >> 5); I < nbr; I += (int64_t)gridDim.x * wpb)
    for (int64_t b = bptr[I] + lane; b < bptr[I + 1]; b += 32) atomicAdd(&tcnt[bcol[b]], 1);
}

__global__ void k_tfill(int64_t nbr, const int64_t* __restrict__ bptr, const int32_t* __restrict__ bcol,
                        const int64_t* __restrict__ tptr, int32_t* __restrict__ tfill, int32_t* __restrict__ trow) {
  const int lane = threadIdx.x & 31;
  const int64_t wpb = blockDim.x >> 5;
  for (int64_t I = blockIdx.x * wpb + (threadIdx.x >> 5); I < nbr; I += (int64_t)gridDim.x * wpb)
    for (int64_t b = bptr[I] + lane; b < bptr[I + 1]; b += 32) {
      const int32_t J = bcol[b];
      trow[tptr[J] + atomicAdd(&tfill[J], 1)] = (int32_t)I;
    }
}

__device__ __forceinline__ bool better(const double* w, int64_t u, int64_t v) {
  return w[u] > w[v] || (w[u] == w[v] && u < v);
}

// state: 0 undecided, 1 in D, 2 out (in the current MIS round), 3 out.
// fixed (may be NULL): rows that never enter the set (interface rows of the
// Section 5 Schur-complement preconditioner); they are out from the start.
__global__ void k_is_init(int64_t p, const int64_t* __restrict__ bptr, const int32_t* __restrict__ bcol,
                          const int64_t* __restrict__ tptr, const int32_t* __restrict__ trow,
                          const double* __restrict__ w, double ddtol, const int32_t* __restrict__ fixed,
                          int32_t* __restrict__ pending, int32_t* __restrict__ state,
                          unsigned long long* remaining) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < p; v += (int64_t)gridDim.x * blockDim.x) {
    int cnt = 0;
    for (int64_t b = bptr[v]; b < bptr[v + 1]; ++b) {
      const int64_t u = bcol[b];
      if (u != v && better(w, u, v)) ++cnt;
    }
    for (int64_t t = tptr[v]; t < tptr[v + 1]; ++t) {
      const int64_t u = trow[t];
      if (u != v && better(w, u, v)) ++cnt;
    }
    pending[v] = cnt;
    if (w[v] < ddtol || (fixed && fixed[v])) {  // too weakly dominant or fixed: never a pivot (forced into C)
      state[v] = 2;
      atomicAdd(remaining, (unsigned long long)-1LL);
    } else {
      state[v] = 0;
    }
  }
}

__global__ void k_is_round_a(int64_t p, const int64_t* __restrict__ bptr, const int32_t* __restrict__ bcol,
                             const int64_t* __restrict__ tptr, const int32_t* __restrict__ trow,
                             const int32_t* __restrict__ pending, int32_t* __restrict__ state,
                             unsigned long long* remaining) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < p; v += (int64_t)gridDim.x * blockDim.x) {
    if (state[v] != 0 || pending[v] != 0) continue;
    state[v] = 1;
    long long dec = 1;
    for (int64_t b = bptr[v]; b < bptr[v + 1]; ++b) {
      const int32_t u = bcol[b];
      if (u != v && atomicCAS(&state[u], 0, 2) == 0) ++dec;
    }
    for (int64_t t = tptr[v]; t < tptr[v + 1]; ++t) {
      const int32_t u = trow[t];
      if (u != v && atomicCAS(&state[u], 0, 2) == 0) ++dec;
    }
    atomicAdd(remaining, (unsigned long long)(-dec));
  }
}

__global__ void k_is_round_b(int64_t p, const int64_t* __restrict__ bptr, const int32_t* __restrict__ bcol,
                             const int64_t* __restrict__ tptr, const int32_t* __restrict__ trow,
                             const double* __restrict__ w, int32_t* __restrict__ pending,
                             int32_t* __restrict__ state) {
  for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < p; u += (int64_t)gridDim.x * blockDim.x) {
    if (state[u] != 2) continue;
    state[u] = 3;
    for (int64_t b = bptr[u]; b < bptr[u + 1]; ++b) {
      const int64_t x = bcol[b];
      if (x != u && better(w, u, x)) atomicSub(&pending[x], 1);
    }
    for (int64_t t = tptr[u]; t < tptr[u + 1]; ++t) {
      const int64_t x = trow[t];
      if (x != u && better(w, u, x)) atomicSub(&pending[x], 1);
    }
  }
}

__global__ void k_is_flags(int64_t p, const int32_t* __restrict__ state, int32_t* __restrict__ isD,
                           int32_t* __restrict__ isC) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < p; v += (int64_t)gridDim.x * blockDim.x) {
    const bool d = state[v] == 1;
    isD[v] = d ? 1 : 0;
    isC[v] = d ? 0 : 1;
  }
}

__global__ void k_is_positions(int64_t p, const int32_t* __restrict__ isD, const int64_t* __restrict__ scanD,
                               const int64_t* __restrict__ scanC, int64_t nD, int32_t* __restrict__ newpos,
                               int32_t* __restrict__ pI) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < p; v += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = isD[v] ? scanD[v] : nD + scanC[v];
    newpos[v] = (int32_t)k;
    pI[k] = (int32_t)v;
  }
}

__global__ void k_perm_sizes(int64_t p, const int32_t* __restrict__ pI, const int32_t* __restrict__ rsz,
                             int32_t* __restrict__ out) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < p; k += (int64_t)gridDim.x * blockDim.x)
    out[k] = rsz[pI[k]];
}

// ---- A7: gather of D, F, E, C -----------------------------------------------
// PASS 0: counts per part row; PASS 1: bcol of every part and the source block
// of every destination block.
template <int PASS>
__global__ void k_gather(int64_t p, int64_t nD, const int64_t* __restrict__ bptr, const int32_t* __restrict__ bcol,
                         const int32_t* __restrict__ newpos, int64_t* __restrict__ cntF, int64_t* __restrict__ cntE,
                         int64_t* __restrict__ cntC, const int64_t* __restrict__ pF, const int64_t* __restrict__ pE,
                         const int64_t* __restrict__ pC, int32_t* __restrict__ colF, int32_t* __restrict__ colE,
                         int32_t* __restrict__ colC, int64_t* __restrict__ srcD, int64_t* __restrict__ srcF,
                         int64_t* __restrict__ srcE, int64_t* __restrict__ srcC, int* st) {
  const int lane = threadIdx.x & 31;
  const int64_t wpb = blockDim.x >> 5;
  for (int64_t Y = blockIdx.x * wpb + (threadIdx.x >> 5); Y < p; Y += (int64_t)gridDim.x * wpb) {
    const int64_t k = newpos[Y];
    const bool rowD = k < nD;
    int64_t baseX = 0, baseY = 0;  // running destinations: rowD: F ; else: E (X) and C (Y)
    if (PASS == 1) {
      if (rowD)
        baseX = pF[k];
      else {
        baseX = pE[k - nD];
        baseY = pC[k - nD];
      }
    }
    int cX = 0, cY = 0, diag = 0;
    for (int64_t b0 = bptr[Y]; b0 < bptr[Y + 1]; b0 += 32) {
      const int64_t b = b0 + lane;
      const bool valid = b < bptr[Y + 1];
      int32_t Z = valid ? bcol[b] : -1;
      const int64_t nz = valid ? newpos[Z] : -1;
      const bool colD = valid && nz < nD;
      const bool isdiag = valid && Z == Y;
      bool toX, toY;
      if (rowD) {
        toX = valid && !colD;  // F
        toY = false;
        if (valid && colD && !isdiag) dev_fail(st, DEV_INTERNAL);  // D supernodes are uncoupled
        if (isdiag && PASS == 1) srcD[k] = b;
        diag += isdiag ? 1 : 0;
      } else {
        toX = colD;             // E
        toY = valid && !colD;   // C
      }
      const unsigned mX = __ballot_sync(0xffffffffu, toX), mY = __ballot_sync(0xffffffffu, toY);
      if (PASS == 1) {
        const unsigned lt = (1u << lane) - 1u;
        if (toX) {
          const int64_t d = baseX + __popc(mX & lt);
          if (rowD) {
            colF[d] = (int32_t)(nz - nD);
            srcF[d] = b;
          } else {
            colE[d] = (int32_t)nz;
            srcE[d] = b;
          }
        }
        if (toY) {
          const int64_t d = baseY + __popc(mY & lt);
          colC[d] = (int32_t)(nz - nD);
          srcC[d] = b;
        }
        baseX += __popc(mX);
        baseY += __popc(mY);
      }
      cX += __popc(mX);
      cY += __popc(mY);
    }
    diag = warp_sum_i(diag);
    if (PASS == 0 && lane == 0) {
      if (rowD) {
        cntF[k] = cX;
        if (diag != 1) dev_fail(st, DEV_ESINGULAR);  // a missing pivot block is zero
      } else {
        cntE[k - nD] = cX;
        cntC[k - nD] = cY;
      }
    }
  }
}

template <typename TS, typename TD>
__global__ void k_copy_blocks(int64_t nblocks, const int64_t* __restrict__ src, const int64_t* __restrict__ svoff,
                              const TS* __restrict__ sval, const int64_t* __restrict__ dvoff, TD* __restrict__ dval) {
  const int lane = threadIdx.x & 31;
  const int64_t wpb = blockDim.x >> 5;
  for (int64_t d = blockIdx.x * wpb + (threadIdx.x >> 5); d < nblocks; d += (int64_t)gridDim.x * wpb) {
    const int64_t b = src[d];
    const int64_t n = svoff[b + 1] - svoff[b];
    for (int64_t e = lane; e < n; e += 32) dval[dvoff[d] + e] = (TD)sval[svoff[b] + e];
  }
}

// ---- A7: batched GEPP ------------------------------------------------------
constexpr int KAPPA_MAX = 64;  // largest block given a condition estimate

// One pivot block, one thread: GEPP, then (mixed factor) the 1-norm
// condition estimate from the explicit inverse columns, the FP64 tag and the
// FP32 copy.
__device__ void gepp_item_thread(int64_t y, const int32_t* __restrict__ sz, const int64_t* __restrict__ roff,
                                 const int64_t* __restrict__ voff, double* __restrict__ val,
                                 int32_t* __restrict__ piv, int mixed, double cond_thr, int32_t* __restrict__ ptag,
                                 float* __restrict__ val32, int* st) {
  const int m = sz[y];
  double* a = val + voff[y];
  int32_t* pv = piv + roff[y];
  double norm1 = 0.0;
  if (mixed) {
    for (int j = 0; j < m; ++j) {
      double s = 0.0;
      for (int i = 0; i < m; ++i) s += fabs(a[i * m + j]);
      norm1 = fmax(norm1, s);
    }
  }
  for (int k = 0; k < m; ++k) {
    int p = k;
    double best = fabs(a[k * m + k]);
    for (int i = k + 1; i < m; ++i) {
      const double v = fabs(a[i * m + k]);
      if (v > best) {
        best = v;
        p = i;
      }
    }
    if (best == 0.0) {
      dev_fail(st, DEV_ESINGULAR);
      return;
    }
    pv[k] = p;
    if (p != k)
      for (int j = 0; j < m; ++j) {
        const double t = a[k * m + j];
        a[k * m + j] = a[p * m + j];
        a[p * m + j] = t;
      }
    const double d = a[k * m + k];
    for (int i = k + 1; i < m; ++i) {
      const double l = __ddiv_rn(a[i * m + k], d);
      a[i * m + k] = l;
      for (int j = k + 1; j < m; ++j) a[i * m + j] = __dsub_rn(a[i * m + j], __dmul_rn(l, a[k * m + j]));
    }
  }
  if (mixed) {
    int tag = 1;
    if (m <= KAPPA_MAX) {
      // ||D^{-1}||_1 from the explicit inverse columns
      double inv1 = 0.0;
      double x[KAPPA_MAX];
      for (int j = 0; j < m; ++j) {
        for (int i = 0; i < m; ++i) x[i] = (i == j) ? 1.0 : 0.0;
        for (int k = 0; k < m; ++k)
          if (pv[k] != k) {
            const double t = x[k];
            x[k] = x[pv[k]];
            x[pv[k]] = t;
          }
        for (int i = 1; i < m; ++i)
          for (int k = 0; k < i; ++k) x[i] -= a[i * m + k] * x[k];
        for (int i = m - 1; i >= 0; --i) {
          double s = x[i];
          for (int k = i + 1; k < m; ++k) s -= a[i * m + k] * x[k];
          x[i] = s / a[i * m + i];
        }
        double cs = 0.0;
        for (int i = 0; i < m; ++i) cs += fabs(x[i]);
        inv1 = fmax(inv1, cs);
      }
      tag = (norm1 * inv1 > cond_thr) ? 1 : 0;
    }
    ptag[y] = tag;
    for (int e = 0; e < m * m; ++e) val32[voff[y] + e] = (float)a[e];
  }
}

// The same for one block with the 32 lanes of a warp: pivot search by a warp
// reduction (largest magnitude, lowest row on ties), multipliers and the
// trailing update over lanes, column sums and inverse columns over lanes;
// every element receives the sequential algorithm's operations in its order,
// so the result equals gepp_item_thread's bit for bit.
__device__ void gepp_item_warp(int64_t y, int lane, const int32_t* __restrict__ sz,
                               const int64_t* __restrict__ roff, const int64_t* __restrict__ voff,
                               double* __restrict__ val, int32_t* __restrict__ piv, int mixed, double cond_thr,
                               int32_t* __restrict__ ptag, float* __restrict__ val32, int* st) {
  const int m = sz[y];
  double* a = val + voff[y];
  int32_t* pv = piv + roff[y];
  double norm1 = 0.0;
  if (mixed) {
    for (int j = lane; j < m; j += 32) {
      double s = 0.0;
      for (int i = 0; i < m; ++i) s += fabs(a[i * m + j]);
      norm1 = fmax(norm1, s);
    }
    for (int o = 16; o > 0; o >>= 1) norm1 = fmax(norm1, __shfl_xor_sync(0xffffffffu, norm1, o));
  }
  for (int k = 0; k < m; ++k) {
    double best = -1.0;
    int p = 0x7fffffff;
    for (int i = k + lane; i < m; i += 32) {
      const double v = fabs(a[i * m + k]);
      if (v > best) {
        best = v;
        p = i;
      }
    }
    for (int o = 16; o > 0; o >>= 1) {
      const double ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int op = __shfl_xor_sync(0xffffffffu, p, o);
      if (ob > best || (ob == best && op < p)) {
        best = ob;
        p = op;
      }
    }
    if (best == 0.0) {
      if (lane == 0) dev_fail(st, DEV_ESINGULAR);
      return;
    }
    if (lane == 0) pv[k] = p;
    if (p != k)
      for (int j = lane; j < m; j += 32) {
        const double t = a[k * m + j];
        a[k * m + j] = a[p * m + j];
        a[p * m + j] = t;
      }
    __syncwarp();
    const double d = a[k * m + k];
    const int w = m - k - 1;
    for (int r = lane; r < w; r += 32) a[(k + 1 + r) * m + k] = __ddiv_rn(a[(k + 1 + r) * m + k], d);
    __syncwarp();
    for (int e = lane; e < w * w; e += 32) {
      const int r = e / w, c = e - r * w;
      const int i = k + 1 + r, j = k + 1 + c;
      a[i * m + j] = __dsub_rn(a[i * m + j], __dmul_rn(a[i * m + k], a[k * m + j]));
    }
    __syncwarp();
  }
  if (mixed) {
    int tag = 1;
    if (m <= KAPPA_MAX) {
      double inv1 = 0.0;
      for (int j = lane; j < m; j += 32) {
        double x[KAPPA_MAX];
        for (int i = 0; i < m; ++i) x[i] = (i == j) ? 1.0 : 0.0;
        for (int k = 0; k < m; ++k)
          if (pv[k] != k) {
            const double t = x[k];
            x[k] = x[pv[k]];
            x[pv[k]] = t;
          }
        for (int i = 1; i < m; ++i)
          for (int k = 0; k < i; ++k) x[i] -= a[i * m + k] * x[k];
        for (int i = m - 1; i >= 0; --i) {
          double s = x[i];
          for (int k = i + 1; k < m; ++k) s -= a[i * m + k] * x[k];
          x[i] = s / a[i * m + i];
        }
        double cs = 0.0;
        for (int i = 0; i < m; ++i) cs += fabs(x[i]);
        inv1 = fmax(inv1, cs);
      }
      for (int o = 16; o > 0; o >>= 1) inv1 = fmax(inv1, __shfl_xor_sync(0xffffffffu, inv1, o));
      tag = (norm1 * inv1 > cond_thr) ? 1 : 0;
    }
    if (lane == 0) ptag[y] = tag;
    for (int e = lane; e < m * m; e += 32) val32[voff[y] + e] = (float)a[e];
  }
}

// Block-size classes of the queued pivot phase.
constexpr int PQ_NCLASS = 5;
__device__ __forceinline__ int pq_class(int m) { return m <= 4 ? 0 : m <= 8 ? 1 : m <= 16 ? 2 : m <= 32 ? 3 : 4; }

__global__ void k_pq_keys(int64_t nD, const int32_t* __restrict__ sz, unsigned long long* __restrict__ key,
                          int* __restrict__ cnt) {
  for (int64_t y = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; y < nD; y += (int64_t)gridDim.x * blockDim.x) {
    const int c = pq_class(sz[y]);
    key[y] = ((unsigned long long)c << 32) | (unsigned long long)y;
    atomicAdd(&cnt[c], 1);
  }
}

// The pivot phase as one persistent launch over the flattened pivot blocks,
// class by class (items[cstart[c] .. cstart[c+1]) in ascending block order):
// mode[c] = 0 gives each thread an item (a warp claims 32 at a time), 1 gives
// each warp an item.
__global__ void __launch_bounds__(128)
    k_gepp_q(const unsigned long long* __restrict__ items, const int64_t* __restrict__ cstart,
             const int32_t* __restrict__ mode, unsigned long long* __restrict__ ctr, int only,
             const int32_t* __restrict__ sz, const int64_t* __restrict__ roff, const int64_t* __restrict__ voff,
             double* __restrict__ val, int32_t* __restrict__ piv, int mixed, double cond_thr,
             int32_t* __restrict__ ptag, float* __restrict__ val32, int* st) {
  const int lane = threadIdx.x & 31;
  for (int c = 0; c < PQ_NCLASS; ++c) {
    const int64_t c0 = cstart[c], c1 = cstart[c + 1];
    if (c0 == c1 || (only >= 0 && c != only)) continue;
    const int md = mode[c];
    for (;;) {
      long long base = 0;
      if (lane == 0) base = (long long)atomicAdd(&ctr[c], md == 0 ? 32ULL : 1ULL);
      base = __shfl_sync(0xffffffffu, base, 0);
      if (c0 + base >= c1) break;
      if (md == 0) {
        const int64_t q = c0 + base + lane;
        if (q < c1)
          gepp_item_thread((int64_t)(items[q] & 0xffffffffull), sz, roff, voff, val, piv, mixed, cond_thr, ptag,
                           val32, st);
      } else {
        gepp_item_warp((int64_t)(items[c0 + base] & 0xffffffffull), lane, sz, roff, voff, val, piv, mixed,
                       cond_thr, ptag, val32, st);
      }
    }
  }
}

// ---- A8 / A9: W = L^{-1} P F and G = E U^{-1} -----------------------------
// Each lane owns one block of its warp's block row.  X is computed in place
// in a copy of F (resp. E).  The FP32 path uses the FP32 LU unless the pivot
// block is tagged FP64, then it promotes the block to FP64.

// WHICH = 0: W rows (D nodes) from F; WHICH = 1: G rows (C nodes) from E.
template <typename T, int WHICH>
__global__ void k_wg_cand(VBView<T> X, const int32_t* __restrict__ dsz, const int64_t* __restrict__ droff,
                          const int64_t* __restrict__ dvoff, const double* __restrict__ dval,
                          const float* __restrict__ dval32, const int32_t* __restrict__ piv,
                          const int32_t* __restrict__ ptag, double t, double* __restrict__ f2,
                          int8_t* __restrict__ keep) {
  const int lane = threadIdx.x & 31;
  const int64_t wpb = blockDim.x >> 5;
  for (int64_t R = blockIdx.x * wpb + (threadIdx.x >> 5); R < X.nbr; R += (int64_t)gridDim.x * wpb) {
    const int mr = X.rsz[R];
    for (int64_t b = X.bptr[R] + lane; b < X.bptr[R + 1]; b += 32) {
      const int32_t Cc = X.bcol[b];
      const int nc = X.csz[Cc];
      T* x = X.val + X.voff[b];
      const int64_t y = WHICH == 0 ? R : Cc;  // pivot block used
      const int m = dsz[y];
      const bool use64 = (sizeof(T) == sizeof(double)) || (ptag && ptag[y]);
      if (WHICH == 0) {
        if (use64)
          linvp_block<T, double>(dval + dvoff[y], piv + droff[y], m, x, nc);
        else
          linvp_block<T, float>(dval32 + dvoff[y], piv + droff[y], m, x, nc);
      } else {
        if (use64)
          uinv_right_block<T, double>(dval + dvoff[y], m, x, mr);
        else
          uinv_right_block<T, float>(dval32 + dvoff[y], m, x, mr);
      }
      const double f = fro2_d(x, mr * nc);
      f2[b] = f;
      keep[b] = drop_rule(f, mr, nc, t) ? 0 : 1;
    }
  }
}

// Keep at most lfil blocks per row among the kept ones: largest f2, lower
// column on ties (one thread per block row, repeated selection).
__global__ void k_lfil(int64_t nbr, const int64_t* __restrict__ bptr, const int32_t* __restrict__ bcol,
                       const double* __restrict__ f2, int8_t* __restrict__ keep, int lfil, int32_t skip_col_is_row) {
  for (int64_t R = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; R < nbr; R += (int64_t)gridDim.x * blockDim.x) {
    int cnt = 0;
    for (int64_t b = bptr[R]; b < bptr[R + 1]; ++b) cnt += keep[b] && !(skip_col_is_row && bcol[b] == R);
    if (cnt <= lfil) continue;
    // mark the lfil largest with keep = 2, then clear the remaining 1s
    for (int sel = 0; sel < lfil; ++sel) {
      int64_t best = -1;
      for (int64_t b = bptr[R]; b < bptr[R + 1]; ++b) {
        if (keep[b] != 1 || (skip_col_is_row && bcol[b] == R)) continue;
        if (best < 0 || f2[b] > f2[best] || (f2[b] == f2[best] && bcol[b] < bcol[best])) best = b;
      }
      if (best < 0) break;
      keep[best] = 2;
    }
    for (int64_t b = bptr[R]; b < bptr[R + 1]; ++b) {
      if (skip_col_is_row && bcol[b] == R) continue;
      keep[b] = keep[b] == 2 ? 1 : 0;
    }
  }
}

// ---- A10: Schur complement S = C - G W ---------------------------------------
// Pattern: per C row r, the union of C's columns and of the columns of the W
// rows Y with G_rY stored.  PASS 0 counts, PASS 1 writes them ascending.
template <bool GLOBAL, int PASS>
__global__ void __launch_bounds__(LW * 32)
    k_schur_pattern(int64_t nrows, const int32_t* __restrict__ list, const int64_t* __restrict__ Cbptr,
                    const int32_t* __restrict__ Cbcol, const int64_t* __restrict__ Gbptr,
                    const int32_t* __restrict__ Gbcol, const int64_t* __restrict__ Wbptr,
                    const int32_t* __restrict__ Wbcol, int* gtab, uint32_t gcap, int64_t* __restrict__ cnt,
                    const int64_t* __restrict__ Sbptr, int32_t* __restrict__ Sbcol, int32_t* __restrict__ heavy,
                    int* nheavy, int* st) {
  extern __shared__ int smem[];
  __shared__ int nfresh[LW];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int* keys;
  uint32_t cap;
  int limit;
  if (GLOBAL) {
    keys = gtab + ((size_t)blockIdx.x * LW + warp) * gcap;
    cap = gcap;
    limit = (int)gcap;
  } else {
    keys = smem + warp * PAT_CAP;
    cap = PAT_CAP;
    limit = PAT_LIMIT;
  }
  for (int64_t t = (int64_t)blockIdx.x * LW + warp; t < nrows; t += (int64_t)gridDim.x * LW) {
    const int64_t r = list ? list[t] : t;
    for (uint32_t k = lane; k < cap; k += 32) keys[k] = -1;
    if (lane == 0) nfresh[warp] = 0;
    __syncwarp();
    bool full = false;
    for (int64_t b = Cbptr[r] + lane; b < Cbptr[r + 1]; b += 32) {
      bool fresh;
      if (hset_insert(keys, cap - 1, Cbcol[b], &fresh) < 0) {
        full = true;
        break;
      }
      if (fresh) atomicAdd(&nfresh[warp], 1);
    }
    __syncwarp();
    bool over = __any_sync(0xffffffffu, full) || *((volatile int*)&nfresh[warp]) > limit;
    for (int64_t g = Gbptr[r]; g < Gbptr[r + 1] && !over; ++g) {
      const int32_t Y = Gbcol[g];
      for (int64_t b = Wbptr[Y] + lane; b < Wbptr[Y + 1]; b += 32) {
        bool fresh;
        if (hset_insert(keys, cap - 1, Wbcol[b], &fresh) < 0) {
          full = true;
          break;
        }
        if (fresh) atomicAdd(&nfresh[warp], 1);
      }
      __syncwarp();
      over = __any_sync(0xffffffffu, full) || *((volatile int*)&nfresh[warp]) > limit;
    }
    if (over) {
      if (lane == 0) {
        if (GLOBAL)
          dev_fail(st, DEV_INTERNAL);
        else if (PASS == 0)
          heavy[atomicAdd(nheavy, 1)] = (int32_t)r;
      }
      __syncwarp();
      continue;
    }
    const int nf = *((volatile int*)&nfresh[warp]);
    if (PASS == 0) {
      if (lane == 0) cnt[r] = nf;
    } else {
      int base = 0;
      for (uint32_t k0 = 0; k0 < cap; k0 += 32) {
        const uint32_t k = k0 + lane;
        const int key = k < cap ? keys[k] : -1;
        const unsigned bm = __ballot_sync(0xffffffffu, key >= 0);
        __syncwarp();
        if (key >= 0) keys[base + __popc(bm & ((1u << lane) - 1u))] = key;
        base += __popc(bm);
        __syncwarp();
      }
      const int64_t out = Sbptr[r];
      for (int a = lane; a < nf; a += 32) {
        const int key = keys[a];
        int rank = 0;
        for (int q = 0; q < nf; ++q) rank += keys[q] < key ? 1 : 0;
        Sbcol[out + rank] = key;
      }
    }
    __syncwarp();
  }
}

// Upper bound on the distinct columns of the listed S rows (C row plus the
// W rows reached from G), to size the global hash tables of those rows.
__global__ void k_schur_row_bound(int nrows, const int32_t* __restrict__ rows, const int64_t* __restrict__ Cbptr,
                                  const int64_t* __restrict__ Gbptr, const int32_t* __restrict__ Gbcol,
                                  const int64_t* __restrict__ Wbptr, int64_t ncols,
                                  unsigned long long* __restrict__ maxb) {
  const int lane = threadIdx.x & 31;
  const int64_t wpb = blockDim.x >> 5;
  for (int64_t t = blockIdx.x * wpb + (threadIdx.x >> 5); t < nrows; t += (int64_t)gridDim.x * wpb) {
    const int32_t r = rows[t];
    long long b = 0;
    for (int64_t g = Gbptr[r] + lane; g < Gbptr[r + 1]; g += 32) {
      const int32_t Y = Gbcol[g];
      b += Wbptr[Y + 1] - Wbptr[Y];
    }
    b = warp_sum_ll(b) + (Cbptr[r + 1] - Cbptr[r]);
    if (b > ncols) b = ncols;
    if (lane == 0) atomicMax(maxb, (unsigned long long)b);
  }
}

// Numeric phase.  One warp per block row r of S.  The row's values are one
// contiguous run of S (blocks ascending, each row-major), and S has C's row
// partition, so the warp
//   1. stages the row plan in shared memory: S block columns and offsets, the
//      C block feeding each S block, and the (G block, W block) pairs of the
//      row with the S block each pair updates;
//   2. streams the C values into the S run (zero for fill blocks) with
//      coalesced loads and stores;
//   3. for each G block (r, Y) ascending, subtracts G_rY W_Ys from every S
//      block s of W row Y: one lane per column of the W row, the column of W
//      held in registers, the S rows i in batches;
// so every element sees the C value, then the G blocks ascending, each with
// its k terms ascending: the oracle's order.  The run just written stays in
// L2 for the updates.  Rows that exceed the plan's capacities are listed for
// k_schur_numeric_rows.
constexpr int SN_WARPS = 8;   // warps per block
constexpr int SN_NQ = 160;    // S blocks of one row
constexpr int SN_NG = 32;     // G blocks of one row
constexpr int SN_NP = 224;    // (G block, W block) pairs of one row
constexpr int SN_RB = 8;      // S rows updated together
constexpr int SN_MK = 8;      // W column length held in registers
constexpr int SN_CU = 16;     // copy loads in flight per lane

struct SnPlan {
  int64_t gvo[SN_NG];     // value offset of G block g
  int64_t wb0[SN_NG];     // first W block of W row Y_g
  int64_t pwv[SN_NP];     // value offset of the W block of pair t
  int32_t sb[SN_NQ];      // S block columns
  int32_t soff[SN_NQ + 1];  // S block offsets within the run; soff[nq] = run length
  int32_t csrc[SN_NQ];    // C block offset relative to the C row start, or -1
  int32_t lst[SN_NG + 1];   // pairs of G block g: [lst[g], lst[g+1])
  int32_t gm[SN_NG];      // n_Y
  int32_t pq[SN_NP];      // S block of pair t
  int32_t cpre[SN_NP + 1];  // W-row column prefix over the pairs
  unsigned long long fl;     // flops of the rows this warp did (2 n_r n_Y n_s per pair)
};

__device__ __forceinline__ int sn_find(const int32_t* a, int n, int32_t key) {
  int lo = 0, hi = n;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    const int32_t v = a[mid];
    if (v == key) return mid;
    if (v < key)
      lo = mid + 1;
    else
      hi = mid;
  }
  return -1;
}

// One G block's update of the S run with a compile-time pivot size MK = n_Y
// (any number nr of S rows): lane per W-row column, the column of W in
// registers, k ascending per element.
template <typename T, int MK>
__device__ __forceinline__ void sn_update_m(const SnPlan& P, int t0, int cA, int cB, int nr, int lane,
                                            const T* gp, const T* __restrict__ Wv, T* run) {
  int t = t0;
  for (int c = cA + lane; c < cB; c += 32) {
    while (P.cpre[t + 1] <= c) ++t;
    const int j = c - P.cpre[t];
    const int ns = P.cpre[t + 1] - P.cpre[t];
    const T* __restrict__ wv = Wv + P.pwv[t] + j;
    T* dst = run + P.soff[P.pq[t]] + j;
    T wr[MK];
#pragma unroll
    for (int k = 0; k < MK; ++k) wr[k] = wv[k * ns];
    int u = 0;
    for (; u + 2 <= nr; u += 2) {
      T a0 = dst[u * ns], a1 = dst[(u + 1) * ns];
      const T* g0 = gp + u * MK;
#pragma unroll
      for (int k = 0; k < MK; ++k) {
        a0 = msub<T>(a0, g0[k], wr[k]);
        a1 = msub<T>(a1, g0[MK + k], wr[k]);
      }
      dst[u * ns] = a0;
      dst[(u + 1) * ns] = a1;
    }
    if (u < nr) {
      T a0 = dst[u * ns];
      const T* g0 = gp + u * MK;
#pragma unroll
      for (int k = 0; k < MK; ++k) a0 = msub<T>(a0, g0[k], wr[k]);
      dst[u * ns] = a0;
    }
  }
}

// Blocks per SM the register budget aims for: four for FP32 (64 registers),
// two for FP64.
template <typename T>
constexpr int kSnMinBlocks = sizeof(T) == sizeof(float) ? 4 : 2;

template <typename T>
__global__ void __launch_bounds__(SN_WARPS * 32, kSnMinBlocks<T>)
    k_schur_numeric(VBView<T> C, VBView<T> G, VBView<T> W, VBView<T> S, int32_t* __restrict__ slow,
                    int* __restrict__ nslow, unsigned long long* __restrict__ rowctr,
                    unsigned long long* __restrict__ flops, int* st) {
  extern __shared__ __align__(16) unsigned char sn_raw[];
  const int lane = threadIdx.x & 31;
  SnPlan& P = reinterpret_cast<SnPlan*>(sn_raw)[threadIdx.x >> 5];
  const T* __restrict__ Cv = C.val;
  const T* __restrict__ Gv = G.val;
  const T* __restrict__ Wv = W.val;
  if (lane == 0) P.fl = 0;
  for (;;) {
    // rows are handed out one at a time to whichever warp is free
    long long rr = 0;
    if (lane == 0) rr = (long long)atomicAdd(rowctr, 1ULL);
    const int64_t r = __shfl_sync(0xffffffffu, rr, 0);
    if (r >= S.nbr) {
      if (lane == 0 && flops && P.fl) atomicAdd(flops, P.fl);
      break;
    }
    __syncwarp();
    const int64_t s0 = S.bptr[r], s1 = S.bptr[r + 1];
    const int64_t c0 = C.bptr[r], c1 = C.bptr[r + 1];
    const int64_t g0 = G.bptr[r], g1 = G.bptr[r + 1];
    const int nr = S.rsz[r];
    const int64_t vbase = S.voff[s0], vend = S.voff[s1];
    const int64_t cbase = C.voff[c0], cend = C.voff[c1];
    if (s1 - s0 > SN_NQ || g1 - g0 > SN_NG || vend - vbase > INT32_MAX || cend - cbase > INT32_MAX) {
      if (lane == 0) slow[atomicAdd(nslow, 1)] = (int32_t)r;
      continue;
    }
    const int nq = (int)(s1 - s0), ng = (int)(g1 - g0);
    for (int q = lane; q <= nq; q += 32) {
      P.soff[q] = (int32_t)(S.voff[s0 + q] - vbase);
      if (q < nq) {
        P.sb[q] = S.bcol[s0 + q];
        P.csrc[q] = -1;
      }
    }
    int cnt = 0;
    if (lane < ng) {
      const int32_t Y = G.bcol[g0 + lane];
      P.gm[lane] = G.csz[Y];
      P.gvo[lane] = G.voff[g0 + lane];
      const int64_t a = W.bptr[Y];
      P.wb0[lane] = a;
      cnt = (int)(W.bptr[Y + 1] - a);
    }
    int incl = cnt;
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += v;
    }
    const int np = __shfl_sync(0xffffffffu, incl, 31);
    if (lane < ng) P.lst[lane] = incl - cnt;
    if (lane == 0) P.lst[ng] = np;
    if (np > SN_NP) {
      if (lane == 0) slow[atomicAdd(nslow, 1)] = (int32_t)r;
      continue;
    }
    __syncwarp();
    for (int64_t cb = c0 + lane; cb < c1; cb += 32) {
      const int q = sn_find(P.sb, nq, C.bcol[cb]);
      if (q >= 0)
        P.csrc[q] = (int32_t)(C.voff[cb] - cbase);
      else
        dev_fail(st, DEV_INTERNAL);
    }
    int carry = 0;
    long long pf = 0;
    for (int base = 0; base < np; base += 32) {
      const int t = base + lane;
      int ns = 0;
      if (t < np) {
        int lo = 0, hi = ng - 1;  // last g with lst[g] <= t
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (P.lst[mid] <= t)
            lo = mid;
          else
            hi = mid - 1;
        }
        const int64_t wb = P.wb0[lo] + (t - P.lst[lo]);
        int q = sn_find(P.sb, nq, W.bcol[wb]);
        if (q < 0) {
          dev_fail(st, DEV_INTERNAL);
          q = 0;
        }
        P.pq[t] = q;
        P.pwv[t] = W.voff[wb];
        ns = (P.soff[q + 1] - P.soff[q]) / nr;
        pf += 2LL * nr * P.gm[lo] * ns;
      }
      int sc = ns;
      for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, sc, o);
        if (lane >= o) sc += v;
      }
      if (t < np) P.cpre[t + 1] = carry + sc;
      carry += __shfl_sync(0xffffffffu, sc, 31);
    }
    if (lane == 0) P.cpre[0] = 0;
    pf = warp_sum_ll(pf);
    if (lane == 0) P.fl += (unsigned long long)pf;
    __syncwarp();
    // 2. C values (zero for fill) into the run, SN_CU loads in flight per lane
    T* __restrict__ run = S.val + vbase;
    const int vlen = P.soff[nq];
    {
      // the lane's current block: its start, end and C source in registers
      int q = 0, qb = 0, qe = P.soff[1], src = P.csrc[0];
      for (int e0 = 0; e0 < vlen; e0 += 32 * SN_CU) {
        T v[SN_CU];
#pragma unroll
        for (int u = 0; u < SN_CU; ++u) {
          const int e = e0 + u * 32 + lane;
          v[u] = (T)0;
          if (e < vlen) {
            while (qe <= e) {
              ++q;
              qb = qe;
              qe = P.soff[q + 1];
              src = P.csrc[q];
            }
            if (src >= 0) v[u] = Cv[cbase + src + (e - qb)];
          }
        }
#pragma unroll
        for (int u = 0; u < SN_CU; ++u) {
          const int e = e0 + u * 32 + lane;
          if (e < vlen) run[e] = v[u];
        }
      }
    }
    __syncwarp();
    // 3. the G W products, G blocks ascending
    for (int g = 0; g < ng; ++g) {
      const int t0 = P.lst[g], t1 = P.lst[g + 1];
      if (t0 == t1) continue;
      const int m = P.gm[g];
      const T* __restrict__ gp = Gv + P.gvo[g];
      const int cB = P.cpre[t1];
      // compile-time pivot sizes for the blocks of 4-6 unknowns per node
      // and their merges
      if (m >= 4 && m <= 6) {
        if (m == 6)
          sn_update_m<T, 6>(P, t0, P.cpre[t0], cB, nr, lane, gp, Wv, run);
        else if (m == 5)
          sn_update_m<T, 5>(P, t0, P.cpre[t0], cB, nr, lane, gp, Wv, run);
        else
          sn_update_m<T, 4>(P, t0, P.cpre[t0], cB, nr, lane, gp, Wv, run);
        __syncwarp();
        continue;
      }
      if (m == 12) {
        sn_update_m<T, 12>(P, t0, P.cpre[t0], cB, nr, lane, gp, Wv, run);
        __syncwarp();
        continue;
      }
      int t = t0;
      for (int c = P.cpre[t0] + lane; c < cB; c += 32) {
        while (P.cpre[t + 1] <= c) ++t;
        const int j = c - P.cpre[t];
        const int ns = P.cpre[t + 1] - P.cpre[t];
        const T* __restrict__ wv = Wv + P.pwv[t] + j;
        T* __restrict__ dst = run + P.soff[P.pq[t]] + j;
        if (m <= SN_MK) {
          T wr[SN_MK];
#pragma unroll
          for (int k = 0; k < SN_MK; ++k) wr[k] = k < m ? wv[k * ns] : (T)0;
          for (int i0 = 0; i0 < nr; i0 += SN_RB) {
            T a[SN_RB];
#pragma unroll
            for (int u = 0; u < SN_RB; ++u)
              if (i0 + u < nr) a[u] = dst[(i0 + u) * ns];
#pragma unroll
            for (int u = 0; u < SN_RB; ++u) {
              if (i0 + u < nr) {
                const T* gi = gp + (i0 + u) * m;
#pragma unroll
                for (int k = 0; k < SN_MK; ++k)
                  if (k < m) a[u] = msub<T>(a[u], gi[k], wr[k]);
              }
            }
#pragma unroll
            for (int u = 0; u < SN_RB; ++u)
              if (i0 + u < nr) dst[(i0 + u) * ns] = a[u];
          }
        } else {
          for (int i = 0; i < nr; ++i) {
            T a = dst[i * ns];
            for (int k = 0; k < m; ++k) a = msub<T>(a, gp[i * m + k], wv[k * ns]);
            dst[i * ns] = a;
          }
        }
      }
      __syncwarp();
    }
  }
}

// Rows beyond the plan capacities: the same order of operations, one warp per
// listed row, with the row's blocks located by binary search in global memory.
template <typename T>
__global__ void __launch_bounds__(LW * 32)
    k_schur_numeric_rows(VBView<T> C, VBView<T> G, VBView<T> W, VBView<T> S, const int32_t* __restrict__ rows,
                         const int* __restrict__ nrows, unsigned long long* __restrict__ flops, int* st) {
  const int lane = threadIdx.x & 31;
  const int64_t wpb = blockDim.x >> 5;
  const int64_t total = *nrows;
  unsigned long long wfl = 0;
  for (int64_t t = blockIdx.x * wpb + (threadIdx.x >> 5); t < total; t += (int64_t)gridDim.x * wpb) {
    const int64_t r = rows[t];
    const int nr = S.rsz[r];
    const int64_t s0 = S.bptr[r], s1 = S.bptr[r + 1];
    for (int64_t q = s0; q < s1; ++q) {
      const int32_t J = S.bcol[q];
      const int64_t cb = bsearch_i32(C.bcol, C.bptr[r], C.bptr[r + 1], J);
      const int n = nr * S.csz[J];
      T* dst = S.val + S.voff[q];
      for (int e = lane; e < n; e += 32) dst[e] = cb >= 0 ? C.val[C.voff[cb] + e] : (T)0;
    }
    __syncwarp();
    for (int64_t g = G.bptr[r]; g < G.bptr[r + 1]; ++g) {
      const int32_t Y = G.bcol[g];
      const int m = G.csz[Y];
      const T* gb = G.val + G.voff[g];
      for (int64_t wb = W.bptr[Y]; wb < W.bptr[Y + 1]; ++wb) {
        const int32_t sc = W.bcol[wb];
        const int ns = W.csz[sc];
        const int64_t q = bsearch_i32(S.bcol, s0, s1, sc);
        if (q < 0) {
          if (lane == 0) dev_fail(st, DEV_INTERNAL);
          continue;
        }
        const T* wv = W.val + W.voff[wb];
        T* dst = S.val + S.voff[q];
        if (lane == 0) wfl += 2ull * (unsigned long long)nr * (unsigned long long)m * (unsigned long long)ns;
        for (int e = lane; e < nr * ns; e += 32) {
          const int i = e / ns, j = e - i * ns;
          T acc = dst[e];
          for (int k = 0; k < m; ++k) acc = msub<T>(acc, gb[i * m + k], wv[k * ns + j]);
          dst[e] = acc;
        }
      }
      __syncwarp();
    }
  }
  if (lane == 0 && flops && wfl) atomicAdd(flops, wfl);
}

// Last reduction: drop off-diagonal blocks of S below the threshold.
template <typename T>
__global__ void k_schur_drop(VBView<T> S, double t, int8_t* __restrict__ keep) {
  const int lane = threadIdx.x & 31;
  const int64_t wpb = blockDim.x >> 5;
  for (int64_t r = blockIdx.x * wpb + (threadIdx.x >> 5); r < S.nbr; r += (int64_t)gridDim.x * wpb) {
    const int nr = S.rsz[r];
    for (int64_t b = S.bptr[r] + lane; b < S.bptr[r + 1]; b += 32) {
      const int32_t J = S.bcol[b];
      const int nc = S.csz[J];
      keep[b] = (J == r || !drop_rule(fro2_d(S.val + S.voff[b], nr * nc), nr, nc, t)) ? 1 : 0;
    }
  }
}

}  // namespace

// ============================================================================
template <typename TA>
void scale_level_t(VBDev<TA>& A, DBuf<double>& r, DBuf<double>& c, cudaStream_t s) {
  const int64_t n = A.nbr ? d2h(A.roff.p + A.nbr, s) : 0;
  r.alloc(n, s);
  c.alloc(n, s);
  if (!A.nbr) return;
  DBuf<unsigned long long> cmax(n, s);
  cmax.zero();
  const unsigned g = grid_for(A.nbr, LW);
  launch(k_rowmax<TA>, g, LW * 32, 0, s, A.view(), r.p);
  VB_LAUNCH_CHECK();
  launch(k_colmax<TA>, g, LW * 32, 0, s, A.view(), r.p, cmax.p);
  VB_LAUNCH_CHECK();
  launch(k_colinv, grid_for(n, 256), 256, 0, s, n, cmax.p, c.p);
  VB_LAUNCH_CHECK();
  launch(k_apply_scale<TA>, g, LW * 32, 0, s, A.view(), r.p, c.p);
  VB_LAUNCH_CHECK();
}
template void scale_level_t<double>(VBDev<double>&, DBuf<double>&, DBuf<double>&, cudaStream_t);
template void scale_level_t<float>(VBDev<float>&, DBuf<double>&, DBuf<double>&, cudaStream_t);

void scale_level(VBDev<double>& A, DBuf<double>& r, DBuf<double>& c, cudaStream_t s) { scale_level_t(A, r, c, s); }

template <typename TA>
int64_t is_order(const VBDev<TA>& A, double ddtol, DBuf<double>& w, DBuf<int32_t>& pI, DBuf<int32_t>& newpos,
                 cudaStream_t s, const int32_t* fixed) {
  const int64_t p = A.nbr;
  w.alloc(p, s);
  pI.alloc(p, s);
  newpos.alloc(p, s);
  if (!p) return 0;
  const unsigned g = grid_for(p, 256);
  launch(k_weights<TA>, grid_for(p, LW), LW * 32, 0, s, A.view(), w.p);
  VB_LAUNCH_CHECK();
  DBuf<int32_t> tcnt(p, s), trow(A.nnzb, s), pending(p, s), state(p, s);
  DBuf<int64_t> tptr(p + 1, s);
  tcnt.zero();
  const unsigned gw = grid_for(p, LW);
  launch(k_tcount, gw, LW * 32, 0, s, p, A.bptr.p, A.bcol.p, tcnt.p);
  VB_LAUNCH_CHECK();
  scan_i32_to_i64(tcnt.p, tptr.p, p, s);
  tcnt.zero();
  launch(k_tfill, gw, LW * 32, 0, s, p, A.bptr.p, A.bcol.p, tptr.p, tcnt.p, trow.p);
  VB_LAUNCH_CHECK();
  DBuf<unsigned long long> remaining(1, s);
  {
    unsigned long long pp = (unsigned long long)p;
    h2d(remaining.p, &pp, 1, s);
  }
  launch(k_is_init, g, 256, 0, s, p, A.bptr.p, A.bcol.p, tptr.p, trow.p, w.p, ddtol, fixed, pending.p, state.p,
         remaining.p);
  VB_LAUNCH_CHECK();
  for (int64_t round = 0;; ++round) {
    launch(k_is_round_b, g, 256, 0, s, p, A.bptr.p, A.bcol.p, tptr.p, trow.p, w.p, pending.p, state.p);
    VB_LAUNCH_CHECK();
    launch(k_is_round_a, g, 256, 0, s, p, A.bptr.p, A.bcol.p, tptr.p, trow.p, pending.p, state.p, remaining.p);
    VB_LAUNCH_CHECK();
    if (round < 4 || (round & 3) == 3)
      if (d2h(remaining.p, s) == 0) break;
    if (round > p + 8) fail(VB_EINTERNAL, "independent-set rounds did not terminate");
  }
  DBuf<int32_t> isD(p, s), isC(p, s);
  launch(k_is_flags, g, 256, 0, s, p, state.p, isD.p, isC.p);
  VB_LAUNCH_CHECK();
  DBuf<int64_t> scanD(p + 1, s), scanC(p + 1, s);
  scan_i32_to_i64(isD.p, scanD.p, p, s);
  scan_i32_to_i64(isC.p, scanC.p, p, s);
  const int64_t nD = d2h(scanD.p + p, s);
  launch(k_is_positions, g, 256, 0, s, p, isD.p, scanD.p, scanC.p, nD, newpos.p, pI.p);
  VB_LAUNCH_CHECK();
  return nD;
}
template <typename TA>
void level_weights(const VBDev<TA>& A, DBuf<double>& w, cudaStream_t s) {
  const int64_t p = A.nbr;
  w.alloc(std::max<int64_t>(p, 1), s);
  if (!p) return;
  launch(k_weights<TA>, grid_for(p, LW), LW * 32, 0, s, A.view(), w.p);
  VB_LAUNCH_CHECK();
}
template void level_weights<double>(const VBDev<double>&, DBuf<double>&, cudaStream_t);
template void level_weights<float>(const VBDev<float>&, DBuf<double>&, cudaStream_t);

template int64_t is_order<double>(const VBDev<double>&, double, DBuf<double>&, DBuf<int32_t>&, DBuf<int32_t>&,
                                  cudaStream_t, const int32_t*);
template int64_t is_order<float>(const VBDev<float>&, double, DBuf<double>&, DBuf<int32_t>&, DBuf<int32_t>&,
                                 cudaStream_t, const int32_t*);

template <typename TA, typename T>
void gather_parts(const VBDev<TA>& A, const DBuf<int32_t>& pI, const DBuf<int32_t>& newpos, int64_t nD,
                  LevelDev<T>& L, cudaStream_t s, int* dst) {
  const int64_t p = A.nbr, nC = p - nD;
  L.nD = nD;
  L.nC = nC;
  DBuf<int32_t> psz(p, s);
  launch(k_perm_sizes, grid_for(p, 256), 256, 0, s, p, pI.p, A.rsz.p, psz.p);
  VB_LAUNCH_CHECK();
  const int32_t* szD = psz.p;
  const int32_t* szC = psz.p + nD;
  set_partitions(L.D, szD, nD, szD, nD, s);
  set_partitions(L.F, szD, nD, szC, nC, s);
  set_partitions(L.E, szC, nC, szD, nD, s);
  set_partitions(L.C, szC, nC, szC, nC, s);
  DBuf<int64_t> cF(nD, s), cE(nC, s), cC(nC, s);
  const unsigned gw = grid_for(p, LW);
  launch(k_gather<0>, gw, LW * 32, 0, s, p, nD, A.bptr.p, A.bcol.p, newpos.p, cF.p, cE.p, cC.p, nullptr, nullptr,
                                     nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, dst);
  VB_LAUNCH_CHECK();
  check_status(dst, s, "vbarms_factor: gather");
  L.F.bptr.alloc(nD + 1, s);
  L.E.bptr.alloc(nC + 1, s);
  L.C.bptr.alloc(nC + 1, s);
  scan_i64(cF.p, L.F.bptr.p, nD, s);
  scan_i64(cE.p, L.E.bptr.p, nC, s);
  scan_i64(cC.p, L.C.bptr.p, nC, s);
  const int64_t nF = d2h(L.F.bptr.p + nD, s), nE = d2h(L.E.bptr.p + nC, s), nCC = d2h(L.C.bptr.p + nC, s);
  L.F.bcol.alloc(nF, s);
  L.E.bcol.alloc(nE, s);
  L.C.bcol.alloc(nCC, s);
  // D: one block per row, column = row
  {
    std::vector<int64_t> hb(nD + 1);
    std::vector<int32_t> hc(nD);
    for (int64_t k = 0; k <= nD; ++k) hb[k] = k;
    for (int64_t k = 0; k < nD; ++k) hc[k] = (int32_t)k;
    L.D.bptr.alloc(nD + 1, s);
    L.D.bcol.alloc(nD, s);
    h2d(L.D.bptr.p, hb.data(), nD + 1, s);
    h2d(L.D.bcol.p, hc.data(), nD, s);
    VB_CUDA(cudaStreamSynchronize(s));
  }
  DBuf<int64_t> sD(nD, s), sF(nF, s), sE(nE, s), sC(nCC, s);
  launch(k_gather<1>, gw, LW * 32, 0, s, p, nD, A.bptr.p, A.bcol.p, newpos.p, nullptr, nullptr, nullptr, L.F.bptr.p,
                                     L.E.bptr.p, L.C.bptr.p, L.F.bcol.p, L.E.bcol.p, L.C.bcol.p, sD.p, sF.p, sE.p,
                                     sC.p, dst);
  VB_LAUNCH_CHECK();
  finish_offsets(L.D, s);
  finish_offsets(L.F, s);
  finish_offsets(L.E, s);
  finish_offsets(L.C, s);
  if (nD) launch(k_copy_blocks<TA, double>, grid_for(nD, LW), LW * 32, 0, s, nD, sD.p, A.voff.p, A.val.p, L.D.voff.p, L.D.val.p);
  if (nF) launch(k_copy_blocks<TA, T>, grid_for(nF, LW), LW * 32, 0, s, nF, sF.p, A.voff.p, A.val.p, L.F.voff.p, L.F.val.p);
  if (nE) launch(k_copy_blocks<TA, T>, grid_for(nE, LW), LW * 32, 0, s, nE, sE.p, A.voff.p, A.val.p, L.E.voff.p, L.E.val.p);
  if (nCC) launch(k_copy_blocks<TA, T>, grid_for(nCC, LW), LW * 32, 0, s, nCC, sC.p, A.voff.p, A.val.p, L.C.voff.p, L.C.val.p);
  VB_LAUNCH_CHECK();
  check_status(dst, s, "vbarms_factor: gather");
}

namespace {
std::mutex g_pq_mu;
std::map<long long, int> g_pq_mode;  // (device, class, mixed) -> the faster mode
constexpr int64_t kPqTuneMin = 1024;  // items of a class before its modes are timed
}  // namespace

// A7 as one persistent launch over block-size-class queues (A14): the pivot
// blocks are flattened into classes by size (<= 4, <= 8, <= 16, <= 32, more),
// each class run one item per thread or one per warp.  The mode of a class is
// timed on a copy of this level's own blocks of that class the first time the
// process meets it on a device (results do not depend on it), and reused.
void pivot_lu(VBDev<double>& D, DBuf<int32_t>& piv, DBuf<int32_t>& ptag, VBDev<float>& D32, bool mixed,
              double cond_thr, cudaStream_t s, int* dst, PivotTiles* info) {
  const int64_t nD = D.nbr;
  const int64_t nsc = nD ? d2h(D.roff.p + nD, s) : 0;
  piv.alloc(nsc, s);
  ptag.alloc(nD, s);
  if (mixed) {
    copy_vb<float, double>(D, D32, s);
  }
  if (!nD) return;
  DBuf<unsigned long long> items(nD, s);
  DBuf<int> cnt(PQ_NCLASS, s);
  cnt.zero();
  launch(k_pq_keys, grid_for(nD, 256), 256, 0, s, nD, D.rsz.p, items.p, cnt.p);
  VB_LAUNCH_CHECK();
  radix_sort_u64(items, nullptr, nD, 35, s);
  const std::vector<int> hc = d2h_vec(cnt.p, PQ_NCLASS, s);
  std::vector<int64_t> hs(PQ_NCLASS + 1, 0);
  for (int c = 0; c < PQ_NCLASS; ++c) hs[c + 1] = hs[c] + hc[c];
  DBuf<int64_t> cstart(PQ_NCLASS + 1, s);
  h2d(cstart.p, hs.data(), PQ_NCLASS + 1, s);
  int dev = 0, nsm = 0;
  VB_CUDA(cudaGetDevice(&dev));
  VB_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>((int64_t)nsm * 8, (nD + 127) / 128));
  int32_t mode[PQ_NCLASS];
  int source = 0;
  DBuf<int32_t> dmode(PQ_NCLASS, s);
  DBuf<unsigned long long> ctr(PQ_NCLASS, s);
  {
    std::lock_guard<std::mutex> lk(g_pq_mu);
    DBuf<double> sv;
    DBuf<int32_t> sp, st2;
    DBuf<float> s32;
    for (int c = 0; c < PQ_NCLASS; ++c) {
      mode[c] = c >= 2 ? 1 : 0;  // default: a thread per block up to 8, a warp above
      const long long key = ((long long)dev << 8) | ((long long)c << 1) | (mixed ? 1 : 0);
      auto it = g_pq_mode.find(key);
      if (it != g_pq_mode.end()) {
        mode[c] = it->second;
        source = std::max(source, 2);
        continue;
      }
      if (hc[c] < kPqTuneMin) continue;
      if (!sv.p) {
        sv.alloc(std::max<int64_t>(D.nval, 1), s);
        sp.alloc(std::max<int64_t>(nsc, 1), s);
        st2.alloc(nD, s);
        if (mixed) s32.alloc(std::max<int64_t>(D.nval, 1), s);
      }
      float ms[2] = {0.f, 0.f};
      cudaEvent_t e0, e1;
      VB_CUDA(cudaEventCreate(&e0));
      VB_CUDA(cudaEventCreate(&e1));
      for (int md = 0; md < 2; ++md) {
        VB_CUDA(cudaMemcpyAsync(sv.p, D.val.p, D.nval * sizeof(double), cudaMemcpyDeviceToDevice, s));
        int32_t hm[PQ_NCLASS];
        for (int q = 0; q < PQ_NCLASS; ++q) hm[q] = md;
        h2d(dmode.p, hm, PQ_NCLASS, s);
        ctr.zero();
        VB_CUDA(cudaEventRecord(e0, s));
        launch(k_gepp_q, grid, 128, 0, s, items.p, cstart.p, dmode.p, ctr.p, c, D.rsz.p, D.roff.p, D.voff.p, sv.p,
               sp.p, mixed ? 1 : 0, cond_thr, st2.p, mixed ? s32.p : nullptr, dst);
        VB_CUDA(cudaEventRecord(e1, s));
        VB_LAUNCH_CHECK();
        VB_CUDA(cudaEventSynchronize(e1));
        VB_CUDA(cudaEventElapsedTime(&ms[md], e0, e1));
      }
      VB_CUDA(cudaEventDestroy(e0));
      VB_CUDA(cudaEventDestroy(e1));
      mode[c] = ms[1] < ms[0] ? 1 : 0;
      g_pq_mode[key] = mode[c];
      source = std::max(source, 1);
    }
  }
  h2d(dmode.p, mode, PQ_NCLASS, s);
  ctr.zero();
  launch(k_gepp_q, grid, 128, 0, s, items.p, cstart.p, dmode.p, ctr.p, -1, D.rsz.p, D.roff.p, D.voff.p, D.val.p,
         piv.p, mixed ? 1 : 0, cond_thr, ptag.p, mixed ? D32.val.p : nullptr, dst);
  VB_LAUNCH_CHECK();
  check_status(dst, s, "vbarms_factor: pivot LU");
  if (info) {
    for (int c = 0; c < PQ_NCLASS; ++c) {
      info->count[c] = hc[c];
      info->mode[c] = mode[c];
    }
    info->source = source;
  }
}

template <typename T>
void w_or_g(const VBDev<T>& X, int which, const VBDev<double>& D, const VBDev<float>& D32, const DBuf<int32_t>& piv,
            const DBuf<int32_t>& ptag, bool mixed, double t, int lfil, VBDev<T>& out, cudaStream_t s) {
  VBDev<T> cand;
  copy_vb<T, T>(X, cand, s);
  DBuf<double> f2(cand.nnzb, s);
  DBuf<int8_t> keep(cand.nnzb, s);
  if (cand.nbr && cand.nnzb) {
    const unsigned g = grid_for(cand.nbr, LW);
    if (which == 0)
      launch(k_wg_cand<T, 0>, g, LW * 32, 0, s, cand.view(), D.rsz.p, D.roff.p, D.voff.p, D.val.p,
                                            mixed ? D32.val.p : nullptr, piv.p, mixed ? ptag.p : nullptr, t, f2.p,
                                            keep.p);
    else
      launch(k_wg_cand<T, 1>, g, LW * 32, 0, s, cand.view(), D.rsz.p, D.roff.p, D.voff.p, D.val.p,
                                            mixed ? D32.val.p : nullptr, piv.p, mixed ? ptag.p : nullptr, t, f2.p,
                                            keep.p);
    VB_LAUNCH_CHECK();
    if (lfil >= 0) {
      launch(k_lfil, grid_for(cand.nbr, 128), 128, 0, s, cand.nbr, cand.bptr.p, cand.bcol.p, f2.p, keep.p, lfil, 0);
      VB_LAUNCH_CHECK();
    }
  }
  compact_blocks(cand, keep.p, out, s);
}

template <typename T>
void schur(const VBDev<T>& C, const VBDev<T>& G, const VBDev<T>& W, bool last_reduction, double t, VBDev<T>& S,
           cudaStream_t s, int* dst, KernelRec* rec) {
  const int64_t nC = C.nbr;
  VBDev<T> Sf;
  set_partitions(Sf, C.rsz.p, nC, C.rsz.p, nC, s);
  Sf.bptr.alloc(nC + 1, s);
  DBuf<int64_t> cnt(nC, s);
  DBuf<int32_t> heavy(std::max<int64_t>(nC, 1), s);
  DBuf<int> nheavy(1, s);
  nheavy.zero();
  const size_t smem = (size_t)LW * PAT_CAP * sizeof(int);
  VB_CUDA(cudaFuncSetAttribute(k_schur_pattern<false, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  VB_CUDA(cudaFuncSetAttribute(k_schur_pattern<false, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const unsigned gl = grid_for(nC, LW, 152LL * 24);
  if (nC) {
    launch(k_schur_pattern<false, 0>, gl, LW * 32, smem, s, nC, nullptr, C.bptr.p, C.bcol.p, G.bptr.p, G.bcol.p,
                                                        W.bptr.p, W.bcol.p, nullptr, 0, cnt.p, nullptr, nullptr,
                                                        heavy.p, nheavy.p, dst);
    VB_LAUNCH_CHECK();
  }
  const int nh = d2h(nheavy.p, s);
  uint32_t gcap = 0;
  int64_t hb = 0;
  DBuf<int> gtab;
  if (nh > 0) {
    // tables sized by the heaviest listed row, not by the matrix width
    DBuf<unsigned long long> bound(1, s);
    bound.zero();
    launch(k_schur_row_bound, grid_for(nh, LW), LW * 32, 0, s, nh, heavy.p, C.bptr.p, G.bptr.p, G.bcol.p, W.bptr.p,
           nC, bound.p);
    VB_LAUNCH_CHECK();
    const int64_t maxb = (int64_t)d2h(bound.p, s);
    gcap = 1024;
    while ((int64_t)gcap < 2 * maxb + 64) gcap <<= 1;
    int64_t warps = std::max<int64_t>(1, (256LL << 20) / ((int64_t)gcap * 4));
    warps = std::min<int64_t>(warps, nh);
    hb = (warps + LW - 1) / LW;
    gtab.alloc((size_t)hb * LW * gcap, s);
    launch(k_schur_pattern<true, 0>, (unsigned)hb, LW * 32, 0, s, nh, heavy.p, C.bptr.p, C.bcol.p, G.bptr.p, G.bcol.p,
                                                             W.bptr.p, W.bcol.p, gtab.p, gcap, cnt.p, nullptr,
                                                             nullptr, nullptr, nullptr, dst);
    VB_LAUNCH_CHECK();
  }
  check_status(dst, s, "vbarms_factor: Schur pattern");
  scan_i64(cnt.p, Sf.bptr.p, nC, s);
  Sf.nnzb = nC ? d2h(Sf.bptr.p + nC, s) : 0;
  Sf.bcol.alloc(Sf.nnzb, s);
  if (nC) {
    launch(k_schur_pattern<false, 1>, gl, LW * 32, smem, s, nC, nullptr, C.bptr.p, C.bcol.p, G.bptr.p, G.bcol.p,
                                                        W.bptr.p, W.bcol.p, nullptr, 0, nullptr, Sf.bptr.p,
                                                        Sf.bcol.p, nullptr, nullptr, dst);
    VB_LAUNCH_CHECK();
  }
  if (nh > 0) {
    launch(k_schur_pattern<true, 1>, (unsigned)hb, LW * 32, 0, s, nh, heavy.p, C.bptr.p, C.bcol.p, G.bptr.p, G.bcol.p,
                                                             W.bptr.p, W.bcol.p, gtab.p, gcap, nullptr, Sf.bptr.p,
                                                             Sf.bcol.p, nullptr, nullptr, dst);
    VB_LAUNCH_CHECK();
  }
  check_status(dst, s, "vbarms_factor: Schur pattern");
  finish_offsets(Sf, s);
  if (nC) {
    DBuf<int32_t> slow(nC, s);
    DBuf<int> nslow(1, s);
    nslow.zero();
    DBuf<unsigned long long> fl(1, s);  // flops of the numeric phase, counted by its kernels
    fl.zero();
    if (rec) {
      // algorithmic work of the numeric phase: read C, G, W and write S once
      // (values and their index arrays); flops = sum over (r, Y, s) of
      // 2 n_r n_Y n_s
      auto idx = [](const VBDev<T>& M) {
        return 8.0 * (M.nbr + 1) + 4.0 * M.nnzb + 8.0 * (M.nnzb + 1);
      };
      rec->bytes = (double)sizeof(T) * (double)(C.nval + G.nval + W.nval + Sf.nval) + idx(C) + idx(G) + idx(W) +
                   idx(Sf);
      VB_CUDA(cudaEventCreate(&rec->e0));
      VB_CUDA(cudaEventCreate(&rec->e1));
      VB_CUDA(cudaEventRecord(rec->e0, s));
    }
    const size_t psmem = (size_t)SN_WARPS * sizeof(SnPlan);
    VB_CUDA(cudaFuncSetAttribute(k_schur_numeric<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)psmem));
    int dev = 0, nsm = 0, per_sm = 0;
    VB_CUDA(cudaGetDevice(&dev));
    VB_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    VB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_schur_numeric<T>, SN_WARPS * 32, psmem));
    DBuf<unsigned long long> rowctr(1, s);
    rowctr.zero();
    launch(k_schur_numeric<T>, grid_for(nC, SN_WARPS, (int64_t)nsm * std::max(per_sm, 1)), SN_WARPS * 32, psmem, s,
           C.view(), G.view(), W.view(), Sf.view(), slow.p, nslow.p, rowctr.p, fl.p, dst);
    VB_LAUNCH_CHECK();
    launch(k_schur_numeric_rows<T>, 152u * 4, LW * 32, 0, s, C.view(), G.view(), W.view(), Sf.view(), slow.p,
           nslow.p, fl.p, dst);
    VB_LAUNCH_CHECK();
    if (rec) {
      VB_CUDA(cudaEventRecord(rec->e1, s));
      rec->flops = (double)d2h(fl.p, s);
    }
  }
  check_status(dst, s, "vbarms_factor: Schur numeric");
  if (last_reduction && nC) {
    DBuf<int8_t> keep(Sf.nnzb, s);
    launch(k_schur_drop<T>, grid_for(nC, LW), LW * 32, 0, s, Sf.view(), t, keep.p);
    VB_LAUNCH_CHECK();
    compact_blocks(Sf, keep.p, S, s);
  } else {
    S = std::move(Sf);
  }
}

#define VB_LEVEL_INST(TA, T)                                                                                     \
  template void gather_parts<TA, T>(const VBDev<TA>&, const DBuf<int32_t>&, const DBuf<int32_t>&, int64_t,     \
                                    LevelDev<T>&, cudaStream_t, int*);
VB_LEVEL_INST(double, double)
VB_LEVEL_INST(double, float)
VB_LEVEL_INST(float, float)
template void w_or_g<double>(const VBDev<double>&, int, const VBDev<double>&, const VBDev<float>&,
                             const DBuf<int32_t>&, const DBuf<int32_t>&, bool, double, int, VBDev<double>&,
                             cudaStream_t);
template void w_or_g<float>(const VBDev<float>&, int, const VBDev<double>&, const VBDev<float>&,
                            const DBuf<int32_t>&, const DBuf<int32_t>&, bool, double, int, VBDev<float>&,
                            cudaStream_t);
template void schur<double>(const VBDev<double>&, const VBDev<double>&, const VBDev<double>&, bool, double,
                            VBDev<double>&, cudaStream_t, int*, KernelRec*);
template void schur<float>(const VBDev<float>&, const VBDev<float>&, const VBDev<float>&, bool, double,
                           VBDev<float>&, cudaStream_t, int*, KernelRec*);

}  // namespace vb
