// Last-level block ILUT of VBARMS on the GPU (Section 3 dropping rule, the
// block IKJ form of Alg. 3), on the scaled last Schur complement in natural
// order.
//
// Row i is processed by one warp that took ticket i (tickets are handed out
// in row order, so every row a warp waits for is already owned by a running
// warp).  A matrix made of independent diagonal blocks (a batch, or the
// subdomains of a domain decomposition) may instead hand out its rows
// interleaved across the blocks, each block's rows in ascending order: the
// blocks' dependency chains then advance side by side.  The warp keeps its working row in a private workspace (hash table
// column -> slot, dense values): in shared memory when the row fits, else in
// global memory (a shared row whose fill outgrows the buffer starts again in
// the global one).  It eliminates its L part in ascending column order
// including fill -- waiting, with a bounded spin, until row k is published,
// then staging row k's pivot block and U row in shared memory -- drops and
// trims, factors its diagonal block (GEPP) and publishes its L and U rows to
// global pools.  Per element, the operation order is the oracle's, so FP64
// results match it bit for bit; the mixed factor keeps its drop sums, drop
// tests and diagonal GEPP in FP32 (a block whose condition estimate exceeds
// the threshold is factored again in FP64).
//
// A wait that runs out sets VB_ETIMEOUT and raises an abort flag; a row that
// failed publishes the flag value 2 so that its dependants stop too.
// Overflowing a pool or the global workspace sets an overflow code and the
// host repeats the kernel with larger buffers.
#include <algorithm>
#include <type_traits>

#include "internal.h"
#include "level.cuh"
#include "vbsr_ops.cuh"

namespace vb {
namespace {

constexpr int IW = 8;  // warps per block

enum : int { SL_LIVE = 0, SL_LKEPT = 1, SL_DEAD = 2 };

struct Pools {
  // L and U rows: blocks in pool order; per row the first block and count
  int32_t* lcol;
  int64_t* lvo;  // value offset of each pool block
  int32_t* ucol;
  int64_t* uvo;
  int64_t* lstart;
  int32_t* lcnt;
  int64_t* ustart;
  int32_t* ucnt;
  unsigned long long* ctr;  // [0] L blocks, [1] L values, [2] U blocks, [3] U values, [4] ticket, [5] max row need
  int64_t lbcap, lvcap, ubcap, uvcap;
  int32_t* done;
  int* abort;
  int64_t* uvstart;  // value offset of the first U block of each row
  int64_t* uvlen;    // values of the U row (its blocks are contiguous)
  // ticket -> row (nullptr: ticket t is row t); every row's dependencies
  // must come earlier in it
  const int32_t* order;
};

struct Workspace {
  int* keys;      // [HT] per warp
  int* hpos;      // [SMAX]
  int* scol;      // [SMAX]
  int* soff;      // [SMAX]
  int* sstate;    // [SMAX]
  long long* sf2;  // [SMAX] norm key of each slot
  int ht, smax;
  int64_t vmax;
};

template <typename T>
__device__ __forceinline__ T msub(T acc, T a, T b);
template <>
__device__ __forceinline__ double msub<double>(double acc, double a, double b) {
  return __dsub_rn(acc, __dmul_rn(a, b));
}
template <>
__device__ __forceinline__ float msub<float>(float acc, float a, float b) {
  return __fmaf_rn(-a, b, acc);
}

__device__ __forceinline__ bool drop_rule(double f2, int m, int n, double t) {
  const double thr = __dmul_rn(__dmul_rn(t, (double)m), (double)n);
  return f2 < __dmul_rn(thr, thr);
}

// The same rule in FP32 for the mixed factor (FP64 operations are slow on
// this part and would sit on the critical path of every elimination step).
__device__ __forceinline__ bool drop_rule_f(float f2, int m, int n, float t) {
  const float thr = t * (float)m * (float)n;
  return f2 < thr * thr;
}

// Squared Frobenius norms are ranked (lfil) by their bit patterns: for
// non-negative IEEE values the integer order is the value order, so the
// comparisons stay on the integer pipes.  FP64 factor: the double's bits;
// mixed factor: the float's bits.
__device__ __forceinline__ long long norm_key(double f2) { return __double_as_longlong(f2); }
__device__ __forceinline__ long long norm_key(float f2) { return (long long)__float_as_int(f2); }

template <typename T>
__device__ __forceinline__ double fro2_seq(const T* v, int n) {
  double s = 0.0;
  for (int e = 0; e < n; ++e) {
    const double x = (double)v[e];
    s = __dadd_rn(s, __dmul_rn(x, x));
  }
  return s;
}

// x (one row of length m) <- x (P^T L U)^{-1} = x U^{-1} L^{-1} P, with the
// factored pivot block read through L2 (written by another warp).
template <typename T, typename TL>
__device__ void ainv_right_row(const TL* lu, const int32_t* pv, int m, T* x) {
  for (int j = 0; j < m; ++j) {
    TL s = (TL)x[j];
    for (int q = 0; q < j; ++q) s = msub<TL>(s, (TL)x[q], __ldcg(lu + q * m + j));
    x[j] = (T)(s / __ldcg(lu + j * m + j));
  }
  for (int j = m - 1; j >= 0; --j) {
    TL s = (TL)x[j];
    for (int q = j + 1; q < m; ++q) s = msub<TL>(s, (TL)x[q], __ldcg(lu + q * m + j));
    x[j] = (T)s;
  }
  for (int k = m - 1; k >= 0; --k) {
    const int p = __ldcg(pv + k);
    if (p > k && p < m) {  // GEPP interchanges satisfy k <= p < m
      const T t = x[k];
      x[k] = x[p];
      x[p] = t;
    }
  }
}

// Workspace hash: keys[h] = -2 - slot, -1 = empty; the column of a slot is
// scol[slot].  Placement and lookup never run concurrently (separated by
// __syncwarp), and the columns inserted in one phase are distinct.
__device__ __forceinline__ int ws_place(int* keys, uint32_t mask, int slot, int col) {
  uint32_t h = hmix((uint32_t)col) & mask;
  for (uint32_t probe = 0; probe <= mask; ++probe) {
    if (atomicCAS(&keys[h], -1, -2 - slot) == -1) return (int)h;
    h = (h + 1) & mask;
  }
  return -1;
}

__device__ __forceinline__ int ws_lookup(const int* keys, const int* scol, uint32_t mask, int col) {
  uint32_t h = hmix((uint32_t)col) & mask;
  for (uint32_t probe = 0; probe <= mask; ++probe) {
    const int kv = keys[h];
    if (kv == -1) return -1;
    const int s = -2 - kv;
    if (scol[s] == col) return s;
    h = (h + 1) & mask;
  }
  return -1;
}

// Claim a new slot of sz values for column col; returns the slot or -1.
__device__ __forceinline__ int ws_new_slot(int smax, int64_t vmax, int* keys, int* hpos, int* scol, int* soff,
                                           int* sstate, int* nslots, unsigned long long* nvals, uint32_t hmask,
                                           int col, int sz) {
  const int slot = atomicAdd(nslots, 1);
  const long long off = (long long)atomicAdd(nvals, (unsigned long long)sz);
  if (slot >= smax) return -1;
  hpos[slot] = -1;  // the end-of-row reset skips slots that were never placed
  if (off + sz > vmax) return -1;
  scol[slot] = col;
  soff[slot] = (int)off;
  sstate[slot] = SL_LIVE;
  hpos[slot] = ws_place(keys, hmask, slot, col);
  return hpos[slot] < 0 ? -1 : slot;
}

constexpr int SMB = 16;         // pivot blocks up to SMB x SMB have their own shared buffer
constexpr int PVMAX = 64;       // larger ones up to PVMAX are staged in free workspace space
constexpr int MAX_SLOTS = 4096;  // largest workspace (blocks of one working row)

// x (one row of length m) <- x (P^T L U)^{-1} from a staged pivot block
// (values held as doubles; TL is the arithmetic type).
template <typename T, typename TL>
__device__ void ainv_right_row_s(const double* lu, const int* pv, int m, T* x) {
  for (int j = 0; j < m; ++j) {
    TL s = (TL)x[j];
    for (int q = 0; q < j; ++q) s = msub<TL>(s, (TL)x[q], (TL)lu[q * m + j]);
    x[j] = (T)(s / (TL)lu[j * m + j]);
  }
  for (int j = m - 1; j >= 0; --j) {
    TL s = (TL)x[j];
    for (int q = j + 1; q < m; ++q) s = msub<TL>(s, (TL)x[q], (TL)lu[q * m + j]);
    x[j] = (T)s;
  }
  for (int k = m - 1; k >= 0; --k) {
    const int p = pv[k];
    if (p > k && p < m) {
      const T t = x[k];
      x[k] = x[p];
      x[p] = t;
    }
  }
}

// Warp-cooperative copy with eight independent loads in flight per lane.
template <typename T>
__device__ __forceinline__ void warp_copy(T* __restrict__ dst, const T* __restrict__ src, int64_t n, int lane) {
  for (int64_t e0 = lane; e0 < n; e0 += 32 * 8) {
    T v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int64_t e = e0 + 32 * u;
      if (e < n) v[u] = src[e];
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int64_t e = e0 + 32 * u;
      if (e < n) dst[e] = v[u];
    }
  }
}

// Squared Frobenius norm in row-major order (the oracle's summation order),
// with the loads issued eight at a time.
template <typename T>
__device__ __forceinline__ double fro2_batched(const T* __restrict__ v, int n) {
  double s = 0.0;
  for (int e0 = 0; e0 < n; e0 += 8) {
    T x[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) x[u] = e0 + u < n ? v[e0 + u] : (T)0;
#pragma unroll
    for (int u = 0; u < 8; ++u)
      if (e0 + u < n) {
        const double d = (double)x[u];
        s = __dadd_rn(s, __dmul_rn(d, d));
      }
  }
  return s;
}

// Squared Frobenius norm accumulated in FP32 (mixed factor).
template <typename T>
__device__ __forceinline__ float fro2_f32(const T* __restrict__ v, int n) {
  float s = 0.f;
#pragma unroll 4
  for (int e = 0; e < n; ++e) {
    const float x = (float)v[e];
    s = __fmaf_rn(x, x, s);
  }
  return s;
}

constexpr int LCAP = 128;           // pending L columns tracked in shared memory per warp
constexpr int USTAGE_BYTES = 2048;  // U row of a dependency staged in shared memory per warp
constexpr int WS_SLOTS = 64;        // working rows held in shared memory: blocks,
constexpr int WS_HASH = 128;        //   hash positions,
constexpr int WS_VBYTES = 4096;     //   value bytes
constexpr int MSH = 96;             // slot metadata of a global working row staged for the finish

// Per-warp shared memory: the working row when it fits (hash table, slot
// metadata, values), the dependency's pivot block and U row, and the
// bookkeeping of one elimination step.
struct IlutWarp {
  __align__(16) unsigned char vals[WS_VBYTES];
  __align__(16) unsigned char ustage[USTAGE_BYTES];
  __align__(16) unsigned char lu[SMB * SMB * sizeof(double)];  // FP64 or FP32 pivot block
  long long sf2[WS_SLOTS];
  long long wdst[32];  // pool value offset of each written block of a chunk
  int keys[WS_HASH];
  int hpos[WS_SLOTS];
  int scol[WS_SLOTS];
  int soff[WS_SLOTS];
  int sstate[WS_SLOTS];
  int pv[PVMAX];
  int qoff[32];  // workspace value offset of each U block's target
  int quo[32];   // value offset of the U block within the U row
  int qnj[32];
  int qpre[33];  // element prefix of the chunk's U blocks
  int lc[LCAP];  // pending L columns (INT_MAX when processed)
  int ls[LCAP];  // their slots
  int nl, nslots, flag, pad;
  unsigned long long nvals;
};

constexpr size_t ilut_smem() { return IW * sizeof(IlutWarp); }
static_assert(MSH * (3 * sizeof(int) + sizeof(long long)) <= USTAGE_BYTES, "finish staging exceeds the U-row buffer");

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// x (one row of length m) <- x (P^T L U)^{-1} from a staged pivot block
// (values of type TS, arithmetic in TL); x lives in shared memory.
template <typename T, typename TL, typename TS>
__device__ void ainv_right_row_sh(const TS* lu, const int* pv, int m, T* x) {
  for (int j = 0; j < m; ++j) {
    TL s = (TL)x[j];
    for (int q = 0; q < j; ++q) s = msub<TL>(s, (TL)x[q], (TL)lu[q * m + j]);
    x[j] = (T)(s / (TL)lu[j * m + j]);
  }
  for (int j = m - 1; j >= 0; --j) {
    TL s = (TL)x[j];
    for (int q = j + 1; q < m; ++q) s = msub<TL>(s, (TL)x[q], (TL)lu[q * m + j]);
    x[j] = (T)s;
  }
  for (int k = m - 1; k >= 0; --k) {
    const int p = pv[k];
    if (p > k && p < m) {
      const T t = x[k];
      x[k] = x[p];
      x[p] = t;
    }
  }
}

// |x| as an integer key: non-negative IEEE values order like their bit
// patterns, so pivot searches compare integers.
__device__ __forceinline__ long long abs_key(double x) { return __double_as_longlong(x) & 0x7fffffffffffffffLL; }
__device__ __forceinline__ long long abs_key(float x) { return (long long)(__float_as_int(x) & 0x7fffffff); }

template <typename TL>
__device__ __forceinline__ TL div_rn(TL a, TL b);
template <>
__device__ __forceinline__ double div_rn<double>(double a, double b) {
  return __ddiv_rn(a, b);
}
template <>
__device__ __forceinline__ float div_rn<float>(float a, float b) {
  return __fdiv_rn(a, b);
}

// GEPP of the n x n row-major block a (max-abs pivot, ties to the lowest
// row), one warp: each elimination step finds its pivot by a warp reduction,
// then the lanes form the multipliers and update the trailing block, so every
// element receives the operations of the sequential algorithm in its order.
// Pivot rows go to gpiv (and pvs when not null).  Returns false when a pivot
// column is exactly zero.
template <typename TL>
__device__ bool gepp_warp(TL* a, int n, int* pvs, int32_t* gpiv, int lane) {
  for (int kk = 0; kk < n; ++kk) {
    long long key = -1;
    int idx = 0x7fffffff;
    for (int ii = kk + lane; ii < n; ii += 32) {
      const long long v = abs_key(a[ii * n + kk]);
      if (v > key) {
        key = v;
        idx = ii;
      }
    }
    for (int o = 16; o > 0; o >>= 1) {
      const long long ok = __shfl_xor_sync(0xffffffffu, key, o);
      const int oi = __shfl_xor_sync(0xffffffffu, idx, o);
      if (ok > key || (ok == key && oi < idx)) {
        key = ok;
        idx = oi;
      }
    }
    if (key <= 0) return false;
    const int pr = idx;
    if (lane == 0) {
      gpiv[kk] = pr;
      if (pvs) pvs[kk] = pr;
    }
    if (pr != kk)
      for (int jj = lane; jj < n; jj += 32) {
        const TL t = a[kk * n + jj];
        a[kk * n + jj] = a[pr * n + jj];
        a[pr * n + jj] = t;
      }
    __syncwarp();
    const TL d = a[kk * n + kk];
    const int w = n - kk - 1;
    for (int r = lane; r < w; r += 32) {
      TL* l = a + (kk + 1 + r) * n + kk;
      *l = div_rn<TL>(*l, d);
    }
    __syncwarp();
    for (int e = lane; e < w * w; e += 32) {
      const int r = e / w, c = e - r * w;
      const int ii = kk + 1 + r, jj = kk + 1 + c;
      a[ii * n + jj] = msub<TL>(a[ii * n + jj], a[ii * n + kk], a[kk * n + jj]);
    }
    __syncwarp();
  }
  return true;
}

// ||B^{-1}||_1 of a GEPP-factored FP32 block (n <= 32): lane c solves
// B x = e_c through the interchanges, L and U; the result is the largest
// column sum, on every lane.
__device__ float inv_norm1_f32(const float* a, int n, const int* pv, int lane) {
  float cs = 0.f;
  if (lane < n) {
    float x[32];
    for (int ii = 0; ii < n; ++ii) x[ii] = ii == lane ? 1.f : 0.f;
    for (int kk = 0; kk < n; ++kk) {
      const int pk = pv[kk];
      if (pk != kk) {
        const float t = x[kk];
        x[kk] = x[pk];
        x[pk] = t;
      }
    }
    for (int ii = 1; ii < n; ++ii) {
      float sum = x[ii];
      for (int kk = 0; kk < ii; ++kk) sum = __fmaf_rn(-a[ii * n + kk], x[kk], sum);
      x[ii] = sum;
    }
    for (int ii = n - 1; ii >= 0; --ii) {
      float sum = x[ii];
      for (int kk = ii + 1; kk < n; ++kk) sum = __fmaf_rn(-a[ii * n + kk], x[kk], sum);
      x[ii] = __fdiv_rn(sum, a[ii * n + ii]);
    }
    for (int ii = 0; ii < n; ++ii) cs += fabsf(x[ii]);
  }
  for (int o = 16; o > 0; o >>= 1) cs = fmaxf(cs, __shfl_xor_sync(0xffffffffu, cs, o));
  return cs;
}


template <typename T>
__global__ void __launch_bounds__(IW * 32, 2)
    k_ilut(VBView<T> A, Workspace ws, T* __restrict__ wvals_all, Pools P, T* __restrict__ lval,
           T* __restrict__ uval, const int64_t* __restrict__ dgoff, double* __restrict__ dg,
           float* __restrict__ dg32, int32_t* __restrict__ piv, int32_t* __restrict__ ptag, int mixed,
           double cond_thr, double t, int lfil, unsigned long long wait_limit, int* st) {
  extern __shared__ __align__(16) unsigned char ilut_sm[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  IlutWarp& W = reinterpret_cast<IlutWarp*>(ilut_sm)[warp];
  const int64_t wid = (int64_t)blockIdx.x * IW + warp;
  constexpr int USTAGE = USTAGE_BYTES / (int)sizeof(T);
  constexpr int VSH = WS_VBYTES / (int)sizeof(T);
  T* const ustage = reinterpret_cast<T*>(W.ustage);
  const float tf = (float)t, condf = (float)cond_thr;
  volatile int* vflag = &W.flag;
  volatile int* vns = &W.nslots;
  volatile int* vnl = &W.nl;
  int* const gkeys = ws.keys + wid * ws.ht;
  for (int k = lane; k < ws.ht; k += 32) gkeys[k] = -1;
  for (int k = lane; k < WS_HASH; k += 32) W.keys[k] = -1;
  __syncwarp();

  for (;;) {
    long long row = 0;
    if (lane == 0) {
      row = (long long)atomicAdd(P.ctr + 4, 1ULL);
      if (P.order && row < A.nbr) row = P.order[row];
    }
    row = __shfl_sync(0xffffffffu, row, 0);
    if (row >= A.nbr) break;
    const int64_t i = row;
    const int ni = A.rsz[i];
    const int64_t b0 = A.bptr[i], b1 = A.bptr[i + 1];
    const int64_t v0 = A.voff[b0], nv = A.voff[b1] - v0;
    const int nb = (int)(b1 - b0);
    // The working row lives in shared memory when it leaves room for fill; a
    // row whose fill outgrows that restarts in the warp's global workspace
    // (nothing of it is visible before its finish, so the restart is exact).
    bool in_sh = nb <= WS_SLOTS / 2 && nv <= VSH / 2;
    int status_local = 0;
    int* keys;
    int* hpos;
    int* scol;
    int* soff;
    int* sstate;
    long long* sf2;
    T* wv;
    int smax_c;
    int64_t vmax_c;
    uint32_t hmask;
    for (;;) {
      if (in_sh) {
        keys = W.keys, hpos = W.hpos, scol = W.scol, soff = W.soff, sstate = W.sstate, sf2 = W.sf2;
        wv = reinterpret_cast<T*>(W.vals);
        smax_c = WS_SLOTS, vmax_c = VSH, hmask = WS_HASH - 1;
      } else {
        keys = gkeys, hpos = ws.hpos + wid * ws.smax, scol = ws.scol + wid * ws.smax;
        soff = ws.soff + wid * ws.smax, sstate = ws.sstate + wid * ws.smax, sf2 = ws.sf2 + wid * ws.smax;
        wv = wvals_all + wid * ws.vmax;
        smax_c = ws.smax, vmax_c = ws.vmax, hmask = (uint32_t)ws.ht - 1;
      }
      if (lane == 0) {
        W.nslots = 0;
        W.nvals = 0;
        W.flag = 0;
        W.nl = 0;
      }
      __syncwarp();
      // ---- load row i of A into the workspace: slot q is the row's block q
      // and the values arrive as one contiguous copy; columns left of the
      // diagonal enter the list of pending L columns
      if (nb > smax_c || nv > vmax_c) {
        if (lane == 0) {
          *vflag = 1;
          atomicMax(P.ctr + 5, (unsigned long long)nv);
          atomicMax(P.ctr + 6, (unsigned long long)nb);
        }
      } else {
        for (int64_t b = b0 + lane; b < b1; b += 32) {
          const int slot = (int)(b - b0);
          const int32_t J = A.bcol[b];
          scol[slot] = J;
          soff[slot] = (int)(A.voff[b] - v0);
          sstate[slot] = SL_LIVE;
          hpos[slot] = ws_place(keys, hmask, slot, J);  // the table holds 2 smax positions
          if (J < i) {
            const int q = atomicAdd(&W.nl, 1);
            if (q < LCAP) {
              W.lc[q] = J;
              W.ls[q] = slot;
            }
          }
        }
        warp_copy(wv, A.val + v0, nv, lane);
        if (lane == 0) {
          W.nslots = nb;
          W.nvals = (unsigned long long)nv;
        }
      }
      __syncwarp();
      status_local = *vflag ? DEV_OVERFLOW : 0;
      int64_t last = -1;
      // ---- eliminate the L part in ascending column order (including fill)
      while (status_local == 0) {
        // next pending L column: from the list while it has not overflowed,
        // else by a scan of the workspace slots
        int best = 0x7fffffff, bslot = -1, bpos = -1;
        const int nlist = *vnl;
        if (nlist <= LCAP) {
          for (int q = lane; q < nlist; q += 32) {
            const int c = W.lc[q];
            if (c < best) {
              best = c;
              bslot = W.ls[q];
              bpos = q;
            }
          }
        } else {
          const int ns = min(*vns, smax_c);
          for (int sidx = lane; sidx < ns; sidx += 32) {
            const int c = scol[sidx];
            if (sstate[sidx] == SL_LIVE && c > last && c < i && c < best) {
              best = c;
              bslot = sidx;
            }
          }
        }
        const int kmin = warp_min_i(best);
        if (kmin == 0x7fffffff) break;
        const unsigned who = __ballot_sync(0xffffffffu, bslot >= 0 && best == kmin);
        const int owner = __ffs(who) - 1;
        const int sk = __shfl_sync(0xffffffffu, bslot, owner);
        if (lane == owner && bpos >= 0) W.lc[bpos] = 0x7fffffff;
        const int64_t k = kmin;
        last = k;
        // static data of row k: loaded before the wait, used after it
        const int nk = A.rsz[k];
        const int64_t dgk = dgoff[k];
        const int64_t rk = A.roff[k];
        // bounded wait until row k is published; a row that failed publishes
        // 2 (its factors must not be used)
        if (lane == 0 && wait_flag(P.done + k, P.abort, wait_limit, st) != 1) *vflag = 2;
        __syncwarp();
        if (*vflag == 2) {
          status_local = DEV_ETIMEOUT;
          break;
        }
        T* m = wv + soff[sk];
        // the pivot block of k goes to shared memory: its own buffer when
        // small, else the free tail of the value buffer (new slots are only
        // created after the multiplier), sized for FP64
        unsigned char* lus = nullptr;
        if (nk <= SMB) {
          lus = W.lu;
        } else if (nk <= PVMAX) {
          const long long used = in_sh ? ((long long)W.nvals * (long long)sizeof(T) + 15) / 16 * 16 : 0;
          if (used + (long long)nk * nk * (long long)sizeof(double) <= WS_VBYTES) lus = W.vals + used;
        }
        const bool staged = lus != nullptr;
        double* const luD = reinterpret_cast<double*>(lus);
        float* const luF = reinterpret_cast<float*>(lus);
        // round A: the precision tag and the extent of U row k (lanes 0-4),
        // the pivot block of k and its pivots
        long long hv = 0;
        if (lane == 0)
          hv = ptag ? __ldcg(ptag + k) : 1;
        else if (lane == 1)
          hv = __ldcg(P.ustart + k);
        else if (lane == 2)
          hv = __ldcg(P.ucnt + k);
        else if (lane == 3)
          hv = __ldcg(P.uvstart + k);
        else if (lane == 4)
          hv = __ldcg(P.uvlen + k);
        if (staged && nk <= SMB) {  // every load issued before the first store
          constexpr int LV = SMB * SMB / 32;
          using TS = typename std::conditional<sizeof(T) == sizeof(double), double, float>::type;
          const TS* src = sizeof(T) == sizeof(double) ? reinterpret_cast<const TS*>(dg) : reinterpret_cast<const TS*>(dg32);
          TS* dstl = reinterpret_cast<TS*>(lus);
          TS lv[LV];
#pragma unroll
          for (int u = 0; u < LV; ++u) {
            const int e = lane + 32 * u;
            lv[u] = e < nk * nk ? __ldcg(src + dgk + e) : (TS)0;
          }
          const int pvv = lane < nk ? __ldcg(piv + rk + lane) : 0;
#pragma unroll
          for (int u = 0; u < LV; ++u) {
            const int e = lane + 32 * u;
            if (e < nk * nk) dstl[e] = lv[u];
          }
          if (lane < nk) W.pv[lane] = pvv;
        } else if (staged) {
          if (sizeof(T) == sizeof(double))
            for (int e = lane; e < nk * nk; e += 32) luD[e] = __ldcg(dg + dgk + e);
          else
            for (int e = lane; e < nk * nk; e += 32) luF[e] = __ldcg(dg32 + dgk + e);
          if (lane < nk) W.pv[lane] = __ldcg(piv + rk + lane);
        }
        const int tag = (int)__shfl_sync(0xffffffffu, hv, 0);
        const int64_t u0 = __shfl_sync(0xffffffffu, hv, 1);
        const int uc = (int)__shfl_sync(0xffffffffu, hv, 2);
        const int64_t uvs = __shfl_sync(0xffffffffu, hv, 3);
        const int64_t uvl = __shfl_sync(0xffffffffu, hv, 4);
        if (u0 < 0 || uc < 0 || u0 + uc > P.ubcap || uvs < 0 || uvl < 0 || uvs + uvl > P.uvcap) {
          status_local = DEV_INTERNAL;  // never true for a published row: record and skip
          break;
        }
        // round B, in flight during the multiplier: U row k into shared memory
        // (16-byte asynchronous copies; U rows start 16-byte aligned in the
        // pool and their padding is reserved) and the columns and offsets of
        // its first 32 blocks
        const bool ust = uvl <= USTAGE && ((uvs * (int64_t)sizeof(T)) & 15) == 0;
        if (ust) {
          const int nch = (int)((uvl * (int64_t)sizeof(T) + 15) / 16);
          const unsigned char* src = reinterpret_cast<const unsigned char*>(uval + uvs);
          for (int c = lane; c < nch; c += 32) cp_async16(W.ustage + 16 * c, src + 16 * c);
        }
        int32_t pj = -1;
        int64_t puo = 0;
        if (lane < uc) {
          pj = __ldcg(P.ucol + u0 + lane);
          puo = __ldcg(P.uvo + u0 + lane);
        }
        const bool use64 = sizeof(T) == sizeof(double) || tag != 0;
        if (staged && use64 && sizeof(T) != sizeof(double))  // an FP64 pivot block of the mixed factor
          for (int e = lane; e < nk * nk; e += 32) luD[e] = __ldcg(dg + dgk + e);
        __syncwarp();
        // the multiplier m = a_ik (P^T L U)_k^{-1}, in place, one lane per row
        if (staged) {
          for (int a = lane; a < ni; a += 32) {
            if (use64)
              ainv_right_row_sh<T, double>(luD, W.pv, nk, m + a * nk);
            else
              ainv_right_row_sh<T, float>(luF, W.pv, nk, m + a * nk);
          }
        } else {
          for (int a = lane; a < ni; a += 32) {
            if (use64)
              ainv_right_row<T, double>(dg + dgk, piv + rk, nk, m + a * nk);
            else
              ainv_right_row<T, float>(dg32 + dgk, piv + rk, nk, m + a * nk);
          }
        }
        __syncwarp();
        long long key = 0;
        bool dropped;
        if (sizeof(T) == sizeof(double)) {  // the oracle's summation order
          double f2 = 0.0;
          if (lane == 0) f2 = fro2_seq(m, ni * nk);
          f2 = __shfl_sync(0xffffffffu, f2, 0);
          dropped = drop_rule(f2, ni, nk, t);
          key = norm_key(f2);
        } else {  // mixed factor: FP32 squares summed by a warp reduction
          float sf = 0.f;
          for (int e = lane; e < ni * nk; e += 32) {
            const float x = (float)m[e];
            sf = __fmaf_rn(x, x, sf);
          }
          for (int o = 16; o > 0; o >>= 1) sf += __shfl_xor_sync(0xffffffffu, sf, o);
          dropped = drop_rule_f(sf, ni, nk, tf);
          key = norm_key(sf);
        }
        if (ust) cp_async_wait_all();
        if (dropped) {
          if (lane == 0) sstate[sk] = SL_DEAD;
          __syncwarp();
          continue;
        }
        if (lane == 0) {
          sstate[sk] = SL_LKEPT;
          sf2[sk] = key;
        }
        __syncwarp();
        // U row k in chunks of 32 blocks: look up or create the target blocks
        // (probe, then place, separated by __syncwarp), then update all
        // elements of the chunk with lanes spread over the flattened elements.
        for (int q0 = 0; q0 < uc && status_local == 0; q0 += 32) {
          const int q = q0 + lane;
          int32_t j = -1;
          int slot = -1;
          int64_t uo = 0;
          bool missing = false;
          if (q < uc) {
            if (q0 == 0) {
              j = pj;
              uo = puo;
            } else {
              j = __ldcg(P.ucol + u0 + q);
              uo = __ldcg(P.uvo + u0 + q);
            }
            if (j <= k || j >= A.nbr || uo < uvs || uo + (int64_t)nk * A.rsz[j] > uvs + uvl) {
              *vflag = 4;  // a published U block lies right of k inside its row's extent
              j = -1;
            } else {
              slot = ws_lookup(keys, scol, hmask, j);
              missing = slot < 0;
            }
          }
          __syncwarp();
          if (missing) {
            const int sz = ni * A.rsz[j];
            slot = ws_new_slot(smax_c, vmax_c, keys, hpos, scol, soff, sstate, &W.nslots, &W.nvals, hmask, j, sz);
            if (slot < 0) {
              *vflag = 1;
            } else {
              T* z = wv + soff[slot];
#pragma unroll 4
              for (int e = 0; e < sz; ++e) z[e] = (T)0;
              if (j < i) {  // fill in the L part: pending for a later step
                const int pq = atomicAdd(&W.nl, 1);
                if (pq < LCAP) {
                  W.lc[pq] = j;
                  W.ls[pq] = slot;
                }
              }
            }
          }
          __syncwarp();
          if (*vflag == 1) {
            status_local = DEV_OVERFLOW;
            break;
          }
          if (*vflag == 4) {
            status_local = DEV_INTERNAL;
            break;
          }
          const int nj = j >= 0 ? A.rsz[j] : 0;
          const int sz = ni * nj;
          int incl = sz;
          for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
          }
          const int total = __shfl_sync(0xffffffffu, incl, 31);
          W.qpre[lane] = incl - sz;
          if (lane == 31) W.qpre[32] = total;
          W.qoff[lane] = slot >= 0 ? soff[slot] : 0;
          W.quo[lane] = (int)(uo - uvs);
          W.qnj[lane] = nj;
          __syncwarp();
          const int nq = min(32, uc - q0);
          const T* Ubase = ust ? ustage : uval + uvs;
          // four elements per lane in flight
          for (int e0 = lane; e0 < total; e0 += 128) {
            T acc[4];
            T* dst[4];
            int a4[4], jj4[4], nj4[4], uo4[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const int e = e0 + 32 * u;
              dst[u] = nullptr;
              if (e < total) {
                int lo = 0, hi = nq - 1;  // block tq with qpre[tq] <= e < qpre[tq + 1]
                while (lo < hi) {
                  const int mid = (lo + hi + 1) >> 1;
                  if (W.qpre[mid] <= e)
                    lo = mid;
                  else
                    hi = mid - 1;
                }
                const int njt = W.qnj[lo];
                const int local = e - W.qpre[lo];
                a4[u] = local / njt;
                jj4[u] = local - a4[u] * njt;
                nj4[u] = njt;
                uo4[u] = W.quo[lo];
                dst[u] = wv + W.qoff[lo] + local;
                acc[u] = *dst[u];
              }
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              if (!dst[u]) continue;
              const T* U = Ubase + uo4[u];
              T av = acc[u];
              if (ust) {
                for (int r = 0; r < nk; ++r) av = msub<T>(av, m[a4[u] * nk + r], U[r * nj4[u] + jj4[u]]);
              } else {
                for (int r = 0; r < nk; ++r) av = msub<T>(av, m[a4[u] * nk + r], __ldcg(U + r * nj4[u] + jj4[u]));
              }
              *dst[u] = av;
            }
          }
          __syncwarp();
        }
      }
      if (status_local == DEV_OVERFLOW && in_sh) {
        // the fill outgrew the shared workspace: start the row again in the
        // global one
        for (int q = lane; q < WS_HASH; q += 32) W.keys[q] = -1;
        __syncwarp();
        in_sh = false;
        continue;
      }
      break;
    }
    const int ns = min(*vns, smax_c);
    // ---- finish the row.  A row in the global workspace has its slot
    // metadata staged in shared memory (the U-row stage buffer is free now)
    // so that the scans below read on-chip data; rows with more than MSH
    // slots read the workspace directly.
    int* mcol = reinterpret_cast<int*>(W.ustage);
    int* mst = mcol + MSH;
    int* moff = mst + MSH;
    long long* mf2 = reinterpret_cast<long long*>(moff + MSH);
    const bool msh = !in_sh && ns <= MSH;
    if (msh)
      for (int q = lane; q < ns; q += 32) {
        mcol[q] = scol[q];
        mst[q] = sstate[q];
        moff[q] = soff[q];
        mf2[q] = sf2[q];
      }
    __syncwarp();
    auto COL = [&](int q) { return msh ? mcol[q] : scol[q]; };
    auto ST = [&](int q) { return msh ? mst[q] : sstate[q]; };
    auto OFF = [&](int q) { return msh ? moff[q] : soff[q]; };
    auto F2 = [&](int q) { return msh ? mf2[q] : sf2[q]; };
    auto IS_L = [&](int q) { return ST(q) == SL_LKEPT; };
    auto IS_U = [&](int q) { return ST(q) == SL_LIVE && COL(q) > i; };
    int dslot = -1;
    if (status_local == 0) {
      for (int q = lane; q < ns; q += 32)
        if (COL(q) == i && ST(q) == SL_LIVE) dslot = q;
      dslot = warp_max_i(dslot);
      if (dslot < 0) status_local = DEV_ESINGULAR;
    }
    bool fits = false;
    unsigned long long lb = 0, lvv = 0, ub = 0, uvv = 0;
    int nl = 0, nu = 0;
    long long vl = 0, vu = 0;
    if (status_local == 0) {
      // U part: threshold on the blocks right of the diagonal
      for (int q = lane; q < ns; q += 32) {
        const int c = COL(q);
        if (ST(q) == SL_LIVE && c > i) {
          const int nc = A.rsz[c];
          bool drop;
          long long key;
          if (sizeof(T) == sizeof(double)) {
            const double f2 = fro2_batched(wv + OFF(q), ni * nc);
            drop = drop_rule(f2, ni, nc, t);
            key = norm_key(f2);
          } else {
            const float f2 = fro2_f32(wv + OFF(q), ni * nc);
            drop = drop_rule_f(f2, ni, nc, tf);
            key = norm_key(f2);
          }
          if (msh) mf2[q] = key; else sf2[q] = key;
          if (drop) {
            if (msh) mst[q] = SL_DEAD; else sstate[q] = SL_DEAD;
          }
        }
      }
      __syncwarp();
      // lfil: keep the lfil largest of the L part and of the U part (rank by
      // (norm desc, column asc); ranks computed before any state changes)
      if (lfil >= 0) {
        unsigned cutmask[MAX_SLOTS / 1024] = {};  // bit tq: slot lane + 32 tq is cut
        for (int tq = 0; tq * 32 < ns && tq < MAX_SLOTS / 32; ++tq) {
          const int q = tq * 32 + lane;
          if (q >= ns) continue;
          const bool isL = IS_L(q), isU = IS_U(q);
          if (!isL && !isU) continue;
          const long long fq = F2(q);
          const int cq = COL(q);
          int rank = 0;
          for (int r2 = 0; r2 < ns; ++r2) {
            const bool same = isL ? IS_L(r2) : IS_U(r2);
            if (same) {
              const long long fr = F2(r2);
              if (fr > fq || (fr == fq && COL(r2) < cq)) ++rank;
            }
          }
          if (rank >= lfil) cutmask[tq >> 5] |= 1u << (tq & 31);
        }
        __syncwarp();
        for (int tq = 0; tq < MAX_SLOTS / 32; ++tq)
          if (cutmask[tq >> 5] & (1u << (tq & 31))) {
            const int q = tq * 32 + lane;
            if (msh) mst[q] = SL_DEAD; else sstate[q] = SL_DEAD;
          }
        __syncwarp();
      }
      for (int q = lane; q < ns; q += 32) {
        const int c = COL(q);
        if (IS_L(q)) {
          ++nl;
          vl += (long long)ni * A.rsz[c];
        } else if (IS_U(q)) {
          ++nu;
          vu += (long long)ni * A.rsz[c];
        }
      }
      nl = warp_sum_i(nl);
      nu = warp_sum_i(nu);
      vl = warp_sum_ll(vl);
      vu = warp_sum_ll(vu);
      // U rows are reserved in whole 16-byte units so that every row starts
      // 16-byte aligned (the readers stage them with 16-byte copies)
      constexpr long long UQ = 16 / (long long)sizeof(T);
      const long long vu_pad = (vu + UQ - 1) / UQ * UQ;
      if (lane == 0) {
        lb = atomicAdd(P.ctr + 0, (unsigned long long)nl);
        lvv = atomicAdd(P.ctr + 1, (unsigned long long)vl);
        ub = atomicAdd(P.ctr + 2, (unsigned long long)nu);
        uvv = atomicAdd(P.ctr + 3, (unsigned long long)vu_pad);
      }
      lb = __shfl_sync(0xffffffffu, lb, 0);
      lvv = __shfl_sync(0xffffffffu, lvv, 0);
      ub = __shfl_sync(0xffffffffu, ub, 0);
      uvv = __shfl_sync(0xffffffffu, uvv, 0);
      fits = (int64_t)(lb + nl) <= P.lbcap && (int64_t)(lvv + vl) <= P.lvcap && (int64_t)(ub + nu) <= P.ubcap &&
             (int64_t)(uvv + vu_pad) <= P.uvcap;
      if (!fits) status_local = DEV_OVERFLOW;
      if (status_local == 0) {
        // GEPP of the diagonal block, in shared memory when it fits.  FP64
        // factor: FP64 in the oracle's operation order.  Mixed factor: FP32
        // GEPP and 1-norm condition estimate (explicit inverse columns); a
        // block above the threshold, larger than 32, or singular in FP32 is
        // factored again in FP64 and tagged.
        const T* srcd = wv + OFF(dslot);
        // staging: the small-block buffer, else the U-row buffer (free now)
        // of a shared working row or the value buffer of a global one
        unsigned char* gb = nullptr;
        int gcap = 0;
        if (ni <= SMB) {
          gb = W.lu, gcap = (int)sizeof(W.lu);
        } else if (ni <= PVMAX) {
          if (in_sh)
            gb = W.ustage, gcap = USTAGE_BYTES;
          else
            gb = W.vals, gcap = WS_VBYTES;
        }
        const bool gs32 = gb && ni * ni * 4 <= gcap, gs64 = gb && ni * ni * 8 <= gcap;
        int* pvs = gb ? W.pv : nullptr;
        int32_t* gpiv = piv + A.roff[i];
        bool ok = true, tag64 = true;
        if (sizeof(T) == sizeof(float)) {
          const bool gsh = gs32;
          float* a = gsh ? reinterpret_cast<float*>(gb) : dg32 + dgoff[i];
          for (int e = lane; e < ni * ni; e += 32) a[e] = (float)srcd[e];
          __syncwarp();
          float norm1 = 0.f;
          for (int jj = lane; jj < ni; jj += 32) {
            float sum = 0.f;
            for (int ii = 0; ii < ni; ++ii) sum += fabsf(a[ii * ni + jj]);
            norm1 = fmaxf(norm1, sum);
          }
          for (int o = 16; o > 0; o >>= 1) norm1 = fmaxf(norm1, __shfl_xor_sync(0xffffffffu, norm1, o));
          __syncwarp();
          if (ni <= 32 && gepp_warp<float>(a, ni, pvs, gpiv, lane)) {
            const float kappa = norm1 * inv_norm1_f32(a, ni, pvs ? pvs : gpiv, lane);
            tag64 = !(kappa <= condf);
            if (!tag64) {
              for (int e = lane; e < ni * ni; e += 32) {
                if (gsh) dg32[dgoff[i] + e] = a[e];
                dg[dgoff[i] + e] = (double)a[e];
              }
            }
          }
          __syncwarp();
        }
        if (tag64) {
          const bool gsh = gs64;
          double* a = gsh ? reinterpret_cast<double*>(gb) : dg + dgoff[i];
          for (int e = lane; e < ni * ni; e += 32) a[e] = (double)srcd[e];
          __syncwarp();
          ok = gepp_warp<double>(a, ni, pvs, gpiv, lane);
          if (ok)
            for (int e = lane; e < ni * ni; e += 32) {
              if (gsh) dg[dgoff[i] + e] = a[e];
              if (mixed) dg32[dgoff[i] + e] = (float)a[e];
            }
        }
        if (!ok)
          status_local = DEV_ESINGULAR;
        else if (mixed && lane == 0)
          ptag[i] = tag64 ? 1 : 0;
      }
    }
    // Write the kept blocks of one part in column order: per chunk of 32
    // slots the ranks come from the staged metadata, then the chunk's values
    // are copied with lanes over the flattened elements, eight loads in
    // flight per lane.
    auto write_part = [&](bool isL, unsigned long long bstart, unsigned long long vstart, int32_t* pcol,
                          int64_t* pvo, T* pval) {
      for (int s0 = 0; s0 < ns; s0 += 32) {
        const int q = s0 + lane;
        int sz = 0;
        int64_t src = 0, dstv = 0;
        if (q < ns && (isL ? IS_L(q) : IS_U(q))) {
          const int c = COL(q);
          int rank = 0;
          long long vo = 0;
          for (int r2 = 0; r2 < ns; ++r2) {
            const int cr = COL(r2);
            if (cr < c && (isL ? IS_L(r2) : IS_U(r2))) {
              ++rank;
              vo += (long long)ni * A.rsz[cr];
            }
          }
          sz = ni * A.rsz[c];
          src = OFF(q);
          dstv = (int64_t)vstart + vo;
          pcol[bstart + rank] = c;
          pvo[bstart + rank] = dstv;
        }
        int incl = sz;
        for (int o = 1; o < 32; o <<= 1) {
          const int v = __shfl_up_sync(0xffffffffu, incl, o);
          if (lane >= o) incl += v;
        }
        const int total = __shfl_sync(0xffffffffu, incl, 31);
        W.qpre[lane] = incl - sz;
        W.qoff[lane] = (int)src;
        W.wdst[lane] = dstv;
        __syncwarp();
        for (int e0 = lane; e0 < total; e0 += 32 * 8) {
          T v[8];
          int64_t d8[8];
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            const int e = e0 + 32 * u;
            d8[u] = -1;
            if (e < total) {
              int lo = 0, hi = 31;
              while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (W.qpre[mid] <= e)
                  lo = mid;
                else
                  hi = mid - 1;
              }
              // skip empty entries that share the same prefix
              while (lo < 31 && W.qpre[lo + 1] <= e) ++lo;
              const int local = e - W.qpre[lo];
              v[u] = wv[W.qoff[lo] + local];
              d8[u] = W.wdst[lo] + local;
            }
          }
#pragma unroll
          for (int u = 0; u < 8; ++u)
            if (d8[u] >= 0) pval[d8[u]] = v[u];
        }
        __syncwarp();
      }
    };
    if (status_local == 0) {
      write_part(false, ub, uvv, P.ucol, P.uvo, uval);
      if (lane == 0) {
        P.ustart[i] = (int64_t)ub;
        P.ucnt[i] = nu;
        P.uvstart[i] = (int64_t)uvv;
        P.uvlen[i] = (int64_t)vu;
      }
    }
    if (status_local != 0 && lane == 0) {
      dev_fail(st, status_local);
      atomicExch(P.abort, 1);
      P.lcnt[i] = 0;
      P.ucnt[i] = 0;
      P.lstart[i] = 0;
      P.ustart[i] = 0;
      P.uvstart[i] = 0;
      P.uvlen[i] = 0;
    }
    if (lane == 0) {  // what the row asked for, to size a retry
      atomicMax(P.ctr + 5, W.nvals);
      atomicMax(P.ctr + 6, (unsigned long long)W.nslots);
    }
    // publish the row (its U part and pivot block): every lane's writes are
    // made visible device-wide before lane 0 raises the flag
    __threadfence();
    __syncwarp();
    if (lane == 0) atomicExch(&P.done[i], status_local == 0 ? 1 : 2);
    // the L part is read by no other row: written after publishing
    if (status_local == 0) {
      write_part(true, lb, lvv, P.lcol, P.lvo, lval);
      if (lane == 0) {
        P.lstart[i] = (int64_t)lb;
        P.lcnt[i] = nl;
      }
    }
    // clear the hash positions this row used
    if (in_sh) {
      for (int q = lane; q < WS_HASH; q += 32) W.keys[q] = -1;
    } else {
      for (int q = lane; q < ns; q += 32)
        if (hpos[q] >= 0) keys[hpos[q]] = -1;
    }
    __syncwarp();
  }
}

// Gather the pooled rows into VBCSR (warp per row).
template <typename T>
__global__ void k_pool_to_vb(int64_t nbr, const int64_t* __restrict__ start, const int32_t* __restrict__ pcol,
                             const int64_t* __restrict__ pvo, const T* __restrict__ pval,
                             const int64_t* __restrict__ bptr, const int64_t* __restrict__ voff,
                             int32_t* __restrict__ bcol, T* __restrict__ val) {
  const int lane = threadIdx.x & 31;
  const int64_t wpb = blockDim.x >> 5;
  for (int64_t i = blockIdx.x * wpb + (threadIdx.x >> 5); i < nbr; i += (int64_t)gridDim.x * wpb) {
    const int64_t n = bptr[i + 1] - bptr[i];
    if (!voff) {  // first pass: columns only (the value offsets do not exist yet)
      for (int64_t q = lane; q < n; q += 32) bcol[bptr[i] + q] = pcol[start[i] + q];
      continue;
    }
    for (int64_t q = 0; q < n; ++q) {
      const int64_t d = bptr[i] + q;
      const int64_t sz = voff[d + 1] - voff[d];
      const int64_t src = pvo[start[i] + q];
      for (int64_t e = lane; e < sz; e += 32) val[voff[d] + e] = pval[src + e];
    }
  }
}

__global__ void k_sq_sizes(int64_t n, const int32_t* __restrict__ sz, int64_t* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (int64_t)sz[i] * sz[i];
}

__global__ void k_count_to_i64(int64_t n, const int32_t* __restrict__ c, int64_t* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = c[i];
}

__global__ void k_iota(int64_t n, int64_t* __restrict__ bptr, int32_t* __restrict__ bcol) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i <= n; i += (int64_t)gridDim.x * blockDim.x) {
    bptr[i] = i;
    if (i < n) bcol[i] = (int32_t)i;
  }
}

}  // namespace

template <typename T>
void ilut_last(LastDev<T>& X, double t, int lfil, bool mixed, double cond_thr, uint64_t wait_limit, cudaStream_t s,
               int* dst, const int32_t* order) {
  const VBDev<T>& A = X.A;
  const int64_t p = A.nbr;
  const int64_t n = p ? d2h(A.roff.p + p, s) : 0;
  // pivot blocks: block diagonal structure
  set_partitions(X.Dg, A.rsz.p, p, A.rsz.p, p, s);
  X.Dg.bptr.alloc(p + 1, s);
  X.Dg.bcol.alloc(p, s);
  launch(k_iota, grid_for(p + 1, 256), 256, 0, s, p, X.Dg.bptr.p, X.Dg.bcol.p);
  VB_LAUNCH_CHECK();
  X.Dg.nnzb = p;
  X.Dg.voff.alloc(p + 1, s);
  {
    DBuf<int64_t> sq(p, s);
    if (p) {
      launch(k_sq_sizes, grid_for(p, 256), 256, 0, s, p, A.rsz.p, sq.p);
      VB_LAUNCH_CHECK();
    }
    scan_i64(sq.p, X.Dg.voff.p, p, s);
  }
  X.Dg.nval = p ? d2h(X.Dg.voff.p + p, s) : 0;
  X.Dg.val.alloc(X.Dg.nval, s);
  X.piv.alloc(n, s);
  X.ptag.alloc(p, s);
  X.ptag.zero();
  if (mixed) copy_vb<float, double>(X.Dg, X.Dg32, s);
  set_partitions(X.L, A.rsz.p, p, A.rsz.p, p, s);
  set_partitions(X.U, A.rsz.p, p, A.rsz.p, p, s);
  if (p == 0) {
    X.L.bptr.alloc(1, s);
    X.L.bptr.zero();
    X.U.bptr.alloc(1, s);
    X.U.bptr.zero();
    X.L.voff.alloc(1, s);
    X.L.voff.zero();
    X.U.voff.alloc(1, s);
    X.U.voff.zero();
    return;
  }

  int dev = 0;
  VB_CUDA(cudaGetDevice(&dev));
  int nsm = 0;
  VB_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  // L and U each hold about half of the last-level matrix on the configured
  // workloads; the pools start at its full size and grow on overflow (retry)
  int64_t lbcap = std::max<int64_t>(A.nnzb, 1024), lvcap = std::max<int64_t>(A.nval, 1 << 16);
  int64_t ubcap = lbcap, uvcap = lvcap + 4 * p;  // U rows are padded to 16 bytes
  int smax = 1024;
  int64_t vmax = 32768;
  const int blocks_per_sm = 2;  // two blocks of IW warps share the shared memory of an SM
  for (int attempt = 0; attempt < 6; ++attempt) {
    const int64_t nblocks = std::max<int64_t>(1, std::min<int64_t>((int64_t)nsm * blocks_per_sm, (p + IW - 1) / IW));
    const int64_t nwarps = nblocks * IW;
    int ht = 1;
    while (ht < 2 * smax) ht <<= 1;
    DBuf<int> keys(nwarps * ht, s), hpos(nwarps * smax, s), scol(nwarps * smax, s), sstate(nwarps * smax, s);
    DBuf<int> soff(nwarps * smax, s);
    DBuf<long long> sf2(nwarps * smax, s);
    DBuf<T> wvals(nwarps * vmax, s);
    Workspace ws{keys.p, hpos.p, scol.p, soff.p, sstate.p, sf2.p, ht, smax, vmax};
    DBuf<int32_t> lcol(lbcap, s), ucol(ubcap, s), lcnt(p, s), ucnt(p, s), done(p, s);
    DBuf<int64_t> lvo(lbcap, s), uvo(ubcap, s), lstart(p, s), ustart(p, s), uvstart(p, s), uvlen(p, s);
    DBuf<T> lval(lvcap, s), uval(uvcap, s);
    DBuf<unsigned long long> ctr(8, s);
    DBuf<int> abort(1, s);
    ctr.zero();
    done.zero();
    abort.zero();
    X.piv.zero();
    Pools P{lcol.p, lvo.p,  ucol.p, uvo.p,  lstart.p, lcnt.p,  ustart.p,  ucnt.p,   ctr.p,
            lbcap,  lvcap,  ubcap,  uvcap,  done.p,   abort.p, uvstart.p, uvlen.p, order};
    VB_CUDA(cudaFuncSetAttribute(k_ilut<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ilut_smem()));
    launch(k_ilut<T>, (unsigned)nblocks, IW * 32, ilut_smem(), s, A.view(), ws, wvals.p, P, lval.p, uval.p,
           X.Dg.voff.p,
                                                     X.Dg.val.p, mixed ? X.Dg32.val.p : nullptr, X.piv.p,
                                                     mixed ? X.ptag.p : nullptr, mixed ? 1 : 0, cond_thr, t, lfil,
                                                     (unsigned long long)wait_limit, dst);
    VB_LAUNCH_CHECK();
    const int st = d2h(dst, s);
    if (st == DEV_OVERFLOW) {
      VB_CUDA(cudaMemsetAsync(dst, 0, sizeof(int), s));
      std::vector<unsigned long long> c = d2h_vec(ctr.p, 8, s);
      lbcap = std::max<int64_t>(2 * lbcap, (int64_t)c[0] + 1024);
      lvcap = std::max<int64_t>(2 * lvcap, (int64_t)c[1] + 4096);
      ubcap = std::max<int64_t>(2 * ubcap, (int64_t)c[2] + 1024);
      uvcap = std::max<int64_t>(2 * uvcap, (int64_t)c[3] + 4096);
      while ((int64_t)c[5] > vmax) vmax *= 2;
      if ((int64_t)c[6] > smax) {
        while (smax < (int)c[6] && smax < MAX_SLOTS) smax *= 2;
        if ((int64_t)c[6] > MAX_SLOTS) fail(VB_ENOMEM, "last-level ILUT: a working row exceeds 4096 blocks");
      }
      continue;
    }
    check_status(dst, s, "vbarms_factor: last-level block ILUT");
    // assemble L and U
    for (int which = 0; which < 2; ++which) {
      VBDev<T>& M = which == 0 ? X.L : X.U;
      DBuf<int32_t>& cnt = which == 0 ? lcnt : ucnt;
      DBuf<int64_t>& start = which == 0 ? lstart : ustart;
      DBuf<int32_t>& pcol = which == 0 ? lcol : ucol;
      DBuf<int64_t>& pvo = which == 0 ? lvo : uvo;
      DBuf<T>& pval = which == 0 ? lval : uval;
      M.bptr.alloc(p + 1, s);
      DBuf<int64_t> c64(p, s);
      launch(k_count_to_i64, grid_for(p, 256), 256, 0, s, p, cnt.p, c64.p);
      VB_LAUNCH_CHECK();
      scan_i64(c64.p, M.bptr.p, p, s);
      M.nnzb = d2h(M.bptr.p + p, s);
      M.bcol.alloc(M.nnzb, s);
      // bcol first (needed by the offsets), then offsets, then values
      launch(k_pool_to_vb<T>, grid_for(p, 8), 256, 0, s, p, start.p, pcol.p, pvo.p, pval.p, M.bptr.p, nullptr,
                                                       M.bcol.p, nullptr);
      VB_LAUNCH_CHECK();
      finish_offsets(M, s);
      launch(k_pool_to_vb<T>, grid_for(p, 8), 256, 0, s, p, start.p, pcol.p, pvo.p, pval.p, M.bptr.p, M.voff.p,
                                                       M.bcol.p, M.val.p);
      VB_LAUNCH_CHECK();
    }
    return;
  }
  fail(VB_ENOMEM, "vbarms_factor: last-level ILUT workspace could not be sized");
}

namespace {
__global__ void k_dom_start(int64_t p, int ndom, const int32_t* __restrict__ dom, int64_t* __restrict__ start) {
  for (int d = blockIdx.x * blockDim.x + threadIdx.x; d <= ndom; d += gridDim.x * blockDim.x) {
    int64_t lo = 0, hi = p;  // first row with dom >= d
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      if (dom[mid] < d)
        lo = mid + 1;
      else
        hi = mid;
    }
    start[d] = lo;
  }
}

// Row r, the j-th of block d, goes to position
//   sum_{d'} min(len_d', j) + #{d' < d : len_d' > j},
// its place when the blocks' rows are dealt out one per block in turn.
__global__ void k_ticket_pos(int64_t p, int ndom, const int32_t* __restrict__ dom, const int64_t* __restrict__ start,
                             int32_t* __restrict__ order) {
  extern __shared__ int64_t lens[];
  for (int d = threadIdx.x; d < ndom; d += blockDim.x) lens[d] = start[d + 1] - start[d];
  __syncthreads();
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < p; r += (int64_t)gridDim.x * blockDim.x) {
    const int d = dom[r];
    const int64_t j = r - start[d];
    int64_t pos = 0;
    for (int e = 0; e < ndom; ++e) {
      const int64_t le = lens[e];
      pos += le < j ? le : j;
      if (e < d && le > j) ++pos;
    }
    order[pos] = (int32_t)r;
  }
}

__global__ void k_take_i32(int64_t n, const int32_t* __restrict__ src, const int32_t* __restrict__ idx,
                           int32_t* __restrict__ dst) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
    dst[k] = src[idx[k]];
}
}  // namespace

void ticket_order(const int32_t* dom, int64_t p, int ndom, DBuf<int32_t>& order, cudaStream_t s) {
  if (p == 0 || ndom <= 1 || ndom > kTicketMaxDom) {
    order = DBuf<int32_t>();
    return;
  }
  DBuf<int64_t> start(ndom + 1, s);
  launch(k_dom_start, grid_for(ndom + 1, 256), 256, 0, s, p, ndom, dom, start.p);
  VB_LAUNCH_CHECK();
  order.alloc(p, s);
  launch(k_ticket_pos, grid_for(p, 256), 256, (size_t)ndom * sizeof(int64_t), s, p, ndom, dom, start.p, order.p);
  VB_LAUNCH_CHECK();
}

void take_i32(const int32_t* src, const int32_t* idx, int64_t n, int32_t* dst, cudaStream_t s) {
  if (n == 0) return;
  launch(k_take_i32, grid_for(n, 256), 256, 0, s, n, src, idx, dst);
  VB_LAUNCH_CHECK();
}

template void ilut_last<double>(LastDev<double>&, double, int, bool, double, uint64_t, cudaStream_t, int*,
                                 const int32_t*);
template void ilut_last<float>(LastDev<float>&, double, int, bool, double, uint64_t, cudaStream_t, int*,
                                const int32_t*);

}  // namespace vb

namespace vb {

namespace {

// Level of every row in the dependency DAG of a triangular block pattern:
// lev[i] = 1 + max lev[k] over the row's block columns k (0 without
// blocks).  Warps of a persistent grid take the rows in dependency order
// (forward, for L: ascending, every column below the row; backward, for U:
// descending, every column above) and spin, bounded, on the columns' words:
// a row publishes lev + 1 (-1 when it failed) in its word with one atomic
// store, so the word is both flag and value and needs no fence.  The first
// half of the grid does L, the second U, at the same time.
struct DagSide {
  int64_t p;
  const int64_t* bptr;
  const int32_t* bcol;
  int32_t* word;  // 0 until published, then lev + 1 (or -1)
  unsigned long long* tick;
  int* depth;
};

// The published word, or 0 when the wait gave up (abort raised elsewhere, or
// limit ns passed: DEV_ETIMEOUT recorded and abort raised).
__device__ __forceinline__ int dag_wait(const int32_t* w, int* abort, unsigned long long limit, int* st) {
  int v = ld_relaxed_gpu(w);
  if (v == 0) {
    const unsigned long long t0 = global_ns();
    for (unsigned it = 1;; ++it) {
      v = ld_relaxed_gpu(w);
      if (v != 0) break;
      if ((it & 63) == 0) {
        if (*((volatile int*)abort) != 0) return 0;
        if (global_ns() - t0 > limit) {
          dev_fail(st, DEV_ETIMEOUT);
          atomicExch(abort, 1);
          return 0;
        }
      }
    }
  }
  return v;
}

__global__ void k_dag_level(DagSide fw, DagSide bw, unsigned half, int* __restrict__ abort, unsigned long long limit,
                            int* st) {
  const bool back = blockIdx.x >= half;
  const DagSide D = back ? bw : fw;
  const int lane = threadIdx.x & 31;
  for (;;) {
    long long t = 0;
    if (lane == 0) t = (long long)atomicAdd(D.tick, 1ULL);
    t = __shfl_sync(0xffffffffu, t, 0);
    if (t >= D.p) break;
    const int64_t i = back ? D.p - 1 - t : t;
    int l = 0, bad = 0;
    for (int64_t b = D.bptr[i] + lane; b < D.bptr[i + 1]; b += 32) {
      const int v = dag_wait(D.word + D.bcol[b], abort, limit, st);
      if (v <= 0)
        bad = 1;
      else
        l = max(l, v);  // v = lev[k] + 1
    }
    l = warp_max_i(l);
    bad = __any_sync(0xffffffffu, bad);
    if (lane == 0) {
      if (!bad) atomicMax(D.depth, l + 1);
      atomicExch(D.word + i, bad ? -1 : l + 1);
    }
  }
}

// word = lev + 1 -> lev
__global__ void k_dag_unword(int64_t n, int32_t* __restrict__ w) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    w[i] -= 1;
}

// Stable least-significant-digit radix sort of row ids by their level, 8
// bits a pass: per block of RS_T ids a digit histogram, one scan over
// (digit, block), then every id goes to its digit's range after the ids of
// earlier blocks and of earlier warps and lanes of its own block.
constexpr int RS_T = 256;

__global__ void k_rs_init(int64_t n, bool descending, int32_t* __restrict__ v) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    v[i] = (int32_t)(descending ? n - 1 - i : i);
}

__global__ void __launch_bounds__(RS_T) k_rs_hist(int64_t n, const int32_t* __restrict__ v,
                                                  const int32_t* __restrict__ key, int shift, int64_t nblk,
                                                  int32_t* __restrict__ hist) {
  __shared__ int h[256];
  for (int d = threadIdx.x; d < 256; d += blockDim.x) h[d] = 0;
  __syncthreads();
  const int64_t e = blockIdx.x * (int64_t)RS_T + threadIdx.x;
  if (e < n) atomicAdd(&h[(key[v[e]] >> shift) & 255], 1);
  __syncthreads();
  for (int d = threadIdx.x; d < 256; d += blockDim.x) hist[(int64_t)d * nblk + blockIdx.x] = h[d];
}

__global__ void __launch_bounds__(RS_T) k_rs_scatter(int64_t n, const int32_t* __restrict__ v,
                                                     const int32_t* __restrict__ key, int shift, int64_t nblk,
                                                     const int64_t* __restrict__ base, int32_t* __restrict__ out) {
  __shared__ int cnt[RS_T / 32][256];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int x = threadIdx.x; x < (RS_T / 32) * 256; x += blockDim.x) (&cnt[0][0])[x] = 0;
  __syncthreads();
  const int64_t e = blockIdx.x * (int64_t)RS_T + threadIdx.x;
  const bool has = e < n;
  const int32_t id = has ? v[e] : 0;
  const int d = has ? (key[id] >> shift) & 255 : 256;
  const unsigned peers = __match_any_sync(0xffffffffu, d);
  const int rank = __popc(peers & ((1u << lane) - 1u));
  if (has && rank == 0) cnt[warp][d] = __popc(peers);
  __syncthreads();
  if (has) {
    int off = 0;
    for (int w = 0; w < warp; ++w) off += cnt[w][d];
    out[base[(int64_t)d * nblk + blockIdx.x] + off + rank] = id;
  }
}

}  // namespace

// Level orders of the last level's L (forward sweep) and U (backward sweep)
// on the device: the levels of both dependency DAGs (k_dag_level), then each
// side's rows sorted by level, rows ascending (L) / descending (U) within a
// level.
template <typename T>
void level_orders(LastDev<T>& X, uint64_t wait_limit, int* dst, cudaStream_t s) {
  const int64_t p = X.L.nbr;
  X.lorder.alloc(std::max<int64_t>(p, 1), s);
  X.uorder.alloc(std::max<int64_t>(p, 1), s);
  X.ldepth = X.udepth = 0;
  if (p == 0) return;
  DBuf<int32_t> lev(2 * p, s);
  DBuf<unsigned long long> tick(2, s);
  DBuf<int> abort(1, s), dmax(2, s);
  lev.zero();
  tick.zero();
  abort.zero();
  dmax.zero();
  int dev = 0, nsm = 0;
  VB_CUDA(cudaGetDevice(&dev));
  VB_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  const unsigned half = (unsigned)std::max<int64_t>(1, std::min<int64_t>((int64_t)nsm * 4, (p + 7) / 8));
  DagSide fw{p, X.L.bptr.p, X.L.bcol.p, lev.p, tick.p, dmax.p};
  DagSide bw{p, X.U.bptr.p, X.U.bcol.p, lev.p + p, tick.p + 1, dmax.p + 1};
  launch(k_dag_level, 2 * half, 256, 0, s, fw, bw, half, abort.p, (unsigned long long)wait_limit, dst);
  VB_LAUNCH_CHECK();
  check_status(dst, s, "vbarms_factor: level order of the triangular sweeps");
  launch(k_dag_unword, grid_for(2 * p, 256), 256, 0, s, 2 * p, lev.p);
  VB_LAUNCH_CHECK();
  const std::vector<int> dd = d2h_vec(dmax.p, 2, s);
  X.ldepth = dd[0];
  X.udepth = dd[1];
  const int64_t nblk = (p + RS_T - 1) / RS_T;
  DBuf<int32_t> hist(256 * nblk, s);
  DBuf<int64_t> base(256 * nblk + 1, s);
  for (int side = 0; side < 2; ++side) {
    const int32_t* key = lev.p + side * p;
    const int64_t depth = side == 0 ? X.ldepth : X.udepth;
    DBuf<int32_t> a(p, s), b(p, s);
    launch(k_rs_init, grid_for(p, 256), 256, 0, s, p, side == 1, a.p);
    VB_LAUNCH_CHECK();
    for (int shift = 0; shift < 31 && (1LL << shift) < depth; shift += 8) {
      launch(k_rs_hist, (unsigned)nblk, RS_T, 0, s, p, a.p, key, shift, nblk, hist.p);
      VB_LAUNCH_CHECK();
      scan_i32_to_i64(hist.p, base.p, 256 * nblk, s);
      launch(k_rs_scatter, (unsigned)nblk, RS_T, 0, s, p, a.p, key, shift, nblk, base.p, b.p);
      VB_LAUNCH_CHECK();
      std::swap(a, b);
    }
    (side == 0 ? X.lorder : X.uorder) = std::move(a);
  }
}

template void level_orders<double>(LastDev<double>&, uint64_t, int*, cudaStream_t);
template void level_orders<float>(LastDev<float>&, uint64_t, int*, cudaStream_t);

}  // namespace vb
