// Last-level block ILUT of VBARMS on the GPU (Section 3 dropping rule, the
// block IKJ form of Alg. 3), on the scaled last Schur complement in natural
// order.
//
// Row i is processed by one warp that took ticket i (tickets are handed out
// in row order, so every row a warp waits for is already owned by a running
// warp).  A matrix made of independent diagonal blocks (a batch, or the
// subdomains of a domain decomposition) may instead hand out its rows
// interleaved across the blocks, each block's rows in ascending order: the
// blocks' dependency chains then advance side by side.
//
// The warp keeps its working row in a private workspace (hash table column ->
// slot, dense values): in shared memory when the row fits, else in global
// memory (a shared row whose fill would outgrow the buffer moves, slots and
// values as they are, to the global one before the blocks that overflow it are
// created).  The size of the shared workspace is chosen by timing from the
// last-level matrix (rows of a few large blocks, or rows of many small ones).
// The warp eliminates its L part in ascending column order including fill.
// For each column k it needs row k's factored pivot block and its U row:
// row k publishes them as one record (below) and a 64-bit word in done[k]
// telling where the record lies, so the dependant waits for one word and
// brings the record on chip with one bulk asynchronous copy (completing on an
// mbarrier); the record of the next pending column is fetched ahead while
// the current step computes.  After the last column the warp thresholds its U
// part, applies lfil to L and U (radix selection of the lfil largest norms),
// sorts the kept blocks by column, factors its diagonal block (GEPP) and
// publishes.  Per element, the operation order is the oracle's, so FP64
// results match it bit for bit; the mixed factor keeps its drop sums, drop
// tests and diagonal GEPP in FP32 (a block whose condition estimate exceeds
// the threshold is factored again in FP64).
//
// A wait that runs out sets VB_ETIMEOUT and raises an abort flag; a row that
// failed publishes kRowFailed so that its dependants stop too.  Overflowing a
// pool or the global workspace sets an overflow code and the host repeats the
// kernel with larger buffers.
#include <algorithm>
#include <chrono>
#include <climits>
#include <map>
#include <mutex>
#include <type_traits>

#include "internal.h"
#include "level.cuh"
#include "vbsr_ops.cuh"

namespace vb {
namespace {

enum : int { SL_LIVE = 0, SL_LKEPT = 1, SL_DEAD = 2 };

// ---------------------------------------------------------------------------
// Published rows.  Row k's record, in the U pool, 16-byte aligned:
//   int32 head[4]         ucnt (U blocks), nk, lu64 (1: the pivot LU is stored
//                         in FP64, else in the factor's type), nval (U values)
//   int32 piv[nk]         GEPP interchanges of the pivot block
//   TL lu[nk * nk]        the factored pivot block, row-major
//   int32 ucol[ucnt]      U block columns, ascending
//   int32 urel[ucnt]      each U block's first value within val
//   int32 unj[ucnt]       each U block's column count
//   T val[nval]           the U blocks, row-major, in column order
// every part starting on a 16-byte boundary.  done[k] = (offset << 24) |
// length, both in 16-byte units, once the record is complete; kRowFailed when
// the row failed; 0 before.
constexpr unsigned long long kRowFailed = ~0ull;
constexpr int64_t kRecMaxUnits = (1LL << 24) - 1;

__host__ __device__ __forceinline__ int64_t pad16(int64_t b) { return (b + 15) & ~(int64_t)15; }

struct RecLayout {
  int64_t piv, lu, ucol, urel, unj, val, bytes;
};

__host__ __device__ __forceinline__ RecLayout rec_layout(int ucnt, int nk, int lu64, int64_t nval, int tsize) {
  RecLayout L;
  L.piv = 16;
  L.lu = L.piv + pad16(4LL * nk);
  L.ucol = L.lu + pad16((int64_t)nk * nk * (lu64 ? 8 : tsize));
  L.urel = L.ucol + pad16(4LL * ucnt);
  L.unj = L.urel + pad16(4LL * ucnt);
  L.val = L.unj + pad16(4LL * ucnt);
  L.bytes = L.val + pad16(nval * tsize);
  return L;
}

struct Pools {
  // L rows: blocks in pool order; per row the first block and count
  int32_t* lcol;
  int64_t* lvo;  // value offset of each pool block
  int64_t* lstart;
  int32_t* lcnt;
  unsigned long long* done;  // per row: the published record word
  unsigned long long* ctr;   // [0] L blocks, [1] L values, [2] U record units, [4] ticket,
                             // [5] largest row values asked, [6] largest row slots asked
  int64_t lbcap, lvcap, ucap16;
  int* abort;
  // ticket -> row (nullptr: ticket t is row t); every row's dependencies
  // must come earlier in it
  const int32_t* order;
  // tickets handed out (the rows of the first nticket tickets: every prefix
  // of the ticket order holds its rows' dependencies, so it is factored
  // exactly on its own)
  int64_t nticket;
  // per row (may be NULL): 1 + the largest depth among the rows it waited
  // on (every pending L column, the dropped multipliers' included), i.e. the
  // length of the longest chain of waits ending at the row
  int32_t* depth;
};

// Global fallback workspace, per warp.
struct Workspace {
  int* keys;       // [ht]
  int* hpos;       // [smax]
  int* scol;       // [smax]
  int* soff;       // [smax]
  int* sstate;     // [smax]
  long long* sf2;  // [smax] norm key of each slot
  int* sncl;       // [smax] column count of each slot's block
  int* fin;        // [2 smax] candidate lists of the finish
  unsigned long long* srt;  // [4 smax] kept lists being sorted
  int ht, smax;
  int64_t vmax;
};

// Shared workspace of one warp, sized at launch (byte offsets in the warp's
// region; every part 16-byte aligned).
struct IlutGeom {
  int slots, hash, vbytes, stage, lcap;
  int o_misc, o_stage, o_vals, o_keys, o_hpos, o_scol, o_soff, o_sst, o_sf2, o_sncl, o_lc, o_ls;
  int bytes;
};

// Geometries chosen by timing, per device, precision and class of row sizes
// (the process keeps them), and the smallest matrix that is timed.
std::mutex g_geom_mu;
std::map<long long, struct IlutGeom> g_geom;
constexpr int64_t kTuneMinRows = 65536;

constexpr int PVMAX = 64;
struct IlutMisc {
  unsigned long long mbar[2];  // completion of the bulk copy into stage buffer b
  unsigned long long nvals;
  long long wdst[32];  // destination offset of each block of a copied chunk
  int hist[256];       // radix selection of the lfil cut
  int qoff[32];        // workspace value offset of each U block's target
  int quo[32];         // value offset of the U block within the record values
  int qnj[32];
  int qpre[33];        // element prefix of a chunk's blocks
  int pv[PVMAX];       // GEPP interchanges of the row's own diagonal block
  float lu32[64];      // the row's FP32 pivot LU (at most 8 x 8) for its record
  float mbuf[64];      // a step's FP32 multiplier (at most 64 values) for its update
  int nl, nslots, flag, pad;
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
                                           int* sstate, int* sncl, int* nslots, unsigned long long* nvals,
                                           uint32_t hmask, int col, int ncl, int sz) {
  const int slot = atomicAdd(nslots, 1);
  const long long off = (long long)atomicAdd(nvals, (unsigned long long)sz);
  if (slot >= smax) return -1;
  hpos[slot] = -1;  // the end-of-row reset skips slots that were never placed
  if (off + sz > vmax) return -1;
  scol[slot] = col;
  soff[slot] = (int)off;
  sstate[slot] = SL_LIVE;
  sncl[slot] = ncl;
  hpos[slot] = ws_place(keys, hmask, slot, col);
  return hpos[slot] < 0 ? -1 : slot;
}

constexpr int MAX_SLOTS = 4096;  // largest workspace (blocks of one working row)

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
  for (int e0 = 0; e0 < n; e0 += 16) {  // sixteen loads in flight, summed in element order
    float x[16];
#pragma unroll
    for (int u = 0; u < 16; ++u) x[u] = e0 + u < n ? (float)v[e0 + u] : 0.f;
#pragma unroll
    for (int u = 0; u < 16; ++u)
      if (e0 + u < n) s = __fmaf_rn(x[u], x[u], s);
  }
  return s;
}

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

// ---- pivot blocks of at most 8 rows (FP32), held in registers ---------------
// The block size is a template argument, so every loop is unrolled and no
// array is indexed at run time.  Each routine gives every element the
// operations of its generic counterpart (ainv_right_row_sh, gepp_warp,
// inv_norm1_f32) in the same order, so the results are identical bit for
// bit; only the latency of the dependent chain changes.

// x (one row of length N, shared or global memory) <- x (P^T L U)^{-1}.
template <int N>
__device__ __forceinline__ void ainv_right_row_n(const float* lu, const int* pv, float* x, float* x2) {
  float r[N];
#pragma unroll
  for (int j = 0; j < N; ++j) r[j] = x[j];
#pragma unroll
  for (int j = 0; j < N; ++j) {
    float s = r[j];
#pragma unroll
    for (int q = 0; q < j; ++q) s = msub<float>(s, r[q], lu[q * N + j]);
    r[j] = s / lu[j * N + j];
  }
#pragma unroll
  for (int j = N - 1; j >= 0; --j) {
    float s = r[j];
#pragma unroll
    for (int q = j + 1; q < N; ++q) s = msub<float>(s, r[q], lu[q * N + j]);
    r[j] = s;
  }
#pragma unroll
  for (int k = N - 1; k >= 0; --k) {
    const int p = pv[k];
#pragma unroll
    for (int q = k + 1; q < N; ++q)
      if (q == p) {
        const float t = r[k];
        r[k] = r[q];
        r[q] = t;
      }
  }
#pragma unroll
  for (int j = 0; j < N; ++j) x[j] = r[j];
  if (x2) {
#pragma unroll
    for (int j = 0; j < N; ++j) x2[j] = r[j];
  }
}

// GEPP of the N x N row-major block a (shared memory), row i in lane i's
// registers: the pivot is the largest |a_ik| (lowest row on ties) found by a
// warp max-reduction of the keys and a ballot; interchanges and the pivot
// row travel by shuffles.  Pivot rows go to gpiv (and pvs when not null).
template <int N>
__device__ __forceinline__ bool gepp_n(float* a, int* pvs, int32_t* gpiv, int lane) {
  float r[N];
#pragma unroll
  for (int j = 0; j < N; ++j) r[j] = lane < N ? a[lane * N + j] : 0.f;
  bool ok = true;
#pragma unroll
  for (int k = 0; k < N; ++k) {
    const unsigned key = (lane >= k && lane < N) ? (unsigned)abs_key(r[k]) + 1u : 0u;
    const unsigned mk = __reduce_max_sync(0xffffffffu, key);
    if (mk <= 1u) {  // the pivot column is exactly zero
      ok = false;
      break;
    }
    const int p = __ffs(__ballot_sync(0xffffffffu, key == mk)) - 1;
    if (lane == 0) {
      gpiv[k] = p;
      if (pvs) pvs[k] = p;
    }
    if (p != k) {
#pragma unroll
      for (int j = 0; j < N; ++j) {
        const float vk = __shfl_sync(0xffffffffu, r[j], k);
        const float vp = __shfl_sync(0xffffffffu, r[j], p);
        if (lane == k) r[j] = vp;
        if (lane == p) r[j] = vk;
      }
    }
    float u[N];
#pragma unroll
    for (int j = k; j < N; ++j) u[j] = __shfl_sync(0xffffffffu, r[j], k);
    if (lane > k && lane < N) {
      const float l = div_rn<float>(r[k], u[k]);
      r[k] = l;
#pragma unroll
      for (int j = k + 1; j < N; ++j) r[j] = msub<float>(r[j], l, u[j]);
    }
  }
  if (lane < N) {
#pragma unroll
    for (int j = 0; j < N; ++j) a[lane * N + j] = r[j];
  }
  __syncwarp();
  return ok;
}

// ||B^{-1}||_1 of a GEPP-factored N x N block: lane c solves B x = e_c in
// registers; the largest column sum, on every lane.
template <int N>
__device__ __forceinline__ float inv_norm1_n(const float* a, const int* pv, int lane) {
  float cs = 0.f;
  if (lane < N) {
    float x[N];
#pragma unroll
    for (int ii = 0; ii < N; ++ii) x[ii] = ii == lane ? 1.f : 0.f;
#pragma unroll
    for (int kk = 0; kk < N; ++kk) {
      const int pk = pv[kk];
#pragma unroll
      for (int q = kk + 1; q < N; ++q)
        if (q == pk) {
          const float t = x[kk];
          x[kk] = x[q];
          x[q] = t;
        }
    }
#pragma unroll
    for (int ii = 1; ii < N; ++ii) {
      float sum = x[ii];
#pragma unroll
      for (int kk = 0; kk < ii; ++kk) sum = __fmaf_rn(-a[ii * N + kk], x[kk], sum);
      x[ii] = sum;
    }
#pragma unroll
    for (int ii = N - 1; ii >= 0; --ii) {
      float sum = x[ii];
#pragma unroll
      for (int kk = ii + 1; kk < N; ++kk) sum = __fmaf_rn(-a[ii * N + kk], x[kk], sum);
      x[ii] = __fdiv_rn(sum, a[ii * N + ii]);
    }
#pragma unroll
    for (int ii = 0; ii < N; ++ii) cs += fabsf(x[ii]);
  }
  for (int o = 16; o > 0; o >>= 1) cs = fmaxf(cs, __shfl_xor_sync(0xffffffffu, cs, o));
  return cs;
}

// Dispatch on the block size (false / a negative norm: larger than 8, the
// caller takes the generic routine).
__device__ __forceinline__ bool ainv_right_row_small(const float* lu, const int* pv, int m, float* x, float* x2) {
  switch (m) {
    case 1: ainv_right_row_n<1>(lu, pv, x, x2); return true;
    case 2: ainv_right_row_n<2>(lu, pv, x, x2); return true;
    case 3: ainv_right_row_n<3>(lu, pv, x, x2); return true;
    case 4: ainv_right_row_n<4>(lu, pv, x, x2); return true;
    case 5: ainv_right_row_n<5>(lu, pv, x, x2); return true;
    case 6: ainv_right_row_n<6>(lu, pv, x, x2); return true;
    case 7: ainv_right_row_n<7>(lu, pv, x, x2); return true;
    case 8: ainv_right_row_n<8>(lu, pv, x, x2); return true;
    default: return false;
  }
}
__device__ __forceinline__ bool gepp_small(float* a, int n, int* pvs, int32_t* gpiv, int lane) {
  switch (n) {
    case 1: return gepp_n<1>(a, pvs, gpiv, lane);
    case 2: return gepp_n<2>(a, pvs, gpiv, lane);
    case 3: return gepp_n<3>(a, pvs, gpiv, lane);
    case 4: return gepp_n<4>(a, pvs, gpiv, lane);
    case 5: return gepp_n<5>(a, pvs, gpiv, lane);
    case 6: return gepp_n<6>(a, pvs, gpiv, lane);
    case 7: return gepp_n<7>(a, pvs, gpiv, lane);
    default: return gepp_n<8>(a, pvs, gpiv, lane);
  }
}
__device__ __forceinline__ float inv_norm1_small(const float* a, int n, const int* pv, int lane) {
  switch (n) {
    case 1: return inv_norm1_n<1>(a, pv, lane);
    case 2: return inv_norm1_n<2>(a, pv, lane);
    case 3: return inv_norm1_n<3>(a, pv, lane);
    case 4: return inv_norm1_n<4>(a, pv, lane);
    case 5: return inv_norm1_n<5>(a, pv, lane);
    case 6: return inv_norm1_n<6>(a, pv, lane);
    case 7: return inv_norm1_n<7>(a, pv, lane);
    default: return inv_norm1_n<8>(a, pv, lane);
  }
}

// ---------------------------------------------------------------------------
// Bulk asynchronous copies into shared memory, completing on an mbarrier.
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
}

// Orders this thread's generic-proxy view of memory with the async proxy
// (the bulk copies): taken by a producer after writing a record and by a
// consumer after acquiring its flag, before issuing the copy.
__device__ __forceinline__ void fence_proxy_async_all() { asm volatile("fence.proxy.async;" ::: "memory"); }

__device__ __forceinline__ void bulk_load(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ bool mbar_test(unsigned long long* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait for phase `parity` of bar to complete; false when limit ns
// passed first.
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity, unsigned long long limit) {
  if (mbar_test(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  for (unsigned it = 1;; ++it) {
    if (mbar_test(bar, parity)) return true;
    if ((it & 15) == 0 && global_ns() - t0 > limit) return false;
  }
}

__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.b64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

// The published word of a row, waiting for it as wait_flag does (relaxed
// polls with backoff, the abort word and the time budget every 16th poll,
// one acquire fence at the end).  0 when the wait gave up.
__device__ __forceinline__ unsigned long long wait_word(const unsigned long long* w, int* abort,
                                                        unsigned long long limit, int* st) {
  unsigned long long v = ld_relaxed_u64(w);
  if (v == 0) {
    const unsigned long long t0 = global_ns();
    unsigned nsl = 32;
    for (unsigned it = 1;; ++it) {
      __nanosleep(nsl);
      if (nsl < 256) nsl <<= 1;
      v = ld_relaxed_u64(w);
      if (v != 0) break;
      if ((it & 15) == 0) {
        if (*((volatile int*)abort) != 0) return 0;
        if (global_ns() - t0 > limit) {
          dev_fail(st, DEV_ETIMEOUT);
          atomicExch(abort, 1);
          return 0;
        }
      }
    }
  }
  asm volatile("fence.acq_rel.gpu;" ::: "memory");
  return v;
}

// Ascending bitonic sort of a[0, n2) (n2 a power of two) by one warp.
__device__ void warp_bitonic_sort(unsigned long long* a, int n2, int lane) {
  for (int k = 2; k <= n2; k <<= 1)
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int x = lane; x < n2; x += 32) {
        const int y = x ^ j;
        if (y > x) {
          const unsigned long long u = a[x], v = a[y];
          if ((u > v) == ((x & k) == 0)) {
            a[x] = v;
            a[y] = u;
          }
        }
      }
      __syncwarp();
    }
}

// lfil (Section 3 dropping rule with the lfil bound of the paper's ARMS
// parameters): of the n candidate slots cand[], keep the lfil with the
// largest norm keys, lower column first on equal keys; the others become
// SL_DEAD and cand[] is compacted to the kept ones.  The lfil-th largest key
// is found by radix selection, 8 bits a pass from the top (keybytes passes:
// the keys are the bit patterns of non-negative FP64 or FP32 norms, so their
// integer order is their value order).  Returns the number kept.
__device__ int lfil_cut(int* cand, int n, int lfil, const long long* sf2, const int* scol, int* sstate, int* hist,
                        int keybytes, int lane) {
  if (lfil < 0 || n <= lfil) return n;
  if (lfil == 0) {
    for (int c = lane; c < n; c += 32) sstate[cand[c]] = SL_DEAD;
    __syncwarp();
    return 0;
  }
  unsigned long long prefix = 0, pmask = 0;
  int want = lfil;  // keys still to take at or below the current prefix
  for (int d = keybytes - 1; d >= 0; --d) {
    const int shift = 8 * d;
    for (int b = lane; b < 256; b += 32) hist[b] = 0;
    __syncwarp();
    for (int base = 0; base < n; base += 32) {
      const int c = base + lane;
      int bin = -1;
      if (c < n) {
        const unsigned long long key = (unsigned long long)sf2[cand[c]];
        if ((key & pmask) == prefix) bin = (int)((key >> shift) & 255);
      }
      // lanes with the same bin add once (keys of one row crowd a few bins)
      const unsigned peers = __match_any_sync(0xffffffffu, bin);
      if (bin >= 0 && (__ffs(peers) - 1) == lane) atomicAdd(&hist[bin], __popc(peers));
    }
    __syncwarp();
    // lane l holds bins 255 - 8 l - u, u = 0..7 (the highest bins first)
    int cnt[8];
    int s = 0;
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      cnt[u] = hist[255 - 8 * lane - u];
      s += cnt[u];
    }
    int incl = s;
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += v;
    }
    const int excl = incl - s;
    int bin = -1, above = 0;
    if (excl < want && want <= incl) {
      int run = excl;
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        if (bin < 0 && run + cnt[u] >= want) {
          bin = 255 - 8 * lane - u;
          above = run;
        }
        run += cnt[u];
      }
    }
    const unsigned who = __ballot_sync(0xffffffffu, bin >= 0);
    const int src = __ffs(who) - 1;
    bin = __shfl_sync(0xffffffffu, bin, src);
    above = __shfl_sync(0xffffffffu, above, src);
    want -= above;
    prefix |= (unsigned long long)bin << shift;
    pmask |= 255ull << shift;
    __syncwarp();
  }
  // keys above prefix are kept; of the keys equal to it, the `want` with the
  // lowest columns.  Every cut slot is marked first (the tie ranks read the
  // whole list), then the list is compacted.
  for (int c = lane; c < n; c += 32) {
    const int q = cand[c];
    const unsigned long long key = (unsigned long long)sf2[q];
    bool keep = key > prefix;
    if (key == prefix) {
      const int col = scol[q];
      int rank = 0;
      for (int c2 = 0; c2 < n; ++c2) {
        const int q2 = cand[c2];
        if ((unsigned long long)sf2[q2] == prefix && scol[q2] < col) ++rank;
      }
      keep = rank < want;
    }
    if (!keep) sstate[q] = SL_DEAD;
  }
  __syncwarp();
  int kept = 0;
  for (int base = 0; base < n; base += 32) {
    const int c = base + lane;
    const int q = c < n ? cand[c] : -1;
    const bool keep = q >= 0 && sstate[q] != SL_DEAD;
    __syncwarp();
    const unsigned bk = __ballot_sync(0xffffffffu, keep);
    if (keep) cand[kept + __popc(bk & ((1u << lane) - 1u))] = q;
    kept += __popc(bk);
    __syncwarp();
  }
  return kept;
}

// The kept blocks of one part in column order: srt[p] = col << 32 | slot for
// p < k (n2 = the next power of two, padded with ~0).  Returns n2.
__device__ int sort_by_column(const int* cand, int k, const int* scol, unsigned long long* srt, int lane) {
  int n2 = 1;
  while (n2 < k) n2 <<= 1;
  if (k <= 32) {  // the keys are distinct: each goes to its rank
    const unsigned long long key =
        lane < k ? ((unsigned long long)(unsigned)scol[cand[lane]] << 32) | (unsigned)cand[lane] : ~0ull;
    int rank = 0;
    for (int j = 0; j < k; ++j) rank += __shfl_sync(0xffffffffu, key, j) < key ? 1 : 0;
    if (lane < k)
      srt[rank] = key;
    else if (lane < n2)
      srt[lane] = ~0ull;
    __syncwarp();
    return n2;
  }
  for (int p = lane; p < n2; p += 32)
    srt[p] = p < k ? ((unsigned long long)(unsigned)scol[cand[p]] << 32) | (unsigned)cand[p] : ~0ull;
  __syncwarp();
  warp_bitonic_sort(srt, n2, lane);
  return n2;
}

// Copy blocks to consecutive destinations, 32 blocks a round: block b of the
// round has sz[b] values at src offset so[b] and goes to dst offset dof[b];
// lanes walk the round's flattened values, eight loads in flight per lane.
template <typename T>
__device__ __forceinline__ void copy_round(IlutMisc& M, int sz, int so, long long dof, const T* __restrict__ src,
                                           T* __restrict__ dst, int lane) {
  int incl = sz;
  for (int o = 1; o < 32; o <<= 1) {
    const int v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += v;
  }
  const int total = __shfl_sync(0xffffffffu, incl, 31);
  M.qpre[lane] = incl - sz;
  if (lane == 31) M.qpre[32] = total;
  M.qoff[lane] = so;
  M.wdst[lane] = dof;
  __syncwarp();
  for (int e0 = lane; e0 < total; e0 += 32 * 8) {
    T v[8];
    long long d8[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int e = e0 + 32 * u;
      d8[u] = -1;
      if (e < total) {
        int lo = 0, hi = 31;  // last block with qpre <= e (empty blocks share a prefix)
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (M.qpre[mid] <= e)
            lo = mid;
          else
            hi = mid - 1;
        }
        const int local = e - M.qpre[lo];
        v[u] = src[M.qoff[lo] + local];
        d8[u] = M.wdst[lo] + local;
      }
    }
#pragma unroll
    for (int u = 0; u < 8; ++u)
      if (d8[u] >= 0) dst[d8[u]] = v[u];
  }
  __syncwarp();
}



template <typename T>
__global__ void __launch_bounds__(256, 2)
    k_ilut(VBView<T> A, IlutGeom g, Workspace ws, T* __restrict__ wvals_all, Pools P, T* __restrict__ lval,
           unsigned char* __restrict__ upool, const int64_t* __restrict__ dgoff, double* __restrict__ dg,
           float* __restrict__ dg32, int32_t* __restrict__ piv, int32_t* __restrict__ ptag, int mixed,
           double cond_thr, double t, int lfil, unsigned long long wait_limit, int* st) {
  extern __shared__ __align__(128) unsigned char ilut_sm[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned char* const wb = ilut_sm + (size_t)warp * g.bytes;
  IlutMisc& M = *reinterpret_cast<IlutMisc*>(wb + g.o_misc);
  unsigned char* const stage0 = wb + g.o_stage;
  unsigned char* const stage1 = stage0 + g.stage;
  T* const sh_vals = reinterpret_cast<T*>(wb + g.o_vals);
  int* const sh_keys = reinterpret_cast<int*>(wb + g.o_keys);
  int* const sh_hpos = reinterpret_cast<int*>(wb + g.o_hpos);
  int* const sh_scol = reinterpret_cast<int*>(wb + g.o_scol);
  int* const sh_soff = reinterpret_cast<int*>(wb + g.o_soff);
  int* const sh_sst = reinterpret_cast<int*>(wb + g.o_sst);
  long long* const sh_sf2 = reinterpret_cast<long long*>(wb + g.o_sf2);
  int* const sh_sncl = reinterpret_cast<int*>(wb + g.o_sncl);
  int* const lc = reinterpret_cast<int*>(wb + g.o_lc);  // pending L columns (INT_MAX when processed)
  int* const ls = reinterpret_cast<int*>(wb + g.o_ls);  // their slots
  const int64_t wid = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;
  const int VSH = g.vbytes / (int)sizeof(T);
  const float tf = (float)t, condf = (float)cond_thr;
  constexpr int TS = (int)sizeof(T);
  volatile int* vflag = &M.flag;
  volatile int* vns = &M.nslots;
  volatile int* vnl = &M.nl;
  int* const gkeys = ws.keys + wid * ws.ht;
  for (int k = lane; k < ws.ht; k += 32) gkeys[k] = -1;
  for (int k = lane; k < g.hash; k += 32) sh_keys[k] = -1;
  if (lane == 0) {
    mbar_init(&M.mbar[0]);
    mbar_init(&M.mbar[1]);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncwarp();
  // stage buffer bookkeeping, the same in every lane: the column whose record
  // a buffer holds (-1: free), whether its copy still has to be waited for,
  // and the parity of its mbarrier's next phase
  int btag0 = -1, btag1 = -1;
  bool bpend0 = false, bpend1 = false;
  unsigned bph0 = 0, bph1 = 0;
  auto drain = [&]() {  // wait (bounded) for copies in flight and free both buffers
    if (bpend0) {
      if (mbar_wait(&M.mbar[0], bph0, wait_limit)) bph0 ^= 1;
      bpend0 = false;
    }
    if (bpend1) {
      if (mbar_wait(&M.mbar[1], bph1, wait_limit)) bph1 ^= 1;
      bpend1 = false;
    }
    btag0 = btag1 = -1;
  };

  for (;;) {
    long long row = 0;
    if (lane == 0) {
      row = (long long)atomicAdd(P.ctr + 4, 1ULL);
      if (row >= P.nticket)
        row = A.nbr;
      else if (P.order)
        row = P.order[row];
    }
    row = __shfl_sync(0xffffffffu, row, 0);
    if (row >= A.nbr) break;
    const int64_t i = row;
    int maxdep = 0;  // lane 0: the deepest row waited on
    const int ni = A.rsz[i];
    const int64_t b0 = A.bptr[i], b1 = A.bptr[i + 1];
    const int64_t v0 = A.voff[b0], nv = A.voff[b1] - v0;
    const int nb = (int)(b1 - b0);
    // The working row lives in shared memory when it leaves room for fill; a
    // row whose fill outgrows that restarts in the warp's global workspace
    // (nothing of it is visible before its finish, so the restart is exact).
    bool in_sh = nb <= g.slots / 2 && nv <= VSH / 2;
    int status_local = 0;
    int* keys;
    int* hpos;
    int* scol;
    int* soff;
    int* sstate;
    long long* sf2;
    int* sncl;
    T* wv;
    int smax_c;
    int64_t vmax_c;
    uint32_t hmask;
    for (;;) {
      if (in_sh) {
        keys = sh_keys, hpos = sh_hpos, scol = sh_scol, soff = sh_soff, sstate = sh_sst, sf2 = sh_sf2;
        sncl = sh_sncl;
        wv = sh_vals;
        smax_c = g.slots, vmax_c = VSH, hmask = (uint32_t)g.hash - 1;
      } else {
        keys = gkeys, hpos = ws.hpos + wid * ws.smax, scol = ws.scol + wid * ws.smax;
        soff = ws.soff + wid * ws.smax, sstate = ws.sstate + wid * ws.smax, sf2 = ws.sf2 + wid * ws.smax;
        sncl = ws.sncl + wid * ws.smax;
        wv = wvals_all + wid * ws.vmax;
        smax_c = ws.smax, vmax_c = ws.vmax, hmask = (uint32_t)ws.ht - 1;
      }
      if (lane == 0) {
        M.nslots = 0;
        M.nvals = 0;
        M.flag = 0;
        M.nl = 0;
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
          sncl[slot] = A.rsz[J];
          hpos[slot] = ws_place(keys, hmask, slot, J);  // the table holds 2 smax positions
          if (J < i) {
            const int q = atomicAdd(&M.nl, 1);
            if (q < g.lcap) {
              lc[q] = J;
              ls[q] = slot;
            }
          }
        }
        warp_copy(wv, A.val + v0, nv, lane);
        if (lane == 0) {
          M.nslots = nb;
          M.nvals = (unsigned long long)nv;
        }
      }
      __syncwarp();
      status_local = *vflag ? DEV_OVERFLOW : 0;
      int64_t last = -1;
      // ---- eliminate the L part in ascending column order (including fill)
      while (status_local == 0) {
        // the next pending L column and the one after it: from the list while
        // it has not overflowed, else by a scan of the workspace slots
        int c1 = INT_MAX, s1 = -1, p1 = -1, c2 = INT_MAX;
        const int nlist = *vnl;
        if (nlist <= g.lcap) {
          for (int q = lane; q < nlist; q += 32) {
            const int c = lc[q];
            if (c < c1) {
              c2 = c1;
              c1 = c;
              s1 = ls[q];
              p1 = q;
            } else if (c < c2) {
              c2 = c;
            }
          }
        } else {
          const int ns = min(*vns, smax_c);
          for (int sidx = lane; sidx < ns; sidx += 32) {
            const int c = scol[sidx];
            if (sstate[sidx] == SL_LIVE && c > last && c < i) {
              if (c < c1) {
                c2 = c1;
                c1 = c;
                s1 = sidx;
              } else if (c < c2) {
                c2 = c;
              }
            }
          }
        }
        const int kmin = warp_min_i(c1);
        if (kmin == INT_MAX) break;
        const unsigned who = __ballot_sync(0xffffffffu, s1 >= 0 && c1 == kmin);
        const int owner = __ffs(who) - 1;
        const int sk = __shfl_sync(0xffffffffu, s1, owner);
        const int knext = warp_min_i(lane == owner ? c2 : c1);
        if (lane == owner && p1 >= 0) lc[p1] = INT_MAX;
        const int64_t k = kmin;
        last = k;
        const int nk = A.rsz[k];
        // ---- row k's record: already fetched ahead into a stage buffer, or
        // fetched now (a bounded wait for its word, then one bulk copy); a
        // record too large for a buffer is read in place
        int bi = btag0 == (int)k ? 0 : (btag1 == (int)k ? 1 : -1);
        const unsigned char* rec = nullptr;
        int64_t rlen = 0;
        // the word of the next pending column is loaded now and looked at
        // after the multiplier, so that its latency hides behind this step
        const bool want_pf = knext != INT_MAX && btag0 != knext && btag1 != knext;
        unsigned long long w2 = 0;
        if (want_pf && lane == 0) w2 = ld_relaxed_u64(P.done + knext);
        if (bi < 0) {
          unsigned long long word = 0;
          if (lane == 0) word = wait_word(P.done + k, P.abort, wait_limit, st);
          word = __shfl_sync(0xffffffffu, word, 0);
          if (word == 0 || word == kRowFailed) {
            status_local = DEV_ETIMEOUT;
            break;
          }
          rlen = (int64_t)(word & 0xFFFFFFull) * 16;
          const unsigned char* src = upool + (int64_t)(word >> 24) * 16;
          if (rlen <= g.stage) {
            // a free buffer, else one holding a record fetched ahead for a
            // later column: its copy is waited for before the buffer is reused
            bi = btag0 < 0 ? 0 : (btag1 < 0 ? 1 : 0);
            bool ok = true;
            if (bi == 0 && bpend0) {
              ok = mbar_wait(&M.mbar[0], bph0, wait_limit);
              if (ok) bph0 ^= 1;
              bpend0 = !ok;
            } else if (bi == 1 && bpend1) {
              ok = mbar_wait(&M.mbar[1], bph1, wait_limit);
              if (ok) bph1 ^= 1;
              bpend1 = !ok;
            }
            if (!__all_sync(0xffffffffu, ok)) {
              if (lane == 0) dev_fail(st, DEV_ETIMEOUT);
              status_local = DEV_ETIMEOUT;
              break;
            }
            if (lane == 0) {
              fence_proxy_async_all();
              bulk_load(bi ? stage1 : stage0, src, (unsigned)rlen, &M.mbar[bi]);
            }
            if (bi) {
              btag1 = (int)k;
              bpend1 = true;
            } else {
              btag0 = (int)k;
              bpend0 = true;
            }
          } else {
            rec = src;
          }
        }
        if (bi >= 0) {
          bool ok = true;
          if (bi == 0 && bpend0) {
            ok = mbar_wait(&M.mbar[0], bph0, wait_limit);
            if (ok) bph0 ^= 1;
            bpend0 = !ok;
          } else if (bi == 1 && bpend1) {
            ok = mbar_wait(&M.mbar[1], bph1, wait_limit);
            if (ok) bph1 ^= 1;
            bpend1 = !ok;
          }
          if (!__all_sync(0xffffffffu, ok)) {
            if (lane == 0) dev_fail(st, DEV_ETIMEOUT);
            status_local = DEV_ETIMEOUT;
            break;
          }
          rec = bi ? stage1 : stage0;
        }
        const bool staged = bi >= 0;
        if (P.depth && lane == 0) maxdep = max(maxdep, ld_relaxed_gpu(P.depth + k));
        // header: U blocks, pivot size, pivot precision, U values
        int hv = 0;
        if (lane < 4) hv = staged ? reinterpret_cast<const int*>(rec)[lane] : __ldcg(reinterpret_cast<const int*>(rec) + lane);
        const int ucnt = __shfl_sync(0xffffffffu, hv, 0);
        const int hnk = __shfl_sync(0xffffffffu, hv, 1);
        const int lu64 = __shfl_sync(0xffffffffu, hv, 2);
        const int uval_n = __shfl_sync(0xffffffffu, hv, 3);
        const RecLayout RL = rec_layout(ucnt, nk, lu64, uval_n, TS);
        if (hnk != nk || ucnt < 0 || uval_n < 0 || (!staged && RL.bytes > rlen && rlen) ||
            (staged && RL.bytes > g.stage)) {
          status_local = DEV_INTERNAL;  // never true for a published row: record and skip
          break;
        }
        const int* rpiv = reinterpret_cast<const int*>(rec + RL.piv);
        const int* rcol = reinterpret_cast<const int*>(rec + RL.ucol);
        const int* rrel = reinterpret_cast<const int*>(rec + RL.urel);
        const int* rnj = reinterpret_cast<const int*>(rec + RL.unj);
        const T* rval = reinterpret_cast<const T*>(rec + RL.val);
        T* m = wv + soff[sk];
        // the multiplier m = a_ik (P^T L U)_k^{-1}, in place, one lane per row;
        // an FP32 multiplier of at most 64 values is also kept in M.mbuf, where
        // the drop test and the update read it
        bool mb = false;
        if constexpr (std::is_same<T, float>::value) mb = staged && !lu64 && nk <= 8 && ni * nk <= 64;
        const T* msrc = m;
        if constexpr (std::is_same<T, float>::value)
          if (mb) msrc = M.mbuf;
        for (int a = lane; a < ni; a += 32) {
          if (staged) {
            if (lu64)
              ainv_right_row_sh<T, double, double>(reinterpret_cast<const double*>(rec + RL.lu), rpiv, nk, m + a * nk);
            else {
              bool small = false;
              if constexpr (std::is_same<T, float>::value)
                small = ainv_right_row_small(reinterpret_cast<const float*>(rec + RL.lu), rpiv, nk, m + a * nk,
                                             mb ? M.mbuf + a * nk : nullptr);
              if (!small)
                ainv_right_row_sh<T, float, T>(reinterpret_cast<const T*>(rec + RL.lu), rpiv, nk, m + a * nk);
            }
          } else {
            if (lu64)
              ainv_right_row<T, double>(reinterpret_cast<const double*>(rec + RL.lu), rpiv, nk, m + a * nk);
            else
              ainv_right_row<T, T>(reinterpret_cast<const T*>(rec + RL.lu), rpiv, nk, m + a * nk);
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
            const float x = (float)msrc[e];
            sf = __fmaf_rn(x, x, sf);
          }
          for (int o = 16; o > 0; o >>= 1) sf += __shfl_xor_sync(0xffffffffu, sf, o);
          dropped = drop_rule_f(sf, ni, nk, tf);
          key = norm_key(sf);
        }
        // the next pending column's record, fetched ahead while the update
        // computes, when its row was already published at the start of the
        // step, no buffer holds it yet and a buffer is free (the current
        // step's buffer holds k)
        if (want_pf) {
          const int ob = btag0 < 0 ? 0 : (btag1 < 0 ? 1 : -1);
          int go = 0;
          if (ob >= 0 && lane == 0 && w2 != 0 && w2 != kRowFailed && (int64_t)(w2 & 0xFFFFFFull) * 16 <= g.stage) {
            asm volatile("fence.acq_rel.gpu;" ::: "memory");
            fence_proxy_async_all();
            bulk_load(ob ? stage1 : stage0, upool + (int64_t)(w2 >> 24) * 16, (unsigned)((w2 & 0xFFFFFFull) * 16),
                      &M.mbar[ob]);
            go = 1;
          }
          go = __shfl_sync(0xffffffffu, go, 0);
          if (go) {
            if (ob) {
              btag1 = knext;
              bpend1 = true;
            } else {
              btag0 = knext;
              bpend0 = true;
            }
          }
        }
        if (dropped) {
          if (lane == 0) sstate[sk] = SL_DEAD;
          __syncwarp();
          if (bi == 0) btag0 = -1;
          if (bi == 1) btag1 = -1;
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
        for (int q0 = 0; q0 < ucnt && status_local == 0; q0 += 32) {
          const int q = q0 + lane;
          int32_t j = -1;
          int slot = -1;
          int uo = 0, njq = 0;
          bool missing = false;
          if (q < ucnt) {
            j = staged ? rcol[q] : __ldcg(rcol + q);
            uo = staged ? rrel[q] : __ldcg(rrel + q);
            njq = staged ? rnj[q] : __ldcg(rnj + q);
            if (j <= k || j >= A.nbr || uo < 0 || njq <= 0 || (int64_t)uo + (int64_t)nk * njq > uval_n) {
              *vflag = 4;  // a published U block lies right of k inside its record
              j = -1;
            } else {
              slot = ws_lookup(keys, scol, hmask, j);
              missing = slot < 0;
            }
          }
          __syncwarp();
          // A shared working row that this chunk's new blocks would overflow
          // moves to the warp's global workspace first: slot numbers (so the
          // pending L columns and the lookups above), value offsets and the
          // multiplier's values stay as they are; the global hash is rebuilt.
          // (When the global workspace is too small as well, the creation
          // below fails and the row takes the overflow path.)
          if (in_sh) {
            const unsigned mm = __ballot_sync(0xffffffffu, missing);
            if (mm) {
              const int add_s = __popc(mm);
              const int add_v = warp_sum_i(missing ? ni * njq : 0);
              const int ns0 = *vns;
              const long long nv0 = (long long)M.nvals;
              if ((ns0 + add_s > smax_c || nv0 + add_v > vmax_c) && ns0 + add_s <= ws.smax &&
                  nv0 + add_v <= ws.vmax) {
                int* const gh = ws.hpos + wid * ws.smax;
                int* const gc = ws.scol + wid * ws.smax;
                int* const go = ws.soff + wid * ws.smax;
                int* const gs = ws.sstate + wid * ws.smax;
                long long* const gf = ws.sf2 + wid * ws.smax;
                int* const gn = ws.sncl + wid * ws.smax;
                T* const gv = wvals_all + wid * ws.vmax;
                for (int q = lane; q < ns0; q += 32) {
                  gc[q] = scol[q];
                  go[q] = soff[q];
                  gs[q] = sstate[q];
                  gf[q] = sf2[q];
                  gn[q] = sncl[q];
                }
                for (long long e = lane; e < nv0; e += 32) gv[e] = wv[e];
                __syncwarp();
                const uint32_t gmask = (uint32_t)ws.ht - 1;
                for (int q = lane; q < ns0; q += 32) gh[q] = ws_place(gkeys, gmask, q, gc[q]);
                for (int q = lane; q < g.hash; q += 32) sh_keys[q] = -1;
                __syncwarp();
                keys = gkeys, hpos = gh, scol = gc, soff = go, sstate = gs, sf2 = gf, sncl = gn;
                wv = gv;
                smax_c = ws.smax, vmax_c = ws.vmax, hmask = gmask;
                in_sh = false;
                m = wv + soff[sk];
                if (!mb) msrc = m;
              }
            }
          }
          if (missing) {
            const int sz = ni * njq;
            slot = ws_new_slot(smax_c, vmax_c, keys, hpos, scol, soff, sstate, sncl, &M.nslots, &M.nvals, hmask, j,
                               njq, sz);
            if (slot < 0) {
              *vflag = 1;
            } else {
              T* z = wv + soff[slot];
#pragma unroll 4
              for (int e = 0; e < sz; ++e) z[e] = (T)0;
              if (j < i) {  // fill in the L part: pending for a later step
                const int pq = atomicAdd(&M.nl, 1);
                if (pq < g.lcap) {
                  lc[pq] = j;
                  ls[pq] = slot;
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
          const int nj = j >= 0 ? njq : 0;
          const int sz = ni * nj;
          int incl = sz;
          for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
          }
          const int total = __shfl_sync(0xffffffffu, incl, 31);
          M.qpre[lane] = incl - sz;
          if (lane == 31) M.qpre[32] = total;
          M.qoff[lane] = slot >= 0 ? soff[slot] : 0;
          M.quo[lane] = uo;
          M.qnj[lane] = nj;
          __syncwarp();
          const int nq = min(32, ucnt - q0);
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
                  if (M.qpre[mid] <= e)
                    lo = mid;
                  else
                    hi = mid - 1;
                }
                const int njt = M.qnj[lo];
                const int local = e - M.qpre[lo];
                a4[u] = local / njt;
                jj4[u] = local - a4[u] * njt;
                nj4[u] = njt;
                uo4[u] = M.quo[lo];
                dst[u] = wv + M.qoff[lo] + local;
                acc[u] = *dst[u];
              }
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              if (!dst[u]) continue;
              const T* U = rval + uo4[u];
              T av = acc[u];
              if (staged) {
                for (int r = 0; r < nk; ++r) av = msub<T>(av, msrc[a4[u] * nk + r], U[r * nj4[u] + jj4[u]]);
              } else {
                for (int r = 0; r < nk; ++r) av = msub<T>(av, msrc[a4[u] * nk + r], __ldcg(U + r * nj4[u] + jj4[u]));
              }
              *dst[u] = av;
            }
          }
          __syncwarp();
        }
        if (bi == 0) btag0 = -1;
        if (bi == 1) btag1 = -1;
      }
      if (status_local == DEV_OVERFLOW && in_sh) {
        // the fill outgrew the shared workspace: start the row again in the
        // global one (records fetched ahead stay valid)
        for (int q = lane; q < g.hash; q += 32) sh_keys[q] = -1;
        __syncwarp();
        in_sh = false;
        continue;
      }
      break;
    }
    drain();  // every record fetched ahead has been used, unless the row failed
    const int ns = min(*vns, smax_c);
    // A row that ends in the global workspace has its slot metadata copied
    // to the shared working-row region (unused by such a row) when it fits,
    // so that the scans of the finish read on-chip data; its values stay in
    // the global workspace.
    bool meta_sh = false;
    if (!in_sh && status_local == 0) {
      const int region = g.o_lc - g.o_vals;  // vals, hash and slot arrays of the shared workspace
      if (ns * 24 <= region) {
        meta_sh = true;
        long long* mf2 = reinterpret_cast<long long*>(wb + g.o_vals);
        int* mcol = reinterpret_cast<int*>(mf2 + ns);
        int* mst = mcol + ns;
        int* mncl = mst + ns;
        int* moff = mncl + ns;
        for (int q = lane; q < ns; q += 32) {
          mf2[q] = sf2[q];
          mcol[q] = scol[q];
          mst[q] = sstate[q];
          mncl[q] = sncl[q];
          moff[q] = soff[q];
        }
        __syncwarp();
        sf2 = mf2, scol = mcol, sstate = mst, sncl = mncl, soff = moff;
      }
    }
    // ---- finish the row.
    int dslot = -1;
    if (status_local == 0) {
      for (int q = lane; q < ns; q += 32)
        if (scol[q] == i && sstate[q] == SL_LIVE) dslot = q;
      dslot = warp_max_i(dslot);
      if (dslot < 0) status_local = DEV_ESINGULAR;
    }
    // GEPP of the diagonal block, in shared memory when it fits (the stage
    // buffers are free now).  FP64 factor: FP64 in the oracle's operation
    // order.  Mixed factor: FP32 GEPP and 1-norm condition estimate (explicit
    // inverse columns); a block above the threshold, larger than 32, or
    // singular in FP32 is factored again in FP64 and tagged.
    bool tag64 = sizeof(T) == sizeof(double);
    bool lu_sm = false;  // the FP32 pivot LU is in M.lu32
    if (status_local == 0) {
      const T* srcd = wv + soff[dslot];
      unsigned char* gb = stage0;
      const int gcap = 2 * g.stage;
      const bool gs32 = ni * ni * 4 <= gcap, gs64 = ni * ni * 8 <= gcap;
      int* pvs = ni <= PVMAX ? M.pv : nullptr;
      int32_t* gpiv = piv + A.roff[i];
      bool ok = true;
      if (sizeof(T) == sizeof(float)) {
        tag64 = true;
        float* a = gs32 ? reinterpret_cast<float*>(gb) : dg32 + dgoff[i];
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
        const bool small = ni <= 8 && pvs;  // registers; M.pv holds the interchanges
        if (small ? gepp_small(a, ni, pvs, gpiv, lane) : (ni <= 32 && gepp_warp<float>(a, ni, pvs, gpiv, lane))) {
          const float kappa = norm1 * (small ? inv_norm1_small(a, ni, pvs, lane)
                                             : inv_norm1_f32(a, ni, pvs ? pvs : gpiv, lane));
          tag64 = !(kappa <= condf);
          if (!tag64) {
            lu_sm = small;
            for (int e = lane; e < ni * ni; e += 32) {
              if (gs32) dg32[dgoff[i] + e] = a[e];
              dg[dgoff[i] + e] = (double)a[e];
              if (small) M.lu32[e] = a[e];
            }
          }
        }
        __syncwarp();
      }
      if (tag64) {
        double* a = gs64 ? reinterpret_cast<double*>(gb) : dg + dgoff[i];
        for (int e = lane; e < ni * ni; e += 32) a[e] = (double)srcd[e];
        __syncwarp();
        ok = gepp_warp<double>(a, ni, pvs, gpiv, lane);
        if (ok)
          for (int e = lane; e < ni * ni; e += 32) {
            if (gs64) dg[dgoff[i] + e] = a[e];
            if (mixed) dg32[dgoff[i] + e] = (float)a[e];
          }
      }
      __syncwarp();
      if (!ok)
        status_local = DEV_ESINGULAR;
      else if (mixed && lane == 0)
        ptag[i] = tag64 ? 1 : 0;
    }
    // U part: threshold on the blocks right of the diagonal (norm keys kept
    // for lfil)
    if (status_local == 0) {
      for (int q = lane; q < ns; q += 32) {
        const int c = scol[q];
        if (sstate[q] == SL_LIVE && c > i) {
          const int nc = sncl[q];
          bool drop;
          long long kq;
          if (sizeof(T) == sizeof(double)) {
            const double f2 = fro2_batched(wv + soff[q], ni * nc);
            drop = drop_rule(f2, ni, nc, t);
            kq = norm_key(f2);
          } else {
            const float f2 = fro2_f32(wv + soff[q], ni * nc);
            drop = drop_rule_f(f2, ni, nc, tf);
            kq = norm_key(f2);
          }
          sf2[q] = kq;
          if (drop) sstate[q] = SL_DEAD;
        }
      }
      __syncwarp();
    }
    // candidate lists of the kept L blocks and the surviving U blocks, the
    // lfil cut of each, then each part sorted by column; in the stage buffers
    // when they fit, else in the warp's global finish space
    int nL = 0, nU = 0, n2L = 0, n2U = 0;
    int* candL = nullptr;
    int* candU = nullptr;
    unsigned long long* srtL = nullptr;
    unsigned long long* srtU = nullptr;
    if (status_local == 0) {
      int cl = 0, cu = 0;
      for (int q = lane; q < ns; q += 32) {
        const int s = sstate[q];
        cl += s == SL_LKEPT;
        cu += s == SL_LIVE && scol[q] > i;
      }
      cl = warp_sum_i(cl);
      cu = warp_sum_i(cu);
      int p2l = 1, p2u = 1;
      while (p2l < cl) p2l <<= 1;
      while (p2u < cu) p2u <<= 1;
      const int64_t need = 4LL * (cl + cu) + 8LL * (p2l + p2u) + 16;
      if (need <= 2LL * g.stage) {
        candL = reinterpret_cast<int*>(stage0);
        candU = candL + cl;
        srtL = reinterpret_cast<unsigned long long*>(stage0 + ((4LL * (cl + cu) + 15) & ~15LL));
        srtU = srtL + p2l;
      } else {
        candL = ws.fin + wid * 2 * ws.smax;
        candU = candL + ws.smax;
        srtL = ws.srt + wid * 4 * ws.smax;
        srtU = srtL + 2 * ws.smax;
      }
      for (int base = 0; base < ns; base += 32) {
        const int q = base + lane;
        bool isL = false, isU = false;
        if (q < ns) {
          const int s = sstate[q];
          isL = s == SL_LKEPT;
          isU = s == SL_LIVE && scol[q] > i;
        }
        const unsigned bL = __ballot_sync(0xffffffffu, isL), bU = __ballot_sync(0xffffffffu, isU);
        const unsigned lt = (1u << lane) - 1u;
        if (isL) candL[nL + __popc(bL & lt)] = q;
        if (isU) candU[nU + __popc(bU & lt)] = q;
        nL += __popc(bL);
        nU += __popc(bU);
      }
      __syncwarp();
      // lfil: keep the lfil largest of the L part and of the U part
      nL = lfil_cut(candL, nL, lfil, sf2, scol, sstate, M.hist, TS, lane);
      nU = lfil_cut(candU, nU, lfil, sf2, scol, sstate, M.hist, TS, lane);
      n2L = sort_by_column(candL, nL, scol, srtL, lane);
      n2U = sort_by_column(candU, nU, scol, srtU, lane);
    }
    // sizes, then the pool space: the U record and the L blocks
    long long vl = 0, vu = 0;
    unsigned long long lb = 0, lvv = 0, roff16 = 0;
    int64_t rbytes = 0;
    int lu64r = 0;
    if (status_local == 0) {
      for (int p = lane; p < nL; p += 32) vl += (long long)ni * sncl[(int)(srtL[p] & 0xffffffffu)];
      for (int p = lane; p < nU; p += 32) vu += (long long)ni * sncl[(int)(srtU[p] & 0xffffffffu)];
      vl = warp_sum_ll(vl);
      vu = warp_sum_ll(vu);
      lu64r = (sizeof(T) == sizeof(double) || tag64) ? 1 : 0;
      const RecLayout RL = rec_layout(nU, ni, lu64r, vu, TS);
      rbytes = RL.bytes;
      if (lane == 0) {
        lb = atomicAdd(P.ctr + 0, (unsigned long long)nL);
        lvv = atomicAdd(P.ctr + 1, (unsigned long long)vl);
        roff16 = atomicAdd(P.ctr + 2, (unsigned long long)(rbytes / 16));
      }
      lb = __shfl_sync(0xffffffffu, lb, 0);
      lvv = __shfl_sync(0xffffffffu, lvv, 0);
      roff16 = __shfl_sync(0xffffffffu, roff16, 0);
      const bool fits = (int64_t)(lb + nL) <= P.lbcap && (int64_t)(lvv + vl) <= P.lvcap &&
                        (int64_t)roff16 + rbytes / 16 <= P.ucap16 && rbytes / 16 <= kRecMaxUnits &&
                        vu <= INT_MAX;
      if (!fits) status_local = DEV_OVERFLOW;
    }
    // the U record: header, pivots, pivot LU, columns, value offsets, values
    if (status_local == 0) {
      const RecLayout RL = rec_layout(nU, ni, lu64r, vu, TS);
      unsigned char* r = upool + (int64_t)roff16 * 16;
      if (lane == 0) {
        int* h = reinterpret_cast<int*>(r);
        h[0] = nU;
        h[1] = ni;
        h[2] = lu64r;
        h[3] = (int)vu;
      }
      const int32_t* gpiv = piv + A.roff[i];
      for (int a = lane; a < ni; a += 32) reinterpret_cast<int*>(r + RL.piv)[a] = ni <= PVMAX ? M.pv[a] : gpiv[a];
      for (int e = lane; e < ni * ni; e += 32) {
        if (lu64r)
          reinterpret_cast<double*>(r + RL.lu)[e] = dg[dgoff[i] + e];
        else
          reinterpret_cast<float*>(r + RL.lu)[e] = lu_sm ? M.lu32[e] : dg32[dgoff[i] + e];
      }
      int* rcol = reinterpret_cast<int*>(r + RL.ucol);
      int* rrel = reinterpret_cast<int*>(r + RL.urel);
      int* rnjw = reinterpret_cast<int*>(r + RL.unj);
      T* rv = reinterpret_cast<T*>(r + RL.val);
      int carry = 0;
      for (int p0 = 0; p0 < nU; p0 += 32) {
        const int p = p0 + lane;
        int sz = 0, so = 0;
        if (p < nU) {
          const int c = (int)(srtU[p] >> 32), q = (int)(srtU[p] & 0xffffffffu);
          const int nc = sncl[q];
          sz = ni * nc;
          so = soff[q];
          rcol[p] = c;
          rnjw[p] = nc;
        }
        int incl = sz;
        for (int o = 1; o < 32; o <<= 1) {
          const int v = __shfl_up_sync(0xffffffffu, incl, o);
          if (lane >= o) incl += v;
        }
        const int rel = carry + incl - sz;
        if (p < nU) rrel[p] = rel;
        copy_round<T>(M, sz, so, rel, wv, rv, lane);
        carry += __shfl_sync(0xffffffffu, incl, 31);
      }
    }
    if (status_local != 0 && lane == 0) {
      dev_fail(st, status_local);
      atomicExch(P.abort, 1);
      P.lcnt[i] = 0;
      P.lstart[i] = 0;
    }
    if (lane == 0) {  // what the row asked for, to size a retry
      atomicMax(P.ctr + 5, M.nvals);
      atomicMax(P.ctr + 6, (unsigned long long)M.nslots);
    }
    if (P.depth && lane == 0) P.depth[i] = maxdep + 1;
    // publish the row: every lane's writes are made visible device-wide (and
    // to the bulk copies of the readers) before lane 0 sets the word
    fence_proxy_async_all();
    __threadfence();
    __syncwarp();
    if (lane == 0)
      atomicExch(P.done + i, status_local == 0 ? ((unsigned long long)roff16 << 24) | (unsigned long long)(rbytes / 16)
                                               : kRowFailed);
    // the L part is read by no other row: written after publishing, in
    // column order
    if (status_local == 0) {
      long long carry = 0;
      for (int p0 = 0; p0 < nL; p0 += 32) {
        const int p = p0 + lane;
        int sz = 0, so = 0;
        if (p < nL) {
          const int c = (int)(srtL[p] >> 32), q = (int)(srtL[p] & 0xffffffffu);
          sz = ni * sncl[q];
          so = soff[q];
          P.lcol[lb + p] = c;
        }
        int incl = sz;
        for (int o = 1; o < 32; o <<= 1) {
          const int v = __shfl_up_sync(0xffffffffu, incl, o);
          if (lane >= o) incl += v;
        }
        const long long dof = (long long)lvv + carry + incl - sz;
        if (p < nL) P.lvo[lb + p] = dof;
        copy_round<T>(M, sz, so, dof, wv, lval, lane);
        carry += __shfl_sync(0xffffffffu, incl, 31);
      }
      if (lane == 0) {
        P.lstart[i] = (int64_t)lb;
        P.lcnt[i] = nL;
      }
    }
    (void)n2L;
    (void)n2U;
    // clear the hash positions this row used (and the shared hash when the
    // finish staged metadata over it)
    if (in_sh || meta_sh) {
      for (int q = lane; q < g.hash; q += 32) sh_keys[q] = -1;
    }
    if (!in_sh) {
      for (int q = lane; q < ns; q += 32)
        if (hpos[q] >= 0) keys[hpos[q]] = -1;
    }
    __syncwarp();
  }
  drain();
}

// Gather the pooled L rows into VBCSR (warp per row).
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

// U rows from the published records: counts (pass 0), columns (pass 1, after
// the row pointers), values (pass 2, after the value offsets).  A record's
// values are its row's blocks in column order, the VBCSR layout of the row.
template <typename T>
__global__ void k_rec_to_vb(int64_t nbr, int pass, const unsigned long long* __restrict__ done,
                            const unsigned char* __restrict__ upool, int32_t* __restrict__ cnt,
                            const int64_t* __restrict__ bptr, const int64_t* __restrict__ voff,
                            int32_t* __restrict__ bcol, T* __restrict__ val) {
  const int lane = threadIdx.x & 31;
  const int64_t wpb = blockDim.x >> 5;
  for (int64_t i = blockIdx.x * wpb + (threadIdx.x >> 5); i < nbr; i += (int64_t)gridDim.x * wpb) {
    const unsigned char* r = upool + (int64_t)(done[i] >> 24) * 16;
    const int* h = reinterpret_cast<const int*>(r);
    const int ucnt = h[0];
    if (pass == 0) {
      if (lane == 0) cnt[i] = ucnt;
      continue;
    }
    const RecLayout RL = rec_layout(ucnt, h[1], h[2], h[3], (int)sizeof(T));
    if (pass == 1) {
      for (int q = lane; q < ucnt; q += 32) bcol[bptr[i] + q] = reinterpret_cast<const int*>(r + RL.ucol)[q];
      continue;
    }
    const T* src = reinterpret_cast<const T*>(r + RL.val);
    T* dst = val + voff[bptr[i]];
    for (int e = lane; e < h[3]; e += 32) dst[e] = src[e];
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

// Row statistics of the last-level matrix for the choice of the workspace:
// [0] block rows with more than 24 blocks, [1] largest row in blocks.
__global__ void k_row_stats(int64_t nbr, const int64_t* __restrict__ bptr, unsigned long long* __restrict__ out) {
  unsigned long long big = 0, mx = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nbr; i += (int64_t)gridDim.x * blockDim.x) {
    const unsigned long long nb = (unsigned long long)(bptr[i + 1] - bptr[i]);
    big += nb > 24;
    mx = nb > mx ? nb : mx;
  }
  for (int o = 16; o > 0; o >>= 1) {
    big += __shfl_xor_sync(0xffffffffu, big, o);
    const unsigned long long v = __shfl_xor_sync(0xffffffffu, mx, o);
    mx = v > mx ? v : mx;
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(out, big);
    atomicMax(out + 1, mx);
  }
}

}  // namespace

// Shared workspace of one warp: slots, value bytes, stage-buffer bytes and
// pending-column capacity, every part 16-byte aligned.
static IlutGeom make_geom(int slots, int vbytes, int stage, int lcap) {
  IlutGeom G{};
  G.slots = slots;
  G.hash = 1;
  while (G.hash < 2 * slots) G.hash <<= 1;
  G.vbytes = vbytes;
  G.stage = stage;
  G.lcap = lcap;
  auto up = [](int v, int a) { return (v + a - 1) / a * a; };
  int o = 0;
  G.o_misc = o;
  o = up(o + (int)sizeof(IlutMisc), 128);
  G.o_stage = o;
  o += 2 * stage;
  G.o_vals = o;
  o = up(o + vbytes, 16);
  G.o_keys = o;
  o = up(o + 4 * G.hash, 16);
  G.o_hpos = o;
  o = up(o + 4 * slots, 16);
  G.o_scol = o;
  o = up(o + 4 * slots, 16);
  G.o_soff = o;
  o = up(o + 4 * slots, 16);
  G.o_sst = o;
  o = up(o + 4 * slots, 16);
  G.o_sf2 = o;
  o = up(o + 8 * slots, 16);
  G.o_sncl = o;
  o = up(o + 4 * slots, 16);
  G.o_lc = o;
  o = up(o + 4 * lcap, 16);
  G.o_ls = o;
  o = up(o + 4 * lcap, 128);
  G.bytes = o;
  return G;
}



namespace {
// m = the largest a[i]
__global__ void k_max_i32(int64_t n, const int32_t* __restrict__ a, unsigned long long* __restrict__ m) {
  unsigned long long v = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    v = max(v, (unsigned long long)a[i]);
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
  if ((threadIdx.x & 31) == 0 && v) atomicMax(m, v);
}

}  // namespace

template <typename T>
void ilut_last(LastDev<T>& X, double t, int lfil, bool mixed, double cond_thr, uint64_t wait_limit, cudaStream_t s,
               int* dst, const int32_t* order) {
  IlutInfo* info = &X.info;
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
  int nsm = 0, smem_sm = 0, smem_block = 0;
  VB_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  VB_CUDA(cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
  VB_CUDA(cudaDeviceGetAttribute(&smem_block, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  // Shared workspace per warp ("tile shape" of the kernel): chosen by timing
  // the candidates below on a prefix of this matrix's own tickets (every
  // prefix of the ticket order is factored exactly on its own), the fastest
  // kept per device, precision and class of row sizes for the rest of the
  // process; small matrices take the measured default.  The candidates span
  // what the configured workloads were measured to prefer: 64 or 128 slots,
  // 2 to 8 KB of values, 16 down to 6 warps per SM.  The prefix is 1/64 of
  // the tickets (2 048 to 16 384), so the two or three timings add at most about
  // 5 % to the first factorization of a class.
  DBuf<unsigned long long> rstat(2, s);
  rstat.zero();
  launch(k_row_stats, grid_for(p, 256), 256, 0, s, p, A.bptr.p, rstat.p);
  VB_LAUNCH_CHECK();
  const std::vector<unsigned long long> rs = d2h_vec(rstat.p, 2, s);
  const bool wide = rs[0] * 4 > (unsigned long long)p;
  const bool f64 = sizeof(T) == sizeof(double);
  std::vector<IlutGeom> cands;
  cands.push_back((wide && f64) ? make_geom(128, 8192, 2048, 256) : make_geom(64, 2048, 2048, wide ? 256 : 128));
  cands.push_back(make_geom(64, 4096, 2048, 128));
  // Fewer warps per SM means fewer rows in flight; a prefix under-weights
  // that window, which a matrix of narrow rows depends on (on the 3M-unknown
  // workload the prefix preferred 12 warps per SM, which ran the whole matrix
  // 12 % slower than 16), so only wide rows also time the 128-slot shape.
  if (wide) cands.push_back(make_geom(128, f64 ? 8192 : 4096, 2048, 256));
  const int reserve = 1024;  // shared memory the system keeps per block
  // warps per block and blocks per SM of a geometry: the most warps per SM
  // (at most 16)
  auto shape = [&](const IlutGeom& G, int& wpb, int& bps) {
    wpb = 0, bps = 0;
    for (int w = 8; w >= 1; --w) {
      if (w * G.bytes > smem_block) continue;
      int b = smem_sm / (w * G.bytes + reserve);
      while (w * b > 16) --b;
      if (b >= 1 && w * b > wpb * bps) wpb = w, bps = b;
    }
    return wpb >= 1;
  };
  // L pool: the L blocks; U pool: one record per row.  L and U each hold
  // about half of the last-level matrix on the configured workloads; the
  // pools start at its full size and grow on overflow (retry)
  int64_t lbcap = std::max<int64_t>(A.nnzb, 1024), lvcap = std::max<int64_t>(A.nval, 1 << 16);
  int64_t ucap16 = (A.nval * (int64_t)sizeof(T) + X.Dg.nval * 8 + 8 * A.nnzb + 64 * p) / 16 + 4096;
  int smax = 1024;
  int64_t vmax = 32768;
  // buffers of one launch
  struct Run {
    DBuf<int32_t> lcol, lcnt, depth;
    DBuf<int64_t> lvo, lstart;
    DBuf<unsigned long long> done, ctr;
    DBuf<T> lval;
    DBuf<unsigned char> upool;
  };
  // one launch of the kernel over the first nticket tickets with geometry G;
  // returns the device status (the time of the launch in *ms when asked)
  auto run = [&](const IlutGeom& G, int64_t nticket, Run& R, float* ms, bool track = false) -> int {
    int wpb = 0, bps = 0;
    if (!shape(G, wpb, bps)) fail(VB_EINTERNAL, "last-level ILUT: shared workspace exceeds a block");
    const size_t smem = (size_t)wpb * G.bytes;
    const int64_t nblocks = std::max<int64_t>(1, std::min<int64_t>((int64_t)nsm * bps, (nticket + wpb - 1) / wpb));
    const int64_t nwarps = nblocks * wpb;
    int ht = 1;
    while (ht < 2 * smax) ht <<= 1;
    DBuf<int> keys(nwarps * ht, s), hpos(nwarps * smax, s), scol(nwarps * smax, s), sstate(nwarps * smax, s);
    DBuf<int> soff(nwarps * smax, s), sncl(nwarps * smax, s), fin(nwarps * 2 * smax, s);
    DBuf<long long> sf2(nwarps * smax, s);
    DBuf<unsigned long long> srt(nwarps * 4 * smax, s);
    DBuf<T> wvals(nwarps * vmax, s);
    Workspace ws{keys.p, hpos.p, scol.p, soff.p, sstate.p, sf2.p, sncl.p, fin.p, srt.p, ht, smax, vmax};
    R.lcol.alloc(lbcap, s);
    R.lcnt.alloc(p, s);
    R.lvo.alloc(lbcap, s);
    R.lstart.alloc(p, s);
    R.done.alloc(p, s);
    R.lval.alloc(lvcap, s);
    R.upool.alloc(ucap16 * 16, s);
    R.ctr.alloc(8, s);
    if (track) {
      R.depth.alloc(p, s);
      R.depth.zero();
    }
    DBuf<int> abort(1, s);
    R.ctr.zero();
    R.done.zero();
    abort.zero();
    X.piv.zero();
    Pools P{R.lcol.p, R.lvo.p, R.lstart.p, R.lcnt.p, R.done.p, R.ctr.p, lbcap, lvcap, ucap16, abort.p, order,
            nticket, R.depth.p};
    VB_CUDA(cudaFuncSetAttribute(k_ilut<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (ms) {
      VB_CUDA(cudaEventCreate(&e0));
      VB_CUDA(cudaEventCreate(&e1));
      VB_CUDA(cudaEventRecord(e0, s));
    }
    launch(k_ilut<T>, (unsigned)nblocks, wpb * 32, smem, s, A.view(), G, ws, wvals.p, P, R.lval.p, R.upool.p,
           X.Dg.voff.p, X.Dg.val.p, mixed ? X.Dg32.val.p : nullptr, X.piv.p, mixed ? X.ptag.p : nullptr,
           mixed ? 1 : 0, cond_thr, t, lfil, (unsigned long long)wait_limit, dst);
    VB_LAUNCH_CHECK();
    if (ms) {
      VB_CUDA(cudaEventRecord(e1, s));
      VB_CUDA(cudaEventSynchronize(e1));
      VB_CUDA(cudaEventElapsedTime(ms, e0, e1));
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
    }
    if (info) {
      info->warps_per_sm = wpb * bps;
    }
    return d2h(dst, s);
  };
  // the geometry: cached, tuned on a prefix, or the default
  IlutGeom G = cands[0];
  {
    int m1 = 0, m2 = 0;
    const double mb = (double)A.nnzb / (double)p, mv = (double)A.nval / (double)p;
    while ((1 << m1) < mb) ++m1;
    while ((1 << m2) < mv) ++m2;
    const long long key = ((long long)dev << 40) | ((long long)sizeof(T) << 32) | ((long long)wide << 24) |
                          ((long long)m1 << 8) | (long long)m2;
    std::lock_guard<std::mutex> lk(g_geom_mu);
    auto it = g_geom.find(key);
    if (it != g_geom.end()) {
      G = it->second;
      if (info) info->source = 2;
    } else if (p >= kTuneMinRows) {
      const int64_t m = std::min<int64_t>(std::max<int64_t>(p / 64, 2048), 16384);
      const auto t0 = std::chrono::steady_clock::now();
      float best = 0.f;
      int bi = -1;
      for (size_t c = 0; c < cands.size(); ++c) {
        Run R;
        float ms = 0.f;
        const int st = run(cands[c], m, R, &ms);
        if (st != DEV_OK) {
          VB_CUDA(cudaMemsetAsync(dst, 0, sizeof(int), s));
          if (st == DEV_ETIMEOUT || st == DEV_INTERNAL) check_status(dst, s, "last-level ILUT tuning");
          continue;
        }
        if (bi < 0 || ms < best) best = ms, bi = (int)c;
      }
      if (bi >= 0) G = cands[bi];
      g_geom[key] = G;
      if (info) {
        info->source = 1;
        info->tune_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
      }
    }
  }
  if (info) {
    info->slots = G.slots;
    info->vbytes = G.vbytes;
  }
  for (int attempt = 0; attempt < 6; ++attempt) {
    Run R;
    const int st = run(G, p, R, nullptr, true);
    auto& lcol = R.lcol;
    auto& lcnt = R.lcnt;
    auto& lvo = R.lvo;
    auto& lstart = R.lstart;
    auto& done = R.done;
    auto& lval = R.lval;
    auto& upool = R.upool;
    auto& ctr = R.ctr;
    if (st == DEV_OVERFLOW) {
      VB_CUDA(cudaMemsetAsync(dst, 0, sizeof(int), s));
      std::vector<unsigned long long> c = d2h_vec(ctr.p, 8, s);
      lbcap = std::max<int64_t>(2 * lbcap, (int64_t)c[0] + 1024);
      lvcap = std::max<int64_t>(2 * lvcap, (int64_t)c[1] + 4096);
      ucap16 = std::max<int64_t>(2 * ucap16, (int64_t)c[2] + 4096);
      while ((int64_t)c[5] > vmax) vmax *= 2;
      if ((int64_t)c[6] > smax) {
        while (smax < (int)c[6] && smax < MAX_SLOTS) smax *= 2;
        if ((int64_t)c[6] > MAX_SLOTS) fail(VB_ENOMEM, "last-level ILUT: a working row exceeds 4096 blocks");
      }
      continue;
    }
    check_status(dst, s, "vbarms_factor: last-level block ILUT");
    if (info) {  // the longest chain of waits
      DBuf<unsigned long long> mx(1, s);
      mx.zero();
      launch(k_max_i32, grid_for(p, 256), 256, 0, s, p, R.depth.p, mx.p);
      VB_LAUNCH_CHECK();
      info->chain = (long long)d2h(mx.p, s);
    }
    // assemble L from its pool
    {
      VBDev<T>& M = X.L;
      M.bptr.alloc(p + 1, s);
      DBuf<int64_t> c64(p, s);
      launch(k_count_to_i64, grid_for(p, 256), 256, 0, s, p, lcnt.p, c64.p);
      VB_LAUNCH_CHECK();
      scan_i64(c64.p, M.bptr.p, p, s);
      M.nnzb = d2h(M.bptr.p + p, s);
      M.bcol.alloc(M.nnzb, s);
      // bcol first (needed by the offsets), then offsets, then values
      launch(k_pool_to_vb<T>, grid_for(p, 8), 256, 0, s, p, lstart.p, lcol.p, lvo.p, lval.p, M.bptr.p, nullptr,
             M.bcol.p, nullptr);
      VB_LAUNCH_CHECK();
      finish_offsets(M, s);
      launch(k_pool_to_vb<T>, grid_for(p, 8), 256, 0, s, p, lstart.p, lcol.p, lvo.p, lval.p, M.bptr.p, M.voff.p,
             M.bcol.p, M.val.p);
      VB_LAUNCH_CHECK();
    }
    // assemble U from the records
    {
      VBDev<T>& M = X.U;
      M.bptr.alloc(p + 1, s);
      DBuf<int32_t> ucnt(p, s);
      DBuf<int64_t> c64(p, s);
      launch(k_rec_to_vb<T>, grid_for(p, 8), 256, 0, s, p, 0, done.p, upool.p, ucnt.p, nullptr, nullptr, nullptr,
             nullptr);
      launch(k_count_to_i64, grid_for(p, 256), 256, 0, s, p, ucnt.p, c64.p);
      VB_LAUNCH_CHECK();
      scan_i64(c64.p, M.bptr.p, p, s);
      M.nnzb = d2h(M.bptr.p + p, s);
      M.bcol.alloc(M.nnzb, s);
      launch(k_rec_to_vb<T>, grid_for(p, 8), 256, 0, s, p, 1, done.p, upool.p, nullptr, M.bptr.p, nullptr, M.bcol.p,
             nullptr);
      VB_LAUNCH_CHECK();
      finish_offsets(M, s);
      launch(k_rec_to_vb<T>, grid_for(p, 8), 256, 0, s, p, 2, done.p, upool.p, nullptr, M.bptr.p, M.voff.p, M.bcol.p,
             M.val.p);
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
