// Groups of more than one supernode in Step 3 (Section 3: "the diagonal
// blocks D_i of D are block sparse"), and the partial factorization of such
// a level by the two sweeps of Section 3.1 inside each group.
//
// Group ordering (readings of the cited ARMS greedy):
//   supernodes are visited by (weight desc, index asc) (R5); an unmarked
//   eligible one seeds a group, which grows breadth first -- members in the
//   order they joined, each member's neighbours in ascending order -- by
//   unmarked eligible supernodes until it holds gs of them; the members and
//   all their neighbours are then marked.  Every group's marks decide the
//   next seeds, so the greedy is one warp walking the visit order (its
//   lanes test 32 candidates and scan a member's adjacency at a time).  The
//   groups are then listed by their smallest member, members ascending.
//
// Grouped level, every step of a row in the oracle's order:
//   sweep 1, one warp per group, its rows in order: the row of [D, F] in a
//   dense workspace over the group's columns and the union of its members'
//   F columns (the fill of a row stays inside both); each group column
//   k < y still present (fill included) gives m = w_k U_k^{-1} (drop test),
//   w_j -= m ubar_kj over row k of the group part and of W; lfil trims the
//   multipliers; the updated pivot block is GEPP factored; the rest becomes
//   L_y^{-1} P_y w_j (drop test, lfil on the group part and on W apart);
//   sweep 2, one warp per row of [E, C]: the E part in a workspace over the
//   members of the groups it touches, eliminated the same way (G
//   candidates, fill only inside a group), lfil; S = C - G W follows from
//   the Schur kernels of the single-supernode levels.
// Outputs go to per-row slots sized by these bounds and are compacted into
// VBCSR afterwards.
#include <algorithm>
#include <climits>

#include "blockops.cuh"
#include "internal.h"
#include "level.cuh"
#include "vbsr_ops.cuh"

namespace vb {
namespace {

constexpr int GR_GSMAX = 64;      // largest group
constexpr int GR_UCAP = 1024;     // columns of a row's workspace (union of F columns, or G workspace)
constexpr int GR_CCAP = 4096;     // concatenated F columns of a group, before the union
constexpr int GR_WARPS = 2;       // warps per block of the sweeps

int bits_of(unsigned long long x) {
  int b = 0;
  while (b < 64 && (x >> b) != 0) ++b;
  return std::max(b, 1);
}

// ---- symmetric block adjacency without self loops ---------------------------
__global__ void k_gr_pairs(int64_t p, const int64_t* __restrict__ bptr, const int32_t* __restrict__ bcol,
                           unsigned long long* __restrict__ key) {
  const int lane = threadIdx.x & 31;
  const int64_t wpb = blockDim.x >> 5;
  const unsigned long long sentinel = (unsigned long long)p * (unsigned long long)p;
  for (int64_t I = blockIdx.x * wpb + (threadIdx.x >> 5); I < p; I += (int64_t)gridDim.x * wpb)
    for (int64_t b = bptr[I] + lane; b < bptr[I + 1]; b += 32) {
      const unsigned long long J = (unsigned long long)bcol[b];
      if (J == (unsigned long long)I) {
        key[2 * b] = sentinel;
        key[2 * b + 1] = sentinel;
      } else {
        key[2 * b] = (unsigned long long)I * (unsigned long long)p + J;
        key[2 * b + 1] = J * (unsigned long long)p + (unsigned long long)I;
      }
    }
}

__global__ void k_gr_first(int64_t m, unsigned long long sentinel, const unsigned long long* __restrict__ key,
                           int32_t* __restrict__ first) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < m; k += (int64_t)gridDim.x * blockDim.x)
    first[k] = (key[k] != sentinel && (k == 0 || key[k] != key[k - 1])) ? 1 : 0;
}

__global__ void k_gr_unique(int64_t m, int64_t p, const unsigned long long* __restrict__ key,
                            const int32_t* __restrict__ first, const int64_t* __restrict__ pos,
                            int32_t* __restrict__ acol, int32_t* __restrict__ rowcnt) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < m; k += (int64_t)gridDim.x * blockDim.x)
    if (first[k]) {
      const unsigned long long x = key[k];
      const int64_t i = (int64_t)(x / (unsigned long long)p);
      acol[pos[k]] = (int32_t)(x - (unsigned long long)i * (unsigned long long)p);
      atomicAdd(&rowcnt[i], 1);
    }
}

// ---- visit order: weight descending, index ascending (stable sort) ---------
__global__ void k_gr_wkey(int64_t p, const double* __restrict__ w, unsigned long long* __restrict__ key,
                          int32_t* __restrict__ idx) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < p; v += (int64_t)gridDim.x * blockDim.x) {
    key[v] = ~(unsigned long long)__double_as_longlong(w[v]);  // w >= 0: larger weight, smaller key
    idx[v] = (int32_t)v;
  }
}

__global__ void k_gr_fill(int64_t n, int32_t v, int32_t* __restrict__ a) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    a[i] = v;
}

// ---- the greedy, one warp ------------------------------------------------------
__global__ void __launch_bounds__(32) k_gr_greedy(int64_t p, const int32_t* __restrict__ order,
                                                  const int64_t* __restrict__ aptr, const int32_t* __restrict__ acol,
                                                  const double* __restrict__ w, double ddtol,
                                                  const int32_t* __restrict__ fixed, int gs, int32_t* mark,
                                                  int32_t* __restrict__ gid, int* __restrict__ ngroups) {
  __shared__ int32_t grp[GR_GSMAX];
  const int lane = threadIdx.x & 31;
  volatile const int32_t* vm = mark;
  int G = 0;
  for (int64_t base = 0; base < p; base += 32) {
    const int64_t i = base + lane;
    const int v = i < p ? order[i] : -1;
    const bool elig = v >= 0 && !(w[v] < ddtol) && !(fixed && fixed[v]);
    unsigned pend = __ballot_sync(0xffffffffu, elig);
    while (pend) {
      const bool ok = ((pend >> lane) & 1u) && vm[v] == 0;
      const unsigned cand = __ballot_sync(0xffffffffu, ok);
      if (!cand) break;
      const int src = __ffs(cand) - 1;
      const int seed = __shfl_sync(0xffffffffu, v, src);
      pend &= ~((2u << src) - 1u);
      if (lane == 0) {
        grp[0] = seed;
        mark[seed] = 1;
        gid[seed] = G;
      }
      __syncwarp();
      int n = 1;
      for (int head = 0; head < n && n < gs; ++head) {
        const int u = grp[head];
        const int64_t a1 = aptr[u + 1];
        for (int64_t a0 = aptr[u]; a0 < a1 && n < gs; a0 += 32) {
          const int64_t a = a0 + lane;
          int z = -1;
          bool take = false;
          if (a < a1) {
            z = acol[a];
            take = vm[z] == 0 && !(w[z] < ddtol) && !(fixed && fixed[z]);
          }
          const unsigned tm = __ballot_sync(0xffffffffu, take);
          const int rank = __popc(tm & ((1u << lane) - 1u));
          const int room = gs - n;
          if (take && rank < room) {
            grp[n + rank] = z;
            mark[z] = 1;
            gid[z] = G;
          }
          n += min(__popc(tm), room);
          __syncwarp();
        }
      }
      for (int k = 0; k < n; ++k) {
        const int u = grp[k];
        for (int64_t a = aptr[u] + lane; a < aptr[u + 1]; a += 32) mark[acol[a]] = 1;
      }
      __syncwarp();
      ++G;
    }
  }
  if (lane == 0) *ngroups = G;
}

// The same greedy with the marks and the eligibility flags as bit masks in
// shared memory (level matrices of up to GR_SHMAX supernodes): mark tests
// cost a shared load, and the members' neighbours are marked in one pass
// over their flattened adjacency.  Same result as k_gr_greedy.
constexpr int64_t GR_SHMAX = 880000;  // supernodes whose two masks fit in 220 KB

__global__ void k_gr_elig(int64_t p, const double* __restrict__ w, double ddtol, const int32_t* __restrict__ fixed,
                          uint32_t* __restrict__ elig) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < p; v += (int64_t)gridDim.x * blockDim.x) {
    if (!(w[v] < ddtol) && !(fixed && fixed[v])) atomicOr(&elig[v >> 5], 1u << (v & 31));
  }
}

__global__ void __launch_bounds__(32) k_gr_greedy_sh(int64_t p, const int32_t* __restrict__ order,
                                                     const int64_t* __restrict__ aptr,
                                                     const int32_t* __restrict__ acol,
                                                     const uint32_t* __restrict__ elig_g, int gs,
                                                     int32_t* __restrict__ gid, int* __restrict__ ngroups) {
  extern __shared__ uint32_t gr_sh[];
  __shared__ int32_t grp[GR_GSMAX];
  __shared__ int64_t nb0[GR_GSMAX];
  __shared__ int32_t nbc[GR_GSMAX + 1];
  const int lane = threadIdx.x & 31;
  const int64_t nwd = (p + 31) >> 5;
  uint32_t* mark = gr_sh;
  uint32_t* elig = gr_sh + nwd;
  for (int64_t q = lane; q < nwd; q += 32) {
    mark[q] = 0u;
    elig[q] = elig_g[q];
  }
  __syncwarp();
  auto marked = [&](int v) { return (mark[v >> 5] >> (v & 31)) & 1u; };
  auto eligible = [&](int v) { return (elig[v >> 5] >> (v & 31)) & 1u; };
  auto setmark = [&](int v) { atomicOr(&mark[v >> 5], 1u << (v & 31)); };
  int G = 0;
  for (int64_t base = 0; base < p; base += 32) {
    const int64_t i = base + lane;
    const int v = i < p ? order[i] : -1;
    const bool el = v >= 0 && eligible(v);
    unsigned pend = __ballot_sync(0xffffffffu, el);
    while (pend) {
      const bool ok = ((pend >> lane) & 1u) && !marked(v);
      const unsigned cand = __ballot_sync(0xffffffffu, ok);
      if (!cand) break;
      const int src = __ffs(cand) - 1;
      const int seed = __shfl_sync(0xffffffffu, v, src);
      pend &= ~((2u << src) - 1u);
      if (lane == 0) {
        grp[0] = seed;
        setmark(seed);
        gid[seed] = G;
      }
      __syncwarp();
      int n = 1;
      for (int head = 0; head < n && n < gs; ++head) {
        const int u = grp[head];
        const int64_t a1 = aptr[u + 1];
        for (int64_t a0 = aptr[u]; a0 < a1 && n < gs; a0 += 32) {
          const int64_t a = a0 + lane;
          int z = -1;
          bool take = false;
          if (a < a1) {
            z = acol[a];
            take = !marked(z) && eligible(z);
          }
          const unsigned tm = __ballot_sync(0xffffffffu, take);
          const int rank = __popc(tm & ((1u << lane) - 1u));
          const int room = gs - n;
          if (take && rank < room) {
            grp[n + rank] = z;
            setmark(z);
            gid[z] = G;
          }
          n += min(__popc(tm), room);
          __syncwarp();
        }
      }
      // every member's neighbours, in one pass over the flattened lists
      for (int k = lane; k < n; k += 32) {
        const int u = grp[k];
        nb0[k] = aptr[u];
        nbc[k] = (int32_t)(aptr[u + 1] - aptr[u]);
      }
      __syncwarp();
      if (lane == 0) {
        int acc = 0;
        for (int k = 0; k < n; ++k) {
          const int c = nbc[k];
          nbc[k] = acc;
          acc += c;
        }
        nbc[n] = acc;
      }
      __syncwarp();
      const int tot = nbc[n];
      int k = 0;
      for (int e = lane; e < tot; e += 32) {
        while (nbc[k + 1] <= e) ++k;
        setmark(acol[nb0[k] + (e - nbc[k])]);
      }
      __syncwarp();
      ++G;
    }
  }
  if (lane == 0) *ngroups = G;
}

// ---- group ranks and the ordering ------------------------------------------
__global__ void k_gr_gmin(int64_t p, const int32_t* __restrict__ gid, int32_t* __restrict__ gmin,
                          int32_t* __restrict__ gcnt) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < p; v += (int64_t)gridDim.x * blockDim.x)
    if (gid[v] >= 0) {
      atomicMin(&gmin[gid[v]], (int32_t)v);
      atomicAdd(&gcnt[gid[v]], 1);
    }
}

__global__ void k_gr_gkey(int64_t ng, const int32_t* __restrict__ gmin, unsigned long long* __restrict__ key) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < ng; g += (int64_t)gridDim.x * blockDim.x)
    key[g] = ((unsigned long long)(uint32_t)gmin[g] << 32) | (unsigned long long)g;
}

__global__ void k_gr_rank(int64_t ng, const unsigned long long* __restrict__ key, const int32_t* __restrict__ gcnt,
                          int32_t* __restrict__ rank, int32_t* __restrict__ rsize) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < ng; q += (int64_t)gridDim.x * blockDim.x) {
    const int32_t g = (int32_t)(key[q] & 0xffffffffull);
    rank[g] = (int32_t)q;
    rsize[q] = gcnt[g];
  }
}

__global__ void k_gr_flags(int64_t p, const int32_t* __restrict__ gid, int32_t* __restrict__ inD,
                           int32_t* __restrict__ inC) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < p; v += (int64_t)gridDim.x * blockDim.x) {
    inD[v] = gid[v] >= 0 ? 1 : 0;
    inC[v] = gid[v] >= 0 ? 0 : 1;
  }
}

// D members keyed by (group rank, member); C rows placed ascending.
__global__ void k_gr_place(int64_t p, int64_t nD, const int32_t* __restrict__ gid, const int32_t* __restrict__ rank,
                           const int64_t* __restrict__ sD, const int64_t* __restrict__ sC,
                           unsigned long long* __restrict__ mkey, int32_t* __restrict__ pI) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < p; v += (int64_t)gridDim.x * blockDim.x) {
    if (gid[v] >= 0)
      mkey[sD[v]] = ((unsigned long long)(uint32_t)rank[gid[v]] << 32) | (unsigned long long)v;
    else
      pI[nD + sC[v]] = (int32_t)v;
  }
}

__global__ void k_gr_dlist(int64_t nD, const unsigned long long* __restrict__ mkey, int32_t* __restrict__ pI) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nD; q += (int64_t)gridDim.x * blockDim.x)
    pI[q] = (int32_t)(mkey[q] & 0xffffffffull);
}

__global__ void k_gr_newpos(int64_t p, const int32_t* __restrict__ pI, int32_t* __restrict__ newpos) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < p; k += (int64_t)gridDim.x * blockDim.x)
    newpos[pI[k]] = (int32_t)k;
}

}  // namespace

namespace {

// ---- gather of a grouped level -------------------------------------------------
// PASS 0: counts of the D (group), F, E, C blocks of every new row; PASS 1:
// columns (new numbering) and source blocks, in A's column order (ascending
// for D, F, C; E rows are sorted afterwards).
template <int PASS>
__global__ void k_gr_gather(int64_t p, int64_t nD, const int64_t* __restrict__ bptr, const int32_t* __restrict__ bcol,
                            const int32_t* __restrict__ newpos, int32_t* __restrict__ cD, int32_t* __restrict__ cF,
                            int32_t* __restrict__ cE, int32_t* __restrict__ cC, const int64_t* __restrict__ pD,
                            const int64_t* __restrict__ pF, const int64_t* __restrict__ pE,
                            const int64_t* __restrict__ pC, int32_t* __restrict__ colD, int32_t* __restrict__ colF,
                            int32_t* __restrict__ colE, int32_t* __restrict__ colC, int64_t* __restrict__ srcD,
                            int64_t* __restrict__ srcF, int64_t* __restrict__ srcE, int64_t* __restrict__ srcC) {
  const int lane = threadIdx.x & 31;
  const int64_t wpb = blockDim.x >> 5;
  for (int64_t Y = blockIdx.x * wpb + (threadIdx.x >> 5); Y < p; Y += (int64_t)gridDim.x * wpb) {
    const int64_t k = newpos[Y];
    const bool rowD = k < nD;
    int64_t oX = 0, oY = 0;
    if (PASS == 1) {
      oX = rowD ? pD[k] : pE[k - nD];
      oY = rowD ? pF[k] : pC[k - nD];
    }
    int nX = 0, nY = 0;
    for (int64_t b0 = bptr[Y]; b0 < bptr[Y + 1]; b0 += 32) {
      const int64_t b = b0 + lane;
      const bool valid = b < bptr[Y + 1];
      const int64_t nz = valid ? newpos[bcol[b]] : -1;
      const bool toX = valid && nz < nD;   // D (row in D) or E
      const bool toY = valid && nz >= nD;  // F (row in D) or C
      const unsigned mX = __ballot_sync(0xffffffffu, toX), mY = __ballot_sync(0xffffffffu, toY);
      if (PASS == 1) {
        const unsigned lt = (1u << lane) - 1u;
        if (toX) {
          const int64_t d = oX + __popc(mX & lt);
          (rowD ? colD : colE)[d] = (int32_t)nz;
          (rowD ? srcD : srcE)[d] = b;
        }
        if (toY) {
          const int64_t d = oY + __popc(mY & lt);
          (rowD ? colF : colC)[d] = (int32_t)(nz - nD);
          (rowD ? srcF : srcC)[d] = b;
        }
        oX += __popc(mX);
        oY += __popc(mY);
      }
      nX += __popc(mX);
      nY += __popc(mY);
    }
    if (PASS == 0 && lane == 0) {
      if (rowD) {
        cD[k] = nX;
        cF[k] = nY;
      } else {
        cE[k - nD] = nX;
        cC[k - nD] = nY;
      }
    }
  }
}

// Sort every row's (column, source) pairs by column (columns unique in a
// row): each entry's rank is the number of smaller columns.
__global__ void k_gr_sort_rows(int64_t nrows, const int64_t* __restrict__ bptr, const int32_t* __restrict__ cin,
                               const int64_t* __restrict__ sin, int32_t* __restrict__ cout,
                               int64_t* __restrict__ sout) {
  const int lane = threadIdx.x & 31;
  const int64_t wpb = blockDim.x >> 5;
  for (int64_t r = blockIdx.x * wpb + (threadIdx.x >> 5); r < nrows; r += (int64_t)gridDim.x * wpb) {
    const int64_t b0 = bptr[r], b1 = bptr[r + 1];
    for (int64_t b = b0 + lane; b < b1; b += 32) {
      const int32_t c = cin[b];
      int64_t rk = 0;
      for (int64_t q = b0; q < b1; ++q) rk += cin[q] < c ? 1 : 0;
      cout[b0 + rk] = c;
      sout[b0 + rk] = sin[b];
    }
  }
}

template <typename TS, typename TD>
__global__ void k_gr_copy_blocks(int64_t nblocks, const int64_t* __restrict__ src, const int64_t* __restrict__ svoff,
                                 const TS* __restrict__ sval, const int64_t* __restrict__ dvoff,
                                 TD* __restrict__ dval) {
  const int lane = threadIdx.x & 31;
  const int64_t wpb = blockDim.x >> 5;
  for (int64_t d = blockIdx.x * wpb + (threadIdx.x >> 5); d < nblocks; d += (int64_t)gridDim.x * wpb) {
    const int64_t b = src[d];
    const int64_t n = svoff[b + 1] - svoff[b];
    for (int64_t e = lane; e < n; e += 32) dval[dvoff[d] + e] = (TD)sval[svoff[b] + e];
  }
}

__global__ void k_gr_group_of(int64_t ng, const int64_t* __restrict__ gptr, int32_t* __restrict__ dgid) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < ng; g += (int64_t)gridDim.x * blockDim.x)
    for (int64_t y = gptr[g]; y < gptr[g + 1]; ++y) dgid[y] = (int32_t)g;
}

// ---- warp helpers ----------------------------------------------------------
__device__ void gr_bitonic(int32_t* a, int n2, int lane) {
  for (int k = 2; k <= n2; k <<= 1)
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = lane; i < n2; i += 32) {
        const int l = i ^ j;
        if (l > i) {
          const bool up = (i & k) == 0;
          const int32_t x = a[i], y = a[l];
          if ((x > y) == up) {
            a[i] = y;
            a[l] = x;
          }
        }
      }
      __syncwarp();
    }
}

__device__ __forceinline__ int gr_find(const int32_t* a, int n, int32_t key) {
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

// w (r x n) -= m (r x k) * u (k x n): lanes over the elements of w, each
// element's terms in order (the oracle's sub_prod)
template <typename TU>
__device__ __forceinline__ void gr_sub_prod(double* w, const double* m, const TU* u, int r, int k, int n, int lane) {
  for (int e = lane; e < r * n; e += 32) {
    const int i = e / n, j = e - i * n;
    double a = w[e];
    for (int q = 0; q < k; ++q) a = __dsub_rn(a, __dmul_rn(m[i * k + q], (double)u[q * n + j]));
    w[e] = a;
  }
}

// x (r x m) <- x U^{-1}, rows over lanes (the oracle's apply_Uinv_right per row)
__device__ __forceinline__ void gr_uinv_right(const double* lu, int m, double* x, int r, int lane) {
  for (int i = lane; i < r; i += 32) uinv_right_block<double, double>(lu, m, x + i * m, 1);
}

// x (m x n) <- L^{-1} P x, columns over lanes (the oracle's apply_LinvP per column)
__device__ __forceinline__ void gr_linvp(const double* lu, const int32_t* pv, int m, double* x, int n, int lane) {
  for (int j = lane; j < n; j += 32) {
    for (int k = 0; k < m; ++k)
      if (pv[k] != k) {
        const double t = x[k * n + j];
        x[k * n + j] = x[pv[k] * n + j];
        x[pv[k] * n + j] = t;
      }
    for (int i = 1; i < m; ++i)
      for (int k = 0; k < i; ++k) x[i * n + j] = __dsub_rn(x[i * n + j], __dmul_rn(lu[i * m + k], x[k * n + j]));
  }
}

// Keep at most lfil of n candidates (largest f2, lower column on ties); the
// kept ones flagged in keep[].  The warp's lanes rank one candidate each.
__device__ void gr_lfil(int n, const int32_t* col, const double* f2, int8_t* keep, int lfil, int lane) {
  __syncwarp();
  const bool all = lfil < 0 || n <= lfil;
  for (int i = lane; i < n; i += 32) {
    int better = 0;
    if (!all)
      for (int j = 0; j < n; ++j)
        if (f2[j] > f2[i] || (f2[j] == f2[i] && col[j] < col[i])) ++better;
    keep[i] = all || better < lfil ? 1 : 0;
  }
  __syncwarp();
}

// ---- F-column union of every group -----------------------------------------
// ulist[F.bptr[gptr[g]] ...] = the sorted union of the group members' F
// columns; ucnt[g], uwid[g] (scalar width).  Fails with DEV_OVERFLOW when a
// union exceeds GR_UCAP blocks.
__global__ void __launch_bounds__(GR_WARPS * 32)
    k_gr_union(int64_t ng, const int64_t* __restrict__ gptr, const int64_t* __restrict__ Fbptr,
               const int32_t* __restrict__ Fbcol, const int32_t* __restrict__ csz, int32_t* __restrict__ ulist,
               int32_t* __restrict__ ucnt, int64_t* __restrict__ uwid, int* st) {
  __shared__ int32_t buf[GR_WARPS][GR_CCAP];
  const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
  int32_t* a = buf[wi];
  for (int64_t g = blockIdx.x * GR_WARPS + wi; g < ng; g += (int64_t)gridDim.x * GR_WARPS) {
    const int64_t b0 = Fbptr[gptr[g]], b1 = Fbptr[gptr[g + 1]];
    const int64_t n = b1 - b0;
    if (n > GR_CCAP) {
      if (lane == 0) {
        dev_fail(st, DEV_OVERFLOW);
        ucnt[g] = 0;
        uwid[g] = 0;
      }
      continue;
    }
    int n2 = 1;
    while (n2 < n) n2 <<= 1;
    for (int i = lane; i < n2; i += 32) a[i] = i < n ? Fbcol[b0 + i] : INT_MAX;
    __syncwarp();
    gr_bitonic(a, n2, lane);
    int cnt = 0;
    long long wid = 0;
    for (int i0 = 0; i0 < n; i0 += 32) {
      const int i = i0 + lane;
      const bool keep = i < n && (i == 0 || a[i] != a[i - 1]);
      const int32_t c = i < n ? a[i] : 0;
      const unsigned km = __ballot_sync(0xffffffffu, keep);
      if (keep) ulist[b0 + cnt + __popc(km & ((1u << lane) - 1u))] = c;
      wid += keep ? csz[c] : 0;
      cnt += __popc(km);
    }
    wid = warp_sum_ll(wid);
    if (lane == 0) {
      ucnt[g] = cnt;
      uwid[g] = wid;
      if (cnt > GR_UCAP) dev_fail(st, DEV_OVERFLOW);
    }
    __syncwarp();
  }
}

// Per-row slot capacities of sweep 1: Lg and Ug rows take at most the group's
// size in blocks and ny times its scalar width in values; W rows the union's.
__global__ void k_gr_caps1(int64_t ng, const int64_t* __restrict__ gptr, const int32_t* __restrict__ dsz,
                           const int32_t* __restrict__ ucnt, const int64_t* __restrict__ uwid,
                           int64_t* __restrict__ capG, int64_t* __restrict__ vcapG, int64_t* __restrict__ capW,
                           int64_t* __restrict__ vcapW) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < ng; g += (int64_t)gridDim.x * blockDim.x) {
    int64_t gw = 0;
    for (int64_t y = gptr[g]; y < gptr[g + 1]; ++y) gw += dsz[y];
    for (int64_t y = gptr[g]; y < gptr[g + 1]; ++y) {
      capG[y] = gptr[g + 1] - gptr[g];
      vcapG[y] = (int64_t)dsz[y] * gw;
      capW[y] = ucnt[g];
      vcapW[y] = (int64_t)dsz[y] * uwid[g];
    }
  }
}

// Per-row capacities of sweep 2: the members of the groups an E row touches.
__global__ void k_gr_caps2(int64_t nC, const int64_t* __restrict__ Ebptr, const int32_t* __restrict__ Ebcol,
                           const int32_t* __restrict__ dgid, const int64_t* __restrict__ gptr,
                           const int64_t* __restrict__ droff, const int32_t* __restrict__ csz,
                           int64_t* __restrict__ cap, int64_t* __restrict__ vcap) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < nC; r += (int64_t)gridDim.x * blockDim.x) {
    int64_t nb = 0, sw = 0;
    int last = -1;
    for (int64_t b = Ebptr[r]; b < Ebptr[r + 1]; ++b) {
      const int g = dgid[Ebcol[b]];
      if (g == last) continue;
      last = g;
      nb += gptr[g + 1] - gptr[g];
      sw += droff[gptr[g + 1]] - droff[gptr[g]];
    }
    cap[r] = nb;
    vcap[r] = (int64_t)csz[r] * sw;
  }
}

// ---- sweep 1: one warp per group --------------------------------------------
struct GrOut {  // per-row slots of one output matrix
  const int64_t* slot;  // first block slot of the row
  const int64_t* vslot;  // first value slot of the row
  int32_t* col;         // slot columns
  int32_t* cnt;         // kept blocks per row
};

template <typename T>
__global__ void __launch_bounds__(GR_WARPS * 32)
    k_gr_sweep1(int64_t ng, const int64_t* __restrict__ gptr, VBView<double> Dm, VBView<T> F,
                const int32_t* __restrict__ ulist, const int32_t* __restrict__ ucnt, const int32_t* __restrict__ Csz,
                const int64_t* __restrict__ Dvo, double* __restrict__ Dlu, int32_t* __restrict__ piv,
                GrOut oL, T* __restrict__ Lv, GrOut oU, T* __restrict__ Uv, GrOut oW, T* __restrict__ Wv,
                double* __restrict__ wsall, int64_t wcap, double t, int lfil, int* st) {
  __shared__ int32_t s_ucol[GR_WARPS][GR_UCAP];
  __shared__ int32_t s_uoff[GR_WARPS][GR_UCAP + 1];
  __shared__ int8_t s_fp[GR_WARPS][GR_UCAP];
  __shared__ int8_t s_keep[GR_WARPS][GR_UCAP];
  __shared__ double s_f2[GR_WARPS][GR_UCAP];
  __shared__ int32_t s_cc[GR_WARPS][GR_UCAP];
  __shared__ int32_t s_doff[GR_WARPS][GR_GSMAX + 1];
  __shared__ int8_t s_dp[GR_WARPS][GR_GSMAX];
  const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
  const int64_t gw = (int64_t)blockIdx.x * GR_WARPS + wi;
  double* ws = wsall + gw * wcap;
  int32_t* ucol = s_ucol[wi];
  int32_t* uoff = s_uoff[wi];
  int8_t* fp = s_fp[wi];
  int8_t* keep = s_keep[wi];
  double* f2 = s_f2[wi];
  int32_t* cc = s_cc[wi];
  int32_t* doff = s_doff[wi];
  int8_t* dp = s_dp[wi];
  for (int64_t g = gw; g < ng; g += (int64_t)gridDim.x * GR_WARPS) {
    const int64_t y0 = gptr[g], y1 = gptr[g + 1];
    const int gsz = (int)(y1 - y0);
    const int nu = ucnt[g];
    const int64_t ub = F.bptr[y0];
    for (int u = lane; u < nu; u += 32) ucol[u] = ulist[ub + u];
    __syncwarp();
    if (lane == 0) {
      int o = 0;
      for (int u = 0; u < nu; ++u) {
        uoff[u] = o;
        o += Csz[ucol[u]];
      }
      uoff[nu] = o;
      o = 0;
      for (int k = 0; k < gsz; ++k) {
        doff[k] = o;
        o += Dm.rsz[y0 + k];
      }
      doff[gsz] = o;
    }
    __syncwarp();
    const int uw = uoff[nu], gwid = doff[gsz];
    for (int64_t y = y0; y < y1; ++y) {
      const int yy = (int)(y - y0);
      const int ny = Dm.rsz[y];
      double* wF = ws;                   // F part: block u at ny * uoff[u]
      double* wD = ws + (int64_t)ny * uw;  // group part: member kk at ny * doff[kk]
      if ((int64_t)ny * (uw + gwid) > wcap) {
        if (lane == 0) dev_fail(st, DEV_OVERFLOW);
        break;
      }
      for (int64_t e = lane; e < (int64_t)ny * (uw + gwid); e += 32) ws[e] = 0.0;
      for (int u = lane; u < nu; u += 32) fp[u] = 0;
      for (int k = lane; k < gsz; k += 32) dp[k] = 0;
      __syncwarp();
      // the row of [D, F]
      for (int64_t b = F.bptr[y]; b < F.bptr[y + 1]; ++b) {
        const int u = gr_find(ucol, nu, F.bcol[b]);
        if (u < 0) {
          if (lane == 0) dev_fail(st, DEV_INTERNAL);
          continue;
        }
        const int n = ny * F.csz[F.bcol[b]];
        for (int e = lane; e < n; e += 32) wF[(int64_t)ny * uoff[u] + e] = (double)F.val[F.voff[b] + e];
        if (lane == 0) fp[u] = 1;
      }
      for (int64_t b = Dm.bptr[y]; b < Dm.bptr[y + 1]; ++b) {
        const int kk = Dm.bcol[b] - (int)y0;
        const int n = ny * Dm.rsz[y0 + kk];
        for (int e = lane; e < n; e += 32) wD[(int64_t)ny * doff[kk] + e] = Dm.val[Dm.voff[b] + e];
        if (lane == 0) dp[kk] = 1;
      }
      __syncwarp();
      // L part: group columns before y, ascending, fill included
      int nl = 0;
      for (int kk = 0; kk < yy; ++kk) {
        if (!dp[kk]) continue;
        const int64_t k = y0 + kk;
        const int nk = Dm.rsz[k];
        double* m = wD + (int64_t)ny * doff[kk];
        gr_uinv_right(Dlu + Dvo[k], nk, m, ny, lane);
        __syncwarp();
        double fr = 0.0;
        if (lane == 0) fr = fro2_d(m, ny * nk);
        fr = __shfl_sync(0xffffffffu, fr, 0);
        if (drop_rule(fr, ny, nk, t)) {
          if (lane == 0) dp[kk] = 0;
          __syncwarp();
          continue;
        }
        // updates from row k of Ubar (group part) and of W
        const int64_t us = oU.slot[k], uvs = oU.vslot[k];
        int64_t vo = uvs;
        for (int q = 0; q < oU.cnt[k]; ++q) {
          const int jj = oU.col[us + q] - (int)y0;
          const int nj = Dm.rsz[y0 + jj];
          gr_sub_prod<T>(wD + (int64_t)ny * doff[jj], m, Uv + vo, ny, nk, nj, lane);
          if (lane == 0) dp[jj] = 1;
          vo += (int64_t)nk * nj;
        }
        const int64_t ws0 = oW.slot[k];
        vo = oW.vslot[k];
        for (int q = 0; q < oW.cnt[k]; ++q) {
          const int32_t c = oW.col[ws0 + q];
          const int u = gr_find(ucol, nu, c);
          const int nc = Csz[c];
          if (u < 0) {
            if (lane == 0) dev_fail(st, DEV_INTERNAL);
            vo += (int64_t)nk * nc;
            continue;
          }
          gr_sub_prod<T>(wF + (int64_t)ny * uoff[u], m, Wv + vo, ny, nk, nc, lane);
          if (lane == 0) fp[u] = 1;
          vo += (int64_t)nk * nc;
        }
        if (lane == 0) {
          cc[nl] = (int32_t)k;
          f2[nl] = fr;
          dp[kk] = 2;  // a kept multiplier, no longer part of the row
        }
        ++nl;
        __syncwarp();
      }
      // lfil on the multipliers, then the kept ones in ascending column order
      gr_lfil(nl, cc, f2, keep, lfil, lane);
      {
        int64_t vo = oL.vslot[y];
        int c = 0;
        for (int q = 0; q < nl; ++q) {
          if (!keep[q]) continue;
          const int kk = cc[q] - (int)y0;
          const int nk = Dm.rsz[cc[q]];
          const double* m = wD + (int64_t)ny * doff[kk];
          for (int e = lane; e < ny * nk; e += 32) Lv[vo + e] = (T)m[e];
          if (lane == 0) oL.col[oL.slot[y] + c] = cc[q];
          vo += (int64_t)ny * nk;
          ++c;
        }
        if (lane == 0) oL.cnt[y] = c;
      }
      __syncwarp();
      // the pivot block
      if (!dp[yy]) {
        if (lane == 0) dev_fail(st, DEV_ESINGULAR);
        break;
      }
      double* lu = Dlu + Dvo[y];
      int32_t* pv = piv + Dm.roff[y];
      for (int e = lane; e < ny * ny; e += 32) lu[e] = wD[(int64_t)ny * doff[yy] + e];
      __syncwarp();
      const bool ok = gepp_block_warp(lu, ny, pv, lane);
      if (!ok) {
        if (lane == 0) dev_fail(st, DEV_ESINGULAR);
        break;
      }
      __syncwarp();
      // U part, group columns after y: L_y^{-1} P_y w_j, drop test, lfil
      int nc = 0;
      for (int jj = yy + 1; jj < gsz; ++jj) {
        if (!dp[jj]) continue;
        const int nj = Dm.rsz[y0 + jj];
        double* x = wD + (int64_t)ny * doff[jj];
        gr_linvp(lu, pv, ny, x, nj, lane);
        __syncwarp();
        double fr = 0.0;
        if (lane == 0) fr = fro2_d(x, ny * nj);
        fr = __shfl_sync(0xffffffffu, fr, 0);
        if (!drop_rule(fr, ny, nj, t)) {
          if (lane == 0) {
            cc[nc] = (int32_t)(y0 + jj);
            f2[nc] = fr;
          }
          ++nc;
        }
        __syncwarp();
      }
      gr_lfil(nc, cc, f2, keep, lfil, lane);
      {
        int64_t vo = oU.vslot[y];
        int c = 0;
        for (int q = 0; q < nc; ++q) {
          if (!keep[q]) continue;
          const int jj = cc[q] - (int)y0;
          const int nj = Dm.rsz[cc[q]];
          const double* x = wD + (int64_t)ny * doff[jj];
          for (int e = lane; e < ny * nj; e += 32) Uv[vo + e] = (T)x[e];
          if (lane == 0) oU.col[oU.slot[y] + c] = cc[q];
          vo += (int64_t)ny * nj;
          ++c;
        }
        if (lane == 0) oU.cnt[y] = c;
      }
      __syncwarp();
      // W part
      nc = 0;
      for (int u = 0; u < nu; ++u) {
        if (!fp[u]) continue;
        const int ns = Csz[ucol[u]];
        double* x = wF + (int64_t)ny * uoff[u];
        gr_linvp(lu, pv, ny, x, ns, lane);
        __syncwarp();
        double fr = 0.0;
        if (lane == 0) fr = fro2_d(x, ny * ns);
        fr = __shfl_sync(0xffffffffu, fr, 0);
        if (!drop_rule(fr, ny, ns, t)) {
          if (lane == 0) {
            cc[nc] = u;
            f2[nc] = fr;
          }
          ++nc;
        }
        __syncwarp();
      }
      // lfil compares columns: the union is sorted, so u orders like the column
      gr_lfil(nc, cc, f2, keep, lfil, lane);
      {
        int64_t vo = oW.vslot[y];
        int c = 0;
        for (int q = 0; q < nc; ++q) {
          if (!keep[q]) continue;
          const int u = cc[q];
          const int ns = Csz[ucol[u]];
          const double* x = wF + (int64_t)ny * uoff[u];
          for (int e = lane; e < ny * ns; e += 32) Wv[vo + e] = (T)x[e];
          if (lane == 0) oW.col[oW.slot[y] + c] = ucol[u];
          vo += (int64_t)ny * ns;
          ++c;
        }
        if (lane == 0) oW.cnt[y] = c;
      }
      __syncwarp();
    }
  }
}

// ---- sweep 2: one warp per row of [E, C] ------------------------------------
template <typename T>
__global__ void __launch_bounds__(GR_WARPS * 32)
    k_gr_sweep2(int64_t nC, VBView<T> E, const int32_t* __restrict__ dgid, const int64_t* __restrict__ gptr,
                const int32_t* __restrict__ dsz, const int64_t* __restrict__ Dvo, const double* __restrict__ Dlu,
                GrOut oU, const T* __restrict__ Uv, GrOut oG, T* __restrict__ Gv, double* __restrict__ wsall,
                int64_t wcap, double t, int lfil, int* st) {
  __shared__ int32_t s_col[GR_WARPS][GR_UCAP];
  __shared__ int32_t s_off[GR_WARPS][GR_UCAP + 1];
  __shared__ int8_t s_pr[GR_WARPS][GR_UCAP];
  __shared__ int8_t s_keep[GR_WARPS][GR_UCAP];
  __shared__ double s_f2[GR_WARPS][GR_UCAP];
  __shared__ int32_t s_cc[GR_WARPS][GR_UCAP];
  const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
  const int64_t gw = (int64_t)blockIdx.x * GR_WARPS + wi;
  double* ws = wsall + gw * wcap;
  int32_t* col = s_col[wi];
  int32_t* off = s_off[wi];
  int8_t* pr = s_pr[wi];
  int8_t* keep = s_keep[wi];
  double* f2 = s_f2[wi];
  int32_t* cc = s_cc[wi];
  for (int64_t r = gw; r < nC; r += (int64_t)gridDim.x * GR_WARPS) {
    const int nr = E.rsz[r];
    // the workspace columns: every member of the groups the row touches
    if (lane == 0) {
      int n = 0, o = 0, last = -1;
      bool over = false;
      for (int64_t b = E.bptr[r]; b < E.bptr[r + 1] && !over; ++b) {
        const int g = dgid[E.bcol[b]];
        if (g == last) continue;
        last = g;
        for (int64_t y = gptr[g]; y < gptr[g + 1]; ++y) {
          if (n >= GR_UCAP) {
            over = true;
            break;
          }
          col[n] = (int32_t)y;
          off[n] = o;
          o += dsz[y];
          ++n;
        }
      }
      off[n] = over ? -1 : o;
      cc[0] = n;
    }
    __syncwarp();
    const int n = cc[0];
    const int width = off[n];
    if (width < 0 || (int64_t)nr * width > wcap) {
      if (lane == 0) {
        dev_fail(st, DEV_OVERFLOW);
        oG.cnt[r] = 0;
      }
      continue;
    }
    for (int64_t e = lane; e < (int64_t)nr * width; e += 32) ws[e] = 0.0;
    for (int i = lane; i < n; i += 32) pr[i] = 0;
    __syncwarp();
    for (int64_t b = E.bptr[r]; b < E.bptr[r + 1]; ++b) {
      const int i = gr_find(col, n, E.bcol[b]);
      const int len = nr * dsz[E.bcol[b]];
      for (int e = lane; e < len; e += 32) ws[(int64_t)nr * off[i] + e] = (double)E.val[E.voff[b] + e];
      if (lane == 0) pr[i] = 1;
    }
    __syncwarp();
    int nc = 0;
    for (int i = 0; i < n; ++i) {
      if (!pr[i]) continue;
      const int64_t k = col[i];
      const int nk = dsz[k];
      double* m = ws + (int64_t)nr * off[i];
      gr_uinv_right(Dlu + Dvo[k], nk, m, nr, lane);
      __syncwarp();
      double fr = 0.0;
      if (lane == 0) fr = fro2_d(m, nr * nk);
      fr = __shfl_sync(0xffffffffu, fr, 0);
      if (drop_rule(fr, nr, nk, t)) {
        if (lane == 0) pr[i] = 0;
        __syncwarp();
        continue;
      }
      const int64_t us = oU.slot[k];
      int64_t vo = oU.vslot[k];
      for (int q = 0; q < oU.cnt[k]; ++q) {
        const int32_t j = oU.col[us + q];
        const int nj = dsz[j];
        const int jx = i + (int)(j - k);  // the group's members are consecutive columns
        gr_sub_prod<T>(ws + (int64_t)nr * off[jx], m, Uv + vo, nr, nk, nj, lane);
        if (lane == 0) pr[jx] = 1;
        vo += (int64_t)nk * nj;
      }
      if (lane == 0) {
        cc[nc] = (int32_t)i;
        f2[nc] = fr;
        pr[i] = 2;
      }
      ++nc;
      __syncwarp();
    }
    // lfil compares columns: workspace positions order like the columns
    gr_lfil(nc, cc, f2, keep, lfil, lane);
    {
      int64_t vo = oG.vslot[r];
      int c = 0;
      for (int q = 0; q < nc; ++q) {
        if (!keep[q]) continue;
        const int i = cc[q];
        const int nk = dsz[col[i]];
        const double* m = ws + (int64_t)nr * off[i];
        for (int e = lane; e < nr * nk; e += 32) Gv[vo + e] = (T)m[e];
        if (lane == 0) oG.col[oG.slot[r] + c] = col[i];
        vo += (int64_t)nr * nk;
        ++c;
      }
      if (lane == 0) oG.cnt[r] = c;
    }
    __syncwarp();
  }
}

// Compaction of slot rows into VBCSR: columns (first launch) and values.
template <typename T>
__global__ void k_gr_compact(int64_t nrows, const int64_t* __restrict__ slot, const int64_t* __restrict__ vslot,
                             const int32_t* __restrict__ scol, const T* __restrict__ sval,
                             const int64_t* __restrict__ bptr, int32_t* __restrict__ bcol,
                             const int64_t* __restrict__ voff, T* __restrict__ val) {
  const int lane = threadIdx.x & 31;
  const int64_t wpb = blockDim.x >> 5;
  for (int64_t r = blockIdx.x * wpb + (threadIdx.x >> 5); r < nrows; r += (int64_t)gridDim.x * wpb) {
    const int64_t b0 = bptr[r], nb = bptr[r + 1] - b0;
    if (!voff) {
      for (int64_t q = lane; q < nb; q += 32) bcol[b0 + q] = scol[slot[r] + q];
    } else {
      const int64_t len = voff[b0 + nb] - voff[b0];
      for (int64_t e = lane; e < len; e += 32) val[voff[b0] + e] = sval[vslot[r] + e];
    }
  }
}

// m = max over rows of a[r] + b[r] (b may be NULL)
__global__ void k_gr_max2(int64_t n, const int64_t* __restrict__ a, const int64_t* __restrict__ b,
                          unsigned long long* __restrict__ m) {
  unsigned long long v = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t x = a[i] + (b ? b[i] : 0);
    if ((unsigned long long)x > v) v = (unsigned long long)x;
  }
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
    if (w > v) v = w;
  }
  if ((threadIdx.x & 31) == 0 && v) atomicMax(m, v);
}

__global__ void k_gr_i32_to_i64(int64_t n, const int32_t* __restrict__ a, int64_t* __restrict__ b) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = a[i];
}

__global__ void k_gr_iota(int64_t n, int64_t* __restrict__ bptr, int32_t* __restrict__ bcol) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i <= n; i += (int64_t)gridDim.x * blockDim.x) {
    bptr[i] = i;
    if (i < n) bcol[i] = (int32_t)i;
  }
}

__global__ void k_gr_sq(int64_t n, const int32_t* __restrict__ sz, int64_t* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (int64_t)sz[i] * sz[i];
}

// Slots of one output: block and value capacities per row, scanned.
struct GrSlots {
  DBuf<int64_t> slot, vslot;
  DBuf<int32_t> col, cnt;
  DBuf<unsigned char> vraw;
  int64_t nslot = 0, nval = 0;
  template <typename T>
  void make(const DBuf<int64_t>& cap, const DBuf<int64_t>& vcap, int64_t nrows, cudaStream_t s) {
    slot.alloc(nrows + 1, s);
    vslot.alloc(nrows + 1, s);
    scan_i64(cap.p, slot.p, nrows, s);
    scan_i64(vcap.p, vslot.p, nrows, s);
    nslot = nrows ? d2h(slot.p + nrows, s) : 0;
    nval = nrows ? d2h(vslot.p + nrows, s) : 0;
    col.alloc(std::max<int64_t>(nslot, 1), s);
    cnt.alloc(std::max<int64_t>(nrows, 1), s);
    cnt.zero();
    vraw.alloc(std::max<int64_t>(nval, 1) * sizeof(T), s);
  }
  GrOut out() { return GrOut{slot.p, vslot.p, col.p, cnt.p}; }
};

// The VBCSR of kept slots (partitions: rows rsz, columns csz).
template <typename T>
void gr_assemble(GrSlots& S, int64_t nrows, const int32_t* rsz, const int32_t* csz, int64_t ncols, VBDev<T>& M,
                 cudaStream_t s) {
  set_partitions(M, rsz, nrows, csz, ncols, s);
  M.bptr.alloc(nrows + 1, s);
  {
    DBuf<int64_t> c64(std::max<int64_t>(nrows, 1), s);
    if (nrows) {
      launch(k_gr_i32_to_i64, grid_for(nrows, 256), 256, 0, s, nrows, S.cnt.p, c64.p);
      VB_LAUNCH_CHECK();
    }
    scan_i64(c64.p, M.bptr.p, nrows, s);
  }
  M.nnzb = nrows ? d2h(M.bptr.p + nrows, s) : 0;
  M.bcol.alloc(std::max<int64_t>(M.nnzb, 1), s);
  const T* sv = reinterpret_cast<const T*>(S.vraw.p);
  if (nrows) {
    launch(k_gr_compact<T>, grid_for(nrows, 8), 256, 0, s, nrows, S.slot.p, S.vslot.p, S.col.p, sv, M.bptr.p,
           M.bcol.p, (const int64_t*)nullptr, (T*)nullptr);
    VB_LAUNCH_CHECK();
  }
  finish_offsets(M, s);
  if (nrows && M.nval) {
    launch(k_gr_compact<T>, grid_for(nrows, 8), 256, 0, s, nrows, S.slot.p, S.vslot.p, S.col.p, sv, M.bptr.p,
           M.bcol.p, M.voff.p, M.val.p);
    VB_LAUNCH_CHECK();
  }
}

}  // namespace

template <typename TA>
int64_t group_order(const VBDev<TA>& A, double ddtol, int gs, const int32_t* fixed, DBuf<double>& w,
                    DBuf<int32_t>& pI, DBuf<int32_t>& newpos, DBuf<int64_t>& gptr, int64_t& ngroups,
                    cudaStream_t s) {
  const int64_t p = A.nbr;
  if (gs < 1 || gs > GR_GSMAX) fail(VB_EINVAL, "group size must lie in [1, 64]");
  level_weights<TA>(A, w, s);
  pI.alloc(std::max<int64_t>(p, 1), s);
  newpos.alloc(std::max<int64_t>(p, 1), s);
  ngroups = 0;
  if (!p) {
    gptr.alloc(1, s);
    gptr.zero();
    return 0;
  }
  // adjacency of A + A^T, rows ascending, no self loops
  const int64_t m = 2 * A.nnzb;
  const unsigned long long sentinel = (unsigned long long)p * (unsigned long long)p;
  DBuf<unsigned long long> pk(std::max<int64_t>(m, 1), s);
  DBuf<int64_t> aptr(p + 1, s);
  DBuf<int32_t> acol;
  {
    if (m) {
      launch(k_gr_pairs, grid_for(p, 8), 256, 0, s, p, A.bptr.p, A.bcol.p, pk.p);
      VB_LAUNCH_CHECK();
      radix_sort_u64(pk, nullptr, m, bits_of(sentinel), s);
    }
    DBuf<int32_t> first(std::max<int64_t>(m, 1), s), rowcnt(p, s);
    DBuf<int64_t> pos(m + 1, s);
    rowcnt.zero();
    if (m) {
      launch(k_gr_first, grid_for(m, 256), 256, 0, s, m, sentinel, pk.p, first.p);
      VB_LAUNCH_CHECK();
    }
    scan_i32_to_i64(first.p, pos.p, m, s);
    const int64_t E = m ? d2h(pos.p + m, s) : 0;
    acol.alloc(std::max<int64_t>(E, 1), s);
    if (m) {
      launch(k_gr_unique, grid_for(m, 256), 256, 0, s, m, p, pk.p, first.p, pos.p, acol.p, rowcnt.p);
      VB_LAUNCH_CHECK();
    }
    scan_i32_to_i64(rowcnt.p, aptr.p, p, s);
  }
  // visit order
  DBuf<int32_t> order(p, s);
  {
    DBuf<unsigned long long> wk(p, s);
    launch(k_gr_wkey, grid_for(p, 256), 256, 0, s, p, w.p, wk.p, order.p);
    VB_LAUNCH_CHECK();
    radix_sort_u64(wk, &order, p, 64, s);
  }
  // the greedy
  DBuf<int32_t> gid(p, s);
  DBuf<int> ng_dev(1, s);
  launch(k_gr_fill, grid_for(p, 256), 256, 0, s, p, -1, gid.p);
  if (p <= GR_SHMAX) {
    const int64_t nwd = (p + 31) >> 5;
    DBuf<uint32_t> elig(nwd, s);
    elig.zero();
    launch(k_gr_elig, grid_for(p, 256), 256, 0, s, p, w.p, ddtol, fixed, elig.p);
    const size_t smem = (size_t)2 * nwd * sizeof(uint32_t);
    VB_CUDA(cudaFuncSetAttribute(k_gr_greedy_sh, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    launch(k_gr_greedy_sh, 1, 32, smem, s, p, order.p, aptr.p, acol.p, elig.p, gs, gid.p, ng_dev.p);
  } else {
    DBuf<int32_t> mark(p, s);
    mark.zero();
    launch(k_gr_greedy, 1, 32, 0, s, p, order.p, aptr.p, acol.p, w.p, ddtol, fixed, gs, mark.p, gid.p, ng_dev.p);
  }
  VB_LAUNCH_CHECK();
  const int64_t ng = d2h(ng_dev.p, s);
  ngroups = ng;
  // groups by smallest member; D = members keyed by (rank, member); C ascending
  DBuf<int32_t> gmin(std::max<int64_t>(ng, 1), s), gcnt(std::max<int64_t>(ng, 1), s),
      rank(std::max<int64_t>(ng, 1), s), rsize(std::max<int64_t>(ng, 1), s);
  gptr.alloc(ng + 1, s);
  if (ng) {
    launch(k_gr_fill, grid_for(ng, 256), 256, 0, s, ng, INT_MAX, gmin.p);
    gcnt.zero();
    launch(k_gr_gmin, grid_for(p, 256), 256, 0, s, p, gid.p, gmin.p, gcnt.p);
    VB_LAUNCH_CHECK();
    DBuf<unsigned long long> gk(ng, s);
    launch(k_gr_gkey, grid_for(ng, 256), 256, 0, s, ng, gmin.p, gk.p);
    VB_LAUNCH_CHECK();
    radix_sort_u64(gk, nullptr, ng, 32 + bits_of((unsigned long long)p), s);  // (smallest member, group)
    launch(k_gr_rank, grid_for(ng, 256), 256, 0, s, ng, gk.p, gcnt.p, rank.p, rsize.p);
    VB_LAUNCH_CHECK();
  }
  scan_i32_to_i64(rsize.p, gptr.p, ng, s);
  DBuf<int32_t> inD(p, s), inC(p, s);
  DBuf<int64_t> sD(p + 1, s), sC(p + 1, s);
  launch(k_gr_flags, grid_for(p, 256), 256, 0, s, p, gid.p, inD.p, inC.p);
  VB_LAUNCH_CHECK();
  scan_i32_to_i64(inD.p, sD.p, p, s);
  scan_i32_to_i64(inC.p, sC.p, p, s);
  const int64_t nD = d2h(sD.p + p, s);
  DBuf<unsigned long long> mkey(std::max<int64_t>(nD, 1), s);
  launch(k_gr_place, grid_for(p, 256), 256, 0, s, p, nD, gid.p, rank.p, sD.p, sC.p, mkey.p, pI.p);
  VB_LAUNCH_CHECK();
  if (nD) {
    radix_sort_u64(mkey, nullptr, nD, 32 + bits_of((unsigned long long)std::max<int64_t>(ng, 1)), s);
    launch(k_gr_dlist, grid_for(nD, 256), 256, 0, s, nD, mkey.p, pI.p);
    VB_LAUNCH_CHECK();
  }
  launch(k_gr_newpos, grid_for(p, 256), 256, 0, s, p, pI.p, newpos.p);
  VB_LAUNCH_CHECK();
  return nD;
}

template int64_t group_order<double>(const VBDev<double>&, double, int, const int32_t*, DBuf<double>&,
                                     DBuf<int32_t>&, DBuf<int32_t>&, DBuf<int64_t>&, int64_t&, cudaStream_t);
template int64_t group_order<float>(const VBDev<float>&, double, int, const int32_t*, DBuf<double>&,
                                    DBuf<int32_t>&, DBuf<int32_t>&, DBuf<int64_t>&, int64_t&, cudaStream_t);

namespace {
// Level solve of a grouped level (one thread per group, its rows in order):
// u_y = L_y^{-1} P_y (f_y - sum_k m_yk u_k) forward, in place in bh.
template <typename T>
__global__ void k_gr_fwd(int64_t ng, const int64_t* __restrict__ gptr, VBView<T> Lg, const int64_t* __restrict__ Dvo,
                         const double* __restrict__ Dlu, const int32_t* __restrict__ piv, double* __restrict__ bh) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < ng; g += (int64_t)gridDim.x * blockDim.x)
    for (int64_t y = gptr[g]; y < gptr[g + 1]; ++y) {
      const int ny = Lg.rsz[y];
      double* u = bh + Lg.roff[y];
      for (int64_t b = Lg.bptr[y]; b < Lg.bptr[y + 1]; ++b) {
        const int32_t k = Lg.bcol[b];
        const int nk = Lg.csz[k];
        const T* m = Lg.val + Lg.voff[b];
        const double* uk = bh + Lg.coff[k];
        for (int a = 0; a < ny; ++a) {
          double v = u[a];
          for (int q = 0; q < nk; ++q) v = __dsub_rn(v, __dmul_rn((double)m[a * nk + q], uk[q]));
          u[a] = v;
        }
      }
      const double* lu = Dlu + Dvo[y];
      const int32_t* pv = piv + Lg.roff[y];
      for (int k = 0; k < ny; ++k)
        if (pv[k] != k) {
          const double t = u[k];
          u[k] = u[pv[k]];
          u[pv[k]] = t;
        }
      for (int i = 1; i < ny; ++i)
        for (int k = 0; k < i; ++k) u[i] = __dsub_rn(u[i], __dmul_rn(lu[i * ny + k], u[k]));
    }
}

// Backward: x_y = U_y^{-1} (bh_y - sum_j ubar_yj x_j), rows in reverse order
// (bh already holds u - W z).
template <typename T>
__global__ void k_gr_bwd(int64_t ng, const int64_t* __restrict__ gptr, VBView<T> Ug, const int64_t* __restrict__ Dvo,
                         const double* __restrict__ Dlu, const double* __restrict__ bh, double* __restrict__ xh) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < ng; g += (int64_t)gridDim.x * blockDim.x)
    for (int64_t y = gptr[g + 1] - 1; y >= gptr[g]; --y) {
      const int ny = Ug.rsz[y];
      double* x = xh + Ug.roff[y];
      for (int a = 0; a < ny; ++a) x[a] = bh[Ug.roff[y] + a];
      for (int64_t b = Ug.bptr[y]; b < Ug.bptr[y + 1]; ++b) {
        const int32_t j = Ug.bcol[b];
        const int nj = Ug.csz[j];
        const T* um = Ug.val + Ug.voff[b];
        const double* xj = xh + Ug.coff[j];
        for (int a = 0; a < ny; ++a) {
          double v = x[a];
          for (int q = 0; q < nj; ++q) v = __dsub_rn(v, __dmul_rn((double)um[a * nj + q], xj[q]));
          x[a] = v;
        }
      }
      const double* lu = Dlu + Dvo[y];
      for (int i = ny - 1; i >= 0; --i) {
        double v = x[i];
        for (int k = i + 1; k < ny; ++k) v = __dsub_rn(v, __dmul_rn(lu[i * ny + k], x[k]));
        x[i] = __ddiv_rn(v, lu[i * ny + i]);
      }
    }
}

__global__ void k_gr_sizes_by(int64_t n, int64_t off, const int32_t* __restrict__ pI, const int32_t* __restrict__ rsz,
                              int32_t* __restrict__ out) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
    out[k] = rsz[pI[off + k]];
}
}  // namespace

template <typename T>
void grouped_forward(const LevelDev<T>& L, double* bh, cudaStream_t s) {
  if (!L.ngroups) return;
  launch(k_gr_fwd<T>, grid_for(L.ngroups, 128), 128, 0, s, L.ngroups, L.gptr.p, L.Lg.view(), L.D.voff.p, L.D.val.p,
         L.piv.p, bh);
  VB_LAUNCH_CHECK();
}

template <typename T>
void grouped_backward(const LevelDev<T>& L, const double* bh, double* xh, cudaStream_t s) {
  if (!L.ngroups) return;
  launch(k_gr_bwd<T>, grid_for(L.ngroups, 128), 128, 0, s, L.ngroups, L.gptr.p, L.Ug.view(), L.D.voff.p, L.D.val.p,
         bh, xh);
  VB_LAUNCH_CHECK();
}
template void grouped_forward<double>(const LevelDev<double>&, double*, cudaStream_t);
template void grouped_forward<float>(const LevelDev<float>&, double*, cudaStream_t);
template void grouped_backward<double>(const LevelDev<double>&, const double*, double*, cudaStream_t);
template void grouped_backward<float>(const LevelDev<float>&, const double*, double*, cudaStream_t);

template <typename TA, typename T>
void grouped_level(const VBDev<TA>& A, const DBuf<int32_t>& pI, const DBuf<int32_t>& newpos, int64_t nD,
                   const DBuf<int64_t>& gptr, int64_t ngroups, double t, int lfil, LevelDev<T>& L, cudaStream_t s,
                   int* dst) {
  const int64_t p = A.nbr, nC = p - nD;
  L.nD = nD;
  L.nC = nC;
  L.grouped = true;
  L.ngroups = ngroups;
  L.gptr.alloc(ngroups + 1, s);
  VB_CUDA(cudaMemcpyAsync(L.gptr.p, gptr.p, (ngroups + 1) * sizeof(int64_t), cudaMemcpyDeviceToDevice, s));
  DBuf<int32_t> szD(std::max<int64_t>(nD, 1), s), szC(std::max<int64_t>(nC, 1), s);
  if (nD) launch(k_gr_sizes_by, grid_for(nD, 256), 256, 0, s, nD, (int64_t)0, pI.p, A.rsz.p, szD.p);
  if (nC) launch(k_gr_sizes_by, grid_for(nC, 256), 256, 0, s, nC, nD, pI.p, A.rsz.p, szC.p);
  VB_LAUNCH_CHECK();
  // the four parts
  VBDev<double> Dm;
  set_partitions(Dm, szD.p, nD, szD.p, nD, s);
  set_partitions(L.F, szD.p, nD, szC.p, nC, s);
  set_partitions(L.E, szC.p, nC, szD.p, nD, s);
  set_partitions(L.C, szC.p, nC, szC.p, nC, s);
  DBuf<int32_t> cD(std::max<int64_t>(nD, 1), s), cF(std::max<int64_t>(nD, 1), s), cE(std::max<int64_t>(nC, 1), s),
      cC(std::max<int64_t>(nC, 1), s);
  launch(k_gr_gather<0>, grid_for(p, 8), 256, 0, s, p, nD, A.bptr.p, A.bcol.p, newpos.p, cD.p, cF.p, cE.p, cC.p,
         nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr);
  VB_LAUNCH_CHECK();
  check_status(dst, s, "vbarms_factor: grouped gather");
  Dm.bptr.alloc(nD + 1, s);
  L.F.bptr.alloc(nD + 1, s);
  L.E.bptr.alloc(nC + 1, s);
  L.C.bptr.alloc(nC + 1, s);
  scan_i32_to_i64(cD.p, Dm.bptr.p, nD, s);
  scan_i32_to_i64(cF.p, L.F.bptr.p, nD, s);
  scan_i32_to_i64(cE.p, L.E.bptr.p, nC, s);
  scan_i32_to_i64(cC.p, L.C.bptr.p, nC, s);
  Dm.nnzb = nD ? d2h(Dm.bptr.p + nD, s) : 0;
  L.F.nnzb = nD ? d2h(L.F.bptr.p + nD, s) : 0;
  L.E.nnzb = nC ? d2h(L.E.bptr.p + nC, s) : 0;
  L.C.nnzb = nC ? d2h(L.C.bptr.p + nC, s) : 0;
  Dm.bcol.alloc(std::max<int64_t>(Dm.nnzb, 1), s);
  L.F.bcol.alloc(std::max<int64_t>(L.F.nnzb, 1), s);
  L.E.bcol.alloc(std::max<int64_t>(L.E.nnzb, 1), s);
  L.C.bcol.alloc(std::max<int64_t>(L.C.nnzb, 1), s);
  DBuf<int64_t> sD(std::max<int64_t>(Dm.nnzb, 1), s), sF(std::max<int64_t>(L.F.nnzb, 1), s),
      sE0(std::max<int64_t>(L.E.nnzb, 1), s), sE(std::max<int64_t>(L.E.nnzb, 1), s),
      sC(std::max<int64_t>(L.C.nnzb, 1), s);
  DBuf<int32_t> colE0(std::max<int64_t>(L.E.nnzb, 1), s);
  launch(k_gr_gather<1>, grid_for(p, 8), 256, 0, s, p, nD, A.bptr.p, A.bcol.p, newpos.p, nullptr, nullptr, nullptr,
         nullptr, Dm.bptr.p, L.F.bptr.p, L.E.bptr.p, L.C.bptr.p, Dm.bcol.p, L.F.bcol.p, colE0.p, L.C.bcol.p, sD.p,
         sF.p, sE0.p, sC.p);
  VB_LAUNCH_CHECK();
  if (nC) {
    launch(k_gr_sort_rows, grid_for(nC, 8), 256, 0, s, nC, L.E.bptr.p, colE0.p, sE0.p, L.E.bcol.p, sE.p);
    VB_LAUNCH_CHECK();
  }
  finish_offsets(Dm, s);
  finish_offsets(L.F, s);
  finish_offsets(L.E, s);
  finish_offsets(L.C, s);
  if (Dm.nnzb) launch(k_gr_copy_blocks<TA, double>, grid_for(Dm.nnzb, 8), 256, 0, s, Dm.nnzb, sD.p, A.voff.p, A.val.p,
                      Dm.voff.p, Dm.val.p);
  if (L.F.nnzb) launch(k_gr_copy_blocks<TA, T>, grid_for(L.F.nnzb, 8), 256, 0, s, L.F.nnzb, sF.p, A.voff.p, A.val.p,
                       L.F.voff.p, L.F.val.p);
  if (L.E.nnzb) launch(k_gr_copy_blocks<TA, T>, grid_for(L.E.nnzb, 8), 256, 0, s, L.E.nnzb, sE.p, A.voff.p, A.val.p,
                       L.E.voff.p, L.E.val.p);
  if (L.C.nnzb) launch(k_gr_copy_blocks<TA, T>, grid_for(L.C.nnzb, 8), 256, 0, s, L.C.nnzb, sC.p, A.voff.p, A.val.p,
                       L.C.voff.p, L.C.val.p);
  VB_LAUNCH_CHECK();
  // pivot blocks (block diagonal, LU after the group elimination)
  set_partitions(L.D, szD.p, nD, szD.p, nD, s);
  L.D.bptr.alloc(nD + 1, s);
  L.D.bcol.alloc(std::max<int64_t>(nD, 1), s);
  launch(k_gr_iota, grid_for(nD + 1, 256), 256, 0, s, nD, L.D.bptr.p, L.D.bcol.p);
  VB_LAUNCH_CHECK();
  L.D.nnzb = nD;
  L.D.voff.alloc(nD + 1, s);
  {
    DBuf<int64_t> sq(std::max<int64_t>(nD, 1), s);
    if (nD) launch(k_gr_sq, grid_for(nD, 256), 256, 0, s, nD, szD.p, sq.p);
    VB_LAUNCH_CHECK();
    scan_i64(sq.p, L.D.voff.p, nD, s);
  }
  L.D.nval = nD ? d2h(L.D.voff.p + nD, s) : 0;
  L.D.val.alloc(std::max<int64_t>(L.D.nval, 1), s);
  const int64_t nsd = nD ? d2h(L.D.roff.p + nD, s) : 0;
  L.piv.alloc(std::max<int64_t>(nsd, 1), s);
  L.ptag.alloc(std::max<int64_t>(nD, 1), s);
  launch(k_gr_fill, grid_for(std::max<int64_t>(nD, 1), 256), 256, 0, s, std::max<int64_t>(nD, 1), 1, L.ptag.p);
  VB_LAUNCH_CHECK();
  int dev = 0, nsm = 0;
  VB_CUDA(cudaGetDevice(&dev));
  VB_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  // sweep 1
  DBuf<int32_t> ulist(std::max<int64_t>(L.F.nnzb, 1), s), ucnt(std::max<int64_t>(ngroups, 1), s);
  DBuf<int64_t> uwid(std::max<int64_t>(ngroups, 1), s);
  if (ngroups) {
    launch(k_gr_union, grid_for(ngroups, GR_WARPS), GR_WARPS * 32, 0, s, ngroups, gptr.p, L.F.bptr.p, L.F.bcol.p,
           szC.p, ulist.p, ucnt.p, uwid.p, dst);
    VB_LAUNCH_CHECK();
  }
  if (d2h(dst, s) == DEV_OVERFLOW)
    fail(VB_ENOMEM, "grouped level: a group's F columns exceed 1024 blocks (use a smaller group size)");
  check_status(dst, s, "vbarms_factor: grouped level");
  GrSlots SL, SU, SW, SG;
  int64_t wcap1 = 1, wcap2 = 1;
  {
    DBuf<int64_t> capG(std::max<int64_t>(nD, 1), s), vcapG(std::max<int64_t>(nD, 1), s),
        capW(std::max<int64_t>(nD, 1), s), vcapW(std::max<int64_t>(nD, 1), s);
    if (ngroups) {
      launch(k_gr_caps1, grid_for(ngroups, 256), 256, 0, s, ngroups, gptr.p, szD.p, ucnt.p, uwid.p, capG.p, vcapG.p,
             capW.p, vcapW.p);
      VB_LAUNCH_CHECK();
    }
    SL.make<T>(capG, vcapG, nD, s);
    SU.make<T>(capG, vcapG, nD, s);
    SW.make<T>(capW, vcapW, nD, s);
    // one row's workspace: ny times the group's and the union's widths
    DBuf<unsigned long long> mx(1, s);
    mx.zero();
    if (nD) {
      launch(k_gr_max2, grid_for(nD, 256), 256, 0, s, nD, vcapG.p, vcapW.p, mx.p);
      VB_LAUNCH_CHECK();
    }
    wcap1 = std::max<int64_t>((int64_t)d2h(mx.p, s), 1);
  }
  const unsigned nb1 = (unsigned)std::max<int64_t>(1, std::min<int64_t>((ngroups + GR_WARPS - 1) / GR_WARPS,
                                                                          (int64_t)nsm * 8));
  DBuf<double> ws((size_t)nb1 * GR_WARPS * wcap1, s);
  if (ngroups) {
    launch(k_gr_sweep1<T>, nb1, GR_WARPS * 32, 0, s, ngroups, gptr.p, Dm.view(), L.F.view(), ulist.p, ucnt.p, szC.p,
           L.D.voff.p, L.D.val.p, L.piv.p, SL.out(), reinterpret_cast<T*>(SL.vraw.p), SU.out(),
           reinterpret_cast<T*>(SU.vraw.p), SW.out(), reinterpret_cast<T*>(SW.vraw.p), ws.p, wcap1, t, lfil, dst);
    VB_LAUNCH_CHECK();
  }
  if (d2h(dst, s) == DEV_OVERFLOW) fail(VB_ENOMEM, "grouped level: a row exceeds the sweep workspace");
  check_status(dst, s, "vbarms_factor: grouped level (first sweep)");
  gr_assemble<T>(SL, nD, szD.p, szD.p, nD, L.Lg, s);
  gr_assemble<T>(SU, nD, szD.p, szD.p, nD, L.Ug, s);
  gr_assemble<T>(SW, nD, szD.p, szC.p, nC, L.W, s);
  SL = GrSlots();
  SW = GrSlots();
  // sweep 2 (reads Ubar's group part from its slots, which SU still holds)
  DBuf<int32_t> dgid(std::max<int64_t>(nD, 1), s);
  if (ngroups) {
    launch(k_gr_group_of, grid_for(ngroups, 256), 256, 0, s, ngroups, gptr.p, dgid.p);
    VB_LAUNCH_CHECK();
  }
  {
    DBuf<int64_t> cap(std::max<int64_t>(nC, 1), s), vcap(std::max<int64_t>(nC, 1), s);
    if (nC) {
      launch(k_gr_caps2, grid_for(nC, 256), 256, 0, s, nC, L.E.bptr.p, L.E.bcol.p, dgid.p, gptr.p, L.D.roff.p,
             szC.p, cap.p, vcap.p);
      VB_LAUNCH_CHECK();
    }
    SG.make<T>(cap, vcap, nC, s);
    DBuf<unsigned long long> mx(1, s);
    mx.zero();
    if (nC) {
      launch(k_gr_max2, grid_for(nC, 256), 256, 0, s, nC, vcap.p, (const int64_t*)nullptr, mx.p);
      VB_LAUNCH_CHECK();
    }
    wcap2 = std::max<int64_t>((int64_t)d2h(mx.p, s), 1);
  }
  if (nC) {
    const unsigned nb2 = (unsigned)std::max<int64_t>(1, std::min<int64_t>((nC + GR_WARPS - 1) / GR_WARPS,
                                                                           (int64_t)nsm * 8));
    ws.alloc((size_t)nb2 * GR_WARPS * wcap2, s);
    launch(k_gr_sweep2<T>, nb2, GR_WARPS * 32, 0, s, nC, L.E.view(), dgid.p, gptr.p, szD.p, L.D.voff.p, L.D.val.p,
           SU.out(), reinterpret_cast<const T*>(SU.vraw.p), SG.out(), reinterpret_cast<T*>(SG.vraw.p), ws.p, wcap2,
           t, lfil, dst);
    VB_LAUNCH_CHECK();
  }
  if (d2h(dst, s) == DEV_OVERFLOW)
    fail(VB_ENOMEM, "grouped level: an E row touches groups beyond the sweep workspace");
  check_status(dst, s, "vbarms_factor: grouped level (second sweep)");
  gr_assemble<T>(SG, nC, szC.p, szD.p, nD, L.G, s);
}

#define VB_GR_INST(TA, T)                                                                                        \
  template void grouped_level<TA, T>(const VBDev<TA>&, const DBuf<int32_t>&, const DBuf<int32_t>&, int64_t,     \
                                     const DBuf<int64_t>&, int64_t, double, int, LevelDev<T>&, cudaStream_t, int*);
VB_GR_INST(double, double)
VB_GR_INST(double, float)
VB_GR_INST(float, float)

}  // namespace vb
