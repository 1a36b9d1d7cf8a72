// Step 1 of VBARMS on the GPU: angle-based row-pattern compression
// (Section 2.1) and the VBCSR block permutation P_B A P_B^T (Eq. 3).
//
//   A1  row lengths, CSR validation, CSC transpose of the pattern
//   A2  per row i, the overlaps |P_i n P_j| for j > i (the upper part of
//       C C^T) counted in a per-warp shared-memory hash table; similar pairs
//       (cos >= tau, one exactly rounded FP64 product) are emitted
//   A3  the natural-order leader greedy, which is the lexicographically first
//       maximal independent set of the similarity graph: computed in
//       deterministic rounds, each non-leader joins its smallest similar
//       leader
//   A4  block ordering (leaders ascending, members ascending) and VBCSR
//       assembly with zero-padded dense blocks, values copied bit-exactly
#include "internal.h"
#include "vbsr_ops.cuh"

namespace vb {
namespace {

constexpr int CW = 8;          // warps per block in the hashing kernels
constexpr int SIM_CAP = 1024;  // per-warp shared hash capacity (power of 2)
constexpr int SIM_LIMIT = 640; // distinct keys before a row moves to the global-table path

// ---- A1 ------------------------------------------------------------------
__global__ void k_validate(int64_t n, const int64_t* __restrict__ rowptr, const int32_t* __restrict__ colind,
                           int32_t* __restrict__ len, int* st) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p0 = rowptr[i], p1 = rowptr[i + 1];
    if (i == 0 && p0 != 0) dev_fail(st, DEV_EINVAL);
    if (p1 < p0 || p1 - p0 > n) {
      dev_fail(st, DEV_EINVAL);
      len[i] = 0;
      continue;
    }
    int32_t prev = -1;
    for (int64_t p = p0; p < p1; ++p) {
      const int32_t c = colind[p];
      if (c < 0 || c >= n || c <= prev) {
        dev_fail(st, DEV_EINVAL);
        break;
      }
      prev = c;
    }
    len[i] = (int32_t)(p1 - p0);
  }
}

__global__ void k_col_count(int64_t nnz, const int32_t* __restrict__ colind, int32_t* __restrict__ ccnt) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < nnz; p += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(&ccnt[colind[p]], 1);
}

__global__ void k_col_fill(int64_t n, const int64_t* __restrict__ rowptr, const int32_t* __restrict__ colind,
                           const int64_t* __restrict__ cptr, int32_t* __restrict__ cfill, int32_t* __restrict__ crow) {
  const int lane = threadIdx.x & 31;
  const int64_t wpb = blockDim.x >> 5;
  for (int64_t i = blockIdx.x * wpb + (threadIdx.x >> 5); i < n; i += (int64_t)gridDim.x * wpb) {
    for (int64_t p = rowptr[i] + lane; p < rowptr[i + 1]; p += 32) {
      const int32_t c = colind[p];
      const int32_t k = atomicAdd(&cfill[c], 1);
      crow[cptr[c] + k] = (int32_t)i;
    }
  }
}

// ---- A2 ------------------------------------------------------------------
// One warp per row i.  The row's columns are taken 32 at a time: one round of
// loads gives their extents in the CSC, then the lanes walk the chunk's
// (column, row j) entries flattened, eight loads in flight per lane, and
// count |P_i n P_j| for j > i in a hash table (atomic inserts and counts, so
// entries of different columns may meet in one pass).  GLOBAL = false: table
// in shared memory (SIM_CAP); rows whose candidate set outgrows SIM_LIMIT are
// deferred to a list.  GLOBAL = true: table in global memory (gcap per warp),
// rows from the list.
template <bool GLOBAL>
__global__ void __launch_bounds__(CW * 32)
    k_similar(int64_t nrows, const int32_t* __restrict__ rows, const int64_t* __restrict__ rowptr,
              const int32_t* __restrict__ colind, const int64_t* __restrict__ cptr,
              const int32_t* __restrict__ crow, const int32_t* __restrict__ len, double tau2, int* gtab,
              uint32_t gcap, int64_t* __restrict__ simstart, int32_t* __restrict__ simcnt,
              int32_t* __restrict__ simbuf, int64_t simcap, unsigned long long* simtotal,
              int32_t* __restrict__ heavy, int* nheavy, int* st) {
  extern __shared__ int smem[];
  __shared__ int nfresh[CW];
  __shared__ int64_t ccs[CW][32];  // CSC start of each column of the chunk
  __shared__ int cpre[CW][33];     // entry prefix over the chunk's columns
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int *keys, *cnt;
  uint32_t cap;
  int limit;
  if (GLOBAL) {
    keys = gtab + ((size_t)blockIdx.x * CW + warp) * 2 * gcap;
    cnt = keys + gcap;
    cap = gcap;
    limit = (int)gcap;
  } else {
    keys = smem + warp * 2 * SIM_CAP;
    cnt = keys + SIM_CAP;
    cap = SIM_CAP;
    limit = SIM_LIMIT;
  }
  for (int64_t t = (int64_t)blockIdx.x * CW + warp; t < nrows; t += (int64_t)gridDim.x * CW) {
    const int64_t i = rows ? rows[t] : t;
    const int ni = len[i];
    if (ni == 0) {
      if (lane == 0) {
        simstart[i] = 0;
        simcnt[i] = 0;
      }
      continue;
    }
    for (uint32_t k = lane; k < cap; k += 32) {
      keys[k] = -1;
      cnt[k] = 0;
    }
    if (lane == 0) nfresh[warp] = 0;
    __syncwarp();
    bool over = false;
    const int64_t pe = rowptr[i + 1];
    for (int64_t p0 = rowptr[i]; p0 < pe && !over; p0 += 32) {
      int64_t cs = 0, ce = 0;
      if (p0 + lane < pe) {
        const int32_t c = colind[p0 + lane];
        cs = cptr[c];
        ce = cptr[c + 1];
      }
      const int lc = (int)(ce - cs);
      int incl = lc;
      for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
      }
      const int tot = __shfl_sync(0xffffffffu, incl, 31);
      ccs[warp][lane] = cs;
      cpre[warp][lane] = incl - lc;
      if (lane == 31) cpre[warp][32] = tot;
      __syncwarp();
      bool full = false;
      int tc = 0;  // column of the lane's current entry (entries only move forward)
      for (int e0 = lane; e0 < tot && !full; e0 += 32 * 8) {
        int32_t jv[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int e = e0 + 32 * u;
          jv[u] = -1;
          if (e < tot) {
            while (cpre[warp][tc + 1] <= e) ++tc;
            jv[u] = crow[ccs[warp][tc] + (e - cpre[warp][tc])];
          }
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int32_t j = jv[u];
          if (j <= i || full) continue;
          bool fresh;
          const int slot = hset_insert(keys, cap - 1, j, &fresh);
          if (slot < 0) {
            full = true;
            continue;
          }
          atomicAdd(&cnt[slot], 1);
          if (fresh) atomicAdd(&nfresh[warp], 1);
        }
      }
      __syncwarp();
      const int nf = *((volatile int*)&nfresh[warp]);
      if (__any_sync(0xffffffffu, full) || nf > limit) over = true;
    }
    if (over) {
      if (lane == 0) {
        if (GLOBAL) {
          dev_fail(st, DEV_INTERNAL);
        } else {
          heavy[atomicAdd(nheavy, 1)] = (int32_t)i;
          simcnt[i] = 0;
          simstart[i] = 0;
        }
      }
      __syncwarp();
      continue;
    }
    // similar iff c^2 >= tau^2 |P_i| |P_j| (one exactly rounded product)
    int mine = 0;
    for (uint32_t k = lane; k < cap; k += 32) {
      const int j = keys[k];
      if (j >= 0) {
        const long long c = cnt[k];
        const long long nn = (long long)ni * (long long)len[j];
        if ((double)(c * c) >= __dmul_rn(tau2, (double)nn)) ++mine;
      }
    }
    const int total = warp_sum_i(mine);
    unsigned long long off = 0;
    if (lane == 0 && total) off = atomicAdd(simtotal, (unsigned long long)total);
    off = __shfl_sync(0xffffffffu, off, 0);
    if (lane == 0) {
      simstart[i] = (int64_t)off;
      simcnt[i] = total;
    }
    if (total && (int64_t)(off + total) <= simcap) {
      int64_t base = (int64_t)off;
      for (uint32_t k0 = 0; k0 < cap; k0 += 32) {
        const uint32_t k = k0 + lane;
        bool m = false;
        int j = -1;
        if (k < cap) {
          j = keys[k];
          if (j >= 0) {
            const long long c = cnt[k];
            const long long nn = (long long)ni * (long long)len[j];
            m = (double)(c * c) >= __dmul_rn(tau2, (double)nn);
          }
        }
        const unsigned b = __ballot_sync(0xffffffffu, m);
        if (m) simbuf[base + __popc(b & ((1u << lane) - 1u))] = j;
        base += __popc(b);
      }
    }
    __syncwarp();
  }
}

// Upper bound of the candidate count of the deferred rows (global tables).
__global__ void k_heavy_bound(int nheavy, const int32_t* __restrict__ heavy, const int64_t* __restrict__ rowptr,
                              const int32_t* __restrict__ colind, const int64_t* __restrict__ cptr, int64_t n,
                              unsigned long long* maxb) {
  const int lane = threadIdx.x & 31;
  const int64_t wpb = blockDim.x >> 5;
  for (int64_t t = blockIdx.x * wpb + (threadIdx.x >> 5); t < nheavy; t += (int64_t)gridDim.x * wpb) {
    const int32_t i = heavy[t];
    long long b = 0;
    for (int64_t p = rowptr[i] + lane; p < rowptr[i + 1]; p += 32) b += cptr[colind[p] + 1] - cptr[colind[p]];
    b = warp_sum_ll(b);
    if (b > n) b = n;
    if (lane == 0) atomicMax(maxb, (unsigned long long)b);
  }
}

// ---- A3 ------------------------------------------------------------------
// pending[j] = number of similar i < j (the leaders that could claim j).
__global__ void k_pending(int64_t n, const int64_t* __restrict__ simstart, const int32_t* __restrict__ simcnt,
                          const int32_t* __restrict__ simbuf, int32_t* __restrict__ pending) {
  const int lane = threadIdx.x & 31;
  const int64_t wpb = blockDim.x >> 5;
  for (int64_t i = blockIdx.x * wpb + (threadIdx.x >> 5); i < n; i += (int64_t)gridDim.x * wpb)
    for (int64_t q = lane; q < simcnt[i]; q += 32) atomicAdd(&pending[simbuf[simstart[i] + q]], 1);
}

// state: 0 undecided, 1 leader, 2 claimed in the current MIS round, 3 claimed.
__global__ void k_round_a(int64_t n, const int64_t* __restrict__ simstart, const int32_t* __restrict__ simcnt,
                          const int32_t* __restrict__ simbuf, const int32_t* __restrict__ pending,
                          int32_t* __restrict__ state, unsigned long long* remaining) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    if (state[v] != 0 || pending[v] != 0) continue;
    state[v] = 1;
    unsigned long long dec = 1;
    for (int64_t q = 0; q < simcnt[v]; ++q) {
      const int32_t j = simbuf[simstart[v] + q];
      if (atomicCAS(&state[j], 0, 2) == 0) ++dec;
    }
    atomicAdd(remaining, (unsigned long long)(-(long long)dec));
  }
}

__global__ void k_round_b(int64_t n, const int64_t* __restrict__ simstart, const int32_t* __restrict__ simcnt,
                          const int32_t* __restrict__ simbuf, int32_t* __restrict__ pending,
                          int32_t* __restrict__ state) {
  for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < n; u += (int64_t)gridDim.x * blockDim.x) {
    if (state[u] != 2) continue;
    state[u] = 3;
    for (int64_t q = 0; q < simcnt[u]; ++q) atomicSub(&pending[simbuf[simstart[u] + q]], 1);
  }
}

// group[j] = smallest leader similar to j (leaders: themselves).
__global__ void k_groups(int64_t n, const int64_t* __restrict__ simstart, const int32_t* __restrict__ simcnt,
                         const int32_t* __restrict__ simbuf, const int32_t* __restrict__ state,
                         int32_t* __restrict__ group, int32_t* __restrict__ isleader) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    const bool lead = state[v] == 1;
    isleader[v] = lead ? 1 : 0;
    if (!lead) continue;
    atomicMin(&group[v], (int32_t)v);
    for (int64_t q = 0; q < simcnt[v]; ++q) atomicMin(&group[simbuf[simstart[v] + q]], (int32_t)v);
  }
}

__global__ void k_block_of(int64_t n, const int32_t* __restrict__ group, const int64_t* __restrict__ lead_scan,
                           int32_t* __restrict__ blk, int32_t* __restrict__ bsz, int* st) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
    const int32_t g = group[r];
    if (g < 0 || g > r) {
      dev_fail(st, DEV_INTERNAL);
      blk[r] = 0;
      continue;
    }
    const int32_t b = (int32_t)lead_scan[g];
    blk[r] = b;
    atomicAdd(&bsz[b], 1);
  }
}

// rank of r among its group's members (members ascending, leader first).
__global__ void k_member_rank(int64_t n, const int64_t* __restrict__ simstart, const int32_t* __restrict__ simcnt,
                              const int32_t* __restrict__ simbuf, const int32_t* __restrict__ group,
                              const int32_t* __restrict__ blk, const int64_t* __restrict__ boff,
                              int32_t* __restrict__ offin, int32_t* __restrict__ perm) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
    const int32_t v = group[r];
    int32_t rank = 0;
    if (v != r) {
      rank = 1;
      for (int64_t q = 0; q < simcnt[v]; ++q) {
        const int32_t j = simbuf[simstart[v] + q];
        if (j < r && group[j] == v) ++rank;
      }
    }
    offin[r] = rank;
    const int64_t pos = boff[blk[r]] + rank;
    if (pos < boff[blk[r] + 1]) perm[pos] = (int32_t)r;  // always true unless the grouping is inconsistent
  }
}

// ---- A4 ------------------------------------------------------------------
// One warp per block row I: the distinct block columns J = blk[c] of its rows.
// PASS 0 counts them, PASS 1 writes them ascending.
template <bool GLOBAL, int PASS>
__global__ void __launch_bounds__(CW * 32)
    k_block_pattern(int64_t nrowsI, const int32_t* __restrict__ list, const int64_t* __restrict__ boff,
                    const int32_t* __restrict__ perm, const int64_t* __restrict__ rowptr,
                    const int32_t* __restrict__ colind, const int32_t* __restrict__ blk, int* gtab, uint32_t gcap,
                    int64_t* __restrict__ bcnt, const int64_t* __restrict__ bptr, int32_t* __restrict__ bcol,
                    int32_t* __restrict__ heavy, int* nheavy, int* st) {
  extern __shared__ int smem[];
  __shared__ int nfresh[CW];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int* keys;
  uint32_t cap;
  int limit;
  if (GLOBAL) {
    keys = gtab + ((size_t)blockIdx.x * CW + warp) * gcap;
    cap = gcap;
    limit = (int)gcap;
  } else {
    keys = smem + warp * SIM_CAP;
    cap = SIM_CAP;
    limit = SIM_LIMIT;
  }
  for (int64_t t = (int64_t)blockIdx.x * CW + warp; t < nrowsI; t += (int64_t)gridDim.x * CW) {
    const int64_t I = list ? list[t] : t;
    for (uint32_t k = lane; k < cap; k += 32) keys[k] = -1;
    if (lane == 0) nfresh[warp] = 0;
    __syncwarp();
    bool over = false;
    for (int64_t m = boff[I]; m < boff[I + 1] && !over; ++m) {
      const int32_t r = perm[m];
      bool full = false;
      for (int64_t p = rowptr[r] + lane; p < rowptr[r + 1]; p += 32) {
        bool fresh;
        if (hset_insert(keys, cap - 1, blk[colind[p]], &fresh) < 0) {
          full = true;
          break;
        }
        if (fresh) atomicAdd(&nfresh[warp], 1);
      }
      __syncwarp();
      const int nf = *((volatile int*)&nfresh[warp]);
      over = __any_sync(0xffffffffu, full) || nf > limit;
    }
    if (over) {  // deferred to the global-table pass (pass 1 skips it)
      if (lane == 0) {
        if (GLOBAL)
          dev_fail(st, DEV_INTERNAL);
        else if (PASS == 0)
          heavy[atomicAdd(nheavy, 1)] = (int32_t)I;
      }
      __syncwarp();
      continue;
    }
    const int nf = *((volatile int*)&nfresh[warp]);
    if (PASS == 0) {
      if (lane == 0) bcnt[I] = nf;
    } else {
      // compact the keys to the front of the table, then rank-sort in place
      // into bcol[bptr[I] ...].
      int base = 0;
      for (uint32_t k0 = 0; k0 < cap; k0 += 32) {
        const uint32_t k = k0 + lane;
        const int key = k < cap ? keys[k] : -1;
        const unsigned b = __ballot_sync(0xffffffffu, key >= 0);
        __syncwarp();
        if (key >= 0) keys[base + __popc(b & ((1u << lane) - 1u))] = key;
        base += __popc(b);
        __syncwarp();
      }
      const int64_t out = bptr[I];
      for (int a = lane; a < nf; a += 32) {
        const int key = keys[a];
        int rank = 0;
        for (int q = 0; q < nf; ++q) rank += keys[q] < key ? 1 : 0;
        bcol[out + rank] = key;
      }
    }
    __syncwarp();
  }
}

// Scatter the CSR values into the zero-padded blocks (warp per original row).
__global__ void k_scatter_values(int64_t n, const int64_t* __restrict__ rowptr, const int32_t* __restrict__ colind,
                                 const double* __restrict__ val, const int32_t* __restrict__ blk,
                                 const int32_t* __restrict__ offin, const int32_t* __restrict__ bsz,
                                 const int64_t* __restrict__ bptr, const int32_t* __restrict__ bcol,
                                 const int64_t* __restrict__ voff, double* __restrict__ bval, int* st) {
  const int lane = threadIdx.x & 31;
  const int64_t wpb = blockDim.x >> 5;
  for (int64_t r = blockIdx.x * wpb + (threadIdx.x >> 5); r < n; r += (int64_t)gridDim.x * wpb) {
    const int32_t I = blk[r], a = offin[r];
    for (int64_t p = rowptr[r] + lane; p < rowptr[r + 1]; p += 32) {
      const int32_t c = colind[p];
      const int32_t J = blk[c];
      const int64_t b = bsearch_i32(bcol, bptr[I], bptr[I + 1], J);
      if (b < 0) {
        dev_fail(st, DEV_INTERNAL);
        continue;
      }
      bval[voff[b] + (int64_t)a * bsz[J] + offin[c]] = val[p];
    }
  }
}

}  // namespace

void validate_csr(int64_t n, const int64_t* rowptr, const int32_t* colind, int32_t* len, cudaStream_t s, int* dst) {
  if (n) {
    launch(k_validate, grid_for(n, 256), 256, 0, s, n, rowptr, colind, len, dst);
    VB_LAUNCH_CHECK();
  }
}

void compress_device(int64_t n, const int64_t* rowptr, const int32_t* colind, const double* val, double tau,
                     cudaStream_t s, int* dst, Compressed& out) {
  out.n = n;
  out.nnz = n ? d2h(rowptr + n, s) : 0;
  const int64_t nnz = out.nnz;
  DBuf<int32_t> len(n, s);
  if (n) {
    launch(k_validate, grid_for(n, 256), 256, 0, s, n, rowptr, colind, len.p, dst);
    VB_LAUNCH_CHECK();
  }
  check_status(dst, s, "vbarms_compress: CSR validation");

  // CSC pattern (column lists; their order is irrelevant: only counts are used)
  DBuf<int32_t> ccnt(n, s), crow(nnz, s);
  DBuf<int64_t> cptr(n + 1, s);
  ccnt.zero();
  if (nnz) {
    launch(k_col_count, grid_for(nnz, 256, 152LL * 64), 256, 0, s, nnz, colind, ccnt.p);
    VB_LAUNCH_CHECK();
  }
  scan_i32_to_i64(ccnt.p, cptr.p, n, s);
  ccnt.zero();
  if (n) {
    launch(k_col_fill, grid_for(n, 8), 256, 0, s, n, rowptr, colind, cptr.p, ccnt.p, crow.p);
    VB_LAUNCH_CHECK();
  }
  ccnt.release();

  // A2: similar pairs
  const double tau2 = tau * tau;
  DBuf<int64_t> simstart(n, s);
  DBuf<int32_t> simcnt(n, s), heavy(n, s);
  DBuf<unsigned long long> counters(2, s);  // [0] simtotal, [1] heavy bound
  DBuf<int> nheavy(1, s);
  int64_t simcap = std::max<int64_t>(1024, 8 * n);
  DBuf<int32_t> simbuf;
  const size_t smem_sim = (size_t)CW * 2 * SIM_CAP * sizeof(int);
  VB_CUDA(cudaFuncSetAttribute(k_similar<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_sim));
  for (int attempt = 0; attempt < 2; ++attempt) {
    simbuf.alloc(simcap, s);
    counters.zero();
    nheavy.zero();
    if (n) {
      launch(k_similar<false>, grid_for(n, CW, 152LL * 24), CW * 32, smem_sim, s, 
          n, nullptr, rowptr, colind, cptr.p, crow.p, len.p, tau2, nullptr, 0, simstart.p, simcnt.p, simbuf.p,
          simcap, counters.p, heavy.p, nheavy.p, dst);
      VB_LAUNCH_CHECK();
    }
    const int nh = d2h(nheavy.p, s);
    if (nh > 0) {
      launch(k_heavy_bound, grid_for(nh, 8), 256, 0, s, nh, heavy.p, rowptr, colind, cptr.p, n, counters.p + 1);
      VB_LAUNCH_CHECK();
      const uint64_t bound = d2h(counters.p + 1, s);
      uint32_t gcap = 1024;
      while (gcap < 2 * bound + 64) gcap <<= 1;
      const int64_t budget = 256LL << 20;  // bytes of global tables
      int64_t warps = std::max<int64_t>(1, budget / ((int64_t)gcap * 8));
      warps = std::min<int64_t>(warps, nh);
      const int64_t blocks = (warps + CW - 1) / CW;
      DBuf<int> gtab((size_t)blocks * CW * 2 * gcap, s);
      launch(k_similar<true>, (unsigned)blocks, CW * 32, 0, s, nh, heavy.p, rowptr, colind, cptr.p, crow.p, len.p,
                                                          tau2, gtab.p, gcap, simstart.p, simcnt.p, simbuf.p,
                                                          simcap, counters.p, nullptr, nullptr, dst);
      VB_LAUNCH_CHECK();
    }
    check_status(dst, s, "vbarms_compress: similarity");
    const uint64_t total = d2h(counters.p, s);
    if ((int64_t)total <= simcap) break;
    if (attempt == 1) fail(VB_EINTERNAL, "vbarms_compress: similarity buffer sizing");
    simcap = (int64_t)total + 1024;
  }
  cptr.release();
  crow.release();

  // A3: leaders in deterministic rounds
  DBuf<int32_t> pending(n, s), state(n, s), group(n, s), isleader(n, s);
  pending.zero();
  state.zero();
  group.fill_bytes(0x7f);
  if (n) {
    launch(k_pending, grid_for(n, 8), 256, 0, s, n, simstart.p, simcnt.p, simbuf.p, pending.p);
    VB_LAUNCH_CHECK();
  }
  DBuf<unsigned long long> remaining(1, s);
  {
    unsigned long long nn = (unsigned long long)n;
    h2d(remaining.p, &nn, 1, s);
  }
  for (int64_t round = 0; n > 0; ++round) {
    launch(k_round_a, grid_for(n, 256), 256, 0, s, n, simstart.p, simcnt.p, simbuf.p, pending.p, state.p, remaining.p);
    VB_LAUNCH_CHECK();
    launch(k_round_b, grid_for(n, 256), 256, 0, s, n, simstart.p, simcnt.p, simbuf.p, pending.p, state.p);
    VB_LAUNCH_CHECK();
    if ((round & 3) == 3 || round < 4) {
      if (d2h(remaining.p, s) == 0) break;
    }
    if (round > n + 8) fail(VB_EINTERNAL, "vbarms_compress: leader rounds did not terminate");
  }
  if (n) {
    launch(k_groups, grid_for(n, 256), 256, 0, s, n, simstart.p, simcnt.p, simbuf.p, state.p, group.p, isleader.p);
    VB_LAUNCH_CHECK();
  }
  DBuf<int64_t> lead_scan(n + 1, s);
  scan_i32_to_i64(isleader.p, lead_scan.p, n, s);
  const int64_t p = n ? d2h(lead_scan.p + n, s) : 0;
  DBuf<int32_t> blk(n, s), offin(n, s), bsz(p, s);
  bsz.zero();
  if (n) {
    launch(k_block_of, grid_for(n, 256), 256, 0, s, n, group.p, lead_scan.p, blk.p, bsz.p, dst);
    VB_LAUNCH_CHECK();
  }
  check_status(dst, s, "vbarms_compress: grouping");
  DBuf<int64_t> boff(p + 1, s);
  scan_i32_to_i64(bsz.p, boff.p, p, s);
  out.perm.alloc(n, s);
  if (n) {
    launch(k_member_rank, grid_for(n, 256), 256, 0, s, n, simstart.p, simcnt.p, simbuf.p, group.p, blk.p, boff.p,
                                                   offin.p, out.perm.p);
    VB_LAUNCH_CHECK();
  }
  pending.release();
  state.release();
  isleader.release();
  lead_scan.release();
  simbuf.release();
  heavy.release();
  assemble_vbcsr(n, rowptr, colind, val, p, bsz, boff, blk.p, offin.p, s, dst, out);
}

// A4: VBCSR of P_B A P_B^T from a grouping of the rows (out.perm already set).
void assemble_vbcsr(int64_t n, const int64_t* rowptr, const int32_t* colind, const double* val, int64_t p,
                    DBuf<int32_t>& bsz, DBuf<int64_t>& boff, const int32_t* blkp, const int32_t* offinp,
                    cudaStream_t s, int* dst, Compressed& out) {
  const int64_t nnz = out.nnz;
  DBuf<int32_t> heavy(std::max<int64_t>(n, 1), s);
  DBuf<int> nheavy(1, s);
  VBDev<double>& A = out.A;
  A.nbr = A.nbc = p;
  A.same_partition = true;
  A.rsz = std::move(bsz);
  A.roff = std::move(boff);
  A.bptr.alloc(p + 1, s);
  DBuf<int64_t> bcnt(p, s);
  const size_t smem_pat = (size_t)CW * SIM_CAP * sizeof(int);
  VB_CUDA(cudaFuncSetAttribute(k_block_pattern<false, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_pat));
  VB_CUDA(cudaFuncSetAttribute(k_block_pattern<false, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_pat));
  nheavy.zero();
  if (p) {
    launch(k_block_pattern<false, 0>, grid_for(p, CW, 152LL * 24), CW * 32, smem_pat, s, 
        p, nullptr, A.roff.p, out.perm.p, rowptr, colind, blkp, nullptr, 0, bcnt.p, nullptr, nullptr, heavy.p,
        nheavy.p, dst);
    VB_LAUNCH_CHECK();
  }
  const int nhb = d2h(nheavy.p, s);
  uint32_t gcapb = 0;
  DBuf<int> gtabb;
  int64_t hblocks = 0;
  if (nhb > 0) {
    // block rows with many distinct block columns use global tables sized by
    // the block count (an upper bound on the distinct columns)
    gcapb = 1024;
    while ((int64_t)gcapb < 2 * p + 64) gcapb <<= 1;
    int64_t warps = std::max<int64_t>(1, (256LL << 20) / ((int64_t)gcapb * 4));
    warps = std::min<int64_t>(warps, nhb);
    hblocks = (warps + CW - 1) / CW;
    gtabb.alloc((size_t)hblocks * CW * gcapb, s);
    launch(k_block_pattern<true, 0>, (unsigned)hblocks, CW * 32, 0, s, nhb, heavy.p, A.roff.p, out.perm.p, rowptr,
                                                                  colind, blkp, gtabb.p, gcapb, bcnt.p, nullptr,
                                                                  nullptr, nullptr, nullptr, dst);
    VB_LAUNCH_CHECK();
  }
  check_status(dst, s, "vbarms_compress: block pattern");
  scan_i64(bcnt.p, A.bptr.p, p, s);
  A.nnzb = p ? d2h(A.bptr.p + p, s) : 0;
  A.bcol.alloc(A.nnzb, s);
  if (p) {
    // the light pass skips the deferred rows (marked again, then ignored)
    DBuf<int> dummy(1, s);
    dummy.zero();
    DBuf<int32_t> hv2(std::max<int>(nhb, 1), s);
    launch(k_block_pattern<false, 1>, grid_for(p, CW, 152LL * 24), CW * 32, smem_pat, s, 
        p, nullptr, A.roff.p, out.perm.p, rowptr, colind, blkp, nullptr, 0, nullptr, A.bptr.p, A.bcol.p, hv2.p,
        dummy.p, dst);
    VB_LAUNCH_CHECK();
  }
  if (nhb > 0) {
    launch(k_block_pattern<true, 1>, (unsigned)hblocks, CW * 32, 0, s, nhb, heavy.p, A.roff.p, out.perm.p, rowptr,
                                                                  colind, blkp, gtabb.p, gcapb, nullptr, A.bptr.p,
                                                                  A.bcol.p, nullptr, nullptr, dst);
    VB_LAUNCH_CHECK();
  }
  check_status(dst, s, "vbarms_compress: block pattern");
  finish_offsets(A, s);
  A.val.zero();
  if (n) {
    launch(k_scatter_values, grid_for(n, 8), 256, 0, s, n, rowptr, colind, val, blkp, offinp, A.rsz.p, A.bptr.p,
                                                     A.bcol.p, A.voff.p, A.val.p, dst);
    VB_LAUNCH_CHECK();
  }
  check_status(dst, s, "vbarms_compress: value scatter");
  out.av_bd = A.nval ? (double)nnz / (double)A.nval : 0.0;
  out.av_bs = p ? (double)n / (double)p : 0.0;
}

}  // namespace vb
