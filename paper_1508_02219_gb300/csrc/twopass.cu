// Two-pass checksum and angle compression of VBARMS on the GPU (Section 2.1,
// the variant that first groups rows of identical pattern, then scans the
// other rows again):
//   T1  classes of identical stored row patterns (list_classes: a hash of
//       each sorted pattern, a sort, exact comparisons); a class of two or
//       more nonempty rows is a group, groups in ascending order of their
//       smallest row, which carries the group's pattern
//   T2  every other nonempty row j joins the first group g whose pattern
//       passes the angle test |P_j n P_g|^2 >= tau^2 |P_j| |P_g| (one exactly
//       rounded product, as in the one-pass method); the groups' patterns do
//       not change as rows join, so every row decides on its own: one warp
//       per row counts its overlaps with the groups that share a column (a
//       shared-memory hash over the column lists of the groups' patterns)
//   T3  blocks in ascending order of their smallest row, rows ascending (a
//       joining row may precede its group's rows).
#include <climits>

#include "internal.h"

namespace vb {
namespace {

constexpr int TW = 4;       // warps per block of the second pass (32 KB of hash)
constexpr int THC = 1024;   // hash positions per warp

__global__ void k_class_count(int64_t n, const int32_t* __restrict__ leader, int32_t* __restrict__ cnt) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(&cnt[leader[v]], 1);
}

// group leaders: the smallest row of a class of two or more nonempty rows
__global__ void k_group_flag(int64_t n, const int64_t* __restrict__ rowptr, const int32_t* __restrict__ leader,
                             const int32_t* __restrict__ cnt, int32_t* __restrict__ isg) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
    isg[v] = (leader[v] == (int32_t)v && cnt[v] >= 2 && rowptr[v + 1] > rowptr[v]) ? 1 : 0;
}

__global__ void k_group_ref(int64_t n, const int32_t* __restrict__ isg, const int64_t* __restrict__ gscan,
                            const int64_t* __restrict__ rowptr, int32_t* __restrict__ ref,
                            int64_t* __restrict__ rlen) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
    if (isg[v]) {
      ref[gscan[v]] = (int32_t)v;
      rlen[gscan[v]] = rowptr[v + 1] - rowptr[v];
    }
}

// (column, group) pairs of the groups' patterns, key = column << 32 | group
__global__ void k_ref_pairs(int64_t ng, const int32_t* __restrict__ ref, const int64_t* __restrict__ roff,
                            const int64_t* __restrict__ rowptr, const int32_t* __restrict__ colind,
                            unsigned long long* __restrict__ key) {
  const int lane = threadIdx.x & 31;
  const int64_t wpb = blockDim.x >> 5;
  for (int64_t g = blockIdx.x * wpb + (threadIdx.x >> 5); g < ng; g += (int64_t)gridDim.x * wpb) {
    const int32_t r = ref[g];
    for (int64_t q = rowptr[r] + lane; q < rowptr[r + 1]; q += 32)
      key[roff[g] + (q - rowptr[r])] = ((unsigned long long)(unsigned)colind[q] << 32) | (unsigned long long)g;
  }
}

__global__ void k_col_groups(int64_t m, const unsigned long long* __restrict__ key, int32_t* __restrict__ cg,
                             int32_t* __restrict__ ccnt) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < m; k += (int64_t)gridDim.x * blockDim.x) {
    cg[k] = (int32_t)(key[k] & 0xffffffffull);
    atomicAdd(&ccnt[key[k] >> 32], 1);
  }
}

// |P_a n P_b| of two sorted patterns.
__device__ int64_t overlap(const int32_t* __restrict__ a, int64_t na, const int32_t* __restrict__ b, int64_t nb) {
  int64_t i = 0, j = 0, c = 0;
  while (i < na && j < nb) {
    if (a[i] == b[j]) {
      ++c;
      ++i;
      ++j;
    } else if (a[i] < b[j]) {
      ++i;
    } else {
      ++j;
    }
  }
  return c;
}

// The second pass, one warp per row: join[j] = the first group passing the
// angle test, -1 when none does; -2 for rows of a group and empty rows.
__global__ void __launch_bounds__(TW * 32)
    k_join(int64_t n, const int64_t* __restrict__ rowptr, const int32_t* __restrict__ colind,
           const int32_t* __restrict__ leader, const int32_t* __restrict__ cnt, const int64_t* __restrict__ cptr,
           const int32_t* __restrict__ cg, const int32_t* __restrict__ ref, const int64_t* __restrict__ rlen,
           double tau2, int32_t* __restrict__ join) {
  __shared__ int hkey[TW][THC];
  __shared__ int hcnt[TW][THC];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int* keys = hkey[warp];
  int* cts = hcnt[warp];
  for (int q = lane; q < THC; q += 32) {
    keys[q] = -1;
    cts[q] = 0;
  }
  __syncwarp();
  const int64_t wpb = blockDim.x >> 5;
  for (int64_t j = blockIdx.x * wpb + warp; j < n; j += (int64_t)gridDim.x * wpb) {
    const int64_t p0 = rowptr[j], nj = rowptr[j + 1] - p0;
    const bool grouped = cnt[leader[j]] >= 2 && nj > 0;
    if (grouped || nj == 0) {
      if (lane == 0) join[j] = -2;
      continue;
    }
    // candidate bound: the groups listed under the row's columns
    long long bound = 0;
    for (int64_t q = lane; q < nj; q += 32) bound += cptr[colind[p0 + q] + 1] - cptr[colind[p0 + q]];
    bound = warp_sum_ll(bound);
    int best = INT_MAX;
    if (bound <= THC / 2) {
      for (int64_t q = 0; q < nj; ++q) {
        const int32_t c = colind[p0 + q];
        for (int64_t e = cptr[c] + lane; e < cptr[c + 1]; e += 32) {
          bool fresh;
          const int slot = hset_insert(keys, THC - 1, cg[e], &fresh);
          if (slot >= 0) atomicAdd(&cts[slot], 1);
        }
      }
      __syncwarp();
      for (int q = lane; q < THC; q += 32) {
        const int g = keys[q];
        if (g >= 0) {
          const long long c = cts[q];
          if ((double)(c * c) >= tau2 * (double)(nj * rlen[g])) best = min(best, g);
        }
      }
      __syncwarp();
      for (int q = lane; q < THC; q += 32) {
        keys[q] = -1;
        cts[q] = 0;
      }
      __syncwarp();
    } else {
      // many candidates: exact overlaps by merging the sorted patterns
      for (int64_t q = 0; q < nj; ++q) {
        const int32_t c = colind[p0 + q];
        for (int64_t e = cptr[c] + lane; e < cptr[c + 1]; e += 32) {
          const int g = cg[e];
          if (g >= best) continue;
          const int32_t r = ref[g];
          const long long ov = overlap(colind + p0, nj, colind + rowptr[r], rlen[g]);
          if ((double)(ov * ov) >= tau2 * (double)(nj * rlen[g])) best = min(best, g);
        }
      }
    }
    best = warp_min_i(best);
    if (lane == 0) join[j] = best == INT_MAX ? -1 : best;
  }
}

__global__ void k_gmin(int64_t n, const int32_t* __restrict__ join, int32_t* __restrict__ gmin) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
    if (join[v] >= 0) atomicMin(&gmin[join[v]], (int32_t)v);
}

__global__ void k_two_pass_lead(int64_t n, const int32_t* __restrict__ leader, const int32_t* __restrict__ join,
                                const int64_t* __restrict__ gscan, const int32_t* __restrict__ isg,
                                const int32_t* __restrict__ gmin, int32_t* __restrict__ lead) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    const int32_t jv = join[v];
    if (jv >= 0)
      lead[v] = gmin[jv];
    else if (jv == -2 && isg[leader[v]])
      lead[v] = gmin[gscan[leader[v]]];
    else
      lead[v] = (int32_t)v;
  }
}

}  // namespace

void two_pass_compress_device(int64_t n, const int64_t* rowptr, const int32_t* colind, const double* val,
                              double tau, cudaStream_t s, int* dst, Compressed& out) {
  out.n = n;
  out.nnz = n ? d2h(rowptr + n, s) : 0;
  {
    DBuf<int32_t> len(std::max<int64_t>(n, 1), s);
    if (n) validate_csr(n, rowptr, colind, len.p, s, dst);
  }
  check_status(dst, s, "vbarms_compress_two_pass: CSR validation");
  DBuf<int32_t> lead(std::max<int64_t>(n, 1), s);
  if (n) {
    // T1: classes of identical row patterns; the groups
    DBuf<int32_t> leader(n, s), cnt(n, s), isg(n, s);
    list_classes(n, rowptr, colind, leader.p, s);
    cnt.zero();
    launch(k_class_count, grid_for(n, 256), 256, 0, s, n, leader.p, cnt.p);
    VB_LAUNCH_CHECK();
    launch(k_group_flag, grid_for(n, 256), 256, 0, s, n, rowptr, leader.p, cnt.p, isg.p);
    VB_LAUNCH_CHECK();
    DBuf<int64_t> gscan(n + 1, s);
    scan_i32_to_i64(isg.p, gscan.p, n, s);
    const int64_t ng = d2h(gscan.p + n, s);
    DBuf<int32_t> ref(std::max<int64_t>(ng, 1), s), gmin(std::max<int64_t>(ng, 1), s), join(n, s);
    DBuf<int64_t> rlen(std::max<int64_t>(ng, 1), s), roff(ng + 1, s);
    DBuf<int64_t> cptr(n + 1, s);
    DBuf<int32_t> ccnt(n, s);
    ccnt.zero();
    DBuf<int32_t> cg;
    if (ng) {
      launch(k_group_ref, grid_for(n, 256), 256, 0, s, n, isg.p, gscan.p, rowptr, ref.p, rlen.p);
      VB_LAUNCH_CHECK();
      scan_i64(rlen.p, roff.p, ng, s);
      const int64_t m = d2h(roff.p + ng, s);
      DBuf<unsigned long long> key(m, s);
      launch(k_ref_pairs, grid_for(ng, 8), 256, 0, s, ng, ref.p, roff.p, rowptr, colind, key.p);
      VB_LAUNCH_CHECK();
      int cbits = 1;
      while (cbits < 62 && (1LL << cbits) <= n) ++cbits;
      int gbits = 1;
      while (gbits < 31 && (1LL << gbits) <= ng) ++gbits;
      // sort by (column, group): low 32 bits hold the group, so the sorted
      // range covers bits 0..31 and the column's bits above
      radix_sort_u64(key, nullptr, m, 32 + cbits, s);
      cg.alloc(m, s);
      launch(k_col_groups, grid_for(m, 256), 256, 0, s, m, key.p, cg.p, ccnt.p);
      VB_LAUNCH_CHECK();
      (void)gbits;
      VB_CUDA(cudaMemcpyAsync(gmin.p, ref.p, ng * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
    }
    scan_i32_to_i64(ccnt.p, cptr.p, n, s);
    // T2: the other rows
    launch(k_join, grid_for(n, TW, 152LL * 16), TW * 32, 0, s, n, rowptr, colind, leader.p, cnt.p, cptr.p,
           ng ? cg.p : nullptr, ref.p, rlen.p, tau * tau, join.p);
    VB_LAUNCH_CHECK();
    if (ng) {
      launch(k_gmin, grid_for(n, 256), 256, 0, s, n, join.p, gmin.p);
      VB_LAUNCH_CHECK();
    }
    launch(k_two_pass_lead, grid_for(n, 256), 256, 0, s, n, leader.p, join.p, gscan.p, isg.p, gmin.p, lead.p);
    VB_LAUNCH_CHECK();
  }
  assemble_from_leaders(n, rowptr, colind, val, lead.p, s, dst, out);
}

}  // namespace vb
