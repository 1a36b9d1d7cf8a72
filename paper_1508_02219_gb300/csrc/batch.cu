// Batching of independent matrices: the block-diagonal union of several
// compressed matrices, so that one factorization (one launch per phase)
// serves all of them.  Every step of the method is local to a connected
// component of the block graph -- the scalings are row/column maxima, the
// greedy independent set decides each supernode from its own neighbours in
// (weight desc, index asc) order, P_I keeps the components' blocks in
// ascending order, W, G and S never couple two components, and the last
// level runs in natural order -- so the union's factors restricted to one
// matrix are that matrix's own factors, operation for operation.
#include <algorithm>

#include "internal.h"
#include "vbsr_ops.cuh"

namespace vb {
namespace {

// dst[e] = src[m][e - start[m]] + add[m] for e in [start[m], start[m + 1]):
// one launch concatenates one array of every part.
template <typename V>
__global__ void k_cat(int nparts, const int64_t* __restrict__ start, const V* const* __restrict__ src,
                      const V* __restrict__ add, V* __restrict__ dst) {
  const int64_t total = start[nparts];
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    int lo = 0, hi = nparts - 1;  // last part with start <= e
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (start[mid] <= e)
        lo = mid;
      else
        hi = mid - 1;
    }
    dst[e] = src[lo][e - start[lo]] + add[lo];
  }
}

// Concatenate one array over the parts: counts[m] entries of part m, shifted
// by add[m]; when tail is set, dst gets one more entry, tail_value.
template <typename V>
void cat(const std::vector<const V*>& src, const std::vector<int64_t>& counts, const std::vector<V>& add, V* dst,
         cudaStream_t s, bool tail = false, V tail_value = V(0)) {
  const int np = (int)src.size();
  std::vector<int64_t> start(np + 1, 0);
  for (int m = 0; m < np; ++m) start[m + 1] = start[m] + counts[m];
  DBuf<int64_t> dstart(np + 1, s);
  DBuf<const V*> dsrc(np, s);
  DBuf<V> dadd(np, s);
  h2d(dstart.p, start.data(), np + 1, s);
  h2d(dsrc.p, src.data(), np, s);
  h2d(dadd.p, add.data(), np, s);
  if (start[np] > 0) {
    launch(k_cat<V>, grid_for(start[np], 256), 256, 0, s, np, dstart.p, dsrc.p, dadd.p, dst);
    VB_LAUNCH_CHECK();
  }
  if (tail) h2d(dst + start[np], &tail_value, 1, s);
  // the host arrays above must outlive the copies
  VB_CUDA(cudaStreamSynchronize(s));
}

__global__ void k_part_ids(int nparts, const int64_t* __restrict__ start, int32_t* __restrict__ dom) {
  const int64_t total = start[nparts];
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    int lo = 0, hi = nparts - 1;  // last part with start <= e
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (start[mid] <= e)
        lo = mid;
      else
        hi = mid - 1;
    }
    dom[e] = lo;
  }
}

}  // namespace

void union_part_ids(const std::vector<const Compressed*>& parts, cudaStream_t s, DBuf<int32_t>& dom) {
  const int np = (int)parts.size();
  std::vector<int64_t> start(np + 1, 0);
  for (int m = 0; m < np; ++m) start[m + 1] = start[m] + parts[m]->A.nbr;
  dom.alloc(std::max<int64_t>(start[np], 1), s);
  if (start[np] == 0) return;
  DBuf<int64_t> dstart(np + 1, s);
  h2d(dstart.p, start.data(), np + 1, s);
  launch(k_part_ids, grid_for(start[np], 256), 256, 0, s, np, dstart.p, dom.p);
  VB_LAUNCH_CHECK();
  VB_CUDA(cudaStreamSynchronize(s));  // the host array must outlive the copy
}

void compressed_union(const std::vector<const Compressed*>& parts, cudaStream_t s, Compressed& out) {
  const int np = (int)parts.size();
  std::vector<int64_t> nbr(np), nnzb(np), nval(np), n(np);
  std::vector<int64_t> p_off(np + 1, 0), n_off(np + 1, 0), b_off(np + 1, 0), v_off(np + 1, 0);
  double area = 0;
  int64_t nnz = 0;
  for (int m = 0; m < np; ++m) {
    const Compressed& c = *parts[m];
    if (!c.A.same_partition) fail(VB_EINVAL, "batched factorization: a part is not square-partitioned");
    nbr[m] = c.A.nbr, nnzb[m] = c.A.nnzb, nval[m] = c.A.nval, n[m] = c.n;
    p_off[m + 1] = p_off[m] + nbr[m];
    n_off[m + 1] = n_off[m] + n[m];
    b_off[m + 1] = b_off[m] + nnzb[m];
    v_off[m + 1] = v_off[m] + nval[m];
    nnz += c.nnz;
    area += c.av_bd > 0 ? (double)c.nnz / c.av_bd : 0.0;
  }
  if (p_off[np] > INT32_MAX || n_off[np] > INT32_MAX)
    fail(VB_EINVAL, "batched factorization: the batch exceeds 2^31 rows or blocks");
  VBDev<double>& U = out.A;
  U.nbr = U.nbc = p_off[np];
  U.nnzb = b_off[np];
  U.nval = v_off[np];
  U.same_partition = true;
  out.n = n_off[np];
  out.nnz = nnz;
  out.av_bd = area > 0 ? (double)nnz / area : 0.0;
  out.av_bs = U.nbr ? (double)out.n / (double)U.nbr : 0.0;
  U.rsz.alloc(U.nbr, s);
  U.roff.alloc(U.nbr + 1, s);
  U.bptr.alloc(U.nbr + 1, s);
  U.bcol.alloc(U.nnzb, s);
  U.voff.alloc(U.nnzb + 1, s);
  U.val.alloc(U.nval, s);
  out.perm.alloc(out.n, s);
  std::vector<const int32_t*> s_rsz(np), s_bcol(np), s_perm(np);
  std::vector<const int64_t*> s_roff(np), s_bptr(np), s_voff(np);
  std::vector<const double*> s_val(np);
  std::vector<int32_t> a_zero32(np, 0), a_p(np), a_n(np);
  std::vector<int64_t> a_n64(np), a_b(np), a_v(np);
  std::vector<double> a_zero(np, 0.0);
  for (int m = 0; m < np; ++m) {
    const VBDev<double>& A = parts[m]->A;
    s_rsz[m] = A.rsz.p, s_bcol[m] = A.bcol.p, s_perm[m] = parts[m]->perm.p;
    s_roff[m] = A.roff.p, s_bptr[m] = A.bptr.p, s_voff[m] = A.voff.p, s_val[m] = A.val.p;
    a_p[m] = (int32_t)p_off[m], a_n[m] = (int32_t)n_off[m];
    a_n64[m] = n_off[m], a_b[m] = b_off[m], a_v[m] = v_off[m];
  }
  cat<int32_t>(s_rsz, nbr, a_zero32, U.rsz.p, s);
  cat<int64_t>(s_roff, nbr, a_n64, U.roff.p, s, true, n_off[np]);
  cat<int64_t>(s_bptr, nbr, a_b, U.bptr.p, s, true, b_off[np]);
  cat<int32_t>(s_bcol, nnzb, a_p, U.bcol.p, s);
  cat<int64_t>(s_voff, nnzb, a_v, U.voff.p, s, true, v_off[np]);
  cat<double>(s_val, nval, a_zero, U.val.p, s);
  cat<int32_t>(s_perm, n, a_n, out.perm.p, s);
}

}  // namespace vb
