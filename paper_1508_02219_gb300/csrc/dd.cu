// Section 5 global preconditioners on one GPU: block Jacobi and (restricted)
// additive Schwarz with VBARMS as the local solver.
//
// Subdomain i is a contiguous range W_i^0 of the compressed block rows
// (part(I) = floor(N * roff_I / n)), extended delta times by the block graph
// of A + A^T (W_i^d = adj(W_i^{d-1})); its local matrix A_i = R_i A R_i keeps
// the stored blocks with row and column in W_i^delta, in ascending order.
// All A_i are laid out as one block-diagonal union (subdomain-major) and
// factored by one multilevel factorization: every step of the method is
// local to a connected component, so the union's factors restricted to
// subdomain i are A_i's own.  Applying the preconditioner gathers R_i x of
// every subdomain into the union vector, runs one union solve, and then adds
// the local results (additive; block Jacobi when delta = 0) or takes each
// row from the subdomain that owns it (restricted).
//
// Subdomain membership is a bit mask per block row (32 subdomains a word), so
// every set operation is a word-wise OR and the result does not depend on
// the order in which threads run.
#include "prec.cuh"
#include "vbsr_ops.cuh"

namespace vb {
namespace {

constexpr int DCH = 256;  // block rows per chunk (one block of threads) of the union listing

__global__ void k_dd_init(int64_t p, int64_t n, int nparts, int nw, const int64_t* __restrict__ roff,
                          int32_t* __restrict__ part, uint32_t* __restrict__ mask) {
  for (int64_t I = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; I < p; I += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(((int64_t)nparts * roff[I]) / n);
    part[I] = i;
    for (int w = 0; w < nw; ++w) mask[I * nw + w] = w == (i >> 5) ? (1u << (i & 31)) : 0u;
  }
}

// One overlap level, next = adj(old) on the graph of A + A^T (next starts as
// a copy of old): a stored block (I, J) hands J's subdomains to I (an OR over
// the warp's blocks) and I's subdomains to J (an atomic OR, issued only for
// bits J does not hold yet).
__global__ void k_dd_expand(VBView<double> A, int nw, const uint32_t* __restrict__ old,
                            uint32_t* __restrict__ next) {
  const int lane = threadIdx.x & 31;
  const int64_t wpb = blockDim.x >> 5;
  for (int64_t I = blockIdx.x * wpb + (threadIdx.x >> 5); I < A.nbr; I += (int64_t)gridDim.x * wpb) {
    const int64_t b0 = A.bptr[I], b1 = A.bptr[I + 1];
    for (int w = 0; w < nw; ++w) {
      const uint32_t oI = old[I * nw + w];
      uint32_t acc = 0;
      for (int64_t b = b0 + lane; b < b1; b += 32) {
        const int64_t J = A.bcol[b];
        const uint32_t oJ = old[J * nw + w];
        acc |= oJ;
        if (oI & ~oJ) atomicOr(&next[J * nw + w], oI);
      }
      acc = __reduce_or_sync(0xffffffffu, acc);
      if (lane == 0 && (acc & ~oI)) atomicOr(&next[I * nw + w], acc);
    }
  }
}

// Members of subdomain i among the DCH block rows of chunk c: cnt[i * nch + c]
// (count pass), then their union positions base[i * nch + c] + rank (fill
// pass): the union lists subdomain 0's block rows ascending, then 1's, ...
template <bool FILL>
__global__ void k_dd_list(int64_t p, int nparts, int nw, int64_t nch, const uint32_t* __restrict__ mask,
                          int32_t* __restrict__ cnt, const int64_t* __restrict__ base, int32_t* __restrict__ ug,
                          int32_t* __restrict__ ud) {
  __shared__ int wc[DCH / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int64_t c = blockIdx.x; c < nch; c += gridDim.x) {
    const int64_t I = c * DCH + threadIdx.x;
    for (int w = 0; w < nw; ++w) {
      const uint32_t word = I < p ? mask[I * nw + w] : 0u;
      for (int bit = 0; bit < 32 && w * 32 + bit < nparts; ++bit) {
        const int i = w * 32 + bit;
        const bool has = (word >> bit) & 1u;
        const unsigned bal = __ballot_sync(0xffffffffu, has);
        if (lane == 0) wc[warp] = __popc(bal);
        __syncthreads();
        if (!FILL) {
          if (threadIdx.x == 0) {
            int s = 0;
            for (int k = 0; k < DCH / 32; ++k) s += wc[k];
            cnt[(int64_t)i * nch + c] = s;
          }
        } else if (has) {
          int pre = 0;
          for (int k = 0; k < warp; ++k) pre += wc[k];
          const int64_t pos = base[(int64_t)i * nch + c] + pre + __popc(bal & ((1u << lane) - 1u));
          ug[pos] = (int32_t)I;
          ud[pos] = i;
        }
        __syncthreads();
      }
    }
  }
}

__global__ void k_dd_dstart(int nparts, int64_t nch, const int64_t* __restrict__ base, int64_t* __restrict__ dstart) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i <= nparts; i += gridDim.x * blockDim.x)
    dstart[i] = base[(int64_t)i * nch];
}

__device__ __forceinline__ bool dd_member(const uint32_t* mask, int nw, int64_t J, int i) {
  return (mask[J * nw + (i >> 5)] >> (i & 31)) & 1u;
}

// Union row k (block row ug[k] of A in subdomain ud[k]): its blocks are those
// of A's row with the column in the subdomain; count pass, then the union
// column (the union row of (ud[k], J), found by binary search in the
// subdomain's ascending list) and the source block.
template <bool FILL>
__global__ void k_dd_rows(int64_t m, VBView<double> A, int nw, const uint32_t* __restrict__ mask,
                          const int32_t* __restrict__ ug, const int32_t* __restrict__ ud,
                          const int64_t* __restrict__ dstart, int32_t* __restrict__ cnt,
                          const int64_t* __restrict__ ubptr, int32_t* __restrict__ ubcol, int64_t* __restrict__ srcb) {
  const int lane = threadIdx.x & 31;
  const int64_t wpb = blockDim.x >> 5;
  for (int64_t k = blockIdx.x * wpb + (threadIdx.x >> 5); k < m; k += (int64_t)gridDim.x * wpb) {
    const int64_t I = ug[k];
    const int i = ud[k];
    const int64_t b0 = A.bptr[I], b1 = A.bptr[I + 1];
    int64_t pos = FILL ? ubptr[k] : 0;
    int c = 0;
    for (int64_t bb = b0; bb < b1; bb += 32) {
      const int64_t b = bb + lane;
      const bool in = b < b1 && dd_member(mask, nw, A.bcol[b], i);
      const unsigned bal = __ballot_sync(0xffffffffu, in);
      if (FILL && in) {
        const int64_t d = pos + __popc(bal & ((1u << lane) - 1u));
        ubcol[d] = (int32_t)bsearch_i32(ug, dstart[i], dstart[i + 1], A.bcol[b]);
        srcb[d] = b;
      }
      pos += __popc(bal);
      c += __popc(bal);
    }
    if (!FILL && lane == 0) cnt[k] = c;
  }
}

__global__ void k_dd_values(int64_t m, const int64_t* __restrict__ ubptr, const int64_t* __restrict__ uvoff,
                            const int64_t* __restrict__ srcb, const int64_t* __restrict__ avoff,
                            const double* __restrict__ aval, double* __restrict__ uval) {
  const int lane = threadIdx.x & 31;
  const int64_t wpb = blockDim.x >> 5;
  for (int64_t k = blockIdx.x * wpb + (threadIdx.x >> 5); k < m; k += (int64_t)gridDim.x * wpb)
    for (int64_t d = ubptr[k]; d < ubptr[k + 1]; ++d) {
      const int64_t s0 = avoff[srcb[d]], len = uvoff[d + 1] - uvoff[d];
      for (int64_t e = lane; e < len; e += 32) uval[uvoff[d] + e] = aval[s0 + e];
    }
}

__global__ void k_dd_take_rsz(int64_t m, const int32_t* __restrict__ ug, const int32_t* __restrict__ rsz,
                              int32_t* __restrict__ ursz) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < m; k += (int64_t)gridDim.x * blockDim.x)
    ursz[k] = rsz[ug[k]];
}

// gidx: union scalar row -> scalar row of A; src: scalar row of A -> its copy
// in the owning subdomain.
__global__ void k_dd_maps(int64_t m, const int32_t* __restrict__ ug, const int32_t* __restrict__ ud,
                          const int32_t* __restrict__ part, const int32_t* __restrict__ rsz,
                          const int64_t* __restrict__ roff, const int64_t* __restrict__ uroff,
                          int32_t* __restrict__ gidx, int32_t* __restrict__ src) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < m; k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t I = ug[k];
    const bool own = ud[k] == part[I];
    for (int a = 0; a < rsz[I]; ++a) {
      gidx[uroff[k] + a] = (int32_t)(roff[I] + a);
      if (own) src[roff[I] + a] = (int32_t)(uroff[k] + a);
    }
  }
}

// The copies of every block row of A, in subdomain order (additive sum).
template <bool FILL>
__global__ void k_dd_copies(int64_t p, int nparts, int nw, const uint32_t* __restrict__ mask,
                            const int32_t* __restrict__ ug, const int64_t* __restrict__ dstart,
                            int32_t* __restrict__ ccnt, const int64_t* __restrict__ cptr, int32_t* __restrict__ clist) {
  for (int64_t I = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; I < p; I += (int64_t)gridDim.x * blockDim.x) {
    int c = 0;
    for (int w = 0; w < nw; ++w) {
      uint32_t word = mask[I * nw + w];
      if constexpr (!FILL) {
        c += __popc(word);
      } else {
        while (word) {
          const int i = w * 32 + __ffs(word) - 1;
          word &= word - 1;
          clist[cptr[I] + c] = (int32_t)bsearch_i32(ug, dstart[i], dstart[i + 1], (int32_t)I);
          ++c;
        }
      }
    }
    if constexpr (!FILL) ccnt[I] = c;
  }
}

__global__ void k_dd_add(int64_t p, const int32_t* __restrict__ rsz, const int64_t* __restrict__ roff,
                         const int64_t* __restrict__ cptr, const int32_t* __restrict__ clist,
                         const int64_t* __restrict__ uroff, const double* __restrict__ yu, double* __restrict__ y) {
  const int lane = threadIdx.x & 31;
  const int64_t wpb = blockDim.x >> 5;
  for (int64_t I = blockIdx.x * wpb + (threadIdx.x >> 5); I < p; I += (int64_t)gridDim.x * wpb)
    for (int a = lane; a < rsz[I]; a += 32) {
      double acc = 0.0;
      for (int64_t c = cptr[I]; c < cptr[I + 1]; ++c) acc = __dadd_rn(acc, yu[uroff[clist[c]] + a]);
      y[roff[I] + a] = acc;
    }
}

__global__ void k_dd_iota(int64_t n, int32_t* __restrict__ v) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    v[i] = (int32_t)i;
}

__global__ void k_dd_count_nz(int64_t n, const double* __restrict__ v, unsigned long long* __restrict__ out) {
  unsigned long long c = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    c += v[i] != 0.0;
  c = (unsigned long long)warp_sum_ll((long long)c);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(out, c);
}

}  // namespace

void dd_build(const Compressed& A, int nparts, int overlap, bool restricted, cudaStream_t s, DDLayout& L,
              Compressed& U) {
  const VBDev<double>& M = A.A;
  const int64_t p = M.nbr, n = A.n;
  if (!M.same_partition) fail(VB_EINVAL, "vbarms_dd_factor: the matrix is not square-partitioned");
  if (nparts < 1 || nparts > kDDMaxParts) fail(VB_EINVAL, "vbarms_dd_factor: nparts must lie in [1, 4096]");
  if (overlap < 0) fail(VB_EINVAL, "vbarms_dd_factor: overlap < 0");
  L.nparts = nparts;
  L.overlap = overlap;
  L.restricted = restricted;
  L.n = n;
  L.p = p;
  const int nw = (nparts + 31) / 32;
  L.part.alloc(std::max<int64_t>(p, 1), s);
  L.rsz.alloc(std::max<int64_t>(p, 1), s);
  L.roff.alloc(p + 1, s);
  if (p) {
    VB_CUDA(cudaMemcpyAsync(L.rsz.p, M.rsz.p, p * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
  }
  VB_CUDA(cudaMemcpyAsync(L.roff.p, M.roff.p, (p + 1) * sizeof(int64_t), cudaMemcpyDeviceToDevice, s));
  DBuf<uint32_t> mask(std::max<int64_t>(p * nw, 1), s), next(std::max<int64_t>(p * nw, 1), s);
  if (p) {
    launch(k_dd_init, grid_for(p, 256), 256, 0, s, p, n, nparts, nw, M.roff.p, L.part.p, mask.p);
    VB_LAUNCH_CHECK();
  }
  for (int d = 0; d < overlap && p; ++d) {
    VB_CUDA(cudaMemcpyAsync(next.p, mask.p, p * nw * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s));
    launch(k_dd_expand, grid_for(p, 8), 256, 0, s, M.view(), nw, mask.p, next.p);
    VB_LAUNCH_CHECK();
    std::swap(mask, next);
  }
  // the union's block rows, subdomain-major
  const int64_t nch = std::max<int64_t>((p + DCH - 1) / DCH, 1);
  DBuf<int32_t> cnt(nparts * nch, s);
  DBuf<int64_t> base(nparts * nch + 1, s);
  launch(k_dd_list<false>, grid_for(nch, 1), DCH, 0, s, p, nparts, nw, nch, mask.p, cnt.p, nullptr, nullptr, nullptr);
  VB_LAUNCH_CHECK();
  scan_i32_to_i64(cnt.p, base.p, nparts * nch, s);
  const int64_t m = d2h(base.p + nparts * nch, s);
  if (m > INT32_MAX) fail(VB_EINVAL, "vbarms_dd_factor: the subdomains exceed 2^31 block rows in total");
  L.m = m;
  L.ug.alloc(std::max<int64_t>(m, 1), s);
  L.ud.alloc(std::max<int64_t>(m, 1), s);
  L.dstart.alloc(nparts + 1, s);
  launch(k_dd_list<true>, grid_for(nch, 1), DCH, 0, s, p, nparts, nw, nch, mask.p, nullptr, base.p, L.ug.p, L.ud.p);
  VB_LAUNCH_CHECK();
  launch(k_dd_dstart, grid_for(nparts + 1, 256), 256, 0, s, nparts, nch, base.p, L.dstart.p);
  VB_LAUNCH_CHECK();

  // the union matrix
  VBDev<double>& V = U.A;
  {
    DBuf<int32_t> ursz(std::max<int64_t>(m, 1), s);
    if (m) {
      launch(k_dd_take_rsz, grid_for(m, 256), 256, 0, s, m, L.ug.p, M.rsz.p, ursz.p);
      VB_LAUNCH_CHECK();
    }
    set_partitions(V, ursz.p, m, ursz.p, m, s);
  }
  V.bptr.alloc(m + 1, s);
  {
    DBuf<int32_t> rc(std::max<int64_t>(m, 1), s);
    if (m) {
      launch(k_dd_rows<false>, grid_for(m, 8), 256, 0, s, m, M.view(), nw, mask.p, L.ug.p, L.ud.p, L.dstart.p, rc.p,
             nullptr, nullptr, nullptr);
      VB_LAUNCH_CHECK();
    }
    scan_i32_to_i64(rc.p, V.bptr.p, m, s);
  }
  V.nnzb = m ? d2h(V.bptr.p + m, s) : 0;
  V.bcol.alloc(std::max<int64_t>(V.nnzb, 1), s);
  DBuf<int64_t> srcb(std::max<int64_t>(V.nnzb, 1), s);
  if (m) {
    launch(k_dd_rows<true>, grid_for(m, 8), 256, 0, s, m, M.view(), nw, mask.p, L.ug.p, L.ud.p, L.dstart.p, nullptr,
           V.bptr.p, V.bcol.p, srcb.p);
    VB_LAUNCH_CHECK();
  }
  finish_offsets(V, s);
  if (m && V.nval) {
    launch(k_dd_values, grid_for(m, 8), 256, 0, s, m, V.bptr.p, V.voff.p, srcb.p, M.voff.p, M.val.p, V.val.p);
    VB_LAUNCH_CHECK();
  }
  U.n = V.nrows_scalar(s);
  L.nu = U.n;
  if (U.n > INT32_MAX) fail(VB_EINVAL, "vbarms_dd_factor: the subdomains exceed 2^31 rows in total");
  U.perm.alloc(std::max<int64_t>(U.n, 1), s);
  if (U.n) {
    launch(k_dd_iota, grid_for(U.n, 256), 256, 0, s, U.n, U.perm.p);
    VB_LAUNCH_CHECK();
  }
  {
    DBuf<unsigned long long> nz(1, s);
    nz.zero();
    if (V.nval) {
      launch(k_dd_count_nz, grid_for(V.nval, 256), 256, 0, s, V.nval, V.val.p, nz.p);
      VB_LAUNCH_CHECK();
    }
    U.nnz = (int64_t)d2h(nz.p, s);
  }
  U.av_bd = U.av_bs = 0.0;

  // application maps
  L.uroff.alloc(m + 1, s);
  VB_CUDA(cudaMemcpyAsync(L.uroff.p, V.roff.p, (m + 1) * sizeof(int64_t), cudaMemcpyDeviceToDevice, s));
  L.gidx.alloc(std::max<int64_t>(U.n, 1), s);
  L.src.alloc(std::max<int64_t>(n, 1), s);
  if (m) {
    launch(k_dd_maps, grid_for(m, 256), 256, 0, s, m, L.ug.p, L.ud.p, L.part.p, M.rsz.p, M.roff.p, V.roff.p,
           L.gidx.p, L.src.p);
    VB_LAUNCH_CHECK();
  }
  if (!restricted) {
    DBuf<int32_t> cc(std::max<int64_t>(p, 1), s);
    L.cptr.alloc(p + 1, s);
    if (p) {
      launch(k_dd_copies<false>, grid_for(p, 256), 256, 0, s, p, nparts, nw, mask.p, L.ug.p, L.dstart.p, cc.p,
             nullptr, nullptr);
      VB_LAUNCH_CHECK();
    }
    scan_i32_to_i64(cc.p, L.cptr.p, p, s);
    const int64_t nc = p ? d2h(L.cptr.p + p, s) : 0;
    L.clist.alloc(std::max<int64_t>(nc, 1), s);
    if (p) {
      launch(k_dd_copies<true>, grid_for(p, 256), 256, 0, s, p, nparts, nw, mask.p, L.ug.p, L.dstart.p, nullptr,
             L.cptr.p, L.clist.p);
      VB_LAUNCH_CHECK();
    }
  }
  VB_CUDA(cudaStreamSynchronize(s));
}

namespace {
// y (A's P_B numbering) from the union solve yu: the owning subdomain's rows
// (restricted) or the sum over the copies in subdomain order (additive).
void dd_combine(const DDLayout& L, const double* yu, double* y, cudaStream_t s) {
  if (L.restricted) {
    if (L.n) gather_dev(y, yu, L.src.p, L.n, s);
  } else if (L.p) {
    launch(k_dd_add, grid_for(L.p, 8), 256, 0, s, L.p, L.rsz.p, L.roff.p, L.cptr.p, L.clist.p, L.uroff.p, yu, y);
    VB_LAUNCH_CHECK();
  }
}
inline size_t al256(size_t v) { return (v + 255) & ~(size_t)255; }
}  // namespace

// y = sum_i Q_i^T A_i^{-1} R_i x in the P_B numbering of A (xu, yu: union
// vectors of L.nu entries).
void dd_apply(const DDLayout& L, PrecBase& inner, const double* x, double* y, double* xu, double* yu,
              cudaStream_t s) {
  if (L.nu) gather_dev(xu, x, L.gidx.p, L.nu, s);
  inner.apply_perm(xu, yu);
  dd_combine(L, yu, y, s);
}

size_t PrecDD::scratch_bytes() const {
  return 2 * al256((size_t)n * 8) + 2 * al256((size_t)L.nu * 8) + inner->scratch_bytes();
}

// The same in the original numbering with caller scratch only (the union's
// own numbering is the identity, so the inner call's permutation is a copy).
void PrecDD::apply_with_scratch(const double* x, double* y, unsigned char* scratch, int nsm) {
  size_t o = 0;
  double* xp = (double*)(scratch + o);
  o += al256((size_t)n * 8);
  double* yp = (double*)(scratch + o);
  o += al256((size_t)n * 8);
  double* xs = (double*)(scratch + o);
  o += al256((size_t)L.nu * 8);
  double* ys = (double*)(scratch + o);
  o += al256((size_t)L.nu * 8);
  if (n) gather_dev(xp, x, perm.p, n, s);
  if (L.nu) gather_dev(xs, xp, L.gidx.p, L.nu, s);
  inner->apply_with_scratch(xs, ys, scratch + o, nsm);
  dd_combine(L, ys, yp, s);
  if (n) scatter_dev(y, yp, perm.p, n, s);
}

}  // namespace vb
