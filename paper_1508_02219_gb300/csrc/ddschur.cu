// Section 5 Schur-complement global preconditioner on one GPU (eq. paral,
// eq. gschur, eq. loc_var_schur).
//
// Subdomain i is the contiguous range of compressed block rows with
// part(I) = floor(N * roff_I / n).  A block row is an interface row when a
// stored block of A couples it, as row or as column, to another subdomain;
// the others are interior.  The union of the local matrices A_i lists each
// subdomain's interior rows, then its interface rows (each ascending), so
// A_i = [[B_i, F_i], [E_i, C_i]], and is factored once with the interface
// rows kept out of every independent set: they reach the last level behind
// the remaining interior rows, and the trailing part of its block ILUT is the
// LU of the approximate local Schur complement S_i = C_i - E_i B_i^{-1} F_i.
//
// One application to r = (f_i, g_i):
//   z   = interface part of the union solve of r       (= S_i^{-1} g'_i)
//   y   = msteps steps of GMRES (y_0 = 0, modified Gram-Schmidt, Givens) on
//         (I + S^{-1} E) y = z, E the blocks E_ij between interface rows of
//         different subdomains, S^{-1} v = interface part of the union solve
//         of (0, v): the global system preconditioned by blockdiag(S_i)
//   u_i = interior part of the union solve of r whose last-level backward
//         sweep keeps the interface unknowns at y (B_i^{-1}(f_i - F_i y_i))
// The inner GMRES is driven from the host: its dot products are the
// deterministic two-stage reductions of the outer FGMRES, its small
// Hessenberg problem is solved on the host in FP64.
//
// Subdomain ranges are contiguous and increasing, so the interface rows in
// the union's order are simply the interface rows of A in ascending order:
// that is the interface numbering of E and of the interface vector.
#include <cmath>

#include "prec.cuh"
#include "vbsr_ops.cuh"

namespace vb {
namespace {

__global__ void k_ds_part(int64_t p, int64_t n, int nparts, const int64_t* __restrict__ roff,
                          int32_t* __restrict__ part) {
  for (int64_t I = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; I < p; I += (int64_t)gridDim.x * blockDim.x)
    part[I] = (int32_t)(((int64_t)nparts * roff[I]) / n);
}

// A stored block (I, J) between two subdomains makes I and J interface rows
// (every writer stores 1, so the result does not depend on the order).
__global__ void k_ds_iface(int64_t p, const int64_t* __restrict__ bptr, const int32_t* __restrict__ bcol,
                           const int32_t* __restrict__ part, int32_t* __restrict__ iface) {
  const int lane = threadIdx.x & 31;
  const int64_t wpb = blockDim.x >> 5;
  for (int64_t I = blockIdx.x * wpb + (threadIdx.x >> 5); I < p; I += (int64_t)gridDim.x * wpb) {
    const int32_t pi = part[I];
    bool any = false;
    for (int64_t b = bptr[I] + lane; b < bptr[I + 1]; b += 32) {
      const int32_t J = bcol[b];
      if (part[J] != pi) {
        iface[J] = 1;
        any = true;
      }
    }
    if (__any_sync(0xffffffffu, any) && lane == 0) iface[I] = 1;
  }
}

// First block row of every subdomain (empty subdomains start where the next
// non-empty one does); dstart[nparts] = p.
__global__ void k_ds_dstart(int64_t p, int nparts, const int32_t* __restrict__ part, int64_t* __restrict__ dstart) {
  for (int64_t I = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; I <= p; I += (int64_t)gridDim.x * blockDim.x) {
    const int prev = I == 0 ? -1 : part[I - 1];
    const int cur = I == p ? nparts : part[I];
    for (int q = prev + 1; q <= cur; ++q) dstart[q] = I;
  }
}

// Union position of every block row: its subdomain's start, then the interior
// rows before it, or all the subdomain's interior rows and the interface rows
// before it (sint/sif: exclusive scans of the interior/interface flags).
__global__ void k_ds_upos(int64_t p, const int32_t* __restrict__ part, const int32_t* __restrict__ iface,
                          const int64_t* __restrict__ dstart, const int64_t* __restrict__ sint,
                          const int64_t* __restrict__ sif, int32_t* __restrict__ upos, int32_t* __restrict__ ug,
                          int32_t* __restrict__ ud, int32_t* __restrict__ ufix) {
  for (int64_t I = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; I < p; I += (int64_t)gridDim.x * blockDim.x) {
    const int q = part[I];
    const int64_t s0 = dstart[q], s1 = dstart[q + 1];
    const int64_t k = iface[I] ? s0 + (sint[s1] - sint[s0]) + (sif[I] - sif[s0]) : s0 + (sint[I] - sint[s0]);
    upos[I] = (int32_t)k;
    ug[k] = (int32_t)I;
    ud[k] = q;
    ufix[k] = iface[I];
  }
}

// isint = 1 - iface; gsz = iface ? rsz : 0
__global__ void k_ds_flags(int64_t p, const int32_t* __restrict__ iface, const int32_t* __restrict__ rsz,
                           int32_t* __restrict__ isint, int32_t* __restrict__ gsz) {
  for (int64_t I = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; I < p; I += (int64_t)gridDim.x * blockDim.x) {
    isint[I] = 1 - iface[I];
    gsz[I] = iface[I] ? rsz[I] : 0;
  }
}

__global__ void k_ds_nint(int nparts, const int64_t* __restrict__ dstart, const int64_t* __restrict__ sint,
                          int64_t* __restrict__ nint) {
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nparts; q += gridDim.x * blockDim.x)
    nint[q] = sint[dstart[q + 1]] - sint[dstart[q]];
}

__global__ void k_ds_take_rsz(int64_t m, const int32_t* __restrict__ rows, const int32_t* __restrict__ rsz,
                              int32_t* __restrict__ out) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < m; k += (int64_t)gridDim.x * blockDim.x)
    out[k] = rsz[rows[k]];
}

// Rows of the union (SAME = true: blocks inside the row's subdomain, union
// columns, interior columns first) or of E (SAME = false: blocks to other
// subdomains, interface columns).  Count pass, then columns and source
// blocks; a warp compacts its row in order with ballots.
template <bool SAME, bool FILL>
__global__ void k_ds_rows(int64_t m, const int32_t* __restrict__ rows, const int64_t* __restrict__ bptr,
                          const int32_t* __restrict__ bcol, const int32_t* __restrict__ part,
                          const int32_t* __restrict__ iface, const int32_t* __restrict__ colmap,
                          int32_t* __restrict__ cnt, const int64_t* __restrict__ obptr, int32_t* __restrict__ obcol,
                          int64_t* __restrict__ srcb) {
  const int lane = threadIdx.x & 31;
  const int64_t wpb = blockDim.x >> 5;
  for (int64_t k = blockIdx.x * wpb + (threadIdx.x >> 5); k < m; k += (int64_t)gridDim.x * wpb) {
    const int64_t I = rows[k];
    const int32_t pi = part[I];
    const int64_t b0 = bptr[I], b1 = bptr[I + 1];
    int64_t pos = FILL ? obptr[k] : 0;
    int c = 0;
    for (int pass = 0; pass < (SAME ? 2 : 1); ++pass)
      for (int64_t bb = b0; bb < b1; bb += 32) {
        const int64_t b = bb + lane;
        bool in = false;
        if (b < b1) {
          const int32_t J = bcol[b];
          in = SAME ? (part[J] == pi && iface[J] == pass) : part[J] != pi;
        }
        const unsigned bal = __ballot_sync(0xffffffffu, in);
        if (FILL && in) {
          const int64_t d = pos + __popc(bal & ((1u << lane) - 1u));
          obcol[d] = colmap[bcol[b]];
          srcb[d] = b;
        }
        pos += __popc(bal);
        c += __popc(bal);
      }
    if (!FILL && lane == 0) cnt[k] = c;
  }
}

__global__ void k_ds_values(int64_t m, const int64_t* __restrict__ obptr, const int64_t* __restrict__ ovoff,
                            const int64_t* __restrict__ srcb, const int64_t* __restrict__ avoff,
                            const double* __restrict__ aval, double* __restrict__ oval) {
  const int lane = threadIdx.x & 31;
  const int64_t wpb = blockDim.x >> 5;
  for (int64_t k = blockIdx.x * wpb + (threadIdx.x >> 5); k < m; k += (int64_t)gridDim.x * wpb)
    for (int64_t d = obptr[k]; d < obptr[k + 1]; ++d) {
      const int64_t s0 = avoff[srcb[d]], len = ovoff[d + 1] - ovoff[d];
      for (int64_t e = lane; e < len; e += 32) oval[ovoff[d] + e] = aval[s0 + e];
    }
}

// gidx: union scalar row -> scalar row of A; gpos: interface scalar -> union
// scalar row (gsoff: exclusive scan of the interface rows' sizes over A).
__global__ void k_ds_maps(int64_t p, const int32_t* __restrict__ rsz, const int64_t* __restrict__ roff,
                          const int32_t* __restrict__ upos, const int64_t* __restrict__ uroff,
                          const int32_t* __restrict__ iface, const int64_t* __restrict__ gsoff,
                          int32_t* __restrict__ gidx, int32_t* __restrict__ gpos) {
  for (int64_t I = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; I < p; I += (int64_t)gridDim.x * blockDim.x) {
    const int64_t u0 = uroff[upos[I]];
    for (int a = 0; a < rsz[I]; ++a) {
      gidx[u0 + a] = (int32_t)(roff[I] + a);
      if (iface[I]) gpos[gsoff[I] + a] = (int32_t)(u0 + a);
    }
  }
}

// The interface rows of A in ascending order (their interface numbering).
__global__ void k_ds_iflist(int64_t p, const int32_t* __restrict__ iface, const int64_t* __restrict__ sif,
                            int32_t* __restrict__ ifrows) {
  for (int64_t I = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; I < p; I += (int64_t)gridDim.x * blockDim.x)
    if (iface[I]) ifrows[sif[I]] = (int32_t)I;
}

__global__ void k_ds_i64_to_i32(int64_t n, const int64_t* __restrict__ a, int32_t* __restrict__ b) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = (int32_t)a[i];
}

__global__ void k_ds_iota(int64_t n, int32_t* __restrict__ v) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    v[i] = (int32_t)i;
}

// out = v + t
__global__ void k_ds_add(int64_t n, const double* __restrict__ v, const double* __restrict__ t,
                         double* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = __dadd_rn(v[i], t[i]);
}

__global__ void k_ds_count_nz(int64_t n, const double* __restrict__ v, unsigned long long* __restrict__ out) {
  unsigned long long c = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    c += v[i] != 0.0;
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(out, c);
}

// Rows `rows` of A restricted by SAME into M (partitions already set).
template <bool SAME>
void ds_submatrix(const VBDev<double>& A, const DBuf<int32_t>& rows, int64_t m, const int32_t* part,
                  const int32_t* iface, const int32_t* colmap, VBDev<double>& M, cudaStream_t s) {
  M.bptr.alloc(m + 1, s);
  {
    DBuf<int32_t> rc(std::max<int64_t>(m, 1), s);
    if (m) {
      launch(k_ds_rows<SAME, false>, grid_for(m, 8), 256, 0, s, m, rows.p, A.bptr.p, A.bcol.p, part, iface, colmap,
             rc.p, nullptr, nullptr, nullptr);
      VB_LAUNCH_CHECK();
    }
    scan_i32_to_i64(rc.p, M.bptr.p, m, s);
  }
  M.nnzb = m ? d2h(M.bptr.p + m, s) : 0;
  M.bcol.alloc(std::max<int64_t>(M.nnzb, 1), s);
  DBuf<int64_t> srcb(std::max<int64_t>(M.nnzb, 1), s);
  if (m) {
    launch(k_ds_rows<SAME, true>, grid_for(m, 8), 256, 0, s, m, rows.p, A.bptr.p, A.bcol.p, part, iface, colmap,
           nullptr, M.bptr.p, M.bcol.p, srcb.p);
    VB_LAUNCH_CHECK();
  }
  finish_offsets(M, s);
  if (m && M.nval) {
    launch(k_ds_values, grid_for(m, 8), 256, 0, s, m, M.bptr.p, M.voff.p, srcb.p, A.voff.p, A.val.p, M.val.p);
    VB_LAUNCH_CHECK();
  }
}

inline size_t al256(size_t v) { return (v + 255) & ~(size_t)255; }

// Scratch of one application (each piece 256-byte aligned): five union
// vectors, the Krylov basis (msteps + 1 interface vectors), four interface
// vectors, the Hessenberg column and the reduction scratch, then (static
// path) the permuted x and y and the inner solve's own scratch.
struct DSPlan {
  size_t xu, zu, tu, su, fu, V, w, t, z, yg, hcol, red, xp, yp, inner, total;
};

DSPlan ds_plan(const DDSLayout& L, int64_t n, size_t inner_bytes) {
  DSPlan P{};
  size_t o = 0;
  auto take = [&o](size_t bytes) {
    const size_t at = o;
    o = al256(o + bytes);
    return at;
  };
  const size_t nu = (size_t)L.n * 8, ng = (size_t)L.ng * 8;
  P.xu = take(nu);
  P.zu = take(nu);
  P.tu = take(nu);
  P.su = take(nu);
  P.fu = take(nu);
  P.V = take((size_t)(L.msteps + 1) * ng);
  P.w = take(ng);
  P.t = take(ng);
  P.z = take(ng);
  P.yg = take(ng);
  P.hcol = take((size_t)(L.msteps + 2) * 8);
  P.red = take(512 * 8);
  P.xp = take((size_t)n * 8);
  P.yp = take((size_t)n * 8);
  P.inner = take(inner_bytes);
  P.total = o;
  return P;
}

// One application in the union's own numbering (xu -> ru): solve(x, y, fixv)
// is the union solve (fixv: interface unknowns kept at those values).
template <typename Solve>
void ds_apply_union(const DDSLayout& L, unsigned char* sc, const DSPlan& P, cudaStream_t s, Solve&& solve) {
  const int64_t nu = L.n, ng = L.ng;
  const int m = L.msteps;
  double* xu = (double*)(sc + P.xu);
  double* zu = (double*)(sc + P.zu);
  double* tu = (double*)(sc + P.tu);
  double* su = (double*)(sc + P.su);
  double* fu = (double*)(sc + P.fu);
  double* V = (double*)(sc + P.V);
  double* w = (double*)(sc + P.w);
  double* t = (double*)(sc + P.t);
  double* z = (double*)(sc + P.z);
  double* yg = (double*)(sc + P.yg);
  double* hcol = (double*)(sc + P.hcol);
  double* red = (double*)(sc + P.red);
  // z = S^{-1} g' from the local solves of r
  solve(xu, zu, nullptr);
  if (ng) {
    gather_dev(z, zu, L.gpos.p, ng, s);
    VB_CUDA(cudaMemsetAsync(yg, 0, ng * sizeof(double), s));
    dot_dev(z, z, ng, hcol, red, s);
    const double beta = std::sqrt(d2h(hcol, s));
    if (beta != 0.0) {
      std::vector<double> H((size_t)(m + 1) * m, 0.0), cs(m), sn(m), gv(m + 1, 0.0), yv(m);
      VB_CUDA(cudaMemcpyAsync(hcol + m + 1, &beta, sizeof(double), cudaMemcpyHostToDevice, s));
      scale_dev(V, z, hcol + m + 1, ng, s);
      gv[0] = beta;
      int j = 0;
      for (; j < m; ++j) {
        double* vj = V + (size_t)j * ng;
        // w = v_j + S^{-1} E v_j
        spmv_vb(L.E, L.Erb.p, ng, vj, w, s);
        VB_CUDA(cudaMemsetAsync(tu, 0, nu * sizeof(double), s));
        scatter_dev(tu, w, L.gpos.p, ng, s);
        solve(tu, su, nullptr);
        gather_dev(t, su, L.gpos.p, ng, s);
        launch(k_ds_add, grid_for(ng, 256), 256, 0, s, ng, vj, t, w);
        VB_LAUNCH_CHECK();
        for (int i = 0; i <= j; ++i) {
          dot_dev(w, V + (size_t)i * ng, ng, hcol + i, red, s);
          axpy_dev(w, V + (size_t)i * ng, hcol + i, -1.0, ng, s);
        }
        dot_dev(w, w, ng, hcol + j + 1, red, s);
        const std::vector<double> hc = d2h_vec(hcol, j + 2, s);
        const double hn = std::sqrt(hc[j + 1]);
        for (int i = 0; i <= j; ++i) H[(size_t)i * m + j] = hc[i];
        H[(size_t)(j + 1) * m + j] = hn;
        for (int i = 0; i < j; ++i) {
          const double a = H[(size_t)i * m + j], c = H[(size_t)(i + 1) * m + j];
          H[(size_t)i * m + j] = cs[i] * a + sn[i] * c;
          H[(size_t)(i + 1) * m + j] = -sn[i] * a + cs[i] * c;
        }
        const double a = H[(size_t)j * m + j], c = H[(size_t)(j + 1) * m + j];
        const double d = std::sqrt(a * a + c * c);
        cs[j] = d > 0.0 ? a / d : 1.0;
        sn[j] = d > 0.0 ? c / d : 0.0;
        H[(size_t)j * m + j] = d;
        H[(size_t)(j + 1) * m + j] = 0.0;
        gv[j + 1] = -sn[j] * gv[j];
        gv[j] = cs[j] * gv[j];
        if (hn == 0.0) {
          ++j;
          break;
        }
        VB_CUDA(cudaMemcpyAsync(hcol + m + 1, &hn, sizeof(double), cudaMemcpyHostToDevice, s));
        scale_dev(V + (size_t)(j + 1) * ng, w, hcol + m + 1, ng, s);
      }
      for (int i = j - 1; i >= 0; --i) {
        double sacc = gv[i];
        for (int k = i + 1; k < j; ++k) sacc -= H[(size_t)i * m + k] * yv[k];
        yv[i] = H[(size_t)i * m + i] != 0.0 ? sacc / H[(size_t)i * m + i] : 0.0;
      }
      for (int i = 0; i < j; ++i) axpy_host(yg, V + (size_t)i * ng, yv[i], ng, s);
    }
  }
  // recovery: the union solve of r with the interface unknowns kept at y
  VB_CUDA(cudaMemsetAsync(fu, 0, nu * sizeof(double), s));
  if (ng) scatter_dev(fu, yg, L.gpos.p, ng, s);
  solve(xu, zu, fu);
  if (ng) scatter_dev(zu, yg, L.gpos.p, ng, s);
}

}  // namespace

void dds_build(const Compressed& A, int nparts, int msteps, cudaStream_t s, DDSLayout& L, Compressed& U) {
  const VBDev<double>& M = A.A;
  const int64_t p = M.nbr, n = A.n;
  if (!M.same_partition) fail(VB_EINVAL, "vbarms_dd_schur_factor: the matrix is not square-partitioned");
  L.nparts = nparts;
  L.msteps = msteps;
  L.n = n;
  L.p = p;
  const int64_t p1 = std::max<int64_t>(p, 1);
  L.part.alloc(p1, s);
  L.iface.alloc(p1, s);
  L.iface.zero();
  L.dstart.alloc(nparts + 1, s);
  L.nint.alloc(nparts, s);
  if (p) {
    launch(k_ds_part, grid_for(p, 256), 256, 0, s, p, n, nparts, M.roff.p, L.part.p);
    launch(k_ds_iface, grid_for(p, 8), 256, 0, s, p, M.bptr.p, M.bcol.p, L.part.p, L.iface.p);
    VB_LAUNCH_CHECK();
  }
  launch(k_ds_dstart, grid_for(p + 1, 256), 256, 0, s, p, nparts, L.part.p, L.dstart.p);
  VB_LAUNCH_CHECK();
  // union order: each subdomain's interior rows, then its interface rows
  DBuf<int32_t> isint(p1, s), gsz(p1, s), upos(p1, s);
  DBuf<int64_t> sint(p + 1, s), sif(p + 1, s), gsoff(p + 1, s);
  if (p) {
    launch(k_ds_flags, grid_for(p, 256), 256, 0, s, p, L.iface.p, M.rsz.p, isint.p, gsz.p);
    VB_LAUNCH_CHECK();
  }
  scan_i32_to_i64(isint.p, sint.p, p, s);
  scan_i32_to_i64(L.iface.p, sif.p, p, s);
  scan_i32_to_i64(gsz.p, gsoff.p, p, s);
  L.ngb = p ? (int64_t)d2h(sif.p + p, s) : 0;
  L.ng = p ? (int64_t)d2h(gsoff.p + p, s) : 0;
  L.ug.alloc(p1, s);
  L.ud.alloc(p1, s);
  L.ufix.alloc(p1, s);
  if (p) {
    launch(k_ds_upos, grid_for(p, 256), 256, 0, s, p, L.part.p, L.iface.p, L.dstart.p, sint.p, sif.p, upos.p, L.ug.p,
           L.ud.p, L.ufix.p);
    VB_LAUNCH_CHECK();
  }
  launch(k_ds_nint, grid_for(nparts, 256), 256, 0, s, nparts, L.dstart.p, sint.p, L.nint.p);
  VB_LAUNCH_CHECK();

  // the union matrix: blocks inside a subdomain, union columns
  VBDev<double>& V = U.A;
  {
    DBuf<int32_t> ursz(p1, s);
    if (p) {
      launch(k_ds_take_rsz, grid_for(p, 256), 256, 0, s, p, L.ug.p, M.rsz.p, ursz.p);
      VB_LAUNCH_CHECK();
    }
    set_partitions(V, ursz.p, p, ursz.p, p, s);
  }
  ds_submatrix<true>(M, L.ug, p, L.part.p, L.iface.p, upos.p, V, s);
  U.n = n;
  U.perm.alloc(std::max<int64_t>(n, 1), s);
  if (n) {
    launch(k_ds_iota, grid_for(n, 256), 256, 0, s, n, U.perm.p);
    VB_LAUNCH_CHECK();
  }
  {
    DBuf<unsigned long long> nz(1, s);
    nz.zero();
    if (V.nval) {
      launch(k_ds_count_nz, grid_for(V.nval, 256), 256, 0, s, V.nval, V.val.p, nz.p);
      VB_LAUNCH_CHECK();
    }
    U.nnz = (int64_t)d2h(nz.p, s);
  }
  U.av_bd = U.av_bs = 0.0;

  // maps between the union, A and the interface vector
  L.gidx.alloc(std::max<int64_t>(n, 1), s);
  L.gpos.alloc(std::max<int64_t>(L.ng, 1), s);
  if (p) {
    launch(k_ds_maps, grid_for(p, 256), 256, 0, s, p, M.rsz.p, M.roff.p, upos.p, V.roff.p, L.iface.p, gsoff.p,
           L.gidx.p, L.gpos.p);
    VB_LAUNCH_CHECK();
  }

  // E: blocks between interface rows of different subdomains, on the
  // interface numbering (the interface rows of A in ascending order)
  {
    const int64_t m = L.ngb;
    DBuf<int32_t> ifrows(std::max<int64_t>(m, 1), s), ersz(std::max<int64_t>(m, 1), s), gcol(p1, s);
    if (p) {
      launch(k_ds_iflist, grid_for(p, 256), 256, 0, s, p, L.iface.p, sif.p, ifrows.p);
      launch(k_ds_i64_to_i32, grid_for(p, 256), 256, 0, s, p, sif.p, gcol.p);
      VB_LAUNCH_CHECK();
    }
    if (m) {
      launch(k_ds_take_rsz, grid_for(m, 256), 256, 0, s, m, ifrows.p, M.rsz.p, ersz.p);
      VB_LAUNCH_CHECK();
    }
    set_partitions(L.E, ersz.p, m, ersz.p, m, s);
    ds_submatrix<false>(M, ifrows, m, L.part.p, L.iface.p, gcol.p, L.E, s);
    if (L.ng) rowblk_map(L.E, L.ng, L.Erb, s);
  }
  VB_CUDA(cudaStreamSynchronize(s));
}

size_t PrecDDS::scratch_bytes() const {
  return ds_plan(L, n, inner->scratch_bytes()).total;
}

void PrecDDS::apply_perm(const double* x, double* y) {
  const DSPlan P = ds_plan(L, n, 0);
  if (work.n < P.total) work.alloc(P.total, s);
  unsigned char* sc = work.p;
  if (L.n) gather_dev((double*)(sc + P.xu), x, L.gidx.p, L.n, s);
  ds_apply_union(L, sc, P, s, [this](const double* a, double* b, const double* fixv) {
    inner->apply_fixed(a, b, fixv);
  });
  if (L.n) scatter_dev(y, (double*)(sc + P.zu), L.gidx.p, L.n, s);
}

void PrecDDS::apply_with_scratch(const double* x, double* y, unsigned char* scratch, int nsm) {
  const DSPlan P = ds_plan(L, n, inner->scratch_bytes());
  double* xp = (double*)(scratch + P.xp);
  double* yp = (double*)(scratch + P.yp);
  unsigned char* isc = scratch + P.inner;
  if (n) gather_dev(xp, x, perm.p, n, s);
  if (L.n) gather_dev((double*)(scratch + P.xu), xp, L.gidx.p, L.n, s);
  ds_apply_union(L, scratch, P, s, [this, isc, nsm](const double* a, double* b, const double* fixv) {
    inner->solve_scratch(a, b, isc, nsm, fixv);
  });
  if (L.n) scatter_dev(yp, (double*)(scratch + P.zu), L.gidx.p, L.n, s);
  if (n) scatter_dev(y, yp, perm.p, n, s);
}

}  // namespace vb
