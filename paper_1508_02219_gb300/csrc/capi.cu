// The C ABI of the library (include/vbarms.h): handles, the multilevel
// factorization driver (Steps 2-4 per level, Eq. 7-8, last-level ILUT) and
// the FGMRES outer loop.
#include <chrono>
#include <cmath>
#include <memory>

#include "prec.cuh"
#include "vbsr_ops.cuh"

using namespace vb;

struct vbarms_vbsr_st {
  cudaStream_t s = nullptr;
  int dev = 0;  // the device current when the handle was created
  Compressed C;
  DBuf<int> status;
  DBuf<int64_t> rowblk;  // scalar row -> block row, for the SpMV
};

namespace {

thread_local std::string g_err;

vb_status set_err(vb_status st, const std::string& m) {
  g_err = m;
  return st;
}

template <typename F>
vb_status guarded(F&& f) {
  try {
    f();
    g_err.clear();
    return VB_OK;
  } catch (const Error& e) {
    return set_err(e.st, e.msg);
  } catch (const std::bad_alloc&) {
    return set_err(VB_ENOMEM, "host allocation failed");
  } catch (const std::exception& e) {
    return set_err(VB_EINTERNAL, e.what());
  }
}

struct PhaseTimer {
  cudaStream_t s;
  std::vector<std::pair<int, cudaEvent_t>> marks;
  explicit PhaseTimer(cudaStream_t st) : s(st) {}
  void mark(int phase_ending) {
    cudaEvent_t e;
    VB_CUDA(cudaEventCreate(&e));
    VB_CUDA(cudaEventRecord(e, s));
    marks.push_back({phase_ending, e});
  }
  void accumulate(double* out) {
    VB_CUDA(cudaStreamSynchronize(s));
    for (size_t i = 1; i < marks.size(); ++i) {
      float ms = 0;
      VB_CUDA(cudaEventElapsedTime(&ms, marks[i - 1].second, marks[i].second));
      if (marks[i].first >= 0) out[marks[i].first] += ms * 1e-3;
    }
  }
  ~PhaseTimer() {
    for (auto& m : marks) cudaEventDestroy(m.second);
  }
};

// dom (device, may be NULL): for a matrix made of ndom independent diagonal
// blocks, the block of each block row (nondecreasing); it follows the rows
// through the levels so that the last-level ILUT can interleave the blocks.
// fixed (device, may be NULL): one flag per block row; flagged rows never
// enter an independent set, so they reach the last level (Section 5, the
// interface rows of the Schur-complement preconditioner).
template <typename T>
std::unique_ptr<PrecDev<T>> factor_impl(const vbarms_vbsr_st& Ah, const FactorOpts& o, const int32_t* dom = nullptr,
                                        int ndom = 0, const int32_t* fixed = nullptr) {
  auto P = std::make_unique<PrecDev<T>>();
  cudaStream_t s = Ah.s;
  P->s = s;
  P->dev = Ah.dev;
  P->n = Ah.C.n;
  P->precision = o.precision;
  P->wait_limit = o.wait_limit;
  P->status.alloc(1, s);
  P->status.zero();
  int* dst = P->status.p;
  P->perm.alloc(Ah.C.n, s);
  if (Ah.C.n)
    VB_CUDA(cudaMemcpyAsync(P->perm.p, Ah.C.perm.p, Ah.C.n * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
  const bool mixed = o.precision == VB_FP32_MIXED;
  PhaseTimer tm(s);
  tm.mark(-1);
  // current level input: FP64 (the compressed matrix) or T (a Schur complement)
  const VBDev<double>* cur64 = &Ah.C.A;
  VBDev<T> curT;
  bool cur_is64 = true;
  double fill = 0;
  const bool track = dom && ndom > 1 && ndom <= kTicketMaxDom && Ah.C.A.nbr > 0;
  DBuf<int32_t> dcur;
  if (track) {
    dcur.alloc(Ah.C.A.nbr, s);
    VB_CUDA(cudaMemcpyAsync(dcur.p, dom, Ah.C.A.nbr * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
  }
  DBuf<int32_t> fcur;
  if (fixed) {
    fcur.alloc(std::max<int64_t>(Ah.C.A.nbr, 1), s);
    if (Ah.C.A.nbr)
      VB_CUDA(cudaMemcpyAsync(fcur.p, fixed, Ah.C.A.nbr * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
  }
  for (int l = 0; l < o.nlev; ++l) {
    const int64_t p = cur_is64 ? cur64->nbr : curT.nbr;
    if (p == 0) break;
    LevelDev<T> L;
    DBuf<int32_t> newpos;
    DBuf<int64_t> gptr;
    int64_t nD = 0, ngroups = 0;
    if (cur_is64) {
      copy_vb<double, double>(*cur64, L.A64, s);
      scale_level_t<double>(L.A64, L.r, L.c, s);
      tm.mark(PH_SCALE);
      if (o.group_size > 1)
        nD = group_order<double>(L.A64, o.ddtol, o.group_size, fixed ? fcur.p : nullptr, L.w, L.pI, newpos, gptr,
                                 ngroups, s);
      else
        nD = is_order<double>(L.A64, o.ddtol, L.w, L.pI, newpos, s, fixed ? fcur.p : nullptr);
      tm.mark(PH_ORDER);
      if (nD == 0) break;
      if (o.group_size > 1)
        grouped_level<double, T>(L.A64, L.pI, newpos, nD, gptr, ngroups, o.droptol, o.lfil, L, s, dst);
      else
        gather_parts<double, T>(L.A64, L.pI, newpos, nD, L, s, dst);
    } else {
      copy_vb<T, T>(curT, L.AT, s);
      scale_level_t<T>(L.AT, L.r, L.c, s);
      tm.mark(PH_SCALE);
      if (o.group_size > 1)
        nD = group_order<T>(L.AT, o.ddtol, o.group_size, fixed ? fcur.p : nullptr, L.w, L.pI, newpos, gptr, ngroups,
                            s);
      else
        nD = is_order<T>(L.AT, o.ddtol, L.w, L.pI, newpos, s, fixed ? fcur.p : nullptr);
      tm.mark(PH_ORDER);
      if (nD == 0) break;
      if (o.group_size > 1)
        grouped_level<T, T>(L.AT, L.pI, newpos, nD, gptr, ngroups, o.droptol, o.lfil, L, s, dst);
      else
        gather_parts<T, T>(L.AT, L.pI, newpos, nD, L, s, dst);
    }
    tm.mark(PH_GATHER);
    if (track) {  // the next level's rows are the C rows, in P_I order
      DBuf<int32_t> dn(std::max<int64_t>(p - nD, 1), s);
      take_i32(dcur.p, L.pI.p + nD, p - nD, dn.p, s);
      dcur = std::move(dn);
    }
    if (fixed) {
      DBuf<int32_t> fn(std::max<int64_t>(p - nD, 1), s);
      take_i32(fcur.p, L.pI.p + nD, p - nD, fn.p, s);
      fcur = std::move(fn);
    }
    if (!L.grouped) {  // grouped levels made D, W and G in their two sweeps
      pivot_lu(L.D, L.piv, L.ptag, L.D32, mixed, o.fp64_pivot_cond, s, dst, &L.tiles);
      tm.mark(PH_PIVOT);
      w_or_g<T>(L.F, 0, L.D, L.D32, L.piv, L.ptag, mixed, o.droptol, o.lfil, L.W, s);
      tm.mark(PH_W);
      w_or_g<T>(L.E, 1, L.D, L.D32, L.piv, L.ptag, mixed, o.droptol, o.lfil, L.G, s);
      tm.mark(PH_G);
    }
    KernelRec rec;
    rec.kernel = 0;
    rec.level = l;
    schur<T>(L.C, L.G, L.W, l == o.nlev - 1 || o.schur_drop_all, o.droptol, L.S, s, dst, &rec);
    P->krec.push_back(rec);
    tm.mark(PH_SCHUR);
    fill += (double)(L.D.nval + L.W.nval + L.G.nval + L.Lg.nval + L.Ug.nval);
    LevelMaps M;
    if (cur_is64)
      build_level_maps<T>(L, L.A64.rsz.p, L.A64.roff.p, L.A64.nbr, M, s);
    else
      build_level_maps<T>(L, L.AT.rsz.p, L.AT.roff.p, L.AT.nbr, M, s);
    // the next level starts from S; F, E, C are no longer needed by the solve
    if (o.keep_factors) {
      copy_vb<T, T>(L.S, curT, s);
    } else {
      // released once consumed: the scaled level matrix, F, E, C; S moves on
      curT = std::move(L.S);
      L.A64 = VBDev<double>();
      L.AT = VBDev<T>();
      L.F = VBDev<T>();
      L.E = VBDev<T>();
      L.C = VBDev<T>();
    }
    cur_is64 = false;
    P->maps.push_back(std::move(M));
    P->lev.push_back(std::move(L));
    tm.mark(-1);
  }
  // last level: scale, then block ILUT
  LastDev<T>& X = P->last;
  if (cur_is64)
    copy_vb<T, double>(*cur64, X.A, s);
  else
    X.A = std::move(curT);
  scale_level_t<T>(X.A, X.r, X.c, s);
  DBuf<int32_t> tickets;
  if (track) ticket_order(dcur.p, X.A.nbr, ndom, tickets, s);
  ilut_last<T>(X, o.droptol, o.lfil, mixed, o.fp64_pivot_cond, o.wait_limit, s, dst, tickets.p);
  if (fixed) X.fixed = std::move(fcur);
  tm.mark(PH_ILUT);
  level_orders<T>(X, o.wait_limit, dst, s);
  fill += (double)(X.Dg.nval + X.L.nval + X.U.nval);
  tm.accumulate(P->phase_s);
  for (auto& r : P->krec) {
    float ms = 0;
    if (r.e0 && r.e1) {
      VB_CUDA(cudaEventElapsedTime(&ms, r.e0, r.e1));
      r.ms = ms;
    }
  }
  P->mem_ratio = Ah.C.nnz ? fill / (double)Ah.C.nnz : 0.0;
  return P;
}

// Step 1 with either grouping: angle-based (compress_device) or graph-based
// (graph_compress_device); host arrays are copied to the device first.
template <typename F>
vb_status compress_entry(const char* who, int64_t n, const int64_t* rowptr, const int32_t* colind, const double* val,
                         int on_device, void* stream, vbarms_vbsr* out, F&& group) {
  if (!out) return set_err(VB_EINVAL, std::string(who) + ": out is NULL");
  if (n > 0 && !rowptr) return set_err(VB_EINVAL, "rowptr is NULL");
  if (n > 0 && !on_device && rowptr[n] > 0 && (!colind || !val)) return set_err(VB_EINVAL, "colind/val NULL");
  if (n > 0 && on_device && (!colind || !val)) return set_err(VB_EINVAL, "colind/val NULL");
  if (n >= (int64_t)1 << 31) return set_err(VB_EINVAL, "n must fit in int32");
  auto h = std::make_unique<vbarms_vbsr_st>();
  vb_status st = guarded([&] {
    cudaStream_t s = (cudaStream_t)stream;
    h->s = s;
    h->dev = current_device();
    h->status.alloc(1, s);
    h->status.zero();
    const int64_t* d_rowptr = rowptr;
    const int32_t* d_colind = colind;
    const double* d_val = val;
    DBuf<int64_t> rp;
    DBuf<int32_t> ci;
    DBuf<double> vv;
    int64_t nnz = 0;
    if (!on_device) {
      nnz = n ? rowptr[n] : 0;
      if (n && rowptr[0] != 0) fail(VB_EINVAL, "rowptr[0] != 0");
      if (nnz < 0) fail(VB_EINVAL, "negative nnz");
      rp.alloc(n + 1, s);
      ci.alloc(nnz, s);
      vv.alloc(nnz, s);
      h2d(rp.p, rowptr, n + 1, s);
      h2d(ci.p, colind, nnz, s);
      h2d(vv.p, val, nnz, s);
      d_rowptr = rp.p;
      d_colind = ci.p;
      d_val = vv.p;
    } else if (n == 0) {
      rp.alloc(1, s);
      rp.zero();
      d_rowptr = rp.p;
    }
    group(n, d_rowptr, d_colind, d_val, s, h->status.p, h->C);
    VB_CUDA(cudaStreamSynchronize(s));
  });
  if (st != VB_OK) return st;
  *out = h.release();
  return VB_OK;
}

}  // namespace

void vb::set_last_error(const std::string& msg) { g_err = msg; }

// ============================================================================
extern "C" {

void vbarms_opts_default(vbarms_opts* opt) {
  if (!opt) return;
  opt->precision = VB_FP64;
  opt->fp64_pivot_cond = 1e4;
  opt->ddtol = 0.0;
  opt->wait_limit = 0;
  opt->schur_drop_all = 0;
  opt->keep_factors = 1;
  opt->group_size = 1;
}

const char* vbarms_last_error(void) { return g_err.c_str(); }

vb_status vbarms_compress(int64_t n, const int64_t* rowptr, const int32_t* colind, const double* val, int on_device,
                          double tau, void* stream, vbarms_vbsr* out) {
  if (n < 0 || !(tau > 0.0 && tau <= 1.0)) return set_err(VB_EINVAL, "n < 0 or tau outside (0, 1]");
  return compress_entry("vbarms_compress", n, rowptr, colind, val, on_device, stream, out,
                        [&](int64_t nn, const int64_t* r, const int32_t* c, const double* v, cudaStream_t s, int* dst,
                            Compressed& C) { compress_device(nn, r, c, v, tau, s, dst, C); });
}

vb_status vbarms_compress_two_pass(int64_t n, const int64_t* rowptr, const int32_t* colind, const double* val,
                                   int on_device, double tau, void* stream, vbarms_vbsr* out) {
  if (n < 0 || !(tau > 0.0 && tau <= 1.0)) return set_err(VB_EINVAL, "n < 0 or tau outside (0, 1]");
  return compress_entry("vbarms_compress_two_pass", n, rowptr, colind, val, on_device, stream, out,
                        [&](int64_t nn, const int64_t* r, const int32_t* c, const double* v, cudaStream_t s, int* dst,
                            Compressed& C) { two_pass_compress_device(nn, r, c, v, tau, s, dst, C); });
}

vb_status vbarms_compress_graph(int64_t n, const int64_t* rowptr, const int32_t* colind, const double* val,
                                int on_device, double mu, void* stream, vbarms_vbsr* out) {
  if (n < 0 || !(mu >= 0.0)) return set_err(VB_EINVAL, "n < 0 or mu < 0");
  return compress_entry("vbarms_compress_graph", n, rowptr, colind, val, on_device, stream, out,
                        [&](int64_t nn, const int64_t* r, const int32_t* c, const double* v, cudaStream_t s, int* dst,
                            Compressed& C) { graph_compress_device(nn, r, c, v, mu, s, dst, C); });
}

vb_status vbarms_vbsr_from_blocks(int64_t nblk, const int32_t* bsz, const int64_t* bptr, const int32_t* bcol,
                                  const int64_t* voff, const double* val, void* stream, vbarms_vbsr* out) {
  if (!out || nblk < 0) return set_err(VB_EINVAL, "invalid arguments");
  auto h = std::make_unique<vbarms_vbsr_st>();
  vb_status st = guarded([&] {
    cudaStream_t s = (cudaStream_t)stream;
    h->s = s;
    h->dev = current_device();
    h->status.alloc(1, s);
    h->status.zero();
    int64_t n = 0;
    for (int64_t I = 0; I < nblk; ++I) {
      if (bsz[I] <= 0) fail(VB_EINVAL, "block sizes must be positive");
      n += bsz[I];
    }
    const int64_t nnzb = bptr[nblk];
    for (int64_t I = 0; I < nblk; ++I) {
      if (bptr[I + 1] < bptr[I]) fail(VB_EINVAL, "bptr not monotone");
      for (int64_t b = bptr[I]; b < bptr[I + 1]; ++b) {
        if (bcol[b] < 0 || bcol[b] >= nblk || (b > bptr[I] && bcol[b] <= bcol[b - 1]))
          fail(VB_EINVAL, "block columns out of range or not ascending");
        if (voff[b + 1] - voff[b] != (int64_t)bsz[I] * bsz[bcol[b]]) fail(VB_EINVAL, "voff inconsistent");
      }
    }
    Compressed& C = h->C;
    C.n = n;
    C.perm.alloc(n, s);
    std::vector<int32_t> id(n);
    for (int64_t i = 0; i < n; ++i) id[i] = (int32_t)i;
    h2d(C.perm.p, id.data(), n, s);
    DBuf<int32_t> dsz(nblk, s);
    h2d(dsz.p, bsz, nblk, s);
    set_partitions(C.A, dsz.p, nblk, dsz.p, nblk, s);
    C.A.nnzb = nnzb;
    C.A.nval = voff[nnzb];
    C.A.bptr.alloc(nblk + 1, s);
    C.A.bcol.alloc(nnzb, s);
    C.A.voff.alloc(nnzb + 1, s);
    C.A.val.alloc(C.A.nval, s);
    h2d(C.A.bptr.p, bptr, nblk + 1, s);
    h2d(C.A.bcol.p, bcol, nnzb, s);
    h2d(C.A.voff.p, voff, nnzb + 1, s);
    h2d(C.A.val.p, val, C.A.nval, s);
    int64_t nz = 0;
    for (int64_t e = 0; e < C.A.nval; ++e) nz += val[e] != 0.0;
    C.nnz = nz;
    C.av_bd = C.A.nval ? (double)nz / (double)C.A.nval : 0;
    C.av_bs = nblk ? (double)n / (double)nblk : 0;
    VB_CUDA(cudaStreamSynchronize(s));
  });
  if (st != VB_OK) return st;
  *out = h.release();
  return VB_OK;
}

vb_status vbarms_vbsr_query(vbarms_vbsr A, int64_t* n, int64_t* nblk, int64_t* nnzb, int64_t* nval, double* av_bd,
                            double* av_bs) {
  if (!A) return set_err(VB_EINVAL, "NULL handle");
  if (n) *n = A->C.n;
  if (nblk) *nblk = A->C.A.nbr;
  if (nnzb) *nnzb = A->C.A.nnzb;
  if (nval) *nval = A->C.A.nval;
  if (av_bd) *av_bd = A->C.av_bd;
  if (av_bs) *av_bs = A->C.av_bs;
  return VB_OK;
}

vb_status vbarms_vbsr_export(vbarms_vbsr A, int32_t* perm, int32_t* bsz, int64_t* bptr, int32_t* bcol,
                             int64_t* voff, double* val) {
  if (!A) return set_err(VB_EINVAL, "NULL handle");
  return guarded([&] {
    DeviceScope ds(A->dev);
    cudaStream_t s = A->s;
    if (perm && A->C.n) VB_CUDA(cudaMemcpyAsync(perm, A->C.perm.p, A->C.n * 4, cudaMemcpyDeviceToHost, s));
    export_vb(A->C.A, s, nullptr, nullptr, nullptr, nullptr, bsz, nullptr, bptr, bcol, voff, val);
  });
}

vb_status vbarms_factor(vbarms_vbsr A, int nlev, double droptol, int lfil, const vbarms_opts* opt,
                        vbarms_prec* out) {
  if (!A || !out) return set_err(VB_EINVAL, "NULL handle");
  if (nlev < 0 || !(droptol >= 0.0)) return set_err(VB_EINVAL, "nlev < 0 or droptol < 0");
  vbarms_opts d;
  vbarms_opts_default(&d);
  if (!opt) opt = &d;
  if (opt->precision != VB_FP64 && opt->precision != VB_FP32_MIXED) return set_err(VB_EINVAL, "precision");
  if (opt->group_size < 1 || opt->group_size > 64) return set_err(VB_EINVAL, "group_size must lie in [1, 64]");
  FactorOpts o{nlev, droptol, lfil, opt->precision, opt->fp64_pivot_cond, opt->ddtol,
               opt->wait_limit ? opt->wait_limit : (uint64_t)kDefaultWaitNs, opt->schur_drop_all != 0,
               opt->keep_factors != 0, opt->group_size};
  auto h = std::make_unique<vbarms_prec_st>();
  vb_status st = guarded([&] {
    DeviceScope ds(A->dev);
    if (o.precision == VB_FP64)
      h->impl = factor_impl<double>(*A, o);
    else
      h->impl = factor_impl<float>(*A, o);
  });
  if (st != VB_OK) {
    cudaStreamSynchronize(A->s);
    return st;
  }
  *out = h.release();
  return VB_OK;
}

vb_status vbarms_factor_batched(int nmat, const vbarms_vbsr* A, const int* nlev, const double* droptol,
                                const int* lfil, const vbarms_opts* opt, vbarms_prec* out) {
  if (nmat < 0 || (nmat > 0 && (!A || !nlev || !droptol || !lfil || !out)))
    return set_err(VB_EINVAL, "NULL argument or nmat < 0");
  for (int m = 0; m < nmat; ++m) {
    if (!A[m]) return set_err(VB_EINVAL, "NULL matrix handle");
    if (nlev[m] < 0 || !(droptol[m] >= 0.0)) return set_err(VB_EINVAL, "nlev < 0 or droptol < 0");
    if (A[m]->dev != A[0]->dev) return set_err(VB_EINVAL, "the matrices of a batch live on different devices");
  }
  vbarms_opts d;
  vbarms_opts_default(&d);
  if (!opt) opt = &d;
  if (opt->precision != VB_FP64 && opt->precision != VB_FP32_MIXED) return set_err(VB_EINVAL, "precision");
  if (opt->group_size < 1 || opt->group_size > 64) return set_err(VB_EINVAL, "group_size must lie in [1, 64]");
  std::vector<std::unique_ptr<vbarms_prec_st>> res(nmat);
  vb_status st = guarded([&] {
    // matrices with the same (nlev, droptol, lfil) form one batch: one
    // factorization of their block-diagonal union
    std::vector<char> taken(nmat, 0);
    for (int m0 = 0; m0 < nmat; ++m0) {
      if (taken[m0]) continue;
      std::vector<int> members;
      for (int m = m0; m < nmat; ++m)
        if (!taken[m] && nlev[m] == nlev[m0] && droptol[m] == droptol[m0] && lfil[m] == lfil[m0]) {
          members.push_back(m);
          taken[m] = 1;
        }
      DeviceScope ds(A[members[0]]->dev);
      cudaStream_t s = A[members[0]]->s;
      for (int m : members)
        if (A[m]->s != s) VB_CUDA(cudaStreamSynchronize(A[m]->s));
      vbarms_vbsr_st U;
      U.s = s;
      U.dev = A[members[0]]->dev;
      std::vector<const Compressed*> parts;
      for (int m : members) parts.push_back(&A[m]->C);
      compressed_union(parts, s, U.C);
      DBuf<int32_t> dom;
      union_part_ids(parts, s, dom);
      FactorOpts o{nlev[m0], droptol[m0], lfil[m0], opt->precision, opt->fp64_pivot_cond, opt->ddtol,
                   opt->wait_limit ? opt->wait_limit : (uint64_t)kDefaultWaitNs, opt->schur_drop_all != 0,
               opt->keep_factors != 0, opt->group_size};
      std::shared_ptr<PrecBase> P;
      if (o.precision == VB_FP64)
        P = factor_impl<double>(U, o, dom.p, (int)parts.size());
      else
        P = factor_impl<float>(U, o, dom.p, (int)parts.size());
      int64_t off = 0;
      for (int m : members) {
        res[m] = std::make_unique<vbarms_prec_st>();
        res[m]->impl = P;
        res[m]->off = off;
        res[m]->len = A[m]->C.n;
        off += A[m]->C.n;
      }
      VB_CUDA(cudaStreamSynchronize(s));
    }
  });
  if (st != VB_OK) return st;
  for (int m = 0; m < nmat; ++m) out[m] = res[m].release();
  return VB_OK;
}

vb_status vbarms_dd_factor(vbarms_vbsr A, int nparts, int overlap, int restricted, int nlev, double droptol, int lfil,
                           const vbarms_opts* opt, vbarms_prec* out) {
  if (!A || !out) return set_err(VB_EINVAL, "NULL handle");
  if (nlev < 0 || !(droptol >= 0.0)) return set_err(VB_EINVAL, "nlev < 0 or droptol < 0");
  if (nparts < 1 || nparts > kDDMaxParts || overlap < 0)
    return set_err(VB_EINVAL, "nparts must lie in [1, 4096] and overlap must be >= 0");
  vbarms_opts d;
  vbarms_opts_default(&d);
  if (!opt) opt = &d;
  if (opt->precision != VB_FP64 && opt->precision != VB_FP32_MIXED) return set_err(VB_EINVAL, "precision");
  if (opt->group_size < 1 || opt->group_size > 64) return set_err(VB_EINVAL, "group_size must lie in [1, 64]");
  FactorOpts o{nlev, droptol, lfil, opt->precision, opt->fp64_pivot_cond, opt->ddtol,
               opt->wait_limit ? opt->wait_limit : (uint64_t)kDefaultWaitNs, opt->schur_drop_all != 0,
               opt->keep_factors != 0, opt->group_size};
  auto h = std::make_unique<vbarms_prec_st>();
  vb_status st = guarded([&] {
    DeviceScope ds(A->dev);
    cudaStream_t s = A->s;
    auto D = std::make_unique<PrecDD>();
    D->s = s;
    D->dev = A->dev;
    D->n = A->C.n;
    D->precision = o.precision;
    D->wait_limit = o.wait_limit;
    D->perm.alloc(std::max<int64_t>(A->C.n, 1), s);
    if (A->C.n)
      VB_CUDA(cudaMemcpyAsync(D->perm.p, A->C.perm.p, A->C.n * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
    D->status.alloc(1, s);
    D->status.zero();
    // the subdomains' block-diagonal union, factored once; its rows carry
    // their subdomain so that the last-level ILUT interleaves the subdomains
    vbarms_vbsr_st U;
    U.s = s;
    U.dev = A->dev;
    dd_build(A->C, nparts, overlap, restricted != 0, s, D->L, U.C);
    if (o.precision == VB_FP64)
      D->inner = factor_impl<double>(U, o, D->L.ud.p, nparts);
    else
      D->inner = factor_impl<float>(U, o, D->L.ud.p, nparts);
    for (int i = 0; i < PH_COUNT; ++i) D->phase_s[i] = D->inner->phase_s[i];
    D->mem_ratio = D->inner->mem_ratio;
    D->krec = std::move(D->inner->krec);
    D->inner->krec.clear();
    h->impl = std::move(D);
  });
  if (st != VB_OK) {
    cudaStreamSynchronize(A->s);
    return st;
  }
  *out = h.release();
  return VB_OK;
}

vb_status vbarms_dd_schur_factor(vbarms_vbsr A, int nparts, int msteps, int nlev, double droptol, int lfil,
                                 const vbarms_opts* opt, vbarms_prec* out) {
  if (!A || !out) return set_err(VB_EINVAL, "NULL handle");
  if (nlev < 0 || !(droptol >= 0.0)) return set_err(VB_EINVAL, "nlev < 0 or droptol < 0");
  if (nparts < 1 || nparts > kDDMaxParts) return set_err(VB_EINVAL, "nparts must lie in [1, 4096]");
  if (msteps < 1 || msteps > 1000) return set_err(VB_EINVAL, "msteps must lie in [1, 1000]");
  vbarms_opts d;
  vbarms_opts_default(&d);
  if (!opt) opt = &d;
  if (opt->precision != VB_FP64 && opt->precision != VB_FP32_MIXED) return set_err(VB_EINVAL, "precision");
  if (opt->group_size < 1 || opt->group_size > 64) return set_err(VB_EINVAL, "group_size must lie in [1, 64]");
  FactorOpts o{nlev, droptol, lfil, opt->precision, opt->fp64_pivot_cond, opt->ddtol,
               opt->wait_limit ? opt->wait_limit : (uint64_t)kDefaultWaitNs, opt->schur_drop_all != 0,
               opt->keep_factors != 0, opt->group_size};
  auto h = std::make_unique<vbarms_prec_st>();
  vb_status st = guarded([&] {
    DeviceScope ds(A->dev);
    cudaStream_t s = A->s;
    auto D = std::make_unique<PrecDDS>();
    D->s = s;
    D->dev = A->dev;
    D->n = A->C.n;
    D->precision = o.precision;
    D->wait_limit = o.wait_limit;
    D->perm.alloc(std::max<int64_t>(A->C.n, 1), s);
    if (A->C.n)
      VB_CUDA(cudaMemcpyAsync(D->perm.p, A->C.perm.p, A->C.n * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
    D->status.alloc(1, s);
    D->status.zero();
    // the union of the A_i, interface rows last in each, factored once with
    // the interface rows fixed; its rows carry their subdomain so that the
    // last-level ILUT interleaves the subdomains
    vbarms_vbsr_st U;
    U.s = s;
    U.dev = A->dev;
    dds_build(A->C, nparts, msteps, s, D->L, U.C);
    if (o.precision == VB_FP64)
      D->inner = factor_impl<double>(U, o, D->L.ud.p, nparts, D->L.ufix.p);
    else
      D->inner = factor_impl<float>(U, o, D->L.ud.p, nparts, D->L.ufix.p);
    for (int i = 0; i < PH_COUNT; ++i) D->phase_s[i] = D->inner->phase_s[i];
    D->mem_ratio = D->inner->mem_ratio;
    D->krec = std::move(D->inner->krec);
    D->inner->krec.clear();
    h->impl = std::move(D);
  });
  if (st != VB_OK) {
    cudaStreamSynchronize(A->s);
    return st;
  }
  *out = h.release();
  return VB_OK;
}

vb_status vbarms_dd_schur_layout(vbarms_prec M, int* nparts, int* msteps, int64_t* ng, int64_t* ngb, int32_t* part,
                                 int32_t* iface, int32_t* rows, int64_t* nint) {
  if (!M) return set_err(VB_EINVAL, "NULL handle");
  auto* D = dynamic_cast<PrecDDS*>(M->impl.get());
  if (!D) return set_err(VB_EINVAL, "not a Schur-complement preconditioner");
  return guarded([&] {
    DeviceScope ds(D->dev);
    const DDSLayout& L = D->L;
    if (nparts) *nparts = L.nparts;
    if (msteps) *msteps = L.msteps;
    if (ng) *ng = L.ng;
    if (ngb) *ngb = L.ngb;
    if (part && L.p) VB_CUDA(cudaMemcpyAsync(part, L.part.p, L.p * sizeof(int32_t), cudaMemcpyDeviceToHost, D->s));
    if (iface && L.p)
      VB_CUDA(cudaMemcpyAsync(iface, L.iface.p, L.p * sizeof(int32_t), cudaMemcpyDeviceToHost, D->s));
    if (rows && L.p) VB_CUDA(cudaMemcpyAsync(rows, L.ug.p, L.p * sizeof(int32_t), cudaMemcpyDeviceToHost, D->s));
    if (nint) VB_CUDA(cudaMemcpyAsync(nint, L.nint.p, L.nparts * sizeof(int64_t), cudaMemcpyDeviceToHost, D->s));
    VB_CUDA(cudaStreamSynchronize(D->s));
  });
}

vb_status vbarms_dd_layout(vbarms_prec M, int* nparts, int* overlap, int* restricted, int64_t* union_blocks,
                           int32_t* part, int64_t* dstart, int32_t* rows) {
  if (!M) return set_err(VB_EINVAL, "NULL handle");
  auto* D = dynamic_cast<PrecDD*>(M->impl.get());
  if (!D) return set_err(VB_EINVAL, "not a domain-decomposition preconditioner");
  return guarded([&] {
    DeviceScope ds(D->dev);
    const DDLayout& L = D->L;
    if (nparts) *nparts = L.nparts;
    if (overlap) *overlap = L.overlap;
    if (restricted) *restricted = L.restricted ? 1 : 0;
    if (union_blocks) *union_blocks = L.m;
    if (part && L.p) VB_CUDA(cudaMemcpyAsync(part, L.part.p, L.p * sizeof(int32_t), cudaMemcpyDeviceToHost, D->s));
    if (dstart)
      VB_CUDA(cudaMemcpyAsync(dstart, L.dstart.p, (L.nparts + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost, D->s));
    if (rows && L.m) VB_CUDA(cudaMemcpyAsync(rows, L.ug.p, L.m * sizeof(int32_t), cudaMemcpyDeviceToHost, D->s));
    VB_CUDA(cudaStreamSynchronize(D->s));
  });
}

vb_status vbarms_apply(vbarms_prec M, const double* x, double* y) {
  if (!M || !x || !y) return set_err(VB_EINVAL, "NULL argument");
  if (x == y) return set_err(VB_EINVAL, "x and y must not alias");
  return guarded([&] {
    PrecBase& P = *M->impl;
    DeviceScope ds(P.dev);
    DBuf<double> xp(P.n, P.s), yp(P.n, P.s);
    if (M->len < 0) {
      gather_dev(xp.p, x, P.perm.p, P.n, P.s);
      P.apply_perm(xp.p, yp.p);
      scatter_dev(y, yp.p, P.perm.p, P.n, P.s);
    } else {
      // one matrix of a batch: the batch's preconditioner is block diagonal,
      // so it acts on x placed in the matrix's rows and zero elsewhere
      DBuf<double> xu(P.n, P.s), yu(P.n, P.s);
      xu.zero();
      if (M->len)
        VB_CUDA(cudaMemcpyAsync(xu.p + M->off, x, M->len * sizeof(double), cudaMemcpyDeviceToDevice, P.s));
      gather_dev(xp.p, xu.p, P.perm.p, P.n, P.s);
      P.apply_perm(xp.p, yp.p);
      scatter_dev(yu.p, yp.p, P.perm.p, P.n, P.s);
      if (M->len)
        VB_CUDA(cudaMemcpyAsync(y, yu.p + M->off, M->len * sizeof(double), cudaMemcpyDeviceToDevice, P.s));
    }
    check_status(P.status_dev(), P.s, "vbarms_apply");
  });
}

vb_status vbarms_apply_batched(int nmat, const vbarms_prec* M, const double* const* x, double* const* y) {
  if (nmat < 0 || (nmat > 0 && (!M || !x || !y))) return set_err(VB_EINVAL, "NULL argument or nmat < 0");
  for (int m = 0; m < nmat; ++m) {
    if (!M[m] || !x[m] || !y[m]) return set_err(VB_EINVAL, "NULL handle or vector");
    if (x[m] == y[m]) return set_err(VB_EINVAL, "x and y must not alias");
  }
  return guarded([&] {
    // one application per shared factorization: every matrix's x goes to its
    // rows of the batch vector
    std::vector<char> done(nmat, 0);
    for (int m0 = 0; m0 < nmat; ++m0) {
      if (done[m0]) continue;
      PrecBase& P = *M[m0]->impl;
      DeviceScope ds(P.dev);
      DBuf<double> xu(P.n, P.s), yu(P.n, P.s), xp(P.n, P.s), yp(P.n, P.s);
      xu.zero();
      for (int m = m0; m < nmat; ++m) {
        if (done[m] || M[m]->impl.get() != &P) continue;
        const int64_t off = M[m]->len < 0 ? 0 : M[m]->off, len = M[m]->size();
        if (len) VB_CUDA(cudaMemcpyAsync(xu.p + off, x[m], len * sizeof(double), cudaMemcpyDeviceToDevice, P.s));
      }
      gather_dev(xp.p, xu.p, P.perm.p, P.n, P.s);
      P.apply_perm(xp.p, yp.p);
      scatter_dev(yu.p, yp.p, P.perm.p, P.n, P.s);
      for (int m = m0; m < nmat; ++m) {
        if (done[m] || M[m]->impl.get() != &P) continue;
        const int64_t off = M[m]->len < 0 ? 0 : M[m]->off, len = M[m]->size();
        if (len) VB_CUDA(cudaMemcpyAsync(y[m], yu.p + off, len * sizeof(double), cudaMemcpyDeviceToDevice, P.s));
        done[m] = 1;
      }
      check_status(P.status_dev(), P.s, "vbarms_apply_batched");
    }
  });
}

vb_status fgmres_solve(vbarms_vbsr A, vbarms_prec M, const double* b, double* x, double rtol, int restart,
                       int maxit, int* iters, double* relres) {
  if (!A || !b || !x) return set_err(VB_EINVAL, "NULL argument");
  if (restart < 1 || maxit < 0 || !(rtol >= 0.0)) return set_err(VB_EINVAL, "restart < 1, maxit < 0 or rtol < 0");
  if (M && M->size() != A->C.n) return set_err(VB_EINVAL, "preconditioner and matrix sizes differ");
  if (M && M->impl->dev != A->dev) return set_err(VB_EINVAL, "preconditioner and matrix live on different devices");
  bool conv = false;
  vb_status st = guarded([&] {
    DeviceScope ds(A->dev);
    cudaStream_t s = A->s;
    const int64_t n = A->C.n;
    const int m = restart;
    const int32_t* perm = A->C.perm.p;
    if (n && !A->rowblk.p) rowblk_map(A->C.A, n, A->rowblk, s);
    DBuf<double> bp(n, s), xp(n, s), r(n, s), w(n, s), V((size_t)(m + 1) * n, s), Z((size_t)m * n, s);
    DBuf<double> hcol(m + 2, s), red(512, s);
    gather_dev(bp.p, b, perm, n, s);
    gather_dev(xp.p, x, perm, n, s);
    dot_dev(bp.p, bp.p, n, hcol.p, red.p, s);
    const double bnorm = std::sqrt(d2h(hcol.p, s));
    int it = 0;
    double rnorm = 0;
    if (bnorm == 0.0) {
      VB_CUDA(cudaMemsetAsync(x, 0, n * sizeof(double), s));
      VB_CUDA(cudaStreamSynchronize(s));
      if (iters) *iters = 0;
      if (relres) *relres = 0.0;
      conv = true;
      return;
    }
    const double target = rtol * bnorm;
    std::vector<double> H((size_t)(m + 1) * m), cs(m), sn(m), gv(m + 1), yv(m);
    // one matrix of a batch: the batch preconditioner acts on v placed in the
    // matrix's rows (its permuted rows are the same contiguous range) and
    // zero elsewhere
    const bool view = M && M->len >= 0;
    DBuf<double> vu, zu;
    if (view) {
      vu.alloc(M->impl->n, s);
      zu.alloc(M->impl->n, s);
      vu.zero();
    }
    for (;;) {
      // true residual r = b - A x
      spmv_vb(A->C.A, A->rowblk.p, n, xp.p, w.p, s);
      sub_dev(r.p, bp.p, w.p, n, s);
      dot_dev(r.p, r.p, n, hcol.p, red.p, s);
      rnorm = std::sqrt(d2h(hcol.p, s));
      if (rnorm <= target || it >= maxit) break;
      VB_CUDA(cudaMemcpyAsync(hcol.p + m + 1, &rnorm, sizeof(double), cudaMemcpyHostToDevice, s));
      scale_dev(V.p, r.p, hcol.p + m + 1, n, s);
      std::fill(gv.begin(), gv.end(), 0.0);
      gv[0] = rnorm;
      int j = 0;
      for (; j < m && it < maxit; ++j) {
        double* vj = V.p + (size_t)j * n;
        double* zj = Z.p + (size_t)j * n;
        // flexible step: z_j = M^{-1} v_j, w = A z_j, modified Gram-Schmidt
        if (view) {
          if (n) VB_CUDA(cudaMemcpyAsync(vu.p + M->off, vj, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
          M->impl->apply_perm(vu.p, zu.p);
          if (n) VB_CUDA(cudaMemcpyAsync(zj, zu.p + M->off, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
        } else if (M)
          M->impl->apply_perm(vj, zj);
        else
          VB_CUDA(cudaMemcpyAsync(zj, vj, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
        spmv_vb(A->C.A, A->rowblk.p, n, zj, w.p, s);
        for (int i = 0; i <= j; ++i) {
          dot_dev(w.p, V.p + (size_t)i * n, n, hcol.p + i, red.p, s);
          axpy_dev(w.p, V.p + (size_t)i * n, hcol.p + i, -1.0, n, s);
        }
        dot_dev(w.p, w.p, n, hcol.p + j + 1, red.p, s);
        std::vector<double> hc = d2h_vec(hcol.p, j + 2, s);
        if (M) check_status(M->impl->status_dev(), s, "fgmres_solve: preconditioner");
        const double hn = std::sqrt(hc[j + 1]);
        for (int i = 0; i <= j; ++i) H[(size_t)i * m + j] = hc[i];
        H[(size_t)(j + 1) * m + j] = hn;
        ++it;
        // Givens rotations of the new Hessenberg column
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
        if (hn == 0.0 || std::fabs(gv[j + 1]) <= target) {
          ++j;
          break;
        }
        VB_CUDA(cudaMemcpyAsync(hcol.p + m + 1, &hn, sizeof(double), cudaMemcpyHostToDevice, s));
        scale_dev(V.p + (size_t)(j + 1) * n, w.p, hcol.p + m + 1, n, s);
      }
      // x <- x + Z y with the triangular solve of the rotated Hessenberg
      for (int i = j - 1; i >= 0; --i) {
        double sacc = gv[i];
        for (int k = i + 1; k < j; ++k) sacc -= H[(size_t)i * m + k] * yv[k];
        yv[i] = H[(size_t)i * m + i] != 0.0 ? sacc / H[(size_t)i * m + i] : 0.0;
      }
      for (int i = 0; i < j; ++i) axpy_host(xp.p, Z.p + (size_t)i * n, yv[i], n, s);
    }
    scatter_dev(x, xp.p, perm, n, s);
    VB_CUDA(cudaStreamSynchronize(s));
    if (iters) *iters = it;
    if (relres) *relres = rnorm / bnorm;
    conv = rnorm <= target;
  });
  if (st != VB_OK) return st;
  return conv ? VB_OK : set_err(VB_ENOCONV, "FGMRES reached maxit");
}

vb_status vbarms_prec_stats(vbarms_prec M, int* levels_used, double* mem_ratio, double* phase_s) {
  if (!M) return set_err(VB_EINVAL, "NULL handle");
  if (levels_used) *levels_used = M->impl->levels();
  if (mem_ratio) *mem_ratio = M->impl->mem_ratio;
  if (phase_s)
    for (int i = 0; i < PH_COUNT; ++i) phase_s[i] = M->impl->phase_s[i];
  return VB_OK;
}

uint64_t vbarms_launch_count(void) { return g_launch_count.load(); }

uint64_t vbarms_alloc_count(void) { return g_alloc_count.load(); }

vb_status vbarms_prec_ilut_chain(vbarms_prec M, int64_t* links) {
  if (!M) return set_err(VB_EINVAL, "NULL handle");
  if (links) *links = M->impl->ilut_info().chain;
  return VB_OK;
}

vb_status vbarms_prec_pivot_tiles(vbarms_prec M, int lev, int* counts, int* modes, int* source) {
  if (!M) return set_err(VB_EINVAL, "NULL handle");
  return guarded([&] {
    const PivotTiles T = M->impl->pivot_tiles(lev);
    for (int c = 0; c < 5; ++c) {
      if (counts) counts[c] = T.count[c];
      if (modes) modes[c] = T.mode[c];
    }
    if (source) *source = T.source;
  });
}

vb_status vbarms_prec_ilut_geometry(vbarms_prec M, int* slots, int* value_bytes, int* warps_per_sm, int* source,
                                    double* tune_s) {
  if (!M) return set_err(VB_EINVAL, "NULL handle");
  const IlutInfo I = M->impl->ilut_info();
  if (slots) *slots = I.slots;
  if (value_bytes) *value_bytes = I.vbytes;
  if (warps_per_sm) *warps_per_sm = I.warps_per_sm;
  if (source) *source = I.source;
  if (tune_s) *tune_s = I.tune_s;
  return VB_OK;
}

vb_status vbarms_prec_kernel_stats(vbarms_prec M, int kernel, int* launches, double* ms, double* bytes,
                                   double* flops) {
  if (!M) return set_err(VB_EINVAL, "NULL handle");
  int n = 0;
  double t = 0, b = 0, f = 0;
  for (const auto& r : M->impl->krec) {
    if (r.kernel != kernel || r.ms < 0) continue;
    ++n;
    t += r.ms;
    b += r.bytes;
    f += r.flops;
  }
  if (launches) *launches = n;
  if (ms) *ms = t;
  if (bytes) *bytes = b;
  if (flops) *flops = f;
  return VB_OK;
}

vb_status vbarms_prec_export(vbarms_prec M, int lev, int which, int64_t* nbr, int64_t* nbc, int64_t* nnzb,
                             int64_t* nval, int32_t* rsz, int32_t* csz, int64_t* bptr, int32_t* bcol,
                             int64_t* voff, double* val) {
  if (!M) return set_err(VB_EINVAL, "NULL handle");
  return guarded([&] {
    DeviceScope ds(M->impl->dev);
    M->impl->export_mat(lev, which, nbr, nbc, nnzb, nval, rsz, csz, bptr, bcol, voff, val);
  });
}

vb_status vbarms_prec_vector(vbarms_prec M, int lev, int which, double* d, int32_t* iv, int64_t* len) {
  if (!M) return set_err(VB_EINVAL, "NULL handle");
  return guarded([&] {
    DeviceScope ds(M->impl->dev);
    M->impl->export_vec(lev, which, d, iv, len);
  });
}

// Destruction runs on the handle's device (its buffers are freed on its
// stream); a failure to select that device still frees the host side.
void vbarms_vbsr_destroy(vbarms_vbsr A) {
  if (!A) return;
  try {
    DeviceScope ds(A->dev);
    cudaStreamSynchronize(A->s);
    delete A;
  } catch (const Error&) {
    delete A;
  }
}

void vbarms_prec_destroy(vbarms_prec M) {
  if (!M) return;
  if (!M->impl) {
    delete M;
    return;
  }
  try {
    DeviceScope ds(M->impl->dev);
    cudaStreamSynchronize(M->impl->s);
    delete M;
  } catch (const Error&) {
    delete M;
  }
}

}  // extern "C"
