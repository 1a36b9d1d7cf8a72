// The multilevel factorization object and the solve-phase entry points.
#pragma once

#include <memory>

#include "internal.h"
#include "level.cuh"

namespace vb {

enum Phase { PH_SCALE = 0, PH_ORDER, PH_GATHER, PH_PIVOT, PH_W, PH_G, PH_SCHUR, PH_ILUT, PH_COUNT };

// Per level: the scalar permutation of P_I (new scalar position -> old).
struct LevelMaps {
  DBuf<int32_t> sperm;
  DBuf<int64_t> grow, wrow;  // scalar row -> block row of G and W (solve phase)
  int64_t n = 0, nf = 0;
};

struct PrecBase {
  cudaStream_t s = nullptr;
  int dev = 0;  // the device the factorization lives on
  int64_t n = 0;
  int precision = VB_FP64;
  uint64_t wait_limit = 0;
  double phase_s[PH_COUNT] = {0};
  double mem_ratio = 0;
  DBuf<int32_t> perm;  // P_B of the matrix the factorization was built from
  DBuf<int> status;
  std::vector<KernelRec> krec;  // timed launches (Schur numeric per level)
  virtual ~PrecBase() {
    for (auto& r : krec) {
      if (r.e0) cudaEventDestroy(r.e0);
      if (r.e1) cudaEventDestroy(r.e1);
    }
  }
  virtual int levels() const = 0;
  // y = M^{-1} x, both in the block-permuted (P_B) numbering, device FP64.
  // Enqueues work only; read `status` (check_status) after synchronizing.
  virtual void apply_perm(const double* x, double* y) = 0;
  virtual void export_mat(int lev, int which, int64_t* nbr, int64_t* nbc, int64_t* nnzb, int64_t* nval,
                          int32_t* rsz, int32_t* csz, int64_t* bptr, int32_t* bcol, int64_t* voff,
                          double* val) = 0;
  // Bytes of caller-provided scratch that apply_with_scratch needs.
  virtual size_t scratch_bytes() const = 0;
  // y = M^{-1} x (original numbering) using only the given device scratch
  // (256-byte aligned, scratch_bytes() long): allocates nothing.
  virtual void apply_with_scratch(const double* x, double* y, unsigned char* scratch, int nsm) = 0;
  virtual void export_vec(int lev, int which, double* d, int32_t* iv, int64_t* len) = 0;
  // How the last-level ILUT ran.
  virtual IlutInfo ilut_info() const = 0;
  // How level lev's pivot phase ran (size classes and their modes).
  virtual PivotTiles pivot_tiles(int lev) const = 0;
  // The device status word the solve kernels report to.
  virtual int* status_dev() { return status.p; }
  // Factorizations with fixed rows (the Schur-complement preconditioner's
  // local solver): the solve with the fixed rows' unknowns given, in the
  // factorization's own numbering, with its own buffers or with scratch.
  virtual void apply_fixed(const double*, double*, const double*) {
    fail(VB_EINTERNAL, "this factorization has no fixed rows");
  }
  virtual void solve_scratch(const double*, double*, unsigned char*, int, const double*) {
    fail(VB_EINTERNAL, "this factorization has no scratch solve");
  }
};

template <typename T>
struct PrecDev : PrecBase {
  std::vector<LevelDev<T>> lev;
  std::vector<LevelMaps> maps;
  LastDev<T> last;
  // solve-phase scratch, allocated on the first apply
  bool prepared = false;
  int nsm = 0;
  int64_t nlast = 0;
  DBuf<double> work;
  DBuf<int32_t> flags;
  DBuf<unsigned long long> tick;
  DBuf<int> abort_flag;
  DBuf<double> fwork;  // fixed values on the levels (apply_fixed)
  void prepare_apply();
  int levels() const override { return (int)lev.size(); }
  void apply_perm(const double* x, double* y) override;
  // The same with the fixed rows' unknowns given (fixv, this numbering):
  // the last level's backward sweep keeps them instead of solving for them.
  void apply_fixed(const double* x, double* y, const double* fixv) override;
  size_t scratch_bytes() const override;
  void apply_with_scratch(const double* x, double* y, unsigned char* scratch, int nsm) override;
  // Alg. 2 in this numbering (x, y not permuted) with scratch_bytes() of
  // scratch; fixv as in apply_fixed (may be NULL).
  void solve_scratch(const double* x, double* y, unsigned char* scratch, int nsm, const double* fixv) override;
  void export_mat(int lev, int which, int64_t* nbr, int64_t* nbc, int64_t* nnzb, int64_t* nval, int32_t* rsz,
                  int32_t* csz, int64_t* bptr, int32_t* bcol, int64_t* voff, double* val) override;
  void export_vec(int lev, int which, double* d, int32_t* iv, int64_t* len) override;
  IlutInfo ilut_info() const override { return last.info; }
  PivotTiles pivot_tiles(int l) const override {
    if (l < 0 || l >= (int)lev.size()) fail(VB_EINVAL, "level out of range");
    return lev[l].tiles;
  }
};

// Section 5 global preconditioners (dd.cu): the subdomains of A, their
// block-diagonal union and the maps between union and global vectors.
constexpr int kDDMaxParts = 4096;

struct DDLayout {
  int nparts = 0, overlap = 0;
  bool restricted = true;
  int64_t n = 0, p = 0;    // scalar and block rows of A
  int64_t m = 0, nu = 0;   // block and scalar rows of the union
  DBuf<int32_t> part;      // subdomain owning each block row of A
  DBuf<int32_t> rsz;       // block sizes of A
  DBuf<int64_t> roff;      // scalar offsets of A's block rows
  DBuf<int32_t> ug, ud;    // per union block row: block row of A, subdomain
  DBuf<int64_t> dstart;    // first union block row of each subdomain (nparts + 1)
  DBuf<int64_t> uroff;     // scalar offsets of the union's block rows
  DBuf<int32_t> gidx;      // union scalar row -> scalar row of A
  DBuf<int32_t> src;       // scalar row of A -> its row in the owning subdomain
  DBuf<int64_t> cptr;      // additive: copies of each block row of A ...
  DBuf<int32_t> clist;     // ... as union block rows, in subdomain order
};

void dd_build(const Compressed& A, int nparts, int overlap, bool restricted, cudaStream_t s, DDLayout& L,
              Compressed& U);
void dd_apply(const DDLayout& L, PrecBase& inner, const double* x, double* y, double* xu, double* yu,
              cudaStream_t s);

// Block Jacobi / (restricted) additive Schwarz with the factorization of the
// subdomains' union as the local solver.
struct PrecDD : PrecBase {
  std::unique_ptr<PrecBase> inner;
  DDLayout L;
  DBuf<double> xu, yu;
  int levels() const override { return inner->levels(); }
  void apply_perm(const double* x, double* y) override {
    if (!xu.p && L.nu) {
      xu.alloc(L.nu, s);
      yu.alloc(L.nu, s);
    }
    dd_apply(L, *inner, x, y, xu.p, yu.p, s);
  }
  size_t scratch_bytes() const override;
  void apply_with_scratch(const double* x, double* y, unsigned char* scratch, int nsm) override;
  void export_mat(int lev, int which, int64_t* nbr, int64_t* nbc, int64_t* nnzb, int64_t* nval, int32_t* rsz,
                  int32_t* csz, int64_t* bptr, int32_t* bcol, int64_t* voff, double* val) override {
    inner->export_mat(lev, which, nbr, nbc, nnzb, nval, rsz, csz, bptr, bcol, voff, val);
  }
  void export_vec(int lev, int which, double* d, int32_t* iv, int64_t* len) override {
    inner->export_vec(lev, which, d, iv, len);
  }
  IlutInfo ilut_info() const override { return inner->ilut_info(); }
  PivotTiles pivot_tiles(int l) const override { return inner->pivot_tiles(l); }
  int* status_dev() override { return inner->status_dev(); }
};

// Section 5 Schur-complement global preconditioner (ddschur.cu): the
// interior/interface split of the subdomains, their union (each subdomain's
// interior rows, then its interface rows) and the interface couplings E_ij.
struct DDSLayout {
  int nparts = 0, msteps = 0;
  int64_t n = 0, p = 0;      // scalar and block rows of A (and of the union)
  int64_t ng = 0, ngb = 0;   // interface scalars and interface block rows
  DBuf<int32_t> part, iface; // per block row of A: subdomain, interface flag
  DBuf<int32_t> ug, ud, ufix;// per union block row: block row of A, subdomain, interface flag
  DBuf<int64_t> dstart;      // first union block row of each subdomain (nparts + 1)
  DBuf<int64_t> nint;        // interior block rows of each subdomain
  DBuf<int32_t> gidx;        // union scalar row -> scalar row of A
  DBuf<int32_t> gpos;        // interface scalar -> union scalar row
  VBDev<double> E;           // E_ij on the interface numbering (interface rows ascending)
  DBuf<int64_t> Erb;         // scalar row of E -> its block row
};

void dds_build(const Compressed& A, int nparts, int msteps, cudaStream_t s, DDSLayout& L, Compressed& U);

// One application: local solves, msteps of GMRES on the global interface
// system preconditioned by the local Schur complements, recovery of the
// interior unknowns.
struct PrecDDS : PrecBase {
  std::unique_ptr<PrecBase> inner;  // the union's factorization, interface rows fixed
  DDSLayout L;
  DBuf<unsigned char> work;         // apply_perm's scratch (allocated on first use)
  int levels() const override { return inner->levels(); }
  void apply_perm(const double* x, double* y) override;
  size_t scratch_bytes() const override;
  void apply_with_scratch(const double* x, double* y, unsigned char* scratch, int nsm) override;
  void export_mat(int lev, int which, int64_t* nbr, int64_t* nbc, int64_t* nnzb, int64_t* nval, int32_t* rsz,
                  int32_t* csz, int64_t* bptr, int32_t* bcol, int64_t* voff, double* val) override {
    inner->export_mat(lev, which, nbr, nbc, nnzb, nval, rsz, csz, bptr, bcol, voff, val);
  }
  void export_vec(int lev, int which, double* d, int32_t* iv, int64_t* len) override {
    inner->export_vec(lev, which, d, iv, len);
  }
  IlutInfo ilut_info() const override { return inner->ilut_info(); }
  PivotTiles pivot_tiles(int l) const override { return inner->pivot_tiles(l); }
  int* status_dev() override { return inner->status_dev(); }
};

// Record the message vbarms_last_error() returns on this thread.
void set_last_error(const std::string& msg);

// Build the scalar permutation of level L.
template <typename T>
void build_level_maps(const LevelDev<T>& L, const int32_t* rsz, const int64_t* roff, int64_t p, LevelMaps& M,
                      cudaStream_t s);

// y = A x on a VBCSR matrix (FP64), scalar rows in order; rowblk maps each
// of the n scalar rows to its block row (rowblk_map builds it).
void spmv_vb(const VBDev<double>& A, const int64_t* rowblk, int64_t n, const double* x, double* y,
             cudaStream_t s);
void rowblk_map(const VBDev<double>& A, int64_t n, DBuf<int64_t>& rb, cudaStream_t s);

// Vector kernels used by FGMRES (deterministic two-stage reductions; scratch
// holds at least 512 doubles).
void dot_dev(const double* x, const double* y, int64_t n, double* out, double* scratch, cudaStream_t s);
void axpy_dev(double* y, const double* x, const double* alpha_dev, double sign, int64_t n, cudaStream_t s);
void axpy_host(double* y, const double* x, double alpha, int64_t n, cudaStream_t s);
void scale_dev(double* y, const double* x, const double* div_dev, int64_t n, cudaStream_t s);
void sub_dev(double* r, const double* b, const double* ax, int64_t n, cudaStream_t s);
void gather_dev(double* y, const double* x, const int32_t* idx, int64_t n, cudaStream_t s);
void scatter_dev(double* y, const double* x, const int32_t* idx, int64_t n, cudaStream_t s);

}  // namespace vb

// Opaque handle of the C ABI: a factorization, or one matrix of a batched
// factorization (then its rows are [off, off + len) of the batch's original
// numbering and impl is shared by the batch).
struct vbarms_prec_st {
  std::shared_ptr<vb::PrecBase> impl;
  int64_t off = 0;
  int64_t len = -1;  // -1: the whole factorization
  int64_t size() const { return len < 0 ? impl->n : len; }
};
