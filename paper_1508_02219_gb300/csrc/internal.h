// Internal interfaces between the translation units of the library.
#pragma once

#include "common.cuh"

namespace vb {

// Result of Step 1 (Section 2.1, Eq. 3).
struct Compressed {
  int64_t n = 0, nnz = 0;
  DBuf<int32_t> perm;  // perm[k] = original row at permuted position k
  VBDev<double> A;     // P_B A P_B^T, square partition (same_partition)
  double av_bd = 0, av_bs = 0;
};

void compress_device(int64_t n, const int64_t* rowptr, const int32_t* colind, const double* val, double tau,
                     cudaStream_t s, int* dstatus, Compressed& out);

// A1: CSR validation (columns in range, ascending, unique; rowptr monotone)
// into the status word; len[i] = row lengths.
void validate_csr(int64_t n, const int64_t* rowptr, const int32_t* colind, int32_t* len, cudaStream_t s, int* dst);

// A4: the VBCSR matrix P_B A P_B^T of a grouping of the rows into p blocks:
// bsz/boff block sizes and offsets, blk[r] the block of row r, offin[r] its
// place in the block, out.perm and out.nnz already set.
void assemble_vbcsr(int64_t n, const int64_t* rowptr, const int32_t* colind, const double* val, int64_t p,
                    DBuf<int32_t>& bsz, DBuf<int64_t>& boff, const int32_t* blk, const int32_t* offin,
                    cudaStream_t s, int* dstatus, Compressed& out);

// leader[v] = the smallest u whose CSR list (ptr, col; sorted lists) equals
// v's: classes of identical lists, by a hash, a sort and exact comparisons.
void list_classes(int64_t n, const int64_t* ptr, const int32_t* col, int32_t* leader, cudaStream_t s);

// VBCSR of the grouping whose every row r belongs to the group of lead[r],
// the group's smallest row (lead[lead[r]] = lead[r]); blocks in ascending
// order of their smallest row, rows ascending.
void assemble_from_leaders(int64_t n, const int64_t* rowptr, const int32_t* colind, const double* val,
                           const int32_t* lead, cudaStream_t s, int* dst, Compressed& out);

// Two-pass checksum and angle compression (Section 2.1, readings T1-T3):
// classes of identical nonempty row patterns with two or more rows form the
// groups (ordered by smallest row); every other row joins the first group
// whose pattern passes the angle test cos >= tau, else stays alone.
void two_pass_compress_device(int64_t n, const int64_t* rowptr, const int32_t* colind, const double* val,
                              double tau, cudaStream_t s, int* dst, Compressed& out);

// Graph-based compression (Section 2.2, Alg. 1) with minimum block density
// mu: exact classes of identical closed neighbourhoods of A + A^T, then the
// merge pass; the same VBCSR assembly as compress_device.
void graph_compress_device(int64_t n, const int64_t* rowptr, const int32_t* colind, const double* val, double mu,
                           cudaStream_t s, int* dstatus, Compressed& out);

// The block-diagonal union of several compressed matrices, for batched
// factorization: parts keep their order, their block and scalar rows are
// numbered consecutively.
void compressed_union(const std::vector<const Compressed*>& parts, cudaStream_t s, Compressed& out);
// dom[k] = the part that block row k of the union comes from.
void union_part_ids(const std::vector<const Compressed*>& parts, cudaStream_t s, DBuf<int32_t>& dom);

// How a level's pivot phase ran: pivot blocks per size class (<= 4, <= 8,
// <= 16, <= 32, more), the mode of each class (0: a thread per block, 1: a
// warp per block) and how the modes were chosen (0 default, 1 timed on this
// level's blocks, 2 taken from an earlier timing in this process).
struct PivotTiles {
  int count[5] = {0, 0, 0, 0, 0};
  int mode[5] = {0, 0, 1, 1, 1};
  int source = 0;
};

// One reduction level (Steps 2-4) on the device.
template <typename T>
struct LevelDev {
  VBDev<double> A64;      // scaled level matrix when it is FP64 (FP64 mode, level 1)
  VBDev<T> AT;            // scaled level matrix when it is of type T != double
  DBuf<double> r, c, w;   // Step 2 scalings, Step 3 weights
  DBuf<int32_t> pI;       // new order: pI[k] = supernode at position k
  int64_t nD = 0, nC = 0;
  VBDev<double> D;        // pivot blocks, GEPP LU in place (FP64)
  VBDev<float> D32;       // FP32 copy of the LU (mixed precision)
  DBuf<int32_t> piv;      // GEPP interchanges, per scalar row of D
  DBuf<int32_t> ptag;     // 1 = pivot block kept in FP64 (mixed precision)
  VBDev<T> F, E, C, W, G, S;
  // groups of more than one supernode (Step 3 with block-sparse D_i)
  bool grouped = false;
  int64_t ngroups = 0;
  DBuf<int64_t> gptr;     // group boundaries over the D rows
  VBDev<T> Lg, Ug;        // group multipliers (below), group part of Ubar (above)
  PivotTiles tiles;       // how the pivot phase ran
};

// How the last-level ILUT ran: its per-warp shared workspace (slots, value
// bytes), warps per SM, and whether the geometry was the default (0), timed
// on a prefix of this matrix (1, tune_s seconds) or taken from an earlier
// timing of a matrix of the same class (2).
struct IlutInfo {
  int slots = 0, vbytes = 0, warps_per_sm = 0, source = 0;
  long long chain = 0;  // rows on the longest chain of waits of the final run
  double tune_s = 0;
};

template <typename T>
struct LastDev {
  VBDev<T> A;  // scaled last-level matrix
  DBuf<double> r, c;
  VBDev<double> Dg;  // pivot LU (FP64)
  VBDev<float> Dg32;
  DBuf<int32_t> piv, ptag;
  VBDev<T> L, U;
  // rows of L (U) sorted by their level in the dependency DAG of the forward
  // (backward) sweep: the triangular solves take rows in this order
  DBuf<int32_t> lorder, uorder;
  int64_t ldepth = 0, udepth = 0;
  IlutInfo info;
  // rows kept out of every independent set (the interface rows of the
  // Schur-complement preconditioner), one flag per row; empty when none
  DBuf<int32_t> fixed;
};

// Level orders of the last level's triangular sweeps (L forward: row i
// depends on its columns k < i; U backward: on its columns j > i), computed
// on the device with bounded waits (wait_limit ns; failures go to dst).
template <typename T>
void level_orders(LastDev<T>& X, uint64_t wait_limit, int* dst, cudaStream_t s);

struct FactorOpts {
  int nlev;
  double droptol;
  int lfil;
  int precision;
  double fp64_pivot_cond;
  double ddtol;
  uint64_t wait_limit;
  bool schur_drop_all;
  bool keep_factors;
  int group_size;  // supernodes per independent group (Step 3)
};

// Step 2: two-sided max-abs scaling in place (FP64 values).
void scale_level(VBDev<double>& A, DBuf<double>& r, DBuf<double>& c, cudaStream_t s);
template <typename T>
void scale_level_t(VBDev<T>& A, DBuf<double>& r, DBuf<double>& c, cudaStream_t s);

}  // namespace vb
