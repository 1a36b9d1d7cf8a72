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

// The block-diagonal union of several compressed matrices, for batched
// factorization: parts keep their order, their block and scalar rows are
// numbered consecutively.
void compressed_union(const std::vector<const Compressed*>& parts, cudaStream_t s, Compressed& out);
// dom[k] = the part that block row k of the union comes from.
void union_part_ids(const std::vector<const Compressed*>& parts, cudaStream_t s, DBuf<int32_t>& dom);

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
};

// Step 2: two-sided max-abs scaling in place (FP64 values).
void scale_level(VBDev<double>& A, DBuf<double>& r, DBuf<double>& c, cudaStream_t s);
template <typename T>
void scale_level_t(VBDev<T>& A, DBuf<double>& r, DBuf<double>& c, cudaStream_t s);

}  // namespace vb
