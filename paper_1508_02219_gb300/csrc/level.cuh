// Host entry points of the per-level kernels (Steps 2-4) and of the
// last-level block ILUT and the solve phase.
#pragma once

#include "internal.h"

namespace vb {

// Step 3: weights, independent set, P_I.  Returns nD.  fixed (device, may
// be NULL): rows kept out of the set.
template <typename TA>
int64_t is_order(const VBDev<TA>& A, double ddtol, DBuf<double>& w, DBuf<int32_t>& pI, DBuf<int32_t>& newpos,
                 cudaStream_t s, const int32_t* fixed = nullptr);

// Step 3 weights w(Y) = ||A_YY||_F / sum_Z ||A_YZ||_F (R5).
template <typename TA>
void level_weights(const VBDev<TA>& A, DBuf<double>& w, cudaStream_t s);

// Step 3 with groups of up to gs supernodes (the diagonal blocks D_i of D
// block sparse): pI lists the groups by smallest member (members ascending),
// then C ascending; gptr[ngroups + 1] bounds the groups over the D rows.
// Returns nD.
template <typename TA>
int64_t group_order(const VBDev<TA>& A, double ddtol, int gs, const int32_t* fixed, DBuf<double>& w,
                    DBuf<int32_t>& pI, DBuf<int32_t>& newpos, DBuf<int64_t>& gptr, int64_t& ngroups,
                    cudaStream_t s);

// Steps 3-4 of a grouped level (Section 3.1's two sweeps inside each group):
// D (pivot LU after the group elimination), piv, the group multipliers Lg,
// the group part Ug of Ubar, W = Ltilde^{-1} F and G = E Ubar^{-1}; F, E, C
// gathered.  S follows from schur() as for ungrouped levels.
template <typename TA, typename T>
void grouped_level(const VBDev<TA>& A, const DBuf<int32_t>& pI, const DBuf<int32_t>& newpos, int64_t nD,
                   const DBuf<int64_t>& gptr, int64_t ngroups, double t, int lfil, LevelDev<T>& L, cudaStream_t s,
                   int* dst);

// The level solve of a grouped level: forward u = Ltilde^{-1} P f in place
// in bh (its D part), backward xh = Ubar^{-1} bh (bh already holds u - W z).
template <typename T>
void grouped_forward(const LevelDev<T>& L, double* bh, cudaStream_t s);
template <typename T>
void grouped_backward(const LevelDev<T>& L, const double* bh, double* xh, cudaStream_t s);

// Eq. 4: the D (FP64 pivot blocks), F, E, C parts of P_I A P_I^T.
template <typename TA, typename T>
void gather_parts(const VBDev<TA>& A, const DBuf<int32_t>& pI, const DBuf<int32_t>& newpos, int64_t nD,
                  LevelDev<T>& L, cudaStream_t s, int* dst);

// Batched GEPP of the pivot blocks (in place), with the mixed-precision tag:
// one persistent launch over block-size-class queues; info (may be NULL)
// receives the classes' sizes and modes.
void pivot_lu(VBDev<double>& D, DBuf<int32_t>& piv, DBuf<int32_t>& ptag, VBDev<float>& D32, bool mixed,
              double cond_thr, cudaStream_t s, int* dst, PivotTiles* info = nullptr);

// which = 0: W = L^{-1} P F from F;  which = 1: G = E U^{-1} from E.
template <typename T>
void w_or_g(const VBDev<T>& X, int which, const VBDev<double>& D, const VBDev<float>& D32, const DBuf<int32_t>& piv,
            const DBuf<int32_t>& ptag, bool mixed, double t, int lfil, VBDev<T>& out, cudaStream_t s);

// Timing record of one launch of a measured kernel (CUDA events on the
// launching stream) with its algorithmic bytes and flops.
struct KernelRec {
  int kernel = 0;  // 0 = Schur numeric
  int level = 0;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  double bytes = 0, flops = 0, ms = -1;
};

// Eq. 6: S = C - G W (drop at the last reduction).  rec (may be NULL)
// receives the timing of the numeric launch.
template <typename T>
void schur(const VBDev<T>& C, const VBDev<T>& G, const VBDev<T>& W, bool last_reduction, double t, VBDev<T>& S,
           cudaStream_t s, int* dst, KernelRec* rec);

// Last level: block ILUT in natural order (Alg. 3 in block form).  order
// (may be NULL) hands the rows out in another sequence that keeps every
// row's dependencies before it (ticket_order).
template <typename T>
void ilut_last(LastDev<T>& X, double t, int lfil, bool mixed, double cond_thr, uint64_t wait_limit, cudaStream_t s,
               int* dst, const int32_t* order = nullptr);

// For a matrix of independent diagonal blocks (dom[r]: the block of row r,
// nondecreasing, values in [0, ndom)): the rows interleaved round-robin over
// the blocks, each block's rows ascending.  Leaves order empty when ndom is
// above kTicketMaxDom.
constexpr int kTicketMaxDom = 4096;
void ticket_order(const int32_t* dom, int64_t p, int ndom, DBuf<int32_t>& order, cudaStream_t s);
// dst[k] = src[idx[k]]
void take_i32(const int32_t* src, const int32_t* idx, int64_t n, int32_t* dst, cudaStream_t s);

// Solve phase (Alg. 2) helpers.
template <typename T>
struct PrecDev;

}  // namespace vb
