// Structural helpers on device VBCSR matrices: block-size offsets,
// compaction by keep flags, precision conversion, block-row lookups.
#pragma once

#include "common.cuh"

namespace vb {

// vsz[b] = rsz[row(b)] * csz[bcol[b]]  (warp per block row)
__global__ void k_block_sizes(int64_t nbr, const int64_t* __restrict__ bptr, const int32_t* __restrict__ bcol,
                              const int32_t* __restrict__ rsz, const int32_t* __restrict__ csz,
                              int64_t* __restrict__ vsz);

// Given bptr/bcol and partitions, allocate and fill voff (and nval).
template <typename T>
void finish_offsets(VBDev<T>& M, cudaStream_t s);

// dst = the blocks of src whose keep[b] != 0 (same partitions, order kept).
template <typename T>
void compact_blocks(const VBDev<T>& src, const int8_t* keep, VBDev<T>& dst, cudaStream_t s);

// Copy partition arrays of dst from given device sizes.
template <typename T>
void set_partitions(VBDev<T>& M, const int32_t* rsz, int64_t nbr, const int32_t* csz, int64_t nbc,
                    cudaStream_t s);

template <typename TD, typename TS>
void convert_values(const VBDev<TS>& src, VBDev<TD>& dst, cudaStream_t s);

// Deep copy (structure and values) with optional type conversion.
template <typename TD, typename TS>
void copy_vb(const VBDev<TS>& src, VBDev<TD>& dst, cudaStream_t s);

// Host export of a device VBCSR (values converted to double).
template <typename T>
void export_vb(const VBDev<T>& M, cudaStream_t s, int64_t* nbr, int64_t* nbc, int64_t* nnzb, int64_t* nval,
               int32_t* rsz, int32_t* csz, int64_t* bptr, int32_t* bcol, int64_t* voff, double* val);

}  // namespace vb
