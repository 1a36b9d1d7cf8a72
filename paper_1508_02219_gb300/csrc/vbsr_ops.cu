// Structural helpers on device VBCSR matrices.
#include "vbsr_ops.cuh"

namespace vb {

__global__ void k_block_sizes(int64_t nbr, const int64_t* __restrict__ bptr, const int32_t* __restrict__ bcol,
                              const int32_t* __restrict__ rsz, const int32_t* __restrict__ csz,
                              int64_t* __restrict__ vsz) {
  const int lane = threadIdx.x & 31;
  const int64_t wpb = blockDim.x >> 5;
  for (int64_t I = blockIdx.x * wpb + (threadIdx.x >> 5); I < nbr; I += (int64_t)gridDim.x * wpb) {
    const int64_t m = rsz[I];
    for (int64_t b = bptr[I] + lane; b < bptr[I + 1]; b += 32) vsz[b] = m * csz[bcol[b]];
  }
}

template <typename T>
void finish_offsets(VBDev<T>& M, cudaStream_t s) {
  M.nnzb = M.nbr ? d2h(M.bptr.p + M.nbr, s) : 0;
  M.voff.alloc(M.nnzb + 1, s);
  if (M.nnzb) {
    DBuf<int64_t> vsz(M.nnzb, s);
    launch(k_block_sizes, grid_for(M.nbr, 8), 256, 0, s, M.nbr, M.bptr.p, M.bcol.p, M.rsz.p, M.csz_p(), vsz.p);
    VB_LAUNCH_CHECK();
    scan_i64(vsz.p, M.voff.p, M.nnzb, s);
    M.nval = d2h(M.voff.p + M.nnzb, s);
  } else {
    M.voff.zero();
    M.nval = 0;
  }
  M.val.alloc(M.nval, s);
}

namespace {

__global__ void k_count_keep(int64_t nbr, const int64_t* __restrict__ bptr, const int8_t* __restrict__ keep,
                             int64_t* __restrict__ cnt) {
  const int lane = threadIdx.x & 31;
  const int64_t wpb = blockDim.x >> 5;
  for (int64_t I = blockIdx.x * wpb + (threadIdx.x >> 5); I < nbr; I += (int64_t)gridDim.x * wpb) {
    int c = 0;
    for (int64_t b = bptr[I] + lane; b < bptr[I + 1]; b += 32) c += keep[b] ? 1 : 0;
    c = warp_sum_i(c);
    if (lane == 0) cnt[I] = c;
  }
}

// dst index of every kept block (order preserved), written into map[b].
__global__ void k_keep_map(int64_t nbr, const int64_t* __restrict__ bptr, const int8_t* __restrict__ keep,
                           const int64_t* __restrict__ dptr, const int32_t* __restrict__ bcol,
                           int32_t* __restrict__ dcol, int64_t* __restrict__ map) {
  const int lane = threadIdx.x & 31;
  const int64_t wpb = blockDim.x >> 5;
  for (int64_t I = blockIdx.x * wpb + (threadIdx.x >> 5); I < nbr; I += (int64_t)gridDim.x * wpb) {
    int64_t base = dptr[I];
    for (int64_t b0 = bptr[I]; b0 < bptr[I + 1]; b0 += 32) {
      int64_t b = b0 + lane;
      bool k = b < bptr[I + 1] && keep[b];
      unsigned m = __ballot_sync(0xffffffffu, k);
      if (k) {
        int64_t d = base + __popc(m & ((1u << lane) - 1u));
        dcol[d] = bcol[b];
        map[b] = d;
      } else if (b < bptr[I + 1]) {
        map[b] = -1;
      }
      base += __popc(m);
    }
  }
}

template <typename T>
__global__ void k_copy_kept(int64_t nbr, const int64_t* __restrict__ bptr, const int64_t* __restrict__ map,
                            const int64_t* __restrict__ svoff, const int64_t* __restrict__ dvoff,
                            const T* __restrict__ sval, T* __restrict__ dval) {
  const int lane = threadIdx.x & 31;
  const int64_t wpb = blockDim.x >> 5;
  for (int64_t I = blockIdx.x * wpb + (threadIdx.x >> 5); I < nbr; I += (int64_t)gridDim.x * wpb) {
    for (int64_t b = bptr[I]; b < bptr[I + 1]; ++b) {
      int64_t d = map[b];
      if (d < 0) continue;
      const int64_t n = svoff[b + 1] - svoff[b];
      for (int64_t e = lane; e < n; e += 32) dval[dvoff[d] + e] = sval[svoff[b] + e];
    }
  }
}

template <typename TD, typename TS>
__global__ void k_convert(int64_t n, const TS* __restrict__ src, TD* __restrict__ dst) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = (TD)src[i];
}

}  // namespace

template <typename T>
void set_partitions(VBDev<T>& M, const int32_t* rsz, int64_t nbr, const int32_t* csz, int64_t nbc,
                    cudaStream_t s) {
  M.nbr = nbr;
  M.nbc = nbc;
  set_partition(M.rsz, M.roff, rsz, nbr, s);
  if (csz == rsz && nbc == nbr) {
    M.same_partition = true;
  } else {
    M.same_partition = false;
    set_partition(M.csz, M.coff, csz, nbc, s);
  }
}

template <typename T>
void compact_blocks(const VBDev<T>& src, const int8_t* keep, VBDev<T>& dst, cudaStream_t s) {
  set_partitions(dst, src.rsz.p, src.nbr, src.csz_p(), src.nbc, s);
  dst.bptr.alloc(src.nbr + 1, s);
  DBuf<int64_t> cnt(src.nbr, s);
  const unsigned g = grid_for(src.nbr, 8);
  if (src.nbr) {
    launch(k_count_keep, g, 256, 0, s, src.nbr, src.bptr.p, keep, cnt.p);
    VB_LAUNCH_CHECK();
  }
  scan_i64(cnt.p, dst.bptr.p, src.nbr, s);
  dst.nnzb = src.nbr ? d2h(dst.bptr.p + src.nbr, s) : 0;
  dst.bcol.alloc(dst.nnzb, s);
  DBuf<int64_t> map(src.nnzb, s);
  if (src.nbr) {
    launch(k_keep_map, g, 256, 0, s, src.nbr, src.bptr.p, keep, dst.bptr.p, src.bcol.p, dst.bcol.p, map.p);
    VB_LAUNCH_CHECK();
  }
  finish_offsets(dst, s);
  if (src.nbr && dst.nval) {
    launch(k_copy_kept<T>, g, 256, 0, s, src.nbr, src.bptr.p, map.p, src.voff.p, dst.voff.p, src.val.p, dst.val.p);
    VB_LAUNCH_CHECK();
  }
}

template <typename TD, typename TS>
void convert_values(const VBDev<TS>& src, VBDev<TD>& dst, cudaStream_t s) {
  if (src.nval)
    launch(k_convert<TD, TS>, grid_for(src.nval, 256, 152LL * 32), 256, 0, s, src.nval, src.val.p, dst.val.p);
  VB_LAUNCH_CHECK();
}

template <typename TD, typename TS>
void copy_vb(const VBDev<TS>& src, VBDev<TD>& dst, cudaStream_t s) {
  set_partitions(dst, src.rsz.p, src.nbr, src.csz_p(), src.nbc, s);
  dst.nnzb = src.nnzb;
  dst.nval = src.nval;
  dst.bptr.alloc(src.nbr + 1, s);
  dst.bcol.alloc(src.nnzb, s);
  dst.voff.alloc(src.nnzb + 1, s);
  dst.val.alloc(src.nval, s);
  VB_CUDA(cudaMemcpyAsync(dst.bptr.p, src.bptr.p, (src.nbr + 1) * sizeof(int64_t), cudaMemcpyDeviceToDevice, s));
  if (src.nnzb) VB_CUDA(cudaMemcpyAsync(dst.bcol.p, src.bcol.p, src.nnzb * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
  VB_CUDA(cudaMemcpyAsync(dst.voff.p, src.voff.p, (src.nnzb + 1) * sizeof(int64_t), cudaMemcpyDeviceToDevice, s));
  convert_values(src, dst, s);
}

template <typename T>
void export_vb(const VBDev<T>& M, cudaStream_t s, int64_t* nbr, int64_t* nbc, int64_t* nnzb, int64_t* nval,
               int32_t* rsz, int32_t* csz, int64_t* bptr, int32_t* bcol, int64_t* voff, double* val) {
  if (!M.bptr.p) fail(VB_EINVAL, "this factor was released after use (vbarms_opts.keep_factors = 0)");
  if (nbr) *nbr = M.nbr;
  if (nbc) *nbc = M.nbc;
  if (nnzb) *nnzb = M.nnzb;
  if (nval) *nval = M.nval;
  if (rsz && M.nbr) VB_CUDA(cudaMemcpyAsync(rsz, M.rsz.p, M.nbr * 4, cudaMemcpyDeviceToHost, s));
  if (csz && M.nbc) VB_CUDA(cudaMemcpyAsync(csz, M.csz_p(), M.nbc * 4, cudaMemcpyDeviceToHost, s));
  if (bptr) VB_CUDA(cudaMemcpyAsync(bptr, M.bptr.p, (M.nbr + 1) * 8, cudaMemcpyDeviceToHost, s));
  if (bcol && M.nnzb) VB_CUDA(cudaMemcpyAsync(bcol, M.bcol.p, M.nnzb * 4, cudaMemcpyDeviceToHost, s));
  if (voff) VB_CUDA(cudaMemcpyAsync(voff, M.voff.p, (M.nnzb + 1) * 8, cudaMemcpyDeviceToHost, s));
  if (val && M.nval) {
    if (sizeof(T) == sizeof(double)) {
      VB_CUDA(cudaMemcpyAsync(val, M.val.p, M.nval * 8, cudaMemcpyDeviceToHost, s));
    } else {
      DBuf<double> tmp(M.nval, s);
      launch(k_convert<double, T>, grid_for(M.nval, 256, 152LL * 32), 256, 0, s, M.nval, M.val.p, tmp.p);
      VB_LAUNCH_CHECK();
      VB_CUDA(cudaMemcpyAsync(val, tmp.p, M.nval * 8, cudaMemcpyDeviceToHost, s));
      VB_CUDA(cudaStreamSynchronize(s));
    }
  }
  VB_CUDA(cudaStreamSynchronize(s));
}

#define VB_INST(T)                                                                                              \
  template void finish_offsets<T>(VBDev<T>&, cudaStream_t);                                                   \
  template void compact_blocks<T>(const VBDev<T>&, const int8_t*, VBDev<T>&, cudaStream_t);                   \
  template void set_partitions<T>(VBDev<T>&, const int32_t*, int64_t, const int32_t*, int64_t, cudaStream_t); \
  template void export_vb<T>(const VBDev<T>&, cudaStream_t, int64_t*, int64_t*, int64_t*, int64_t*, int32_t*,   \
                             int32_t*, int64_t*, int32_t*, int64_t*, double*);
VB_INST(double)
VB_INST(float)
template void convert_values<float, double>(const VBDev<double>&, VBDev<float>&, cudaStream_t);
template void convert_values<double, float>(const VBDev<float>&, VBDev<double>&, cudaStream_t);
template void convert_values<double, double>(const VBDev<double>&, VBDev<double>&, cudaStream_t);
template void convert_values<float, float>(const VBDev<float>&, VBDev<float>&, cudaStream_t);
template void copy_vb<float, double>(const VBDev<double>&, VBDev<float>&, cudaStream_t);
template void copy_vb<double, double>(const VBDev<double>&, VBDev<double>&, cudaStream_t);
template void copy_vb<float, float>(const VBDev<float>&, VBDev<float>&, cudaStream_t);
template void copy_vb<double, float>(const VBDev<float>&, VBDev<double>&, cudaStream_t);

}  // namespace vb
