// Solve phase of VBARMS on the GPU: Alg. 2 (VBARMS_Solve) over the levels,
// the sync-free block triangular solves of the last level, the VBCSR SpMV and
// the vector kernels of FGMRES.
//
// Vectors are FP64.  FP64 factors are applied in the oracle's operation
// order; FP32 factors are promoted to FP64 as they are read.
#include <type_traits>
#include "prec.cuh"
#include "vbsr_ops.cuh"

namespace vb {
namespace {

constexpr int SW = 8;
constexpr int TRI_R = 4;  // scalar rows per lane in the triangular solves (blocks up to 128)

template <typename T>
__device__ __forceinline__ double ld(const T* p) {
  return (double)*p;
}

// bh[q] = r[sp[q]] * b[sp[q]]
__global__ void k_gather_scale(int64_t n, const int32_t* __restrict__ sp, const double* __restrict__ r,
                               const double* __restrict__ b, double* __restrict__ bh) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
    const int32_t o = sp[q];
    bh[q] = __dmul_rn(r[o], b[o]);
  }
}

// x[sp[q]] = c[sp[q]] * xh[q]
__global__ void k_scatter_scale(int64_t n, const int32_t* __restrict__ sp, const double* __restrict__ c,
                                const double* __restrict__ xh, double* __restrict__ x) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
    const int32_t o = sp[q];
    x[o] = __dmul_rn(c[o], xh[q]);
  }
}

__global__ void k_mul(int64_t n, const double* __restrict__ a, const double* __restrict__ b, double* __restrict__ y) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x)
    y[q] = __dmul_rn(a[q], b[q]);
}

// u <- L^{-1} P u per pivot block (one thread per block).
template <typename TL>
__device__ void pivot_forward(const TL* lu, const int32_t* pv, int m, double* u) {
  for (int k = 0; k < m; ++k)
    if (pv[k] != k) {
      const double t = u[k];
      u[k] = u[pv[k]];
      u[pv[k]] = t;
    }
  for (int i = 1; i < m; ++i)
    for (int k = 0; k < i; ++k) u[i] = __dsub_rn(u[i], __dmul_rn(ld(lu + i * m + k), u[k]));
}

template <typename TL>
__device__ void pivot_backward(const TL* lu, int m, double* u) {
  for (int i = m - 1; i >= 0; --i) {
    double s = u[i];
    for (int k = i + 1; k < m; ++k) s = __dsub_rn(s, __dmul_rn(ld(lu + i * m + k), u[k]));
    u[i] = __ddiv_rn(s, ld(lu + i * m + i));
  }
}

// u <- U^{-1} L^{-1} P u for an FP32 pivot block in FP32 arithmetic (the
// mixed factor applies its FP32 factors in FP32; vectors stay FP64).  m <= 32.
__device__ void pivot_solve_f32(const float* lu, const int32_t* pv, int m, double* u) {
  float x[32];
  for (int k = 0; k < m; ++k) x[k] = (float)u[k];
  for (int k = 0; k < m; ++k)
    if (pv[k] != k) {
      const float t = x[k];
      x[k] = x[pv[k]];
      x[pv[k]] = t;
    }
  for (int i = 1; i < m; ++i) {
    float s = x[i];
    for (int k = 0; k < i; ++k) s = __fmaf_rn(-lu[i * m + k], x[k], s);
    x[i] = s;
  }
  for (int i = m - 1; i >= 0; --i) {
    float s = x[i];
    for (int k = i + 1; k < m; ++k) s = __fmaf_rn(-lu[i * m + k], x[k], s);
    x[i] = __fdiv_rn(s, lu[i * m + i]);
  }
  for (int k = 0; k < m; ++k) u[k] = (double)x[k];
}

__global__ void k_pivot_fwd(int64_t nD, const int32_t* __restrict__ sz, const int64_t* __restrict__ roff,
                            const int64_t* __restrict__ voff, const double* __restrict__ lu64,
                            const float* __restrict__ lu32, const int32_t* __restrict__ ptag,
                            const int32_t* __restrict__ piv, double* __restrict__ u) {
  for (int64_t y = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; y < nD; y += (int64_t)gridDim.x * blockDim.x) {
    if (lu32 && !ptag[y])
      pivot_forward<float>(lu32 + voff[y], piv + roff[y], sz[y], u + roff[y]);
    else
      pivot_forward<double>(lu64 + voff[y], piv + roff[y], sz[y], u + roff[y]);
  }
}

__global__ void k_pivot_bwd(int64_t nD, const int32_t* __restrict__ sz, const int64_t* __restrict__ roff,
                            const int64_t* __restrict__ voff, const double* __restrict__ lu64,
                            const float* __restrict__ lu32, const int32_t* __restrict__ ptag,
                            const double* __restrict__ u, double* __restrict__ x) {
  for (int64_t y = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; y < nD; y += (int64_t)gridDim.x * blockDim.x) {
    const int m = sz[y];
    for (int a = 0; a < m; ++a) x[roff[y] + a] = u[roff[y] + a];
    if (lu32 && !ptag[y])
      pivot_backward<float>(lu32 + voff[y], m, x + roff[y]);
    else
      pivot_backward<double>(lu64 + voff[y], m, x + roff[y]);
  }
}

// y_row -= M x  for every scalar row of a VBCSR M (one thread per scalar row,
// blocks in order, then the entries of the row).
template <typename T>
__global__ void k_bsr_sub(VBView<T> M, const int64_t* __restrict__ rowblk, int64_t nrows,
                          const double* __restrict__ x, double* __restrict__ y) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nrows; q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t I = rowblk[q];
    const int a = (int)(q - M.roff[I]);
    if (sizeof(T) == sizeof(float)) {
      // FP32 factor blocks: products summed in FP32, the result in FP64
      float acc = 0.f;
      for (int64_t b = M.bptr[I]; b < M.bptr[I + 1]; ++b) {
        const int32_t J = M.bcol[b];
        const int nc = M.csz[J];
        const T* v = M.val + M.voff[b] + (int64_t)a * nc;
        const double* xj = x + M.coff[J];
        for (int k = 0; k < nc; ++k) acc = __fmaf_rn((float)v[k], (float)xj[k], acc);
      }
      y[q] = y[q] - (double)acc;
      continue;
    }
    double s = y[q];
    for (int64_t b = M.bptr[I]; b < M.bptr[I + 1]; ++b) {
      const int32_t J = M.bcol[b];
      const int nc = M.csz[J];
      const T* v = M.val + M.voff[b] + (int64_t)a * nc;
      const double* xj = x + M.coff[J];
      for (int k = 0; k < nc; ++k) s = __dsub_rn(s, __dmul_rn(ld(v + k), xj[k]));
    }
    y[q] = s;
  }
}

// y = A x (FP64), one thread per scalar row.
__global__ void k_spmv(VBView<double> A, const int64_t* __restrict__ rowblk, int64_t nrows,
                       const double* __restrict__ x, double* __restrict__ y) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nrows; q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t I = rowblk[q];
    const int a = (int)(q - A.roff[I]);
    double s = 0.0;
    for (int64_t b = A.bptr[I]; b < A.bptr[I + 1]; ++b) {
      const int32_t J = A.bcol[b];
      const int nc = A.csz[J];
      const double* v = A.val + A.voff[b] + (int64_t)a * nc;
      const double* xj = x + A.coff[J];
      for (int k = 0; k < nc; ++k) s = __dadd_rn(s, __dmul_rn(v[k], xj[k]));
    }
    y[q] = s;
  }
}

__global__ void k_rowblk(int64_t nbr, const int64_t* __restrict__ roff, int64_t* __restrict__ rowblk) {
  const int lane = threadIdx.x & 31;
  const int64_t wpb = blockDim.x >> 5;
  for (int64_t I = blockIdx.x * wpb + (threadIdx.x >> 5); I < nbr; I += (int64_t)gridDim.x * wpb)
    for (int64_t q = roff[I] + lane; q < roff[I + 1]; q += 32) rowblk[q] = I;
}

// Bounded wait until row k is published (wait_flag); false when the wait gave
// up or row k failed (a failed row publishes 2).
__device__ __forceinline__ bool wait_row(const int32_t* done, int64_t k, int* abort, unsigned long long limit,
                                         int* st) {
  return wait_flag(done + k, abort, limit, st) == 1;
}

constexpr int TRI_MR = 16;      // block rows up to this size use the lane-per-block path
constexpr int TRI_STAGE = 1024;  // values of a row staged in shared memory per warp
constexpr int TRI_XQ = 16;       // dependency values loaded in one batch

constexpr int TRI_PIV = 72;  // per warp: an FP32 pivot LU of up to 8 x 8 and its 8 interchanges

template <typename T>
constexpr size_t tri_smem() {
  return (size_t)SW * TRI_STAGE * sizeof(T) + (size_t)SW * 32 * TRI_R * sizeof(double) +
         (size_t)SW * TRI_PIV * sizeof(float);
}

// The calling warp's pivot-block buffer in the sweep's shared memory.
template <typename T>
__device__ __forceinline__ float* tri_piv_buf(unsigned char* sm) {
  return (float*)(sm + (size_t)SW * TRI_STAGE * sizeof(T) + (size_t)SW * 32 * TRI_R * sizeof(double)) +
         (size_t)(threadIdx.x >> 5) * TRI_PIV;
}

// Sync-free block triangular sweep over the last-level factors, one warp per
// block row, rows handed out in level order (order[ticket]): every dependency
// of a row sits in an earlier level and so holds an earlier ticket.
//   forward  (BWD = false): y_i <- y_i - sum_{k<i} L_ik y_k        (in place)
//   backward (BWD = true):  x_i <- D_i^{-1} (y_i - sum_{j>i} U_ij x_j)
//                           (rows flagged in fixed keep the x_i in out)
// Rows of up to TRI_MR scalars: the row's block values (static) are staged in
// shared memory before any wait; every lane then owns some blocks of the row,
// waits for its own dependency, loads that dependency's values in one batch
// and accumulates its products privately; a warp reduction forms the update.
// The row's latency is its slowest dependency plus one batched load and a
// reduction.  Larger rows use lanes over scalar rows.
template <typename T, bool BWD>
__global__ void __launch_bounds__(SW * 32)
    k_tri(VBView<T> M, const int64_t* __restrict__ dgoff, const double* __restrict__ lu64,
          const float* __restrict__ lu32, const int32_t* __restrict__ ptag, const int32_t* __restrict__ piv,
          const double* __restrict__ rhs, double* __restrict__ out, const int32_t* __restrict__ order,
          int32_t* __restrict__ done, unsigned long long* ticket, int* abort, unsigned long long wait_limit,
          int* st, const int32_t* __restrict__ fixed) {
  extern __shared__ __align__(16) unsigned char tri_sm[];
  T* stage = (T*)tri_sm + (size_t)(threadIdx.x >> 5) * TRI_STAGE;
  double* sv = (double*)(tri_sm + (size_t)SW * TRI_STAGE * sizeof(T)) + (size_t)(threadIdx.x >> 5) * 32 * TRI_R;
  const int lane = threadIdx.x & 31;
  for (;;) {
    long long t0 = 0;
    if (lane == 0) t0 = (long long)atomicAdd(ticket, 1ULL);
    t0 = __shfl_sync(0xffffffffu, t0, 0);
    if (t0 >= M.nbr) break;
    const int64_t i = order[t0];
    if (BWD && fixed && fixed[i]) {  // the caller gave this row's unknowns (already in out)
      if (lane == 0) atomicExch(&done[i], 1);
      continue;
    }
    const int ni = M.rsz[i];
    const int64_t r0 = M.roff[i];
    bool failed = false;
    // backward sweep, FP32 pivot block of at most 8 rows: the pivot LU and its
    // interchanges are static, so they come into shared memory before the
    // waits below and the final solve reads them on chip
    if (BWD && lu32 && ni <= 8 && !ptag[i]) {
      float* slu = tri_piv_buf<T>(tri_sm);
      const int64_t lo = dgoff[i];
      for (int e = lane; e < ni * ni; e += 32) slu[e] = lu32[lo + e];
      if (lane < ni) reinterpret_cast<int32_t*>(slu + 64)[lane] = piv[r0 + lane];
    }
    if (ni <= TRI_MR) {
      const int64_t b0 = M.bptr[i], b1 = M.bptr[i + 1];
      const int64_t v0 = M.voff[b0];
      const int64_t nv = M.voff[b1] - v0;
      const bool staged = nv <= TRI_STAGE;
      if (staged) {
#pragma unroll 4
        for (int64_t e = lane; e < nv; e += 32) stage[e] = M.val[v0 + e];
      }
      const double r_self = lane < ni ? rhs[r0 + lane] : 0.0;
      __syncwarp();
      // FP32 factors are applied in FP32 (the products and their sums), FP64
      // ones in FP64; the row's result is formed in FP64
      using TA = typename std::conditional<sizeof(T) == sizeof(float), float, double>::type;
      TA part[TRI_MR];
#pragma unroll
      for (int a = 0; a < TRI_MR; ++a) part[a] = 0.0;
      for (int64_t b = b0 + lane; b < b1; b += 32) {
        const int32_t k = M.bcol[b];
        const int nk = M.csz[k];
        const T* v = staged ? stage + (M.voff[b] - v0) : M.val + M.voff[b];
        if (!wait_row(done, k, abort, wait_limit, st)) {
          failed = true;
          break;
        }
        const double* xk = out + M.coff[k];
        for (int q0 = 0; q0 < nk; q0 += TRI_XQ) {
          TA xq[TRI_XQ];
#pragma unroll
          for (int q = 0; q < TRI_XQ; ++q) xq[q] = q0 + q < nk ? (TA)__ldcg(xk + q0 + q) : (TA)0;
#pragma unroll
          for (int q = 0; q < TRI_XQ; ++q) {
            if (q0 + q >= nk) break;
#pragma unroll
            for (int a = 0; a < TRI_MR; ++a)
              if (a < ni) part[a] = fma((TA)v[a * nk + q0 + q], xq[q], part[a]);
          }
        }
      }
      failed = __any_sync(0xffffffffu, failed);
#pragma unroll
      for (int a = 0; a < TRI_MR; ++a)
        for (int o = 16; o > 0; o >>= 1) part[a] += __shfl_xor_sync(0xffffffffu, part[a], o);
      if (!failed && lane < ni) {
        double sa = 0.0;
#pragma unroll
        for (int a = 0; a < TRI_MR; ++a)
          if (a == lane) sa = part[a];
        sv[lane] = r_self - sa;
      }
    } else {
      double s[TRI_R];
#pragma unroll
      for (int t = 0; t < TRI_R; ++t) s[t] = lane + 32 * t < ni ? rhs[r0 + lane + 32 * t] : 0.0;
      if (ni > 32 * TRI_R) {
        if (lane == 0) dev_fail(st, DEV_INTERNAL);
        failed = true;
      }
      for (int64_t b = M.bptr[i]; b < M.bptr[i + 1] && !failed; ++b) {
        const int32_t k = M.bcol[b];
        bool ok = true;
        if (lane == 0) ok = wait_row(done, k, abort, wait_limit, st);
        failed = !__shfl_sync(0xffffffffu, ok, 0);
        if (failed) break;
        const int nk = M.csz[k];
        const double* xk = out + M.coff[k];
#pragma unroll
        for (int t = 0; t < TRI_R; ++t) {
          const int a = lane + 32 * t;
          if (a < ni) {
            const T* v = M.val + M.voff[b] + (int64_t)a * nk;
            for (int q = 0; q < nk; ++q) s[t] = fma(-ld(v + q), __ldcg(xk + q), s[t]);
          }
        }
      }
#pragma unroll
      for (int t = 0; t < TRI_R; ++t)
        if (!failed && lane + 32 * t < ni) sv[lane + 32 * t] = s[t];
    }
    __syncwarp();
    if (!failed) {
      if (BWD && lane == 0) {
        if (lu32 && ni <= 8 && !ptag[i]) {  // the pivot block staged on chip before the waits
          const float* slu = tri_piv_buf<T>(tri_sm);
          pivot_solve_f32(slu, reinterpret_cast<const int32_t*>(slu + 64), ni, sv);
        } else if (lu32 && !ptag[i] && ni <= 32) {
          pivot_solve_f32(lu32 + dgoff[i], piv + r0, ni, sv);
        } else if (lu32 && !ptag[i]) {
          pivot_forward<float>(lu32 + dgoff[i], piv + r0, ni, sv);
          pivot_backward<float>(lu32 + dgoff[i], ni, sv);
        } else {
          pivot_forward<double>(lu64 + dgoff[i], piv + r0, ni, sv);
          pivot_backward<double>(lu64 + dgoff[i], ni, sv);
        }
      }
      __syncwarp();
      for (int a = lane; a < ni; a += 32) out[r0 + a] = sv[a];
    }
    __threadfence();  // every lane's writes before the flag
    __syncwarp();
    if (lane == 0) atomicExch(&done[i], failed ? 2 : 1);
  }
}

// Deterministic two-stage dot product.
constexpr int RT = 256;
constexpr int RB = 512;

__global__ void __launch_bounds__(RT) k_dot_partial(const double* __restrict__ x, const double* __restrict__ y,
                                                    int64_t n, double* __restrict__ part) {
  __shared__ double red[RT / 32];
  double s = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)RT + threadIdx.x; i < n; i += (int64_t)gridDim.x * RT) s += x[i] * y[i];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < RT / 32 ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (threadIdx.x == 0) part[blockIdx.x] = v;
  }
}

__global__ void k_dot_final(const double* __restrict__ part, int nb, double* __restrict__ out) {
  __shared__ double red[RB];
  double s = 0.0;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) s += part[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0];
}

__global__ void k_axpy_dev(double* __restrict__ y, const double* __restrict__ x, const double* __restrict__ a,
                           double sign, int64_t n) {
  const double al = sign * *a;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] += al * x[i];
}
__global__ void k_axpy_host(double* __restrict__ y, const double* __restrict__ x, double a, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] += a * x[i];
}
__global__ void k_scale_dev(double* __restrict__ y, const double* __restrict__ x, const double* __restrict__ d,
                            int64_t n) {
  const double dv = *d;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = x[i] / dv;
}
__global__ void k_sub(double* __restrict__ r, const double* __restrict__ b, const double* __restrict__ ax, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    r[i] = b[i] - ax[i];
}
__global__ void k_gather(double* __restrict__ y, const double* __restrict__ x, const int32_t* __restrict__ idx,
                         int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = x[idx[i]];
}
__global__ void k_scatter(double* __restrict__ y, const double* __restrict__ x, const int32_t* __restrict__ idx,
                          int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[idx[i]] = x[i];
}

__global__ void k_sperm(int64_t p, const int32_t* __restrict__ pI, const int32_t* __restrict__ rsz,
                        const int64_t* __restrict__ roff, const int64_t* __restrict__ newoff,
                        int32_t* __restrict__ sperm) {
  const int lane = threadIdx.x & 31;
  const int64_t wpb = blockDim.x >> 5;
  for (int64_t k = blockIdx.x * wpb + (threadIdx.x >> 5); k < p; k += (int64_t)gridDim.x * wpb) {
    const int32_t Y = pI[k];
    for (int a = lane; a < rsz[Y]; a += 32) sperm[newoff[k] + a] = (int32_t)(roff[Y] + a);
  }
}

__global__ void k_perm_sizes2(int64_t p, const int32_t* __restrict__ pI, const int32_t* __restrict__ rsz,
                              int32_t* __restrict__ out) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < p; k += (int64_t)gridDim.x * blockDim.x)
    out[k] = rsz[pI[k]];
}

}  // namespace

// --------------------------------------------------------------------------
void dot_dev(const double* x, const double* y, int64_t n, double* out, double* scratch, cudaStream_t s) {
  const int nb = (int)std::min<int64_t>(RB, std::max<int64_t>(1, (n + RT - 1) / RT));
  launch(k_dot_partial, nb, RT, 0, s, x, y, n, scratch);
  launch(k_dot_final, 1, RB, 0, s, scratch, nb, out);
  VB_LAUNCH_CHECK();
}
void axpy_dev(double* y, const double* x, const double* a, double sign, int64_t n, cudaStream_t s) {
  if (n) launch(k_axpy_dev, grid_for(n, 256, 152LL * 16), 256, 0, s, y, x, a, sign, n);
  VB_LAUNCH_CHECK();
}
void axpy_host(double* y, const double* x, double a, int64_t n, cudaStream_t s) {
  if (n) launch(k_axpy_host, grid_for(n, 256, 152LL * 16), 256, 0, s, y, x, a, n);
  VB_LAUNCH_CHECK();
}
void scale_dev(double* y, const double* x, const double* d, int64_t n, cudaStream_t s) {
  if (n) launch(k_scale_dev, grid_for(n, 256, 152LL * 16), 256, 0, s, y, x, d, n);
  VB_LAUNCH_CHECK();
}
void sub_dev(double* r, const double* b, const double* ax, int64_t n, cudaStream_t s) {
  if (n) launch(k_sub, grid_for(n, 256, 152LL * 16), 256, 0, s, r, b, ax, n);
  VB_LAUNCH_CHECK();
}
void gather_dev(double* y, const double* x, const int32_t* idx, int64_t n, cudaStream_t s) {
  if (n) launch(k_gather, grid_for(n, 256, 152LL * 16), 256, 0, s, y, x, idx, n);
  VB_LAUNCH_CHECK();
}
void scatter_dev(double* y, const double* x, const int32_t* idx, int64_t n, cudaStream_t s) {
  if (n) launch(k_scatter, grid_for(n, 256, 152LL * 16), 256, 0, s, y, x, idx, n);
  VB_LAUNCH_CHECK();
}

// Row-block map of a VBCSR (scalar row -> block row), cached per matrix.
static void make_rowblk(int64_t nbr, const int64_t* roff, int64_t n, DBuf<int64_t>& rb, cudaStream_t s) {
  rb.alloc(n, s);
  if (nbr) launch(k_rowblk, grid_for(nbr, 8), 256, 0, s, nbr, roff, rb.p);
  VB_LAUNCH_CHECK();
}

void spmv_vb(const VBDev<double>& A, const int64_t* rowblk, int64_t n, const double* x, double* y,
             cudaStream_t s) {
  if (n) launch(k_spmv, grid_for(n, 128, 152LL * 32), 128, 0, s, A.view(), rowblk, n, x, y);
  VB_LAUNCH_CHECK();
}

void rowblk_map(const VBDev<double>& A, int64_t n, DBuf<int64_t>& rb, cudaStream_t s) {
  make_rowblk(A.nbr, A.roff.p, n, rb, s);
}

template <typename T>
void build_level_maps(const LevelDev<T>& L, const int32_t* rsz, const int64_t* roff, int64_t p, LevelMaps& M,
                      cudaStream_t s) {
  M.n = p ? d2h(roff + p, s) : 0;
  M.sperm.alloc(M.n, s);
  DBuf<int32_t> psz(p, s);
  DBuf<int64_t> newoff(p + 1, s);
  if (p) {
    launch(k_perm_sizes2, grid_for(p, 256), 256, 0, s, p, L.pI.p, rsz, psz.p);
    VB_LAUNCH_CHECK();
  }
  scan_i32_to_i64(psz.p, newoff.p, p, s);
  M.nf = p ? d2h(newoff.p + L.nD, s) : 0;
  if (p) {
    launch(k_sperm, grid_for(p, 8), 256, 0, s, p, L.pI.p, rsz, roff, newoff.p, M.sperm.p);
    VB_LAUNCH_CHECK();
  }
}
template void build_level_maps<double>(const LevelDev<double>&, const int32_t*, const int64_t*, int64_t,
                                       LevelMaps&, cudaStream_t);
template void build_level_maps<float>(const LevelDev<float>&, const int32_t*, const int64_t*, int64_t, LevelMaps&,
                                      cudaStream_t);

// --------------------------------------------------------------------------
// The sweeps use more than 48 KB of dynamic shared memory: opt in once per
// device for each instantiation.
template <typename T>
void tri_attributes() {
  static bool set_on[64] = {};
  int dev = 0;
  VB_CUDA(cudaGetDevice(&dev));
  if (dev >= 0 && dev < 64 && set_on[dev]) return;
  VB_CUDA(cudaFuncSetAttribute(k_tri<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tri_smem<T>()));
  VB_CUDA(cudaFuncSetAttribute(k_tri<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tri_smem<T>()));
  if (dev >= 0 && dev < 64) set_on[dev] = true;
}

template <typename T>
void PrecDev<T>::prepare_apply() {
  tri_attributes<T>();
  if (prepared) return;
  const int nl = (int)lev.size();
  int64_t total = 0;
  for (int l = 0; l < nl; ++l) {
    total += 2 * maps[l].n;
    LevelMaps& M = maps[l];
    const LevelDev<T>& L = lev[l];
    if (M.n - M.nf > 0) make_rowblk(L.G.nbr, L.G.roff.p, M.n - M.nf, M.grow, s);
    if (M.nf > 0) make_rowblk(L.W.nbr, L.W.roff.p, M.nf, M.wrow, s);
  }
  nlast = last.A.nbr ? last.A.nrows_scalar(s) : 0;
  total += 2 * nlast;
  work.alloc(std::max<int64_t>(total, 1), s);
  flags.alloc(2 * std::max<int64_t>(last.A.nbr, 1), s);
  tick.alloc(2, s);
  abort_flag.alloc(1, s);
  int dev = 0;
  VB_CUDA(cudaGetDevice(&dev));
  VB_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  prepared = true;
}

namespace {
constexpr int kMaxLev = 64;  // fixed host arrays: the scratch path allocates nothing

// Device buffers of one application of Alg. 2.
struct SolveBufs {
  double* bh[kMaxLev];          // per level: P_I S_1 b, then y = U^{-1}(u - W z)
  double* xh[kMaxLev];          // per level: [y; z] before S_2 P_I^T
  const int64_t* grow[kMaxLev]; // scalar row -> block row of G
  const int64_t* wrow[kMaxLev]; // scalar row -> block row of W
  double* fv[kMaxLev + 1];      // fixed values per level (fv[0]: the caller's)
  double* yy;                   // last level: S_1 g, then L^{-1} S_1 g
  double* xx;                   // last level: U^{-1} L^{-1} S_1 g
  int32_t* flags;               // 2 p_last completion flags
  unsigned long long* tick;     // 2 tickets
  int* abort;
  int nsm;
};

// fv_next[q] = fv[sp[nf + q]] / c[sp[nf + q]]: the fixed values of the C rows
// in the next level's variables (the backward sweep forms x = c * z there).
__global__ void k_fix_down(int64_t n, const int32_t* __restrict__ sp, const double* __restrict__ c,
                           const double* __restrict__ fv, double* __restrict__ fnext) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
    const int32_t o = sp[q];
    fnext[q] = __ddiv_rn(fv[o], c[o]);
  }
}

// Last level: the fixed rows' unknowns before the column scaling.
__global__ void k_fix_last(int64_t p, const int64_t* __restrict__ roff, const int32_t* __restrict__ fixed,
                           const double* __restrict__ fv, const double* __restrict__ c, double* __restrict__ xx) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < p; i += (int64_t)gridDim.x * blockDim.x) {
    if (!fixed[i]) continue;
    for (int64_t q = roff[i]; q < roff[i + 1]; ++q) xx[q] = __ddiv_rn(fv[q], c[q]);
  }
}

// Alg. 2 over all levels, in the factorization's own numbering; enqueues
// work only.  fixv (may be NULL; factorizations with fixed rows only): the
// values the last level's backward sweep takes for its fixed rows instead of
// solving for them (Section 5, the recovery u_i = B_i^{-1}(f_i - F_i y_i)).
template <typename T>
void solve_core(const PrecDev<T>& P, const double* in, double* out, const SolveBufs& B, const double* fixv) {
  cudaStream_t s = P.s;
  const int nl = (int)P.lev.size();
  const bool mixed = sizeof(T) != sizeof(double);
  const auto& last = P.last;
  // forward sweep down the levels: u = L^{-1} P f, g' = g - G u
  for (int l = 0; l < nl; ++l) {
    const LevelDev<T>& L = P.lev[l];
    const LevelMaps& M = P.maps[l];
    const double* b = l == 0 ? in : B.bh[l - 1] + P.maps[l - 1].nf;
    if (M.n) launch(k_gather_scale, grid_for(M.n, 256), 256, 0, s, M.n, M.sperm.p, L.r.p, b, B.bh[l]);
    if (L.grouped)
      grouped_forward<T>(L, B.bh[l], s);
    else if (L.nD)
      launch(k_pivot_fwd, grid_for(L.nD, 128), 128, 0, s, L.nD, L.D.rsz.p, L.D.roff.p, L.D.voff.p, L.D.val.p,
             mixed ? L.D32.val.p : nullptr, L.ptag.p, L.piv.p, B.bh[l]);
    const int64_t ng = M.n - M.nf;
    if (ng && L.G.nnzb)
      launch(k_bsr_sub<T>, grid_for(ng, 128), 128, 0, s, L.G.view(), B.grow[l], ng, B.bh[l], B.bh[l] + M.nf);
    if (fixv && ng)
      launch(k_fix_down, grid_for(ng, 256), 256, 0, s, ng, M.sperm.p + M.nf, L.c.p, l == 0 ? fixv : B.fv[l],
             B.fv[l + 1]);
    VB_LAUNCH_CHECK();
  }
  // last level: z = S2 (L U)^{-1} S1 g
  {
    const int64_t nl_last = nl == 0 ? P.n : P.maps[nl - 1].n - P.maps[nl - 1].nf;
    const double* g = nl == 0 ? in : B.bh[nl - 1] + P.maps[nl - 1].nf;
    double* z = nl == 0 ? out : B.xh[nl - 1] + P.maps[nl - 1].nf;
    if (nl_last) {
      launch(k_mul, grid_for(nl_last, 256), 256, 0, s, nl_last, last.r.p, g, B.yy);
      const int64_t p = last.A.nbr;
      const int32_t* fixed = fixv ? last.fixed.p : nullptr;
      if (fixed)
        launch(k_fix_last, grid_for(p, 256), 256, 0, s, p, last.A.roff.p, fixed, nl == 0 ? fixv : B.fv[nl],
               last.c.p, B.xx);
      // the buffers keep the previous call's contents: clear what starts at 0
      VB_CUDA(cudaMemsetAsync(B.flags, 0, 2 * p * sizeof(int32_t), s));
      VB_CUDA(cudaMemsetAsync(B.tick, 0, 2 * sizeof(unsigned long long), s));
      VB_CUDA(cudaMemsetAsync(B.abort, 0, sizeof(int), s));
      const unsigned nb = (unsigned)std::max<int64_t>(1, std::min<int64_t>((int64_t)B.nsm * 2, (p + SW - 1) / SW));
      launch(k_tri<T, false>, nb, SW * 32, tri_smem<T>(), s, last.L.view(), nullptr, nullptr, nullptr, nullptr,
             nullptr, B.yy, B.yy, last.lorder.p, B.flags, B.tick, B.abort, (unsigned long long)P.wait_limit,
             P.status.p, nullptr);
      launch(k_tri<T, true>, nb, SW * 32, tri_smem<T>(), s, last.U.view(), last.Dg.voff.p, last.Dg.val.p,
             mixed ? last.Dg32.val.p : nullptr, last.ptag.p, last.piv.p, B.yy, B.xx, last.uorder.p, B.flags + p,
             B.tick + 1, B.abort, (unsigned long long)P.wait_limit, P.status.p, fixed);
      launch(k_mul, grid_for(nl_last, 256), 256, 0, s, nl_last, last.c.p, B.xx, z);
      VB_LAUNCH_CHECK();
    }
  }
  // backward sweep up the levels: y = U^{-1} (u - W z), x = S2 P_I^T [y; z]
  for (int l = nl - 1; l >= 0; --l) {
    const LevelDev<T>& L = P.lev[l];
    const LevelMaps& M = P.maps[l];
    double* xo = l == 0 ? out : B.xh[l - 1] + P.maps[l - 1].nf;
    if (M.nf && L.W.nnzb)
      launch(k_bsr_sub<T>, grid_for(M.nf, 128), 128, 0, s, L.W.view(), B.wrow[l], M.nf, B.xh[l] + M.nf, B.bh[l]);
    if (L.grouped)
      grouped_backward<T>(L, B.bh[l], B.xh[l], s);
    else if (L.nD)
      launch(k_pivot_bwd, grid_for(L.nD, 128), 128, 0, s, L.nD, L.D.rsz.p, L.D.roff.p, L.D.voff.p, L.D.val.p,
             mixed ? L.D32.val.p : nullptr, L.ptag.p, B.bh[l], B.xh[l]);
    if (M.n) launch(k_scatter_scale, grid_for(M.n, 256), 256, 0, s, M.n, M.sperm.p, L.c.p, B.xh[l], xo);
    VB_LAUNCH_CHECK();
  }
}

// Doubles of fixed-value work: the C rows of every level.
template <typename T>
int64_t fixed_work(const PrecDev<T>& P) {
  if (!P.last.fixed.p) return 0;
  int64_t t = 0;
  for (const auto& M : P.maps) t += M.n - M.nf;
  return t;
}
}  // namespace

template <typename T>
void PrecDev<T>::apply_perm(const double* x, double* y) {
  apply_fixed(x, y, nullptr);
}

template <typename T>
void PrecDev<T>::apply_fixed(const double* x, double* y, const double* fixv) {
  prepare_apply();
  const int nl = (int)lev.size();
  if (nl > kMaxLev) fail(VB_EINVAL, "more than 64 levels");
  if (fixv && !last.fixed.p) fail(VB_EINVAL, "the factorization has no fixed rows");
  SolveBufs B{};
  double* wp = work.p;
  for (int l = 0; l < nl; ++l) {
    B.bh[l] = wp;
    wp += maps[l].n;
    B.xh[l] = wp;
    wp += maps[l].n;
    B.grow[l] = maps[l].grow.p;
    B.wrow[l] = maps[l].wrow.p;
  }
  B.yy = wp;
  B.xx = wp + nlast;
  if (fixv) {
    const int64_t nf = fixed_work(*this);
    if ((int64_t)fwork.n < nf) fwork.alloc(std::max<int64_t>(nf, 1), s);
    double* fp = fwork.p;
    for (int l = 0; l < nl; ++l) {
      B.fv[l + 1] = fp;
      fp += maps[l].n - maps[l].nf;
    }
  }
  B.flags = flags.p;
  B.tick = tick.p;
  B.abort = abort_flag.p;
  B.nsm = nsm;
  solve_core(*this, x, y, B, fixv);
}

// ---- the same solve with caller-provided scratch (no allocation) ----------
// Layout of the scratch, each piece 256-byte aligned: the permuted x and y
// (n doubles each), the per-level work vectors (2 n_l doubles each), the
// last-level vectors (2 n_last doubles), the row->block maps of G and W
// (n_l int64 per level), the last-level flags (2 p_last int32), two tickets,
// the abort word, and (factorizations with fixed rows) the fixed-value work.
namespace {
struct ScratchPlan {
  size_t xp, yp, work, maps, flags, tick, abort, fwork, total;
};

inline size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

template <typename T>
ScratchPlan plan_scratch(const PrecDev<T>& P) {
  ScratchPlan sp{};
  size_t o = 0;
  int64_t nwork = 0, nmap = 0;
  for (const auto& M : P.maps) {
    nwork += 2 * M.n;
    nmap += M.n;
  }
  const int64_t nlast = P.maps.empty() ? P.n : P.maps.back().n - P.maps.back().nf;
  nwork += 2 * nlast;
  sp.xp = o;
  o = align256(o + (size_t)P.n * 8);
  sp.yp = o;
  o = align256(o + (size_t)P.n * 8);
  sp.work = o;
  o = align256(o + (size_t)nwork * 8);
  sp.maps = o;
  o = align256(o + (size_t)nmap * 8);
  sp.flags = o;
  o = align256(o + (size_t)(2 * P.last.A.nbr) * 4);
  sp.tick = o;
  o = align256(o + 2 * 8);
  sp.abort = o;
  o = align256(o + 4);
  sp.fwork = o;
  o = align256(o + (size_t)fixed_work(P) * 8);
  sp.total = o;
  return sp;
}
}  // namespace

template <typename T>
size_t PrecDev<T>::scratch_bytes() const {
  return plan_scratch(*this).total;
}

template <typename T>
void PrecDev<T>::apply_with_scratch(const double* x, double* y, unsigned char* scratch, int nsm_dev) {
  const ScratchPlan sp = plan_scratch(*this);
  double* xp = (double*)(scratch + sp.xp);
  double* yp = (double*)(scratch + sp.yp);
  gather_dev(xp, x, perm.p, n, s);
  solve_scratch(xp, yp, scratch, nsm_dev, nullptr);
  scatter_dev(y, yp, perm.p, n, s);
}

template <typename T>
void PrecDev<T>::solve_scratch(const double* x, double* y, unsigned char* scratch, int nsm_dev, const double* fixv) {
  tri_attributes<T>();
  const ScratchPlan sp = plan_scratch(*this);
  const int nl = (int)lev.size();
  if (nl > kMaxLev) fail(VB_EINVAL, "more than 64 levels");
  if (fixv && !last.fixed.p) fail(VB_EINVAL, "the factorization has no fixed rows");
  double* wp = (double*)(scratch + sp.work);
  int64_t* mp = (int64_t*)(scratch + sp.maps);
  double* fp = (double*)(scratch + sp.fwork);
  SolveBufs B{};
  for (int l = 0; l < nl; ++l) {
    B.bh[l] = wp;
    wp += maps[l].n;
    B.xh[l] = wp;
    wp += maps[l].n;
    int64_t* gm = mp;
    int64_t* wm = mp + (maps[l].n - maps[l].nf);
    mp += maps[l].n;
    const LevelDev<T>& L = lev[l];
    if (maps[l].n - maps[l].nf > 0 && L.G.nbr)
      launch(k_rowblk, grid_for(L.G.nbr, 8), 256, 0, s, L.G.nbr, L.G.roff.p, gm);
    if (maps[l].nf > 0 && L.W.nbr) launch(k_rowblk, grid_for(L.W.nbr, 8), 256, 0, s, L.W.nbr, L.W.roff.p, wm);
    VB_LAUNCH_CHECK();
    B.grow[l] = gm;
    B.wrow[l] = wm;
    if (fixv) {
      B.fv[l + 1] = fp;
      fp += maps[l].n - maps[l].nf;
    }
  }
  const int64_t nl_last = maps.empty() ? n : maps.back().n - maps.back().nf;
  B.yy = wp;
  B.xx = wp + nl_last;
  B.flags = (int32_t*)(scratch + sp.flags);
  B.tick = (unsigned long long*)(scratch + sp.tick);
  B.abort = (int*)(scratch + sp.abort);
  B.nsm = nsm_dev;
  solve_core(*this, x, y, B, fixv);
}

template <typename T>
void PrecDev<T>::export_mat(int l, int which, int64_t* nbr, int64_t* nbc, int64_t* nnzb, int64_t* nval,
                            int32_t* rsz, int32_t* csz, int64_t* bptr, int32_t* bcol, int64_t* voff, double* val) {
  const int nl = (int)lev.size();
  if (l < 0 || l > nl) fail(VB_EINVAL, "level out of range");
  if (l == nl) {
    switch (which) {
      case 0: return export_vb(last.A, s, nbr, nbc, nnzb, nval, rsz, csz, bptr, bcol, voff, val);
      case 1: return export_vb(last.Dg, s, nbr, nbc, nnzb, nval, rsz, csz, bptr, bcol, voff, val);
      case 8: return export_vb(last.L, s, nbr, nbc, nnzb, nval, rsz, csz, bptr, bcol, voff, val);
      case 9: return export_vb(last.U, s, nbr, nbc, nnzb, nval, rsz, csz, bptr, bcol, voff, val);
    }
    fail(VB_EINVAL, "matrix selector out of range");
  }
  const LevelDev<T>& L = lev[l];
  switch (which) {
    case 0:
      if (L.A64.nbr || !L.AT.nbr) return export_vb(L.A64, s, nbr, nbc, nnzb, nval, rsz, csz, bptr, bcol, voff, val);
      return export_vb(L.AT, s, nbr, nbc, nnzb, nval, rsz, csz, bptr, bcol, voff, val);
    case 1: return export_vb(L.D, s, nbr, nbc, nnzb, nval, rsz, csz, bptr, bcol, voff, val);
    case 2: return export_vb(L.F, s, nbr, nbc, nnzb, nval, rsz, csz, bptr, bcol, voff, val);
    case 3: return export_vb(L.E, s, nbr, nbc, nnzb, nval, rsz, csz, bptr, bcol, voff, val);
    case 4: return export_vb(L.C, s, nbr, nbc, nnzb, nval, rsz, csz, bptr, bcol, voff, val);
    case 5: return export_vb(L.W, s, nbr, nbc, nnzb, nval, rsz, csz, bptr, bcol, voff, val);
    case 6: return export_vb(L.G, s, nbr, nbc, nnzb, nval, rsz, csz, bptr, bcol, voff, val);
    case 7: return export_vb(L.S, s, nbr, nbc, nnzb, nval, rsz, csz, bptr, bcol, voff, val);
    case 10:
      if (!L.grouped) fail(VB_EINVAL, "not a grouped level");
      return export_vb(L.Lg, s, nbr, nbc, nnzb, nval, rsz, csz, bptr, bcol, voff, val);
    case 11:
      if (!L.grouped) fail(VB_EINVAL, "not a grouped level");
      return export_vb(L.Ug, s, nbr, nbc, nnzb, nval, rsz, csz, bptr, bcol, voff, val);
  }
  fail(VB_EINVAL, "matrix selector out of range");
}

template <typename T>
void PrecDev<T>::export_vec(int l, int which, double* d, int32_t* iv, int64_t* len) {
  const int nl = (int)lev.size();
  if (l < 0 || l > nl) fail(VB_EINVAL, "level out of range");
  const DBuf<double>* dv = nullptr;
  const DBuf<int32_t>* ivb = nullptr;
  if (l == nl) {
    if (which == 0) dv = &last.r;
    if (which == 1) dv = &last.c;
    if (which == 4) ivb = &last.piv;
    if (which == 5) ivb = &last.ptag;
  } else {
    const LevelDev<T>& L = lev[l];
    if (which == 0) dv = &L.r;
    if (which == 1) dv = &L.c;
    if (which == 2) dv = &L.w;
    if (which == 3) ivb = &L.pI;
    if (which == 4) ivb = &L.piv;
    if (which == 5) ivb = &L.ptag;
    if (which == 6) {  // group boundaries of a grouped level (ngroups + 1)
      if (!L.grouped) fail(VB_EINVAL, "not a grouped level");
      const std::vector<int64_t> g = d2h_vec(L.gptr.p, L.ngroups + 1, s);
      if (len) *len = (int64_t)g.size();
      if (iv)
        for (size_t k = 0; k < g.size(); ++k) iv[k] = (int32_t)g[k];
      return;
    }
  }
  if (!dv && !ivb) fail(VB_EINVAL, "vector selector out of range");
  const int64_t n = dv ? (int64_t)dv->n : (int64_t)ivb->n;
  if (len) *len = n;
  if (dv && d && n) VB_CUDA(cudaMemcpyAsync(d, dv->p, n * 8, cudaMemcpyDeviceToHost, s));
  if (ivb && iv && n) VB_CUDA(cudaMemcpyAsync(iv, ivb->p, n * 4, cudaMemcpyDeviceToHost, s));
  VB_CUDA(cudaStreamSynchronize(s));
}

template struct PrecDev<double>;
template struct PrecDev<float>;

}  // namespace vb
