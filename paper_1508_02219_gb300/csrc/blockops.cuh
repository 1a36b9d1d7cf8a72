// Dense block operations shared by the reduction levels (level.cu) and the
// grouped levels (groups.cu): each element's terms in the oracle's order,
// separately rounded in FP64 (fused in FP32, the mixed factor's rule).
#pragma once

#include "common.cuh"

namespace vb {

template <typename T>
__device__ __forceinline__ T msub(T acc, T a, T b);
template <>
__device__ __forceinline__ double msub<double>(double acc, double a, double b) {
  return __dsub_rn(acc, __dmul_rn(a, b));
}
template <>
__device__ __forceinline__ float msub<float>(float acc, float a, float b) {
  return __fmaf_rn(-a, b, acc);
}

// X (m x n) <- L^{-1} P X for a GEPP-factored pivot block (lu, pv).
template <typename T, typename TL>
__device__ void linvp_block(const TL* lu, const int32_t* pv, int m, T* x, int n) {
  for (int k = 0; k < m; ++k)
    if (pv[k] != k)
      for (int j = 0; j < n; ++j) {
        const T t = x[k * n + j];
        x[k * n + j] = x[pv[k] * n + j];
        x[pv[k] * n + j] = t;
      }
  for (int i = 1; i < m; ++i)
    for (int k = 0; k < i; ++k) {
      const TL l = lu[i * m + k];
      for (int j = 0; j < n; ++j) x[i * n + j] = (T)msub<TL>((TL)x[i * n + j], l, (TL)x[k * n + j]);
    }
}

template <typename T, typename TL>
__device__ void uinv_right_block(const TL* lu, int m, T* x, int r) {
  for (int i = 0; i < r; ++i)
    for (int j = 0; j < m; ++j) {
      TL s = (TL)x[i * m + j];
      for (int k = 0; k < j; ++k) s = msub<TL>(s, (TL)x[i * m + k], lu[k * m + j]);
      x[i * m + j] = (T)(s / lu[j * m + j]);
    }
}

__device__ __forceinline__ double fro2_d(const double* v, int n) {
  double s = 0.0;
  for (int e = 0; e < n; ++e) s = __dadd_rn(s, __dmul_rn(v[e], v[e]));
  return s;
}
// FP32 blocks (the FP32 levels of the mixed factor): the sum of squares in
// FP32, returned as a double
__device__ __forceinline__ double fro2_d(const float* v, int n) {
  float s = 0.f;
  for (int e = 0; e < n; ++e) s = __fmaf_rn(v[e], v[e], s);
  return (double)s;
}

__device__ __forceinline__ bool drop_rule(double f2, int m, int n, double t) {
  const double thr = __dmul_rn(__dmul_rn(t, (double)m), (double)n);
  return f2 < __dmul_rn(thr, thr);
}

// GEPP of one m x m block in place (max-abs pivot, lowest row on ties);
// false on an exactly zero pivot.
__device__ __forceinline__ bool gepp_block(double* a, int m, int32_t* pv) {
  for (int k = 0; k < m; ++k) {
    int p = k;
    double best = fabs(a[k * m + k]);
    for (int i = k + 1; i < m; ++i) {
      const double v = fabs(a[i * m + k]);
      if (v > best) {
        best = v;
        p = i;
      }
    }
    if (best == 0.0) return false;
    pv[k] = p;
    if (p != k)
      for (int j = 0; j < m; ++j) {
        const double t = a[k * m + j];
        a[k * m + j] = a[p * m + j];
        a[p * m + j] = t;
      }
    const double d = a[k * m + k];
    for (int i = k + 1; i < m; ++i) {
      const double l = __ddiv_rn(a[i * m + k], d);
      a[i * m + k] = l;
      for (int j = k + 1; j < m; ++j) a[i * m + j] = __dsub_rn(a[i * m + j], __dmul_rn(l, a[k * m + j]));
    }
  }
  return true;
}

// The same with the 32 lanes of a warp: the pivot by a warp reduction
// (largest magnitude, lowest row on ties), the multipliers and the trailing
// update over lanes; every element receives gepp_block's operations in its
// order, so the factors are the same bit for bit.  All lanes return the
// same value.
__device__ __forceinline__ bool gepp_block_warp(double* a, int m, int32_t* pv, int lane) {
  for (int k = 0; k < m; ++k) {
    double best = -1.0;
    int p = 0x7fffffff;
    for (int i = k + lane; i < m; i += 32) {
      const double v = fabs(a[i * m + k]);
      if (v > best) {
        best = v;
        p = i;
      }
    }
    for (int o = 16; o > 0; o >>= 1) {
      const double ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int op = __shfl_xor_sync(0xffffffffu, p, o);
      if (ob > best || (ob == best && op < p)) {
        best = ob;
        p = op;
      }
    }
    if (best == 0.0) return false;
    if (lane == 0) pv[k] = p;
    if (p != k)
      for (int j = lane; j < m; j += 32) {
        const double t = a[k * m + j];
        a[k * m + j] = a[p * m + j];
        a[p * m + j] = t;
      }
    __syncwarp();
    const double d = a[k * m + k];
    const int w = m - k - 1;
    for (int r = lane; r < w; r += 32) a[(k + 1 + r) * m + k] = __ddiv_rn(a[(k + 1 + r) * m + k], d);
    __syncwarp();
    for (int e = lane; e < w * w; e += 32) {
      const int r = e / w, c = e - r * w;
      const int i = k + 1 + r, j = k + 1 + c;
      a[i * m + j] = __dsub_rn(a[i * m + j], __dmul_rn(a[i * m + k], a[k * m + j]));
    }
    __syncwarp();
  }
  return true;
}

}  // namespace vb
