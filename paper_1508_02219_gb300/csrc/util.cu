// Host/device plumbing: status word readback, prefix sums, partitions.
#include "common.cuh"

namespace vb {

std::atomic<unsigned long long> g_launch_count{0};
std::atomic<unsigned long long> g_alloc_count{0};

void DeviceScope::throw_cuda_error(const char* what) {
  fail(VB_ECUDA, std::string(what) + " failed: no usable device for this handle");
}

int current_device() {
  int d = 0;
  VB_CUDA(cudaGetDevice(&d));
  return d;
}

void check_status(int* dst, cudaStream_t s, const char* where) {
  int st = d2h(dst, s);
  if (st == DEV_OK) return;
  VB_CUDA(cudaMemsetAsync(dst, 0, sizeof(int), s));
  switch (st) {
    case DEV_EINVAL: fail(VB_EINVAL, std::string(where) + ": invalid input");
    case DEV_ESINGULAR: fail(VB_ESINGULAR, std::string(where) + ": exactly singular pivot block");
    case DEV_ETIMEOUT: fail(VB_ETIMEOUT, std::string(where) + ": bounded device wait ran out");
    default: fail(VB_EINTERNAL, std::string(where) + ": device status " + std::to_string(st));
  }
}

namespace {

constexpr int SCAN_T = 512;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_T * SCAN_ITEMS;

template <typename TIn>
__global__ void __launch_bounds__(SCAN_T) k_tile_sums(const TIn* __restrict__ in, int64_t n,
                                                      int64_t* __restrict__ sums) {
  __shared__ long long red[SCAN_T / 32];
  const int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
  long long s = 0;
  for (int i = threadIdx.x; i < SCAN_TILE; i += SCAN_T) {
    int64_t idx = base + i;
    if (idx < n) s += (long long)in[idx];
  }
  s = warp_sum_ll(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    long long v = threadIdx.x < SCAN_T / 32 ? red[threadIdx.x] : 0;
    v = warp_sum_ll(v);
    if (threadIdx.x == 0) sums[blockIdx.x] = v;
  }
}

// out[idx + 1] = tile_off[tile] + inclusive prefix within the tile.
template <typename TIn>
__global__ void __launch_bounds__(SCAN_T) k_tile_scan(const TIn* __restrict__ in, int64_t n,
                                                      int64_t* __restrict__ out,
                                                      const int64_t* __restrict__ tile_off) {
  __shared__ long long wsum[SCAN_T / 32];
  const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
  long long v[SCAN_ITEMS];
  long long run = 0;
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; ++k) {
    int64_t idx = base + k;
    run += idx < n ? (long long)in[idx] : 0;
    v[k] = run;
  }
  // exclusive scan of per-thread totals across the block
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  long long incl = run;
  for (int o = 1; o < 32; o <<= 1) {
    long long t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  if (lane == 31) wsum[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    long long w = lane < SCAN_T / 32 ? wsum[lane] : 0;
    for (int o = 1; o < 32; o <<= 1) {
      long long t = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += t;
    }
    if (lane < SCAN_T / 32) wsum[lane] = w;  // inclusive per warp
  }
  __syncthreads();
  long long before = (incl - run) + (warp ? wsum[warp - 1] : 0) + (tile_off ? tile_off[blockIdx.x] : 0);
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; ++k) {
    int64_t idx = base + k;
    if (idx < n) out[idx + 1] = before + v[k];
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) out[0] = 0;
}

template <typename TIn>
void scan_impl(const TIn* in, int64_t* out, int64_t n, cudaStream_t s) {
  if (n <= 0) {
    VB_CUDA(cudaMemsetAsync(out, 0, sizeof(int64_t), s));
    return;
  }
  const int64_t tiles = (n + SCAN_TILE - 1) / SCAN_TILE;
  if (tiles == 1) {
    launch(k_tile_scan<TIn>, 1, SCAN_T, 0, s, in, n, out, nullptr);
    VB_LAUNCH_CHECK();
    return;
  }
  DBuf<int64_t> sums(tiles, s), offs(tiles + 1, s);
  launch(k_tile_sums<TIn>, (unsigned)tiles, SCAN_T, 0, s, in, n, sums.p);
  VB_LAUNCH_CHECK();
  scan_impl<int64_t>(sums.p, offs.p, tiles, s);
  launch(k_tile_scan<TIn>, (unsigned)tiles, SCAN_T, 0, s, in, n, out, offs.p);
  VB_LAUNCH_CHECK();
}

}  // namespace

void scan_i64(const int64_t* in, int64_t* out, int64_t n, cudaStream_t s) { scan_impl<int64_t>(in, out, n, s); }
void scan_i32_to_i64(const int32_t* in, int64_t* out, int64_t n, cudaStream_t s) {
  scan_impl<int32_t>(in, out, n, s);
}

void set_partition(DBuf<int32_t>& sz, DBuf<int64_t>& off, const int32_t* src, int64_t nb, cudaStream_t s) {
  sz.alloc(nb, s);
  off.alloc(nb + 1, s);
  if (nb) VB_CUDA(cudaMemcpyAsync(sz.p, src, nb * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
  scan_i32_to_i64(sz.p, off.p, nb, s);
}

}  // namespace vb
