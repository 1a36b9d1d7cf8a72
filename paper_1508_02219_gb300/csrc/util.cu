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


// --------------------------------------------------------------------------
// Stable least-significant-digit radix sort of 64-bit keys, 8 bits a pass:
// per tile of RS_T keys a digit histogram, one scan over (digit, tile), then
// every key goes to its digit's range after the keys of earlier tiles and of
// earlier warps and lanes of its own tile.
namespace {
constexpr int RS64_T = 256;

__global__ void __launch_bounds__(RS64_T) k_rs64_hist(int64_t n, const unsigned long long* __restrict__ key, int shift,
                                                      int64_t ntile, int32_t* __restrict__ hist) {
  __shared__ int h[256];
  for (int d = threadIdx.x; d < 256; d += blockDim.x) h[d] = 0;
  __syncthreads();
  const int64_t e = blockIdx.x * (int64_t)RS64_T + threadIdx.x;
  if (e < n) atomicAdd(&h[(key[e] >> shift) & 255], 1);
  __syncthreads();
  for (int d = threadIdx.x; d < 256; d += blockDim.x) hist[(int64_t)d * ntile + blockIdx.x] = h[d];
}

__global__ void __launch_bounds__(RS64_T) k_rs64_scatter(int64_t n, const unsigned long long* __restrict__ key,
                                                         const int32_t* __restrict__ val, int shift, int64_t ntile,
                                                         const int64_t* __restrict__ base,
                                                         unsigned long long* __restrict__ okey,
                                                         int32_t* __restrict__ oval) {
  __shared__ int cnt[RS64_T / 32][256];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int x = threadIdx.x; x < (RS64_T / 32) * 256; x += blockDim.x) (&cnt[0][0])[x] = 0;
  __syncthreads();
  const int64_t e = blockIdx.x * (int64_t)RS64_T + threadIdx.x;
  const bool has = e < n;
  const unsigned long long k = has ? key[e] : 0ull;
  const int d = has ? (int)((k >> shift) & 255) : 256;
  const unsigned peers = __match_any_sync(0xffffffffu, d);
  const int rank = __popc(peers & ((1u << lane) - 1u));
  if (has && rank == 0) cnt[warp][d] = __popc(peers);
  __syncthreads();
  if (has) {
    int off = 0;
    for (int w = 0; w < warp; ++w) off += cnt[w][d];
    const int64_t pos = base[(int64_t)d * ntile + blockIdx.x] + off + rank;
    okey[pos] = k;
    if (val) oval[pos] = val[e];
  }
}
}  // namespace

void radix_sort_u64(DBuf<unsigned long long>& keys, DBuf<int32_t>* vals, int64_t n, int key_bits, cudaStream_t s) {
  if (n <= 1) return;
  const int64_t ntile = (n + RS64_T - 1) / RS64_T;
  DBuf<int32_t> hist(256 * ntile, s);
  DBuf<int64_t> base(256 * ntile + 1, s);
  DBuf<unsigned long long> k2(n, s);
  DBuf<int32_t> v2;
  if (vals) v2.alloc(n, s);
  for (int shift = 0; shift < key_bits; shift += 8) {
    launch(k_rs64_hist, (unsigned)ntile, RS64_T, 0, s, n, keys.p, shift, ntile, hist.p);
    VB_LAUNCH_CHECK();
    scan_i32_to_i64(hist.p, base.p, 256 * ntile, s);
    launch(k_rs64_scatter, (unsigned)ntile, RS64_T, 0, s, n, keys.p, vals ? vals->p : nullptr, shift, ntile, base.p,
           k2.p, vals ? v2.p : nullptr);
    VB_LAUNCH_CHECK();
    std::swap(keys, k2);
    if (vals) std::swap(*vals, v2);
  }
}

}  // namespace vb
