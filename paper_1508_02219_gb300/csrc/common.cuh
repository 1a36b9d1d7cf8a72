// Shared device/host plumbing of the VBARMS CUDA library: error handling,
// stream-ordered device buffers, prefix sums, hashing and the device VBCSR
// container.  No step of the method lives here.
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <cstring>
#include <string>
#include <utility>
#include <vector>

#include "vbarms.h"

namespace vb {

struct Error {
  vb_status st;
  std::string msg;
};

[[noreturn]] inline void fail(vb_status st, const std::string& msg) { throw Error{st, msg}; }

#define VB_CUDA(call)                                                                        \
  do {                                                                                       \
    cudaError_t e_ = (call);                                                                 \
    if (e_ != cudaSuccess)                                                                   \
      ::vb::fail(e_ == cudaErrorMemoryAllocation ? VB_ENOMEM : VB_ECUDA,                     \
                 std::string(#call) + ": " + cudaGetErrorString(e_));                        \
  } while (0)

#define VB_LAUNCH_CHECK() VB_CUDA(cudaGetLastError())

// Every kernel of the library is launched through launch(), which counts it.
extern std::atomic<unsigned long long> g_launch_count;
// Every device allocation of the library goes through DBuf::alloc, which
// counts it.
extern std::atomic<unsigned long long> g_alloc_count;

// Makes device dev current for the lifetime of the object and restores the
// device that was current before.  Handles remember the device they were
// created on; every entry point that works with a handle runs inside one.
struct DeviceScope {
  int prev = -1, dev = 0;
  explicit DeviceScope(int d) : dev(d) {
    if (cudaGetDevice(&prev) != cudaSuccess) {
      prev = -1;
      (void)cudaGetLastError();
      throw_cuda_error("cudaGetDevice");
    }
    if (prev != dev && cudaSetDevice(dev) != cudaSuccess) {
      (void)cudaGetLastError();
      prev = -1;
      throw_cuda_error("cudaSetDevice");
    }
  }
  ~DeviceScope() {
    if (prev >= 0 && prev != dev) cudaSetDevice(prev);
  }
  DeviceScope(const DeviceScope&) = delete;
  DeviceScope& operator=(const DeviceScope&) = delete;
  [[noreturn]] static void throw_cuda_error(const char* what);
};

// The device current in this thread (VB_ECUDA when there is none).
int current_device();

template <typename... KArgs, typename... Args>
inline void launch(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, Args&&... args) {
  kernel<<<grid, block, smem, s>>>(std::forward<Args>(args)...);
  g_launch_count.fetch_add(1, std::memory_order_relaxed);
}

// Device status word shared by the kernels of one call: first error wins.
enum DevCode : int {
  DEV_OK = 0,
  DEV_EINVAL = 1,
  DEV_ESINGULAR = 4,
  DEV_ETIMEOUT = 5,
  DEV_OVERFLOW = 100,  // a scratch capacity was too small: the host retries
  DEV_INTERNAL = 7,
};

__device__ __forceinline__ void dev_fail(int* st, int code) { atomicCAS(st, 0, code); }

// Device-wide nanosecond timer (bounds the spin waits by time).
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Default time budget of a bounded device wait: 30 s.
constexpr unsigned long long kDefaultWaitNs = 30ull * 1000 * 1000 * 1000;

__device__ __forceinline__ int ld_relaxed_gpu(const int32_t* p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Publication flags of the sync-free kernels: a producer writes its data,
// fences (__threadfence) and sets the flag to 1, or to 2 when it failed.  A
// consumer waits here: relaxed polls with exponential backoff, the shared
// abort word and the time budget looked at only every 16th poll (so that
// waiting warps do not crowd one L2 line), then one acquire fence, which pairs
// with the producer's fence.  Returns the flag, or 0 when the wait gave up:
// abort raised elsewhere, or limit ns passed (then DEV_ETIMEOUT is recorded
// and abort raised).
__device__ __forceinline__ int wait_flag(const int32_t* flag, int* abort, unsigned long long limit, int* st) {
  int v = ld_relaxed_gpu(flag);
  if (v == 0) {
    const unsigned long long t0 = global_ns();
    unsigned nsl = 32;
    for (unsigned it = 1;; ++it) {
      __nanosleep(nsl);
      if (nsl < 256) nsl <<= 1;
      v = ld_relaxed_gpu(flag);
      if (v != 0) break;
      if ((it & 15) == 0) {
        if (*((volatile int*)abort) != 0) return 0;
        if (global_ns() - t0 > limit) {
          dev_fail(st, DEV_ETIMEOUT);
          atomicExch(abort, 1);
          return 0;
        }
      }
    }
  }
  asm volatile("fence.acq_rel.gpu;" ::: "memory");
  return v;
}

// --------------------------------------------------------------------------
// Stream-ordered device buffer (cudaMallocAsync / cudaFreeAsync).
template <typename T>
struct DBuf {
  T* p = nullptr;
  size_t n = 0;
  cudaStream_t s = nullptr;

  DBuf() = default;
  DBuf(size_t count, cudaStream_t st) { alloc(count, st); }
  DBuf(const DBuf&) = delete;
  DBuf& operator=(const DBuf&) = delete;
  DBuf(DBuf&& o) noexcept : p(o.p), n(o.n), s(o.s) { o.p = nullptr, o.n = 0; }
  DBuf& operator=(DBuf&& o) noexcept {
    if (this != &o) {
      release();
      p = o.p, n = o.n, s = o.s;
      o.p = nullptr, o.n = 0;
    }
    return *this;
  }
  ~DBuf() { release(); }

  void alloc(size_t count, cudaStream_t st) {
    release();
    s = st;
    n = count;
    if (count) {
      cudaError_t e = cudaMallocAsync((void**)&p, count * sizeof(T), st);
      if (e != cudaSuccess) {
        p = nullptr;
        n = 0;
        (void)cudaGetLastError();
        fail(VB_ENOMEM, "device allocation of " + std::to_string(count * sizeof(T)) + " bytes failed");
      }
      g_alloc_count.fetch_add(1, std::memory_order_relaxed);
    }
  }
  void zero() {
    if (n) VB_CUDA(cudaMemsetAsync(p, 0, n * sizeof(T), s));
  }
  void fill_bytes(int b) {
    if (n) VB_CUDA(cudaMemsetAsync(p, b, n * sizeof(T), s));
  }
  void release() {
    if (p) cudaFreeAsync(p, s);
    p = nullptr;
    n = 0;
  }
  T* get() const { return p; }
};

template <typename T>
T d2h(const T* dptr, cudaStream_t s) {
  T v;
  VB_CUDA(cudaMemcpyAsync(&v, dptr, sizeof(T), cudaMemcpyDeviceToHost, s));
  VB_CUDA(cudaStreamSynchronize(s));
  return v;
}

template <typename T>
std::vector<T> d2h_vec(const T* dptr, size_t n, cudaStream_t s) {
  std::vector<T> v(n);
  if (n) {
    VB_CUDA(cudaMemcpyAsync(v.data(), dptr, n * sizeof(T), cudaMemcpyDeviceToHost, s));
    VB_CUDA(cudaStreamSynchronize(s));
  }
  return v;
}

template <typename T>
void h2d(T* dptr, const T* h, size_t n, cudaStream_t s) {
  if (n) VB_CUDA(cudaMemcpyAsync(dptr, h, n * sizeof(T), cudaMemcpyHostToDevice, s));
}

// Read the device status word, reset it, and turn a failure into an Error.
void check_status(int* dst, cudaStream_t s, const char* where);

inline unsigned grid_for(int64_t work, int per_block, int64_t cap = 152LL * 64) {
  int64_t g = (work + per_block - 1) / per_block;
  if (g < 1) g = 1;
  if (g > cap) g = cap;
  return (unsigned)g;
}

// --------------------------------------------------------------------------
// Exclusive prefix sum: out[0] = 0, out[i+1] = out[i] + in[i] (out has n+1
// entries).  in and out must not overlap.  Read the total from out[n].
void scan_i64(const int64_t* in, int64_t* out, int64_t n, cudaStream_t s);
void scan_i32_to_i64(const int32_t* in, int64_t* out, int64_t n, cudaStream_t s);

// Stable ascending sort of keys[0, n) on their low key_bits bits (8 bits a
// pass), moving vals (may be NULL) alongside.  The buffers are swapped with
// scratch ones: keys and *vals hold the result.
void radix_sort_u64(DBuf<unsigned long long>& keys, DBuf<int32_t>* vals, int64_t n, int key_bits, cudaStream_t s);

// --------------------------------------------------------------------------
// Integer hash-set helpers (open addressing, linear probing, key -1 = empty).
__device__ __forceinline__ uint32_t hmix(uint32_t x) {
  x ^= x >> 16;
  x *= 0x7feb352du;
  x ^= x >> 15;
  x *= 0x846ca68bu;
  x ^= x >> 16;
  return x;
}

// Insert key into keys[0..mask]; returns the slot, or -1 when the table is
// full.  *fresh tells whether this call created the entry.
__device__ __forceinline__ int hset_insert(int* keys, uint32_t mask, int key, bool* fresh) {
  uint32_t h = hmix((uint32_t)key) & mask;
  for (uint32_t probe = 0; probe <= mask; ++probe) {
    int k = atomicCAS(&keys[h], -1, key);
    if (k == -1) {
      *fresh = true;
      return (int)h;
    }
    if (k == key) {
      *fresh = false;
      return (int)h;
    }
    h = (h + 1) & mask;
  }
  *fresh = false;
  return -1;
}

__device__ __forceinline__ int hset_find(const int* keys, uint32_t mask, int key) {
  uint32_t h = hmix((uint32_t)key) & mask;
  for (uint32_t probe = 0; probe <= mask; ++probe) {
    int k = keys[h];
    if (k == key) return (int)h;
    if (k == -1) return -1;
    h = (h + 1) & mask;
  }
  return -1;
}

__device__ __forceinline__ int warp_sum_i(int v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ long long warp_sum_ll(long long v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ int warp_min_i(int v) {
  for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ int warp_max_i(int v) {
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Binary search of key in the ascending array a[lo, hi); returns index or -1.
__device__ __forceinline__ int64_t bsearch_i32(const int32_t* a, int64_t lo, int64_t hi, int32_t key) {
  while (lo < hi) {
    int64_t mid = (lo + hi) >> 1;
    int32_t v = a[mid];
    if (v == key) return mid;
    if (v < key)
      lo = mid + 1;
    else
      hi = mid;
  }
  return -1;
}

// --------------------------------------------------------------------------
// Device VBCSR matrix: block rows/cols of variable size, each stored block a
// dense row-major rsz[I] x csz[J] array; blocks of a block row contiguous.
template <typename T>
struct VBView {
  int64_t nbr, nbc;
  const int32_t* rsz;
  const int32_t* csz;
  const int64_t* roff;
  const int64_t* coff;
  const int64_t* bptr;
  const int32_t* bcol;
  const int64_t* voff;
  T* val;
};

template <typename T>
struct VBDev {
  int64_t nbr = 0, nbc = 0, nnzb = 0, nval = 0;
  DBuf<int32_t> rsz, csz;
  DBuf<int64_t> roff, coff;
  DBuf<int64_t> bptr;
  DBuf<int32_t> bcol;
  DBuf<int64_t> voff;
  DBuf<T> val;
  bool same_partition = false;  // csz/coff alias rsz/roff

  VBView<T> view() const {
    VBView<T> v;
    v.nbr = nbr;
    v.nbc = nbc;
    v.rsz = rsz.p;
    v.roff = roff.p;
    v.csz = same_partition ? rsz.p : csz.p;
    v.coff = same_partition ? roff.p : coff.p;
    v.bptr = bptr.p;
    v.bcol = bcol.p;
    v.voff = voff.p;
    v.val = val.p;
    return v;
  }
  const int32_t* csz_p() const { return same_partition ? rsz.p : csz.p; }
  const int64_t* coff_p() const { return same_partition ? roff.p : coff.p; }
  int64_t nrows_scalar(cudaStream_t s) const { return nbr ? d2h(roff.p + nbr, s) : 0; }
};

// Set partition arrays (sizes -> offsets) from device sizes.
void set_partition(DBuf<int32_t>& sz, DBuf<int64_t>& off, const int32_t* src, int64_t nb, cudaStream_t s);

}  // namespace vb
