// vbarms_apply_static: the preconditioner solve with no device allocation.
//
// Some callers cannot allocate device memory at the point where they apply
// the preconditioner: solver loops with a fixed memory budget that forbid
// allocator calls once set-up is over, and hosts whose device memory belongs
// to another runtime's pool (an embedding application that hands this
// library no allocator of its own).  For them this entry point runs the same
// solve as vbarms_apply, with all of its scratch in one fixed-size device
// array defined in this file.
#include <mutex>
#include <string>

#include "prec.cuh"

// Scratch of vbarms_apply_static: VB_APPLY_STATIC_BYTES bytes that every GPU
// which loads the library holds until the process exits.  In host code the
// name g_apply_scratch is only a host-side stand-in, not a device address;
// the address used on the GPU comes from cudaGetSymbolAddress below.
#define VB_APPLY_STATIC_BYTES (64ull << 20)
static __device__ __align__(256) unsigned char g_apply_scratch[VB_APPLY_STATIC_BYTES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char* g_addr[kMaxDevices] = {};
int g_nsm[kMaxDevices] = {};

// Set-up, once per device and with that device current (the caller makes the
// handle's device current first): the device address of the scratch array
// (return code checked) and the device's SM count.
vb_status setup_device(int dev, unsigned char** addr, int* nsm) {
  if (dev < 0 || dev >= kMaxDevices) {
    vb::set_last_error("vbarms_apply_static: device ordinal beyond the supported 64");
    return VB_ECUDA;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_apply_scratch);
    if (e != cudaSuccess) {
      vb::set_last_error(std::string("vbarms_apply_static: cudaGetSymbolAddress failed: ") +
                         cudaGetErrorString(e));
      return VB_ECUDA;
    }
    int sm = 0;
    e = cudaDeviceGetAttribute(&sm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) {
      vb::set_last_error(std::string("vbarms_apply_static: ") + cudaGetErrorString(e));
      return VB_ECUDA;
    }
    g_addr[dev] = (unsigned char*)p;
    g_nsm[dev] = sm;
  }
  *addr = g_addr[dev];
  *nsm = g_nsm[dev];
  return VB_OK;
}

}  // namespace

extern "C" {

uint64_t vbarms_apply_static_max_bytes(void) { return VB_APPLY_STATIC_BYTES; }

vb_status vbarms_apply_static_need(vbarms_prec M, uint64_t* bytes) {
  if (!M || !bytes) {
    vb::set_last_error("vbarms_apply_static_need: NULL argument");
    return VB_EINVAL;
  }
  if (M->len >= 0) {
    vb::set_last_error("vbarms_apply_static_need: a handle of a batched factorization");
    return VB_EINVAL;
  }
  *bytes = (uint64_t)M->impl->scratch_bytes();
  vb::set_last_error("");
  return VB_OK;
}

vb_status vbarms_apply_static(vbarms_prec M, const double* x, double* y) {
  if (!M || !x || !y) {
    vb::set_last_error("vbarms_apply_static: NULL argument");
    return VB_EINVAL;
  }
  if (x == y) {
    vb::set_last_error("vbarms_apply_static: x and y must not alias");
    return VB_EINVAL;
  }
  if (M->len >= 0) {
    vb::set_last_error("vbarms_apply_static: a handle of a batched factorization; use vbarms_apply");
    return VB_EINVAL;
  }
  try {
    vb::PrecBase& P = *M->impl;
    const size_t need = P.scratch_bytes();
    if (need > VB_APPLY_STATIC_BYTES) {
      vb::set_last_error("vbarms_apply_static: this factorization needs " + std::to_string(need) +
                         " bytes of scratch, above the fixed maximum of " + std::to_string(VB_APPLY_STATIC_BYTES) +
                         " bytes; use vbarms_apply");
      return VB_EINVAL;
    }
    // the handle's device, whatever device is current: the scratch address
    // belongs to it
    vb::DeviceScope ds(P.dev);
    unsigned char* scratch = nullptr;
    int nsm = 0;
    const vb_status st = setup_device(P.dev, &scratch, &nsm);
    if (st != VB_OK) return st;
    P.apply_with_scratch(x, y, scratch, nsm);
    vb::check_status(P.status_dev(), P.s, "vbarms_apply_static");
  } catch (const vb::Error& err) {
    vb::set_last_error(err.msg);
    return err.st;
  }
  vb::set_last_error("");
  return VB_OK;
}

}  // extern "C"
