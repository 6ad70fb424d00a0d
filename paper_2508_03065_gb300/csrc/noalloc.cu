// Allocation-free forward synthesis for callers that cannot allocate device
// memory.
//
// Some callers of this library are not allowed to call cudaMalloc: a plug-in
// running inside a host application that owns every device buffer through its
// own pool, or a real-time audio thread that must never enter the CUDA
// allocator (an allocation can synchronise the device and block for an
// unbounded time). msrc_synthesize_noalloc serves them: the scratch memory the
// synthesis needs (image table, sort buffers, prefiltered rows, partial sums)
// lives in a fixed device array that is part of this library's image, so the
// call itself allocates nothing. The caller still provides the signal x and
// the output y.
//
// The array costs every GPU that loads the library kNoAllocScratchBytes of
// device memory until the process exits. It is committed when the library's
// device code is loaded on a GPU; with lazy module loading (the CUDA default)
// that happens at the first allocation-free call there, which therefore
// belongs in the caller's set-up phase. msrc_noalloc_errors reads the device
// error word that the calls leave in the array.
#include <cstdint>
#include <cstdio>
#include <mutex>
#include <string>

#include "msrc.h"

namespace msrc {
void set_last_error(const char* msg);
}

namespace {

constexpr size_t kNoAllocScratchBytes = size_t(MSRC_NOALLOC_SCRATCH_BYTES);
constexpr int kMaxDevices = 64;

// The scratch itself. In host code `g_noalloc_scratch` names a host-side
// stand-in, not device memory: its device address comes from
// cudaGetSymbolAddress on each device.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_setup_mutex;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device (looked up once
// per device, with that device current).
msrc_status scratch_for_current_device(void** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    msrc::set_last_error((std::string("cudaGetDevice: ") + cudaGetErrorString(e)).c_str());
    return MSRC_ERR_CUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) {
    msrc::set_last_error("device index out of range for the scratch table");
    return MSRC_ERR_UNSUPPORTED;
  }
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      msrc::set_last_error((std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e)).c_str());
      return MSRC_ERR_CUDA;
    }
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return MSRC_OK;
}

}  // namespace

extern "C" {

msrc_status msrc_synthesize_noalloc(msrc_room_t room, const float* x_dev, int64_t n_in, float* y_dev,
                                    int64_t n_out, void* stream) {
  if (!room || !x_dev || !y_dev) {
    msrc::set_last_error("null room, x or y");
    return MSRC_ERR_INVALID_ARG;
  }
  size_t need = 0;
  msrc_status s = msrc_workspace_size(&room, 1, &n_in, &n_out, &need, nullptr);
  if (s != MSRC_OK) return s;
  if (need > kNoAllocScratchBytes) {
    char buf[256];
    snprintf(buf, sizeof(buf),
             "scene needs %zu bytes of scratch; the allocation-free entry point holds at most %zu "
             "(use msrc_synthesize with a caller workspace)",
             need, kNoAllocScratchBytes);
    msrc::set_last_error(buf);
    return MSRC_ERR_WORKSPACE;
  }
  void* scratch = nullptr;
  s = scratch_for_current_device(&scratch);
  if (s != MSRC_OK) return s;
  // msrc_synthesize clears the scratch header it relies on (error word, work
  // counter) on the stream before its kernels; every other scratch byte is
  // written before it is read within the call.
  return msrc_synthesize(&room, 1, &x_dev, &n_in, &y_dev, &n_out, scratch, kNoAllocScratchBytes, stream);
}

msrc_status msrc_noalloc_errors(void* stream, uint32_t* flags) {
  if (!flags) {
    msrc::set_last_error("null flags");
    return MSRC_ERR_INVALID_ARG;
  }
  // the scratch's first word is the error word of the last allocation-free
  // call on this device (the workspace header of msrc_synthesize)
  void* scratch = nullptr;
  msrc_status s = scratch_for_current_device(&scratch);
  if (s != MSRC_OK) return s;
  return msrc_workspace_errors(scratch, stream, flags);
}

}  // extern "C"
