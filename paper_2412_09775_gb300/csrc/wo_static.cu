// wo_static.cu - wo_reconstruct_static: the reconstruction with a workspace
// that lives in the library itself instead of in caller-allocated memory.
//
// Some callers cannot allocate device memory at the point where they need a
// reconstruction: a plugin running inside a host application that owns the
// whole device-memory budget, code that sits behind a caching allocator it is
// not allowed to bypass, or a latency-bound loop that must not pay the
// implicit device synchronisation of cudaMalloc/cudaFree.  For them this entry
// point takes the same inputs and outputs as wo_reconstruct but uses a
// file-scope device array as its workspace.  It calls no cudaMalloc, cudaFree
// or other allocating routine.
#include <mutex>

#include "wo_internal.h"

// The scratch array: every GPU that loads this library holds these bytes
// until the process exits.
static __device__ __align__(256) unsigned char g_wo_static_scratch[WO_STATIC_SCRATCH_BYTES];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_static_mu;
void* g_static_ptr[kMaxDevices] = {};
}  // namespace

extern "C" wo_status wo_reconstruct_static(const void* d_tf, unsigned kinds, const float* d_data,
                                           const float* h_background, const float* h_eta, int eta_flag,
                                           int mode, float* d_f, int n_tiles, int Z, int Y, int X,
                                           wo_stream stream) {
  // The array's name is only a host-side stand-in in host code: its device
  // address is looked up with the device current.  The first call on a device
  // does the lookup (and loads the array there); every later call outside
  // stream capture looks it up again, so a context that was reset or replaced
  // since is followed; a call made while `stream` is being captured uses the
  // address found by the last call on that device.
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return WO_ERR_CUDA;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing((cudaStream_t)stream, &cap) != cudaSuccess) return WO_ERR_CUDA;
  void* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_static_mu);
    if (!g_static_ptr[dev] || cap == cudaStreamCaptureStatusNone) {
      if (cap != cudaStreamCaptureStatusNone) return WO_ERR_CUDA;  // first call on a device inside a capture
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_wo_static_scratch) != cudaSuccess || !p) return WO_ERR_CUDA;
      g_static_ptr[dev] = p;
    }
    scratch = g_static_ptr[dev];
  }
  const size_t need = wo_workspace_bytes(n_tiles, Z, Y, X, kinds);
  if (need > (size_t)WO_STATIC_SCRATCH_BYTES) return WO_ERR_WORKSPACE;
  // need == 0 (invalid shape or kinds) falls through to wo_reconstruct's own
  // validation, which returns the matching status.  Every workspace byte the
  // reconstruction reads it first writes (or zeroes) in the same call, so
  // nothing in the shared array has to be cleared between calls; the array's
  // status block is not read by this entry point.
  return wo_reconstruct(d_tf, kinds, d_data, h_background, h_eta, eta_flag, mode, d_f, n_tiles, Z, Y, X,
                        scratch, (size_t)WO_STATIC_SCRATCH_BYTES, stream);
}
