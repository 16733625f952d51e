// ssb_reconstruct_static: the single-candidate SSB reconstruction without any
// caller-provided or library-allocated scratch buffer.
//
// Who needs it: a caller that cannot (or must not) allocate device memory at
// the point where it wants a phase image -- for example a detector-acquisition
// plugin whose host application owns every device buffer, or a real-time loop
// whose memory is fixed at start-up and which must not call cudaMalloc because
// that call can synchronise the device and stall the stream of incoming frames.
// Such a caller passes only its inputs (G, aberrations) and outputs (phase,
// variance, status); the working memory comes from the array below, which is
// part of the library's device image and is loaded once per GPU.
//
// Rules of use:
// * The array holds EER4D_STATIC_SCRATCH_BYTES (8 MiB); a plan whose
//   single-candidate scratch is larger (scans beyond about 1024 x 1024) is
//   rejected with EER4D_ESCRATCH before anything is enqueued.
// * Every call on a device shares the one array and it keeps the previous
//   call's contents.  Nothing in it has to start at zero: every word the call
//   reads is first written by an earlier kernel of the same call.  Calls whose
//   work overlaps on the GPU (different streams, or host threads, without an
//   ordering between them) race on the array and give wrong results; order
//   them on one stream.
// * The first call on each device looks up the array's device address with
//   cudaGetSymbolAddress (with that device current); make that first call
//   before any stream capture.  The address is kept for the life of the
//   process: it assumes the device's primary context is not reset
//   (cudaDeviceReset) while the library is in use; after a reset the kept
//   address is stale.
#include <mutex>

#include "common.cuh"

namespace {

static __device__ __align__(256) unsigned char g_static_scratch[EER4D_STATIC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

// Device address of g_static_scratch on device `dev` (the current device);
// host code must not use the symbol itself, which is a host-side stand-in.
cudaError_t scratch_address(int dev, void** out) {
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return e;
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" int ssb_reconstruct_static(const eer4d_plan* p, const void* d_G, const double* d_aberr,
                                      float* d_phase, double* d_var, uint32_t* d_status,
                                      void* stream) {
  if (!p || !d_G || !d_aberr) return EER4D_EINVAL;
  if (trotter_scratch_bytes(p, 1, TROT_FWD) > (size_t)EER4D_STATIC_SCRATCH_BYTES)
    return EER4D_ESCRATCH;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  void* scratch = nullptr;
  if (e == cudaSuccess) e = scratch_address(dev, &scratch);
  if (e != cudaSuccess) return cuda_status(e);
  return cuda_status(launch_trotter(p, static_cast<const float2*>(d_G), d_aberr, 1, TROT_FWD,
                                    scratch, nullptr, d_phase, d_var, nullptr, nullptr, d_status,
                                    (cudaStream_t)stream));
}
