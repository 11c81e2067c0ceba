// noalloc.cu -- pic_poisson_solve_static: the standalone Poisson solve with
// its scratch in a fixed device array of this library instead of memory the
// caller allocates.
//
// Who needs it: callers that must not allocate device memory while they run,
// e.g. an application whose own memory pool already owns the device (so a
// cudaMalloc would fail or fragment that pool), or a control loop with a hard
// latency budget that cannot accept cudaMalloc's implicit device-wide
// synchronisation.  Such a caller passes only its inputs and outputs.
//
// Cost of the design: the array below (kStaticScratchBytes) is reserved on
// every GPU that loads the library, for as long as the process lives.  All
// calls on a device share it: two calls that overlap on the GPU (different
// streams, or host threads racing) corrupt each other's scratch, so callers
// must serialise them.  Each call clears what must start at zero.
#include <cstring>

#include "../../include/pic.h"
#include "common.cuh"
#include "launch.h"

namespace {

constexpr size_t kStaticScratchBytes = PIC_POISSON_STATIC_BYTES;

// File-scope device array; host code must not pass its name to a kernel (on
// the host the name is only a stand-in) -- kernels get the address fetched by
// cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_scratch[kStaticScratchBytes];

// Device address of g_scratch on the current device.  Looked up on every
// call (the lookup is cheap next to the synchronous solve): a cached address
// would go stale if the application reset the device or its primary context,
// which reloads the module at another address.  The first lookup on a device
// loads this library's device code there.
int scratch_address(void** out) {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
  if (e != cudaSuccess || !p) return PIC_ERR_CUDA;
  *out = p;
  return PIC_OK;
}

}  // namespace

extern "C" int pic_poisson_solve_static(int nr, int nz, double R, double L, double tol,
                                        int max_iter, const double* Q_dev, double* phi_dev,
                                        void* cuda_stream, int* iters, double* resid) {
  if (nr < 2 || nz < 2 || (nr & 1) || (nz & 1) || !(R > 0) || !(L > 0) || !(tol > 0) ||
      max_iter < 1 || !Q_dev || !phi_dev)
    return PIC_ERR_INVALID;
  const size_t need = pic::poisson_work_bytes(nr, nz);
  if (need + 256 > kStaticScratchBytes) return PIC_ERR_CAPACITY;  // grid above the fixed maximum
  void* base = nullptr;
  int rc = scratch_address(&base);
  if (rc != PIC_OK) return rc;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  int dev = 0, sms = 1;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return PIC_ERR_CUDA;
  // the previous call's contents stay in the array: clear the workspace and
  // the result words
  if (cudaMemsetAsync(base, 0, need + 256, st) != cudaSuccess) return PIC_ERR_CUDA;
  char* tail = (char*)base + need;
  int* status = (int*)tail;
  int* it_dev = (int*)(tail + 16);
  double* res_dev = (double*)(tail + 32);
  if (pic::launch_poisson_in_place(base, nr, nz, R, L, nr + 1, 0, sms, Q_dev, phi_dev, tol, max_iter, status,
                                   it_dev, res_dev, st) != cudaSuccess)
    return PIC_ERR_CUDA;
  int hs[2] = {0, 0};
  double hr = 0.0;
  cudaError_t e = cudaMemcpyAsync(&hs[0], status, 4, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hs[1], it_dev, 4, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hr, res_dev, 8, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return PIC_ERR_CUDA;
  if (iters) *iters = hs[1];
  if (resid) *resid = hr;
  if (hs[0] & pic::ST_TIMEOUT) return PIC_ERR_TIMEOUT;
  if (hs[0] & pic::ST_NONCONV) return PIC_ERR_NONCONVERGED;
  return PIC_OK;
}
