// stokes_vanka_noalloc: the Vanka patch-solve sum y = M_l^-1 x of one level
// without any device allocation, for callers that must not allocate device
// memory while they run (for example code that runs inside a region where
// the memory budget is fixed, or that is driven from a context in which
// cudaMalloc is not permitted).  Its scratch - the copy of x in the cycle
// precision, the patch-major solutions and the result before conversion -
// lives in one file-scope device array of kScratchBytes; the handle
// (factors, index lists) must have been set up and factorised beforehand.
#include <mutex>
#include <string>

#include "common.cuh"
#include "stokes_dcamg.h"

namespace {

constexpr size_t kScratchBytes = size_t(32) << 20;  // 32 MiB, held by every GPU that loads the library

static __device__ __align__(256) unsigned char g_vanka_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device, looked up
// once per device (the array's host-side name is not a device address).
int scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return sd::set_error(STOKES_ERR_CUDA, cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return sd::set_error(STOKES_ERR_INVALID_ARG, "device index out of range");
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_vanka_scratch);
    if (e != cudaSuccess)
      return sd::set_error(STOKES_ERR_CUDA, (std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e)).c_str());
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return STOKES_OK;
}

inline size_t up256(size_t b) { return (b + 255) / 256 * 256; }

template <typename T>
int run(const sd::VankaView& v, unsigned char* scratch, const double* x, double* y) {
  T* xin = reinterpret_cast<T*>(scratch);
  T* yp = reinterpret_cast<T*>(scratch + up256(sizeof(T) * v.n));
  T* out = reinterpret_cast<T*>(scratch + up256(sizeof(T) * v.n) + up256(sizeof(T) * v.pat->nslots));
  cudaError_t e = sd::cast_copy<double, T>(v.n, x, xin, v.st);
  if (e == cudaSuccess) e = sd::vanka_apply<T, T>(*v.pat, xin, yp, v.st);
  if (e == cudaSuccess) e = sd::vanka_scatter<T>(*v.pat, v.n, yp, out, 1.0, 0, nullptr, nullptr, nullptr, v.st);
  if (e == cudaSuccess) e = sd::cast_copy<T, double>(v.n, out, y, v.st);
  if (e != cudaSuccess) return sd::set_error(STOKES_ERR_CUDA, cudaGetErrorString(e));
  return STOKES_OK;
}

}  // namespace

extern "C" int stokes_vanka_noalloc(stokes_handle* h, int32_t level, const double* x_dev, double* y_dev) {
  if (!h || !x_dev || !y_dev) return sd::set_error(STOKES_ERR_INVALID_ARG, "null argument");
  sd::VankaView v;
  int rc = sd::vanka_level_view(h, level, &v);
  if (rc != STOKES_OK) return rc;
  const size_t elem = v.fp32 ? 4 : 8;
  const size_t need = up256(elem * v.n) + up256(elem * v.pat->nslots) + up256(elem * v.n);
  if (need > kScratchBytes)
    return sd::set_error(STOKES_ERR_INVALID_ARG,
                         ("stokes_vanka_noalloc: level " + std::to_string(level) + " needs " + std::to_string(need) +
                          " bytes of scratch; the fixed buffer holds " + std::to_string(kScratchBytes))
                             .c_str());
  void* scratch = nullptr;
  rc = scratch_address(&scratch);
  if (rc != STOKES_OK) return rc;
  rc = sd::stream_join_in(h);
  if (rc != STOKES_OK) return rc;
  rc = v.fp32 ? run<float>(v, static_cast<unsigned char*>(scratch), x_dev, y_dev)
              : run<double>(v, static_cast<unsigned char*>(scratch), x_dev, y_dev);
  if (rc != STOKES_OK) return rc;
  // a bounded wait of the bulk-copy apply that ran out leaves part of the
  // patch solutions unwritten; the scatter then read what an earlier call
  // left in the shared scratch, so y is unusable: read the level's flag
  // (this waits for the call's work on the handle's stream)
  int flag = 0;
  cudaError_t e = cudaMemcpyAsync(&flag, v.pat->err, sizeof(int), cudaMemcpyDeviceToHost, v.st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(v.st);
  if (e != cudaSuccess) return sd::set_error(STOKES_ERR_CUDA, cudaGetErrorString(e));
  if (flag)
    return sd::set_error(STOKES_ERR_CUDA, ("stokes_vanka_noalloc: a bulk-copy pipeline wait of level " +
                                           std::to_string(level) + " timed out (flag " + std::to_string(flag) +
                                           "); the output is unusable")
                                              .c_str());
  return sd::stream_join_out(h);
}
