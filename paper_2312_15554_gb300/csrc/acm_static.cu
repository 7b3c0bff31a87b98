// acm_static.cu -- acm_fft_r2c_static: the 3D real-to-complex transform with
// no device allocation at all.
//
// Some callers cannot let a library allocate device memory: an application
// that gives every component a fixed device-memory budget managed by its own
// allocator, or a latency-critical loop that must not call cudaMalloc/cudaFree
// (they can synchronise the device). For them this entry point keeps its
// working spectrum in a file-scope __device__ array of fixed size that every
// GPU loading the library holds until the process exits; the caller passes
// only the input and the output.
//
// Host code never dereferences or passes the array's name (on the host it is a
// stand-in, not a device address): the first call on a device, with that
// device current, resolves the real addresses with cudaGetSymbolAddress and
// uploads the twiddle table; later calls on that device reuse them.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "acm.h"
#include "acm_ops.h"

using namespace acm;

namespace {

// Maximum working spectrum: n0 * n1 * (n2/2 + 4) complex values of the chosen
// precision must fit in ACM_STATIC_SCRATCH_BYTES.
constexpr size_t STATIC_SCRATCH_BYTES = ACM_STATIC_SCRATCH_BYTES;

static __device__ __align__(256) unsigned char g_scratch[STATIC_SCRATCH_BYTES];
static __device__ __align__(256) double g_tw64[2 * TW_MAX];
static __device__ __align__(256) float g_tw32[2 * TW_MAX];

constexpr int MAX_DEVICES = 64;

struct DeviceSetup {
  bool ready = false;
  void* scratch = nullptr;
  void* tw32 = nullptr;
  void* tw64 = nullptr;
};

DeviceSetup g_dev[MAX_DEVICES];
std::mutex g_mu;

bool pow2_in_range(int n) { return n >= 8 && n <= 512 && (n & (n - 1)) == 0; }

// One-time set-up on the current device: device addresses of the arrays and
// the twiddle tables W_1024^k (computed in FP64 on the host).
acm_status setup_current_device(int dev, DeviceSetup** out) {
  std::lock_guard<std::mutex> lock(g_mu);
  DeviceSetup& s = g_dev[dev];
  if (!s.ready) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess) {
      cudaGetLastError();
      return ACM_ERR_CUDA;
    }
    s.scratch = p;
    if (cudaGetSymbolAddress(&p, g_tw32) != cudaSuccess) {
      cudaGetLastError();
      return ACM_ERR_CUDA;
    }
    s.tw32 = p;
    if (cudaGetSymbolAddress(&p, g_tw64) != cudaSuccess) {
      cudaGetLastError();
      return ACM_ERR_CUDA;
    }
    s.tw64 = p;
    static double h64[2 * TW_MAX];
    static float h32[2 * TW_MAX];
    const double PI = 3.14159265358979323846;
    for (int k = 0; k < TW_MAX; ++k) {
      h64[2 * k] = std::cos(2.0 * PI * k / TW_MAX);
      h64[2 * k + 1] = -std::sin(2.0 * PI * k / TW_MAX);
      h32[2 * k] = (float)h64[2 * k];
      h32[2 * k + 1] = (float)h64[2 * k + 1];
    }
    // a copy from pageable memory may return before its DMA lands; the device
    // synchronisation orders the tables before work on any (non-blocking) stream
    if (cudaMemcpy(s.tw64, h64, sizeof(h64), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(s.tw32, h32, sizeof(h32), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaDeviceSynchronize() != cudaSuccess) {
      cudaGetLastError();
      return ACM_ERR_CUDA;
    }
    s.ready = true;
  }
  *out = &s;
  return ACM_OK;
}

// device memory of the current device `dev` (the kernels run there and read
// and write the buffers directly), or managed memory
bool on_device(const void* p, int dev) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return (a.type == cudaMemoryTypeDevice && a.device == dev) || a.type == cudaMemoryTypeManaged;
}

template <typename T>
acm_status run(const Geo& g, const void* in, void* out, void* scratch, const void* tw, cudaStream_t st) {
  const size_t cs = 2 * sizeof(T);
  Sym<T> none = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  if (Ops<T>::x_r2c(g, 1, 1, scratch, g.S, in, g.V, tw, st) != cudaSuccess ||
      Ops<T>::pass(g, 1, P_FWD, 1, 1, scratch, g.S, none, tw, nullptr, nullptr, nullptr, nullptr, nullptr, st) !=
          cudaSuccess ||
      Ops<T>::pass(g, 0, P_FWD, 1, 1, scratch, g.S, none, tw, nullptr, nullptr, nullptr, nullptr, nullptr, st) !=
          cudaSuccess ||
      cudaMemcpy2DAsync(out, g.Pu * cs, scratch, g.P * cs, g.Pu * cs, (size_t)g.n0 * g.n1,
                        cudaMemcpyDeviceToDevice, st) != cudaSuccess) {
    cudaGetLastError();
    return ACM_ERR_CUDA;
  }
  return ACM_OK;
}

}  // namespace

extern "C" acm_status acm_fft_r2c_static(int n0, int n1, int n2, int fp64, const void* in, void* out,
                                         void* cuda_stream) {
  if (!in || !out || (fp64 != 0 && fp64 != 1)) return ACM_ERR_ARG;
  if (!pow2_in_range(n0) || !pow2_in_range(n1) || !pow2_in_range(n2)) return ACM_ERR_UNSUPPORTED_SIZE;
  Geo g;
  g.n0 = n0;
  g.n1 = n1;
  g.n2 = n2;
  g.Pu = n2 / 2 + 1;
  g.P = n2 / 2 + 4;
  g.V = (long long)n0 * n1 * n2;
  g.S = (long long)n0 * n1 * g.P;
  g.hs = 0;
  g.us = 0;
  g.lph = 1;
  const size_t need = (size_t)g.S * (fp64 ? 2 * sizeof(double) : 2 * sizeof(float));
  if (need > STATIC_SCRATCH_BYTES) return ACM_ERR_UNSUPPORTED_SIZE;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) {
    cudaGetLastError();
    return ACM_ERR_CUDA;
  }
  if (!on_device(in, dev) || !on_device(out, dev)) return ACM_ERR_ARG;
  DeviceSetup* s = nullptr;
  acm_status st = setup_current_device(dev, &s);
  if (st != ACM_OK) return st;
  const cudaStream_t stream = (cudaStream_t)cuda_stream;
  return fp64 ? run<double>(g, in, out, s->scratch, s->tw64, stream)
              : run<float>(g, in, out, s->scratch, s->tw32, stream);
}
