// fftmech_fft_noalloc: the stand-alone Stockham transform of fftmech_fft
// without any device allocation. fftmech_fft allocates the twiddle tables of
// every new length with cudaMalloc; this variant keeps them in one file-scope
// device array of fixed size instead (no counterpart in the paper).
#include <cuda_runtime.h>

#include <mutex>

#include "fftmech.h"
#include "fftmech_internal.cuh"
#include "host_plan.cuh"

using namespace fftmech;

namespace {

constexpr int kMaxN = FFTMECH_FFT_NOALLOC_MAX_N;
// Layout: x and y plans in double, then x and y plans in float; a slot holds
// the twiddles and pass multipliers of a plan of length up to kMaxN (the
// layout the transform kernels copy to shared memory).
constexpr size_t kSlotD = tw_smem_bytes<double>(kMaxN);
constexpr size_t kSlotF = tw_smem_bytes<float>(kMaxN);
constexpr size_t kScratchBytes = 2 * kSlotD + 2 * kSlotF;
constexpr int kMaxDevices = 64;

}  // namespace

// The scratch array. Every GPU that loads the library holds it until the
// process exits; each call overwrites the entries it uses.
static __device__ __align__(256) unsigned char g_fft_noalloc_scratch[kScratchBytes];

namespace {

std::mutex g_mu;                      // serialises calls: host buffers and the device array
void* g_scratch_dev[kMaxDevices];     // device address of the array, per device
cx<double> g_tw[2 * kMaxN];           // host FP64 twiddles of the x and y plans (no heap use)
alignas(16) unsigned char g_stage[kScratchBytes];  // host image of the slots

// One slot image: twiddles rounded to T, then the pass multipliers.
template <typename T>
void fill_slot(const HostPlan& p, const cx<double>* tw, unsigned char* slot) {
  cx<T>* t = reinterpret_cast<cx<T>*>(slot);
  for (int i = 0; i < p.n - 1; ++i) {
    t[i].re = (T)tw[i].re;
    t[i].im = (T)tw[i].im;
  }
  plan_multipliers(p.n, p.npass, p.radix, reinterpret_cast<unsigned int*>(slot + tw_smem_twiddles<T>(p.n)));
}

// Device address of the scratch array on `dev` (current device). The first
// call on a device looks it up; later calls reuse it.
cudaError_t scratch_address(int dev, unsigned char** out) {
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  if (!g_scratch_dev[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_fft_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_dev[dev] = p;
  }
  *out = static_cast<unsigned char*>(g_scratch_dev[dev]);
  return cudaSuccess;
}

bool on_device(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

template <typename T>
cudaError_t run(HostPlan& px, HostPlan& py, int inverse, void* data, const Shape2& sh, cudaStream_t st) {
  const int nx = px.n, ny = py.n;
  cudaError_t e = launch_rowfft_f<T>(px.fam, nx, ny, (cx<T>*)data, dev_plan<T>(px), inverse, sh, st);
  if (e == cudaSuccess && ny > 1) {
    Spec<T> sp{};
    e = launch_colpass_f<T>(py.fam, nx, ny, (cx<T>*)data, dev_plan<T>(py), sp, sh, COL_PLAIN, inverse,
                            nullptr, nullptr, nullptr, st);
  }
  return e;
}

}  // namespace

extern "C" fftmech_status fftmech_fft_noalloc(int ndim, const int n[3], int precision, int inverse,
                                              void* data, void* stream) {
  if (!n || !data || (ndim != 1 && ndim != 2)) return FFTMECH_ERR_INVALID_ARG;
  if (precision != FFTMECH_FP64 && precision != FFTMECH_MIXED) return FFTMECH_ERR_INVALID_ARG;
  const int nx = n[0], ny = ndim == 2 ? n[1] : 1;
  if (!factor_ok(nx) || !factor_ok(ny) || nx < 2) return FFTMECH_ERR_UNSUPPORTED_SIZE;
  if (nx > kMaxN || ny > kMaxN) return FFTMECH_ERR_UNSUPPORTED_SIZE;  // beyond the fixed array
  if (!on_device(data)) return FFTMECH_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(g_mu);
  int dev = 0, nsm = 0, optin = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
    return FFTMECH_ERR_CUDA;
  unsigned char* base = nullptr;
  if (scratch_address(dev, &base) != cudaSuccess) return FFTMECH_ERR_CUDA;
  HostPlan px, py;
  factor_plan(nx, px);
  factor_plan(ny, py);
  fill_twiddles(px, g_tw);
  fill_twiddles(py, g_tw + kMaxN);
  cudaStream_t st = (cudaStream_t)stream;
  const bool fp64 = precision == FFTMECH_FP64;
  // launch shapes first: a size the kernels cannot take is rejected before
  // anything is queued on the stream
  Shape2 sh{};
  const bool shp = fp64 ? choose_shape_fft<double>(px, py, nsm, (size_t)optin, sh)
                        : choose_shape_fft<float>(px, py, nsm, (size_t)optin, sh);
  if (!shp) return FFTMECH_ERR_UNSUPPORTED_SIZE;
  px.tw_d = reinterpret_cast<cx<double>*>(base);
  py.tw_d = reinterpret_cast<cx<double>*>(base + kSlotD);
  px.tw_f = reinterpret_cast<cx<float>*>(base + 2 * kSlotD);
  py.tw_f = reinterpret_cast<cx<float>*>(base + 2 * kSlotD + kSlotF);
  // Every byte a launch reads (twiddles and multipliers, the first
  // tw_smem_bytes(n) bytes of a slot) is written here first, so nothing in
  // the array has to start at zero.
  cudaError_t e = cudaSuccess;
  if (fp64) {
    fill_slot<double>(px, g_tw, g_stage);
    fill_slot<double>(py, g_tw + kMaxN, g_stage + kSlotD);
    e = cudaMemcpyAsync(px.tw_d, g_stage, tw_smem_bytes<double>(nx), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(py.tw_d, g_stage + kSlotD, tw_smem_bytes<double>(ny), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = run<double>(px, py, inverse, data, sh, st);
  } else {
    fill_slot<float>(px, g_tw, g_stage + 2 * kSlotD);
    fill_slot<float>(py, g_tw + kMaxN, g_stage + 2 * kSlotD + kSlotF);
    e = cudaMemcpyAsync(px.tw_f, g_stage + 2 * kSlotD, tw_smem_bytes<float>(nx), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(py.tw_f, g_stage + 2 * kSlotD + kSlotF, tw_smem_bytes<float>(ny), cudaMemcpyHostToDevice,
                          st);
    if (e == cudaSuccess) e = run<float>(px, py, inverse, data, sh, st);
  }
  // Whatever happened after the first copy was queued, the stream is drained
  // before the lock is released: the next call may then overwrite the array
  // and the host image without racing with copies or transforms of this one.
  const cudaError_t es = cudaStreamSynchronize(st);
  if (e == cudaSuccess) e = es;
  return e == cudaSuccess ? FFTMECH_OK : FFTMECH_ERR_CUDA;
}
