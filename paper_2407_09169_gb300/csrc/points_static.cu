// Point evaluation of the PDF without any allocation.
//
// qtt_observe(..., QTT_OBS_POINTS, ...) allocates device buffers for the
// query and its scratch on every call and frees them afterwards.  Some
// callers cannot allow that: processes whose device memory is entirely
// reserved by their own pool (a framework's caching allocator that holds the
// whole GPU), and monitoring loops that probe the PDF every step and must not
// pay the implicit device-wide synchronisation of cudaFree.
// qtt_observe_points_noalloc serves them: the query flags, the per-point
// scratch vectors and the results live in one file-scope device array of
// fixed size, so the call performs no cudaMalloc, cudaFree or other
// allocating routine.  It still copies the query in and the values out on the
// context's stream and synchronises that stream before it returns.
//
// The array is shared by every call in the process (and is resident on every
// GPU that loads the library until the process exits); calls whose work
// overlaps on the GPU race on it, so callers must serialise them.
#include <cstdint>
#include <cstring>
#include <mutex>
#include <stdexcept>
#include <string>

#include "engine.hpp"

namespace qtt {

namespace {

// Capacity of the shared scratch array.
constexpr size_t kPointsScratchBytes = (size_t)4 << 20;

static __device__ __align__(256) unsigned char g_points_scratch[kPointsScratchBytes];

// Device ordinals served by the per-device address cache below.
constexpr int kMaxDevices = 64;

// The host-side name g_points_scratch is only a stand-in symbol; the device
// address of the array is looked up once per device (with that device
// current) and cached.
void* scratch_address(int device) {
  static std::mutex mu;
  static void* addr[kMaxDevices] = {nullptr};
  static bool ready[kMaxDevices] = {false};
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess) {
    cudaGetLastError();
    throw std::runtime_error("CUDA error: cudaGetDeviceCount failed");
  }
  if (device < 0 || device >= ndev || device >= kMaxDevices)
    throw std::runtime_error("EINVAL: device ordinal " + std::to_string(device) + " out of range");
  std::lock_guard<std::mutex> lock(mu);
  if (!ready[device]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_points_scratch);
    if (e != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      throw std::runtime_error(std::string("CUDA error: cudaGetSymbolAddress of the point scratch failed: ") +
                               cudaGetErrorString(e));
    }
    addr[device] = p;
    ready[device] = true;
  }
  return addr[device];
}

// The point-evaluation kernel reading the index bits as the caller's 0/1
// doubles (the same warp routine as the allocating path, which reads bytes).
// One warp per point; its two scratch rows sit in the shared array.
__global__ void eval_points_flags_kernel(Chain f, int npts, const double* flags, int max_bond, double* out,
                                         double* work) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= npts) return;
  double* v = work + (size_t)warp * 2 * max_bond;
  const double* fl = flags + (size_t)warp * f.n;
  const double val = eval_point_warp(f, [fl](int n) { return fl[n] != 0.0; }, v, v + max_bond);
  if (lane == 0) out[warp] = val;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

size_t Engine::points_noalloc_capacity() const {
  // per point: its value, its N flags and two scratch rows of the largest
  // bond of the context; three 256-byte alignment paddings are reserved
  const size_t per = 8 + 8 * (size_t)N_ + 16 * (size_t)max_bond_;
  const size_t usable = kPointsScratchBytes - 3 * 256;
  return usable / per;
}

void Engine::points_noalloc(double* inout, int npts) {
  if (npts <= 0) return;
  const size_t cap = points_noalloc_capacity();
  if ((size_t)npts > cap)
    throw std::runtime_error("EINVAL: " + std::to_string(npts) + " points exceed the fixed scratch of the "
                             "allocation-free evaluation (at most " + std::to_string(cap) +
                             " points for this context: 8 + 8 N + 16 x its largest bond (" + std::to_string(max_bond_) + ") bytes "
                             "each in a 4 MiB shared array)");
  int device = 0;
  if (cudaGetDevice(&device) != cudaSuccess) {
    cudaGetLastError();
    throw std::runtime_error("CUDA error: cudaGetDevice failed");
  }
  unsigned char* base = (unsigned char*)scratch_address(device);
  double* vals = (double*)base;
  double* flags = (double*)(base + align256((size_t)npts * 8));
  double* work = (double*)((unsigned char*)flags + align256((size_t)npts * N_ * 8));
  if (cudaMemcpyAsync(flags, inout, (size_t)npts * N_ * sizeof(double), cudaMemcpyHostToDevice, st_) != cudaSuccess)
    throw std::runtime_error("CUDA error: copy of the point query failed");
  const int warps_per_block = 8;
  count_launches(1);
  eval_points_flags_kernel<<<(npts + warps_per_block - 1) / warps_per_block, 32 * warps_per_block, 0, st_>>>(
      f_.chain(), npts, flags, max_bond_, vals, work);
  if (cudaGetLastError() != cudaSuccess) throw std::runtime_error("CUDA error: point evaluation launch failed");
  if (cudaMemcpyAsync(inout, vals, (size_t)npts * sizeof(double), cudaMemcpyDeviceToHost, st_) != cudaSuccess)
    throw std::runtime_error("CUDA error: copy of the point values failed");
  if (cudaStreamSynchronize(st_) != cudaSuccess) throw std::runtime_error("CUDA error: point evaluation failed");
}

}  // namespace qtt
