// Point evaluation of the PDF without any allocation.
//
// qtt_observe(..., QTT_OBS_POINTS, ...) allocates device buffers for the
// query and its scratch on every call and frees them afterwards.  Some
// callers cannot allow that: code running while a CUDA stream is being
// captured into a graph (allocation is not permitted there), monitoring loops
// that probe the PDF every step and must not pay the implicit device-wide
// synchronisation of cudaFree, and processes whose device memory is entirely
// reserved by their own pool.  qtt_observe_points_noalloc serves them: the
// query flags, the per-point scratch vectors and the results live in one
// file-scope device array of fixed size, so the call performs no cudaMalloc,
// cudaFree or other allocating routine.
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

// The host-side name g_points_scratch is only a stand-in symbol; the device
// address of the array is looked up once per device (with that device
// current) and cached.
void* scratch_address(int device) {
  static std::mutex mu;
  static void* addr[kMaxSites] = {nullptr};
  static bool ready[kMaxSites] = {false};
  if (device < 0 || device >= kMaxSites) throw std::runtime_error("EINVAL: device ordinal out of range");
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

// Variant of the point-evaluation kernel that reads the index bits as the
// caller's 0/1 doubles.  One warp per point; the running row vector (and its
// double buffer) sits in the scratch.  Every entry a warp reads has been
// written by it first (v[0] before the first site, then v[0..br) per site),
// so the scratch needs no clearing between calls.
__global__ void eval_points_flags_kernel(Chain f, int npts, const double* flags, int max_bond, double* out,
                                         double* work) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= npts) return;
  double* v = work + (size_t)warp * 2 * max_bond;
  double* v2 = v + max_bond;
  if (lane == 0) v[0] = 1.0;
  __syncwarp();
  for (int n = 0; n < f.n; ++n) {
    const int bl = f.bond[n], br = f.bond[n + 1];
    const int s = flags[(size_t)warp * f.n + n] != 0.0 ? 1 : 0;
    const double* A = f.core[n];
    for (int c = lane; c < br; c += 32) {
      double acc = 0.0;
      for (int b = 0; b < bl; ++b) acc += v[b] * A[((size_t)b * 2 + s) * br + c];
      v2[c] = acc;
    }
    __syncwarp();
    for (int c = lane; c < br; c += 32) v[c] = v2[c];
    __syncwarp();
  }
  if (lane == 0) out[warp] = v[0];
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

size_t Engine::points_noalloc_capacity() const {
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
                             " points for this grid and chi_max; 4 MiB shared array)");
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
