// Allocation-free variant of the forward transform (no counterpart in the paper).
//
// Some callers cannot call cudaMalloc at the time they transform a field: code
// running inside another framework's CUDA-graph capture (where device allocation
// is not permitted), or hosts that freeze their device-memory budget after start-up
// and route every allocation through their own pool.  mlx_forward_noalloc serves
// them: it performs exactly the work of mlx_forward, but the intermediate Fourier
// coefficients (the phi-transformed and z-transformed planes between the FFT
// kernels and the Legendre contraction) live in the file-scope device array below
// instead of the context's workspace.  It calls no cudaMalloc, cudaFree or other
// allocating routine.
//
// The array has a fixed size (kScratchBytes) and exists on every GPU that loads
// this library until the process exits.  In host code `g_noalloc_scratch` is only
// a host-side stand-in for the symbol, not a device address; its device address is
// looked up once per device with cudaGetSymbolAddress, with that device current,
// on the first call made on that device (under a lock, so that host threads making
// their first calls together look it up once).  Make that first call before any
// stream capture begins.  The cached address belongs to the device's primary
// context: like every context of this library, it does not survive
// cudaDeviceReset.  Every call on a device shares the one array and leaves the last
// call's contents behind; the kernels overwrite every element they later read, so
// nothing needs clearing.  Calls whose work overlaps on the GPU (different streams,
// or different contexts on the same device) race on the array: serialise them.
#include "mlx_internal.cuh"

#include <atomic>
#include <mutex>

namespace {

constexpr size_t kScratchBytes = (size_t)16 << 20;   // 16 MiB
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::atomic<void*> g_scratch_addr[kMaxDevices];
std::mutex g_scratch_lock;

size_t round256(size_t b) { return (b + 255) / 256 * 256; }

}  // namespace

extern "C" int mlx_forward_noalloc(mlx_ctx* c, const void* phys, void* spec, mlx_stream stream) {
  if (!c || !phys || !spec) return MLX_EINVAL;
  if ((((uintptr_t)phys) & 15u) || (((uintptr_t)spec) & 15u)) return MLX_EINVAL;
  const size_t es = elem_size(c->precision);
  const size_t mixed_b = round256(es * 2 * (size_t)c->K * c->M * c->nr);
  const size_t zm_b = c->nz > 1 ? round256(es * 2 * (size_t)c->nz * c->M * c->nr) : 0;
  if (mixed_b + zm_b > kScratchBytes) {
    c->last_err = "mlx_forward_noalloc: this grid needs " + std::to_string(mixed_b + zm_b) +
                  " bytes of scratch, above the fixed limit of " + std::to_string(kScratchBytes) +
                  " bytes; use mlx_forward";
    return MLX_EINVAL;
  }
  int dev = 0;
  MLX_CUDA_TRY(c, cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) {
    c->last_err = "mlx_forward_noalloc: device ordinal " + std::to_string(dev) + " is beyond the " +
                  std::to_string(kMaxDevices) + " devices this entry point supports";
    return MLX_EINVAL;
  }
  void* addr = g_scratch_addr[dev].load(std::memory_order_acquire);
  if (!addr) {
    std::lock_guard<std::mutex> lock(g_scratch_lock);
    addr = g_scratch_addr[dev].load(std::memory_order_relaxed);
    if (!addr) {
      MLX_CUDA_TRY(c, cudaGetSymbolAddress(&addr, g_noalloc_scratch));
      g_scratch_addr[dev].store(addr, std::memory_order_release);
    }
  }
  unsigned char* base = static_cast<unsigned char*>(addr);
  // run the forward transform's kernels with the workspace pointers redirected
  void* saved_mixed = c->d_mixed;
  void* saved_zm = c->d_zm;
  c->d_mixed = base;
  c->d_zm = c->nz > 1 ? base + mixed_b : nullptr;
  cudaStream_t st = (cudaStream_t)stream;
  int rc = mlx_fft_forward(c, phys, st);
  if (!rc) rc = mlx_legendre_forward(c, (double2*)spec, st);
  c->d_mixed = saved_mixed;
  c->d_zm = saved_zm;
  return rc;
}
