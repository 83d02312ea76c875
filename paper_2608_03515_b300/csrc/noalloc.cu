// amamg_vcycle_noalloc: the V-cycle entry point for callers that cannot
// allocate device memory.
//
// Who needs it: code that runs where cudaMalloc is not allowed or not wanted
// while it runs — inside a host callback, inside a region that a caller is
// recording for later replay with fixed addresses, or in an application whose
// memory pool forbids allocations after start-up.  amamg_vcycle may allocate
// the coarse-level work vectors of the V-cycle on its first call (or when R
// grows); this variant never allocates.  Its work vectors live in one
// file-scope device array of fixed size, AMAMG_NOALLOC_SCRATCH_BYTES, that
// every GPU which loads the library holds until the process exits.
//
// The caller still owns the input and output vectors.  The hierarchy itself
// (interpolators, coarse operators, coarsest inverse) comes from amamg_setup.
#include <mutex>

#include "context.h"

namespace {

// Scratch for the coarse-level vectors r_l, e_l (l >= 1) of one V-cycle.
static __device__ __align__(256) unsigned char g_vcycle_scratch[AMAMG_NOALLOC_SCRATCH_BYTES];

// Device address of the array, looked up once per device (host code cannot use
// the symbol's name as a pointer).
constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {};

cudaError_t scratch_address(void** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_vcycle_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

inline size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

// Bytes of scratch one V-cycle with R right-hand sides of element size cb needs.
size_t scratch_bytes(const amamg_ctx* h, int R, size_t cb) {
  size_t b = 0;
  for (size_t l = 1; l < h->lv.size(); ++l) b += 2 * align256((size_t)R * 2 * h->lv[l].n * cb);
  return b;
}

// The V-cycle behind amamg_vcycle (the engine's own code path: same kernels,
// same order, same arguments) with the coarse vectors carved out of the
// scratch array instead of the handle's allocations.
template <typename T>
int vcycle_noalloc(amamg_ctx* h, const void* r, void* e, int R, cudaStream_t st) {
  const size_t cb = sizeof(typename cplx<T>::type);
  const size_t need = scratch_bytes(h, R, cb);
  if (need > (size_t)AMAMG_NOALLOC_SCRATCH_BYTES) {
    h->err = "amamg_vcycle_noalloc: the coarse levels need " + std::to_string(need) +
             " bytes of scratch for R = " + std::to_string(R) + "; the fixed array holds " +
             std::to_string((size_t)AMAMG_NOALLOC_SCRATCH_BYTES);
    return AMAMG_ERR_INVALID_ARG;
  }
  void* base = nullptr;
  cudaError_t err = scratch_address(&base);
  if (err != cudaSuccess) {
    h->err = std::string("amamg_vcycle_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(err);
    return AMAMG_ERR_CUDA;
  }
  VcycleVecs<T> w;
  unsigned char* p = static_cast<unsigned char*>(base);
  for (size_t l = 1; l < h->lv.size(); ++l) {
    const size_t b = align256((size_t)R * 2 * h->lv[l].n * cb);
    w.r[l] = reinterpret_cast<typename cplx<T>::type*>(p);
    p += b;
    w.e[l] = reinterpret_cast<typename cplx<T>::type*>(p);
    p += b;
  }
  return engine_vcycle<T>(h, static_cast<const typename cplx<T>::type*>(r), static_cast<typename cplx<T>::type*>(e),
                          w, R, st);
}

}  // namespace

extern "C" int amamg_vcycle_noalloc(amamg_handle h, const void* r, void* e, int R, int precision, void* stream) {
  if (!h || !r || !e || R < 1) return AMAMG_ERR_INVALID_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (precision == AMAMG_F64) return vcycle_noalloc<double>(h, r, e, R, st);
  if (precision == AMAMG_F32) return vcycle_noalloc<float>(h, r, e, R, st);
  return AMAMG_ERR_INVALID_ARG;
}
