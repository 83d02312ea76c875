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

template <typename T>
struct LevelVecs {
  typename cplx<T>::type* r[AMAMG_MAX_LEVELS] = {};
  typename cplx<T>::type* e[AMAMG_MAX_LEVELS] = {};
};

// Bytes of scratch one V-cycle with R right-hand sides of element size cb needs.
size_t scratch_bytes(const amamg_ctx* h, int R, size_t cb) {
  size_t b = 0;
  for (size_t l = 1; l < h->lv.size(); ++l) b += 2 * align256((size_t)R * 2 * h->lv[l].n * cb);
  return b;
}

// The same kernels, in the same order and with the same arguments, as the
// V-cycle behind amamg_vcycle (Algorithm 1, start vector 0, no pre-smoothing,
// post_smooth sweeps), with the coarse vectors taken from the scratch array.
template <typename T>
cudaError_t vcycle_level(amamg_ctx* h, int l, const typename cplx<T>::type* r, typename cplx<T>::type* e,
                         const LevelVecs<T>& w, int R, cudaStream_t st) {
  constexpr bool f64 = sizeof(T) == 8;
  const int Lc = (int)h->lv.size() - 1;
  cudaError_t err;
  if (l == Lc) {
    if constexpr (f64) err = launch_dense_gemv<double2>(h->Ainv, r, e, h->nd, R, st);
    else err = launch_dense_gemv32(h->Ainv32, r, e, h->nd, R, st);
    h->launches++;
    return err;
  }
  const Level& L = h->lv[l];
  if constexpr (f64) err = launch_restrict<double, double2>(r, w.r[l + 1], L.P64, nullptr, L.Nx, L.a, L.Np, L.Nq, R, st);
  else err = launch_restrict<float, __half2>(r, w.r[l + 1], L.P16, L.Ps, L.Nx, L.a, L.Np, L.Nq, R, st);
  if (err != cudaSuccess) return err;
  h->launches++;
  err = vcycle_level<T>(h, l + 1, w.r[l + 1], w.e[l + 1], w, R, st);
  if (err != cudaSuccess) return err;
  const int sweeps = h->prm.post_smooth;
  if (l == 0 && sweeps > 0 && h->fine_fused) {
    // the same choice as the allocating V-cycle: prolongation and red-black
    // sweeps in one launch when a resident shape exists
    const T inv = (T)(1.0 / (h->m0 + 2.0));
    bool fused;
    if constexpr (f64) fused = fine_post_rows<double, double2>(L.Nt, L.Nx, L.a, R) > 0;
    else fused = fine_post_rows<float, __half2>(L.Nt, L.Nx, L.a, R) > 0;
    if (fused) {
      if constexpr (f64)
        err = launch_fine_post<double, double2>(w.e[l + 1], e, r, L.P64, nullptr, h->U64s, inv, nullptr, L.Nt, L.Nx,
                                                L.a, sweeps, R, h->d_owner_flags, h->d_sync, st);
      else
        err = launch_fine_post<float, __half2>(w.e[l + 1], e, r, L.P16, L.Ps, h->U32, inv, nullptr, L.Nt, L.Nx, L.a,
                                               sweeps, R, h->d_owner_flags, h->d_sync, st);
      h->launches++;
      return err;
    }
  }
  if constexpr (f64) err = launch_prolong<double, double2>(w.e[l + 1], e, L.P64, nullptr, L.Nx, L.a, L.Np, L.Nq, R, st);
  else err = launch_prolong<float, __half2>(w.e[l + 1], e, L.P16, L.Ps, L.Nx, L.a, L.Np, L.Nq, R, st);
  if (err != cudaSuccess) return err;
  h->launches++;
  if (l == 0) {
    const T inv = (T)(1.0 / (h->m0 + 2.0));
    const typename cplx<T>::type* U;
    if constexpr (f64) U = h->U64s; else U = h->U32;
    for (int s = 0; s < sweeps; ++s)
      for (int c = 0; c < 2; ++c) {
        err = launch_rb_half<T>(e, r, U, inv, L.Nt, L.Nx, c, R, st);
        if (err != cudaSuccess) return err;
        h->launches++;
      }
    return cudaSuccess;
  }
  const int kind = gs_kind_for<T>(L, R);
  if (sweeps > 0 && kind == GS_DSMEM) {
    const bool bsm = dsmem_blocks_in_smem<T>(L.n, L.off.K);
    if constexpr (f64)
      err = launch_coarse_sweeps_dsmem<double, double2>(e, r, L.Bc64, nullptr, L.Dc64, L.off, L.Nt, L.Nx, L.ncol,
                                                        sweeps, R, bsm, st);
    else
      err = launch_coarse_sweeps_dsmem<float, __half2>(e, r, L.Bc16, L.Bcs, L.Dc32, L.off, L.Nt, L.Nx, L.ncol, sweeps,
                                                       R, bsm, st);
    h->launches++;
    return err;
  }
  if (sweeps > 0 && kind == GS_OWNER) {
    if constexpr (f64)
      err = launch_coarse_sweeps_owner<double, double2>(e, r, L.Bc64, nullptr, L.Dc64, L.off, L.Nt, L.Nx, L.ncol,
                                                       sweeps, R, h->d_owner_flags, h->d_sync, st);
    else
      err = launch_coarse_sweeps_owner<float, __half2>(e, r, L.Bc16, L.Bcs, L.Dc32, L.off, L.Nt, L.Nx, L.ncol, sweeps,
                                                      R, h->d_owner_flags, h->d_sync, st);
    h->launches++;
    return err;
  }
  if (sweeps > 0 && kind == GS_GRID) {
    if constexpr (f64)
      err = launch_coarse_sweeps_grid<double, double2>(e, r, L.Bc64, nullptr, L.Dc64, L.off, L.Nt, L.Nx, L.ncol,
                                                       sweeps, R, h->d_sync, st);
    else
      err = launch_coarse_sweeps_grid<float, __half2>(e, r, L.Bc16, L.Bcs, L.Dc32, L.off, L.Nt, L.Nx, L.ncol, sweeps,
                                                      R, h->d_sync, st);
    h->launches++;
    return err;
  }
  if constexpr (!f64) {
    if (sweeps > 0 && kind == GS_CLUSTER && use_cluster_sweeps<T>(L.n, L.ncol)) {
      err = launch_coarse_sweeps_cluster<float, __half2>(e, r, L.Bc16, L.Bcs, L.Dc32, L.off, L.Nt, L.Nx, L.ncol, sweeps,
                                                         R, st);
      h->launches++;
      return err;
    }
  }
  for (int s = 0; s < sweeps; ++s)
    for (int c = 0; c < L.ncol; ++c) {
      if constexpr (f64)
        err = launch_coarse_colour<double, double2>(e, r, L.Bc64, nullptr, L.Dc64, L.off, L.Nt, L.Nx, L.ncol, c, R, st);
      else
        err = launch_coarse_colour<float, __half2>(e, r, L.Bc16, L.Bcs, L.Dc32, L.off, L.Nt, L.Nx, L.ncol, c, R, st);
      if (err != cudaSuccess) return err;
      h->launches++;
    }
  return cudaSuccess;
}

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
  LevelVecs<T> w;
  unsigned char* p = static_cast<unsigned char*>(base);
  for (size_t l = 1; l < h->lv.size(); ++l) {
    const size_t b = align256((size_t)R * 2 * h->lv[l].n * cb);
    w.r[l] = reinterpret_cast<typename cplx<T>::type*>(p);
    p += b;
    w.e[l] = reinterpret_cast<typename cplx<T>::type*>(p);
    p += b;
  }
  err = vcycle_level<T>(h, 0, static_cast<const typename cplx<T>::type*>(r), static_cast<typename cplx<T>::type*>(e),
                        w, R, st);
  if (err != cudaSuccess) {
    h->err = std::string("amamg_vcycle_noalloc: ") + cudaGetErrorString(err);
    return AMAMG_ERR_CUDA;
  }
  return AMAMG_OK;
}

}  // namespace

extern "C" int amamg_vcycle_noalloc(amamg_handle h, const void* r, void* e, int R, int precision, void* stream) {
  if (!h || !r || !e || R < 1) return AMAMG_ERR_INVALID_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (precision == AMAMG_F64) return vcycle_noalloc<double>(h, r, e, R, st);
  if (precision == AMAMG_F32) return vcycle_noalloc<float>(h, r, e, R, st);
  return AMAMG_ERR_INVALID_ARG;
}
