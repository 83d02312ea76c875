// Conjugate gradients on the normal equations, D^H D x = D^H psi (CGNR), the
// paper's unpreconditioned comparison solver (Sec. 5), with D^H = sigma_3 D
// sigma_3 (Eq. (6)).  Every step runs on the device in FP64:
//
//   w = D p,  alpha = ||z||^2 / ||w||^2,  x += alpha p,  r -= alpha w,
//   z' = D^H r,  beta = ||z'||^2 / ||z||^2,  p = z' + beta p
//
// (r = psi - D x carried by the recurrence, z = D^H r).  The scalars live in
// device memory, so a chunk of CG_CHUNK iterations is captured once as a CUDA
// graph and replayed; the host reads the per-right-hand-side flags after each
// chunk.  A right-hand side whose recursive ||r|| / ||psi|| reaches tol is
// frozen by its flag (the update kernels skip it); when all are frozen the
// true residual decides, and the recurrence restarts from it where it is not
// below tol.  Reductions are deterministic: per-block partial sums, added in a
// fixed order by the last block to finish (ticket).
#include <cmath>
#include <vector>

#include "context.h"

namespace {

constexpr int CG_THREADS = 256;
constexpr int CG_CHUNK = 20;          // iterations per captured graph (even: the zz parity returns to 0)
constexpr int CG_MAX_BLOCKS = 256;    // partial sums per right-hand side

// per right-hand side flags
constexpr int CG_RUNNING = 0;
constexpr int CG_CONVERGED = 1;       // recursive residual below tol (or p's image vanished)
constexpr int CG_OUT_OF_STEPS = 2;
constexpr int CG_NONFINITE = 3;

int cg_blocks(long len) {
  long nb = (len + 8 * CG_THREADS - 1) / (8 * CG_THREADS);
  return (int)(nb < 1 ? 1 : (nb > CG_MAX_BLOCKS ? CG_MAX_BLOCKS : nb));
}

__device__ __forceinline__ double block_sum(double v, double* sh) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  if (wid == 0) {
    v = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  }
  return v;
}

// Last block of right-hand side r to arrive (ticket) adds the partials in
// block order; returns true in that block's thread 0 with the sum in *total.
__device__ __forceinline__ bool last_block_total(double mine, double* __restrict__ partial,
                                                 unsigned* __restrict__ tickets, int r, double* total) {
  __shared__ bool last;
  if (threadIdx.x == 0) {
    partial[(size_t)r * CG_MAX_BLOCKS + blockIdx.x] = mine;
    __threadfence();
    const unsigned t = atomicAdd(tickets + r, 1u);
    last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return false;
  if (threadIdx.x == 0) {
    __threadfence();
    double s = 0.0;
    for (int b = 0; b < (int)gridDim.x; ++b) s += __ldcg(partial + (size_t)r * CG_MAX_BLOCKS + b);
    *total = s;
    tickets[r] = 0;                   // re-armed for the next kernel
  }
  return threadIdx.x == 0;
}

// out[r] = ||v_r||^2
__global__ void __launch_bounds__(CG_THREADS)
k_cg_norm2(const double2* __restrict__ v, long len, double* __restrict__ out, double* __restrict__ partial,
           unsigned* __restrict__ tickets) {
  __shared__ double sh[32];
  const int r = blockIdx.y;
  const double2* a = v + (size_t)r * len;
  double acc = 0.0;
  for (long k = (long)blockIdx.x * blockDim.x + threadIdx.x; k < len; k += (long)gridDim.x * blockDim.x)
    acc += cabs2(a[k]);
  acc = block_sum(acc, sh);
  double tot;
  if (last_block_total(acc, partial, tickets, r, &tot)) out[r] = tot;
}

// x += alpha p, r -= alpha w with alpha = zz[r] / ww[r]; rr[r] = ||r||^2 and the
// flag update (iteration count, convergence, step budget, non-finite values).
// Skipped entirely for right-hand sides whose flag is set.
__global__ void __launch_bounds__(CG_THREADS)
k_cg_update_xr(double2* __restrict__ x, double2* __restrict__ rv, const double2* __restrict__ p,
               const double2* __restrict__ w, long len, const double* __restrict__ zz, const double* __restrict__ ww,
               double* __restrict__ rr, const double* __restrict__ bb, double tol2, int max_iter,
               int* __restrict__ flag, int* __restrict__ iters, double* __restrict__ partial,
               unsigned* __restrict__ tickets) {
  __shared__ double sh[32];
  const int r = blockIdx.y;
  if (flag[r] != CG_RUNNING) return;          // read before any block of r can change it
  const double wn = ww[r];
  const double alpha = wn > 0.0 ? zz[r] / wn : 0.0;
  const size_t o = (size_t)r * len;
  double acc = 0.0;
  for (long k = (long)blockIdx.x * blockDim.x + threadIdx.x; k < len; k += (long)gridDim.x * blockDim.x) {
    x[o + k] += alpha * p[o + k];
    const double2 rn = rv[o + k] - alpha * w[o + k];
    rv[o + k] = rn;
    acc += cabs2(rn);
  }
  acc = block_sum(acc, sh);
  double tot;
  if (last_block_total(acc, partial, tickets, r, &tot)) {
    rr[r] = tot;
    if (!(wn > 0.0)) {                         // p has no image: nothing left to minimise
      flag[r] = isfinite(wn) ? CG_CONVERGED : CG_NONFINITE;
      return;
    }
    const int it = iters[r] + 1;
    iters[r] = it;
    if (!isfinite(tot)) flag[r] = CG_NONFINITE;
    else if (tot <= tol2 * bb[r]) flag[r] = CG_CONVERGED;
    else if (it >= max_iter) flag[r] = CG_OUT_OF_STEPS;
  }
}

// p = z + (zz_new / zz_old) p, skipped for right-hand sides whose flag is set
__global__ void __launch_bounds__(CG_THREADS)
k_cg_update_p(double2* __restrict__ p, const double2* __restrict__ z, long len, const double* __restrict__ zz_old,
              const double* __restrict__ zz_new, const int* __restrict__ flag) {
  const int r = blockIdx.y;
  if (flag[r] != CG_RUNNING) return;
  const double zo = zz_old[r];
  const double beta = zo > 0.0 ? zz_new[r] / zo : 0.0;
  const size_t o = (size_t)r * len;
  for (long k = (long)blockIdx.x * blockDim.x + threadIdx.x; k < len; k += (long)gridDim.x * blockDim.x)
    p[o + k] = z[o + k] + beta * p[o + k];
}

// after the true residual: p = z, flags from rr = ||psi - D x||^2 (a right-hand
// side below tol is done, one out of steps or non-finite stays so, the others
// run again)
__global__ void k_cg_restart_flags(const double* __restrict__ rr, const double* __restrict__ bb, double tol2,
                                   int max_iter, const int* __restrict__ iters, int* __restrict__ flag, int R) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= R) return;
  const double t = rr[r];
  if (!isfinite(t) || !isfinite(bb[r])) flag[r] = CG_NONFINITE;
  else if (t <= tol2 * bb[r]) flag[r] = CG_CONVERGED;
  else if (iters[r] >= max_iter) flag[r] = CG_OUT_OF_STEPS;
  else flag[r] = CG_RUNNING;
}

struct CgWork {
  int R = 0;
  long len = 0;
  double2 *r = nullptr, *p = nullptr, *w = nullptr, *z = nullptr;
  double *zz = nullptr, *ww = nullptr, *rr = nullptr, *bb = nullptr, *partial = nullptr;
  unsigned* tickets = nullptr;
  int *flag = nullptr, *iters = nullptr;
  cudaGraphExec_t chunk = nullptr;
  long long chunk_kernels = 0;
  void release() {
    if (chunk) cudaGraphExecDestroy(chunk);
    chunk = nullptr;
    for (void* q : {(void*)r, (void*)p, (void*)w, (void*)z, (void*)zz, (void*)ww, (void*)rr, (void*)bb,
                    (void*)partial, (void*)tickets, (void*)flag, (void*)iters})
      if (q) cudaFree(q);
    r = p = w = z = nullptr;
    zz = ww = rr = bb = partial = nullptr;
    tickets = nullptr;
    flag = iters = nullptr;
  }
};

#define CG_CK(call)                                                            \
  do {                                                                        \
    cudaError_t e_ = (call);                                                  \
    if (e_ != cudaSuccess) {                                                  \
      h->err = std::string("cgnr: ") + #call + ": " + cudaGetErrorString(e_); \
      return e_ == cudaErrorMemoryAllocation ? AMAMG_ERR_OOM : AMAMG_ERR_CUDA; \
    }                                                                         \
  } while (0)

int cg_alloc(amamg_ctx* h, CgWork& wk, int R, long len) {
  const size_t nv = (size_t)R * len;
  CG_CK(cudaMalloc((void**)&wk.r, nv * sizeof(double2)));
  CG_CK(cudaMalloc((void**)&wk.p, nv * sizeof(double2)));
  CG_CK(cudaMalloc((void**)&wk.w, nv * sizeof(double2)));
  CG_CK(cudaMalloc((void**)&wk.z, nv * sizeof(double2)));
  CG_CK(cudaMalloc((void**)&wk.zz, 2 * (size_t)R * sizeof(double)));
  CG_CK(cudaMalloc((void**)&wk.ww, (size_t)R * sizeof(double)));
  CG_CK(cudaMalloc((void**)&wk.rr, (size_t)R * sizeof(double)));
  CG_CK(cudaMalloc((void**)&wk.bb, (size_t)R * sizeof(double)));
  CG_CK(cudaMalloc((void**)&wk.partial, (size_t)R * CG_MAX_BLOCKS * sizeof(double)));
  CG_CK(cudaMalloc((void**)&wk.tickets, (size_t)R * sizeof(unsigned)));
  CG_CK(cudaMalloc((void**)&wk.flag, (size_t)R * sizeof(int)));
  CG_CK(cudaMalloc((void**)&wk.iters, (size_t)R * sizeof(int)));
  CG_CK(cudaMemset(wk.tickets, 0, (size_t)R * sizeof(unsigned)));
  CG_CK(cudaMemset(wk.iters, 0, (size_t)R * sizeof(int)));
  wk.R = R;
  wk.len = len;
  return AMAMG_OK;
}

// (Re)start: r = psi - D x, rr, flags, z = D^H r, zz[0] = ||z||^2, p = z.
int cg_restart(amamg_ctx* h, CgWork& wk, const double2* psi, double2* x, double tol2, int max_iter,
               cudaStream_t st) {
  const Level& F = h->lv[0];
  const int R = wk.R;
  const long len = wk.len;
  const dim3 g(cg_blocks(len), R);
  const double diag = h->m0 + 2.0;
  CG_CK((launch_dslash<double2, double2, double>(x, wk.r, psi, h->U64s, diag, F.Nt, F.Nx, R, st)));
  k_cg_norm2<<<g, CG_THREADS, 0, st>>>(wk.r, len, wk.rr, wk.partial, wk.tickets);
  CG_CK(cudaGetLastError());
  k_cg_restart_flags<<<(R + 127) / 128, 128, 0, st>>>(wk.rr, wk.bb, tol2, max_iter, wk.iters, wk.flag, R);
  CG_CK(cudaGetLastError());
  CG_CK(launch_dslash_dag(wk.r, wk.z, h->U64s, diag, F.Nt, F.Nx, R, st));
  k_cg_norm2<<<g, CG_THREADS, 0, st>>>(wk.z, len, wk.zz, wk.partial, wk.tickets);
  CG_CK(cudaGetLastError());
  CG_CK(cudaMemcpyAsync(wk.p, wk.z, (size_t)R * len * sizeof(double2), cudaMemcpyDeviceToDevice, st));
  h->launches += 6;
  return AMAMG_OK;
}

// CG_CHUNK iterations (parity of zz alternating, starting at 0)
int cg_chunk(amamg_ctx* h, CgWork& wk, double2* x, double tol2, int max_iter, cudaStream_t st) {
  const Level& F = h->lv[0];
  const int R = wk.R;
  const long len = wk.len;
  const dim3 g(cg_blocks(len), R);
  const double diag = h->m0 + 2.0;
  for (int k = 0; k < CG_CHUNK; ++k) {
    double* zo = wk.zz + (size_t)(k & 1) * R;
    double* zn = wk.zz + (size_t)((k + 1) & 1) * R;
    CG_CK((launch_dslash<double2, double2, double>(wk.p, wk.w, nullptr, h->U64s, diag, F.Nt, F.Nx, R, st)));
    k_cg_norm2<<<g, CG_THREADS, 0, st>>>(wk.w, len, wk.ww, wk.partial, wk.tickets);
    CG_CK(cudaGetLastError());
    k_cg_update_xr<<<g, CG_THREADS, 0, st>>>(x, wk.r, wk.p, wk.w, len, zo, wk.ww, wk.rr, wk.bb, tol2, max_iter,
                                             wk.flag, wk.iters, wk.partial, wk.tickets);
    CG_CK(cudaGetLastError());
    CG_CK(launch_dslash_dag(wk.r, wk.z, h->U64s, diag, F.Nt, F.Nx, R, st));
    k_cg_norm2<<<g, CG_THREADS, 0, st>>>(wk.z, len, zn, wk.partial, wk.tickets);
    CG_CK(cudaGetLastError());
    k_cg_update_p<<<g, CG_THREADS, 0, st>>>(wk.p, wk.z, len, zo, zn, wk.flag);
    CG_CK(cudaGetLastError());
  }
  return AMAMG_OK;
}

int cgnr_on(amamg_ctx* h, const double2* psi, double2* x, int R, int max_iter, double tol, cudaStream_t st,
            amamg_solve_info* info) {
  const long len = 2L * h->lv[0].n;
  CgWork wk;
  int rc = cg_alloc(h, wk, R, len);
  const double tol2 = tol * tol;
  std::vector<int> flag(R), iters(R);
  std::vector<double> rr(R), bb(R);
  if (rc == AMAMG_OK) {
    const dim3 g(cg_blocks(len), R);
    cudaMemsetAsync(x, 0, (size_t)R * len * sizeof(double2), st);
    k_cg_norm2<<<g, CG_THREADS, 0, st>>>(psi, len, wk.bb, wk.partial, wk.tickets);
    h->launches++;
    rc = cudaGetLastError() == cudaSuccess ? AMAMG_OK : AMAMG_ERR_CUDA;
  }
  if (rc == AMAMG_OK) rc = cg_restart(h, wk, psi, x, tol2, max_iter, st);
  // capture one chunk as a graph (eager launches while kernel profiling is on)
  if (rc == AMAMG_OK && h->use_graphs) {
    cudaGraph_t gr = nullptr;
    const long long l0 = h->launches;
    if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) rc = AMAMG_ERR_CUDA;
    if (rc == AMAMG_OK) {
      const int rc2 = cg_chunk(h, wk, x, tol2, max_iter, st);
      const cudaError_t ec = cudaStreamEndCapture(st, &gr);
      if (rc2 != AMAMG_OK || ec != cudaSuccess) rc = rc2 != AMAMG_OK ? rc2 : AMAMG_ERR_CUDA;
    }
    if (rc == AMAMG_OK && cudaGraphInstantiate(&wk.chunk, gr, 0) != cudaSuccess) rc = AMAMG_ERR_CUDA;
    if (gr) cudaGraphDestroy(gr);
    h->launches = l0;
    wk.chunk_kernels = 6LL * CG_CHUNK;
  }
  while (rc == AMAMG_OK) {
    if (wk.chunk) {
      if (cudaGraphLaunch(wk.chunk, st) != cudaSuccess) { rc = AMAMG_ERR_CUDA; break; }
      h->launches += wk.chunk_kernels;
    } else {
      rc = cg_chunk(h, wk, x, tol2, max_iter, st);
      h->launches += 6LL * CG_CHUNK;
      if (rc != AMAMG_OK) break;
    }
    if (cudaMemcpyAsync(flag.data(), wk.flag, R * sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
      rc = AMAMG_ERR_CUDA;
      break;
    }
    bool running = false;
    for (int r = 0; r < R; ++r) running |= flag[r] == CG_RUNNING;
    if (running) continue;
    // every right-hand side stopped: the true residual decides
    rc = cg_restart(h, wk, psi, x, tol2, max_iter, st);
    if (rc != AMAMG_OK) break;
    if (cudaMemcpyAsync(flag.data(), wk.flag, R * sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
      rc = AMAMG_ERR_CUDA;
      break;
    }
    running = false;
    for (int r = 0; r < R; ++r) running |= flag[r] == CG_RUNNING;
    if (!running) break;
  }
  if (rc == AMAMG_OK) {
    if (cudaMemcpyAsync(iters.data(), wk.iters, R * sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(rr.data(), wk.rr, R * sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(bb.data(), wk.bb, R * sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      rc = AMAMG_ERR_CUDA;
  }
  if (rc == AMAMG_ERR_CUDA && h->err.empty()) h->err = std::string("cgnr: ") + cudaGetErrorString(cudaGetLastError());
  int out = rc;
  if (rc == AMAMG_OK) {
    bool nonfinite = false;
    for (int r = 0; r < R; ++r) {
      const int s = flag[r] == CG_CONVERGED ? AMAMG_OK
                  : flag[r] == CG_OUT_OF_STEPS ? AMAMG_NOT_CONVERGED : AMAMG_ERR_NONFINITE;
      if (info) {
        info[r].iterations = iters[r];
        info[r].status = s;
        info[r].true_relres = bb[r] > 0.0 ? std::sqrt(rr[r] / bb[r]) : 0.0;
      }
      if (s == AMAMG_NOT_CONVERGED && out == AMAMG_OK) out = AMAMG_NOT_CONVERGED;
      if (s == AMAMG_ERR_NONFINITE) nonfinite = true;
    }
    if (nonfinite) {
      h->err = "cgnr: non-finite value in a right-hand side or residual";
      out = AMAMG_ERR_NONFINITE;
    }
  }
  cudaStreamSynchronize(st);
  wk.release();
  return out;
}

}  // namespace

extern "C" int amamg_cgnr(amamg_handle h, const void* psi, void* x, int R, int max_iter, double tol, void* stream,
                          amamg_solve_info* info) {
  if (!h || !psi || !x || R < 1 || max_iter < 1 || !(tol > 0.0)) return AMAMG_ERR_INVALID_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  // on the handle's own stream (graph capture needs a non-default stream),
  // ordered after the caller's stream and before what it enqueues next
  if (cudaEventRecord(h->ev_in, st) != cudaSuccess || cudaStreamWaitEvent(h->ws, h->ev_in, 0) != cudaSuccess)
    return AMAMG_ERR_CUDA;
  h->err.clear();
  const int rc = cgnr_on(h, static_cast<const double2*>(psi), static_cast<double2*>(x), R, max_iter, tol, h->ws, info);
  if (cudaEventRecord(h->ev_out, h->ws) != cudaSuccess || cudaStreamWaitEvent(st, h->ev_out, 0) != cudaSuccess)
    return AMAMG_ERR_CUDA;
  return rc;
}

extern "C" int amamg_apply_Ddag(amamg_handle h, const void* in, void* out, int R, void* stream) {
  if (!h || !in || !out || R < 1) return AMAMG_ERR_INVALID_ARG;
  const Level& F = h->lv[0];
  const cudaError_t e = launch_dslash_dag(static_cast<const double2*>(in), static_cast<double2*>(out), h->U64s,
                                          h->m0 + 2.0, F.Nt, F.Nx, R, reinterpret_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) {
    h->err = std::string("amamg_apply_Ddag: ") + cudaGetErrorString(e);
    return AMAMG_ERR_CUDA;
  }
  h->launches++;
  return AMAMG_OK;
}
