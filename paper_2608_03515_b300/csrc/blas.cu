// Krylov vector kernels of the FP64 outer FGMRES (Gram-Schmidt inner products,
// multi-vector updates, norms, scaling) and precision casts.
//
// A basis is one allocation [J][R][len] (vector i of right-hand side r at
// base + (i*R + r)*len).  Inner products are two-pass and deterministic: each
// block writes a partial sum, a second kernel adds the partials in a fixed tree
// order.  len counts complex elements.
#include "kernels.h"

namespace {

constexpr int DOT_THREADS = 256;

template <typename C>
__device__ __forceinline__ C block_reduce(C v, C* sh) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
    v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
  }
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  const int nw = blockDim.x >> 5;
  if (wid == 0) {
    v = lane < nw ? sh[lane] : czero<C>();
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
      v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
    }
  }
  return v;
}

// partial[(r*Jt + i)*nb + blk] = sum over the block's chunk of conj(V_i,r) w_r for
// i < J, and conj(w_r) w_r for i == J when the grid has J + 1 rows (Jt = gridDim.y).
// gate (optional): per right-hand side flag; a block whose flag is 0 does nothing.
__global__ void __launch_bounds__(DOT_THREADS)
k_dots(const double2* __restrict__ V, size_t vi, size_t vr, const double2* __restrict__ w, size_t wr,
       long len, long chunk, double2* __restrict__ partial, int J, const int* __restrict__ gate) {
  __shared__ double2 sh[32];
  const int i = blockIdx.y, r = blockIdx.z, nb = gridDim.x, Jt = gridDim.y;
  if (gate && gate[r] == 0) return;
  const double2* a = (i < J) ? V + i * vi + r * vr : w + r * wr;
  const double2* b = w + r * wr;
  const long start = (long)blockIdx.x * chunk;
  const long end = min(start + chunk, len);
  double2 acc = make_double2(0.0, 0.0);
  for (long k = start + threadIdx.x; k < end; k += blockDim.x) cmacc(acc, a[k], b[k]);
  acc = block_reduce(acc, sh);
  if (threadIdx.x == 0) partial[((size_t)r * Jt + i) * nb + blockIdx.x] = acc;
}

// out[r*ldo + off + i] = sum_b partial[(r*J + i)*nb + b]
// mode 0: store the complex sum (0 for a right-hand side whose gate flag is 0);
// mode 1: the sum is <w, w>: store sqrt(re) in out and 1/sqrt(re) (0 when the
//   norm is 0) in inv; with a gate, only where the flag is set;
// mode 2: as mode 1, and set flag[r] = (<w, w> < eta^2 * ref) where ref =
//   out[r*ldo + ref_off].x is the squared norm before the first Gram-Schmidt
//   pass (DGKS criterion for a second pass).
__global__ void __launch_bounds__(256)
k_reduce_partials(const double2* __restrict__ partial, int nb, int J, double2* __restrict__ out, int ldo,
                  int off, int mode, double* __restrict__ inv, int* __restrict__ flag, int ref_off, double eta2) {
  __shared__ double2 sh[32];
  const int i = blockIdx.x, r = blockIdx.y;
  const bool gated = flag && mode != 2 && flag[r] == 0;
  if (gated) {
    if (threadIdx.x == 0 && mode == 0) out[(size_t)r * ldo + off + i] = make_double2(0.0, 0.0);
    return;
  }
  const double2* p = partial + ((size_t)r * J + i) * nb;
  double2 acc = make_double2(0.0, 0.0);
  for (int b = threadIdx.x; b < nb; b += blockDim.x) acc += p[b];
  acc = block_reduce(acc, sh);
  if (threadIdx.x == 0) {
    if (mode == 0) {
      out[(size_t)r * ldo + off + i] = acc;
    } else {
      // NaN propagates (a NaN or Inf entry must surface as a non-finite norm)
      const double nrm = (acc.x >= 0.0) ? sqrt(acc.x) : ((acc.x < 0.0) ? 0.0 : acc.x);
      out[(size_t)r * ldo + off + i] = make_double2(nrm, 0.0);
      if (inv) inv[r] = nrm > 0.0 ? 1.0 / nrm : 0.0;
      if (mode == 2) flag[r] = (acc.x < eta2 * out[(size_t)r * ldo + ref_off].x) ? 1 : 0;
    }
  }
}

// y_r += sign * sum_{i<J} coef[r*ldc + i] * X_{i,r}
template <typename Cx>
__global__ void __launch_bounds__(256)
k_multi_axpy(double2* __restrict__ y, size_t yr, const Cx* __restrict__ X, size_t xi, size_t xr,
             const double2* __restrict__ coef, int ldc, int J, double sign, long len, const int* __restrict__ gate) {
  const int r = blockIdx.y;
  if (gate && gate[r] == 0) return;
  const double2* c = coef + (size_t)r * ldc;
  for (long k = (long)blockIdx.x * blockDim.x + threadIdx.x; k < len; k += (long)gridDim.x * blockDim.x) {
    double2 acc = make_double2(0.0, 0.0);
    for (int i = 0; i < J; ++i) cmac(acc, c[i], to_c(X[i * xi + r * xr + k], double()));
    y[r * yr + k] += sign * acc;
  }
}

// dst_r = src_r * scale[r]   (scale from device memory)
template <typename Cd>
__global__ void __launch_bounds__(256)
k_scale_copy(Cd* __restrict__ dst, size_t dr, const double2* __restrict__ src, size_t sr,
             const double* __restrict__ scale, long len) {
  const int r = blockIdx.y;
  const double s = scale[r];
  for (long k = (long)blockIdx.x * blockDim.x + threadIdx.x; k < len; k += (long)gridDim.x * blockDim.x)
    dst[r * dr + k] = to_c(s * src[r * sr + k], typename real_of<Cd>::type());
}

// dst_r = src_r * scale[r], and its FP32 rounding in dst32_r
__global__ void __launch_bounds__(256)
k_scale_copy_dual(double2* __restrict__ dst, float2* __restrict__ dst32, size_t dr, const double2* __restrict__ src,
                  size_t sr, const double* __restrict__ scale, long len) {
  const int r = blockIdx.y;
  const double s = scale[r];
  for (long k = (long)blockIdx.x * blockDim.x + threadIdx.x; k < len; k += (long)gridDim.x * blockDim.x) {
    const double2 v = s * src[r * sr + k];
    dst[r * dr + k] = v;
    dst32[r * dr + k] = to_c(v, float());
  }
}

template <typename Cs, typename Cd>
__global__ void __launch_bounds__(256) k_cast(const Cs* __restrict__ src, Cd* __restrict__ dst, long len) {
  for (long k = (long)blockIdx.x * blockDim.x + threadIdx.x; k < len; k += (long)gridDim.x * blockDim.x)
    dst[k] = to_c(src[k], typename real_of<Cd>::type());
}

__device__ __forceinline__ double block_reduce_real(double v, double* sh) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  const int nw = blockDim.x >> 5;
  if (wid == 0) {
    v = lane < nw ? sh[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  }
  return v;
}

// Inner products with the reduction fused in: like k_dots, then the last block
// of each (row, RHS) to finish (atomic ticket after a fence) adds the partials
// in a fixed order, so the result is deterministic, writes it to
// out[r*ldo + off + i] and resets the ticket.  A right-hand side whose gate
// flag is 0 gets zeros.
__global__ void __launch_bounds__(DOT_THREADS)
k_dots_fused(const double2* __restrict__ V, size_t vi, size_t vr, const double2* __restrict__ w, size_t wr,
             long len, long chunk, double2* __restrict__ partial, int J, const int* __restrict__ gate,
             unsigned* __restrict__ tickets, double2* __restrict__ out, int ldo, int off) {
  __shared__ double2 sh[32];
  __shared__ bool last;
  const int i = blockIdx.y, r = blockIdx.z, nb = gridDim.x, Jt = gridDim.y;
  if (gate && gate[r] == 0) {
    if (blockIdx.x == 0 && threadIdx.x == 0) out[(size_t)r * ldo + off + i] = make_double2(0.0, 0.0);
    return;
  }
  const double2* a = (i < J) ? V + i * vi + r * vr : w + r * wr;
  const double2* b = w + r * wr;
  const long start = (long)blockIdx.x * chunk;
  const long end = min(start + chunk, len);
  double2 acc = make_double2(0.0, 0.0);
  for (long k = start + threadIdx.x; k < end; k += blockDim.x) cmacc(acc, a[k], b[k]);
  acc = block_reduce(acc, sh);
  const size_t slot = (size_t)r * Jt + i;
  if (threadIdx.x == 0) {
    partial[slot * nb + blockIdx.x] = acc;
    __threadfence();
    last = atomicAdd(&tickets[slot], 1u) == (unsigned)(nb - 1);
  }
  __syncthreads();
  if (last) {
    double2 t = make_double2(0.0, 0.0);
    for (int bb = threadIdx.x; bb < nb; bb += blockDim.x) t += __ldcg(&partial[slot * nb + bb]);
    t = block_reduce(t, sh);
    if (threadIdx.x == 0) {
      out[(size_t)r * ldo + off + i] = t;
      tickets[slot] = 0;
    }
  }
}

// y_r -= sum_{i<J} coef[r*ldc + i] X_{i,r}, and ||y_r|| of the result with the
// same last-block reduction: out[r*ldo + nrm_off] = ||y_r||, inv[r] = 1/||y_r||
// (0 for a zero vector); mode 2 also sets flag[r] = (||y_r||^2 < eta2 *
// out[r*ldo + ref_off].x) (the DGKS test against the norm before the pass).
// A right-hand side whose gate flag is 0 is left untouched.
__global__ void __launch_bounds__(256)
k_axpy_norm(double2* __restrict__ y, size_t yr, const double2* __restrict__ X, size_t xi, size_t xr,
            const double2* __restrict__ coef, int ldc, int J, long len, const int* __restrict__ gate,
            double* __restrict__ partial, unsigned* __restrict__ tickets, double2* __restrict__ out, int ldo,
            int nrm_off, double* __restrict__ inv, int* __restrict__ flag, int ref_off, double eta2, int mode) {
  __shared__ double sh[32];
  __shared__ bool last;
  const int r = blockIdx.y, nb = gridDim.x;
  if (gate && gate[r] == 0) return;
  const double2* c = coef + (size_t)r * ldc;
  double ss = 0.0;
  for (long k = (long)blockIdx.x * blockDim.x + threadIdx.x; k < len; k += (long)gridDim.x * blockDim.x) {
    double2 acc = make_double2(0.0, 0.0);
    for (int i = 0; i < J; ++i) cmac(acc, c[i], X[i * xi + r * xr + k]);
    const double2 v = y[r * yr + k] - acc;
    y[r * yr + k] = v;
    ss = fma(v.x, v.x, fma(v.y, v.y, ss));
  }
  ss = block_reduce_real(ss, sh);
  if (threadIdx.x == 0) {
    partial[(size_t)r * nb + blockIdx.x] = ss;
    __threadfence();
    last = atomicAdd(&tickets[r], 1u) == (unsigned)(nb - 1);
  }
  __syncthreads();
  if (last) {
    double t = 0.0;
    for (int bb = threadIdx.x; bb < nb; bb += blockDim.x) t += __ldcg(&partial[(size_t)r * nb + bb]);
    t = block_reduce_real(t, sh);
    if (threadIdx.x == 0) {
      // NaN propagates (a NaN or Inf entry must surface as a non-finite norm)
      const double nrm = (t >= 0.0) ? sqrt(t) : ((t < 0.0) ? 0.0 : t);
      out[(size_t)r * ldo + nrm_off] = make_double2(nrm, 0.0);
      inv[r] = nrm > 0.0 ? 1.0 / nrm : 0.0;
      if (mode == 2) flag[r] = (t < eta2 * out[(size_t)r * ldo + ref_off].x) ? 1 : 0;
      tickets[r] = 0;
    }
  }
}

// Stage i (0 <= i <= J) of modified Gram-Schmidt of w_r against v_0..v_{J-1}
// (the inner loop of the Arnoldi step in Saad's flexible GMRES): for i >= 1,
// w_r -= h_{i-1,r} v_{i-1,r} with the previous stage's coefficient; then for
// i < J the inner product h_{i,r} = v_{i,r}^H w_r, for i = J the norm ||w_r||,
// each with the fixed-order last-block reduction of k_dots_fused.  h_{i,r} goes
// to out[r*ldo + i] and a zero to out[r*ldo + off2 + i] (the second-pass slot
// that the least-squares step adds); the norm to out[r*ldo + nrm_off] and its
// inverse to inv[r].  One stage reads w and at most two basis vectors.
__global__ void __launch_bounds__(DOT_THREADS)
k_mgs_stage(double2* __restrict__ w, size_t wr, const double2* __restrict__ V, size_t vi, size_t vr, long len,
            long chunk, int i, int J, double2* __restrict__ partial, int pslots, unsigned* __restrict__ tickets,
            double2* __restrict__ out, int ldo, int off2, int nrm_off, double* __restrict__ inv) {
  __shared__ double2 sh[32];
  __shared__ double shr[32];
  __shared__ bool last;
  const int r = blockIdx.y, nb = gridDim.x;
  double2* y = w + r * wr;
  const double2 c = i >= 1 ? out[(size_t)r * ldo + i - 1] : make_double2(0.0, 0.0);
  const double2* vp = V + (size_t)(i >= 1 ? i - 1 : 0) * vi + r * vr;
  const double2* vn = V + (size_t)(i < J ? i : 0) * vi + r * vr;
  const long start = (long)blockIdx.x * chunk;
  const long end = min(start + chunk, len);
  double2 acc = make_double2(0.0, 0.0);
  double ss = 0.0;
  for (long k = start + threadIdx.x; k < end; k += blockDim.x) {
    double2 yk = y[k];
    if (i >= 1) {
      double2 t = make_double2(0.0, 0.0);
      cmac(t, c, vp[k]);
      yk = yk - t;
      y[k] = yk;
    }
    if (i < J) cmacc(acc, vn[k], yk);
    else ss = fma(yk.x, yk.x, fma(yk.y, yk.y, ss));
  }
  const size_t slot = (size_t)r * pslots + i;
  if (i < J) {
    acc = block_reduce(acc, sh);
  } else {
    ss = block_reduce_real(ss, shr);
    acc = make_double2(ss, 0.0);
  }
  if (threadIdx.x == 0) {
    partial[slot * nb + blockIdx.x] = acc;
    __threadfence();
    last = atomicAdd(&tickets[slot], 1u) == (unsigned)(nb - 1);
  }
  __syncthreads();
  if (last) {
    double2 t = make_double2(0.0, 0.0);
    for (int bb = threadIdx.x; bb < nb; bb += blockDim.x) t += __ldcg(&partial[slot * nb + bb]);
    t = block_reduce(t, sh);
    if (threadIdx.x == 0) {
      if (i < J) {
        out[(size_t)r * ldo + i] = t;
        out[(size_t)r * ldo + off2 + i] = make_double2(0.0, 0.0);
      } else {
        // NaN propagates (a NaN or Inf entry must surface as a non-finite norm)
        const double q = t.x;
        const double nrm = (q >= 0.0) ? sqrt(q) : ((q < 0.0) ? 0.0 : q);
        out[(size_t)r * ldo + nrm_off] = make_double2(nrm, 0.0);
        inv[r] = nrm > 0.0 ? 1.0 / nrm : 0.0;
      }
      tickets[slot] = 0;
    }
  }
}

inline int grid_for(long len) {
  long g = (len + 255) / 256;
  if (g > 148 * 16) g = 148 * 16;
  return (int)(g < 1 ? 1 : g);
}

}  // namespace

int dot_blocks(long len) {
  long nb = (len + 4095) / 4096;
  if (nb > 296) nb = 296;
  return (int)(nb < 1 ? 1 : nb);
}

cudaError_t launch_dots(const double2* V, size_t vi, size_t vr, const double2* w, size_t wr, long len, int J,
                        int R, double2* partial, cudaStream_t st, bool with_self, const int* gate) {
  const int nb = dot_blocks(len);
  const long chunk = (len + nb - 1) / nb;
  dim3 grid(nb, J + (with_self ? 1 : 0), R);
  k_dots<<<grid, DOT_THREADS, 0, st>>>(V, vi, vr, w, wr, len, chunk, partial, J, gate);
  return cudaGetLastError();
}

cudaError_t launch_reduce(const double2* partial, int nb, int J, int R, double2* out, int ldo, int off, int mode,
                          double* inv, cudaStream_t st, int* flag, int ref_off, double eta2) {
  dim3 grid(J, R);
  k_reduce_partials<<<grid, 256, 0, st>>>(partial, nb, J, out, ldo, off, mode, inv, flag, ref_off, eta2);
  return cudaGetLastError();
}

cudaError_t launch_dots_fused(const double2* V, size_t vi, size_t vr, const double2* w, size_t wr, long len, int J,
                              int R, double2* partial, bool with_self, const int* gate, unsigned* tickets,
                              double2* out, int ldo, int off, cudaStream_t st) {
  const int nb = dot_blocks(len);
  const long chunk = (len + nb - 1) / nb;
  dim3 grid(nb, J + (with_self ? 1 : 0), R);
  k_dots_fused<<<grid, DOT_THREADS, 0, st>>>(V, vi, vr, w, wr, len, chunk, partial, J, gate, tickets, out, ldo, off);
  return cudaGetLastError();
}

int axpy_norm_blocks(long len) { return grid_for(len); }

cudaError_t launch_mgs_stage(double2* w, size_t wr, const double2* V, size_t vi, size_t vr, long len, int i, int J,
                             int R, double2* partial, int pslots, unsigned* tickets, double2* out, int ldo, int off2,
                             int nrm_off, double* inv, cudaStream_t st) {
  const int nb = dot_blocks(len);
  const long chunk = (len + nb - 1) / nb;
  k_mgs_stage<<<dim3(nb, R), DOT_THREADS, 0, st>>>(w, wr, V, vi, vr, len, chunk, i, J, partial, pslots, tickets, out,
                                                   ldo, off2, nrm_off, inv);
  return cudaGetLastError();
}

cudaError_t launch_axpy_norm(double2* y, size_t yr, const double2* X, size_t xi, size_t xr, const double2* coef,
                             int ldc, int J, long len, int R, const int* gate, double* partial, unsigned* tickets,
                             double2* out, int ldo, int nrm_off, double* inv, int* flag, int ref_off, double eta2,
                             int mode, cudaStream_t st) {
  dim3 grid(grid_for(len), R);
  k_axpy_norm<<<grid, 256, 0, st>>>(y, yr, X, xi, xr, coef, ldc, J, len, gate, partial, tickets, out, ldo, nrm_off,
                                    inv, flag, ref_off, eta2, mode);
  return cudaGetLastError();
}

template <typename Cx>
cudaError_t launch_multi_axpy(double2* y, size_t yr, const Cx* X, size_t xi, size_t xr, const double2* coef, int ldc,
                              int J, double sign, long len, int R, cudaStream_t st, const int* gate) {
  dim3 grid(grid_for(len), R);
  k_multi_axpy<Cx><<<grid, 256, 0, st>>>(y, yr, X, xi, xr, coef, ldc, J, sign, len, gate);
  return cudaGetLastError();
}

template <typename Cd>
cudaError_t launch_scale_copy(Cd* dst, size_t dr, const double2* src, size_t sr, const double* scale, long len, int R,
                              cudaStream_t st) {
  dim3 grid(grid_for(len), R);
  k_scale_copy<Cd><<<grid, 256, 0, st>>>(dst, dr, src, sr, scale, len);
  return cudaGetLastError();
}

cudaError_t launch_scale_copy_dual(double2* dst, float2* dst32, size_t dr, const double2* src, size_t sr,
                                   const double* scale, long len, int R, cudaStream_t st) {
  dim3 grid(grid_for(len), R);
  k_scale_copy_dual<<<grid, 256, 0, st>>>(dst, dst32, dr, src, sr, scale, len);
  return cudaGetLastError();
}

template <typename Cs, typename Cd>
cudaError_t launch_cast(const Cs* src, Cd* dst, long len, cudaStream_t st) {
  k_cast<Cs, Cd><<<grid_for(len), 256, 0, st>>>(src, dst, len);
  return cudaGetLastError();
}

template cudaError_t launch_multi_axpy<double2>(double2*, size_t, const double2*, size_t, size_t, const double2*, int,
                                                int, double, long, int, cudaStream_t, const int*);
template cudaError_t launch_multi_axpy<float2>(double2*, size_t, const float2*, size_t, size_t, const double2*, int,
                                               int, double, long, int, cudaStream_t, const int*);
template cudaError_t launch_scale_copy<double2>(double2*, size_t, const double2*, size_t, const double*, long, int,
                                                cudaStream_t);
template cudaError_t launch_scale_copy<float2>(float2*, size_t, const double2*, size_t, const double*, long, int,
                                               cudaStream_t);
template cudaError_t launch_cast<double2, float2>(const double2*, float2*, long, cudaStream_t);
template cudaError_t launch_cast<float2, double2>(const float2*, double2*, long, cudaStream_t);

// ---------------------------------------------------------------------------
// Least squares of the outer FGMRES (Saad, Iterative Methods for Sparse Linear
// Systems, Sec. 6.5.3: Givens rotations on the Hessenberg matrix).  A rotation
// that annihilates the subdiagonal entry hn (real, >= 0) of column j, whose
// entry j after the earlier rotations is t, is c = |t| / rho,
// s = (t / |t|) hn / rho, rho = (|t|^2 + hn^2)^(1/2), applied to rows (j, j+1)
// as [c s; -conj(s) c]; g_{j+1} = -conj(s) g_j, g_j = c g_j, and |g_{j+1}| is
// the residual norm of the least-squares solution.  Instead of rotating every
// stored column again, the product Q^H of the rotations is kept: step j needs
// only t = (row j of Q^H) . (column j) (a warp-wide dot product) and updates
// rows j and j+1 of Q^H; at the end of the cycle R = Q^H H and the triangular
// solve give y.  On this GPU's narrow FP64 pipe that is a few dozen FP64
// instructions per step instead of a chain of about 12 j.
namespace {

__device__ __forceinline__ double2 warp_sum_c(double2 v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
    v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
  }
  return v;
}

__global__ void k_ls_init(LsView v, const LsInit* __restrict__ init, int m) {
  const int r = blockIdx.x;
  const LsInit q = init[r];
  const int n1 = m + 1;
  double2* Q = v.Q + (size_t)r * n1 * n1;
  for (int i = threadIdx.x; i < n1 * n1; i += blockDim.x)
    Q[i] = make_double2(i / n1 == i % n1 ? 1.0 : 0.0, 0.0);
  double2* g = v.g + (size_t)r * n1;
  for (int i = threadIdx.x; i < n1; i += blockDim.x) g[i] = make_double2(i == 0 ? q.beta : 0.0, 0.0);
  if (threadIdx.x == 0) {
    int* s = v.st + 4 * r;
    s[0] = q.building; s[1] = 0; s[2] = q.iters; s[3] = 0;
    v.bnorm[r] = q.bnorm;
  }
}

// one warp per right-hand side; every load is issued first (one round trip),
// lane l handles rows l, l + 32 and l + 64 of the column
__global__ void __launch_bounds__(32) k_ls_step(LsView v, const double2* __restrict__ hcol, int ldh, int nrm_off,
                                                int j, int m, double tol, int max_iter, LsOut* __restrict__ out) {
  const int r = blockIdx.x, lane = threadIdx.x;
  const int n1 = m + 1;
  int* s = v.st + 4 * r;
  const int4 st0 = *reinterpret_cast<const int4*>(s);        // building, k, iters, nonfinite
  const double2* hh = hcol + (size_t)r * ldh;
  double2* Q = v.Q + (size_t)r * n1 * n1;
  double2* g = v.g + (size_t)r * n1;
  const double hn = hh[nrm_off].x;
  const double bnorm = v.bnorm[r];
  const double2 gj = g[j];
  double2 h[3], q[3];
#pragma unroll
  for (int u = 0; u < 3; ++u) {
    const int i = lane + 32 * u;
    h[u] = q[u] = make_double2(0.0, 0.0);
    if (i <= j) {
      h[u] = hh[i] + hh[(m + 2) + i];
      q[u] = Q[(size_t)j * n1 + i];
    }
  }
  int4 st1 = st0;
  if (st0.x) {
    double2* Hr = v.Hraw + (size_t)r * n1 * m;
    double2 part = make_double2(0.0, 0.0);
#pragma unroll
    for (int u = 0; u < 3; ++u) {
      const int i = lane + 32 * u;
      if (i <= j) Hr[(size_t)i * m + j] = h[u];
      if (32 * u <= j) part += cmul(q[u], h[u]);            // warp-uniform: FP64 issue is the cost here
    }
    if (lane == 0) Hr[(size_t)(j + 1) * m + j] = make_double2(hn, 0.0);
    const double2 t = warp_sum_c(part);                      // entry j of the column after the earlier rotations
    if (!isfinite(hn)) {
      st1.x = 0; st1.y = 0; st1.w = 1;
    } else {
      const double a2 = t.x * t.x + t.y * t.y;
      double c;
      double2 sv;
      if (hn == 0.0) { c = 1.0; sv = make_double2(0.0, 0.0); }
      else if (a2 == 0.0) { c = 0.0; sv = make_double2(1.0, 0.0); }
      else {
        // c = |t| / rho, s = t hn / (|t| rho), with two reciprocal square roots
        const double ia = rsqrt(a2), irho = rsqrt(fma(hn, hn, a2));
        c = a2 * ia * irho;
        const double f = hn * irho * ia;
        sv = make_double2(t.x * f, t.y * f);
      }
      // rows j and j+1 of Q^H: [c s; -conj(s) c] applied to (row j, e_{j+1})
#pragma unroll
      for (int u = 0; u < 3; ++u) {
        const int i = lane + 32 * u;
        if (i <= j + 1) {
          const double e1 = i == j + 1 ? 1.0 : 0.0;
          Q[(size_t)j * n1 + i] = c * q[u] + e1 * sv;
          Q[(size_t)(j + 1) * n1 + i] = make_double2(e1 * c, 0.0) - cmulc(sv, q[u]);
        }
      }
      const double2 g1 = -1.0 * cmulc(sv, gj);
      const double est2 = cabs2(g1), tb = tol * bnorm;
      st1.y = j + 1;
      st1.z += 1;
      if (est2 <= tb * tb || hn == 0.0 || st1.z >= max_iter) st1.x = 0;
      if (lane == 0) {
        g[j + 1] = g1;
        g[j] = c * gj;
        out[r].est2 = est2;
      }
    }
    if (lane == 0) *reinterpret_cast<int4*>(s) = st1;
  }
  if (lane == 0) {
    out[r].building = st1.x;
    out[r].k = st1.y;
    out[r].iters = st1.z;
    out[r].nonfinite = st1.w;
  }
}

// R[i][c] = sum_{l <= c+1} Q^H[i][l] Hraw[l][c] for i <= c < k: block (c, r),
// lanes over rows
__global__ void __launch_bounds__(64) k_ls_rmat(LsView v, int m) {
  const int c = blockIdx.x, r = blockIdx.y;
  const int* s = v.st + 4 * r;
  const int k = s[3] ? 0 : s[1];
  if (c >= k) return;
  const int n1 = m + 1;
  const double2* Q = v.Q + (size_t)r * n1 * n1;
  const double2* Hr = v.Hraw + (size_t)r * n1 * m;
  double2* Rm = v.Rm + (size_t)r * m * m;
  for (int i = threadIdx.x; i <= c; i += blockDim.x) {
    double2 acc = make_double2(0.0, 0.0);
    for (int l = 0; l <= c + 1; ++l) acc += cmul(Q[(size_t)i * n1 + l], Hr[(size_t)l * m + c]);
    Rm[(size_t)i * m + c] = acc;
  }
}

// back substitution, one warp per right-hand side (column oriented)
__global__ void __launch_bounds__(32) k_ls_backsolve(LsView v, double2* __restrict__ y, int m) {
  const int r = blockIdx.x, lane = threadIdx.x;
  const int* s = v.st + 4 * r;
  const int k = s[3] ? 0 : s[1];
  const double2* Rm = v.Rm + (size_t)r * m * m;
  const double2* g = v.g + (size_t)r * (m + 1);
  double2* yr = y + (size_t)r * m;
  __shared__ double2 tt[64];
  for (int i = lane; i < m; i += 32) {
    tt[i] = i < k ? g[i] : make_double2(0.0, 0.0);
    if (i >= k) yr[i] = make_double2(0.0, 0.0);
  }
  __syncwarp();
  for (int i = k - 1; i >= 0; --i) {
    const double2 d = Rm[(size_t)i * m + i];
    const double idd = 1.0 / (d.x * d.x + d.y * d.y);
    const double2 ti = tt[i];
    const double2 yi = make_double2((ti.x * d.x + ti.y * d.y) * idd, (ti.y * d.x - ti.x * d.y) * idd);
    if (lane == 0) yr[i] = yi;
    for (int l = lane; l < i; l += 32) tt[l] -= cmul(Rm[(size_t)l * m + i], yi);
    __syncwarp();
  }
}

}  // namespace

cudaError_t launch_ls_init(LsView v, const LsInit* init, int R, int m, cudaStream_t st) {
  k_ls_init<<<R, 128, 0, st>>>(v, init, m);
  return cudaGetLastError();
}

cudaError_t launch_ls_step(LsView v, const double2* hcol, int ldh, int nrm_off, int j, int R, int m, double tol,
                           int max_iter, LsOut* out, cudaStream_t st) {
  k_ls_step<<<R, 32, 0, st>>>(v, hcol, ldh, nrm_off, j, m, tol, max_iter, out);
  return cudaGetLastError();
}

cudaError_t launch_ls_solve(LsView v, double2* y, int R, int m, cudaStream_t st) {
  k_ls_rmat<<<dim3(m, R), 64, 0, st>>>(v, m);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_ls_backsolve<<<R, 32, 0, st>>>(v, y, m);
  return cudaGetLastError();
}
