// Coarse-level kernels: the Galerkin operator A_l = P^H A_{l-1} P in block-stencil
// form, its 16-colour block Gauss-Seidel smoother, and the coarsest direct solve.
//
// A_l is stored as K blocks of 2x2 complex per coarse site, [K][4][n] (entry
// 2 alpha + beta, site-major within an entry plane, so consecutive threads read
// consecutive sites).  Offsets are the canonical (dt mod Nt, dx mod Nx) pairs,
// sorted, with (0, 0) first.  FP32 path: __half2 entries with one FP32 scale per
// block ([K][n]).
#include "kernels.h"

namespace {

template <typename T, typename BT>
__device__ __forceinline__ typename cplx<T>::type b_load(const BT* B, const float* sc, int k, int e, int n, int v);

template <>
__device__ __forceinline__ double2 b_load<double, double2>(const double2* B, const float*, int k, int e, int n, int v) {
  return B[((size_t)k * 4 + e) * n + v];
}
template <>
__device__ __forceinline__ float2 b_load<float, __half2>(const __half2* B, const float* sc, int k, int e, int n, int v) {
  return h2c<float>(B[((size_t)k * 4 + e) * n + v], sc[(size_t)k * n + v]);
}

// out = A in  (b == nullptr)  or  out = b - A in
template <typename T, typename BT>
__global__ void __launch_bounds__(256)
k_coarse_apply(const typename cplx<T>::type* __restrict__ in, typename cplx<T>::type* __restrict__ out,
               const typename cplx<T>::type* __restrict__ b, const BT* __restrict__ B,
               const float* __restrict__ Bs, Offsets off, int Nt, int Nx) {
  using C = typename cplx<T>::type;
  const int n = Nt * Nx;
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  const int t = v / Nx, x = v - (v / Nx) * Nx;
  const size_t roff = (size_t)blockIdx.y * 2 * n;
  const C* i0 = in + roff;
  C y0 = czero<C>(), y1 = czero<C>();
  for (int k = 0; k < off.K; ++k) {
    int tw = t + off.dt[k]; tw -= (tw >= Nt) ? Nt : 0;
    int xw = x + off.dx[k]; xw -= (xw >= Nx) ? Nx : 0;
    const int w = tw * Nx + xw;
    const C x0 = i0[w], x1 = i0[n + w];
    y0 += cmul(b_load<T, BT>(B, Bs, k, 0, n, v), x0) + cmul(b_load<T, BT>(B, Bs, k, 1, n, v), x1);
    y1 += cmul(b_load<T, BT>(B, Bs, k, 2, n, v), x0) + cmul(b_load<T, BT>(B, Bs, k, 3, n, v), x1);
  }
  C* o = out + roff;
  if (b) {
    y0 = b[roff + v] - y0;
    y1 = b[roff + n + v] - y1;
  }
  o[v] = y0;
  o[n + v] = y1;
}

// One colour of the 16-colour block Gauss-Seidel sweep on A e = r:
// sites (t, x) with (t mod 4, x mod 4) = (c / 4, c % 4):
// e_v <- A_vv^{-1} (r_v - sum_{k >= 1} A_{v, v+off_k} e_{v+off_k}).
template <typename T, typename BT>
__global__ void __launch_bounds__(256)
k_coarse_colour(typename cplx<T>::type* __restrict__ e, const typename cplx<T>::type* __restrict__ r,
                const BT* __restrict__ B, const float* __restrict__ Bs,
                const typename cplx<T>::type* __restrict__ Dinv, Offsets off, int Nt, int Nx, int colour) {
  using C = typename cplx<T>::type;
  const int n = Nt * Nx;
  const int qx = Nx >> 2;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (n >> 4)) return;
  const int ti = idx / qx;
  const int t = 4 * ti + (colour >> 2);
  const int x = 4 * (idx - ti * qx) + (colour & 3);
  const int v = t * Nx + x;
  const size_t roff = (size_t)blockIdx.y * 2 * n;
  C* e0 = e + roff;
  C s0 = r[roff + v], s1 = r[roff + n + v];
  for (int k = 1; k < off.K; ++k) {
    int tw = t + off.dt[k]; tw -= (tw >= Nt) ? Nt : 0;
    int xw = x + off.dx[k]; xw -= (xw >= Nx) ? Nx : 0;
    const int w = tw * Nx + xw;
    const C x0 = e0[w], x1 = e0[n + w];
    s0 -= cmul(b_load<T, BT>(B, Bs, k, 0, n, v), x0) + cmul(b_load<T, BT>(B, Bs, k, 1, n, v), x1);
    s1 -= cmul(b_load<T, BT>(B, Bs, k, 2, n, v), x0) + cmul(b_load<T, BT>(B, Bs, k, 3, n, v), x1);
  }
  const C d00 = Dinv[v], d01 = Dinv[n + v], d10 = Dinv[2 * n + v], d11 = Dinv[3 * n + v];
  e0[v] = cmul(d00, s0) + cmul(d01, s1);
  e0[n + v] = cmul(d10, s0) + cmul(d11, s1);
}

// y_r = Ainv x_r for the coarsest level: dense FP64 complex matrix, row-major,
// nd x nd; vectors are contiguous nd-element arrays (the [2][Nt][Nx] layout
// flattened).  One warp per row; the row is read once for all R right-hand
// sides (R <= 8 per launch).
template <typename Cv>
__global__ void __launch_bounds__(256)
k_dense_gemv(const double2* __restrict__ A, const Cv* __restrict__ x, Cv* __restrict__ y, int nd, int R) {
  const int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (row >= nd) return;
  double2 acc[8];
#pragma unroll
  for (int r = 0; r < 8; ++r) acc[r] = make_double2(0.0, 0.0);
  const double2* a = A + (size_t)row * nd;
  for (int j = lane; j < nd; j += 32) {
    const double2 aj = a[j];
#pragma unroll
    for (int r = 0; r < 8; ++r)
      if (r < R) acc[r] += cmul(aj, to_c(x[(size_t)r * nd + j], double()));
  }
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    if (r < R) {
      double re = acc[r].x, im = acc[r].y;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        re += __shfl_xor_sync(0xffffffffu, re, o);
        im += __shfl_xor_sync(0xffffffffu, im, o);
      }
      if (lane == 0) y[(size_t)r * nd + row] = to_c(make_double2(re, im), typename real_of<Cv>::type());
    }
  }
}

}  // namespace

template <typename T, typename BT>
cudaError_t launch_coarse_apply(const typename cplx<T>::type* in, typename cplx<T>::type* out,
                                const typename cplx<T>::type* b, const BT* B, const float* Bs,
                                const Offsets& off, int Nt, int Nx, int R, cudaStream_t st) {
  const int n = Nt * Nx;
  dim3 grid((n + 255) / 256, R);
  k_coarse_apply<T, BT><<<grid, 256, 0, st>>>(in, out, b, B, Bs, off, Nt, Nx);
  return cudaGetLastError();
}

template <typename T, typename BT>
cudaError_t launch_coarse_colour(typename cplx<T>::type* e, const typename cplx<T>::type* r, const BT* B,
                                 const float* Bs, const typename cplx<T>::type* Dinv, const Offsets& off,
                                 int Nt, int Nx, int colour, int R, cudaStream_t st) {
  const int m = Nt * Nx / 16;
  const int bs = m < 256 ? ((m + 31) / 32) * 32 : 256;
  dim3 grid((m + bs - 1) / bs, R);
  k_coarse_colour<T, BT><<<grid, bs, 0, st>>>(e, r, B, Bs, Dinv, off, Nt, Nx, colour);
  return cudaGetLastError();
}

template <typename Cv>
cudaError_t launch_dense_gemv(const double2* A, const Cv* x, Cv* y, int nd, int R, cudaStream_t st) {
  for (int r0 = 0; r0 < R; r0 += 8) {
    const int rr = (R - r0) < 8 ? (R - r0) : 8;
    k_dense_gemv<Cv><<<(nd * 32 + 255) / 256, 256, 0, st>>>(A, x + (size_t)r0 * nd, y + (size_t)r0 * nd, nd, rr);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

template cudaError_t launch_coarse_apply<double, double2>(const double2*, double2*, const double2*, const double2*,
                                                          const float*, const Offsets&, int, int, int, cudaStream_t);
template cudaError_t launch_coarse_apply<float, __half2>(const float2*, float2*, const float2*, const __half2*,
                                                         const float*, const Offsets&, int, int, int, cudaStream_t);
template cudaError_t launch_coarse_colour<double, double2>(double2*, const double2*, const double2*, const float*,
                                                           const double2*, const Offsets&, int, int, int, int,
                                                           cudaStream_t);
template cudaError_t launch_coarse_colour<float, __half2>(float2*, const float2*, const __half2*, const float*,
                                                          const float2*, const Offsets&, int, int, int, int,
                                                          cudaStream_t);
template cudaError_t launch_dense_gemv<double2>(const double2*, const double2*, double2*, int, int, cudaStream_t);
template cudaError_t launch_dense_gemv<float2>(const double2*, const float2*, float2*, int, int, cudaStream_t);
