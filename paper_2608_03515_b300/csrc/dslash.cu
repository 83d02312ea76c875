// Fine-level kernels: the Wilson-Dirac stencil of Eq. (3) and the red-black
// site Gauss-Seidel half sweep used as post-smoother on the fine level.
//
// Layout: vectors [R][spin][Nt][Nx] complex, links [mu][Nt][Nx] complex,
// mu = 0 the (antiperiodic) t direction, mu = 1 the periodic x direction.
// The stencil kernels take links with the Eq. (7) boundary sign folded in:
// both hops across the t boundary (forward from t = Nt-1, backward from t = 0)
// use the link U_0(Nt-1, x) and carry the factor -1, so storing -U_0(Nt-1, x)
// gives exactly the same products without a per-site sign.
// One thread per site and right-hand side; neighbours are re-read through L1/L2
// (each input element is needed by 5 threads of adjacent rows/columns).
#include "kernels.h"

namespace {

// h = sum_mu [ (1 - sigma_mu) U_mu(n) psi(n+mu) + (1 + sigma_mu) U_mu(n-mu)^* psi(n-mu) ]
// (boundary sign folded into U, see above), so that
// (D psi)(n) = (m0 + 2) psi(n) - h / 2.  Spin projection: every (1 -/+ sigma)
// has rank one, so each hop needs one complex multiplication by its link.
template <typename T, typename Cin>
__device__ __forceinline__ void hop_sum(const Cin* __restrict__ p0, const Cin* __restrict__ p1,
                                        const typename cplx<T>::type* __restrict__ U,
                                        int t, int x, int Nt, int Nx, int n,
                                        typename cplx<T>::type& h0, typename cplx<T>::type& h1) {
  using C = typename cplx<T>::type;
  const int s = t * Nx + x;
  const int tf = (t + 1 == Nt) ? 0 : t + 1;
  const int tb = (t == 0) ? Nt - 1 : t - 1;
  const int xf = (x + 1 == Nx) ? 0 : x + 1;
  const int xb = (x == 0) ? Nx - 1 : x - 1;
  const int s_tf = tf * Nx + x, s_tb = tb * Nx + x, s_xf = t * Nx + xf, s_xb = t * Nx + xb;

  // t forward: (1 - sigma_0) psi = (g, -g), g = psi_0 - psi_1
  C g = to_c(p0[s_tf], T()) - to_c(p1[s_tf], T());
  g = cmul(U[s], g);
  h0 = g;
  h1 = -g;
  // t backward: (1 + sigma_0) psi = (g, g), g = psi_0 + psi_1, link U_0(n - t)^*
  g = to_c(p0[s_tb], T()) + to_c(p1[s_tb], T());
  g = cmulc(U[s_tb], g);
  h0 += g;
  h1 += g;
  // x forward: (1 - sigma_1) psi = (g, -i g), g = psi_0 + i psi_1
  g = to_c(p0[s_xf], T()) + ci(to_c(p1[s_xf], T()));
  g = cmul(U[n + s], g);
  h0 += g;
  h1 -= ci(g);
  // x backward: (1 + sigma_1) psi = (g, i g), g = psi_0 - i psi_1, link U_1(n - x)^*
  g = to_c(p0[s_xb], T()) - ci(to_c(p1[s_xb], T()));
  g = cmulc(U[n + s_xb], g);
  h0 += g;
  h1 += ci(g);
}

// out = D in   (b == nullptr)   or   out = b - D in   (residual form)
template <typename Cin, typename Cout, typename T>
__global__ void __launch_bounds__(256)
k_dslash(const Cin* __restrict__ in, Cout* __restrict__ out, const Cout* __restrict__ b,
         const typename cplx<T>::type* __restrict__ U, T diag_s, const T* __restrict__ diag_r, int Nt, int Nx) {
  using C = typename cplx<T>::type;
  const T diag = diag_r ? diag_r[blockIdx.y] : diag_s;   // m0 + 2, per right-hand side when given
  const int n = Nt * Nx;
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  const size_t roff = (size_t)blockIdx.y * 2 * n;
  const Cin* p0 = in + roff;
  const Cin* p1 = p0 + n;
  const int t = s / Nx, x = s - (s / Nx) * Nx;
  C h0, h1;
  hop_sum<T>(p0, p1, U, t, x, Nt, Nx, n, h0, h1);
  C y0 = diag * to_c(p0[s], T()) - T(0.5) * h0;
  C y1 = diag * to_c(p1[s], T()) - T(0.5) * h1;
  Cout* o = out + roff;
  if (b) {
    const Cout* bb = b + roff;
    y0 = to_c(bb[s], T()) - y0;
    y1 = to_c(bb[s + n], T()) - y1;
  }
  o[s] = to_c(y0, typename real_of<Cout>::type());
  o[s + n] = to_c(y1, typename real_of<Cout>::type());
}

// Red-black half sweep of colour c on D e = r: for every site n with
// (t + x) mod 2 == c, e(n) <- (r(n) + h(n)/2) / (m0 + 2)  (block = site, whose
// diagonal block is (m0 + 2) I).  One thread per site of the colour.
template <typename T>
__global__ void __launch_bounds__(256)
k_rb_half(typename cplx<T>::type* __restrict__ e, const typename cplx<T>::type* __restrict__ r,
          const typename cplx<T>::type* __restrict__ U, T inv_diag_s, const T* __restrict__ inv_diag_r, int Nt,
          int Nx, int colour) {
  using C = typename cplx<T>::type;
  const T inv_diag = inv_diag_r ? inv_diag_r[blockIdx.y] : inv_diag_s;
  const int n = Nt * Nx;
  const int hx = Nx >> 1;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (n >> 1)) return;
  const int t = idx / hx;
  const int x = 2 * (idx - t * hx) + ((t + colour) & 1);
  const int s = t * Nx + x;
  const size_t roff = (size_t)blockIdx.y * 2 * n;
  C* e0 = e + roff;
  const C* rr = r + roff;
  C h0, h1;
  hop_sum<T>(e0, e0 + n, U, t, x, Nt, Nx, n, h0, h1);
  e0[s] = inv_diag * (rr[s] + T(0.5) * h0);
  e0[s + n] = inv_diag * (rr[s + n] + T(0.5) * h1);
}

// U_0(Nt-1, x) <- -U_0(Nt-1, x) for every x (the boundary sign of Eq. (7))
__global__ void k_fold_boundary_sign(double2* __restrict__ U, int Nt, int Nx) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= Nx) return;
  double2& u = U[(size_t)(Nt - 1) * Nx + x];
  u = make_double2(-u.x, -u.y);
}

}  // namespace

cudaError_t launch_fold_boundary_sign(double2* U, int Nt, int Nx, cudaStream_t st) {
  k_fold_boundary_sign<<<(Nx + 255) / 256, 256, 0, st>>>(U, Nt, Nx);
  return cudaGetLastError();
}

template <typename Cin, typename Cout, typename T>
cudaError_t launch_dslash(const Cin* in, Cout* out, const Cout* b, const typename cplx<T>::type* U,
                          T diag, int Nt, int Nx, int R, cudaStream_t st, const T* diag_r) {
  const int n = Nt * Nx;
  dim3 grid((n + 255) / 256, R);
  k_dslash<Cin, Cout, T><<<grid, 256, 0, st>>>(in, out, b, U, diag, diag_r, Nt, Nx);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_rb_half(typename cplx<T>::type* e, const typename cplx<T>::type* r,
                           const typename cplx<T>::type* U, T inv_diag, int Nt, int Nx, int colour,
                           int R, cudaStream_t st, const T* inv_diag_r) {
  const int half = Nt * Nx / 2;
  dim3 grid((half + 255) / 256, R);
  k_rb_half<T><<<grid, 256, 0, st>>>(e, r, U, inv_diag, inv_diag_r, Nt, Nx, colour);
  return cudaGetLastError();
}

template cudaError_t launch_dslash<double2, double2, double>(const double2*, double2*, const double2*,
                                                             const double2*, double, int, int, int, cudaStream_t,
                                                             const double*);
template cudaError_t launch_dslash<float2, float2, float>(const float2*, float2*, const float2*,
                                                          const float2*, float, int, int, int, cudaStream_t,
                                                          const float*);
template cudaError_t launch_dslash<float2, double2, double>(const float2*, double2*, const double2*,
                                                            const double2*, double, int, int, int, cudaStream_t,
                                                            const double*);
template cudaError_t launch_rb_half<double>(double2*, const double2*, const double2*, double, int, int, int,
                                            int, cudaStream_t, const double*);
template cudaError_t launch_rb_half<float>(float2*, const float2*, const float2*, float, int, int, int, int,
                                           cudaStream_t, const float*);
