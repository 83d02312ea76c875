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
#include <algorithm>
#include <map>
#include <type_traits>
#include <mutex>
#include <utility>

#include "kernels.h"

namespace {

// h = sum_mu [ (1 - sigma_mu) U_mu(n) psi(n+mu) + (1 + sigma_mu) U_mu(n-mu)^* psi(n-mu) ]
// (boundary sign folded into U, see above), so that
// (D psi)(n) = (m0 + 2) psi(n) - h / 2.  Spin projection: every (1 -/+ sigma)
// has rank one, so each hop needs one complex multiplication by its link.
// loads of the vector hop_sum reads: plain, or through L2 (ld.global.cg) when
// other blocks of the same launch wrote it
template <bool CG, typename Cin>
__device__ __forceinline__ Cin hop_ld(const Cin* p) {
  if constexpr (CG) return __ldcg(p);
  else return *p;
}

// NEG1: the lower spin component is read negated, i.e. the hops act on
// sigma_3 psi (the conjugated operator sigma_3 D sigma_3 of Eq. (6))
template <typename T, typename Cin, bool CG = false, bool NEG1 = false>
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
  const T s1 = NEG1 ? T(-1) : T(1);
  C g = to_c(hop_ld<CG>(p0 + s_tf), T()) - s1 * to_c(hop_ld<CG>(p1 + s_tf), T());
  g = cmul(U[s], g);
  h0 = g;
  h1 = -g;
  // t backward: (1 + sigma_0) psi = (g, g), g = psi_0 + psi_1, link U_0(n - t)^*
  g = to_c(hop_ld<CG>(p0 + s_tb), T()) + s1 * to_c(hop_ld<CG>(p1 + s_tb), T());
  g = cmulc(U[s_tb], g);
  h0 += g;
  h1 += g;
  // x forward: (1 - sigma_1) psi = (g, -i g), g = psi_0 + i psi_1
  g = to_c(hop_ld<CG>(p0 + s_xf), T()) + s1 * ci(to_c(hop_ld<CG>(p1 + s_xf), T()));
  g = cmul(U[n + s], g);
  h0 += g;
  h1 -= ci(g);
  // x backward: (1 + sigma_1) psi = (g, i g), g = psi_0 - i psi_1, link U_1(n - x)^*
  g = to_c(hop_ld<CG>(p0 + s_xb), T()) - s1 * ci(to_c(hop_ld<CG>(p1 + s_xb), T()));
  g = cmulc(U[n + s_xb], g);
  h0 += g;
  h1 += ci(g);
}

// The hop sum of one site from its neighbour values (the arithmetic of
// hop_sum, same operations in the same order): f/b = forward/backward
// neighbour, t/x = direction, 0/1 = spin; ut = U_0(n), utb = U_0(n - t),
// ux = U_1(n), uxb = U_1(n - x).
template <typename C>
__device__ __forceinline__ void hop_vals(C ft0, C ft1, C bt0, C bt1, C fx0, C fx1, C bx0, C bx1, C ut, C utb, C ux,
                                         C uxb, C& h0, C& h1) {
  C g = cmul(ut, ft0 - ft1);
  h0 = g;
  h1 = -g;
  g = cmulc(utb, bt0 + bt1);
  h0 += g;
  h1 += g;
  g = cmul(ux, fx0 + ci(fx1));
  h0 += g;
  h1 -= ci(g);
  g = cmulc(uxb, bx0 - ci(bx1));
  h0 += g;
  h1 += ci(g);
}

__device__ __forceinline__ float2 lo2(float4 v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 hi2(float4 v) { return make_float2(v.z, v.w); }

// FP32 out = D in (or b - D in) with two x-adjacent sites (x even) per thread:
// every pair of complex values a thread needs from its own row and the rows
// t +- 1 comes in one 16-byte load, so a thread has twice the bytes in flight
// of k_dslash with half the load instructions.  Per site the arithmetic of
// k_dslash.  Nx must be even.
__global__ void __launch_bounds__(256)
k_dslash32x2(const float2* __restrict__ in, float2* __restrict__ out, const float2* __restrict__ b,
             const float2* __restrict__ U, float diag_s, const float* __restrict__ diag_r, int Nt, int Nx) {
  const float diag = diag_r ? diag_r[blockIdx.y] : diag_s;
  const int n = Nt * Nx, hx = Nx >> 1;
  const int pidx = blockIdx.x * blockDim.x + threadIdx.x;
  if (pidx >= (n >> 1)) return;
  const int t = pidx / hx, x = 2 * (pidx - t * hx);
  const int s = t * Nx + x;
  const int tf = (t + 1 == Nt) ? 0 : t + 1, tb = (t == 0) ? Nt - 1 : t - 1;
  const int xf2 = (x + 2 == Nx) ? 0 : x + 2, xb = (x == 0) ? Nx - 1 : x - 1;
  const size_t roff = (size_t)blockIdx.y * 2 * n;
  const float2* p0 = in + roff;
  const float2* p1 = p0 + n;
  const float4 own0 = *reinterpret_cast<const float4*>(p0 + s), own1 = *reinterpret_cast<const float4*>(p1 + s);
  const float4 ft0 = *reinterpret_cast<const float4*>(p0 + tf * Nx + x);
  const float4 ft1 = *reinterpret_cast<const float4*>(p1 + tf * Nx + x);
  const float4 bt0 = *reinterpret_cast<const float4*>(p0 + tb * Nx + x);
  const float4 bt1 = *reinterpret_cast<const float4*>(p1 + tb * Nx + x);
  const float2 fx0 = p0[t * Nx + xf2], fx1 = p1[t * Nx + xf2];
  const float2 bx0 = p0[t * Nx + xb], bx1 = p1[t * Nx + xb];
  const float4 ut = *reinterpret_cast<const float4*>(U + s);
  const float4 utb = *reinterpret_cast<const float4*>(U + tb * Nx + x);
  const float4 ux = *reinterpret_cast<const float4*>(U + n + s);
  const float2 uxb = U[n + t * Nx + xb];
  float2 h0, h1, y0, y1;
  float4 o0, o1;
  // site x: x-neighbours x + 1 (own pair, upper half) and x - 1
  hop_vals(lo2(ft0), lo2(ft1), lo2(bt0), lo2(bt1), hi2(own0), hi2(own1), bx0, bx1, lo2(ut), lo2(utb), lo2(ux), uxb,
           h0, h1);
  y0 = diag * lo2(own0) - 0.5f * h0;
  y1 = diag * lo2(own1) - 0.5f * h1;
  o0.x = y0.x; o0.y = y0.y; o1.x = y1.x; o1.y = y1.y;
  // site x + 1: x-neighbours x + 2 and x (own pair, lower half); backward link U_1(x)
  hop_vals(hi2(ft0), hi2(ft1), hi2(bt0), hi2(bt1), fx0, fx1, lo2(own0), lo2(own1), hi2(ut), hi2(utb), hi2(ux),
           lo2(ux), h0, h1);
  y0 = diag * hi2(own0) - 0.5f * h0;
  y1 = diag * hi2(own1) - 0.5f * h1;
  o0.z = y0.x; o0.w = y0.y; o1.z = y1.x; o1.w = y1.y;
  if (b) {
    const float4 b0 = *reinterpret_cast<const float4*>(b + roff + s);
    const float4 b1 = *reinterpret_cast<const float4*>(b + roff + n + s);
    o0 = make_float4(b0.x - o0.x, b0.y - o0.y, b0.z - o0.z, b0.w - o0.w);
    o1 = make_float4(b1.x - o1.x, b1.y - o1.y, b1.z - o1.z, b1.w - o1.w);
  }
  *reinterpret_cast<float4*>(out + roff + s) = o0;
  *reinterpret_cast<float4*>(out + roff + n + s) = o1;
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

// out = sigma_3 D sigma_3 in = D^H in (Eq. (6): sigma_3-hermiticity), FP64:
// with phi = sigma_3 in = (in_0, -in_1), (D phi)_0 = diag in_0 - h_0(phi) / 2
// and -(D phi)_1 = diag in_1 + h_1(phi) / 2.
__global__ void __launch_bounds__(256)
k_dslash_dag(const double2* __restrict__ in, double2* __restrict__ out, const double2* __restrict__ U, double diag,
             int Nt, int Nx) {
  const int n = Nt * Nx;
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  const size_t roff = (size_t)blockIdx.y * 2 * n;
  const double2* p0 = in + roff;
  const double2* p1 = p0 + n;
  const int t = s / Nx, x = s - (s / Nx) * Nx;
  double2 h0, h1;
  hop_sum<double, double2, false, true>(p0, p1, U, t, x, Nt, Nx, n, h0, h1);
  out[roff + s] = diag * p0[s] - 0.5 * h0;
  out[roff + n + s] = diag * p1[s] + 0.5 * h1;
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

// P entry of the fused kernel (same layout and rounding as the transfer kernels)
template <typename T, typename PT>
__device__ __forceinline__ typename cplx<T>::type fp_load(const PT* P, const float* scale, size_t idx, int tile);
template <>
__device__ __forceinline__ double2 fp_load<double, double2>(const double2* P, const float*, size_t idx, int) {
  return P[idx];
}
template <>
__device__ __forceinline__ float2 fp_load<float, __half2>(const __half2* P, const float* scale, size_t idx, int tile) {
  return h2c<float>(P[idx], scale[tile]);
}

// Fine-level end of the V-cycle in one cooperative launch: e = P e_c (phase
// 0), then `sweeps` red-black sweeps on D e = r (phases 1, 2, ...: colour 0,
// colour 1, ...).  Block b owns rows [b rows, (b+1) rows) of one right-hand
// side.  A red-black update reads e one
// row up and down, so before phase p a block waits only until the two
// neighbouring row blocks have published phase p - 1 (the owner-sweep scheme:
// flags[block] = base + phases done, base = sync[3], end ticket sync[4],
// bounded polls, time-out flag sync[2]).  Per site the arithmetic is that of
// k_prolong and k_rb_half (same order), so the result equals that of the
// separate launches; e is read through L2 because other blocks wrote it.
constexpr unsigned FINE_SPIN_LIMIT = 1u << 20;

template <typename T, typename PT>
__global__ void __launch_bounds__(256)
k_fine_post(const typename cplx<T>::type* __restrict__ ec, typename cplx<T>::type* __restrict__ e,
            const typename cplx<T>::type* __restrict__ r, const PT* __restrict__ P, const float* __restrict__ Pscale,
            const typename cplx<T>::type* __restrict__ U, T inv_diag_s, const T* __restrict__ inv_diag_r,
            int Nt, int Nx, int a, int sweeps, int rows, unsigned* __restrict__ flags, unsigned* __restrict__ sync) {
  using C = typename cplx<T>::type;
  __shared__ int alive;
  const int nrb = Nt / rows;
  const int rhs = blockIdx.x / nrb, b = blockIdx.x - rhs * nrb;
  const int n = Nt * Nx, Np = Nt / a, Nq = Nx / a, nc = Np * Nq, nrows = 2 * (a * a - 1);
  const T inv_diag = inv_diag_r ? inv_diag_r[rhs] : inv_diag_s;
  C* e0 = e + (size_t)rhs * 2 * n;
  const C* r0 = r + (size_t)rhs * 2 * n;
  const C* c0 = ec + (size_t)rhs * 2 * nc;
  const int t0 = b * rows;
  const unsigned base = *reinterpret_cast<volatile unsigned*>(sync + 3);
  if (threadIdx.x == 0) alive = 1;
  // phase 0: prolongation of the owned rows (both spins of a site per thread)
  for (int idx = threadIdx.x; idx < rows * Nx; idx += blockDim.x) {
    const int t = t0 + idx / Nx, x = idx - (idx / Nx) * Nx;
    const int p = t / a, i = t - p * a, q = x / a, j = x - q * a;
    const int tile = p * Nq + q, l = i * a + j, v = t * Nx + x;
    if (l == 0) {
      __stcg(e0 + v, c0[tile]);
      __stcg(e0 + n + v, c0[nc + tile]);
      continue;
    }
    const int p1 = (p + 1 == Np) ? 0 : p + 1, q1 = (q + 1 == Nq) ? 0 : q + 1;
    const int vtx[4] = {p * Nq + q, p * Nq + q1, p1 * Nq + q, p1 * Nq + q1};
#pragma unroll
    for (int alpha = 0; alpha < 2; ++alpha) {
      const int lr = 2 * (l - 1) + alpha;
      const size_t pb = (size_t)tile * 8 * nrows + lr;
      C acc = czero<C>();
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        cmac(acc, fp_load<T, PT>(P, Pscale, pb + (size_t)(2 * c) * nrows, tile), c0[vtx[c]]);
        cmac(acc, fp_load<T, PT>(P, Pscale, pb + (size_t)(2 * c + 1) * nrows, tile), c0[nc + vtx[c]]);
      }
      __stcg(e0 + (size_t)alpha * n + v, acc);
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicExch(flags + blockIdx.x, base + 1u);
  }
  int p = 1;
  const int hx = Nx >> 1;
  for (int sw = 0; sw < sweeps; ++sw) {
    for (int colour = 0; colour < 2; ++colour, ++p) {
      if (threadIdx.x < 2 && nrb > 1 && alive) {
        int nb = b + (threadIdx.x == 0 ? -1 : 1);
        nb += nb < 0 ? nrb : (nb >= nrb ? -nrb : 0);
        const volatile unsigned* f = flags + rhs * nrb + nb;
        const unsigned want = base + (unsigned)p;
        unsigned it = 0;
        while ((int)(*f - want) < 0) {
          if (++it == FINE_SPIN_LIMIT) {
            atomicExch(sync + 2, 1u);
            alive = 0;
            break;
          }
        }
        __threadfence();
      }
      __syncthreads();
      for (int idx = threadIdx.x; idx < rows * hx; idx += blockDim.x) {
        const int t = t0 + idx / hx;
        const int x = 2 * (idx - (idx / hx) * hx) + ((t + colour) & 1);
        const int s = t * Nx + x;
        C h0, h1;
        hop_sum<T, C, true>(e0, e0 + n, U, t, x, Nt, Nx, n, h0, h1);
        __stcg(e0 + s, inv_diag * (r0[s] + T(0.5) * h0));
        __stcg(e0 + s + n, inv_diag * (r0[s + n] + T(0.5) * h1));
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        __threadfence();
        atomicExch(flags + blockIdx.x, base + (unsigned)p + 1u);
      }
    }
  }
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(sync + 4, 1u) == gridDim.x - 1) {
      sync[4] = 0;
      __threadfence();
      atomicExch(sync + 3, base + (unsigned)p);
    }
  }
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

cudaError_t launch_dslash_dag(const double2* in, double2* out, const double2* U, double diag, int Nt, int Nx, int R,
                              cudaStream_t st) {
  const int n = Nt * Nx;
  dim3 grid((n + 255) / 256, R);
  k_dslash_dag<<<grid, 256, 0, st>>>(in, out, U, diag, Nt, Nx);
  return cudaGetLastError();
}

template <typename Cin, typename Cout, typename T>
cudaError_t launch_dslash(const Cin* in, Cout* out, const Cout* b, const typename cplx<T>::type* U,
                          T diag, int Nt, int Nx, int R, cudaStream_t st, const T* diag_r) {
  const int n = Nt * Nx;
  if constexpr (std::is_same<Cin, float2>::value && std::is_same<Cout, float2>::value) {
    if ((Nx & 1) == 0) {
      dim3 grid((n / 2 + 255) / 256, R);
      k_dslash32x2<<<grid, 256, 0, st>>>(in, out, b, U, diag, diag_r, Nt, Nx);
      return cudaGetLastError();
    }
  }
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

// rows per block of the fused fine post-smoother for R right-hand sides: the
// fewest (a divisor of Nt) whose R Nt / rows blocks of 256 threads are at most
// two per SM and can all be resident; 0 when none (then the separate kernels
// run).  Prolongation is per site, so a block's rows need not be whole tiles.
template <typename T, typename PT>
int fine_post_rows(int Nt, int Nx, int a, int R) {
  // co-resident blocks of 256 threads and SM count, per device (several host
  // threads may ask at once, for GPUs of different kinds)
  static std::mutex mu;
  static std::map<int, std::pair<int, int>> per_device;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  int cap = 0, sms = 0;
  {
    std::lock_guard<std::mutex> lock(mu);
    auto it = per_device.find(dev);
    if (it == per_device.end()) {
      int occ = 0, coop = 0;
      if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess ||
          cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
          cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_fine_post<T, PT>, 256, 0) != cudaSuccess) {
        cudaGetLastError();
        cap = 0;
      } else {
        cap = coop ? sms * occ : 0;
      }
      it = per_device.emplace(dev, std::make_pair(cap, sms)).first;
    }
    cap = it->second.first;
    sms = it->second.second;
  }
  if (cap <= 0 || (Nx & 1) || Nt % a || Nx % a) return 0;
  const long limit = std::min<long>(std::min<long>(cap, 2L * sms), FINE_MAX_BLOCKS);
  for (int rows = 1; rows <= Nt; ++rows) {
    if (Nt % rows) continue;
    if ((long)R * (Nt / rows) <= limit) return rows;
  }
  return 0;
}

template <typename T, typename PT>
cudaError_t launch_fine_post(const typename cplx<T>::type* ec, typename cplx<T>::type* e,
                             const typename cplx<T>::type* r, const PT* P, const float* Pscale,
                             const typename cplx<T>::type* U, T inv_diag, const T* inv_diag_r, int Nt, int Nx, int a,
                             int sweeps, int R, unsigned* flags, unsigned* sync, cudaStream_t st) {
  const int rows = fine_post_rows<T, PT>(Nt, Nx, a, R);
  if (rows <= 0) return cudaErrorNotSupported;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(R * (Nt / rows));
  cfg.blockDim = dim3(256);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_fine_post<T, PT>, ec, e, r, P, Pscale, U, inv_diag, inv_diag_r, Nt, Nx, a,
                            sweeps, rows, flags, sync);
}

template int fine_post_rows<double, double2>(int, int, int, int);
template int fine_post_rows<float, __half2>(int, int, int, int);
template cudaError_t launch_fine_post<double, double2>(const double2*, double2*, const double2*, const double2*,
                                                       const float*, const double2*, double, const double*, int, int,
                                                       int, int, int, unsigned*, unsigned*, cudaStream_t);
template cudaError_t launch_fine_post<float, __half2>(const float2*, float2*, const float2*, const __half2*,
                                                      const float*, const float2*, float, const float*, int, int, int,
                                                      int, int, unsigned*, unsigned*, cudaStream_t);

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
