// Transfer kernels between level l and level l+1 (Sec. 2; interpolator of
// Sec. 4.1, Eq. (16)).
//
// P_l is stored per tile T = (p, q) (the a x a sites whose non-vertex rows take
// their formula from basket W(p, q)) as a dense [8][nrows] column-major block:
// column 2c + beta is corner c (= 2 di + dj, vertex (p+di, q+dj)), spin beta;
// row 2(l-1) + alpha is in-tile site l = i*a + j (l >= 1), spin alpha.  The
// tile's vertex (l = 0) interpolates by identity and is not stored.
//   FP64: double2 entries.  FP32 path: __half2 entries times one FP32 scale per tile.
#include "kernels.h"

namespace {

constexpr int RESTRICT_UNROLL = 4;

template <typename T, typename PT>
__device__ __forceinline__ typename cplx<T>::type p_load(const PT* P, const float* scale, size_t idx, int tile);

template <>
__device__ __forceinline__ double2 p_load<double, double2>(const double2* P, const float*, size_t idx, int) {
  return P[idx];
}
template <>
__device__ __forceinline__ float2 p_load<float, __half2>(const __half2* P, const float* scale, size_t idx, int tile) {
  return h2c<float>(P[idx], scale[tile]);
}

// e_fine = P e_coarse.  One thread per (tile, row); rows nrows, nrows+1 are the
// vertex's two spins (identity).  A row's columns are the corners of its
// basket (row_basket: the tile's own under the tile rule).
template <typename T, typename PT>
__global__ void __launch_bounds__(256)
k_prolong(const typename cplx<T>::type* __restrict__ ec, typename cplx<T>::type* __restrict__ ef,
          const PT* __restrict__ P, const float* __restrict__ Pscale,
          int Nxf, int a, int nrows, int Np, int Nq, int own) {
  using C = typename cplx<T>::type;
  const int rows_tot = nrows + 2;
  const int nc = Np * Nq;
  const int nf = nc * a * a;
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= nc * rows_tot) return;
  const int tile = g / rows_tot;
  const int lr = g - tile * rows_tot;
  const int p = tile / Nq, q = tile - (tile / Nq) * Nq;
  const C* e0 = ec + (size_t)blockIdx.y * 2 * nc;
  C* f0 = ef + (size_t)blockIdx.y * 2 * nf;
  if (lr >= nrows) {
    const int alpha = lr - nrows;
    f0[(size_t)alpha * nf + (p * a) * Nxf + q * a] = e0[(size_t)alpha * nc + tile];
    return;
  }
  const int l = (lr >> 1) + 1, alpha = lr & 1;
  const int i = l / a, j = l - (l / a) * a;
  int dp, dq;
  row_basket(own, p, q, i, j, dp, dq);
  const int pb = (p + dp < 0) ? Np - 1 : p + dp, qb = (q + dq < 0) ? Nq - 1 : q + dq;
  const int p1 = (pb + 1 == Np) ? 0 : pb + 1, q1 = (qb + 1 == Nq) ? 0 : qb + 1;
  const int vtx[4] = {pb * Nq + qb, pb * Nq + q1, p1 * Nq + qb, p1 * Nq + q1};
  C acc = czero<C>();
  const size_t base = (size_t)tile * 8 * nrows + lr;
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    cmac(acc, p_load<T, PT>(P, Pscale, base + (size_t)(2 * c) * nrows, tile), e0[vtx[c]]);
    cmac(acc, p_load<T, PT>(P, Pscale, base + (size_t)(2 * c + 1) * nrows, tile), e0[nc + vtx[c]]);
  }
  f0[(size_t)alpha * nf + (p * a + i) * Nxf + q * a + j] = acc;
}

// k_prolong for many right-hand sides: a thread loads its row's 8 entries of P
// once and applies them to RB right-hand sides (blockIdx.y selects the group);
// per right-hand side the arithmetic of k_prolong.
template <typename T, typename PT, int RB>
__global__ void __launch_bounds__(256)
k_prolong_rb(const typename cplx<T>::type* __restrict__ ec, typename cplx<T>::type* __restrict__ ef,
             const PT* __restrict__ P, const float* __restrict__ Pscale,
             int Nxf, int a, int nrows, int Np, int Nq, int own, int R) {
  using C = typename cplx<T>::type;
  const int rows_tot = nrows + 2;
  const int nc = Np * Nq;
  const int nf = nc * a * a;
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= nc * rows_tot) return;
  const int r0 = blockIdx.y * RB;
  const int nr = R - r0 < RB ? R - r0 : RB;
  const int tile = g / rows_tot;
  const int lr = g - tile * rows_tot;
  const int p = tile / Nq, q = tile - (tile / Nq) * Nq;
  if (lr >= nrows) {
    const int alpha = lr - nrows;
#pragma unroll
    for (int k = 0; k < RB; ++k)
      if (k < nr)
        ef[(size_t)(r0 + k) * 2 * nf + (size_t)alpha * nf + (p * a) * Nxf + q * a] =
            ec[(size_t)(r0 + k) * 2 * nc + (size_t)alpha * nc + tile];
    return;
  }
  const int l = (lr >> 1) + 1, alpha = lr & 1;
  const int i = l / a, j = l - (l / a) * a;
  int dp, dq;
  row_basket(own, p, q, i, j, dp, dq);
  const int pb = (p + dp < 0) ? Np - 1 : p + dp, qb = (q + dq < 0) ? Nq - 1 : q + dq;
  const int p1 = (pb + 1 == Np) ? 0 : pb + 1, q1 = (qb + 1 == Nq) ? 0 : qb + 1;
  const int vtx[4] = {pb * Nq + qb, pb * Nq + q1, p1 * Nq + qb, p1 * Nq + q1};
  const size_t base = (size_t)tile * 8 * nrows + lr;
  C pc[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) pc[c] = p_load<T, PT>(P, Pscale, base + (size_t)c * nrows, tile);
  const size_t fo = (size_t)alpha * nf + (p * a + i) * Nxf + q * a + j;
#pragma unroll
  for (int k = 0; k < RB; ++k) {
    if (k < nr) {
      const C* e0 = ec + (size_t)(r0 + k) * 2 * nc;
      C acc = czero<C>();
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        cmac(acc, pc[2 * c], e0[vtx[c]]);
        cmac(acc, pc[2 * c + 1], e0[nc + vtx[c]]);
      }
      ef[(size_t)(r0 + k) * 2 * nf + fo] = acc;
    }
  }
}

// e_coarse = P^H e_fine.  One warp per coarse vertex v = (p, q): it gathers the
// rows of the four tiles that have v as a corner (tile (p-di, q-dj) sees v as
// its corner c = 2 di + dj) plus v's own fine site (identity row), so every
// coarse value is written once and no atomics are needed.  The 4 nrows
// (corner, row) pairs are dealt round-robin to the lanes; the lanes' partial
// sums (two complex values) are combined by a reduce-scatter, after which lane
// 8 h2 + 16 h1 holds real component q = 2 h1 + h2 of (e_c0, e_c1) and stores it.
template <typename T, typename PT>
__global__ void __launch_bounds__(256)
k_restrict(const typename cplx<T>::type* __restrict__ ef, typename cplx<T>::type* __restrict__ ec,
           const PT* __restrict__ P, const float* __restrict__ Pscale,
           int Nxf, int a, int nrows, int Np, int Nq) {
  using C = typename cplx<T>::type;
  const int nc = Np * Nq;
  const int nf = nc * a * a;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= nc) return;                      // whole warps leave together
  const int p = warp / Nq, q = warp - (warp / Nq) * Nq;
  const C* f0 = ef + (size_t)blockIdx.y * 2 * nf;
  C acc0 = czero<C>(), acc1 = czero<C>();
  // the lane's first RESTRICT_UNROLL pairs: all loads issued, then the
  // arithmetic (a <= 4 needs at most 4 pairs per lane); further pairs (larger
  // tiles) one at a time, in the same order
  C fv[RESTRICT_UNROLL], pa[RESTRICT_UNROLL], pb[RESTRICT_UNROLL];
#pragma unroll
  for (int u = 0; u < RESTRICT_UNROLL; ++u) {
    const int idx = lane + 32 * u;
    if (idx < 4 * nrows) {
      const int c = idx / nrows, lr = idx - c * nrows;
      const int di = c >> 1, dj = c & 1;
      const int pT = (p - di < 0) ? Np - 1 : p - di;
      const int qT = (q - dj < 0) ? Nq - 1 : q - dj;
      const int tile = pT * Nq + qT;
      const size_t base = (size_t)tile * 8 * nrows + (size_t)(2 * c) * nrows;
      const int l = (lr >> 1) + 1, alpha = lr & 1;
      const int i = l / a, j = l - (l / a) * a;
      fv[u] = f0[(size_t)alpha * nf + (pT * a + i) * Nxf + qT * a + j];
      pa[u] = p_load<T, PT>(P, Pscale, base + lr, tile);
      pb[u] = p_load<T, PT>(P, Pscale, base + nrows + lr, tile);
    } else {
      fv[u] = pa[u] = pb[u] = czero<C>();
    }
  }
#pragma unroll
  for (int u = 0; u < RESTRICT_UNROLL; ++u) {
    cmacc(acc0, pa[u], fv[u]);
    cmacc(acc1, pb[u], fv[u]);
  }
  for (int idx = lane + 32 * RESTRICT_UNROLL; idx < 4 * nrows; idx += 32) {
    const int c = idx / nrows, lr = idx - c * nrows;
    const int di = c >> 1, dj = c & 1;
    const int pT = (p - di < 0) ? Np - 1 : p - di;
    const int qT = (q - dj < 0) ? Nq - 1 : q - dj;
    const int tile = pT * Nq + qT;
    const size_t base = (size_t)tile * 8 * nrows + (size_t)(2 * c) * nrows;
    const int l = (lr >> 1) + 1, alpha = lr & 1;
    const int i = l / a, j = l - (l / a) * a;
    const C f = f0[(size_t)alpha * nf + (pT * a + i) * Nxf + qT * a + j];
    cmacc(acc0, p_load<T, PT>(P, Pscale, base + lr, tile), f);
    cmacc(acc1, p_load<T, PT>(P, Pscale, base + nrows + lr, tile), f);
  }
  const bool h1 = (lane & 16) != 0, h2 = (lane & 8) != 0;
  T ka = h1 ? acc1.x : acc0.x, kb = h1 ? acc1.y : acc0.y;
  ka += __shfl_xor_sync(0xffffffffu, h1 ? acc0.x : acc1.x, 16);
  kb += __shfl_xor_sync(0xffffffffu, h1 ? acc0.y : acc1.y, 16);
  T sq = h2 ? kb : ka;
  sq += __shfl_xor_sync(0xffffffffu, h2 ? ka : kb, 8);
#pragma unroll
  for (int o = 4; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
  if ((lane & 7) == 0) {
    const int sv = (p * a) * Nxf + q * a;
    const T* fv = reinterpret_cast<const T*>(f0 + (h1 ? nf : 0) + sv);
    T* e0 = reinterpret_cast<T*>(ec + (size_t)blockIdx.y * 2 * nc + (h1 ? nc : 0) + warp);
    e0[h2] = sq + fv[h2];
  }
}

// k_restrict for many right-hand sides: a warp's lanes load their entries of P
// once (a <= 4: at most RESTRICT_UNROLL pairs per lane) and apply them to RB
// right-hand sides (blockIdx.y selects the group); per right-hand side the
// loads, the accumulation order and the reduce-scatter of k_restrict, so every
// right-hand side gets that kernel's result bit for bit.
template <typename T, typename PT, int RB>
__global__ void __launch_bounds__(256)
k_restrict_rb(const typename cplx<T>::type* __restrict__ ef, typename cplx<T>::type* __restrict__ ec,
              const PT* __restrict__ P, const float* __restrict__ Pscale,
              int Nxf, int a, int nrows, int Np, int Nq, int R) {
  using C = typename cplx<T>::type;
  const int nc = Np * Nq;
  const int nf = nc * a * a;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= nc) return;                      // whole warps leave together
  const int r0 = blockIdx.y * RB;
  const int nr = R - r0 < RB ? R - r0 : RB;
  const int p = warp / Nq, q = warp - (warp / Nq) * Nq;
  C pa[RESTRICT_UNROLL], pb[RESTRICT_UNROLL];
  size_t fidx[RESTRICT_UNROLL];
  bool use[RESTRICT_UNROLL];
#pragma unroll
  for (int u = 0; u < RESTRICT_UNROLL; ++u) {
    const int idx = lane + 32 * u;
    use[u] = idx < 4 * nrows;
    pa[u] = pb[u] = czero<C>();
    fidx[u] = 0;
    if (use[u]) {
      const int c = idx / nrows, lr = idx - c * nrows;
      const int di = c >> 1, dj = c & 1;
      const int pT = (p - di < 0) ? Np - 1 : p - di;
      const int qT = (q - dj < 0) ? Nq - 1 : q - dj;
      const int tile = pT * Nq + qT;
      const size_t base = (size_t)tile * 8 * nrows + (size_t)(2 * c) * nrows;
      const int l = (lr >> 1) + 1, alpha = lr & 1;
      const int i = l / a, j = l - (l / a) * a;
      fidx[u] = (size_t)alpha * nf + (pT * a + i) * Nxf + qT * a + j;
      pa[u] = p_load<T, PT>(P, Pscale, base + lr, tile);
      pb[u] = p_load<T, PT>(P, Pscale, base + nrows + lr, tile);
    }
  }
  const bool h1 = (lane & 16) != 0, h2 = (lane & 8) != 0;
  const int sv = (p * a) * Nxf + q * a;
#pragma unroll 1
  for (int k = 0; k < nr; ++k) {
    const C* f0 = ef + (size_t)(r0 + k) * 2 * nf;
    C fv[RESTRICT_UNROLL];
#pragma unroll
    for (int u = 0; u < RESTRICT_UNROLL; ++u) fv[u] = use[u] ? f0[fidx[u]] : czero<C>();
    C acc0 = czero<C>(), acc1 = czero<C>();
#pragma unroll
    for (int u = 0; u < RESTRICT_UNROLL; ++u) {
      cmacc(acc0, pa[u], fv[u]);
      cmacc(acc1, pb[u], fv[u]);
    }
    T ka = h1 ? acc1.x : acc0.x, kb = h1 ? acc1.y : acc0.y;
    ka += __shfl_xor_sync(0xffffffffu, h1 ? acc0.x : acc1.x, 16);
    kb += __shfl_xor_sync(0xffffffffu, h1 ? acc0.y : acc1.y, 16);
    T sq = h2 ? kb : ka;
    sq += __shfl_xor_sync(0xffffffffu, h2 ? ka : kb, 8);
#pragma unroll
    for (int o = 4; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
    if ((lane & 7) == 0) {
      const T* fvv = reinterpret_cast<const T*>(f0 + (h1 ? nf : 0) + sv);
      T* e0 = reinterpret_cast<T*>(ec + (size_t)(r0 + k) * 2 * nc + (h1 ? nc : 0) + warp);
      e0[h2] = sq + fvv[h2];
    }
  }
}

// e_coarse = P^H e_fine for any ownership rule: one warp per coarse vertex
// v = (p, q) walks the F sites of the four baskets that have v as a corner c
// (W(p - di, q - dj)) and takes the rows each basket owns (row_basket), plus
// v's own fine site (identity row).  Used for the first-lex rule, whose rows of
// a tile come from up to three baskets (k_restrict covers the tile rule).
template <typename T, typename PT>
__global__ void __launch_bounds__(256)
k_restrict_owned(const typename cplx<T>::type* __restrict__ ef, typename cplx<T>::type* __restrict__ ec,
                 const PT* __restrict__ P, const float* __restrict__ Pscale,
                 int Nxf, int a, int nrows, int Np, int Nq, int own) {
  using C = typename cplx<T>::type;
  const int nc = Np * Nq;
  const int nf = nc * a * a;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= nc) return;                      // whole warps leave together
  const int p = warp / Nq, q = warp - (warp / Nq) * Nq;
  const C* f0 = ef + (size_t)blockIdx.y * 2 * nf;
  const int nb = (a + 1) * (a + 1);
  C acc0 = czero<C>(), acc1 = czero<C>();
  for (int idx = lane; idx < 4 * nb; idx += 32) {
    const int c = idx / nb, s = idx - c * nb;
    const int i = s / (a + 1), j = s - (s / (a + 1)) * (a + 1);
    if ((i == 0 || i == a) && (j == 0 || j == a)) continue;          // corners
    const int pB = (p - (c >> 1) < 0) ? Np - 1 : p - (c >> 1);
    const int qB = (q - (c & 1) < 0) ? Nq - 1 : q - (c & 1);
    const int it = (i == a) ? 0 : i, jt = (j == a) ? 0 : j;
    const int pT = (i == a) ? ((pB + 1 == Np) ? 0 : pB + 1) : pB;
    const int qT = (j == a) ? ((qB + 1 == Nq) ? 0 : qB + 1) : qB;
    int dp, dq;
    row_basket(own, pT, qT, it, jt, dp, dq);
    const int po = (pT + dp < 0) ? Np - 1 : pT + dp, qo = (qT + dq < 0) ? Nq - 1 : qT + dq;
    if (po != pB || qo != qB) continue;                              // another basket's row
    const int tile = pT * Nq + qT, l = it * a + jt;
    const size_t base = (size_t)tile * 8 * nrows + (size_t)(2 * c) * nrows + 2 * (l - 1);
    const int site = (pT * a + it) * Nxf + qT * a + jt;
#pragma unroll
    for (int sigma = 0; sigma < 2; ++sigma) {
      const C f = f0[(size_t)sigma * nf + site];
      cmacc(acc0, p_load<T, PT>(P, Pscale, base + sigma, tile), f);
      cmacc(acc1, p_load<T, PT>(P, Pscale, base + nrows + sigma, tile), f);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    acc0.x += __shfl_xor_sync(0xffffffffu, acc0.x, o);
    acc0.y += __shfl_xor_sync(0xffffffffu, acc0.y, o);
    acc1.x += __shfl_xor_sync(0xffffffffu, acc1.x, o);
    acc1.y += __shfl_xor_sync(0xffffffffu, acc1.y, o);
  }
  if (lane == 0) {
    const int sv = (p * a) * Nxf + q * a;
    C* e0 = ec + (size_t)blockIdx.y * 2 * nc;
    e0[warp] = acc0 + f0[sv];
    e0[nc + warp] = acc1 + f0[nf + sv];
  }
}

// Level structure as the transfer kernels index it: role of every site (0
// vertex, 1 edge, 2 interior) and the basket p Nq + q whose formula its row
// takes (row_basket; a vertex: its own tile's basket).
__global__ void k_structure(int Nt, int Nx, int a, int own, int* __restrict__ role, int* __restrict__ owner) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= Nt * Nx) return;
  const int t = s / Nx, x = s - (s / Nx) * Nx;
  const int Np = Nt / a, Nq = Nx / a;
  const int p = t / a, q = x / a, i = t - p * a, j = x - q * a;
  const bool ti = i == 0, xj = j == 0;
  role[s] = (ti && xj) ? 0 : (ti != xj ? 1 : 2);
  int dp = 0, dq = 0;
  if (!(ti && xj)) row_basket(own, p, q, i, j, dp, dq);
  const int pb = (p + dp < 0) ? Np - 1 : p + dp, qb = (q + dq < 0) ? Nq - 1 : q + dq;
  owner[s] = pb * Nq + qb;
}

}  // namespace

cudaError_t launch_structure(int Nt, int Nx, int a, int own, int* role, int* owner, cudaStream_t st) {
  k_structure<<<(Nt * Nx + 255) / 256, 256, 0, st>>>(Nt, Nx, a, own, role, owner);
  return cudaGetLastError();
}

template <typename T, typename PT>
cudaError_t launch_prolong(const typename cplx<T>::type* ec, typename cplx<T>::type* ef, const PT* P,
                           const float* Pscale, int Nxf, int a, int Np, int Nq, int R, cudaStream_t st, int own) {
  const int nrows = 2 * (a * a - 1);
  const int total = Np * Nq * (nrows + 2);
  constexpr int RB = sizeof(T) == 8 ? 4 : 8;       // right-hand sides per group of the blocked kernel
  if (R >= 4) {
    dim3 grid((total + 255) / 256, (R + RB - 1) / RB);
    k_prolong_rb<T, PT, RB><<<grid, 256, 0, st>>>(ec, ef, P, Pscale, Nxf, a, nrows, Np, Nq, own, R);
    return cudaGetLastError();
  }
  dim3 grid((total + 255) / 256, R);
  k_prolong<T, PT><<<grid, 256, 0, st>>>(ec, ef, P, Pscale, Nxf, a, nrows, Np, Nq, own);
  return cudaGetLastError();
}

template <typename T, typename PT>
cudaError_t launch_restrict(const typename cplx<T>::type* ef, typename cplx<T>::type* ec, const PT* P,
                            const float* Pscale, int Nxf, int a, int Np, int Nq, int R, cudaStream_t st, int own) {
  const int nrows = 2 * (a * a - 1);
  const int nc = Np * Nq;
  constexpr int RB = sizeof(T) == 8 ? 4 : 8;       // right-hand sides per group of the blocked kernel
  if (own == OWN_TILE && R >= 4 && 4 * nrows <= 32 * RESTRICT_UNROLL) {
    dim3 grid((nc * 32 + 255) / 256, (R + RB - 1) / RB);
    k_restrict_rb<T, PT, RB><<<grid, 256, 0, st>>>(ef, ec, P, Pscale, Nxf, a, nrows, Np, Nq, R);
    return cudaGetLastError();
  }
  dim3 grid((nc * 32 + 255) / 256, R);
  if (own == OWN_TILE) k_restrict<T, PT><<<grid, 256, 0, st>>>(ef, ec, P, Pscale, Nxf, a, nrows, Np, Nq);
  else k_restrict_owned<T, PT><<<grid, 256, 0, st>>>(ef, ec, P, Pscale, Nxf, a, nrows, Np, Nq, own);
  return cudaGetLastError();
}

template cudaError_t launch_prolong<double, double2>(const double2*, double2*, const double2*, const float*, int,
                                                     int, int, int, int, cudaStream_t, int);
template cudaError_t launch_prolong<float, __half2>(const float2*, float2*, const __half2*, const float*, int, int,
                                                    int, int, int, cudaStream_t, int);
template cudaError_t launch_restrict<double, double2>(const double2*, double2*, const double2*, const float*, int,
                                                      int, int, int, int, cudaStream_t, int);
template cudaError_t launch_restrict<float, __half2>(const float2*, float2*, const __half2*, const float*, int,
                                                     int, int, int, int, cudaStream_t, int);
