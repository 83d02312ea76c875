// Coarse-level kernels: the Galerkin operator A_l = P^H A_{l-1} P in block-stencil
// form, its multicolour block Gauss-Seidel smoother (8 or 16 colours, see
// colour_site), and the coarsest direct solve.
//
// A_l is stored as K blocks of 2x2 complex per coarse site, [K][4][n] (entry
// 2 alpha + beta, site-major within an entry plane, so consecutive threads read
// consecutive sites).  Offsets are the canonical (dt mod Nt, dx mod Nx) pairs,
// sorted, with (0, 0) first.  FP32 path: __half2 entries with one FP32 scale per
// block ([K][n]).
#include <cooperative_groups.h>

#include <algorithm>
#include <cstdlib>
#include <map>
#include <mutex>
#include <vector>

#include "kernels.h"

namespace cg = cooperative_groups;

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
    cmac(y0, b_load<T, BT>(B, Bs, k, 0, n, v), x0);
    cmac(y0, b_load<T, BT>(B, Bs, k, 1, n, v), x1);
    cmac(y1, b_load<T, BT>(B, Bs, k, 2, n, v), x0);
    cmac(y1, b_load<T, BT>(B, Bs, k, 3, n, v), x1);
  }
  C* o = out + roff;
  if (b) {
    y0 = b[roff + v] - y0;
    y1 = b[roff + n + v] - y1;
  }
  o[v] = y0;
  o[n + v] = y1;
}

// The same for many right-hand sides: a thread keeps site v's blocks in
// registers for RB right-hand sides at a time (blockIdx.y selects the group), so
// each 2x2 block is loaded once per RB right-hand sides instead of once per
// right-hand side.  Per right-hand side the arithmetic of k_coarse_apply.
template <typename T, typename BT, int RB>
__global__ void __launch_bounds__(256)
k_coarse_apply_rb(const typename cplx<T>::type* __restrict__ in, typename cplx<T>::type* __restrict__ out,
                  const typename cplx<T>::type* __restrict__ b, const BT* __restrict__ B,
                  const float* __restrict__ Bs, Offsets off, int Nt, int Nx, int R) {
  using C = typename cplx<T>::type;
  const int n = Nt * Nx;
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  const int r0 = blockIdx.y * RB;
  const int nr = R - r0 < RB ? R - r0 : RB;
  const int t = v / Nx, x = v - (v / Nx) * Nx;
  C y0[RB], y1[RB];
#pragma unroll
  for (int j = 0; j < RB; ++j) y0[j] = y1[j] = czero<C>();
  for (int k = 0; k < off.K; ++k) {
    int tw = t + off.dt[k]; tw -= (tw >= Nt) ? Nt : 0;
    int xw = x + off.dx[k]; xw -= (xw >= Nx) ? Nx : 0;
    const int w = tw * Nx + xw;
    const C b00 = b_load<T, BT>(B, Bs, k, 0, n, v), b01 = b_load<T, BT>(B, Bs, k, 1, n, v);
    const C b10 = b_load<T, BT>(B, Bs, k, 2, n, v), b11 = b_load<T, BT>(B, Bs, k, 3, n, v);
#pragma unroll
    for (int j = 0; j < RB; ++j) {
      if (j < nr) {
        const C* i0 = in + (size_t)(r0 + j) * 2 * n;
        const C x0 = i0[w], x1 = i0[n + w];
        cmac(y0[j], b00, x0);
        cmac(y0[j], b01, x1);
        cmac(y1[j], b10, x0);
        cmac(y1[j], b11, x1);
      }
    }
  }
#pragma unroll
  for (int j = 0; j < RB; ++j) {
    if (j < nr) {
      const size_t roff = (size_t)(r0 + j) * 2 * n;
      C a0 = y0[j], a1 = y1[j];
      if (b) {
        a0 = b[roff + v] - a0;
        a1 = b[roff + n + v] - a1;
      }
      out[roff + v] = a0;
      out[roff + n + v] = a1;
    }
  }
}

// Colour-major copies of a smoothed level's operator (built in setup): for
// colour c, site j of the colour (colour_site / site_colour below, m = n / ncol
// sites per colour) and off-diagonal offset k = 1..K-1:
//   Bc[((c (K-1) + k - 1) m + j) 4 + e]   the 2x2 block entries e = 2 alpha + beta,
//   Sc[(c (K-1) + k - 1) m + j]           its FP32 scale (FP16 copy only),
//   Dc[(c m + j) 4 + e]                    the inverse of the diagonal block.
// The four entries of a block are contiguous and consecutive sites of a colour
// are adjacent, so the lanes of a warp read whole sectors.
template <typename T, typename BT>
__device__ __forceinline__ void cm_block(const BT* __restrict__ Bc, const float* __restrict__ Sc, size_t blk,
                                         typename cplx<T>::type (&b)[4]);
template <>
__device__ __forceinline__ void cm_block<double, double2>(const double2* __restrict__ Bc, const float*, size_t blk,
                                                          double2 (&b)[4]) {
#pragma unroll
  for (int e = 0; e < 4; ++e) b[e] = Bc[blk * 4 + e];
}
template <>
__device__ __forceinline__ void cm_block<float, __half2>(const __half2* __restrict__ Bc, const float* __restrict__ Sc,
                                                         size_t blk, float2 (&b)[4]) {
  const uint4 q = *reinterpret_cast<const uint4*>(Bc + blk * 4);      // 16 bytes: the block's 4 half2
  const float sc = Sc[blk];
  const __half2* h = reinterpret_cast<const __half2*>(&q);
#pragma unroll
  for (int e = 0; e < 4; ++e) b[e] = h2c<float>(h[e], sc);
}

// Block Gauss-Seidel update of site j of colour c on A e = r by a group of LPS
// lanes: lane g of the group forms A_{v, v+off_k} e_{v+off_k} for
// k = 1 + g, 1 + g + LPS, ...; the group sums its lanes (xor-shuffle tree, fixed
// order) and its lane 0 writes
// e_v = A_vv^{-1} (r_v - sum_{k >= 1} A_{v, v+off_k} e_{v+off_k}).
// ESMEM: e0 points to shared memory (one block owns the whole level); otherwise
// e0 is global and neighbour values are read through L2 (ld.global.cg) so that
// the kernel is also correct when other thread blocks of a cluster updated them.
// The loop over a lane's offsets is unrolled so that all its loads are in flight
// together; r_v and A_vv^{-1} are loaded before the reduction.
template <typename T, typename BT, int LPS, bool ESMEM>
__device__ __forceinline__ void gs_site(typename cplx<T>::type* __restrict__ e0,
                                        const typename cplx<T>::type* __restrict__ r0,
                                        const BT* __restrict__ Bc, const float* __restrict__ Sc,
                                        const typename cplx<T>::type* __restrict__ Dc, const Offsets& off,
                                        int Nt, int Nx, int ncol, int colour, int j, int g, bool valid) {
  // every lane of the warp calls this (the shuffles need all 32); lanes of
  // groups without a site pass valid = false and only take part in the shuffles
  using C = typename cplx<T>::type;
  const int n = Nt * Nx;
  const int m = n / ncol;
  if (!valid) j = 0;
  int t, x;
  colour_site(ncol, colour, j, Nx, t, x);
  const int v = t * Nx + x;
  const int K1 = off.K - 1;
  C rv0 = czero<C>(), rv1 = czero<C>(), d[4] = {czero<C>(), czero<C>(), czero<C>(), czero<C>()};
  if (valid && g == 0) {
    rv0 = r0[v]; rv1 = r0[n + v];
#pragma unroll
    for (int e = 0; e < 4; ++e) d[e] = Dc[((size_t)colour * m + j) * 4 + e];
  }
  // all of this lane's loads first (they are independent), then the arithmetic
  constexpr int IT = (GS_MAX_OFFDIAG + LPS - 1) / LPS;
  C xv[IT][2], bb[IT][4];
#pragma unroll
  for (int i = 0; i < IT; ++i) {
    const int k = 1 + g + i * LPS;
    if (valid && k < off.K) {
      int tw = t + off.dt[k]; tw -= (tw >= Nt) ? Nt : 0;
      int xw = x + off.dx[k]; xw -= (xw >= Nx) ? Nx : 0;
      const int w = tw * Nx + xw;
      if constexpr (ESMEM) { xv[i][0] = e0[w]; xv[i][1] = e0[n + w]; }
      else { xv[i][0] = __ldcg(e0 + w); xv[i][1] = __ldcg(e0 + n + w); }
      cm_block<T, BT>(Bc, Sc, ((size_t)colour * K1 + (k - 1)) * m + j, bb[i]);
    } else {
      xv[i][0] = xv[i][1] = czero<C>();
      bb[i][0] = bb[i][1] = bb[i][2] = bb[i][3] = czero<C>();
    }
  }
  C s0 = czero<C>(), s1 = czero<C>();
#pragma unroll
  for (int i = 0; i < IT; ++i) {
    cmac(s0, bb[i][0], xv[i][0]);
    cmac(s0, bb[i][1], xv[i][1]);
    cmac(s1, bb[i][2], xv[i][0]);
    cmac(s1, bb[i][3], xv[i][1]);
  }
#pragma unroll
  for (int o = LPS / 2; o > 0; o >>= 1) {
    s0.x += __shfl_xor_sync(0xffffffffu, s0.x, o);
    s0.y += __shfl_xor_sync(0xffffffffu, s0.y, o);
    s1.x += __shfl_xor_sync(0xffffffffu, s1.x, o);
    s1.y += __shfl_xor_sync(0xffffffffu, s1.y, o);
  }
  if (valid && g == 0) {
    const C a0 = rv0 - s0, a1 = rv1 - s1;
    const C y0 = cmul(d[0], a0) + cmul(d[1], a1), y1 = cmul(d[2], a0) + cmul(d[3], a1);
    if constexpr (ESMEM) { e0[v] = y0; e0[n + v] = y1; }
    else { __stcg(e0 + v, y0); __stcg(e0 + n + v, y1); }
  }
}

// gs_site for the same site of nr <= RB right-hand sides (e0, r0: the first
// one's vectors, the others rs elements apart): the lanes load the site's
// blocks and diagonal inverse once and the neighbour values of all nr
// right-hand sides together, then form each right-hand side's update in
// gs_site's order (same sums, same shuffle tree), so every right-hand side
// gets gs_site's result bit for bit.
template <typename T, typename BT, int LPS, int RB>
__device__ __forceinline__ void gs_site_rb(typename cplx<T>::type* __restrict__ e0,
                                           const typename cplx<T>::type* __restrict__ r0, size_t rs, int nr,
                                           const BT* __restrict__ Bc, const float* __restrict__ Sc,
                                           const typename cplx<T>::type* __restrict__ Dc, const Offsets& off,
                                           int Nt, int Nx, int ncol, int colour, int j, int g, bool valid) {
  using C = typename cplx<T>::type;
  const int n = Nt * Nx;
  const int m = n / ncol;
  if (!valid) j = 0;
  int t, x;
  colour_site(ncol, colour, j, Nx, t, x);
  const int v = t * Nx + x;
  const int K1 = off.K - 1;
  C d[4] = {czero<C>(), czero<C>(), czero<C>(), czero<C>()};
  C rv[RB][2];
#pragma unroll
  for (int q = 0; q < RB; ++q) rv[q][0] = rv[q][1] = czero<C>();
  if (valid && g == 0) {
#pragma unroll
    for (int e = 0; e < 4; ++e) d[e] = Dc[((size_t)colour * m + j) * 4 + e];
#pragma unroll
    for (int q = 0; q < RB; ++q)
      if (q < nr) { rv[q][0] = r0[q * rs + v]; rv[q][1] = r0[q * rs + n + v]; }
  }
  constexpr int IT = (GS_MAX_OFFDIAG + LPS - 1) / LPS;
  C bb[IT][4], xv[RB][IT][2];
#pragma unroll
  for (int i = 0; i < IT; ++i) {
    const int k = 1 + g + i * LPS;
    if (valid && k < off.K) {
      int tw = t + off.dt[k]; tw -= (tw >= Nt) ? Nt : 0;
      int xw = x + off.dx[k]; xw -= (xw >= Nx) ? Nx : 0;
      const int w = tw * Nx + xw;
#pragma unroll
      for (int q = 0; q < RB; ++q) {
        if (q < nr) { xv[q][i][0] = __ldcg(e0 + q * rs + w); xv[q][i][1] = __ldcg(e0 + q * rs + n + w); }
        else xv[q][i][0] = xv[q][i][1] = czero<C>();
      }
      cm_block<T, BT>(Bc, Sc, ((size_t)colour * K1 + (k - 1)) * m + j, bb[i]);
    } else {
#pragma unroll
      for (int q = 0; q < RB; ++q) xv[q][i][0] = xv[q][i][1] = czero<C>();
      bb[i][0] = bb[i][1] = bb[i][2] = bb[i][3] = czero<C>();
    }
  }
#pragma unroll
  for (int q = 0; q < RB; ++q) {
    C s0 = czero<C>(), s1 = czero<C>();
#pragma unroll
    for (int i = 0; i < IT; ++i) {
      cmac(s0, bb[i][0], xv[q][i][0]);
      cmac(s0, bb[i][1], xv[q][i][1]);
      cmac(s1, bb[i][2], xv[q][i][0]);
      cmac(s1, bb[i][3], xv[q][i][1]);
    }
#pragma unroll
    for (int o = LPS / 2; o > 0; o >>= 1) {
      s0.x += __shfl_xor_sync(0xffffffffu, s0.x, o);
      s0.y += __shfl_xor_sync(0xffffffffu, s0.y, o);
      s1.x += __shfl_xor_sync(0xffffffffu, s1.x, o);
      s1.y += __shfl_xor_sync(0xffffffffu, s1.y, o);
    }
    if (valid && g == 0 && q < nr) {
      const C a0 = rv[q][0] - s0, a1 = rv[q][1] - s1;
      const C y0 = cmul(d[0], a0) + cmul(d[1], a1), y1 = cmul(d[2], a0) + cmul(d[3], a1);
      __stcg(e0 + q * rs + v, y0);
      __stcg(e0 + q * rs + n + v, y1);
    }
  }
}

// Lanes per site: 8 in FP64 (B300's FP64 pipe is narrow: the sites of a colour
// spread over many SMs, three offsets per lane), 32 in FP32 (all offsets of a
// site loaded at once: the clustered sweep is latency bound).
template <typename T> struct GsLanes { static constexpr int value = 32; };
template <> struct GsLanes<double> { static constexpr int value = 8; };

// One colour of the multicolour sweep (sites of colour c as colour_site maps
// them); LPS lanes per site.
template <typename T, typename BT>
__global__ void __launch_bounds__(256)
k_coarse_colour(typename cplx<T>::type* __restrict__ e, const typename cplx<T>::type* __restrict__ r,
                const BT* __restrict__ B, const float* __restrict__ Bs,
                const typename cplx<T>::type* __restrict__ Dinv, Offsets off, int Nt, int Nx, int ncol, int colour) {
  constexpr int LPS = GsLanes<T>::value;
  const int n = Nt * Nx;
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  const int idx = tid / LPS;
  const int g = tid & (LPS - 1);
  const bool valid = idx < n / ncol;
  const size_t roff = (size_t)blockIdx.y * 2 * n;
  gs_site<T, BT, LPS, false>(e + roff, r + roff, B, Bs, Dinv, off, Nt, Nx, ncol, colour, idx, g, valid);
}

// All colours of `sweeps` sweeps in one launch: one thread block cluster per
// right-hand side, LPS lanes per site, and a cluster barrier (barrier.cluster,
// release/acquire) between colours.  Same arithmetic as k_coarse_colour.
template <typename T, typename BT>
__global__ void __launch_bounds__(1024)
k_coarse_sweeps_cluster(typename cplx<T>::type* __restrict__ e, const typename cplx<T>::type* __restrict__ r,
                        const BT* __restrict__ B, const float* __restrict__ Bs,
                        const typename cplx<T>::type* __restrict__ Dinv, Offsets off, int Nt, int Nx, int ncol,
                        int sweeps) {
  constexpr int LPS = GsLanes<T>::value;
  cg::cluster_group cluster = cg::this_cluster();
  const int n = Nt * Nx;
  const int per_colour = n / ncol;
  const int rank = (int)cluster.block_rank();
  const int csize = (int)cluster.num_blocks();
  const int rhs = blockIdx.x / csize;
  const size_t roff = (size_t)rhs * 2 * n;
  const int g = threadIdx.x & (LPS - 1);
  const int gpb = blockDim.x / LPS;
  const int stride = csize * gpb;
  for (int sw = 0; sw < sweeps; ++sw) {
    for (int colour = 0; colour < ncol; ++colour) {
      // every group runs the same number of iterations (shuffles stay converged)
      for (int base = 0; base < per_colour; base += stride) {
        const int idx = base + rank * gpb + threadIdx.x / LPS;
        const bool valid = idx < per_colour;
        gs_site<T, BT, LPS, false>(e + roff, r + roff, B, Bs, Dinv, off, Nt, Nx, ncol, colour, idx, g, valid);
      }
      cluster.sync();
    }
  }
}

// Software barrier over all blocks of a cooperative launch (co-residency is
// guaranteed by the launch).  sync = {arrival count, generation, error}: a
// block's thread 0 reads the generation, arrives, and either (last arrival)
// resets the count and advances the generation or waits for it to advance,
// at most GRID_SPIN_LIMIT polls (about a second); on time-out it records the
// error and the block returns false (its caller stops).  The fences order the
// block's global stores before its arrival and the other blocks' stores before
// its reads (which go through L2).
constexpr unsigned GRID_SPIN_LIMIT = 1u << 23;
#ifndef AMAMG_GRID_SLEEP_NS
#define AMAMG_GRID_SLEEP_NS 64     // back-off between polls of the generation word
#endif
__device__ __forceinline__ bool grid_barrier(unsigned* sync, unsigned nblocks) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* gen = sync + 1;
    const unsigned g = *gen;
    __threadfence();
    ok = 1;
    if (atomicAdd(sync, 1u) == nblocks - 1) {
      sync[0] = 0;
      __threadfence();
      atomicExch(sync + 1, g + 1);
    } else {
      unsigned it = 0;
      while (*gen == g) {
        if (++it == GRID_SPIN_LIMIT) {
          atomicExch(sync + 2, 1u);
          ok = 0;
          break;
        }
        if (AMAMG_GRID_SLEEP_NS > 0) __nanosleep(AMAMG_GRID_SLEEP_NS);
      }
    }
    __threadfence();
  }
  __syncthreads();
  return ok != 0;
}

// All colours of `sweeps` sweeps in one cooperative launch spread over the
// whole GPU: work units (right-hand side, site of the colour) are dealt to
// groups of LPS lanes across all blocks, the colour phases are separated by
// grid_barrier.  Same arithmetic per site as k_coarse_colour.  For FP64, whose
// pipe is narrow on this GPU, this spreads a colour over every SM instead of
// the 16 SMs of one cluster.
#ifndef AMAMG_GRID_LPS64
#define AMAMG_GRID_LPS64 8         // lanes per site of the FP64 grid sweep
#endif
template <typename T> struct GridLanes { static constexpr int value = 32; };
template <> struct GridLanes<double> { static constexpr int value = AMAMG_GRID_LPS64; };

// RB > 1: a work unit is a site and a group of RB right-hand sides (gs_site_rb:
// the site's blocks loaded once per group), with each right-hand side's
// result unchanged.
template <typename T, typename BT, int RB>
__global__ void __launch_bounds__(256)
k_coarse_sweeps_grid(typename cplx<T>::type* __restrict__ e, const typename cplx<T>::type* __restrict__ r,
                     const BT* __restrict__ B, const float* __restrict__ Bs,
                     const typename cplx<T>::type* __restrict__ Dinv, Offsets off, int Nt, int Nx, int ncol,
                     int sweeps, int R, unsigned* sync) {
  constexpr int LPS = GridLanes<T>::value;
  const int n = Nt * Nx;
  const int per_colour = n / ncol;
  const int ngrp = (R + RB - 1) / RB;
  const long units = (long)ngrp * per_colour;
  const int g = threadIdx.x & (LPS - 1);
  const int gpb = blockDim.x / LPS;
  const long stride = (long)gridDim.x * gpb;
  for (int sw = 0; sw < sweeps; ++sw) {
    for (int colour = 0; colour < ncol; ++colour) {
      // every group runs the same number of iterations (shuffles stay converged)
      for (long base = 0; base < units; base += stride) {
        const long u = base + (long)blockIdx.x * gpb + threadIdx.x / LPS;
        const bool valid = u < units;
        const int grp = valid ? (int)(u / per_colour) : 0;
        const int idx = valid ? (int)(u - (long)grp * per_colour) : 0;
        const size_t roff = (size_t)grp * RB * 2 * n;
        if constexpr (RB == 1) {
          gs_site<T, BT, LPS, false>(e + roff, r + roff, B, Bs, Dinv, off, Nt, Nx, ncol, colour, idx, g, valid);
        } else {
          const int nr = R - grp * RB < RB ? R - grp * RB : RB;
          gs_site_rb<T, BT, LPS, RB>(e + roff, r + roff, (size_t)2 * n, nr, B, Bs, Dinv, off, Nt, Nx, ncol, colour,
                                     idx, g, valid);
        }
      }
      if (!grid_barrier(sync, gridDim.x)) return;
    }
  }
}

// All colours of `sweeps` sweeps in one cooperative launch in which block b of
// a right-hand side owns the sites j in [b cnt, (b+1) cnt) of every colour
// (colour-major numbering of colour_site: for 8 colours a segment of 8 cnt
// sites of one row, for 16 colours a strip of a 4-row band; the same ownership
// as k_coarse_sweeps_dsmem with more, smaller owners).  The block keeps its
// sites' r, diagonal inverses and (BSMEM) off-diagonal blocks in shared
// memory; e lives in global memory.  At start every block lists the other
// blocks that own a neighbour of one of its sites (the operator's offsets are
// symmetric, so these are also the blocks that read its sites).  Instead of a
// barrier over the whole grid, a block updates its sites of colour phase p
// once every listed block has published phase p - 1: no neighbour value it
// reads is stale, and no neighbour still reads a value it is about to
// overwrite.
//
// Split of a site's update around that wait.  When phase p starts, only the
// neighbours of the previous phase's colour can still change (all other
// colours were published at phase p - 2 or earlier, and none changes again
// before this block publishes phase p).  So a site's sum over offsets splits
// into an "early" part over every other offset, which needs no wait, and a
// "late" part over the at most S (4 or 8) offsets of the previous colour.
// The block has three roles:
//   early warps (LE lanes per site, several offsets per lane) form the early
//     sums of phase p + 1 into a double-buffered shared array while phase p
//     runs;
//   post warps (4 S lanes per site: S late slots for each of the four real
//     components of the 2x2 product) wait for phase p's release, load the
//     late neighbours, add the early sum, form
//     e_v = A_vv^{-1} (r_v - sum) and store it;
//   the synchronising warp polls the listed blocks' counters with acquire
//     loads, releases phase p through named barrier 1 (with the early warps'
//     sums of phase p), collects the post warps' stores through named barrier
//     2 and publishes with a release add.
// The early sums of phase p + 1 read only colours other than those of phases
// p and p + 1, which no block writes before this block publishes phase p + 1.
// Few lanes per site keep the FP64 instruction count of a phase low: on this
// GPU's narrow FP64 pipe it sets the time of the early sums and slows the post
// warps that share the pipe.  LE = 8 (four sites per warp, three offsets per
// lane) has the fewest FP64 instructions and is taken when several blocks
// share an SM; with one block per SM, LE = 16 (two sites per warp) spreads the
// early sums over two warps and measured faster (a warp's FP64 instructions
// issue on its own SM sub-partition).
// Phase counters are flags[block] = base + phases done, base = sync[3]
// (advanced by the last block to finish through the ticket sync[4]; every
// block sets its counter to base when it starts, before any neighbour can
// need a value above base).  Polls are bounded (OWNER_SPIN_LIMIT, about
// half a second); a block whose wait times out sets sync[2] and stops waiting,
// so the launch always ends.  withhold >= 0 names a block that never publishes
// (self-test of that time-out path; -1 in every normal launch).
// The sum over offsets is the same as in the other sweeps; its rounding order
// differs (early tree, then late tree).
constexpr unsigned OWNER_SPIN_LIMIT = 1u << 20;
constexpr int OWNER_EARLY_WARPS = 2;   // at most
constexpr int OWNER_POST_WARPS = 4;    // at most

__device__ __forceinline__ void bar_sync_n(int id, int n) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}
__device__ __forceinline__ void bar_arrive_n(int id, int n) {
  asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(n) : "memory");
}
__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void red_release_gpu_add(unsigned* p, unsigned v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Early sums of the warp's sites jb + (lane / LPS) < cnt of colour
// `colour` over their offsets not in lm (all offsets when !use_mask): lane g of
// a site's group takes offsets 1 + g, 1 + g + LPS, ...; the group's
// reduce-scatter leaves component q = 2 h1 + h2 of the sum in lanes with
// (h1, h2) = (bit 2, bit 1) of g, whose even lane writes out[4 jj + q].
template <typename T, typename BT, bool BSMEM, int LPS>
__device__ __forceinline__ void owner_early(const typename cplx<T>::type* __restrict__ e0, const BT* __restrict__ Bc,
                                            const float* __restrict__ Sc, const BT* bs, const float* ss,
                                            const unsigned* lm, bool use_mask, const Offsets& off, int Nt, int Nx,
                                            int ncol, int m, int K1, int cnt, int colour, int j0, int jb, int lane,
                                            T* out) {
  using C = typename cplx<T>::type;
  constexpr int IT = (GS_MAX_OFFDIAG + LPS - 1) / LPS;
  const int n = Nt * Nx;
  const int g = lane & (LPS - 1), jj = jb + lane / LPS;
  const bool valid = jj < cnt;
  const int jjc = valid ? jj : 0, j = j0 + jjc;
  const unsigned mask = use_mask ? lm[colour * cnt + jjc] : 0u;
  int t, x;
  colour_site(ncol, colour, j, Nx, t, x);
  C xv[IT][2], bb[IT][4];
#pragma unroll
  for (int it = 0; it < IT; ++it) {
    const int k = 1 + g + it * LPS;
    if (valid && k < off.K && !((mask >> (k - 1)) & 1u)) {
      int tw = t + off.dt[k]; tw -= (tw >= Nt) ? Nt : 0;
      int xw = x + off.dx[k]; xw -= (xw >= Nx) ? Nx : 0;
      const int w = tw * Nx + xw;
      xv[it][0] = __ldcg(e0 + w);
      xv[it][1] = __ldcg(e0 + n + w);
      if constexpr (BSMEM) {
        const int li = (colour * K1 + (k - 1)) * cnt + jj;
        if constexpr (sizeof(T) == 4) {
#pragma unroll
          for (int d = 0; d < 4; ++d) bb[it][d] = h2c<float>(bs[4 * li + d], ss[li]);
        } else {
#pragma unroll
          for (int d = 0; d < 4; ++d) bb[it][d] = to_c(bs[4 * li + d], T());
        }
      } else {
        cm_block<T, BT>(Bc, Sc, ((size_t)colour * K1 + (k - 1)) * m + j, bb[it]);
      }
    } else {
      xv[it][0] = xv[it][1] = czero<C>();
      bb[it][0] = bb[it][1] = bb[it][2] = bb[it][3] = czero<C>();
    }
  }
  C s0 = czero<C>(), s1 = czero<C>();
#pragma unroll
  for (int it = 0; it < IT; ++it) {
    cmac(s0, bb[it][0], xv[it][0]);
    cmac(s0, bb[it][1], xv[it][1]);
    cmac(s1, bb[it][2], xv[it][0]);
    cmac(s1, bb[it][3], xv[it][1]);
  }
  constexpr int o1 = LPS / 2, o2 = LPS / 4;
  const bool h1 = (g & o1) != 0, h2 = (g & o2) != 0;
  T ka = h1 ? s1.x : s0.x, kb = h1 ? s1.y : s0.y;
  ka += __shfl_xor_sync(0xffffffffu, h1 ? s0.x : s1.x, o1);
  kb += __shfl_xor_sync(0xffffffffu, h1 ? s0.y : s1.y, o1);
  T sq = h2 ? kb : ka;
  sq += __shfl_xor_sync(0xffffffffu, h2 ? ka : kb, o2);
#pragma unroll
  for (int o = o2 / 2; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
  if (valid && (g & (o2 - 1)) == 0) out[4 * jj + 2 * h1 + h2] = sq;
}

template <typename T, typename BT, bool BSMEM, int S, int LE>
__global__ void __launch_bounds__(32 * (OWNER_EARLY_WARPS + OWNER_POST_WARPS + 1), 1)
k_coarse_sweeps_owner(typename cplx<T>::type* __restrict__ e, const typename cplx<T>::type* __restrict__ r,
                      const BT* __restrict__ Bc, const float* __restrict__ Sc,
                      const typename cplx<T>::type* __restrict__ Dc, Offsets off, int Nt, int Nx, int ncol,
                      int sweeps, int cnt, int nearly, int late_half, unsigned* __restrict__ flags,
                      unsigned* __restrict__ sync, int withhold) {
  using C = typename cplx<T>::type;
  static_assert(S == 4 || S == 8, "late slots per component: 4 or 8");
  static_assert(LE == 8 || LE == 16, "early lanes per site: 8 or 16");
  constexpr int LPP = 4 * S, SPP = 32 / LPP;                 // post lanes per site, sites per post warp
  constexpr int SPE = 32 / LE;                               // sites per early warp
  const int n = Nt * Nx, m = n / ncol, K1 = off.K - 1;
  const int nbpr = m / cnt;                                  // owner blocks per right-hand side
  const int rhs = blockIdx.x / nbpr, b = blockIdx.x - rhs * nbpr;
  const int j0 = b * cnt;
  const int own = ncol * cnt;
  const int NT = blockDim.x;
  const int npost = NT / 32 - 1 - nearly;                    // warps: post, then early, then synchronising
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* rs = reinterpret_cast<C*>(smem_raw);                    // [ncol][cnt][2]
  C* ds = rs + 2 * own;                                      // [ncol][cnt][4]
  BT* bs = reinterpret_cast<BT*>(ds + 4 * own);              // [ncol][K1][cnt][4]   (BSMEM)
  T* pre = reinterpret_cast<T*>(bs + (BSMEM ? 4 * K1 * own : 0));   // [2][cnt][4] early sums
  unsigned* lm = reinterpret_cast<unsigned*>(pre + 8 * cnt);         // [ncol][cnt] late-offset bits
  float* ss = reinterpret_cast<float*>(lm + own);                    // [ncol][K1][cnt] (BSMEM, FP16)
  __shared__ unsigned bm[OWNER_MAX_BLOCKS / 32];             // blocks owning a neighbour
  __shared__ short wl[OWNER_MAX_WAIT];                       // ... as a list
  __shared__ int nwait;
  const size_t roff = (size_t)rhs * 2 * n;
  C* e0 = e + roff;
  const C* r0 = r + roff;
  const int words = (nbpr + 31) / 32;
  for (int i = threadIdx.x; i < words; i += NT) bm[i] = 0u;
  for (int i = threadIdx.x; i < own; i += NT) {
    const int c = i / cnt, j = j0 + (i - c * cnt);
    int t, x;
    colour_site(ncol, c, j, Nx, t, x);
    const int v = t * Nx + x;
    rs[2 * i] = r0[v]; rs[2 * i + 1] = r0[n + v];
#pragma unroll
    for (int d = 0; d < 4; ++d) ds[4 * i + d] = Dc[((size_t)c * m + j) * 4 + d];
    lm[i] = 0u;
  }
  if constexpr (BSMEM) {
    for (int i = threadIdx.x; i < K1 * own; i += NT) {
      const int ck = i / cnt, jj = i - ck * cnt;                // ck = c K1 + (k - 1)
      const size_t src = (size_t)ck * m + j0 + jj;
#pragma unroll
      for (int d = 0; d < 4; ++d) bs[4 * i + d] = Bc[src * 4 + d];
      if (Sc) ss[i] = Sc[src];
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < K1 * own; i += NT) {
    const int site = i / K1, k = 1 + (i - site * K1);
    const int c = site / cnt, j = j0 + (site - c * cnt);
    int t, x;
    colour_site(ncol, c, j, Nx, t, x);
    int tw = t + off.dt[k]; tw -= (tw >= Nt) ? Nt : 0;
    int xw = x + off.dx[k]; xw -= (xw >= Nx) ? Nx : 0;
    int cw, jw;
    site_colour(ncol, tw, xw, Nx, cw, jw);
    const int ob = jw / cnt;
    if (ob != b) atomicOr(&bm[ob >> 5], 1u << (ob & 31));
    if (cw == (c == 0 ? ncol - 1 : c - 1)) atomicOr(&lm[site], 1u << (k - 1));
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    // compact the bitmap into wl (warp 0, word order, so the list is sorted)
    int total = 0;
    for (int w0 = 0; w0 < words; w0 += 32) {
      const unsigned word = (w0 + (int)threadIdx.x < words) ? bm[w0 + threadIdx.x] : 0u;
      int cnt_w = __popc(word), incl = cnt_w;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if ((int)threadIdx.x >= o) incl += y;
      }
      int pos = total + incl - cnt_w;
      unsigned bits = word;
      while (bits) {
        const int bit = __ffs(bits) - 1;
        bits &= bits - 1;
        if (pos < OWNER_MAX_WAIT) wl[pos] = (short)((w0 + threadIdx.x) * 32 + bit);
        ++pos;
      }
      total += __shfl_sync(0xffffffffu, incl, 31);
    }
    if (threadIdx.x == 0) {
      nwait = total < OWNER_MAX_WAIT ? total : OWNER_MAX_WAIT;
      if (total > OWNER_MAX_WAIT) atomicExch(sync + 2, 1u);
    }
  }
  const unsigned base = *reinterpret_cast<volatile unsigned*>(sync + 3);
  __syncthreads();
  const int phases = sweeps * ncol;
  const int n_done = 32 * (npost + 1);                       // barrier 2: post warps + synchronising warp

  if (warp == npost + nearly) {
    // synchronising warp
    bool alive = true;
    // the block's counter starts the launch at base (a block withheld in a
    // self-test is behind by a launch's phases until here)
    if (lane == 0) *reinterpret_cast<volatile unsigned*>(flags + blockIdx.x) = base;
    for (int p = 0; p < phases; ++p) {
      if (p > 0 && alive) {
        const unsigned want = base + (unsigned)p;
        bool late = false;
        for (int q = lane; q < nwait && !late; q += 32) {
          const unsigned* f = flags + rhs * nbpr + wl[q];
          unsigned it = 0;
          while ((int)(ld_acquire_gpu(f) - want) < 0) {
            if (++it == OWNER_SPIN_LIMIT) { late = true; break; }
          }
        }
        if (__any_sync(0xffffffffu, late)) {
          if (lane == 0) atomicExch(sync + 2, 1u);
          alive = false;
        }
      }
      __syncwarp();
      bar_arrive_n(1, NT);                                   // phase p may start
      bar_sync_n(2, n_done);                                 // the post warps stored phase p
      if (lane == 0 && (int)blockIdx.x != withhold) red_release_gpu_add(flags + blockIdx.x, 1u);
    }
    if (lane == 0) {
      __threadfence();
      if (atomicAdd(sync + 4, 1u) == gridDim.x - 1) {
        sync[4] = 0;
        __threadfence();
        atomicExch(sync + 3, base + (unsigned)phases);
      }
    }
    return;
  }

  if (warp >= npost) {
    // early warps: phase 0 in full (nothing is late yet), then phase p + 1
    // during phase p
    const int ew = warp - npost;
    for (int jb = ew * SPE; jb < cnt; jb += nearly * SPE)
      owner_early<T, BT, BSMEM, LE>(e0, Bc, Sc, bs, ss, lm, false, off, Nt, Nx, ncol, m, K1, cnt, 0, j0, jb, lane, pre);
    for (int p = 0; p < phases; ++p) {
      bar_sync_n(1, NT);
      if (p + 1 < phases) {
        T* out = pre + 4 * cnt * ((p + 1) & 1);
        for (int jb = ew * SPE; jb < cnt; jb += nearly * SPE)
          owner_early<T, BT, BSMEM, LE>(e0, Bc, Sc, bs, ss, lm, true, off, Nt, Nx, ncol, m, K1, cnt, (p + 1) % ncol,
                                    j0, jb, lane, out);
      }
    }
    return;
  }

  // post warps
  const int sub = lane / LPP, slot = lane & (S - 1), q = (lane % LPP) / S;
  const bool h1 = (q & 2) != 0, h2 = (q & 1) != 0;
  const int gb = sub * LPP;                                  // first lane of this site's group
  for (int p = 0; p < phases; ++p) {
    const int colour = p % ncol;
    const T* prep = pre + 4 * cnt * (p & 1);
    bool first = true;
    for (int jb = warp * SPP; jb < cnt; jb += npost * SPP) {
      // address work first; the first sites' runs before the wait
      const int jj = jb + sub;
      const bool valid = jj < cnt;
      const int jjc = valid ? jj : 0;
      const int i = colour * cnt + jjc, j = j0 + jjc;
      const unsigned mask = p > 0 ? lm[i] : 0u;
      int t, x;
      colour_site(ncol, colour, j, Nx, t, x);
      const bool has = valid && slot < __popc(mask);
      int w = 0;
      C bA = czero<C>(), bB = czero<C>();                    // row h1 of the late block
      if (has) {
        const int k = 1 + (int)__fns(mask, 0u, slot + 1);
        int tw = t + off.dt[k]; tw -= (tw >= Nt) ? Nt : 0;
        int xw = x + off.dx[k]; xw -= (xw >= Nx) ? Nx : 0;
        w = tw * Nx + xw;
        if constexpr (BSMEM) {
          const int li = (colour * K1 + (k - 1)) * cnt + jj;
          if constexpr (sizeof(T) == 4) {
            bA = h2c<float>(bs[4 * li + 2 * h1], ss[li]);
            bB = h2c<float>(bs[4 * li + 2 * h1 + 1], ss[li]);
          } else {
            bA = to_c(bs[4 * li + 2 * h1], T());
            bB = to_c(bs[4 * li + 2 * h1 + 1], T());
          }
        } else {
          C bb[4];
          cm_block<T, BT>(Bc, Sc, ((size_t)colour * K1 + (k - 1)) * m + j, bb);
          bA = h1 ? bb[2] : bb[0];
          bB = h1 ? bb[3] : bb[1];
        }
      }
      if (first) {
        bar_sync_n(1, NT);                                   // neighbours published p - 1; early sums ready
        first = false;
      }
      T cq = T(0);
      if (has) {
        const C x0 = __ldcg(e0 + w), x1 = __ldcg(e0 + n + w);
        // real part (h2 = 0): bA.x x0.x - bA.y x0.y + bB.x x1.x - bB.y x1.y;
        // imaginary part (h2 = 1): bA.x x0.y + bA.y x0.x + bB.x x1.y + bB.y x1.x
        T ca = bA.x * (h2 ? x0.y : x0.x);
        ca = fma(h2 ? bA.y : -bA.y, h2 ? x0.x : x0.y, ca);
        T cb = bB.x * (h2 ? x1.y : x1.x);
        cb = fma(h2 ? bB.y : -bB.y, h2 ? x1.x : x1.y, cb);
        cq = ca + cb;
      }
      for (int o = late_half; o > 0; o >>= 1) cq += __shfl_xor_sync(0xffffffffu, cq, o);
      const T sq = prep[4 * jjc + q] + cq;
      // a = r - s, component q here; every lane gathers all four, and the
      // four slot-0 lanes of the site each form one real component of
      // e = [d0 d1; d2 d3] a  (e_0 = d0 a_0 + d1 a_1, e_1 = d2 a_0 + d3 a_1)
      const T aq = reinterpret_cast<const T*>(rs)[4 * i + q] - sq;
      const T A0 = __shfl_sync(0xffffffffu, aq, gb);
      const T A1 = __shfl_sync(0xffffffffu, aq, gb + S);
      const T A2 = __shfl_sync(0xffffffffu, aq, gb + 2 * S);
      const T A3 = __shfl_sync(0xffffffffu, aq, gb + 3 * S);
      if (valid && slot == 0) {
        const C dA = ds[4 * i + (h1 ? 2 : 0)], dB = ds[4 * i + (h1 ? 3 : 1)];
        const T p0 = h2 ? A1 : A0, p1 = h2 ? A0 : A1, q0 = h2 ? A3 : A2, q1 = h2 ? A2 : A3;
        T oa = dA.x * p0;
        oa = fma(h2 ? dA.y : -dA.y, p1, oa);
        T ob = dB.x * q0;
        ob = fma(h2 ? dB.y : -dB.y, q1, ob);
        const int v = t * Nx + x;
        __stcg(reinterpret_cast<T*>(e0) + 2 * (v + (h1 ? n : 0)) + h2, oa + ob);
      }
    }
    bar_arrive_n(2, n_done);                                 // this warp's stores of phase p are done
  }
}

// All colours of `sweeps` sweeps in one launch on a 16-block thread-block
// cluster per right-hand side, the level distributed over the cluster's shared
// memory.  Block q of the cluster owns sites j in [q per, (q+1) per) of every
// colour (per = n / (16 ncol)): it keeps their e, r and diagonal inverses (and, with
// BSMEM, their off-diagonal blocks) in its shared memory for the whole launch.
// A colour phase reads neighbour values from the owning blocks' shared memory
// (distributed shared memory), writes its own sites locally, and ends with a
// cluster barrier (release/acquire), so no phase touches L2 for e.
template <typename T, typename BT, bool BSMEM>
__global__ void __launch_bounds__(512)
k_coarse_sweeps_dsmem(typename cplx<T>::type* __restrict__ e, const typename cplx<T>::type* __restrict__ r,
                      const BT* __restrict__ Bc, const float* __restrict__ Sc,
                      const typename cplx<T>::type* __restrict__ Dc, Offsets off, int Nt, int Nx, int ncol,
                      int sweeps) {
  using C = typename cplx<T>::type;
  constexpr int LPS = 8;
  constexpr int IT = (GS_MAX_OFFDIAG + LPS - 1) / LPS;
  cg::cluster_group cluster = cg::this_cluster();
  const int q = (int)cluster.block_rank();
  const int rhs = blockIdx.x / DSMEM_CLUSTER;
  const int n = Nt * Nx, m = n / ncol, per = m / DSMEM_CLUSTER, K1 = off.K - 1;
  const int own = ncol * per;                             // sites this block owns (n / 16)
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* es = reinterpret_cast<C*>(smem_raw);                 // [ncol colours][per][2]
  C* rs = es + 2 * own;                                   // [ncol][per][2]
  C* ds = rs + 2 * own;                                   // [ncol][per][4]
  BT* bs = reinterpret_cast<BT*>(ds + 4 * own);           // [ncol][K1][per][4]      (BSMEM)
  float* ss = reinterpret_cast<float*>(bs + (BSMEM ? 4 * K1 * own : 0));   // [ncol][K1][per]  (BSMEM, FP16)
  const size_t roff = (size_t)rhs * 2 * n;
  C* e0 = e + roff;
  const C* r0 = r + roff;
  // load this block's part of the level
  for (int i = threadIdx.x; i < own; i += blockDim.x) {
    const int c = i / per, jj = i - (i / per) * per, j = q * per + jj;
    int t, x;
    colour_site(ncol, c, j, Nx, t, x);
    const int v = t * Nx + x;
    es[2 * i] = e0[v]; es[2 * i + 1] = e0[n + v];
    rs[2 * i] = r0[v]; rs[2 * i + 1] = r0[n + v];
#pragma unroll
    for (int d = 0; d < 4; ++d) ds[4 * i + d] = Dc[((size_t)c * m + j) * 4 + d];
  }
  if constexpr (BSMEM) {
    for (int i = threadIdx.x; i < K1 * own; i += blockDim.x) {
      const int ck = i / per, jj = i - (i / per) * per;               // ck = c K1 + (k - 1)
      const size_t src = (size_t)ck * m + q * per + jj;
#pragma unroll
      for (int d = 0; d < 4; ++d) bs[4 * i + d] = Bc[src * 4 + d];
      if (Sc) ss[i] = Sc[src];
    }
  }
  cluster.sync();
  const int g = threadIdx.x & (LPS - 1);
  const int groups = blockDim.x / LPS;
  for (int sw = 0; sw < sweeps; ++sw) {
    for (int colour = 0; colour < ncol; ++colour) {
      for (int base = 0; base < per; base += groups) {
        const int jj = base + threadIdx.x / LPS;
        const bool valid = jj < per;
        const int j = q * per + (valid ? jj : 0);
        int t, x;
        colour_site(ncol, colour, j, Nx, t, x);
        C xv[IT][2], bb[IT][4];
#pragma unroll
        for (int it = 0; it < IT; ++it) {
          const int k = 1 + g + it * LPS;
          if (valid && k < off.K) {
            int tw = t + off.dt[k]; tw -= (tw >= Nt) ? Nt : 0;
            int xw = x + off.dx[k]; xw -= (xw >= Nx) ? Nx : 0;
            int cw, jw;
            site_colour(ncol, tw, xw, Nx, cw, jw);
            const int qw = jw / per, jjw = jw - qw * per;
            const C* rem = cluster.map_shared_rank(es, qw);
            xv[it][0] = rem[2 * (cw * per + jjw)];
            xv[it][1] = rem[2 * (cw * per + jjw) + 1];
            if constexpr (BSMEM) {
              const int li = (colour * K1 + (k - 1)) * per + jj;
              if constexpr (sizeof(T) == 4) {
#pragma unroll
                for (int d = 0; d < 4; ++d) bb[it][d] = h2c<float>(bs[4 * li + d], ss[li]);
              } else {
#pragma unroll
                for (int d = 0; d < 4; ++d) bb[it][d] = to_c(bs[4 * li + d], T());
              }
            } else {
              cm_block<T, BT>(Bc, Sc, ((size_t)colour * K1 + (k - 1)) * m + j, bb[it]);
            }
          } else {
            xv[it][0] = xv[it][1] = czero<C>();
            bb[it][0] = bb[it][1] = bb[it][2] = bb[it][3] = czero<C>();
          }
        }
        C s0 = czero<C>(), s1 = czero<C>();
#pragma unroll
        for (int it = 0; it < IT; ++it) {
          cmac(s0, bb[it][0], xv[it][0]);
          cmac(s0, bb[it][1], xv[it][1]);
          cmac(s1, bb[it][2], xv[it][0]);
          cmac(s1, bb[it][3], xv[it][1]);
        }
#pragma unroll
        for (int o = LPS / 2; o > 0; o >>= 1) {
          s0.x += __shfl_xor_sync(0xffffffffu, s0.x, o);
          s0.y += __shfl_xor_sync(0xffffffffu, s0.y, o);
          s1.x += __shfl_xor_sync(0xffffffffu, s1.x, o);
          s1.y += __shfl_xor_sync(0xffffffffu, s1.y, o);
        }
        if (valid && g == 0) {
          const int i = colour * per + jj;
          const C a0 = rs[2 * i] - s0, a1 = rs[2 * i + 1] - s1;
          es[2 * i] = cmul(ds[4 * i], a0) + cmul(ds[4 * i + 1], a1);
          es[2 * i + 1] = cmul(ds[4 * i + 2], a0) + cmul(ds[4 * i + 3], a1);
        }
      }
      cluster.sync();
    }
  }
  // write this block's sites back (no block reads remote shared memory after the last barrier)
  for (int i = threadIdx.x; i < own; i += blockDim.x) {
    const int c = i / per, jj = i - (i / per) * per, j = q * per + jj;
    int t, x;
    colour_site(ncol, c, j, Nx, t, x);
    const int v = t * Nx + x;
    e0[v] = es[2 * i];
    e0[n + v] = es[2 * i + 1];
  }
}

// y_r = Ainv x_r for the coarsest level: dense FP64 complex matrix, row-major,
// nd x nd; vectors are contiguous nd-element arrays (the [2][Nt][Nx] layout
// flattened).  One warp per row; the row is read once for all RR right-hand
// sides; four independent row loads per lane are in flight.
template <typename Cv, int RR>
__global__ void __launch_bounds__(256)
k_dense_gemv(const double2* __restrict__ A, const Cv* __restrict__ x, Cv* __restrict__ y, int nd) {
  const int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (row >= nd) return;
  double2 acc[RR];
#pragma unroll
  for (int r = 0; r < RR; ++r) acc[r] = make_double2(0.0, 0.0);
  const double2* a = A + (size_t)row * nd;
  int j = lane;
  for (; j + 96 < nd; j += 128) {
    double2 aj[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) aj[u] = __ldcs(a + j + 32 * u);
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int r = 0; r < RR; ++r) cmac(acc[r], aj[u], to_c(x[(size_t)r * nd + j + 32 * u], double()));
  }
  for (; j < nd; j += 32) {
    const double2 aj = a[j];
#pragma unroll
    for (int r = 0; r < RR; ++r) cmac(acc[r], aj, to_c(x[(size_t)r * nd + j], double()));
  }
#pragma unroll
  for (int r = 0; r < RR; ++r) {
    double re = acc[r].x, im = acc[r].y;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      re += __shfl_xor_sync(0xffffffffu, re, o);
      im += __shfl_xor_sync(0xffffffffu, im, o);
    }
    if (lane == 0) y[(size_t)r * nd + row] = to_c(make_double2(re, im), typename real_of<Cv>::type());
  }
}

// Mixed-precision V-cycle: y_r = Ainv32 x_r with the FP32 rounding of the FP64
// inverse (the factorisation itself is FP64); FP32 arithmetic.  One warp per
// row; a lane reads two complex entries per 16-byte load and keeps eight such
// loads in flight (the 2048 x 2048 matrix of the 256^2 hierarchy is 33.5 MB,
// read once per V-cycle: the kernel is bound by bytes in flight, not FLOPs).
// nd is even (two spins per site) and rows start 16-byte aligned.
template <int RR>
__global__ void __launch_bounds__(256)
k_dense_gemv32(const float2* __restrict__ A, const float2* __restrict__ x, float2* __restrict__ y, int nd) {
  const int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (row >= nd) return;
  float2 acc[RR];
#pragma unroll
  for (int r = 0; r < RR; ++r) acc[r] = make_float2(0.f, 0.f);
  const float4* a4 = reinterpret_cast<const float4*>(A + (size_t)row * nd);
  const int nq = nd >> 1;                       // 16-byte pairs per row
  int q = lane;
  for (; q + 32 * 7 < nq; q += 32 * 8) {
    float4 aq[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) aq[u] = __ldg(a4 + q + 32 * u);
#pragma unroll
    for (int u = 0; u < 8; ++u)
#pragma unroll
      for (int r = 0; r < RR; ++r) {
        const float4 xq = __ldg(reinterpret_cast<const float4*>(x + (size_t)r * nd) + q + 32 * u);
        cmac(acc[r], make_float2(aq[u].x, aq[u].y), make_float2(xq.x, xq.y));
        cmac(acc[r], make_float2(aq[u].z, aq[u].w), make_float2(xq.z, xq.w));
      }
  }
  for (; q < nq; q += 32) {
    const float4 aq = __ldg(a4 + q);
#pragma unroll
    for (int r = 0; r < RR; ++r) {
      const float4 xq = __ldg(reinterpret_cast<const float4*>(x + (size_t)r * nd) + q);
      cmac(acc[r], make_float2(aq.x, aq.y), make_float2(xq.x, xq.y));
      cmac(acc[r], make_float2(aq.z, aq.w), make_float2(xq.z, xq.w));
    }
  }
#pragma unroll
  for (int r = 0; r < RR; ++r) {
    float re = acc[r].x, im = acc[r].y;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      re += __shfl_xor_sync(0xffffffffu, re, o);
      im += __shfl_xor_sync(0xffffffffu, im, o);
    }
    if (lane == 0) y[(size_t)r * nd + row] = make_float2(re, im);
  }
}

}  // namespace

template <typename T, typename BT>
cudaError_t launch_coarse_apply(const typename cplx<T>::type* in, typename cplx<T>::type* out,
                                const typename cplx<T>::type* b, const BT* B, const float* Bs,
                                const Offsets& off, int Nt, int Nx, int R, cudaStream_t st) {
  const int n = Nt * Nx;
  if (R >= 4) {
    // blocks loaded once per group of right-hand sides
    constexpr int RB = sizeof(T) == 8 ? 4 : 8;
    dim3 grid((n + 255) / 256, (R + RB - 1) / RB);
    k_coarse_apply_rb<T, BT, RB><<<grid, 256, 0, st>>>(in, out, b, B, Bs, off, Nt, Nx, R);
    return cudaGetLastError();
  }
  dim3 grid((n + 255) / 256, R);
  k_coarse_apply<T, BT><<<grid, 256, 0, st>>>(in, out, b, B, Bs, off, Nt, Nx);
  return cudaGetLastError();
}

template <typename T, typename BT>
cudaError_t launch_coarse_colour(typename cplx<T>::type* e, const typename cplx<T>::type* r, const BT* B,
                                 const float* Bs, const typename cplx<T>::type* Dinv, const Offsets& off,
                                 int Nt, int Nx, int ncol, int colour, int R, cudaStream_t st) {
  const long threads = (long)(Nt * Nx / ncol) * GsLanes<T>::value;
  const int bs = sizeof(T) == 8 ? 32 : 256;      // FP64: spread the colour over many SMs
  dim3 grid((unsigned)((threads + bs - 1) / bs), R);
  k_coarse_colour<T, BT><<<grid, bs, 0, st>>>(e, r, B, Bs, Dinv, off, Nt, Nx, ncol, colour);
  return cudaGetLastError();
}

int cluster_sweep_threads(int n, int ncol) {
  // FP32 sweep: 32 lanes per site, at most 16 sites per warp and colour
  const long per_colour = n / ncol;
  long warps = (per_colour + CLUSTER_BLOCKS - 1) / CLUSTER_BLOCKS;
  if (warps > 32) {
    if (per_colour > (long)CLUSTER_BLOCKS * 32 * 16) return 1 << 30;   // too large: per-colour launches
    warps = 32;
  }
  return (int)(warps < 1 ? 32 : warps * 32);
}

template <typename T, typename BT>
cudaError_t launch_coarse_sweeps_cluster(typename cplx<T>::type* e, const typename cplx<T>::type* r, const BT* B,
                                         const float* Bs, const typename cplx<T>::type* Dinv, const Offsets& off,
                                         int Nt, int Nx, int ncol, int sweeps, int R, cudaStream_t st) {
  const int bs = cluster_sweep_threads(Nt * Nx, ncol);
  if (bs > 1024) return cudaErrorInvalidValue;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(CLUSTER_BLOCKS * R);
  cfg.blockDim = dim3(bs);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = CLUSTER_BLOCKS;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_coarse_sweeps_cluster<T, BT>, e, r, B, Bs, Dinv, off, Nt, Nx, ncol, sweeps);
}

size_t dsmem_sweep_bytes(int n, int K, size_t cbytes, bool bsmem, size_t bt_bytes) {
  const size_t own = (size_t)n / DSMEM_CLUSTER;            // sites per block
  size_t b = own * (2 + 2 + 4) * cbytes;
  if (bsmem) b += own * (K - 1) * (4 * bt_bytes + 4);
  return b;
}

// Grid sweep: GRID_SWEEP_THREADS threads per block (GRID_SWEEP_THREADS / LPS
// sites per block and pass), as many blocks as the widest colour needs, at most the blocks that
// can be co-resident (cooperative launch).
#ifndef AMAMG_GRID_THREADS
#define AMAMG_GRID_THREADS 64
#endif
constexpr int GRID_SWEEP_THREADS = AMAMG_GRID_THREADS;
constexpr int GRID_RB = 4;       // right-hand sides per work unit of the grid sweep from 4 on
template <typename T, typename BT>
int grid_sweep_blocks(int n, int ncol, int R) {
  // co-resident blocks of the grid sweep variant for R (right-hand sides in
  // groups of GRID_RB from GRID_RB on), per device (several host threads may ask)
  static std::mutex mu;
  static std::map<std::pair<int, int>, int> cap;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return 0; }
  const int rb = R >= GRID_RB ? GRID_RB : 1;
  int c;
  {
    std::lock_guard<std::mutex> lock(mu);
    auto it = cap.find({dev, rb});
    if (it == cap.end()) {
      int sms = 0, occ = 0, coop = 0;
      const void* kern = rb == 1 ? (const void*)k_coarse_sweeps_grid<T, BT, 1>
                                 : (const void*)k_coarse_sweeps_grid<T, BT, GRID_RB>;
      if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess ||
          cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
          cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, GRID_SWEEP_THREADS, 0) != cudaSuccess) {
        cudaGetLastError();
        c = 0;
      } else {
        c = coop ? sms * occ : 0;
      }
      cap[{dev, rb}] = c;
    } else {
      c = it->second;
    }
  }
  if (c <= 0) return 0;
  const long groups = (long)((R + rb - 1) / rb) * (n / ncol);
  const long want = (groups * GridLanes<T>::value + GRID_SWEEP_THREADS - 1) / GRID_SWEEP_THREADS;
  return (int)(want < c ? want : c);
}

template <typename T, typename BT>
cudaError_t launch_coarse_sweeps_grid(typename cplx<T>::type* e, const typename cplx<T>::type* r, const BT* B,
                                      const float* Bs, const typename cplx<T>::type* Dinv, const Offsets& off,
                                      int Nt, int Nx, int ncol, int sweeps, int R, unsigned* sync, cudaStream_t st) {
  const int nb = grid_sweep_blocks<T, BT>(Nt * Nx, ncol, R);
  if (nb <= 0) return cudaErrorNotSupported;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(nb);
  cfg.blockDim = dim3(GRID_SWEEP_THREADS);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (R >= GRID_RB)
    return cudaLaunchKernelEx(&cfg, k_coarse_sweeps_grid<T, BT, GRID_RB>, e, r, B, Bs, Dinv, off, Nt, Nx, ncol,
                              sweeps, R, sync);
  return cudaLaunchKernelEx(&cfg, k_coarse_sweeps_grid<T, BT, 1>, e, r, B, Bs, Dinv, off, Nt, Nx, ncol, sweeps, R,
                            sync);
}

// Owner sweep configuration for a level: the fewest sites per block and colour
// (cnt, a divisor of m = n / ncol, at least OWNER_MIN_CNT) whose R m / cnt
// blocks can all be resident (cooperative launch) and whose neighbour-owner
// lists fit OWNER_MAX_WAIT; enough early warps (4 sites each) and post warps
// (2 or 1 sites each) for the block's sites of a colour, up to
// OWNER_EARLY_WARPS and OWNER_POST_WARPS (more sites take several passes), plus
// the synchronising warp; blocks in shared
// memory when that stays within 100 KB.  Levels with more than 8 late offsets
// per site, or more than 32 off-diagonal offsets, have no owner sweep.
#ifndef AMAMG_OWNER_MIN_CNT
#define AMAMG_OWNER_MIN_CNT 4
#endif
// The dynamic shared memory cap of a kernel is one setting per function and
// device, shared by every host thread of the process.  Setting it to each
// launch's own size lets one thread (a serving worker) lower it between
// another's setting and launch, and a cooperative launch then fails its
// residency check.  So it is raised once, to the device's opt-in maximum
// minus the kernel's static shared memory, and never lowered; occupancy
// follows the size each launch requests.
static cudaError_t allow_max_dyn_smem(const void* kern) {
  static std::mutex mu;
  static std::map<std::pair<int, const void*>, cudaError_t> done;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  const auto key = std::make_pair(dev, kern);
  const auto it = done.find(key);
  if (it != done.end()) return it->second;
  int mx = 0;
  cudaFuncAttributes fa;
  e = cudaDeviceGetAttribute(&mx, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, kern);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, mx - (int)fa.sharedSizeBytes);
  if (e != cudaSuccess) cudaGetLastError();
  done[key] = e;
  return e;
}

static size_t owner_smem(int own, int cnt, int K1, size_t cb, bool bsmem, size_t btb) {
  size_t s = (size_t)own * 6 * cb + (size_t)cnt * 4 * cb + (size_t)own * 4;
  if (bsmem) s += (size_t)own * K1 * (4 * btb + 4);
  return s;
}

// largest number of offsets of a site whose neighbour has the previous colour
// (the late offsets of the owner sweep)
static int owner_max_late(int Nt, int Nx, int ncol, const Offsets& off) {
  int worst = 0;
  for (int t = 0; t < Nt; ++t)
    for (int x = 0; x < Nx; ++x) {
      int c, j;
      site_colour(ncol, t, x, Nx, c, j);
      const int prev = c == 0 ? ncol - 1 : c - 1;
      int count = 0;
      for (int k = 1; k < off.K; ++k) {
        int cw, jw;
        site_colour(ncol, (t + off.dt[k]) % Nt, (x + off.dx[k]) % Nx, Nx, cw, jw);
        count += cw == prev;
      }
      worst = std::max(worst, count);
    }
  return worst;
}

// largest number of other blocks owning a neighbour of one block's sites
static int owner_max_wait(int Nt, int Nx, int ncol, const Offsets& off, int cnt) {
  const int m = Nt * Nx / ncol, nbpr = m / cnt;
  int worst = 0;
  std::vector<int> seen(nbpr, -1);
  for (int b = 0; b < nbpr; ++b) {
    int count = 0;
    for (int c = 0; c < ncol; ++c)
      for (int jj = 0; jj < cnt; ++jj) {
        int t, x;
        colour_site(ncol, c, b * cnt + jj, Nx, t, x);
        for (int k = 1; k < off.K; ++k) {
          int cw, jw;
          site_colour(ncol, (t + off.dt[k]) % Nt, (x + off.dx[k]) % Nx, Nx, cw, jw);
          const int ob = jw / cnt;
          if (ob != b && seen[ob] != b) { seen[ob] = b; ++count; }
        }
      }
    worst = std::max(worst, count);
  }
  return worst;
}

template <typename T, typename BT, int LE>
static auto owner_kernel_le(bool bsmem, int slots) {
  return bsmem ? (slots == 4 ? k_coarse_sweeps_owner<T, BT, true, 4, LE> : k_coarse_sweeps_owner<T, BT, true, 8, LE>)
               : (slots == 4 ? k_coarse_sweeps_owner<T, BT, false, 4, LE> : k_coarse_sweeps_owner<T, BT, false, 8, LE>);
}
template <typename T, typename BT>
static auto owner_kernel(bool bsmem, int slots, int le) {
  return le == 16 ? owner_kernel_le<T, BT, 16>(bsmem, slots) : owner_kernel_le<T, BT, 8>(bsmem, slots);
}

template <typename T, typename BT>
static bool owner_sweep_search(int Nt, int Nx, int K, int ncol, const Offsets& off, int R, OwnerConfig* cfg,
                               int variant) {
  int dev = 0, sms = 0, coop = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) || !coop) {
    cudaGetLastError();
    return false;
  }
  const int m = Nt * Nx / ncol;
  const size_t cb = sizeof(typename cplx<T>::type);
  const int max_late = owner_max_late(Nt, Nx, ncol, off);
  if (K - 1 > 32 || max_late > 8) return false;
  const int S = max_late <= 4 ? 4 : 8;
  int late_half = 0;                                         // first xor offset of the late-slot reduction
  while (2 * late_half < max_late) late_half = late_half ? 2 * late_half : 1;
  if (max_late == 1) late_half = 0;
  const int le_force = (variant & 3) == 1 ? 8 : (variant & 3) == 2 ? 16 : 0;
  int first_fit = 0;                                         // variant & 4: at least twice the first fitting cnt
  for (int cnt = std::min(AMAMG_OWNER_MIN_CNT, m); cnt <= m; ++cnt) {
    if (m % cnt) continue;
    if (first_fit && cnt < 2 * first_fit) continue;
    const int nbpr = m / cnt;
    const long blocks = (long)R * nbpr;
    if (nbpr > OWNER_MAX_BLOCKS || blocks > OWNER_MAX_BLOCKS) continue;
    const int own = ncol * cnt;
    const int le = le_force ? le_force : blocks <= sms ? 16 : 8;   // one block per SM: spread the early sums
    const int spe = 32 / le, spp = 32 / (4 * S);
    const int nearly = std::min((cnt + spe - 1) / spe, OWNER_EARLY_WARPS);
    const int npost = std::min((cnt + spp - 1) / spp, OWNER_POST_WARPS);
    const int threads = 32 * (nearly + npost + 1);
    const bool bsmem = owner_smem(own, cnt, K - 1, cb, true, sizeof(BT)) <= 100 * 1024;
    const size_t smem = owner_smem(own, cnt, K - 1, cb, bsmem, sizeof(BT));
    auto kern = owner_kernel<T, BT>(bsmem, S, le);
    int occ = 0;
    if (allow_max_dyn_smem((const void*)kern) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, threads, smem) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    if (blocks > (long)occ * sms) continue;
    if (owner_max_wait(Nt, Nx, ncol, off, cnt) > OWNER_MAX_WAIT) continue;
    if ((variant & 4) && !first_fit) {
      first_fit = cnt;
      continue;
    }
    cfg->cnt = cnt;
    cfg->late_half = late_half;
    cfg->slots = S;
    cfg->nearly = nearly;
    cfg->early_lanes = le;
    cfg->threads = threads;
    cfg->smem = smem;
    cfg->bsmem = bsmem;
    cfg->blocks = (int)blocks;
    return true;
  }
  return false;
}

// Cached per (element type, device, level shape, offsets, R, variant).
// variant (the autotuner's candidates): bits 0-1 force the early-sum lanes
// (1: 8, 2: 16; 0: by blocks per SM), bit 2 takes at least twice the fewest
// sites per block that fit.
template <typename T, typename BT>
bool owner_sweep_config(int Nt, int Nx, int K, int ncol, const Offsets& off, int R, OwnerConfig* cfg, int variant) {
  static std::mutex mu;
  static std::map<std::vector<int>, std::pair<bool, OwnerConfig>> cache;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return false; }
  std::vector<int> key = {dev, Nt, Nx, K, ncol, R, variant};
  for (int k = 0; k < off.K; ++k) { key.push_back(off.dt[k]); key.push_back(off.dx[k]); }
  std::lock_guard<std::mutex> lock(mu);
  auto it = cache.find(key);
  if (it == cache.end()) {
    OwnerConfig oc;
    const bool ok = owner_sweep_search<T, BT>(Nt, Nx, K, ncol, off, R, &oc, variant);
    it = cache.emplace(key, std::make_pair(ok, oc)).first;
  }
  *cfg = it->second.second;
  return it->second.first;
}

template <typename T, typename BT>
cudaError_t launch_coarse_sweeps_owner(typename cplx<T>::type* e, const typename cplx<T>::type* r, const BT* Bc,
                                       const float* Sc, const typename cplx<T>::type* Dc, const Offsets& off,
                                       int Nt, int Nx, int ncol, int sweeps, int R, unsigned* flags, unsigned* sync,
                                       cudaStream_t st, int withhold, int variant) {
  OwnerConfig oc;
  if (!owner_sweep_config<T, BT>(Nt, Nx, off.K, ncol, off, R, &oc, variant)) return cudaErrorNotSupported;
  auto kern = owner_kernel<T, BT>(oc.bsmem, oc.slots, oc.early_lanes);
  // the shared memory cap of the kernel, raised once to the device maximum
  cudaError_t err = allow_max_dyn_smem((const void*)kern);
  if (err != cudaSuccess) return err;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(oc.blocks);
  cfg.blockDim = dim3(oc.threads);
  cfg.dynamicSmemBytes = oc.smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, e, r, Bc, Sc, Dc, off, Nt, Nx, ncol, sweeps, oc.cnt, oc.nearly,
                            oc.late_half, flags, sync, withhold);
}

// the distributed-shared-memory sweep needs per = n / (16 ncol) whole sites per
// block and colour, at most 64
static bool dsmem_shape_ok(int n, int ncol) {
  const int m = n / ncol;
  return n % ncol == 0 && m % DSMEM_CLUSTER == 0 && m / DSMEM_CLUSTER >= 1 && m / DSMEM_CLUSTER <= 64;
}

// Whether a 16-block cluster with this shared-memory size can be resident on
// the device (queried once per level in setup; the sweep falls back to the
// per-colour kernels otherwise).
template <typename T, typename BT>
bool dsmem_sweeps_possible(int n, int K, int ncol, bool bsmem) {
  if (!dsmem_shape_ok(n, ncol)) return false;
  const size_t smem = dsmem_sweep_bytes(n, K, sizeof(typename cplx<T>::type), bsmem, sizeof(BT));
  if (smem > 200 * 1024) return false;
  auto kern = bsmem ? k_coarse_sweeps_dsmem<T, BT, true> : k_coarse_sweeps_dsmem<T, BT, false>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess ||
      allow_max_dyn_smem((const void*)kern) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  const int per = n / ncol / DSMEM_CLUSTER;
  int threads = ((per * 8 + 31) / 32) * 32;
  threads = threads > 512 ? 512 : threads;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(DSMEM_CLUSTER);
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = smem;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = DSMEM_CLUSTER;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int clusters = 0;
  if (cudaOccupancyMaxActiveClusters(&clusters, (void*)kern, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return clusters >= 1;
}

template <typename T, typename BT>
cudaError_t launch_coarse_sweeps_dsmem(typename cplx<T>::type* e, const typename cplx<T>::type* r, const BT* Bc,
                                       const float* Sc, const typename cplx<T>::type* Dc, const Offsets& off,
                                       int Nt, int Nx, int ncol, int sweeps, int R, bool bsmem, cudaStream_t st) {
  const int n = Nt * Nx;
  if (!dsmem_shape_ok(n, ncol)) return cudaErrorInvalidValue;
  const size_t smem = dsmem_sweep_bytes(n, off.K, sizeof(typename cplx<T>::type), bsmem, sizeof(BT));
  if (smem > 200 * 1024) return cudaErrorInvalidValue;
  auto kern = bsmem ? k_coarse_sweeps_dsmem<T, BT, true> : k_coarse_sweeps_dsmem<T, BT, false>;
  cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (err == cudaSuccess) err = allow_max_dyn_smem((const void*)kern);
  if (err != cudaSuccess) return err;
  const int per = n / ncol / DSMEM_CLUSTER;
  int threads = ((per * 8 + 31) / 32) * 32;
  threads = threads > 512 ? 512 : threads;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(DSMEM_CLUSTER * R);
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = DSMEM_CLUSTER;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, e, r, Bc, Sc, Dc, off, Nt, Nx, ncol, sweeps);
}

template <typename Cv>
cudaError_t launch_dense_gemv(const double2* A, const Cv* x, Cv* y, int nd, int R, cudaStream_t st) {
  const int blocks = (nd * 32 + 255) / 256;
  for (int r0 = 0; r0 < R;) {
    const int left = R - r0;
    const Cv* xx = x + (size_t)r0 * nd;
    Cv* yy = y + (size_t)r0 * nd;
    if (left >= 8) { k_dense_gemv<Cv, 8><<<blocks, 256, 0, st>>>(A, xx, yy, nd); r0 += 8; }
    else if (left >= 4) { k_dense_gemv<Cv, 4><<<blocks, 256, 0, st>>>(A, xx, yy, nd); r0 += 4; }
    else if (left >= 2) { k_dense_gemv<Cv, 2><<<blocks, 256, 0, st>>>(A, xx, yy, nd); r0 += 2; }
    else { k_dense_gemv<Cv, 1><<<blocks, 256, 0, st>>>(A, xx, yy, nd); r0 += 1; }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_dense_gemv32(const float2* A, const float2* x, float2* y, int nd, int R, cudaStream_t st) {
  const int blocks = (nd * 32 + 255) / 256;
  for (int r0 = 0; r0 < R;) {
    const int left = R - r0;
    const float2* xx = x + (size_t)r0 * nd;
    float2* yy = y + (size_t)r0 * nd;
    if (left >= 8) { k_dense_gemv32<8><<<blocks, 256, 0, st>>>(A, xx, yy, nd); r0 += 8; }
    else if (left >= 4) { k_dense_gemv32<4><<<blocks, 256, 0, st>>>(A, xx, yy, nd); r0 += 4; }
    else if (left >= 2) { k_dense_gemv32<2><<<blocks, 256, 0, st>>>(A, xx, yy, nd); r0 += 2; }
    else { k_dense_gemv32<1><<<blocks, 256, 0, st>>>(A, xx, yy, nd); r0 += 1; }
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
                                                           const double2*, const Offsets&, int, int, int, int, int,
                                                           cudaStream_t);
template cudaError_t launch_coarse_colour<float, __half2>(float2*, const float2*, const __half2*, const float*,
                                                          const float2*, const Offsets&, int, int, int, int, int,
                                                          cudaStream_t);
template cudaError_t launch_coarse_sweeps_cluster<float, __half2>(float2*, const float2*, const __half2*, const float*,
                                                                  const float2*, const Offsets&, int, int, int, int,
                                                                  int, cudaStream_t);
template bool owner_sweep_config<double, double2>(int, int, int, int, const Offsets&, int, OwnerConfig*, int);
template bool owner_sweep_config<float, __half2>(int, int, int, int, const Offsets&, int, OwnerConfig*, int);
template cudaError_t launch_coarse_sweeps_owner<double, double2>(double2*, const double2*, const double2*,
                                                                const float*, const double2*, const Offsets&, int, int,
                                                                int, int, int, unsigned*, unsigned*, cudaStream_t, int,
                                                                int);
template cudaError_t launch_coarse_sweeps_owner<float, __half2>(float2*, const float2*, const __half2*, const float*,
                                                               const float2*, const Offsets&, int, int, int, int, int,
                                                               unsigned*, unsigned*, cudaStream_t, int, int);
template int grid_sweep_blocks<double, double2>(int, int, int);
template int grid_sweep_blocks<float, __half2>(int, int, int);
template cudaError_t launch_coarse_sweeps_grid<double, double2>(double2*, const double2*, const double2*, const float*,
                                                                const double2*, const Offsets&, int, int, int, int,
                                                                int, unsigned*, cudaStream_t);
template cudaError_t launch_coarse_sweeps_grid<float, __half2>(float2*, const float2*, const __half2*, const float*,
                                                               const float2*, const Offsets&, int, int, int, int,
                                                               int, unsigned*, cudaStream_t);
template bool dsmem_sweeps_possible<float, __half2>(int, int, int, bool);
template bool dsmem_sweeps_possible<double, double2>(int, int, int, bool);
template cudaError_t launch_coarse_sweeps_dsmem<float, __half2>(float2*, const float2*, const __half2*, const float*,
                                                                const float2*, const Offsets&, int, int, int, int, int,
                                                                bool, cudaStream_t);
template cudaError_t launch_coarse_sweeps_dsmem<double, double2>(double2*, const double2*, const double2*,
                                                                 const float*, const double2*, const Offsets&, int, int,
                                                                 int, int, int, bool, cudaStream_t);
template cudaError_t launch_dense_gemv<double2>(const double2*, const double2*, double2*, int, int, cudaStream_t);
template cudaError_t launch_dense_gemv<float2>(const double2*, const float2*, float2*, int, int, cudaStream_t);
