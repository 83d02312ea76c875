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
        __nanosleep(64);
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
template <typename T, typename BT>
__global__ void __launch_bounds__(256)
k_coarse_sweeps_grid(typename cplx<T>::type* __restrict__ e, const typename cplx<T>::type* __restrict__ r,
                     const BT* __restrict__ B, const float* __restrict__ Bs,
                     const typename cplx<T>::type* __restrict__ Dinv, Offsets off, int Nt, int Nx, int ncol,
                     int sweeps, int R, unsigned* sync) {
  constexpr int LPS = GsLanes<T>::value;
  const int n = Nt * Nx;
  const int per_colour = n / ncol;
  const long units = (long)R * per_colour;
  const int g = threadIdx.x & (LPS - 1);
  const int gpb = blockDim.x / LPS;
  const long stride = (long)gridDim.x * gpb;
  for (int sw = 0; sw < sweeps; ++sw) {
    for (int colour = 0; colour < ncol; ++colour) {
      // every group runs the same number of iterations (shuffles stay converged)
      for (long base = 0; base < units; base += stride) {
        const long u = base + (long)blockIdx.x * gpb + threadIdx.x / LPS;
        const bool valid = u < units;
        const int rhs = valid ? (int)(u / per_colour) : 0;
        const int idx = valid ? (int)(u - (long)rhs * per_colour) : 0;
        const size_t roff = (size_t)rhs * 2 * n;
        gs_site<T, BT, LPS, false>(e + roff, r + roff, B, Bs, Dinv, off, Nt, Nx, ncol, colour, idx, g, valid);
      }
      if (!grid_barrier(sync, gridDim.x)) return;
    }
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
// inverse (the factorisation itself is FP64); FP32 arithmetic.
template <int RR>
__global__ void __launch_bounds__(256)
k_dense_gemv32(const float2* __restrict__ A, const float2* __restrict__ x, float2* __restrict__ y, int nd) {
  const int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (row >= nd) return;
  float2 acc[RR];
#pragma unroll
  for (int r = 0; r < RR; ++r) acc[r] = make_float2(0.f, 0.f);
  const float2* a = A + (size_t)row * nd;
  int j = lane;
  for (; j + 96 < nd; j += 128) {
    float2 aj[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) aj[u] = __ldcs(a + j + 32 * u);
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int r = 0; r < RR; ++r) cmac(acc[r], aj[u], x[(size_t)r * nd + j + 32 * u]);
  }
  for (; j < nd; j += 32) {
    const float2 aj = a[j];
#pragma unroll
    for (int r = 0; r < RR; ++r) cmac(acc[r], aj, x[(size_t)r * nd + j]);
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

// Grid sweep: 64 threads per block (8 FP64 sites or 2 FP32 sites per block and
// pass), as many blocks as the widest colour needs, at most the blocks that
// can be co-resident (cooperative launch).
constexpr int GRID_SWEEP_THREADS = 64;
template <typename T, typename BT>
int grid_sweep_blocks(int n, int ncol, int R) {
  static int cap[2] = {-1, -1};                       // per element type, first device queried
  int& c = cap[sizeof(T) == 8 ? 1 : 0];
  if (c < 0) {
    int dev = 0, sms = 0, occ = 0, coop = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_coarse_sweeps_grid<T, BT>, GRID_SWEEP_THREADS, 0) !=
            cudaSuccess) {
      cudaGetLastError();
      c = 0;
    } else {
      c = coop ? sms * occ : 0;
    }
  }
  if (c <= 0) return 0;
  const long groups = (long)R * (n / ncol);
  const long want = (groups * GsLanes<T>::value + GRID_SWEEP_THREADS - 1) / GRID_SWEEP_THREADS;
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
  return cudaLaunchKernelEx(&cfg, k_coarse_sweeps_grid<T, BT>, e, r, B, Bs, Dinv, off, Nt, Nx, ncol, sweeps, R, sync);
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
      cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
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
  if (err == cudaSuccess) err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
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
