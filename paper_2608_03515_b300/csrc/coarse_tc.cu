// Coarse-level apply y = A_l x for many right-hand sides on the 5th-generation
// tensor cores: FP16 operands, FP32 accumulation in tensor memory.
//
// A_l is the block stencil of the Galerkin operator (Sec. 2): y_v = sum over
// the offsets d of B_{v,d} x_{v+d}, 2x2 complex blocks, |dt|, |dx| <= 2.  The
// 8 coarse sites of a 2 x 4 patch in (t, x) (a super-block: 16 complex rows,
// 8 sites x 2 spins) couple only to the 6 x 8 box of sites around the patch
// (96 complex unknowns), so per super-block the apply is a dense 16 x 96
// complex matrix (zero where no offset reaches) times the 96 x R block of the
// right-hand sides: a GEMM, about 2.3 x the stencil's nonzeros.
//
// Real decomposition (K is not doubled): the MMA's M dimension holds the real
// and imaginary planes of 64 right-hand sides (m = 2 r + p), its N dimension
// the real and imaginary parts of the super-block's 16 complex rows
// (n = 2 i + q), its K dimension the 96 complex unknowns of the box:
//   D[(p, r)][(i, q)] = sum_k X_p[r][k] W_q[i][k],   X_0 = Re x, X_1 = Im x,
//                                                   W_0 = Re B, W_1 = Im B,
//   Re y_r[i] = D[(0, r)][(i, 0)] - D[(1, r)][(i, 1)],
//   Im y_r[i] = D[(0, r)][(i, 1)] + D[(1, r)][(i, 0)].
//
// FP16 scaling (both factor out of the K sum and are applied in the epilogue):
// W with one FP32 scale per operator row (site, spin), s = max over the row of
// max(|Re|, |Im|), entries fp16_rn(v / s); X with one power-of-two scale per
// right-hand side above its largest component (x / s exact, |x / s| < 1).
//
// Layouts.  A K chunk is 8 FP16 values (16 bytes): a 2 x 2 block of sites in
// (t, x) with both spins, value d = 4 tpar + 2 xpar + spin.
//   X staging  [group of 64 RHS][t/2][x/2][r 64][plane p][8]: one site block's
//              chunk for all 128 (r, p) rows is a contiguous 2 KB slab, which
//              is 16 core matrices (8 rows x 16 B) of the canonical no-swizzle
//              K-major layout with 8-row groups 128 B apart;
//   W image    per super-block [chunk c 12][n/8 4][n%8 8][8] (6 KB), the same
//              layout for the N = 32 rows; one FP32 scale per complex row i.
// Box chunk c = 4 ct + cx of super-block (P, Q) (sites t in {2P, 2P+1}, x in
// 4Q..4Q+3) is site block (P - 1 + ct, 2Q - 1 + cx) (periodic); complex row
// i = 8 spin + 4 tl + xl is site (2P + tl, 4Q + xl).
//
// One CTA per SM walks the items: strips of NS (2, or 1 on narrow levels)
// super-blocks along x that share one box of X slabs.  The last warp allocates
// the tensor memory; its lanes issue the bulk copies of an item's W images and
// X box into a stage (whose full barrier counts the bytes) and its lane 0 the
// six K = 16 MMAs per super-block into one of four accumulators (so the MMAs
// run ahead of the epilogue), then commits to the stage's empty barrier and to
// the accumulator's full barrier, which also receives a bulk copy of the
// item's row scales.  NS epilogue warpgroups, one per super-block of a strip,
// read their 32 TMEM lanes per warp, hand the accumulator back, combine the two
// planes of a right-hand side between adjacent lanes (one shuffle per value),
// scale and store y; the warps need no barrier among them.  Waits are polled
// by every lane of a warp and decided by a warp vote.  Every wait is bounded;
// on a time-out the kernel records it, waits (bounded) for its copies in
// flight, frees its tensor memory and returns.
#include <cstdlib>
#include <mutex>

#include "context.h"

namespace {

constexpr int CT_W_HALVES = 12 * 256;                    // 6 KB image per super-block
constexpr uint32_t CT_W_BYTES = CT_W_HALVES * 2;
constexpr uint32_t CT_SLAB_BYTES = 2048;                 // one chunk of 128 (p, r) rows
constexpr uint32_t CT_SMEM_CAP = 227 * 1024;            // dynamic shared memory per CTA
constexpr unsigned CT_SPIN_LIMIT = 1u << 24;
constexpr uint64_t CT_WAIT_NS = 1000000000ull;      // 1 s

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// no-swizzle K-major shared-memory descriptor: start, leading (K) byte offset,
// stride (M/N, 8-row groups) byte offset, descriptor version 1
__device__ __forceinline__ uint64_t desc_noswz(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// instruction descriptor, kind::f16: D FP32, A and B FP16, both K-major
__host__ __device__ constexpr uint32_t idesc_f16(int M, int N) {
  return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mbar_init(uint32_t addr, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(addr), "r"(count) : "memory");
}
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;\n" : "=l"(t));
  return t;
}
// wait for the completion of the phase with the given parity, at most
// CT_SPIN_LIMIT polls and CT_WAIT_NS nanoseconds
__device__ __forceinline__ bool mbar_wait(uint32_t addr, uint32_t parity) {
  uint64_t t0 = 0;
  for (unsigned it = 0; it < CT_SPIN_LIMIT; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(addr), "r"(parity)
        : "memory");
    if (done) return true;
    if ((it & 63u) == 0u) {
      const uint64_t t = global_ns();
      if (it == 0u) t0 = t;
      else if (t - t0 > CT_WAIT_NS) return false;
    }
  }
  return false;
}
__device__ __forceinline__ void mbar_arrive(uint32_t addr) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(addr) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t mbar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(mbar), "r"(bytes) : "memory");
}
// bulk copy global -> shared (16-byte aligned, size a multiple of 16), completing on mbar
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t mbar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(mbar)
               : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }

__device__ __forceinline__ void tc_mma_f16(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                           uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void tc_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(mbar)
               : "memory");
}
__device__ __forceinline__ void tc_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// power-of-two scale s > max component (from the FP32 bits of that maximum) and 1 / s
__device__ __forceinline__ void pow2_scale(unsigned amax_bits, float& s, float& inv) {
  if ((amax_bits & 0x7fffffffu) == 0u) {
    s = inv = 1.f;
    return;
  }
  int E = (int)((amax_bits >> 23) & 0xFFu);
  E = E < 1 ? 1 : (E > 252 ? 252 : E);
  s = __uint_as_float((unsigned)(E + 1) << 23);      // 2^(E - 126)
  inv = __uint_as_float((unsigned)(253 - E) << 23);  // 2^(126 - E)
}

// largest |Re|, |Im| of each right-hand side (FP32 bits, atomically maxed; amax zeroed before)
__global__ void k_ct_amax(const float2* __restrict__ x, unsigned* __restrict__ amax, long per_rhs) {
  const int r = blockIdx.y;
  const float4* xr = reinterpret_cast<const float4*>(x + (size_t)r * per_rhs);
  float m = 0.f;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < per_rhs / 2; i += (long)gridDim.x * blockDim.x) {
    const float4 v = xr[i];
    m = fmaxf(m, fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w))));
  }
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  __shared__ float wm[8];
  if ((threadIdx.x & 31) == 0) wm[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = fmaxf(m, wm[w]);
    atomicMax(amax + r, __float_as_uint(m));
  }
}

// X staging: thread (x pair xp, right-hand side r) of site-block row tp and
// group g reads the 4 x-pairs (tpar, spin) of 16 bytes and writes its 16-byte
// value rows of both planes; rows of right-hand sides >= R are zero
__global__ void __launch_bounds__(256)
k_ct_pack_x(const float2* __restrict__ x, const unsigned* __restrict__ amax, __half* __restrict__ xs, int Nt, int Nx,
            int R) {
  const int NTP = Nt >> 1, NXP = Nx >> 1;
  const int xp = blockIdx.x * 16 + (threadIdx.x & 15);
  const int tp = blockIdx.y >> 2;
  const int r = ((blockIdx.y & 3) << 4) + (threadIdx.x >> 4);
  const int g = blockIdx.z;
  if (xp >= NXP) return;
  const int rg = g * 64 + r;
  const size_t n = (size_t)Nt * Nx;
  __align__(16) __half re[8], im[8];
  if (rg < R) {
    float s, inv;
    pow2_scale(amax[rg], s, inv);
#pragma unroll
    for (int tpar = 0; tpar < 2; ++tpar)
#pragma unroll
      for (int spin = 0; spin < 2; ++spin) {
        const float4 v = *reinterpret_cast<const float4*>(
            x + ((size_t)rg * 2 + spin) * n + (size_t)(2 * tp + tpar) * Nx + 2 * xp);
        const int d0 = 4 * tpar + spin;   // xpar = 0; xpar = 1 is d0 + 2
        re[d0] = __float2half_rn(v.x * inv);
        im[d0] = __float2half_rn(v.y * inv);
        re[d0 + 2] = __float2half_rn(v.z * inv);
        im[d0 + 2] = __float2half_rn(v.w * inv);
      }
  } else {
#pragma unroll
    for (int d = 0; d < 8; ++d) re[d] = im[d] = __float2half_rn(0.f);
  }
  __half* slab = xs + (((size_t)g * NTP + tp) * NXP + xp) * 1024;
  *reinterpret_cast<uint4*>(slab + r * 16) = *reinterpret_cast<const uint4*>(re);
  *reinterpret_cast<uint4*>(slab + r * 16 + 8) = *reinterpret_cast<const uint4*>(im);
}

// W images (zeroed before) and row scales from the FP64 blocks [K][4][n]: one
// thread per (super-block, complex row i)
__global__ void k_ct_pack_w(const double2* __restrict__ B, Offsets off, int Nt, int Nx, __half* __restrict__ W,
                            float* __restrict__ Ws) {
  const int NQ = Nx >> 2;
  const int nsb = (Nt >> 1) * NQ;
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= nsb * 16) return;
  const int sb = g >> 4, i = g & 15;
  const int P = sb / NQ, Q = sb - (sb / NQ) * NQ;
  const int alpha = i >> 3, tl = (i >> 2) & 1, xl = i & 3;
  const int n = Nt * Nx;
  const int v = (2 * P + tl) * Nx + 4 * Q + xl;
  double m = 0.0;
  for (int k = 0; k < off.K; ++k)
    for (int beta = 0; beta < 2; ++beta) {
      const double2 b = B[((size_t)k * 4 + 2 * alpha + beta) * n + v];
      m = fmax(m, fmax(fabs(b.x), fabs(b.y)));
    }
  float s = (float)m;
  if (s == 0.f) s = 1.f;
  Ws[g] = s;
  const double inv = 1.0 / (double)s;
  __half* img = W + (size_t)sb * CT_W_HALVES;
  for (int k = 0; k < off.K; ++k) {
    const int dt = off.dt[k] > Nt / 2 ? off.dt[k] - Nt : off.dt[k];
    const int dx = off.dx[k] > Nx / 2 ? off.dx[k] - Nx : off.dx[k];
    const int tb = tl + dt + 2, xb = xl + dx + 2;   // box position, 0..5 x 0..7
    const int c = (tb >> 1) * 4 + (xb >> 1);
    for (int beta = 0; beta < 2; ++beta) {
      const double2 b = B[((size_t)k * 4 + 2 * alpha + beta) * n + v];
      const int d = 4 * (tb & 1) + 2 * (xb & 1) + beta;
      const int n0 = 2 * i, n1 = 2 * i + 1;
      img[c * 256 + (n0 >> 3) * 64 + (n0 & 7) * 8 + d] = __double2half(b.x * inv);
      img[c * 256 + (n1 >> 3) * 64 + (n1 & 7) * 8 + d] = __double2half(b.y * inv);
    }
  }
}

// Item = a strip of NS super-blocks along x (same P, group g): one stage holds
// their NS operator images (contiguous) and the 3 x (2 NS + 2) slab box they
// share, the MMAs of all NS go to NS column ranges of one accumulator, and the
// epilogue stores NS x 4 adjacent sites per row: the per-item synchronisation
// is paid once per strip.
template <int NS>
struct CtShape {
  static constexpr int NCOL = 2 * NS + 2;                             // x pairs of the box
  static constexpr uint32_t W_BYTES = NS * CT_W_BYTES;
  static constexpr uint32_t X_BYTES = 3 * NCOL * CT_SLAB_BYTES;
  static constexpr uint32_t STAGE = W_BYTES + X_BYTES;
  static constexpr int STAGES = (int)((CT_SMEM_CAP - 1024) / STAGE) > 7 ? 7 : (int)((CT_SMEM_CAP - 1024) / STAGE);
  static constexpr int ACC = 4;                                       // accumulators of 32 NS columns
  static constexpr int THREADS = 32 * (4 * NS + 1);                   // NS epilogue warpgroups + 1 warp
  static constexpr uint32_t TMEM_COLS = 32u * NS * ACC;
  static constexpr int SMEM = STAGES * STAGE + 1024;
  // items loaded ahead of the one multiplied: a refill then reuses the stage of
  // item j - 2, whose MMAs have finished (refilling that of item j - 1 would wait
  // for the round trip of the MMAs just issued); with 2 stages it is j - 1
  static constexpr int LA = STAGES >= 3 ? STAGES - 2 : STAGES - 1;
};

template <int NS>
__global__ void __launch_bounds__(CtShape<NS>::THREADS, 1)
k_coarse_tc(const __half* __restrict__ xs, const __half* __restrict__ W, const float* __restrict__ Ws,
            const unsigned* __restrict__ amax, float2* __restrict__ y, int Nt, int Nx, int R, int ngroups,
            int* __restrict__ err) {
  using SH = CtShape<NS>;
  constexpr int S = SH::STAGES, ACC = SH::ACC;
  extern __shared__ unsigned char sm_raw[];
  __shared__ uint64_t full[S], empty[S], tfull[ACC], tempty[ACC];
  __shared__ __align__(16) float wsm[ACC][16 * NS];   // row scales of the item in each accumulator
  __shared__ uint32_t tmem_base;
  __shared__ volatile int failed;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int NTP = Nt >> 1, NXP = Nx >> 1, NQ = Nx >> 2;
  const int per_row = NQ / NS;                       // strips per row of super-blocks
  const int nstrip = NTP * per_row;
  const int items = nstrip * ngroups;
  const int nj = (int)blockIdx.x < items ? (items - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  const uint32_t sbase = (smem_u32(sm_raw) + 1023u) & ~1023u;
  int epi_failed = 0;
  // item j of this CTA -> group, super-block row P, first super-block column Q0
  auto item_of = [&](int j, int& g, int& P, int& Q0) {
    const int it = (int)blockIdx.x + j * (int)gridDim.x;
    g = it / nstrip;
    const int s = it - g * nstrip;
    P = s / per_row;
    Q0 = (s - P * per_row) * NS;
  };

  if (tid == 0) {
    failed = 0;
    for (int k = 0; k < S; ++k) {
      mbar_init(smem_u32(&full[k]), 1);
      mbar_init(smem_u32(&empty[k]), 1);
    }
    for (int a = 0; a < ACC; ++a) {
      mbar_init(smem_u32(&tfull[a]), 2);     // the MMAs' commit + the row scales' copy
      mbar_init(smem_u32(&tempty[a]), 4 * NS);    // one arrival per epilogue warp
    }
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  constexpr int PW = 4 * NS;                         // the producer warp
  if (warp == PW) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&tmem_base)),
                 "r"(SH::TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t dtmem = tmem_base;

  if (warp == PW && nj > 0) {
    // ---- loads (lanes 0-6 issue one copy each) and MMAs (lane 0)
    // every lane polls; the vote makes a time-out a decision of the whole warp
    auto wait0 = [&](uint32_t bar, uint32_t parity) -> bool {
      return __all_sync(0xffffffffu, mbar_wait(bar, parity) ? 1 : 0) != 0;
    };
    auto load = [&](int j, int st) {
      int g, P, Q0;
      item_of(j, g, P, Q0);
      const uint32_t sa = sbase + st * SH::STAGE;
      const uint32_t fb = smem_u32(&full[st]);
      if (lane == 0) mbar_expect_tx(fb, SH::STAGE);
      __syncwarp();
      if (lane == 0) {
        bulk_g2s(sa, W + (size_t)(P * NQ + Q0) * CT_W_HALVES, SH::W_BYTES, fb);
      } else if (lane <= 6) {
        // box row ct: x pairs 2 Q0 - 1 .. 2 Q0 + 2 NS, adjacent in the staging
        // except across the periodic edge (then two copies, part 0 and 1)
        const int ct = (lane - 1) >> 1, part = (lane - 1) & 1;
        int tp = P - 1 + ct;
        tp += tp < 0 ? NTP : (tp >= NTP ? -NTP : 0);
        const __half* row = xs + ((size_t)g * NTP + tp) * NXP * 1024;
        const uint32_t dst = sa + SH::W_BYTES + ct * SH::NCOL * CT_SLAB_BYTES;
        const int x0 = 2 * Q0 - 1;
        if (x0 < 0) {
          if (part == 0) bulk_g2s(dst, row + (size_t)(NXP - 1) * 1024, CT_SLAB_BYTES, fb);
          else bulk_g2s(dst + CT_SLAB_BYTES, row, (SH::NCOL - 1) * CT_SLAB_BYTES, fb);
        } else if (x0 + SH::NCOL > NXP) {
          const int k = NXP - x0;                         // slabs before the edge
          if (part == 0) bulk_g2s(dst, row + (size_t)x0 * 1024, k * CT_SLAB_BYTES, fb);
          else bulk_g2s(dst + k * CT_SLAB_BYTES, row, (SH::NCOL - k) * CT_SLAB_BYTES, fb);
        } else if (part == 0) {
          bulk_g2s(dst, row + (size_t)x0 * 1024, SH::NCOL * CT_SLAB_BYTES, fb);
        }
      }
      __syncwarp();
    };
    int issued = 0, mma_done = 0;
    for (; issued < SH::LA && issued < nj; ++issued) load(issued, issued);
    const uint32_t idesc = idesc_f16(128, 32);
    bool bad = false;
    for (int j = 0; j < nj && !bad; ++j) {
      const int st = j % S, acc = j % ACC;
      if (!wait0(smem_u32(&full[st]), (uint32_t)((j / S) & 1))) { bad = true; break; }
      if (j >= ACC && !wait0(smem_u32(&tempty[acc]), (uint32_t)(((j / ACC) - 1) & 1))) { bad = true; break; }
      if (lane == 0) {
        int g, P, Q0;
        item_of(j, g, P, Q0);
        // the strip's row scales travel with its accumulator
        const uint32_t tb = smem_u32(&tfull[acc]);
        mbar_expect_tx(tb, 64 * NS);
        bulk_g2s(smem_u32(&wsm[acc][0]), Ws + (size_t)(P * NQ + Q0) * 16, 64 * NS, tb);
        tc_fence_after();
        const uint32_t sw = sbase + st * SH::STAGE, sx = sw + SH::W_BYTES;
#pragma unroll
        for (int k = 0; k < NS; ++k)
#pragma unroll
          for (int kk = 0; kk < 6; ++kk) {
            // chunks (ct, cx0) and (ct, cx0 + 1) of super-block k's window (columns 2k ..)
            const int ct = kk >> 1, cx0 = 2 * (kk & 1);
            tc_mma_f16(dtmem + (uint32_t)(acc * 32 * NS + 32 * k),
                       desc_noswz(sx + (ct * SH::NCOL + 2 * k + cx0) * CT_SLAB_BYTES, CT_SLAB_BYTES, 128),
                       desc_noswz(sw + k * CT_W_BYTES + kk * 1024, 512, 128), idesc, kk > 0 ? 1u : 0u);
          }
        tc_commit(smem_u32(&empty[st]));
        tc_commit(smem_u32(&tfull[acc]));
      }
      __syncwarp();
      mma_done = j + 1;
      const int next = j + SH::LA;
      if (next < nj) {
        const int sn = next % S;
        if (next >= S && !wait0(smem_u32(&empty[sn]), (uint32_t)(((next / S) - 1) & 1))) {
          bad = true;
          break;
        }
        load(next, sn);
        issued = next + 1;
      }
    }
    if (bad && lane == 0) {
      failed = 1;
      // let the copies in flight land and the issued MMAs finish (bounded) before returning
      for (int k = mma_done; k < issued; ++k) mbar_wait(smem_u32(&full[k % S]), (uint32_t)((k / S) & 1));
      if (mma_done > 0) {
        const int k = mma_done - 1;
        mbar_wait(smem_u32(&empty[k % S]), (uint32_t)((k / S) & 1));
        mbar_wait(smem_u32(&tfull[k % ACC]), (uint32_t)((k / ACC) & 1));   // its row-scale copy
      }
    }
    __syncwarp();
  } else if (warp < PW) {
    // ---- epilogue: TMEM -> registers -> y.  Warpgroup h finishes super-block
    // k = h of each strip; lane pair (2 r', 2 r' + 1) of its warp q = warp mod 4
    // (TMEM lanes 32 q ..) holds the two planes p of right-hand side
    // r = 16 q + r'; the p = 0 lane finishes spin 0, the p = 1 lane spin 1.
    const int n = Nt * Nx;
    const int q = warp & 3, h = warp >> 2;
    const int p = lane & 1, r = 16 * q + (lane >> 1);
    int g_cached = -1;
    float sx = 1.f;
    for (int j = 0; j < nj; ++j) {
      const int acc = j % ACC;
      int g, P, Q0;
      item_of(j, g, P, Q0);
      const int rg = g * 64 + r;
      if (g != g_cached) {
        float inv;
        pow2_scale(rg < R ? amax[rg] : 0u, sx, inv);
        g_cached = g;
      }
      const int ok =
          __all_sync(0xffffffffu, (!failed && mbar_wait(smem_u32(&tfull[acc]), (uint32_t)((j / ACC) & 1))) ? 1 : 0);
      if (!ok) { epi_failed = 1; break; }
      tc_fence_after();
      {
        const int k = h;
        float v[32];
        tc_ld32(dtmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(acc * 32 * NS + 32 * k), v);
        // this lane's 8 row scales (spin p, both site rows) of super-block k
        const float4 ws0 = *reinterpret_cast<const float4*>(&wsm[acc][16 * k + 8 * p]);
        const float4 ws1 = *reinterpret_cast<const float4*>(&wsm[acc][16 * k + 8 * p + 4]);
        // v[2 i + q] = D[(r, p)][(i, q)].  The p = 0 lane needs the partner's
        // (p = 1) values of rows i = 0..7, the p = 1 lane the partner's of rows
        // 8..15: send the other half, keep one's own
        float u[16];
#pragma unroll
        for (int c = 0; c < 16; ++c) {
          const float send = p ? v[c] : v[16 + c];
          u[c] = __shfl_xor_sync(0xffffffffu, send, 1);
        }
        // rows i = 8 p + m (m = 4 tl + xl): own D[(r, p)][(i, q)] = v[16 p + 2m + q],
        // partner's D[(r, 1 - p)][(i, q)] = u[2m + q]
        const float wsc[8] = {ws0.x, ws0.y, ws0.z, ws0.w, ws1.x, ws1.y, ws1.z, ws1.w};
        float o[16];
#pragma unroll
        for (int m = 0; m < 8; ++m) {
          const float a0 = p ? u[2 * m] : v[2 * m];                  // D[(r, 0)][(i, 0)]
          const float a1 = p ? u[2 * m + 1] : v[2 * m + 1];          // D[(r, 0)][(i, 1)]
          const float b0 = p ? v[16 + 2 * m] : u[2 * m];             // D[(r, 1)][(i, 0)]
          const float b1 = p ? v[16 + 2 * m + 1] : u[2 * m + 1];     // D[(r, 1)][(i, 1)]
          const float s = sx * wsc[m];
          o[2 * m] = (a0 - b1) * s;
          o[2 * m + 1] = (a1 + b0) * s;
        }
        if (rg < R) {
#pragma unroll
          for (int tl = 0; tl < 2; ++tl) {
            float4* dst = reinterpret_cast<float4*>(y + ((size_t)rg * 2 + p) * n + (size_t)(2 * P + tl) * Nx +
                                                    4 * (Q0 + k));
            dst[0] = make_float4(o[8 * tl], o[8 * tl + 1], o[8 * tl + 2], o[8 * tl + 3]);
            dst[1] = make_float4(o[8 * tl + 4], o[8 * tl + 5], o[8 * tl + 6], o[8 * tl + 7]);
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&tempty[acc]));
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if ((tid == 0 && failed) || (lane == 0 && epi_failed)) atomicExch(err, 1);
  __syncwarp();
  if (warp == PW)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(dtmem), "r"(SH::TMEM_COLS)
                 : "memory");
}

}  // namespace

bool coarse_tc_possible(int Nt, int Nx, const Offsets& off) {
  if (Nt % 2 || Nx % 4 || Nt < 8 || Nx < 8) return false;
  for (int k = 0; k < off.K; ++k) {
    const int dt = off.dt[k] > Nt / 2 ? off.dt[k] - Nt : off.dt[k];
    const int dx = off.dx[k] > Nx / 2 ? off.dx[k] - Nx : off.dx[k];
    if (dt < -2 || dt > 2 || dx < -2 || dx > 2) return false;
  }
  return true;
}

size_t coarse_tc_image_halves(int Nt, int Nx) { return (size_t)(Nt / 2) * (Nx / 4) * CT_W_HALVES; }
size_t coarse_tc_scale_floats(int Nt, int Nx) { return (size_t)(Nt / 2) * (Nx / 4) * 16; }
size_t coarse_tc_stage_halves(int Nt, int Nx, int R) { return (size_t)((R + 63) / 64) * Nt * Nx * 256; }

// strip width: 2 super-blocks where the row of super-blocks splits into pairs
// and the box (6 x pairs) fits the period, else 1.  (Strips of 4 measured
// slower: only two of their 84 KB stages fit in shared memory.)
static int strip_ns(int Nx) {
  const int NQ = Nx / 4, NXP = Nx / 2;
  return (NQ % 2 == 0 && 6 <= NXP) ? 2 : 1;
}

cudaError_t coarse_tc_init() {
  // the shared-memory opt-in is a per-process attribute of each kernel: set it once
  static std::once_flag once;
  static cudaError_t status = cudaSuccess;
  std::call_once(once, [] {
    status = cudaFuncSetAttribute(k_coarse_tc<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, CtShape<1>::SMEM);
    if (status == cudaSuccess)
      status = cudaFuncSetAttribute(k_coarse_tc<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, CtShape<2>::SMEM);
    if (status != cudaSuccess) cudaGetLastError();
  });
  return status;
}

cudaError_t launch_coarse_tc_pack_w(const double2* B, const Offsets& off, int Nt, int Nx, __half* W, float* Ws,
                                    cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(W, 0, coarse_tc_image_halves(Nt, Nx) * sizeof(__half), st);
  if (e != cudaSuccess) return e;
  const int threads = (Nt / 2) * (Nx / 4) * 16;
  k_ct_pack_w<<<(threads + 127) / 128, 128, 0, st>>>(B, off, Nt, Nx, W, Ws);
  return cudaGetLastError();
}

cudaError_t launch_coarse_tc(const float2* x, float2* y, const __half* W, const float* Ws, int Nt, int Nx, int R,
                             __half* stage, unsigned* amax, int* err, cudaStream_t st) {
  const int n = Nt * Nx;
  const int ngroups = (R + 63) / 64;
  cudaError_t e = cudaMemsetAsync(amax, 0, sizeof(unsigned) * R, st);
  if (e != cudaSuccess) return e;
  const long per = 2L * n;                            // complex entries per right-hand side (even)
  int bx = (int)((per / 2 + 255) / 256);
  bx = bx > 64 ? 64 : bx;
  k_ct_amax<<<dim3(bx, R), 256, 0, st>>>(x, amax, per);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_ct_pack_x<<<dim3((Nx / 2 + 15) / 16, (Nt / 2) * 4, ngroups), 256, 0, st>>>(x, amax, stage, Nt, Nx, R);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  int sms = 148, dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                 cudaSuccess) {
    cudaGetLastError();
    sms = 148;
  }
  const int ns = strip_ns(Nx);
  const long items = (long)(Nt / 2) * (Nx / 4 / ns) * ngroups;
  const int grid = (int)(items < sms ? items : sms);
  if (ns == 2)
    k_coarse_tc<2><<<grid, CtShape<2>::THREADS, CtShape<2>::SMEM, st>>>(stage, W, Ws, amax, y, Nt, Nx, R, ngroups, err);
  else
    k_coarse_tc<1><<<grid, CtShape<1>::THREADS, CtShape<1>::SMEM, st>>>(stage, W, Ws, amax, y, Nt, Nx, R, ngroups, err);
  return cudaGetLastError();
}
