// Coarsest-level apply of the mixed-precision V-cycle for many right-hand
// sides on the 5th-generation tensor cores: Y = Ainv32 X, with Ainv32 the FP32
// rounding of the FP64 inverse from setup (nd x nd complex, row-major) and X the
// R coarse right-hand sides.  It is a dense contraction (2 nd^2 R complex
// multiply-adds), so it runs as a tcgen05.mma GEMM with TF32 inputs and FP32
// accumulation in tensor memory.
//
// Real form.  With A stored as interleaved (re, im) floats, row i of A times the
// interleaved vector (x_re, -x_im) gives Re y_i, and times (x_im, x_re) gives
// Im y_i.  So D = A_f Bop^T with A_f = Ainv32 viewed as nd x 2nd floats (the
// MMA's A operand, K-major, read as stored) and Bop (2 Rp x 2nd floats, K-major)
// whose row c < Rp is (x_re, -x_im) of right-hand side c and row Rp + c is
// (x_im, x_re); Rp = R rounded up to a multiple of 8 (rows of padding are 0), so
// N = 2 Rp is a multiple of 16 (<= 256).  y_c[i] = (D[i][c], D[i][Rp + c]).
//
// One CTA per 128 rows (M = 128, cta_group::1).  K runs in chunks of 32 floats
// (128 bytes of every row); each chunk of A (128 rows) and Bop (N rows) is
// copied with cp.async into the canonical no-swizzle K-major layout (8-row x
// 16-byte core matrices, 128 bytes each: core (r/8, c) at (r/8) SBO + c LBO,
// LBO = 128 B, SBO = 1024 B), up to CM_STAGES stages with S - 2 chunks in
// flight ahead of the one being multiplied.  Thread 0 issues the four K = 8
// MMAs of a chunk and commits them to the chunk's mbarrier, which the threads
// wait on before refilling that stage two chunks later.  All waits are bounded; on a
// time-out the kernel records it, lets its copies finish, frees its tensor
// memory and returns.
#include "context.h"

namespace {

constexpr int CM_THREADS = 256;
constexpr int CM_BM = 128;              // rows per CTA (MMA M)
constexpr int CM_BK = 32;               // floats of K per stage
constexpr int CM_STAGES = 6;            // at most; fewer when a stage is large (smem budget CM_SMEM)
constexpr int CM_SMEM = 200 * 1024;
constexpr unsigned CM_SPIN_LIMIT = 1u << 24;
constexpr uint32_t CM_LBO = 128, CM_SBO = 1024;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// shared-memory matrix descriptor (tcgen05): start address, leading (K) and
// stride (M/N) byte offsets in 16-byte units, descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((CM_LBO >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((CM_SBO >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// instruction descriptor, kind::tf32: D FP32, A and B TF32, both K-major, M, N
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }
// wait until at most n (0..3, clamped) of this thread's newest groups are pending
__device__ __forceinline__ void cp_async_wait_n(int n) {
  if (n >= 3) cp_async_wait<3>();
  else if (n == 2) cp_async_wait<2>();
  else if (n == 1) cp_async_wait<1>();
  else cp_async_wait<0>();
}

__device__ __forceinline__ void mbar_init(uint32_t addr, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(addr), "r"(count) : "memory");
}
// bounded wait for the completion of the phase with the given parity
__device__ __forceinline__ bool mbar_wait(uint32_t addr, uint32_t parity) {
  for (unsigned it = 0; it < CM_SPIN_LIMIT; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(addr), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }

__device__ __forceinline__ void tc_mma_tf32(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                            uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void tc_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(mbar)
               : "memory");
}

// 32 consecutive FP32 columns of this thread's TMEM lane
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

// Bop rows from X ([R][nd] complex): row c < Rp = conj(x_c), row Rp + c = i conj(x_c)^*
// = (x_im, x_re); rows of right-hand sides >= R are zero.
__global__ void k_coarsest_bop(const float2* __restrict__ x, float4* __restrict__ bop, int nd, int R, int Rp) {
  const long total = (long)Rp * (nd / 2);              // (right-hand side, pair of complex entries)
  for (long g = (long)blockIdx.x * blockDim.x + threadIdx.x; g < total; g += (long)gridDim.x * blockDim.x) {
    const int c = (int)(g / (nd / 2)), q = (int)(g - (long)c * (nd / 2));
    float4 a = make_float4(0.f, 0.f, 0.f, 0.f), b = a;
    if (c < R) {
      const float4 v = reinterpret_cast<const float4*>(x + (size_t)c * nd)[q];    // x_2q, x_2q+1
      a = make_float4(v.x, -v.y, v.z, -v.w);
      b = make_float4(v.y, v.x, v.w, v.z);
    }
    bop[(size_t)c * (nd / 2) + q] = a;
    bop[(size_t)(Rp + c) * (nd / 2) + q] = b;
  }
}

__global__ void __launch_bounds__(CM_THREADS, 1)
k_coarsest_tc(const float* __restrict__ A, const float* __restrict__ Bop, float2* __restrict__ y, int nd, int R,
              int Rp, uint32_t tmem_cols, int S, int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ uint64_t mbar[CM_STAGES];
  __shared__ uint32_t tmem_base;
  __shared__ int failed;
  const int N = 2 * Rp;
  const int K = 2 * nd;                                  // floats per row
  const int nk = K / CM_BK;
  const int row0 = blockIdx.x * CM_BM;
  const uint32_t a_bytes = CM_BM * CM_BK * 4;            // 16 KB
  const uint32_t b_bytes = (uint32_t)N * CM_BK * 4;
  const uint32_t stage_bytes = a_bytes + b_bytes;
  const uint32_t sbase = smem_u32(sm);
  const int tid = threadIdx.x, warp = tid >> 5;

  if (tid == 0) {
    failed = 0;
    for (int s = 0; s < S; ++s) mbar_init(smem_u32(&mbar[s]), 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&tmem_base)),
                 "r"(tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t dtmem = tmem_base;

  // copies of chunk kt into stage s: A rows row0..row0+127, Bop rows 0..N-1,
  // K floats [kt 32, kt 32 + 32), as 16-byte pieces (row r, piece c of 8)
  auto load_stage = [&](int kt, int s) {
    const uint32_t sa = sbase + s * stage_bytes, sb = sa + a_bytes;
    const int k0 = kt * CM_BK;
    for (int q = tid; q < CM_BM * 8; q += CM_THREADS) {
      const int r = q >> 3, c = q & 7;
      cp_async16(sa + (r >> 3) * CM_SBO + c * CM_LBO + (r & 7) * 16, A + (size_t)(row0 + r) * K + k0 + 4 * c);
    }
    for (int q = tid; q < N * 8; q += CM_THREADS) {
      const int r = q >> 3, c = q & 7;
      cp_async16(sb + (r >> 3) * CM_SBO + c * CM_LBO + (r & 7) * 16, Bop + (size_t)r * K + k0 + 4 * c);
    }
  };

  // S stages, P = S - 2 chunks prefetched ahead: a refill goes to the stage
  // whose MMAs were issued two chunks earlier, so it rarely waits for them
  const int P = S - 2;
  for (int c = 0; c < P; ++c) {
    if (c < nk) load_stage(c, c);
    cp_async_commit();
  }
  const uint32_t idesc = idesc_tf32(CM_BM, N);
  for (int kt = 0; kt < nk; ++kt) {
    const int s = kt % S;
    cp_async_wait_n(P - 1);                              // at most P - 1 newer groups pending: chunk kt landed
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    __syncthreads();                                     // ... for every thread's copies
    if (tid == 0) {
      tc_fence_after();
      const uint32_t sa = sbase + s * stage_bytes, sb = sa + a_bytes;
#pragma unroll
      for (int k8 = 0; k8 < CM_BK / 8; ++k8)             // K = 8 TF32 per MMA = two core matrices
        tc_mma_tf32(dtmem, smem_desc(sa + k8 * 2 * CM_LBO), smem_desc(sb + k8 * 2 * CM_LBO), idesc,
                    (kt > 0 || k8 > 0) ? 1u : 0u);
      tc_commit(smem_u32(&mbar[s]));
    }
    // chunk kt + P goes to the stage of chunk kt - 2 once that chunk's MMAs are done
    const int next = kt + P;
    if (next < nk) {
      const int sn = next % S;
      if (kt >= 2 && !mbar_wait(smem_u32(&mbar[sn]), (uint32_t)(((kt - 2) / S) & 1))) failed = 1;
      __syncthreads();
      if (failed) break;
      load_stage(next, sn);
    }
    cp_async_commit();
  }
  // the last chunk's MMAs (committed to its stage's barrier) end the accumulation
  if (!failed && !mbar_wait(smem_u32(&mbar[(nk - 1) % S]), (uint32_t)(((nk - 1) / S) & 1))) failed = 1;
  cp_async_wait_all();
  __syncthreads();
  tc_fence_after();
  if (!failed && warp < 4) {
    // warp w reads TMEM lanes 32 w .. 32 w + 31 (rows of D); columns c and Rp + c
    const int row = row0 + 32 * warp + (tid & 31);
    const uint32_t lane_base = dtmem + ((uint32_t)(32 * warp) << 16);
    for (int c0 = 0; c0 < Rp; c0 += 32) {
      float re[32], im[32];
      tc_ld32(lane_base + (uint32_t)c0, re);
      tc_ld32(lane_base + (uint32_t)(Rp + c0), im);
#pragma unroll
      for (int j = 0; j < 32; ++j)
        if (c0 + j < R) y[(size_t)(c0 + j) * nd + row] = make_float2(re[j], im[j]);
    }
  }
  if (failed && tid == 0) atomicExch(err, 1);
  tc_fence_before();
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(dtmem), "r"(tmem_cols) : "memory");
}

}  // namespace

bool coarsest_tc_possible(int nd, int R) { return nd % CM_BM == 0 && nd >= CM_BM && R >= 8; }

// stages for N columns of Bop: as many as fit CM_SMEM, at most CM_STAGES (at least 3)
static int tc_stages(int N) {
  const int stage = CM_BM * CM_BK * 4 + N * CM_BK * 4;
  const int S = CM_SMEM / stage;
  return S > CM_STAGES ? CM_STAGES : (S < 3 ? 3 : S);
}

cudaError_t coarsest_tc_init() {
  return cudaFuncSetAttribute(k_coarsest_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, CM_SMEM);
}

size_t coarsest_tc_bop_elems(int nd) { return (size_t)2 * 128 * 2 * nd; }   // floats for up to 128 RHS per launch

cudaError_t launch_coarsest_tc(const float2* A, const float2* x, float2* y, int nd, int R, float* bop, int* err,
                               cudaStream_t st) {
  if (!coarsest_tc_possible(nd, R)) return cudaErrorInvalidValue;
  for (int r0 = 0; r0 < R; r0 += 128) {
    const int Rc = R - r0 < 128 ? R - r0 : 128;
    const int Rp = (Rc + 7) & ~7;
    // Rp columns of each form, read back by whole 32-column TMEM loads: the
    // allocation (a power of two >= 32) covers columns up to Rp + round32(Rp)
    const int N = 2 * Rp;
    const int ncols_needed = Rp + ((Rp + 31) & ~31);
    uint32_t cols = 32;
    while ((int)cols < (N > ncols_needed ? N : ncols_needed)) cols <<= 1;
    if (cols > 512) return cudaErrorInvalidValue;
    const long pairs = (long)Rp * (nd / 2);
    k_coarsest_bop<<<(unsigned)((pairs + 255) / 256 < 4096 ? (pairs + 255) / 256 : 4096), 256, 0, st>>>(
        x + (size_t)r0 * nd, reinterpret_cast<float4*>(bop), nd, Rc, Rp);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int S = tc_stages(N);
    const size_t smem = (size_t)S * (CM_BM * CM_BK * 4 + (size_t)N * CM_BK * 4);
    k_coarsest_tc<<<nd / CM_BM, CM_THREADS, smem, st>>>(reinterpret_cast<const float*>(A), bop, y + (size_t)r0 * nd,
                                                       nd, Rc, Rp, cols, S, err);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}
