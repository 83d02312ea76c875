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
// Tiles are moved by TMA (cp.async.bulk.tensor, 2D boxes of 32 floats x rows,
// 128-byte swizzle, which the shared-memory descriptors of the MMAs name):
// one CTA per 128 rows (M = 128, cta_group::1) and per slice of K (small
// levels split K so that every SM has a CTA; the slices' FP32 partials are
// added in slice order by a second kernel).  One thread drives the pipeline:
// TMA loads of a chunk of 32 floats of every row of A and of Bop into a stage
// (its full barrier counts the bytes), the four K = 8 MMAs of a landed chunk,
// their commit to the stage's empty barrier, which the next load into that
// stage waits for.  All waits are bounded; on a time-out the kernel records
// it, frees its tensor memory and returns.
#include <cuda.h>

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

// 2D TMA load of a box at (x inner, y outer) into shared memory, completing
// on mbarrier mbar (transaction bytes)
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t mbar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];\n"
      ::"r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(mbar)
      : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t mbar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(mbar), "r"(bytes) : "memory");
}

// shared-memory matrix descriptor for the 128-byte swizzled K-major layout that
// TMA writes with CU_TENSOR_MAP_SWIZZLE_128B (rows of 128 bytes, 8-row atoms of
// 1024 bytes: stride byte offset 1024, leading byte offset unused)
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)((1024u >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;                               // SWIZZLE_128B
  return d;
}

// One CTA per 128 rows and K slice (blockIdx.y of gridDim.y slices).  Thread 0
// drives the pipeline: TMA loads of the A and Bop chunks into stage s (full[s],
// with the stage's byte count), MMAs of a landed chunk, commit to empty[s],
// which the next load into that stage waits for.  Out: y directly (one slice)
// or the slice's FP32 partial of D (part[slice][row][column], N columns).
__global__ void __launch_bounds__(CM_THREADS, 1)
k_coarsest_tc(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
              float2* __restrict__ y, float* __restrict__ part, int nd, int R, int Rp, uint32_t tmem_cols, int S,
              int* __restrict__ err) {
  extern __shared__ unsigned char sm_raw[];
  __shared__ uint64_t full[CM_STAGES], empty[CM_STAGES];
  __shared__ uint32_t tmem_base;
  __shared__ int failed;
  const int N = 2 * Rp;
  const int nk_all = (2 * nd) / CM_BK;
  const int per = (nk_all + gridDim.y - 1) / gridDim.y;
  const int kt0 = blockIdx.y * per;
  const int nk = max(0, min(nk_all, kt0 + per) - kt0);
  const int row0 = blockIdx.x * CM_BM;
  const uint32_t a_bytes = CM_BM * CM_BK * 4;             // 16 KB
  const uint32_t b_bytes = (uint32_t)N * CM_BK * 4;
  const uint32_t stage_bytes = a_bytes + b_bytes;        // a multiple of 1024
  const uint32_t sbase = (smem_u32(sm_raw) + 1023u) & ~1023u;   // 1024-byte aligned stages (swizzle atoms)
  const int tid = threadIdx.x, warp = tid >> 5;

  if (tid == 0) {
    failed = 0;
    for (int s = 0; s < S; ++s) {
      mbar_init(smem_u32(&full[s]), 1);
      mbar_init(smem_u32(&empty[s]), 1);
    }
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

  if (tid == 0 && nk > 0) {
    auto load = [&](int c, int st) {
      const uint32_t sa = sbase + st * stage_bytes;
      const uint32_t fb = smem_u32(&full[st]);
      mbar_expect_tx(fb, stage_bytes);
      tma_load_2d(sa, &mapA, (kt0 + c) * CM_BK, row0, fb);
      tma_load_2d(sa + a_bytes, &mapB, (kt0 + c) * CM_BK, 0, fb);
    };
    const int P = S - 1;                                  // chunks in flight ahead of the one multiplied
    for (int c = 0; c < P && c < nk; ++c) load(c, c);
    const uint32_t idesc = idesc_tf32(CM_BM, N);
    for (int kt = 0; kt < nk; ++kt) {
      const int st = kt % S;
      if (!mbar_wait(smem_u32(&full[st]), (uint32_t)((kt / S) & 1))) { failed = 1; break; }
      tc_fence_after();
      const uint32_t sa = sbase + st * stage_bytes, sb = sa + a_bytes;
#pragma unroll
      for (int k8 = 0; k8 < CM_BK / 8; ++k8)              // K = 8 TF32 = 32 bytes of the 128-byte row
        tc_mma_tf32(dtmem, smem_desc_sw128(sa + 32 * k8), smem_desc_sw128(sb + 32 * k8), idesc,
                    (kt > 0 || k8 > 0) ? 1u : 0u);
      tc_commit(smem_u32(&empty[st]));
      const int next = kt + P;
      if (next < nk) {
        const int sn = next % S;
        // the stage's previous chunk (next - S) must have been multiplied
        if (next >= S && !mbar_wait(smem_u32(&empty[sn]), (uint32_t)(((next / S) - 1) & 1))) { failed = 1; break; }
        load(next, sn);
      }
    }
    // the last chunk's MMAs (committed to its stage's empty barrier) end the accumulation
    if (!failed && !mbar_wait(smem_u32(&empty[(nk - 1) % S]), (uint32_t)(((nk - 1) / S) & 1))) failed = 1;
  }
  __syncthreads();
  tc_fence_after();
  if (!failed && nk > 0 && warp < 4) {
    // warp w reads TMEM lanes 32 w .. 32 w + 31 (rows of D)
    const int row = row0 + 32 * warp + (tid & 31);
    const uint32_t lane_base = dtmem + ((uint32_t)(32 * warp) << 16);
    for (int c0 = 0; c0 < Rp; c0 += 32) {
      float re[32], im[32];
      tc_ld32(lane_base + (uint32_t)c0, re);
      tc_ld32(lane_base + (uint32_t)(Rp + c0), im);
      if (gridDim.y == 1) {
#pragma unroll
        for (int j = 0; j < 32; ++j)
          if (c0 + j < R) y[(size_t)(c0 + j) * nd + row] = make_float2(re[j], im[j]);
      } else {
        float* pr = part + ((size_t)blockIdx.y * nd + row) * N;
#pragma unroll
        for (int j = 0; j < 32; ++j)
          if (c0 + j < Rp) {
            pr[c0 + j] = re[j];
            pr[Rp + c0 + j] = im[j];
          }
      }
    }
  }
  if (failed && tid == 0) atomicExch(err, 1);
  tc_fence_before();
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(dtmem), "r"(tmem_cols) : "memory");
}

// y_c[i] = sum over slices (in slice order) of (D[i][c], D[i][Rp + c])
__global__ void k_coarsest_tc_reduce(const float* __restrict__ part, float2* __restrict__ y, int nd, int R, int Rp,
                                     int slices) {
  const long total = (long)R * nd;
  const int N = 2 * Rp;
  for (long g = (long)blockIdx.x * blockDim.x + threadIdx.x; g < total; g += (long)gridDim.x * blockDim.x) {
    const int c = (int)(g / nd), i = (int)(g - (long)c * nd);
    float re = 0.f, im = 0.f;
    for (int sl = 0; sl < slices; ++sl) {
      const float* pr = part + ((size_t)sl * nd + i) * N;
      re += pr[c];
      im += pr[Rp + c];
    }
    y[(size_t)c * nd + i] = make_float2(re, im);
  }
}

}  // namespace

bool coarsest_tc_possible(int nd, int R) { return nd % CM_BM == 0 && nd >= CM_BM && R >= 8; }

// K slices: enough CTAs for one wave over the SMs (at most 16 slices)
static int tc_slices(int nd) {
  int sms = 148, dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                 cudaSuccess) {
    cudaGetLastError();
    sms = 148;
  }
  const int tiles = nd / CM_BM;
  int s = sms / tiles;
  s = s < 1 ? 1 : (s > 16 ? 16 : s);
  const int nk = 2 * nd / CM_BK;
  if (s > nk) s = nk;
  const int per = (nk + s - 1) / s;                     // chunks per slice; every slice gets at least one
  return (nk + per - 1) / per;
}

size_t coarsest_tc_scratch_elems(int nd) {
  // Bop for up to 128 right-hand sides per launch, then the slices' partial D
  return (size_t)2 * 128 * 2 * nd + (size_t)tc_slices(nd) * nd * 256;
}

// stages for N columns of Bop: as many as fit CM_SMEM, at most CM_STAGES (at least 3)
static int tc_stages(int N) {
  const int stage = CM_BM * CM_BK * 4 + N * CM_BK * 4;
  const int S = (CM_SMEM - 1024) / stage;
  return S > CM_STAGES ? CM_STAGES : (S < 3 ? 3 : S);
}

typedef CUresult (*EncodeTiled)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiled encode_fn();

cudaError_t coarsest_tc_init() {
  if (!encode_fn()) return cudaErrorNotSupported;       // no tensor-map encoder: the CUDA-core apply runs
  return cudaFuncSetAttribute(k_coarsest_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, CM_SMEM);
}

static EncodeTiled encode_fn() {
  // looked up once (a function-local static is initialised once, thread-safely)
  static const EncodeTiled fn = []() -> EncodeTiled {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    EncodeTiled f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      f = reinterpret_cast<EncodeTiled>(p);
    cudaGetLastError();
    return f;
  }();
  return fn;
}

// row-major FP32 matrix rows x cols (cols contiguous), boxes of 32 x box_rows,
// 128-byte swizzle
static bool make_map(CUtensorMap* m, const void* base, int rows, int cols, int box_rows) {
  EncodeTiled fn = encode_fn();
  if (!fn) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)cols * 4};
  const cuuint32_t box[2] = {(cuuint32_t)CM_BK, (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(base), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

cudaError_t launch_coarsest_tc(const float2* A, const float2* x, float2* y, int nd, int R, float* scratch, int* err,
                               cudaStream_t st) {
  if (!coarsest_tc_possible(nd, R)) return cudaErrorInvalidValue;
  float* bop = scratch;
  float* part = scratch + (size_t)2 * 128 * 2 * nd;
  const int slices = tc_slices(nd);
  CUtensorMap mapA;
  if (!make_map(&mapA, A, nd, 2 * nd, CM_BM)) return cudaErrorNotSupported;
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
    CUtensorMap mapB;
    if (!make_map(&mapB, bop, N, 2 * nd, N)) return cudaErrorNotSupported;
    const int S = tc_stages(N);
    const size_t smem = (size_t)S * (CM_BM * CM_BK * 4 + (size_t)N * CM_BK * 4) + 1024;
    k_coarsest_tc<<<dim3(nd / CM_BM, slices), CM_THREADS, smem, st>>>(mapA, mapB, y + (size_t)r0 * nd, part, nd, Rc,
                                                                      Rp, cols, S, err);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (slices > 1) {
      const long total = (long)Rc * nd;
      k_coarsest_tc_reduce<<<(unsigned)((total + 255) / 256 < 4096 ? (total + 255) / 256 : 4096), 256, 0, st>>>(
          part, y + (size_t)r0 * nd, nd, Rc, Rp, slices);
      e = cudaGetLastError();
      if (e != cudaSuccess) return e;
    }
  }
  return cudaSuccess;
}
