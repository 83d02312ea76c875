// Gram-Schmidt of the outer FGMRES in double-float arithmetic (opt-in for the
// mixed-precision solve, amamg_params.gs_arith = AMAMG_GS_DF64).
//
// On this GPU the FP64 pipe is narrow (about 2 FP64 FMAs per SM and clock),
// and the classical Gram-Schmidt of the outer solver is bound by it.  A
// double-float value is an unevaluated sum hi + lo of two floats with |lo| <=
// ulp(hi) / 2: about 48 significant bits.  Sums and products of such values
// are formed exactly with the error-free transformations of Knuth (two-sum)
// and of Dekker (two-product, here one fused multiply-add) and renormalised,
// which costs a few FP32 operations per operation -- on the wide FP32 pipe.
// The Krylov basis V is stored as double-float complex entries (hi.re, hi.im,
// lo.re, lo.im: 16 bytes, the size of a complex double), the vector w being
// orthogonalised is converted once per pass, and the reductions across threads
// and blocks are done in double-float too (the block-order of the final sum is
// fixed, so the result is deterministic).  The products and norms handed to
// the host's Hessenberg problem are rounded to double.
#include "context.h"

namespace {

struct dfl {
  float hi, lo;
};

__device__ __forceinline__ dfl two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  const float e = (a - (s - bb)) + (b - bb);
  return {s, e};
}
__device__ __forceinline__ dfl quick_two_sum(float a, float b) {
  const float s = a + b;
  return {s, b - (s - a)};
}
__device__ __forceinline__ dfl df_add(dfl x, dfl y) {
  dfl s = two_sum(x.hi, y.hi);
  const float e = s.lo + (x.lo + y.lo);
  return quick_two_sum(s.hi, e);
}
__device__ __forceinline__ dfl df_mul(dfl x, dfl y) {
  const float p = x.hi * y.hi;
  float e = fmaf(x.hi, y.hi, -p);
  e = fmaf(x.hi, y.lo, fmaf(x.lo, y.hi, e));
  return quick_two_sum(p, e);
}
__device__ __forceinline__ dfl df_neg(dfl x) { return {-x.hi, -x.lo}; }
__device__ __forceinline__ dfl df_from(double d) {
  const float hi = __double2float_rn(d);
  return {hi, __double2float_rn(d - (double)hi)};
}
__device__ __forceinline__ double df_to(dfl x) { return (double)x.hi + (double)x.lo; }
__device__ __forceinline__ dfl df_shfl_xor(dfl x, int o) {
  return {__shfl_xor_sync(0xffffffffu, x.hi, o), __shfl_xor_sync(0xffffffffu, x.lo, o)};
}

// complex double-float entry of a basis vector: float4 (hi.re, hi.im, lo.re, lo.im)
struct dfc {
  dfl re, im;
};
__device__ __forceinline__ dfc load_dfc(const float4* p) {
  const float4 v = *p;
  return {{v.x, v.z}, {v.y, v.w}};
}
__device__ __forceinline__ void store_dfc(float4* p, dfc c) { *p = make_float4(c.re.hi, c.im.hi, c.re.lo, c.im.lo); }
__device__ __forceinline__ dfc dfc_from(double2 d) { return {df_from(d.x), df_from(d.y)}; }

// acc += conj(a) b
__device__ __forceinline__ void dfc_macc(dfc& acc, dfc a, dfc b) {
  acc.re = df_add(acc.re, df_add(df_mul(a.re, b.re), df_mul(a.im, b.im)));
  acc.im = df_add(acc.im, df_add(df_mul(a.re, b.im), df_neg(df_mul(a.im, b.re))));
}
// acc += a b
__device__ __forceinline__ void dfc_mac(dfc& acc, dfc a, dfc b) {
  acc.re = df_add(acc.re, df_add(df_mul(a.re, b.re), df_neg(df_mul(a.im, b.im))));
  acc.im = df_add(acc.im, df_add(df_mul(a.re, b.im), df_mul(a.im, b.re)));
}

constexpr int DF_THREADS = 256;
constexpr int DF_GROUP = 8;                // basis vectors per pass over the block's elements

__device__ __forceinline__ dfl block_sum_df(dfl v, dfl* sh) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = df_add(v, df_shfl_xor(v, o));
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  if (wid == 0) {
    v = lane < (int)(blockDim.x >> 5) ? sh[lane] : dfl{0.f, 0.f};
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = df_add(v, df_shfl_xor(v, o));
  }
  return v;
}

// w (double complex) -> double-float copy wd
__global__ void __launch_bounds__(256)
k_to_df(const double2* __restrict__ w, float4* __restrict__ wd, long n) {
  for (long k = (long)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (long)gridDim.x * blockDim.x)
    store_dfc(wd + k, dfc_from(w[k]));
}

// Loads a double-float partial sum written by another block (through L2).
__device__ __forceinline__ dfl ld_partial(const dfl* p) {
  const float2 v = __ldcg(reinterpret_cast<const float2*>(p));
  return {v.x, v.y};
}

// out[r ldo + off + i] = <V_i, w_r> for i < J (and <w_r, w_r> at i = J when
// with_self).  Blocks take contiguous chunks of the elements and walk their
// chunk once per group of DF_GROUP basis vectors (w read once per group);
// block partial sums partial[(r ps + 2 i + part) nb + block] in double-float;
// the last block of a right-hand side (ticket) adds them in block order (one
// warp per product, a fixed tree).  gate: right-hand sides with flag 0 get 0.
__global__ void __launch_bounds__(DF_THREADS)
k_dots_df(const float4* __restrict__ V, size_t vi, size_t vr, const float4* __restrict__ w, size_t wr, long len,
          long chunk, int J, int with_self, const int* __restrict__ gate, dfl* __restrict__ partial, int ps,
          unsigned* __restrict__ tickets, double2* __restrict__ out, int ldo, int off) {
  __shared__ dfl sh[32];
  __shared__ bool last;
  const int r = blockIdx.z, nb = gridDim.x;
  const int Jt = J + with_self;
  if (gate && gate[r] == 0) {
    if (blockIdx.x == 0 && blockIdx.y == 0)
      for (int i = threadIdx.x; i < Jt; i += blockDim.x) out[(size_t)r * ldo + off + i] = make_double2(0.0, 0.0);
    return;
  }
  const float4* wv = w + r * wr;
  const long start = (long)blockIdx.x * chunk;
  const long end = min(start + chunk, len);
  // this block's group of DF_GROUP basis vectors (blockIdx.y)
  for (int g0 = blockIdx.y * DF_GROUP; g0 < Jt && g0 < (int)(blockIdx.y + 1) * DF_GROUP; g0 += DF_GROUP) {
    dfc acc[DF_GROUP];
#pragma unroll
    for (int u = 0; u < DF_GROUP; ++u) acc[u] = {{0.f, 0.f}, {0.f, 0.f}};
    for (long k = start + threadIdx.x; k < end; k += blockDim.x) {
      const dfc b = load_dfc(wv + k);
#pragma unroll
      for (int u = 0; u < DF_GROUP; ++u) {
        const int i = g0 + u;
        if (i < Jt) {
          const dfc a = (i < J) ? load_dfc(V + i * vi + r * vr + k) : b;
          dfc_macc(acc[u], a, b);
        }
      }
    }
#pragma unroll
    for (int u = 0; u < DF_GROUP; ++u) {
      const int i = g0 + u;
      if (i < Jt) {
        const dfl re = block_sum_df(acc[u].re, sh);
        const dfl im = block_sum_df(acc[u].im, sh);
        if (threadIdx.x == 0) {
          partial[((size_t)r * ps + 2 * i) * nb + blockIdx.x] = re;
          partial[((size_t)r * ps + 2 * i + 1) * nb + blockIdx.x] = im;
        }
      }
    }
  }
  if (threadIdx.x == 0) {
    __threadfence();
    last = atomicAdd(&tickets[r], 1u) == (unsigned)(nb * gridDim.y - 1);
  }
  __syncthreads();
  if (!last) return;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int i = wid; i < Jt; i += blockDim.x >> 5) {
    dfl s0 = {0.f, 0.f}, s1 = {0.f, 0.f};
    for (int bb = lane; bb < nb; bb += 32) {
      s0 = df_add(s0, ld_partial(partial + ((size_t)r * ps + 2 * i) * nb + bb));
      s1 = df_add(s1, ld_partial(partial + ((size_t)r * ps + 2 * i + 1) * nb + bb));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      s0 = df_add(s0, df_shfl_xor(s0, o));
      s1 = df_add(s1, df_shfl_xor(s1, o));
    }
    if (lane == 0) out[(size_t)r * ldo + off + i] = make_double2(df_to(s0), df_to(s1));
  }
  __syncthreads();
  if (threadIdx.x == 0) tickets[r] = 0;
}

// w_r -= sum_{i<J} coef[r ldc + i] V_{i,r} in double-float, and ||w_r||:
// out[r ldo + nrm_off] = ||w_r||, inv[r] = 1 / ||w_r|| (0 for a zero vector);
// mode 2 also sets flag[r] = (||w_r||^2 < eta2 out[r ldo + ref_off].x) (the
// DGKS test).  Right-hand sides whose gate flag is 0 are left untouched.
__global__ void __launch_bounds__(DF_THREADS)
k_axpy_norm_df(float4* __restrict__ w, size_t wr, const float4* __restrict__ V, size_t vi, size_t vr,
               const double2* __restrict__ coef, int ldc, int J, long len, long chunk, const int* __restrict__ gate,
               dfl* __restrict__ partial, unsigned* __restrict__ tickets, double2* __restrict__ out, int ldo,
               int nrm_off, double* __restrict__ inv, int* __restrict__ flag, int ref_off, double eta2, int mode) {
  __shared__ dfl sh[32];
  __shared__ dfc cf[64];
  __shared__ bool last;
  const int r = blockIdx.y, nb = gridDim.x;
  if (gate && gate[r] == 0) return;
  for (int i = threadIdx.x; i < J; i += blockDim.x) cf[i] = dfc_from(coef[(size_t)r * ldc + i]);
  __syncthreads();
  float4* wv = w + r * wr;
  const long start = (long)blockIdx.x * chunk;
  const long end = min(start + chunk, len);
  dfl ss = {0.f, 0.f};
  for (long k = start + threadIdx.x; k < end; k += blockDim.x) {
    dfc acc = {{0.f, 0.f}, {0.f, 0.f}};
    for (int i = 0; i < J; ++i) dfc_mac(acc, cf[i], load_dfc(V + i * vi + r * vr + k));
    dfc v = load_dfc(wv + k);
    v.re = df_add(v.re, df_neg(acc.re));
    v.im = df_add(v.im, df_neg(acc.im));
    store_dfc(wv + k, v);
    ss = df_add(ss, df_add(df_mul(v.re, v.re), df_mul(v.im, v.im)));
  }
  ss = block_sum_df(ss, sh);
  if (threadIdx.x == 0) {
    partial[(size_t)r * nb + blockIdx.x] = ss;
    __threadfence();
    last = atomicAdd(&tickets[r], 1u) == (unsigned)(nb - 1);
  }
  __syncthreads();
  if (!last) return;
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    dfl t = {0.f, 0.f};
    for (int bb = lane; bb < nb; bb += 32) t = df_add(t, ld_partial(partial + (size_t)r * nb + bb));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t = df_add(t, df_shfl_xor(t, o));
    if (lane == 0) {
      const double q = df_to(t);
      // NaN propagates (a NaN or Inf entry must surface as a non-finite norm)
      const double nrm = (q >= 0.0) ? sqrt(q) : ((q < 0.0) ? 0.0 : q);
      out[(size_t)r * ldo + nrm_off] = make_double2(nrm, 0.0);
      inv[r] = nrm > 0.0 ? 1.0 / nrm : 0.0;
      if (mode == 2) flag[r] = (q < eta2 * out[(size_t)r * ldo + ref_off].x) ? 1 : 0;
      tickets[r] = 0;
    }
  }
}

// dst_r = scale[r] src_r in double-float, and its FP32 rounding (the hi parts)
// in dst32_r; src double-float (src_df) or double (src_d)
__global__ void __launch_bounds__(256)
k_scale_copy_df(float4* __restrict__ dst, float2* __restrict__ dst32, size_t dr, const float4* __restrict__ src_df,
                const double2* __restrict__ src_d, size_t sr, const double* __restrict__ scale, long len) {
  const int r = blockIdx.y;
  const dfl s = df_from(scale[r]);
  for (long k = (long)blockIdx.x * blockDim.x + threadIdx.x; k < len; k += (long)gridDim.x * blockDim.x) {
    const dfc v = src_df ? load_dfc(src_df + r * sr + k) : dfc_from(src_d[r * sr + k]);
    dfc o;
    o.re = df_mul(v.re, s);
    o.im = df_mul(v.im, s);
    store_dfc(dst + r * dr + k, o);
    if (dst32) dst32[r * dr + k] = make_float2(o.re.hi, o.im.hi);
  }
}

// element chunks of the inner products (blocks per right-hand side and group
// of basis vectors) and of the update
inline int df_blocks(long len) {
  long nb = (len + 1023) / 1024;
  if (nb > 296) nb = 296;
  return (int)(nb < 1 ? 1 : nb);
}
inline int df_axpy_blocks(long len) {
  long g = (len + 255) / 256;
  if (g > 148 * 16) g = 148 * 16;
  return (int)(g < 1 ? 1 : g);
}

}  // namespace

cudaError_t launch_to_df(const double2* w, void* wd, long n, cudaStream_t st) {
  long g = (n + 255) / 256;
  if (g > 148 * 16) g = 148 * 16;
  k_to_df<<<(unsigned)(g < 1 ? 1 : g), 256, 0, st>>>(w, static_cast<float4*>(wd), n);
  return cudaGetLastError();
}

cudaError_t launch_dots_df(const void* V, size_t vi, size_t vr, const void* w, size_t wr, long len, int J, int R,
                           bool with_self, const int* gate, void* partial, int ps, unsigned* tickets, double2* out,
                           int ldo, int off, cudaStream_t st) {
  const int nb = df_blocks(len);
  const long chunk = (len + nb - 1) / nb;
  const int groups = (J + (with_self ? 1 : 0) + DF_GROUP - 1) / DF_GROUP;
  dim3 grid(nb, groups, R);
  k_dots_df<<<grid, DF_THREADS, 0, st>>>(static_cast<const float4*>(V), vi, vr, static_cast<const float4*>(w), wr,
                                         len, chunk, J, with_self ? 1 : 0, gate, static_cast<dfl*>(partial), ps,
                                         tickets, out, ldo, off);
  return cudaGetLastError();
}

cudaError_t launch_axpy_norm_df(void* w, size_t wr, const void* V, size_t vi, size_t vr, const double2* coef, int ldc,
                                int J, long len, int R, const int* gate, void* partial, unsigned* tickets,
                                double2* out, int ldo, int nrm_off, double* inv, int* flag, int ref_off, double eta2,
                                int mode, cudaStream_t st) {
  if (J > 64) return cudaErrorInvalidValue;
  const int nb = df_axpy_blocks(len);
  const long chunk = (len + nb - 1) / nb;
  dim3 grid(nb, R);
  k_axpy_norm_df<<<grid, DF_THREADS, 0, st>>>(static_cast<float4*>(w), wr, static_cast<const float4*>(V), vi, vr,
                                              coef, ldc, J, len, chunk, gate, static_cast<dfl*>(partial), tickets, out,
                                              ldo, nrm_off, inv, flag, ref_off, eta2, mode);
  return cudaGetLastError();
}

int df_partial_blocks(long len) { return df_blocks(len); }
int df_norm_blocks(long len) { return df_axpy_blocks(len); }

cudaError_t launch_scale_copy_df(void* dst, float2* dst32, size_t dr, const void* src_df, const double2* src_d,
                                 size_t sr, const double* scale, long len, int R, cudaStream_t st) {
  long g = (len + 255) / 256;
  if (g > 148 * 16) g = 148 * 16;
  dim3 grid((unsigned)(g < 1 ? 1 : g), R);
  k_scale_copy_df<<<grid, 256, 0, st>>>(static_cast<float4*>(dst), dst32, dr, static_cast<const float4*>(src_df),
                                        src_d, sr, scale, len);
  return cudaGetLastError();
}
