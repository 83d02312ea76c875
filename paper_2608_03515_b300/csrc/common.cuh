// Shared device helpers: complex arithmetic on double2 / float2, precision traits,
// FP16+scale decoding.  Nothing here is specific to one kernel.
#pragma once
#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <stdint.h>

template <typename T> struct cplx;
template <> struct cplx<double> { using type = double2; };
template <> struct cplx<float>  { using type = float2; };

__host__ __device__ __forceinline__ double2 mk(double r, double i) { return make_double2(r, i); }
__host__ __device__ __forceinline__ float2  mk(float r, float i)  { return make_float2(r, i); }

template <typename C> __host__ __device__ __forceinline__ C czero();
template <> __host__ __device__ __forceinline__ double2 czero<double2>() { return make_double2(0.0, 0.0); }
template <> __host__ __device__ __forceinline__ float2  czero<float2>()  { return make_float2(0.f, 0.f); }

#define CPLX_OPS(C, R)                                                                         \
  __host__ __device__ __forceinline__ C operator+(C a, C b) { return mk(a.x + b.x, a.y + b.y); } \
  __host__ __device__ __forceinline__ C operator-(C a, C b) { return mk(a.x - b.x, a.y - b.y); } \
  __host__ __device__ __forceinline__ C operator-(C a) { return mk(-a.x, -a.y); }               \
  __host__ __device__ __forceinline__ C operator*(R s, C a) { return mk(s * a.x, s * a.y); }     \
  __host__ __device__ __forceinline__ C& operator+=(C& a, C b) { a.x += b.x; a.y += b.y; return a; } \
  __host__ __device__ __forceinline__ C& operator-=(C& a, C b) { a.x -= b.x; a.y -= b.y; return a; } \
  __host__ __device__ __forceinline__ C cmul(C a, C b) { return mk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); } \
  /* conj(a) * b */                                                                             \
  __host__ __device__ __forceinline__ C cmulc(C a, C b) { return mk(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x); } \
  /* a * conj(b) */                                                                             \
  __host__ __device__ __forceinline__ C cmul_conjb(C a, C b) { return mk(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y); } \
  __host__ __device__ __forceinline__ C cconj(C a) { return mk(a.x, -a.y); }                    \
  /* i * a */                                                                                   \
  __host__ __device__ __forceinline__ C ci(C a) { return mk(-a.y, a.x); }                        \
  __host__ __device__ __forceinline__ R cabs2(C a) { return a.x * a.x + a.y * a.y; }

CPLX_OPS(double2, double)
CPLX_OPS(float2, float)
#undef CPLX_OPS

// fused complex multiply-accumulate (4 FMAs): acc + a b, and acc + conj(a) b
__device__ __forceinline__ void cmac(double2& acc, double2 a, double2 b) {
  acc.x = fma(a.x, b.x, acc.x); acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y); acc.y = fma(a.y, b.x, acc.y);
}
__device__ __forceinline__ void cmac(float2& acc, float2 a, float2 b) {
  acc.x = fmaf(a.x, b.x, acc.x); acc.x = fmaf(-a.y, b.y, acc.x);
  acc.y = fmaf(a.x, b.y, acc.y); acc.y = fmaf(a.y, b.x, acc.y);
}
__device__ __forceinline__ void cmacc(double2& acc, double2 a, double2 b) {
  acc.x = fma(a.x, b.x, acc.x); acc.x = fma(a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y); acc.y = fma(-a.y, b.x, acc.y);
}
__device__ __forceinline__ void cmacc(float2& acc, float2 a, float2 b) {
  acc.x = fmaf(a.x, b.x, acc.x); acc.x = fmaf(a.y, b.y, acc.x);
  acc.y = fmaf(a.x, b.y, acc.y); acc.y = fmaf(-a.y, b.x, acc.y);
}

// element conversions between vector precisions
__device__ __forceinline__ double2 to_c(double2 a, double) { return a; }
__device__ __forceinline__ double2 to_c(float2 a, double) { return make_double2(a.x, a.y); }
__device__ __forceinline__ float2 to_c(float2 a, float) { return a; }
__device__ __forceinline__ float2 to_c(double2 a, float) { return make_float2((float)a.x, (float)a.y); }

template <typename C> struct real_of;
template <> struct real_of<double2> { using type = double; };
template <> struct real_of<float2> { using type = float; };

// FP16 pair + FP32 scale -> complex of compute precision
template <typename T>
__device__ __forceinline__ typename cplx<T>::type h2c(__half2 h, float s) {
  float2 f = __half22float2(h);
  return mk((T)(f.x * s), (T)(f.y * s));
}

// canonical (mod N) block offsets of a level operator, passed by value to kernels
#define AMAMG_MAX_OFFSETS 48
// off-diagonal block offsets a smoothed coarse level may have (K - 1); setup
// rejects hierarchies beyond it
#define GS_MAX_OFFDIAG 24
struct Offsets {
  int K;
  int dt[AMAMG_MAX_OFFSETS];
  int dx[AMAMG_MAX_OFFSETS];
};

__host__ __device__ __forceinline__ int wrap(int v, int n) { v %= n; return v < 0 ? v + n : v; }

// Gauss-Seidel colourings of a coarse level (Sec. 5 leaves the ordering open):
// site (t, x) of site j of colour c, and the inverse map.  ncol = 16: colour
// (t mod 4, x mod 4), j = (t / 4) (Nx / 4) + x / 4.  ncol = 8: colour
// (t + 3 x) mod 8, j = t (Nx / 8) + x / 8 (one x per row and colour, since 3 is
// invertible mod 8: x = 3 (c - t) mod 8).
__host__ __device__ __forceinline__ void colour_site(int ncol, int c, int j, int Nx, int& t, int& x) {
  if (ncol == 16) {
    const int qx = Nx >> 2;
    t = 4 * (j / qx) + (c >> 2);
    x = 4 * (j % qx) + (c & 3);
  } else {
    const int ox = Nx >> 3;
    t = j / ox;
    x = 8 * (j % ox) + ((3 * (c - t)) & 7);
  }
}
__host__ __device__ __forceinline__ void site_colour(int ncol, int t, int x, int Nx, int& c, int& j) {
  if (ncol == 16) {
    c = ((t & 3) << 2) | (x & 3);
    j = (t >> 2) * (Nx >> 2) + (x >> 2);
  } else {
    c = (t + 3 * x) & 7;
    j = t * (Nx >> 3) + (x >> 3);
  }
}

// Edge ownership (Sec. 4.1: a border site takes its interpolation formula from
// "the first aggregate it was assigned to").  Row of the non-vertex site at
// in-tile position (i, j) of tile (p, q): its formula comes from basket
// W(p + dp, q + dq) (indices mod the tile counts), where it sits at in-basket
// position (i - a dp, j - a dq), and its stored columns 2c + beta are corner c
// of that basket.
//   OWN_TILE:      the tile's own basket (dp = dq = 0).
//   OWN_FIRST_LEX: of the baskets containing the site, the one of smallest
//                  index p Nq + q: a bottom-border site (i = 0) of a tile with
//                  p >= 1 lies on the top border of W(p-1, q), a left-border
//                  site (j = 0) of a tile with q >= 1 on the right border of
//                  W(p, q-1); on the first tile row / column the periodic
//                  neighbour has the larger index, so the tile's own basket keeps it.
enum OwnerRule : int { OWN_TILE = 0, OWN_FIRST_LEX = 1 };
__host__ __device__ __forceinline__ void row_basket(int own, int p, int q, int i, int j, int& dp, int& dq) {
  dp = 0;
  dq = 0;
  if (own == OWN_FIRST_LEX) {
    if (i == 0 && p >= 1) dp = -1;
    else if (j == 0 && q >= 1) dq = -1;
  }
}
