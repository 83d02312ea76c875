// Setup-phase kernels (Sec. 2 and Sec. 4.1), all in FP64:
//   * batched local ideal interpolation per wirebasket, u_F = -A_FF^{-1} A_FV u_V
//     (Eqs. (14)-(16)), one CTA per basket, dense LU with partial pivoting in
//     shared memory;
//   * Galerkin coarse operator A_H = P^H A P in block-stencil form, one CTA per
//     coarse site, one thread per output entry (deterministic, no atomics);
//   * 2x2 diagonal-block inverses for the coarse smoother;
//   * the coarsest level's dense matrix and its in-place Gauss-Jordan inverse
//     (row partial pivoting; the column unscrambling is a final gather);
//   * FP16 + FP32-scale packing of P and of the coarse blocks.
#include "kernels.h"

namespace {

// ------------------------------------------------------------------ operators
// Block A[(t,x), neighbour] of the level operator.  Wilson: Eq. (3) with the
// Eq. (7) sign; stencil: a Galerkin level in [K][4][n] form.

__device__ __forceinline__ void wilson_nb(const WilsonOp& op, int t, int x, int dir, int& tn, int& xn,
                                          double2 blk[4]) {
  const int Nt = op.Nt, Nx = op.Nx, n = Nt * Nx;
  const int s = t * Nx + x;
  double2 c;
  switch (dir) {
    case 0:
      tn = t; xn = x;
      blk[0] = make_double2(op.diag, 0.0); blk[1] = make_double2(0.0, 0.0);
      blk[2] = make_double2(0.0, 0.0); blk[3] = make_double2(op.diag, 0.0);
      return;
    case 1: {  // n + t: -1/2 sign U_0(n) (1 - sigma_0)
      tn = (t + 1 == Nt) ? 0 : t + 1; xn = x;
      const double sg = (t + 1 == Nt) ? -0.5 : 0.5;
      c = -sg * op.U[s];
      blk[0] = c; blk[1] = -c; blk[2] = -c; blk[3] = c;
      return;
    }
    case 2: {  // n - t: -1/2 sign U_0(n - t)^* (1 + sigma_0)
      tn = (t == 0) ? Nt - 1 : t - 1; xn = x;
      const double sg = (t == 0) ? -0.5 : 0.5;
      c = -sg * cconj(op.U[tn * Nx + x]);
      blk[0] = c; blk[1] = c; blk[2] = c; blk[3] = c;
      return;
    }
    case 3: {  // n + x: -1/2 U_1(n) (1 - sigma_1) = [[c, i c], [-i c, c]]
      tn = t; xn = (x + 1 == Nx) ? 0 : x + 1;
      c = -0.5 * op.U[n + s];
      blk[0] = c; blk[1] = ci(c); blk[2] = -ci(c); blk[3] = c;
      return;
    }
    default: {  // n - x: -1/2 U_1(n - x)^* (1 + sigma_1) = [[c, -i c], [i c, c]]
      tn = t; xn = (x == 0) ? Nx - 1 : x - 1;
      c = -0.5 * cconj(op.U[n + t * Nx + xn]);
      blk[0] = c; blk[1] = -ci(c); blk[2] = ci(c); blk[3] = c;
      return;
    }
  }
}

__device__ __forceinline__ int op_count(const WilsonOp&) { return 5; }
__device__ __forceinline__ int op_count(const StencilOp& op) { return op.off.K; }

__device__ __forceinline__ void op_nb(const WilsonOp& op, int t, int x, int k, int& tn, int& xn, double2 blk[4]) {
  wilson_nb(op, t, x, k, tn, xn, blk);
}
__device__ __forceinline__ void op_nb(const StencilOp& op, int t, int x, int k, int& tn, int& xn, double2 blk[4]) {
  const int n = op.Nt * op.Nx;
  tn = t + op.off.dt[k]; tn -= (tn >= op.Nt) ? op.Nt : 0;
  xn = x + op.off.dx[k]; xn -= (xn >= op.Nx) ? op.Nx : 0;
  const int v = t * op.Nx + x;
#pragma unroll
  for (int e = 0; e < 4; ++e) blk[e] = op.B[((size_t)k * 4 + e) * n + v];
}

// block coupling site (t,x) to the site displaced by (di, dj); false if none
__device__ __forceinline__ bool op_rel(const WilsonOp& op, int t, int x, int di, int dj, double2 blk[4]) {
  int dir;
  if (di == 0 && dj == 0) dir = 0;
  else if (di == 1 && dj == 0) dir = 1;
  else if (di == -1 && dj == 0) dir = 2;
  else if (di == 0 && dj == 1) dir = 3;
  else if (di == 0 && dj == -1) dir = 4;
  else return false;
  int tn, xn;
  wilson_nb(op, t, x, dir, tn, xn, blk);
  return true;
}
__device__ __forceinline__ bool op_rel(const StencilOp& op, int t, int x, int di, int dj, double2 blk[4]) {
  const int ct = wrap(di, op.Nt), cx = wrap(dj, op.Nx);
  for (int k = 0; k < op.off.K; ++k) {
    if (op.off.dt[k] == ct && op.off.dx[k] == cx) {
      const int n = op.Nt * op.Nx, v = t * op.Nx + x;
#pragma unroll
      for (int e = 0; e < 4; ++e) blk[e] = op.B[((size_t)k * 4 + e) * n + v];
      return true;
    }
  }
  return false;
}

__device__ __forceinline__ double2 crecip(double2 a) {
  const double d = 1.0 / (a.x * a.x + a.y * a.y);
  return make_double2(a.x * d, -a.y * d);
}

// ------------------------------------------------------------------ local solves
// One CTA per basket W(p, q).  Basket sites (i, j), 0 <= i, j <= A; F = the
// non-corner sites in i-major order; corners ordered c = 2 (i/A) + (j/A).
// M = [A_FF | A_FV] (NF x (NF + 8)), eliminated in place; X = A_FF^{-1} A_FV.
template <int A, typename Op>
__global__ void __launch_bounds__(128)
k_local_solve(Op op, int Np, int Nq, double2* __restrict__ P, int* __restrict__ err, double rel_tol, int own) {
  constexpr int NB = (A + 1) * (A + 1);
  constexpr int NFS = NB - 4;
  constexpr int NF = 2 * NFS;
  constexpr int NC = NF + 8;
  constexpr int NR = 2 * (A * A - 1);
  __shared__ double2 M[NF][NC];
  __shared__ int fi[NFS], fj[NFS];
  __shared__ int s_piv;
  __shared__ double s_pmax;
  __shared__ double s_scale;
  const int tile = blockIdx.x;
  const int p = tile / Nq, q = tile - (tile / Nq) * Nq;
  const int Nt = op.Nt, Nx = op.Nx;
  if (threadIdx.x == 0) {
    int f = 0;
    for (int i = 0; i <= A; ++i)
      for (int j = 0; j <= A; ++j) {
        const bool corner = (i == 0 || i == A) && (j == 0 || j == A);
        if (!corner) { fi[f] = i; fj[f] = j; ++f; }
      }
  }
  __syncthreads();
  // fill: rows F sites, columns F sites then corners
  for (int pr = threadIdx.x; pr < NFS * (NFS + 4); pr += blockDim.x) {
    const int f = pr / (NFS + 4), g = pr - (pr / (NFS + 4)) * (NFS + 4);
    const int i = fi[f], j = fj[f];
    int i2, j2, col;
    if (g < NFS) { i2 = fi[g]; j2 = fj[g]; col = 2 * g; }
    else { const int c = g - NFS; i2 = (c >> 1) * A; j2 = (c & 1) * A; col = NF + 2 * c; }
    const int t = wrap(p * A + i, Nt), x = wrap(q * A + j, Nx);
    double2 blk[4];
    if (!op_rel(op, t, x, i2 - i, j2 - j, blk)) {
      blk[0] = blk[1] = blk[2] = blk[3] = make_double2(0.0, 0.0);
    }
    M[2 * f][col] = blk[0];
    M[2 * f][col + 1] = blk[1];
    M[2 * f + 1][col] = blk[2];
    M[2 * f + 1][col + 1] = blk[3];
  }
  __syncthreads();
  // scale reference for the singularity test: max |entry| of A_FF
  if (threadIdx.x < 32) {
    double m = 0.0;
    for (int e = threadIdx.x; e < NF * NF; e += 32) m = fmax(m, cabs2(M[e / NF][e - (e / NF) * NF]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (threadIdx.x == 0) s_scale = m;
  }
  __syncthreads();
  for (int k = 0; k < NF; ++k) {
    if (threadIdx.x < 32) {
      double best = -1.0;
      int bi = k;
      for (int i = k + threadIdx.x; i < NF; i += 32) {
        const double v = cabs2(M[i][k]);
        if (v > best) { best = v; bi = i; }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const double ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
      }
      if (threadIdx.x == 0) { s_piv = bi; s_pmax = best; }
    }
    __syncthreads();
    const int pv = s_piv;
    if (pv != k) {
      for (int j = k + threadIdx.x; j < NC; j += blockDim.x) {
        const double2 tmp = M[k][j];
        M[k][j] = M[pv][j];
        M[pv][j] = tmp;
      }
    }
    if (threadIdx.x == 0 && !(s_pmax > rel_tol * rel_tol * s_scale)) {
      atomicOr(err, 1);
      M[k][k] = make_double2(1.0, 0.0);   // keep the arithmetic finite; the status reports the failure
    }
    __syncthreads();
    const double2 inv = crecip(M[k][k]);
    for (int i = k + 1 + threadIdx.x; i < NF; i += blockDim.x) M[i][k] = cmul(M[i][k], inv);
    __syncthreads();
    const int rows = NF - k - 1, cols = NC - k - 1;
    for (int e = threadIdx.x; e < rows * cols; e += blockDim.x) {
      const int i = k + 1 + e / cols, j = k + 1 + (e - (e / cols) * cols);
      M[i][j] -= cmul(M[i][k], M[k][j]);
    }
    __syncthreads();
  }
  // back substitution on the 8 right-hand-side columns
  for (int k = NF - 1; k >= 0; --k) {
    if (threadIdx.x < 8) M[k][NF + threadIdx.x] = cmul(M[k][NF + threadIdx.x], crecip(M[k][k]));
    __syncthreads();
    for (int e = threadIdx.x; e < k * 8; e += blockDim.x) {
      const int i = e >> 3, c = e & 7;
      M[i][NF + c] -= cmul(M[i][k], M[k][NF + c]);
    }
    __syncthreads();
  }
  // the rows this basket owns (row_basket): F site (i, j) lies in tile
  // (p + i / A, q + j / A) at in-tile (i mod A, j mod A) and is stored there;
  // P = -X.  Under the tile rule these are the sites with i, j < A.
  for (int e = threadIdx.x; e < NFS * 2 * 8; e += blockDim.x) {
    const int f = e >> 4, rem = e & 15, alpha = rem >> 3, c8 = rem & 7;
    const int i = fi[f], j = fj[f];
    const int it = (i == A) ? 0 : i, jt = (j == A) ? 0 : j;
    const int pT = (i == A) ? ((p + 1 == Np) ? 0 : p + 1) : p;
    const int qT = (j == A) ? ((q + 1 == Nq) ? 0 : q + 1) : q;
    int dp, dq;
    row_basket(own, pT, qT, it, jt, dp, dq);
    if (wrap(pT + dp, Np) != p || wrap(qT + dq, Nq) != q) continue;
    const int l = it * A + jt;
    const int lr = 2 * (l - 1) + alpha;
    P[((size_t)(pT * Nq + qT) * 8 + c8) * NR + lr] = -M[2 * f + alpha][NF + c8];
  }
}

// ------------------------------------------------------------------ Galerkin
// Interpolation weight P[(site (t,x), spin tau), (vertex (pw,qw), spin beta)].
// The row's stored columns are the corners of its basket (row_basket).
__device__ __forceinline__ double2 p_weight(const double2* __restrict__ P, int t, int x, int tau, int pw, int qw,
                                            int beta, int a, int Np, int Nq, int nrows, int own) {
  const int it = t % a, ix = x % a;
  const int pt = t / a, qt = x / a;
  if (it == 0 && ix == 0) {
    return (pt == pw && qt == qw && tau == beta) ? make_double2(1.0, 0.0) : make_double2(0.0, 0.0);
  }
  const int l = it * a + ix;
  const int lr = 2 * (l - 1) + tau;
  const int tile = pt * Nq + qt;
  int dp, dq;
  row_basket(own, pt, qt, it, ix, dp, dq);
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const int pc = wrap(pt + dp + (c >> 1), Np), qc = wrap(qt + dq + (c & 1), Nq);
    if (pc == pw && qc == qw) return P[((size_t)tile * 8 + 2 * c + beta) * nrows + lr];
  }
  return make_double2(0.0, 0.0);
}

template <typename Op>
__device__ double2 ap_entry(const Op& op, const double2* __restrict__ P, int t, int x, int sigma, int pw, int qw,
                            int beta, int a, int Np, int Nq, int nrows, int own) {
  // (A P)[(s, sigma), (w, beta)] = sum_nb sum_tau A[(s,sigma),(s',tau)] P[(s',tau),(w,beta)]
  double2 acc = make_double2(0.0, 0.0);
  const int nn = op_count(op);
  for (int k = 0; k < nn; ++k) {
    int tn, xn;
    double2 blk[4];
    op_nb(op, t, x, k, tn, xn, blk);
#pragma unroll
    for (int tau = 0; tau < 2; ++tau) {
      const double2 pwv = p_weight(P, tn, xn, tau, pw, qw, beta, a, Np, Nq, nrows, own);
      if (pwv.x != 0.0 || pwv.y != 0.0) acc += cmul(blk[2 * sigma + tau], pwv);
    }
  }
  return acc;
}

// one CTA per coarse site v, thread = (k, alpha, beta) (several passes when
// 4 K exceeds the block): Bc[k][2 alpha + beta][v]
template <typename Op>
__global__ void __launch_bounds__(128)
k_galerkin(Op op, const double2* __restrict__ P, int a, int Np, int Nq, Offsets offc, double2* __restrict__ Bc,
           int own) {
  const int v = blockIdx.x;
  for (int th = threadIdx.x; th < offc.K * 4; th += blockDim.x) {
    const int k = th >> 2, alpha = (th >> 1) & 1, beta = th & 1;
    const int nc = Np * Nq;
    const int p = v / Nq, q = v - (v / Nq) * Nq;
    const int pw = wrap(p + offc.dt[k], Np), qw = wrap(q + offc.dx[k], Nq);
    const int nrows = 2 * (a * a - 1);
    double2 acc = make_double2(0.0, 0.0);
    // v's own fine site: P row is the identity on spin alpha
    acc += ap_entry(op, P, p * a, q * a, alpha, pw, qw, beta, a, Np, Nq, nrows, own);
    // the rows whose basket has v as corner c: the F sites that basket
    // W(p - di, q - dj) owns (under the tile rule: every row of tile (p-di, q-dj))
    for (int c = 0; c < 4; ++c) {
      const int pB = wrap(p - (c >> 1), Np), qB = wrap(q - (c & 1), Nq);
      for (int i = 0; i <= a; ++i)
        for (int j = 0; j <= a; ++j) {
          if ((i == 0 || i == a) && (j == 0 || j == a)) continue;      // corners
          const int it = (i == a) ? 0 : i, jt = (j == a) ? 0 : j;
          const int pT = (i == a) ? wrap(pB + 1, Np) : pB, qT = (j == a) ? wrap(qB + 1, Nq) : qB;
          int dp, dq;
          row_basket(own, pT, qT, it, jt, dp, dq);
          if (wrap(pT + dp, Np) != pB || wrap(qT + dq, Nq) != qB) continue;
          const int l = it * a + jt;
          const int tile = pT * Nq + qT;
          for (int sigma = 0; sigma < 2; ++sigma) {
            const double2 pv = P[((size_t)tile * 8 + 2 * c + alpha) * nrows + 2 * (l - 1) + sigma];
            acc += cmulc(pv, ap_entry(op, P, pT * a + it, qT * a + jt, sigma, pw, qw, beta, a, Np, Nq, nrows, own));
          }
        }
    }
    Bc[((size_t)k * 4 + 2 * alpha + beta) * nc + v] = acc;
  }
}

// Row-sum normalisation of Eq. (16) (N = diag(1 / row sum)): the complex sum
// s of every stored row's 8 weights; the largest |s| of the level goes to
// *smax as the bits of a non-negative double (ordered like unsigned integers).
__global__ void k_rowsum_max(const double2* __restrict__ P, int nrows, int ntiles,
                             unsigned long long* __restrict__ smax) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  double m = 0.0;
  if (g < ntiles * nrows) {
    const int tile = g / nrows, lr = g - (g / nrows) * nrows;
    double2 s = make_double2(0.0, 0.0);
    for (int c8 = 0; c8 < 8; ++c8) s += P[((size_t)tile * 8 + c8) * nrows + lr];
    m = sqrt(cabs2(s));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(smax, (unsigned long long)__double_as_longlong(m));
}

// rows with |s| >= rel_floor * max |s| are divided by s; the others stay and
// are counted
__global__ void k_rowsum_scale(double2* __restrict__ P, int nrows, int ntiles,
                               const unsigned long long* __restrict__ smax, double rel_floor,
                               unsigned* __restrict__ skipped) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= ntiles * nrows) return;
  const int tile = g / nrows, lr = g - (g / nrows) * nrows;
  double2 s = make_double2(0.0, 0.0);
  for (int c8 = 0; c8 < 8; ++c8) s += P[((size_t)tile * 8 + c8) * nrows + lr];
  const double floor_ = rel_floor * __longlong_as_double((long long)*smax);
  if (!(sqrt(cabs2(s)) >= floor_)) {
    atomicAdd(skipped, 1u);
    return;
  }
  const double2 inv = crecip(s);
  for (int c8 = 0; c8 < 8; ++c8) {
    double2& w = P[((size_t)tile * 8 + c8) * nrows + lr];
    w = cmul(w, inv);
  }
}

// ------------------------------------------------------------------ small kernels
__global__ void k_diag_inv(const double2* __restrict__ B, int n, double2* __restrict__ D64, float2* __restrict__ D32,
                           int* __restrict__ err) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  const double2 a = B[v], b = B[n + v], c = B[2 * n + v], d = B[3 * n + v];   // offset 0 = (0, 0)
  const double2 det = cmul(a, d) - cmul(b, c);
  if (cabs2(det) == 0.0) { atomicOr(err, 2); return; }
  const double2 id = crecip(det);
  const double2 r[4] = {cmul(d, id), -cmul(b, id), -cmul(c, id), cmul(a, id)};
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    D64[(size_t)e * n + v] = r[e];
    D32[(size_t)e * n + v] = make_float2((float)r[e].x, (float)r[e].y);
  }
}

__global__ void k_dense_from_blocks(const double2* __restrict__ B, Offsets off, int Nt, int Nx,
                                    double2* __restrict__ Ad) {
  const int n = Nt * Nx, nd = 2 * n;
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= n * off.K) return;
  const int k = g / n, v = g - (g / n) * n;
  const int t = v / Nx, x = v - (v / Nx) * Nx;
  const int w = wrap(t + off.dt[k], Nt) * Nx + wrap(x + off.dx[k], Nx);
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const int al = e >> 1, be = e & 1;
    Ad[(size_t)(al * n + v) * nd + be * n + w] = B[((size_t)k * 4 + e) * n + v];
  }
}

// Gauss-Jordan step k, part 1 (one CTA): pivot search in column k, row swap,
// scaling of the pivot row (its column-k entry becomes 1/pivot), multipliers of
// column k saved to colk (0 at row k).
__global__ void __launch_bounds__(1024)
k_gj_pivot(double2* __restrict__ A, int nd, int k, double2* __restrict__ colk, int* __restrict__ perm,
           int* __restrict__ err, double tol2) {
  __shared__ double sv[32];
  __shared__ int si[32];
  __shared__ int s_p;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  double best = -1.0;
  int bi = k;
  for (int i = k + tid; i < nd; i += blockDim.x) {
    const double v = cabs2(A[(size_t)i * nd + k]);
    if (v > best) { best = v; bi = i; }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double ob = __shfl_xor_sync(0xffffffffu, best, o);
    const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
    if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
  }
  if (lane == 0) { sv[wid] = best; si[wid] = bi; }
  __syncthreads();
  if (wid == 0) {
    const int nw = blockDim.x >> 5;
    best = lane < nw ? sv[lane] : -1.0;
    bi = lane < nw ? si[lane] : nd;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
    }
    if (lane == 0) {
      s_p = bi;
      perm[k] = bi;
      if (!(best > tol2)) atomicOr(err, 4);
    }
  }
  __syncthreads();
  const int p = s_p;
  if (p != k) {
    for (int j = tid; j < nd; j += blockDim.x) {
      const double2 tmp = A[(size_t)k * nd + j];
      A[(size_t)k * nd + j] = A[(size_t)p * nd + j];
      A[(size_t)p * nd + j] = tmp;
    }
  }
  __syncthreads();
  double2 piv = A[(size_t)k * nd + k];
  if (cabs2(piv) == 0.0) piv = make_double2(1.0, 0.0);
  const double2 inv = crecip(piv);
  for (int i = tid; i < nd; i += blockDim.x) colk[i] = (i == k) ? make_double2(0.0, 0.0) : A[(size_t)i * nd + k];
  __syncthreads();
  for (int j = tid; j < nd; j += blockDim.x)
    A[(size_t)k * nd + j] = (j == k) ? inv : cmul(A[(size_t)k * nd + j], inv);
}

// Gauss-Jordan step k, part 2: rows i != k, A[i][j] = (j == k ? 0 : A[i][j]) - colk[i] A[k][j]
__global__ void __launch_bounds__(256)
k_gj_update(double2* __restrict__ A, int nd, int k, const double2* __restrict__ colk) {
  const int i = blockIdx.y;
  if (i == k) return;
  const double2 f = colk[i];
  if (f.x == 0.0 && f.y == 0.0) return;
  const double2* rk = A + (size_t)k * nd;
  double2* ri = A + (size_t)i * nd;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < nd; j += gridDim.x * blockDim.x) {
    const double2 base = (j == k) ? make_double2(0.0, 0.0) : ri[j];
    ri[j] = base - cmul(f, rk[j]);
  }
}

__global__ void k_gather_cols(const double2* __restrict__ X, double2* __restrict__ Y, const int* __restrict__ cols,
                              int nd) {
  const int i = blockIdx.y;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < nd; j += gridDim.x * blockDim.x)
    Y[(size_t)i * nd + j] = X[(size_t)i * nd + cols[j]];
}

// FP16 + scale: one warp per tile; scale = max |re|, |im| over the tile
__global__ void k_pack_P16(const double2* __restrict__ P, int per_tile, int ntiles, __half2* __restrict__ P16,
                           float* __restrict__ scale) {
  const int tile = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (tile >= ntiles) return;
  const double2* src = P + (size_t)tile * per_tile;
  double m = 0.0;
  for (int e = lane; e < per_tile; e += 32) m = fmax(m, fmax(fabs(src[e].x), fabs(src[e].y)));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  float s = (float)m;
  if (s == 0.0f) s = 1.0f;
  const double inv = 1.0 / (double)s;
  for (int e = lane; e < per_tile; e += 32)
    P16[(size_t)tile * per_tile + e] = __halves2half2(__double2half(src[e].x * inv), __double2half(src[e].y * inv));
  if (lane == 0) scale[tile] = s;
}

// one thread per 2x2 block (k, v)
__global__ void k_pack_B16(const double2* __restrict__ B, int K, int n, __half2* __restrict__ B16,
                           float* __restrict__ scale) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= K * n) return;
  const int k = g / n, v = g - (g / n) * n;
  double m = 0.0;
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const double2 b = B[((size_t)k * 4 + e) * n + v];
    m = fmax(m, fmax(fabs(b.x), fabs(b.y)));
  }
  float s = (float)m;
  if (s == 0.0f) s = 1.0f;
  const double inv = 1.0 / (double)s;
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const double2 b = B[((size_t)k * 4 + e) * n + v];
    B16[((size_t)k * 4 + e) * n + v] = __halves2half2(__double2half(b.x * inv), __double2half(b.y * inv));
  }
  scale[(size_t)k * n + v] = s;
}

// Colour-major copies of a smoothed level for the Gauss-Seidel kernels (layout
// described with gs_site): thread per (colour, off-diagonal offset, site of the
// colour) for the blocks, the diagonal inverses by the threads with offset 0.
__global__ void k_pack_colour_major(const double2* __restrict__ B64, const __half2* __restrict__ B16,
                                    const float* __restrict__ Bs, const double2* __restrict__ D64,
                                    const float2* __restrict__ D32, int K, int Nt, int Nx, int ncol,
                                    double2* __restrict__ Bc64, __half2* __restrict__ Bc16, float* __restrict__ Bcs,
                                    double2* __restrict__ Dc64, float2* __restrict__ Dc32) {
  const int n = Nt * Nx, m = n / ncol, K1 = K - 1;
  const long g = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= (long)ncol * K1 * m) return;
  const int j = (int)(g % m);
  const int kk = (int)((g / m) % K1);
  const int c = (int)(g / ((long)m * K1));
  int t, x;
  colour_site(ncol, c, j, Nx, t, x);
  const int v = t * Nx + x, k = kk + 1;
  const size_t blk = ((size_t)c * K1 + kk) * m + j;
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    Bc64[blk * 4 + e] = B64[((size_t)k * 4 + e) * n + v];
    Bc16[blk * 4 + e] = B16[((size_t)k * 4 + e) * n + v];
  }
  Bcs[blk] = Bs[(size_t)k * n + v];
  if (kk == 0) {
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      Dc64[((size_t)c * m + j) * 4 + e] = D64[(size_t)e * n + v];
      Dc32[((size_t)c * m + j) * 4 + e] = D32[(size_t)e * n + v];
    }
  }
}

}  // namespace

cudaError_t launch_pack_colour_major(const double2* B64, const __half2* B16, const float* Bs, const double2* D64,
                                     const float2* D32, int K, int Nt, int Nx, int ncol, double2* Bc64, __half2* Bc16,
                                     float* Bcs, double2* Dc64, float2* Dc32, cudaStream_t st) {
  const long total = (long)ncol * (K - 1) * (Nt * Nx / ncol);
  k_pack_colour_major<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(B64, B16, Bs, D64, D32, K, Nt, Nx, ncol, Bc64,
                                                                     Bc16, Bcs, Dc64, Dc32);
  return cudaGetLastError();
}

template <typename Op>
cudaError_t launch_local_solve(const Op& op, int a, int Np, int Nq, double2* P, int* err, int own, cudaStream_t st) {
  const double rel_tol = 1e-13;
  if (a == 4) k_local_solve<4, Op><<<Np * Nq, 128, 0, st>>>(op, Np, Nq, P, err, rel_tol, own);
  else if (a == 2) k_local_solve<2, Op><<<Np * Nq, 128, 0, st>>>(op, Np, Nq, P, err, rel_tol, own);
  else return cudaErrorInvalidValue;
  return cudaGetLastError();
}

template <typename Op>
cudaError_t launch_galerkin(const Op& op, const double2* P, int a, int Np, int Nq, const Offsets& offc, double2* Bc,
                            int own, cudaStream_t st) {
  k_galerkin<Op><<<Np * Nq, 128, 0, st>>>(op, P, a, Np, Nq, offc, Bc, own);
  return cudaGetLastError();
}

cudaError_t launch_rowsum_normalize(double2* P, int nrows, int ntiles, unsigned long long* smax, unsigned* skipped,
                                    cudaStream_t st) {
  const int total = ntiles * nrows;
  cudaError_t e = cudaMemsetAsync(smax, 0, sizeof(unsigned long long), st);
  if (e != cudaSuccess) return e;
  k_rowsum_max<<<(total + 255) / 256, 256, 0, st>>>(P, nrows, ntiles, smax);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_rowsum_scale<<<(total + 255) / 256, 256, 0, st>>>(P, nrows, ntiles, smax, 1e-12, skipped);
  return cudaGetLastError();
}

cudaError_t launch_diag_inv(const double2* B, int n, double2* D64, float2* D32, int* err, cudaStream_t st) {
  k_diag_inv<<<(n + 255) / 256, 256, 0, st>>>(B, n, D64, D32, err);
  return cudaGetLastError();
}

cudaError_t launch_dense_from_blocks(const double2* B, const Offsets& off, int Nt, int Nx, double2* Ad,
                                     cudaStream_t st) {
  const int total = Nt * Nx * off.K;
  k_dense_from_blocks<<<(total + 255) / 256, 256, 0, st>>>(B, off, Nt, Nx, Ad);
  return cudaGetLastError();
}

cudaError_t launch_gj_step(double2* A, int nd, int k, double2* colk, int* perm, int* err, double tol2,
                           cudaStream_t st) {
  k_gj_pivot<<<1, 1024, 0, st>>>(A, nd, k, colk, perm, err, tol2);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int bx = (nd + 255) / 256;
  dim3 grid(bx < 4 ? bx : 4, nd);
  k_gj_update<<<grid, 256, 0, st>>>(A, nd, k, colk);
  return cudaGetLastError();
}

cudaError_t launch_gather_cols(const double2* X, double2* Y, const int* cols, int nd, cudaStream_t st) {
  const int bx = (nd + 255) / 256;
  dim3 grid(bx < 8 ? bx : 8, nd);
  k_gather_cols<<<grid, 256, 0, st>>>(X, Y, cols, nd);
  return cudaGetLastError();
}

namespace {
// Spin-split interpolation: zero the weights that couple different spins
// (column 2c + beta, row 2(l-1) + alpha with alpha != beta) of every tile.
__global__ void k_spin_split_P(double2* __restrict__ P, int nrows, long total) {
  const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= total) return;
  const int lr = (int)(idx % nrows);
  const int col = (int)((idx / nrows) % 8);
  if ((col & 1) != (lr & 1)) P[idx] = make_double2(0.0, 0.0);
}
}  // namespace

cudaError_t launch_spin_split_P(double2* P, int nrows, int ntiles, cudaStream_t st) {
  const long total = (long)ntiles * 8 * nrows;
  k_spin_split_P<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(P, nrows, total);
  return cudaGetLastError();
}

cudaError_t launch_pack_P16(const double2* P, int per_tile, int ntiles, __half2* P16, float* scale,
                            cudaStream_t st) {
  k_pack_P16<<<(ntiles * 32 + 255) / 256, 256, 0, st>>>(P, per_tile, ntiles, P16, scale);
  return cudaGetLastError();
}

cudaError_t launch_pack_B16(const double2* B, int K, int n, __half2* B16, float* scale, cudaStream_t st) {
  k_pack_B16<<<(K * n + 255) / 256, 256, 0, st>>>(B, K, n, B16, scale);
  return cudaGetLastError();
}

template cudaError_t launch_local_solve<WilsonOp>(const WilsonOp&, int, int, int, double2*, int*, int,
                                                  cudaStream_t);
template cudaError_t launch_local_solve<StencilOp>(const StencilOp&, int, int, int, double2*, int*, int,
                                                   cudaStream_t);
template cudaError_t launch_galerkin<WilsonOp>(const WilsonOp&, const double2*, int, int, int, const Offsets&,
                                               double2*, int, cudaStream_t);
template cudaError_t launch_galerkin<StencilOp>(const StencilOp&, const double2*, int, int, int, const Offsets&,
                                                double2*, int, cudaStream_t);
