// Coarsest-level solve by unpreconditioned restarted GMRES to a relative
// residual of 0.1 from a zero start: the paper's coarsest solver (Sec. 5,
// solver settings), the alternative to the exact solve by the dense inverse.
//
// It runs inside the V-cycle (and so inside each captured Arnoldi step), so
// it cannot return to the host: the whole solve of R right-hand sides is one
// cooperative kernel.  Work units (right-hand side, coarse site) are spread
// over every block; the steps that need global sums end at a grid barrier whose
// last-arriving block adds the blocks' partial sums in block order
// (deterministic), updates the small Hessenberg problem of every right-hand
// side (Givens rotations, in FP64) and publishes the result before releasing
// the others.  Per Arnoldi step:
//   (1) w = A v_j and the inner products <v_i, w>          -> barrier
//   (2) w -= sum h_i v_i, second inner products (CGS2)      -> barrier
//   (3) w -= sum h'_i v_i and ||w||^2                       -> barrier: Givens,
//       residual estimate |g_{j+1}|, end of the cycle for this right-hand side
//       when it is at most tol ||r||.
// The basis is stored unnormalised with the inverse norms s_i kept aside.  At
// the end of a cycle e += V y, then the true residual r - A e decides (a new
// cycle starts from it unless it is below tol ||r||).  A right-hand side that
// is done takes no further part.  Barrier waits are bounded: a time-out sets
// sync[2] (reported by the host like the coarse smoothers' time-outs) and the
// kernel stops.
#include "context.h"

namespace {

constexpr int GM_THREADS = 256;
constexpr unsigned GM_SPIN_LIMIT = 1u << 23;

template <typename T, typename BT>
__device__ __forceinline__ typename cplx<T>::type gm_b(const BT* B, const float* sc, int k, int e, int n, int v);
template <>
__device__ __forceinline__ double2 gm_b<double, double2>(const double2* B, const float*, int k, int e, int n, int v) {
  return B[((size_t)k * 4 + e) * n + v];
}
template <>
__device__ __forceinline__ float2 gm_b<float, __half2>(const __half2* B, const float* sc, int k, int e, int n, int v) {
  return h2c<float>(B[((size_t)k * 4 + e) * n + v], sc[(size_t)k * n + v]);
}

template <typename T, typename BT>
struct GmArgs {
  using C = typename cplx<T>::type;
  const C* r;           // [R][2n] right-hand sides
  C* e;                 // [R][2n] solution (zero start)
  const BT* B;          // [K][4][n] level operator
  const float* Bs;      // its FP32 scales (FP16 copy only)
  Offsets off;
  int Nt, Nx, R, m, max_cycles;
  double tol;
  C* V;                 // [m + 1][R][2n] raw basis
  double2* part;        // [gridDim][R][m + 2] block partial sums
  GmresRhs* st;         // [R] Hessenberg problems (written by the last block of a barrier)
  unsigned* sync;       // {count, generation, time-out}
  int* all_done;        // published by the last block
};

// (A x)_v for both spins of site v of one right-hand side, x scaled by s
// (x read through L2: other blocks wrote it)
template <typename T, typename BT>
__device__ __forceinline__ void gm_apply(const GmArgs<T, BT>& a, const typename cplx<T>::type* x, T s, int v,
                                         typename cplx<T>::type& y0, typename cplx<T>::type& y1) {
  using C = typename cplx<T>::type;
  const int n = a.Nt * a.Nx;
  const int t = v / a.Nx, xx = v - (v / a.Nx) * a.Nx;
  y0 = czero<C>();
  y1 = czero<C>();
  for (int k = 0; k < a.off.K; ++k) {
    int tw = t + a.off.dt[k]; tw -= (tw >= a.Nt) ? a.Nt : 0;
    int xw = xx + a.off.dx[k]; xw -= (xw >= a.Nx) ? a.Nx : 0;
    const int w = tw * a.Nx + xw;
    const C x0 = s * __ldcg(x + w), x1 = s * __ldcg(x + n + w);
    cmac(y0, gm_b<T, BT>(a.B, a.Bs, k, 0, n, v), x0);
    cmac(y0, gm_b<T, BT>(a.B, a.Bs, k, 1, n, v), x1);
    cmac(y1, gm_b<T, BT>(a.B, a.Bs, k, 2, n, v), x0);
    cmac(y1, gm_b<T, BT>(a.B, a.Bs, k, 3, n, v), x1);
  }
}

// Grid barrier; the last block to arrive runs f() with all its threads before
// the others are released.  Every thread fences its own global stores first.
// Returns false after a time-out.
template <typename F>
__device__ __forceinline__ bool gm_barrier(unsigned* sync, F f) {
  __shared__ int last, ok;
  __shared__ unsigned gen0;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    gen0 = *reinterpret_cast<volatile unsigned*>(sync + 1);
    __threadfence();
    last = atomicAdd(sync, 1u) == gridDim.x - 1;
    ok = 1;
  }
  __syncthreads();
  if (last) {
    __threadfence();
    f();
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
      sync[0] = 0;
      __threadfence();
      atomicExch(sync + 1, gen0 + 1);
    }
  } else if (threadIdx.x == 0) {
    const volatile unsigned* gen = sync + 1;
    unsigned it = 0;
    while (*gen == gen0) {
      if (++it == GM_SPIN_LIMIT) {
        atomicExch(sync + 2, 1u);
        ok = 0;
        break;
      }
      __nanosleep(64);
    }
    __threadfence();
  }
  __syncthreads();
  return ok != 0;
}

// sum over blocks of part[.][rhs][idx] (fixed order)
__device__ __forceinline__ double2 gm_total(const double2* part, int R, int m, int rhs, int idx) {
  double2 s = make_double2(0.0, 0.0);
  const int per = m + 2;
  for (int b = 0; b < (int)gridDim.x; ++b) s += __ldcg(part + ((size_t)b * R + rhs) * per + idx);
  return s;
}

template <typename T, typename BT>
__global__ void __launch_bounds__(GM_THREADS)
k_coarsest_gmres(GmArgs<T, BT> a) {
  using C = typename cplx<T>::type;
  // dynamic shared memory, per right-hand side rhs and index i < m + 2:
  //   sp[rhs][i] block partial sums, sc[rhs][i] coefficients of the phase,
  //   ss[rhs][i] inverse basis norms; sf[rhs] 1 while the right-hand side runs
  extern __shared__ double2 smem[];
  const int R = a.R, m = a.m, per = m + 2;
  double2* sp = smem;
  double2* sc = sp + (size_t)R * per;
  double* ss = reinterpret_cast<double*>(sc + (size_t)R * per);
  int* sf = reinterpret_cast<int*>(ss + (size_t)R * per);
  __shared__ int s_any;
  const int n = a.Nt * a.Nx;
  const size_t len = 2 * (size_t)n;
  const long units = (long)R * n;
  const long stride = (long)gridDim.x * blockDim.x;
  auto vec = [&](int i, int rhs) { return a.V + ((size_t)i * R + rhs) * len; };
  // zero the partial sums and copy the phase's per-RHS data from the state
  // (through L2: the last block of the previous barrier wrote it); coef: 0 none,
  // 1 the Hessenberg column j, 2 the second-pass coefficients, 3 y
  auto begin_phase = [&](int j, int coef, bool need_cycle) {
    for (int i = threadIdx.x; i < R * per; i += blockDim.x) {
      const int rhs = i / per, k = i - rhs * per;
      const GmresRhs* q = a.st + rhs;
      sp[i] = make_double2(0.0, 0.0);
      ss[i] = (k <= m) ? __ldcg(q->s + k) : 0.0;
      double2 c = make_double2(0.0, 0.0);
      if (coef == 1 && k <= j) c = __ldcg(q->H + k * GMRES_MAX_M + j);
      else if (coef == 2 && k <= j) c = __ldcg(q->H2 + k);
      else if (coef == 3 && k < GMRES_MAX_M) c = __ldcg(q->y + k);
      sc[i] = c;
      if (k == 0) {
        const int done = __ldcg(&q->done), cdone = __ldcg(&q->cdone);
        sf[rhs] = need_cycle ? (!done && !cdone) : !done;
        if (coef == 3) sf[rhs] = done ? 0 : 1 + __ldcg(&q->k);   // 1 + number of basis vectors in use
      }
    }
    __syncthreads();
  };
  auto publish = [&]() {
    for (int i = threadIdx.x; i < R * per; i += blockDim.x) a.part[(size_t)blockIdx.x * R * per + i] = sp[i];
  };
  auto any_left = [&](int live) {
    if (threadIdx.x == 0) s_any = 0;
    __syncthreads();
    if (live) atomicOr(&s_any, 1);
    __syncthreads();
    if (threadIdx.x == 0) *a.all_done = s_any ? 0 : 1;
  };

  for (int cycle = 0; cycle < a.max_cycles; ++cycle) {
    // ---- residual of the current iterate: v_0 = r - A e, ||v_0||^2
    begin_phase(0, 0, false);
    for (long u = (long)blockIdx.x * blockDim.x + threadIdx.x; u < units; u += stride) {
      const int rhs = (int)(u / n), v = (int)(u - (long)rhs * n);
      if (!sf[rhs]) continue;
      C y0 = czero<C>(), y1 = czero<C>();
      if (cycle > 0) gm_apply<T, BT>(a, a.e + rhs * len, T(1), v, y0, y1);
      const C* rr = a.r + rhs * len;
      const C w0 = rr[v] - y0, w1 = rr[n + v] - y1;
      C* v0 = vec(0, rhs);
      __stcg(v0 + v, w0);
      __stcg(v0 + n + v, w1);
      atomicAdd(&sp[rhs * per].x, (double)(cabs2(w0) + cabs2(w1)));
    }
    __syncthreads();
    publish();
    if (!gm_barrier(a.sync, [&] {
          int live = 0;
          for (int rhs = threadIdx.x; rhs < R; rhs += blockDim.x) {
            GmresRhs* q = a.st + rhs;
            if (__ldcg(&q->done)) continue;
            const double beta = sqrt(gm_total(a.part, R, m, rhs, 0).x);
            double bnorm = __ldcg(&q->bnorm);
            if (cycle == 0) { bnorm = beta; q->bnorm = beta; }
            if (!(beta > a.tol * bnorm) || !isfinite(beta)) { q->done = 1; continue; }
            q->s[0] = 1.0 / beta;
            q->g[0] = make_double2(beta, 0.0);
            q->k = 0;
            q->cdone = 0;
            ++live;
          }
          any_left(live);
        }))
      return;
    if (*reinterpret_cast<volatile int*>(a.all_done)) break;

    int jend = 0;
    for (int j = 0; j < m; ++j) {
      jend = j + 1;
      // ---- (1) w = A (s_j v_j) into slot j + 1, inner products with v_0..v_j
      begin_phase(j, 0, true);
      for (long u = (long)blockIdx.x * blockDim.x + threadIdx.x; u < units; u += stride) {
        const int rhs = (int)(u / n), v = (int)(u - (long)rhs * n);
        if (!sf[rhs]) continue;
        const double* s = ss + rhs * per;
        C w0, w1;
        gm_apply<T, BT>(a, vec(j, rhs), (T)s[j], v, w0, w1);
        C* wv = vec(j + 1, rhs);
        __stcg(wv + v, w0);
        __stcg(wv + n + v, w1);
        for (int i = 0; i <= j; ++i) {
          const C* vi = vec(i, rhs);
          C d = czero<C>();
          cmacc(d, __ldcg(vi + v), w0);
          cmacc(d, __ldcg(vi + n + v), w1);
          atomicAdd(&sp[rhs * per + i].x, (double)d.x * s[i]);
          atomicAdd(&sp[rhs * per + i].y, (double)d.y * s[i]);
        }
      }
      __syncthreads();
      publish();
      if (!gm_barrier(a.sync, [&] {
            for (int e2 = threadIdx.x; e2 < R * (j + 1); e2 += blockDim.x) {
              const int rhs = e2 / (j + 1), i = e2 - rhs * (j + 1);
              GmresRhs* q = a.st + rhs;
              if (__ldcg(&q->done) || __ldcg(&q->cdone)) continue;
              q->H[i * GMRES_MAX_M + j] = gm_total(a.part, R, m, rhs, i);
            }
          }))
        return;
      // ---- (2) w -= sum_i h_i s_i v_i, second inner products
      begin_phase(j, 1, true);
      for (long u = (long)blockIdx.x * blockDim.x + threadIdx.x; u < units; u += stride) {
        const int rhs = (int)(u / n), v = (int)(u - (long)rhs * n);
        if (!sf[rhs]) continue;
        const double* s = ss + rhs * per;
        const double2* h = sc + rhs * per;
        C* wv = vec(j + 1, rhs);
        C w0 = __ldcg(wv + v), w1 = __ldcg(wv + n + v);
        for (int i = 0; i <= j; ++i) {
          const C c = mk((T)(h[i].x * s[i]), (T)(h[i].y * s[i]));
          const C* vi = vec(i, rhs);
          w0 -= cmul(c, __ldcg(vi + v));
          w1 -= cmul(c, __ldcg(vi + n + v));
        }
        __stcg(wv + v, w0);
        __stcg(wv + n + v, w1);
        for (int i = 0; i <= j; ++i) {
          const C* vi = vec(i, rhs);
          C d = czero<C>();
          cmacc(d, __ldcg(vi + v), w0);
          cmacc(d, __ldcg(vi + n + v), w1);
          atomicAdd(&sp[rhs * per + i].x, (double)d.x * s[i]);
          atomicAdd(&sp[rhs * per + i].y, (double)d.y * s[i]);
        }
      }
      __syncthreads();
      publish();
      if (!gm_barrier(a.sync, [&] {
            for (int e2 = threadIdx.x; e2 < R * (j + 1); e2 += blockDim.x) {
              const int rhs = e2 / (j + 1), i = e2 - rhs * (j + 1);
              GmresRhs* q = a.st + rhs;
              if (__ldcg(&q->done) || __ldcg(&q->cdone)) continue;
              q->H2[i] = gm_total(a.part, R, m, rhs, i);
            }
          }))
        return;
      // ---- (3) w -= sum_i h'_i s_i v_i, ||w||^2; Givens and the residual estimate
      begin_phase(j, 2, true);
      for (long u = (long)blockIdx.x * blockDim.x + threadIdx.x; u < units; u += stride) {
        const int rhs = (int)(u / n), v = (int)(u - (long)rhs * n);
        if (!sf[rhs]) continue;
        const double* s = ss + rhs * per;
        const double2* h = sc + rhs * per;
        C* wv = vec(j + 1, rhs);
        C w0 = __ldcg(wv + v), w1 = __ldcg(wv + n + v);
        for (int i = 0; i <= j; ++i) {
          const C c = mk((T)(h[i].x * s[i]), (T)(h[i].y * s[i]));
          const C* vi = vec(i, rhs);
          w0 -= cmul(c, __ldcg(vi + v));
          w1 -= cmul(c, __ldcg(vi + n + v));
        }
        __stcg(wv + v, w0);
        __stcg(wv + n + v, w1);
        atomicAdd(&sp[rhs * per + m + 1].x, (double)(cabs2(w0) + cabs2(w1)));
      }
      __syncthreads();
      publish();
      if (!gm_barrier(a.sync, [&] {
            int live = 0;
            for (int rhs = threadIdx.x; rhs < R; rhs += blockDim.x) {
              GmresRhs* q = a.st + rhs;
              if (__ldcg(&q->done) || __ldcg(&q->cdone)) continue;
              double2* H = q->H;
              for (int i = 0; i <= j; ++i) H[i * GMRES_MAX_M + j] = __ldcg(H + i * GMRES_MAX_M + j) + __ldcg(q->H2 + i);
              const double hn = sqrt(gm_total(a.part, R, m, rhs, m + 1).x);
              // earlier rotations, then the one that annihilates H[j+1][j]
              for (int i = 0; i < j; ++i) {
                const double ci = __ldcg(q->cs + i);
                const double2 si = __ldcg(q->sn + i);
                const double2 x0 = __ldcg(H + i * GMRES_MAX_M + j), x1 = __ldcg(H + (i + 1) * GMRES_MAX_M + j);
                H[i * GMRES_MAX_M + j] = ci * x0 + cmul(si, x1);
                H[(i + 1) * GMRES_MAX_M + j] = ci * x1 - cmulc(si, x0);
              }
              const double2 x0 = __ldcg(H + j * GMRES_MAX_M + j);
              const double ax = sqrt(cabs2(x0));
              double c;
              double2 sv;
              if (hn == 0.0) { c = 1.0; sv = make_double2(0.0, 0.0); }
              else if (ax == 0.0) { c = 0.0; sv = make_double2(1.0, 0.0); }
              else {
                const double rr = hypot(ax, hn);
                c = ax / rr;
                sv = make_double2(x0.x / ax * hn / rr, x0.y / ax * hn / rr);
              }
              q->cs[j] = c;
              q->sn[j] = sv;
              H[j * GMRES_MAX_M + j] = c * x0 + hn * sv;
              const double2 gj = __ldcg(q->g + j);
              const double2 gn = -1.0 * cmulc(sv, gj);
              q->g[j + 1] = gn;
              q->g[j] = c * gj;
              q->s[j + 1] = hn > 0.0 ? 1.0 / hn : 0.0;
              q->k = j + 1;
              q->iters = __ldcg(&q->iters) + 1;
              if (!(sqrt(cabs2(gn)) > a.tol * __ldcg(&q->bnorm)) || hn == 0.0 || !isfinite(hn)) q->cdone = 1;
              else ++live;
            }
            any_left(live);
          }))
        return;
      if (*reinterpret_cast<volatile int*>(a.all_done)) break;
    }
    (void)jend;
    // ---- least squares of every right-hand side (one thread each)
    if (!gm_barrier(a.sync, [&] {
          for (int rhs = threadIdx.x; rhs < R; rhs += blockDim.x) {
            GmresRhs* q = a.st + rhs;
            if (__ldcg(&q->done)) continue;
            const int k = __ldcg(&q->k);
            for (int i = k - 1; i >= 0; --i) {
              double2 sacc = __ldcg(q->g + i);
              for (int l = i + 1; l < k; ++l) sacc -= cmul(__ldcg(q->H + i * GMRES_MAX_M + l), q->y[l]);
              const double2 d = __ldcg(q->H + i * GMRES_MAX_M + i);
              const double dd = cabs2(d);
              q->y[i] = make_double2((sacc.x * d.x + sacc.y * d.y) / dd, (sacc.y * d.x - sacc.x * d.y) / dd);
            }
          }
        }))
      return;
    // ---- e += V diag(s) y
    begin_phase(0, 3, false);
    for (long u = (long)blockIdx.x * blockDim.x + threadIdx.x; u < units; u += stride) {
      const int rhs = (int)(u / n), v = (int)(u - (long)rhs * n);
      const int kk = sf[rhs] - 1;
      if (kk < 0) continue;
      const double* s = ss + rhs * per;
      const double2* y = sc + rhs * per;
      C* ev = a.e + rhs * len;
      C x0 = __ldcg(ev + v), x1 = __ldcg(ev + n + v);
      for (int i = 0; i < kk; ++i) {
        const C c = mk((T)(y[i].x * s[i]), (T)(y[i].y * s[i]));
        const C* vi = vec(i, rhs);
        x0 += cmul(c, __ldcg(vi + v));
        x1 += cmul(c, __ldcg(vi + n + v));
      }
      __stcg(ev + v, x0);
      __stcg(ev + n + v, x1);
    }
    if (!gm_barrier(a.sync, [] {})) return;   // the next residual reads neighbours' e
  }
}

}  // namespace

size_t coarsest_gmres_smem(int R, int m) {
  return (size_t)R * (m + 2) * (2 * sizeof(double2) + sizeof(double)) + (size_t)R * sizeof(int);
}

// Blocks that can be co-resident for GMRES_MAX_R right-hand sides and restart
// m (at most two per SM), 0 without cooperative launches.  Queried once in setup.
template <typename T, typename BT>
int coarsest_gmres_blocks(int m) {
  int dev = 0, sms = 0, occ = 0, coop = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_coarsest_gmres<T, BT>, GM_THREADS,
                                                    coarsest_gmres_smem(GMRES_MAX_R, m)) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  if (!coop || occ <= 0) return 0;
  return sms * (occ < 2 ? occ : 2);
}

template <typename T, typename BT>
cudaError_t launch_coarsest_gmres(const typename cplx<T>::type* r, typename cplx<T>::type* e, const BT* B,
                                  const float* Bs, const Offsets& off, int Nt, int Nx, int R, int m, double tol,
                                  int max_cycles, typename cplx<T>::type* V, double2* part, GmresRhs* st,
                                  unsigned* sync, int* all_done, int max_blocks, cudaStream_t s) {
  const long want = ((long)R * Nt * Nx + GM_THREADS - 1) / GM_THREADS;
  const int nb = (int)(want < max_blocks ? want : max_blocks);
  if (nb <= 0 || m > GMRES_MAX_M || R > GMRES_MAX_R) return cudaErrorNotSupported;
  cudaError_t err = cudaMemsetAsync(st, 0, sizeof(GmresRhs) * R, s);
  if (err == cudaSuccess) err = cudaMemsetAsync(e, 0, sizeof(typename cplx<T>::type) * 2 * (size_t)Nt * Nx * R, s);
  if (err != cudaSuccess) return err;
  GmArgs<T, BT> a;
  a.r = r; a.e = e; a.B = B; a.Bs = Bs; a.off = off; a.Nt = Nt; a.Nx = Nx; a.R = R; a.m = m;
  a.max_cycles = max_cycles; a.tol = tol; a.V = V; a.part = part; a.st = st; a.sync = sync; a.all_done = all_done;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(nb);
  cfg.blockDim = dim3(GM_THREADS);
  cfg.dynamicSmemBytes = coarsest_gmres_smem(R, m);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_coarsest_gmres<T, BT>, a);
}

template int coarsest_gmres_blocks<double, double2>(int);
template int coarsest_gmres_blocks<float, __half2>(int);
template cudaError_t launch_coarsest_gmres<double, double2>(const double2*, double2*, const double2*, const float*,
                                                            const Offsets&, int, int, int, int, double, int,
                                                            double2*, double2*, GmresRhs*, unsigned*, int*, int,
                                                            cudaStream_t);
template cudaError_t launch_coarsest_gmres<float, __half2>(const float2*, float2*, const __half2*, const float*,
                                                           const Offsets&, int, int, int, int, double, int, float2*,
                                                           double2*, GmresRhs*, unsigned*, int*, int, cudaStream_t);
