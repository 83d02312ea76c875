// Host engine and C ABI: hierarchy setup (Sec. 2, Sec. 4.1), the V-cycle of
// Algorithm 1 used as preconditioner, the FP64 flexible GMRES outer solver, and
// the apply/export entry points declared in include/amamg.h.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <set>
#include <utility>

#include "context.h"

namespace {

#define CK(call)                                                              \
  do {                                                                        \
    cudaError_t e_ = (call);                                                  \
    if (e_ != cudaSuccess) {                                                  \
      h->err = std::string(#call) + ": " + cudaGetErrorString(e_);           \
      return e_ == cudaErrorMemoryAllocation ? AMAMG_ERR_OOM : AMAMG_ERR_CUDA; \
    }                                                                         \
  } while (0)

#define CKS(expr)              \
  do {                         \
    int s_ = (expr);           \
    if (s_ != AMAMG_OK) return s_; \
  } while (0)

inline cudaStream_t S(void* s) { return reinterpret_cast<cudaStream_t>(s); }

// ----------------------------------------------------------------- profiling
int cat_id(amamg_ctx* h, const char* name) {
  for (size_t i = 0; i < h->cats.size(); ++i)
    if (h->cats[i].name == name) return (int)i;
  h->cats.push_back(ProfCat{name});
  return (int)h->cats.size() - 1;
}

cudaEvent_t take_event(amamg_ctx* h) {
  if (h->ev_used == h->ev_pool.size()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    h->ev_pool.push_back(e);
  }
  return h->ev_pool[h->ev_used++];
}

// Wraps one kernel launch: counts it and, when profiling, brackets it with events.
template <typename F>
int launch(amamg_ctx* h, const char* name, double bytes, cudaStream_t st, F&& f, double flops = 0.0) {
  ProfRec rec{-1, nullptr, nullptr, bytes, flops};
  if (h->prof) {
    rec.cat = cat_id(h, name);
    rec.a = take_event(h);
    rec.b = take_event(h);
    if (rec.a) cudaEventRecord(rec.a, st);
  }
  cudaError_t e = f();
  if (e != cudaSuccess) {
    h->err = std::string(name) + ": " + cudaGetErrorString(e);
    return AMAMG_ERR_CUDA;
  }
  h->launches++;
  if (h->prof && rec.a && rec.b) {
    cudaEventRecord(rec.b, st);
    h->recs.push_back(rec);
  }
  return AMAMG_OK;
}

int collect_profile(amamg_ctx* h) {
  for (auto& r : h->recs) {
    if (cudaEventSynchronize(r.b) != cudaSuccess) return AMAMG_ERR_CUDA;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, r.a, r.b);
    ProfCat& c = h->cats[r.cat];
    c.launches++;
    c.ms += ms;
    c.bytes += r.bytes;
    c.flops += r.flops;
  }
  h->recs.clear();
  h->ev_used = 0;
  return AMAMG_OK;
}

template <typename P>
int dalloc(amamg_ctx* h, P** p, size_t count) {
  *p = nullptr;
  if (count == 0) return AMAMG_OK;
  // failure injection on the host (AMAMG_FAIL_ALLOC_AFTER=n, read by
  // amamg_setup): the handle's allocation number n + 1 and later report
  // out-of-memory without calling cudaMalloc, so the error paths can be tested
  // without exhausting the device
  if (h->fail_alloc_after >= 0 && h->allocs++ >= h->fail_alloc_after) {
    h->err = "cudaMalloc: out of memory (injected by AMAMG_FAIL_ALLOC_AFTER)";
    return AMAMG_ERR_OOM;
  }
  cudaError_t e = cudaMalloc((void**)p, count * sizeof(P));
  if (e != cudaSuccess) {
    h->err = std::string("cudaMalloc: ") + cudaGetErrorString(e);
    cudaGetLastError();
    return AMAMG_ERR_OOM;
  }
  return AMAMG_OK;
}

template <typename P>
void dfree(P*& p) {
  if (p) cudaFree((void*)p);
  p = nullptr;
}

// ----------------------------------------------------------------- structure
Offsets wilson_offsets(int Nt, int Nx) {
  std::set<std::pair<int, int>> s = {{0, 0}, {1 % Nt, 0}, {(Nt - 1) % Nt, 0}, {0, 1 % Nx}, {0, (Nx - 1) % Nx}};
  Offsets o{};
  o.K = 0;
  for (auto& p : s) { o.dt[o.K] = p.first; o.dx[o.K] = p.second; ++o.K; }
  return o;
}

// Block offsets of P^H A P from the structural patterns (translation invariant
// under the tile ownership rule, so coarse site 0 represents every row): the
// support of coarse column 0 is its own vertex site plus the owned sites of the
// four tiles that have it as a corner; A widens it by its offsets; each reached
// site contributes its vertex (vertex row) or its tile's four corners.
int coarse_offsets_owned(const Offsets& fine, int Nt, int Nx, int a, int own, Offsets* out);

int coarse_offsets(const Offsets& fine, int Nt, int Nx, int a, int own, Offsets* out) {
  if (own != OWN_TILE) return coarse_offsets_owned(fine, Nt, Nx, a, own, out);
  const int Np = Nt / a, Nq = Nx / a;
  std::set<std::pair<int, int>> W;
  std::vector<std::pair<int, int>> supp;
  supp.push_back({0, 0});
  for (int c = 0; c < 4; ++c) {
    const int pT = wrap(-(c >> 1), Np), qT = wrap(-(c & 1), Nq);
    for (int i = 0; i < a; ++i)
      for (int j = 0; j < a; ++j)
        if (i || j) supp.push_back({pT * a + i, qT * a + j});
  }
  for (auto& s : supp) {
    for (int k = 0; k < fine.K; ++k) {
      const int t = wrap(s.first + fine.dt[k], Nt), x = wrap(s.second + fine.dx[k], Nx);
      const int pt = t / a, qt = x / a;
      if (t % a == 0 && x % a == 0) {
        W.insert({pt, qt});
      } else {
        for (int c = 0; c < 4; ++c) W.insert({wrap(pt + (c >> 1), Np), wrap(qt + (c & 1), Nq)});
      }
    }
  }
  if ((int)W.size() > AMAMG_MAX_OFFSETS) return AMAMG_ERR_INVALID_ARG;
  Offsets o{};
  o.K = 0;
  for (auto& p : W) { o.dt[o.K] = p.first; o.dx[o.K] = p.second; ++o.K; }
  *out = o;
  return AMAMG_OK;
}

// The same for an ownership rule that is not translation invariant (first-lex:
// the rows of the first tile row and column come from other baskets than
// elsewhere): the column pattern of every coarse column v, i.e. the rows
// (vertices w) reached from v's support (its vertex site and the F sites its
// four corner baskets own) through A, collected as offsets w - v over all v.
int coarse_offsets_owned(const Offsets& fine, int Nt, int Nx, int a, int own, Offsets* out) {
  const int Np = Nt / a, Nq = Nx / a;
  std::vector<char> hit((size_t)Np * Nq, 0);
  std::vector<std::pair<int, int>> supp;
  for (int pv = 0; pv < Np; ++pv)
    for (int qv = 0; qv < Nq; ++qv) {
      supp.clear();
      supp.push_back({pv * a, qv * a});
      for (int c = 0; c < 4; ++c) {
        const int pB = wrap(pv - (c >> 1), Np), qB = wrap(qv - (c & 1), Nq);
        for (int i = 0; i <= a; ++i)
          for (int j = 0; j <= a; ++j) {
            if ((i == 0 || i == a) && (j == 0 || j == a)) continue;
            const int it = (i == a) ? 0 : i, jt = (j == a) ? 0 : j;
            const int pT = (i == a) ? wrap(pB + 1, Np) : pB, qT = (j == a) ? wrap(qB + 1, Nq) : qB;
            int dp, dq;
            row_basket(own, pT, qT, it, jt, dp, dq);
            if (wrap(pT + dp, Np) == pB && wrap(qT + dq, Nq) == qB) supp.push_back({pT * a + it, qT * a + jt});
          }
      }
      for (auto& sv : supp)
        for (int k = 0; k < fine.K; ++k) {
          const int t = wrap(sv.first + fine.dt[k], Nt), x = wrap(sv.second + fine.dx[k], Nx);
          const int pt = t / a, qt = x / a, it = t % a, jt = x % a;
          if (it == 0 && jt == 0) {
            hit[(size_t)wrap(pt - pv, Np) * Nq + wrap(qt - qv, Nq)] = 1;
          } else {
            int dp, dq;
            row_basket(own, pt, qt, it, jt, dp, dq);
            for (int c = 0; c < 4; ++c)
              hit[(size_t)wrap(pt + dp + (c >> 1) - pv, Np) * Nq + wrap(qt + dq + (c & 1) - qv, Nq)] = 1;
          }
        }
    }
  // row v couples to column v + o for every pair found as (w - v) with w the
  // row: the pattern is symmetric (A's is), so both signs are marked
  for (int dt = 0; dt < Np; ++dt)
    for (int dx = 0; dx < Nq; ++dx)
      if (hit[(size_t)dt * Nq + dx]) hit[(size_t)wrap(-dt, Np) * Nq + wrap(-dx, Nq)] = 2;
  Offsets o{};
  o.K = 0;
  for (int dt = 0; dt < Np; ++dt)
    for (int dx = 0; dx < Nq; ++dx) {
      if (!hit[(size_t)dt * Nq + dx]) continue;
      if (o.K == AMAMG_MAX_OFFSETS) return AMAMG_ERR_INVALID_ARG;
      o.dt[o.K] = dt; o.dx[o.K] = dx; ++o.K;
    }
  *out = o;
  return AMAMG_OK;
}

// Colours of the coarse Gauss-Seidel sweep on level L: the 8 classes
// (t + 3x) mod 8 when both extents are multiples of 8 and no off-diagonal
// coupling (dt, dx) has dt + 3 dx = 0 mod 8 (then a colour holds no two coupled
// sites), else the 16 classes (t mod 4, x mod 4).
int gs_colours(const Level& L) {
  if (L.Nt % 8 || L.Nx % 8) return 16;
  for (int k = 0; k < L.off.K; ++k) {
    const int dt = wrap(L.off.dt[k], L.Nt), dx = wrap(L.off.dx[k], L.Nx);
    if (dt == 0 && dx == 0) continue;
    if ((dt + 3 * dx) % 8 == 0) return 16;
  }
  return 8;
}

// Coarse Gauss-Seidel kernel of a smoothed coarse level, per precision.
// FP64: the owner sweep (all SMs, neighbour waits only), else the grid sweep,
// since one 16-block cluster has the FP64 throughput of only 16 SMs.  FP32, one
// right-hand side: the owner sweep, else the 16-block cluster with the level
// in distributed shared memory, else the grid sweep, else the L2 cluster
// sweep, else one launch per colour; FP32 with R >= 2: the cluster sweep where
// it fits (one cluster per right-hand side, 37 us at 64^2 against 47 us for the
// owner sweep at R = 4), else the R = 1 choice.  AMAMG_COARSE_GS = colour | cluster | dsmem | grid |
// owner forces a kernel where it is available (for measurement); results are
// the same.
void choose_gs_kernels(Level& C) {
  OwnerConfig rc;
  const bool owner64 = owner_sweep_config<double, double2>(C.Nt, C.Nx, C.off.K, C.ncol, C.off, 1, &rc);
  const bool owner32 = owner_sweep_config<float, __half2>(C.Nt, C.Nx, C.off.K, C.ncol, C.off, 1, &rc);
  const bool grid64 = grid_sweep_blocks<double, double2>(C.n, C.ncol, 1) > 0;
  const bool grid32 = grid_sweep_blocks<float, __half2>(C.n, C.ncol, 1) > 0;
  const bool dsm64 = dsmem_sweeps_possible<double, double2>(C.n, C.off.K, C.ncol, false);
  const bool dsm32 = dsmem_sweeps_possible<float, __half2>(C.n, C.off.K, C.ncol,
                                                            dsmem_blocks_in_smem<float>(C.n, C.off.K));
  const bool clu32 = use_cluster_sweeps<float>(C.n, C.ncol);
  C.gs64 = owner64 ? GS_OWNER : grid64 ? GS_GRID : dsm64 ? GS_DSMEM : GS_COLOUR;
  C.gs32 = owner32 ? GS_OWNER : dsm32 ? GS_DSMEM : grid32 ? GS_GRID : clu32 ? GS_CLUSTER : GS_COLOUR;
  C.gs32_multi = dsm32 ? GS_DSMEM : C.gs32;
  const char* env = getenv("AMAMG_COARSE_GS");
  if (!env) return;
  const std::string want(env);
  if (want == "colour") { C.gs64 = C.gs32 = GS_COLOUR; }
  else if (want == "cluster") { C.gs32 = clu32 ? GS_CLUSTER : C.gs32; }
  else if (want == "dsmem") { C.gs64 = dsm64 ? GS_DSMEM : C.gs64; C.gs32 = dsm32 ? GS_DSMEM : C.gs32; }
  else if (want == "grid") { C.gs64 = grid64 ? GS_GRID : C.gs64; C.gs32 = grid32 ? GS_GRID : C.gs32; }
  else if (want == "owner") { C.gs64 = owner64 ? GS_OWNER : C.gs64; C.gs32 = owner32 ? GS_OWNER : C.gs32; }
  C.gs32_multi = C.gs32 == GS_OWNER && dsm32 && want != "owner" ? GS_DSMEM : C.gs32;
}

// ----------------------------------------------------------------- workspace
void clear_graphs(amamg_ctx* h) {
  for (auto g : h->step_graphs)
    if (g) cudaGraphExecDestroy(g);
  h->step_graphs.clear();
  h->step_graph_kernels.clear();
  h->graph_R = 0;
}

int ensure_vcycle_ws(amamg_ctx* h, int R) {
  if (R <= h->Rcap) return AMAMG_OK;
  clear_graphs(h);
  for (auto& L : h->lv) {
    dfree(L.r64); dfree(L.e64); dfree(L.r32); dfree(L.e32);
  }
  for (size_t l = 1; l < h->lv.size(); ++l) {
    Level& L = h->lv[l];
    const size_t m = (size_t)R * 2 * L.n;
    CKS(dalloc(h, &L.r64, m)); CKS(dalloc(h, &L.e64, m));
    CKS(dalloc(h, &L.r32, m)); CKS(dalloc(h, &L.e32, m));
  }
  h->Rcap = R;
  return AMAMG_OK;
}

int ensure_solver_ws(amamg_ctx* h, int R) {
  const int m = h->prm.restart;
  if (R <= h->Rsolve && m <= h->mcap) return AMAMG_OK;
  clear_graphs(h);
  dfree(h->V); dfree(h->Z64); dfree(h->Z32); dfree(h->v32); dfree(h->w); dfree(h->res); dfree(h->wdf); dfree(h->df_part);
  dfree(h->partial); dfree(h->d_h); dfree(h->d_inv); dfree(h->d_flag); dfree(h->d_y); dfree(h->d_tickets); dfree(h->d_npart);
  dfree(h->d_diag64); dfree(h->d_inv64); dfree(h->d_inv32);
  dfree(h->ls_H); dfree(h->ls_Q); dfree(h->ls_R); dfree(h->ls_g); dfree(h->ls_bnorm); dfree(h->ls_st);
  dfree(h->d_lsout); dfree(h->d_lsinit);
  if (h->h_h) cudaFreeHost(h->h_h);
  if (h->h_lsout) cudaFreeHost(h->h_lsout);
  if (h->h_lsinit) cudaFreeHost(h->h_lsinit);
  h->h_h = nullptr;
  h->h_lsout = nullptr;
  h->h_lsinit = nullptr;
  const size_t len = 2 * (size_t)h->lv[0].n;
  CKS(dalloc(h, &h->V, (size_t)(m + 1) * R * len));
  if (h->prm.precision == AMAMG_SOLVE_MIXED) {
    CKS(dalloc(h, &h->Z32, (size_t)m * R * len));
    CKS(dalloc(h, &h->v32, (size_t)R * len));
  } else {
    CKS(dalloc(h, &h->Z64, (size_t)m * R * len));
  }
  CKS(dalloc(h, &h->w, (size_t)R * len));
  CKS(dalloc(h, &h->res, (size_t)R * len));
  if (h->prm.gs_arith == AMAMG_GS_DF64) {
    CKS(dalloc(h, &h->wdf, (size_t)R * len));
    CKS(dalloc(h, &h->df_part, (size_t)R * (2 * (m + 2) * df_partial_blocks((long)len) + df_norm_blocks((long)len))));
  }
  h->partial_elems = (size_t)R * (m + 2) * dot_blocks((long)len);
  CKS(dalloc(h, &h->partial, h->partial_elems));
  CKS(dalloc(h, &h->d_h, (size_t)R * 3 * (m + 2)));
  CKS(dalloc(h, &h->d_inv, (size_t)R));
  CKS(dalloc(h, &h->d_flag, (size_t)R));
  CKS(dalloc(h, &h->d_tickets, (size_t)R * (m + 3)));
  CK(cudaMemset(h->d_tickets, 0, sizeof(unsigned) * (size_t)R * (m + 3)));
  CKS(dalloc(h, &h->d_npart, (size_t)R * axpy_norm_blocks((long)len)));
  CKS(dalloc(h, &h->d_diag64, (size_t)R));
  CKS(dalloc(h, &h->d_inv64, (size_t)R));
  CKS(dalloc(h, &h->d_inv32, (size_t)R));
  CKS(dalloc(h, &h->d_y, (size_t)R * m));
  CKS(dalloc(h, &h->ls_H, (size_t)R * (m + 1) * m));
  CKS(dalloc(h, &h->ls_Q, (size_t)R * (m + 1) * (m + 1)));
  CKS(dalloc(h, &h->ls_R, (size_t)R * m * m));
  CKS(dalloc(h, &h->ls_g, (size_t)R * (m + 1)));
  CKS(dalloc(h, &h->ls_bnorm, (size_t)R));
  CKS(dalloc(h, &h->ls_st, (size_t)R * 4));
  CKS(dalloc(h, &h->d_lsout, (size_t)R));
  CKS(dalloc(h, &h->d_lsinit, (size_t)R));
  CK(cudaMallocHost((void**)&h->h_h, sizeof(double2) * (size_t)R * 3 * (m + 2)));
  CK(cudaMallocHost((void**)&h->h_lsout, sizeof(LsOut) * (size_t)R));
  CK(cudaMallocHost((void**)&h->h_lsinit, sizeof(LsInit) * (size_t)R));
  h->Rsolve = R;
  h->mcap = m;
  return AMAMG_OK;
}

// ----------------------------------------------------------------- level operations
// bytes below are the algorithmic traffic of each launch (each input read once,
// each output written once), used for the achieved-bandwidth figures.

template <typename T>
int op_dslash(amamg_ctx* h, const typename cplx<T>::type* in, typename cplx<T>::type* out,
              const typename cplx<T>::type* b, int R, cudaStream_t st);

template <>
int op_dslash<double>(amamg_ctx* h, const double2* in, double2* out, const double2* b, int R, cudaStream_t st) {
  const Level& L = h->lv[0];
  const double bytes = (double)L.n * (R * (32.0 + 32.0 + (b ? 32.0 : 0.0)) + 32.0);
  return launch(h, b ? "dslash_residual_f64" : "dslash_f64", bytes, st, [&] {
    return launch_dslash<double2, double2, double>(in, out, b, h->U64s, h->m0 + 2.0, L.Nt, L.Nx, R, st, h->cur_diag64);
  }, (double)L.n * R * (b ? 60.0 : 56.0));
}

template <>
int op_dslash<float>(amamg_ctx* h, const float2* in, float2* out, const float2* b, int R, cudaStream_t st) {
  const Level& L = h->lv[0];
  const double bytes = (double)L.n * (R * (16.0 + 16.0 + (b ? 16.0 : 0.0)) + 16.0);
  return launch(h, "dslash_f32", bytes, st, [&] {
    return launch_dslash<float2, float2, float>(in, out, b, h->U32, (float)(h->m0 + 2.0), L.Nt, L.Nx, R, st);
  }, (double)L.n * R * (b ? 60.0 : 56.0));
}

template <typename T>
int op_smooth(amamg_ctx* h, int l, typename cplx<T>::type* e, const typename cplx<T>::type* r, int R, int sweeps,
              cudaStream_t st);

template <typename T>
int smooth_impl(amamg_ctx* h, int l, typename cplx<T>::type* e, const typename cplx<T>::type* r, int R, int sweeps,
                cudaStream_t st) {
  const Level& L = h->lv[l];
  constexpr bool f64 = sizeof(T) == 8;
  const double cb = f64 ? 16.0 : 8.0;
  if (l == 0) {
    const T inv = (T)(1.0 / (h->m0 + 2.0));
    const typename cplx<T>::type* U;
    const T* inv_r;
    if constexpr (f64) { U = h->U64s; inv_r = h->cur_inv64; } else { U = h->U32; inv_r = h->cur_inv32; }
    // half sweep: read r, read + write e on half the sites, links once
    const double bytes = (double)L.n / 2 * (R * 2 * 3 * cb) + (double)L.n * 2 * cb / 2;
    for (int s = 0; s < sweeps; ++s)
      for (int c = 0; c < 2; ++c)
        CKS(launch(h, f64 ? "rb_smooth_f64" : "rb_smooth_f32", bytes, st, [&] {
          return launch_rb_half<T>(e, r, U, inv, L.Nt, L.Nx, c, R, st, inv_r);
        }, (double)L.n / 2 * R * 56.0));
    return AMAMG_OK;
  }
  const double blk = f64 ? 16.0 * 4 : (4.0 * 4 + 4.0);
  const int nc = L.ncol;
  const double bytes = (double)L.n / nc * ((L.off.K - 1) * blk + 4 * cb + R * 2 * 3 * cb);
  const double flops = (double)L.n / nc * R * ((L.off.K - 1) * 32.0 + 36.0);   // one colour
  const std::pair<int, int> choice = gs_choice<T>(L, R);
  const int kind = choice.first, variant = choice.second;
  if (sweeps > 0 && kind == GS_DSMEM) {
    // every colour of every sweep on one 16-block cluster, level in shared memory
    const bool bsm = dsmem_blocks_in_smem<T>(L.n, L.off.K);
    if constexpr (f64)
      return launch(h, "coarse_smooth_f64", bytes * nc * sweeps, st, [&] {
        return launch_coarse_sweeps_dsmem<double, double2>(e, r, L.Bc64, nullptr, L.Dc64, L.off, L.Nt, L.Nx, nc,
                                                           sweeps, R, bsm, st);
      }, flops * nc * sweeps);
    else
      return launch(h, "coarse_smooth_f32", bytes * nc * sweeps, st, [&] {
        return launch_coarse_sweeps_dsmem<float, __half2>(e, r, L.Bc16, L.Bcs, L.Dc32, L.off, L.Nt, L.Nx, nc, sweeps,
                                                          R, bsm, st);
      }, flops * nc * sweeps);
  }
  if (sweeps > 0 && kind == GS_OWNER) {
    // every colour of every sweep in one cooperative launch, neighbour waits only
    if constexpr (f64)
      return launch(h, "coarse_smooth_f64", bytes * nc * sweeps, st, [&] {
        return launch_coarse_sweeps_owner<double, double2>(e, r, L.Bc64, nullptr, L.Dc64, L.off, L.Nt, L.Nx, nc,
                                                          sweeps, R, h->d_owner_flags, h->d_sync, st, -1, variant);
      }, flops * nc * sweeps);
    else
      return launch(h, "coarse_smooth_f32", bytes * nc * sweeps, st, [&] {
        return launch_coarse_sweeps_owner<float, __half2>(e, r, L.Bc16, L.Bcs, L.Dc32, L.off, L.Nt, L.Nx, nc, sweeps,
                                                         R, h->d_owner_flags, h->d_sync, st, -1, variant);
      }, flops * nc * sweeps);
  }
  if (sweeps > 0 && kind == GS_GRID) {
    // every colour of every sweep in one cooperative launch over all SMs
    if constexpr (f64)
      return launch(h, "coarse_smooth_f64", bytes * nc * sweeps, st, [&] {
        return launch_coarse_sweeps_grid<double, double2>(e, r, L.Bc64, nullptr, L.Dc64, L.off, L.Nt, L.Nx, nc,
                                                          sweeps, R, h->d_sync, st);
      }, flops * nc * sweeps);
    else
      return launch(h, "coarse_smooth_f32", bytes * nc * sweeps, st, [&] {
        return launch_coarse_sweeps_grid<float, __half2>(e, r, L.Bc16, L.Bcs, L.Dc32, L.off, L.Nt, L.Nx, nc, sweeps,
                                                         R, h->d_sync, st);
      }, flops * nc * sweeps);
  }
  if constexpr (!f64) {
    if (sweeps > 0 && kind == GS_CLUSTER && use_cluster_sweeps<T>(L.n, nc))
      // every colour of every sweep in one clustered launch
      return launch(h, "coarse_smooth_f32", bytes * nc * sweeps, st, [&] {
        return launch_coarse_sweeps_cluster<float, __half2>(e, r, L.Bc16, L.Bcs, L.Dc32, L.off, L.Nt, L.Nx, nc,
                                                            sweeps, R, st);
      }, flops * nc * sweeps);
  }
  for (int s = 0; s < sweeps; ++s)
    for (int c = 0; c < nc; ++c) {
      int rc;
      if constexpr (f64)
        rc = launch(h, "coarse_smooth_f64", bytes, st, [&] {
          return launch_coarse_colour<double, double2>(e, r, L.Bc64, nullptr, L.Dc64, L.off, L.Nt, L.Nx, nc, c, R,
                                                       st);
        }, flops);
      else
        rc = launch(h, "coarse_smooth_f32", bytes, st, [&] {
          return launch_coarse_colour<float, __half2>(e, r, L.Bc16, L.Bcs, L.Dc32, L.off, L.Nt, L.Nx, nc, c, R, st);
        }, flops);
      CKS(rc);
    }
  return AMAMG_OK;
}

template <typename T>
int op_prolong(amamg_ctx* h, int l, const typename cplx<T>::type* ec, typename cplx<T>::type* ef, int R,
               cudaStream_t st) {
  const Level& L = h->lv[l];
  constexpr bool f64 = sizeof(T) == 8;
  const double cb = f64 ? 16.0 : 8.0;
  const double pbytes = (double)L.nT * 8 * L.nrows * (f64 ? 16.0 : 4.0) + (f64 ? 0.0 : 4.0 * L.nT);
  const double bytes = pbytes + (double)R * 2 * (L.n + h->lv[l + 1].n) * cb;
  if constexpr (f64)
    return launch(h, "prolong_f64", bytes, st, [&] {
      return launch_prolong<double, double2>(ec, ef, L.P64, nullptr, L.Nx, L.a, L.Np, L.Nq, R, st,
                                             h->prm.edge_owner);
    }, (double)L.nT * L.nrows * 64.0 * R);
  else
    return launch(h, "prolong_f32", bytes, st, [&] {
      return launch_prolong<float, __half2>(ec, ef, L.P16, L.Ps, L.Nx, L.a, L.Np, L.Nq, R, st, h->prm.edge_owner);
    }, (double)L.nT * L.nrows * 64.0 * R);
}

// The fine-level end of a V-cycle (prolongation from level 1, then the
// post-smoothing red-black sweeps) as one launch when a resident shape exists.
template <typename T>
bool fine_post_possible(const amamg_ctx* h, int R) {
  if (!h->fine_fused || h->prm.edge_owner != AMAMG_OWNER_TILE) return false;   // the fused kernel reads tile corners
  const Level& L = h->lv[0];
  if constexpr (sizeof(T) == 8) return fine_post_rows<double, double2>(L.Nt, L.Nx, L.a, R) > 0;
  else return fine_post_rows<float, __half2>(L.Nt, L.Nx, L.a, R) > 0;
}

template <typename T>
int op_fine_post(amamg_ctx* h, const typename cplx<T>::type* ec, typename cplx<T>::type* e,
                 const typename cplx<T>::type* r, int R, cudaStream_t st) {
  const Level& L = h->lv[0];
  constexpr bool f64 = sizeof(T) == 8;
  const double cb = f64 ? 16.0 : 8.0;
  const int sweeps = h->prm.post_smooth;
  const double pbytes = (double)L.nT * 8 * L.nrows * (f64 ? 16.0 : 4.0) + (f64 ? 0.0 : 4.0 * L.nT);
  const double bytes = pbytes + (double)R * 2 * (L.n + h->lv[1].n) * cb +
                       2.0 * sweeps * ((double)L.n / 2 * (R * 2 * 3 * cb) + (double)L.n * 2 * cb / 2);
  const double flops = (double)L.nT * L.nrows * 64.0 * R + 2.0 * sweeps * (double)L.n / 2 * R * 56.0;
  const T inv = (T)(1.0 / (h->m0 + 2.0));
  if constexpr (f64)
    return launch(h, "fine_post_f64", bytes, st, [&] {
      return launch_fine_post<double, double2>(ec, e, r, L.P64, nullptr, h->U64s, inv, h->cur_inv64, L.Nt, L.Nx,
                                               L.a, sweeps, R, h->d_owner_flags, h->d_sync, st);
    }, flops);
  else
    return launch(h, "fine_post_f32", bytes, st, [&] {
      return launch_fine_post<float, __half2>(ec, e, r, L.P16, L.Ps, h->U32, inv, h->cur_inv32, L.Nt, L.Nx, L.a,
                                              sweeps, R, h->d_owner_flags, h->d_sync, st);
    }, flops);
}

template <typename T>
int op_restrict(amamg_ctx* h, int l, const typename cplx<T>::type* ef, typename cplx<T>::type* ec, int R,
                cudaStream_t st) {
  const Level& L = h->lv[l];
  constexpr bool f64 = sizeof(T) == 8;
  const double cb = f64 ? 16.0 : 8.0;
  const double pbytes = (double)L.nT * 8 * L.nrows * (f64 ? 16.0 : 4.0) + (f64 ? 0.0 : 4.0 * L.nT);
  const double bytes = pbytes + (double)R * 2 * (L.n + h->lv[l + 1].n) * cb;
  if constexpr (f64)
    return launch(h, "restrict_f64", bytes, st, [&] {
      return launch_restrict<double, double2>(ef, ec, L.P64, nullptr, L.Nx, L.a, L.Np, L.Nq, R, st,
                                              h->prm.edge_owner);
    }, (double)L.nT * L.nrows * 64.0 * R);
  else
    return launch(h, "restrict_f32", bytes, st, [&] {
      return launch_restrict<float, __half2>(ef, ec, L.P16, L.Ps, L.Nx, L.a, L.Np, L.Nq, R, st, h->prm.edge_owner);
    }, (double)L.nT * L.nrows * 64.0 * R);
}

// Right-hand-side count from which the FP32 coarse apply runs on the tensor
// cores (64 right-hand sides fill the MMA's 128 rows with both planes).
constexpr int COARSE_TC_MIN_R = 32;

// The tensor-core coarse apply of level l for R right-hand sides: builds the
// level's FP16 super-block images at the first use and grows the staging
// buffers.  Returns false (the CUDA-core kernel runs) where the level's shape
// or the device does not allow it, or AMAMG_COARSE_TC=0.
bool ensure_coarse_tc(amamg_ctx* h, int l, int R, cudaStream_t st, int* rc) {
  Level& L = h->lv[l];
  *rc = AMAMG_OK;
  if (L.ct_state == 0) {
    const char* env = std::getenv("AMAMG_COARSE_TC");
    L.ct_state = -1;
    if (!(env && std::strcmp(env, "0") == 0) && coarse_tc_possible(L.Nt, L.Nx, L.off) &&
        coarse_tc_init() == cudaSuccess) {
      *rc = dalloc(h, &L.ctW, coarse_tc_image_halves(L.Nt, L.Nx));
      if (*rc == AMAMG_OK) *rc = dalloc(h, &L.ctWs, coarse_tc_scale_floats(L.Nt, L.Nx));
      if (*rc == AMAMG_OK)
        *rc = launch(h, "coarse_tc_images", 0.0, st, [&] {
          return launch_coarse_tc_pack_w(L.B64, L.off, L.Nt, L.Nx, L.ctW, L.ctWs, st);
        });
      if (*rc != AMAMG_OK) {
        dfree(L.ctW);
        dfree(L.ctWs);
        return false;
      }
      L.ct_state = 1;
    }
    cudaGetLastError();
  }
  if (L.ct_state != 1) return false;
  const size_t need = coarse_tc_stage_halves(L.Nt, L.Nx, R);
  if (need > h->ct_stage_cap) {
    dfree(h->ct_stage);
    h->ct_stage_cap = 0;
    if ((*rc = dalloc(h, &h->ct_stage, need)) != AMAMG_OK) return false;
    h->ct_stage_cap = need;
  }
  if (R > h->ct_amax_cap) {
    dfree(h->ct_amax);
    h->ct_amax_cap = 0;
    if ((*rc = dalloc(h, &h->ct_amax, (size_t)R)) != AMAMG_OK) return false;
    h->ct_amax_cap = R;
  }
  return true;
}

template <typename T>
int op_coarse(amamg_ctx* h, int l, const typename cplx<T>::type* in, typename cplx<T>::type* out,
              const typename cplx<T>::type* b, int R, cudaStream_t st) {
  const Level& L = h->lv[l];
  constexpr bool f64 = sizeof(T) == 8;
  const double cb = f64 ? 16.0 : 8.0;
  const double blk = f64 ? 16.0 * 4 : (4.0 * 4 + 4.0);
  const double bytes = (double)L.n * (L.off.K * blk + R * 2 * (b ? 3 : 2) * cb);
  if constexpr (!f64) {
    if (!b && R >= COARSE_TC_MIN_R) {
      int rc = AMAMG_OK;
      if (ensure_coarse_tc(h, l, R, st, &rc))
        return launch(h, "coarse_apply_tc", bytes, st, [&] {
          return launch_coarse_tc(in, out, L.ctW, L.ctWs, L.Nt, L.Nx, R, h->ct_stage, h->ct_amax,
                                  reinterpret_cast<int*>(h->d_sync + 2), st);
        }, (double)L.n * R * L.off.K * 32.0);
      if (rc != AMAMG_OK) return rc;
    }
  }
  if constexpr (f64)
    return launch(h, "coarse_apply_f64", bytes, st, [&] {
      return launch_coarse_apply<double, double2>(in, out, b, L.B64, nullptr, L.off, L.Nt, L.Nx, R, st);
    }, (double)L.n * R * L.off.K * 32.0);
  else
    return launch(h, "coarse_apply_f32", bytes, st, [&] {
      return launch_coarse_apply<float, __half2>(in, out, b, L.B16, L.Bs, L.off, L.Nt, L.Nx, R, st);
    }, (double)L.n * R * L.off.K * 32.0);
}

// The paper's coarsest solver (Sec. 5): GMRES(GMRES_RESTART) to relative
// residual GMRES_TOL from a zero start, at most GMRES_MAX_R right-hand sides per
// launch.  Bytes and FLOPs are not counted (the iteration count is data dependent).
constexpr int GMRES_RESTART = 30;
constexpr double GMRES_TOL = 0.1;
constexpr int GMRES_MAX_CYCLES = 200;

template <typename T>
int op_coarsest_gmres(amamg_ctx* h, const typename cplx<T>::type* r, typename cplx<T>::type* e, int R,
                      cudaStream_t st) {
  using C = typename cplx<T>::type;
  const Level& L = h->lv.back();
  const size_t len = 2 * (size_t)L.n;
  for (int r0 = 0; r0 < R; r0 += GMRES_MAX_R) {
    const int Rc = std::min(GMRES_MAX_R, R - r0);
    const C* rr = r + r0 * len;
    C* ee = e + r0 * len;
    C* V = reinterpret_cast<C*>(h->gm_V);
    if constexpr (sizeof(T) == 8)
      CKS(launch(h, "coarsest_gmres_f64", 0.0, st, [&] {
        return launch_coarsest_gmres<double, double2>(rr, ee, L.B64, nullptr, L.off, L.Nt, L.Nx, Rc, GMRES_RESTART,
                                                      GMRES_TOL, GMRES_MAX_CYCLES, V, h->gm_part, h->gm_st,
                                                      h->d_sync, h->gm_done, h->gm_blocks64, st);
      }));
    else
      CKS(launch(h, "coarsest_gmres_f32", 0.0, st, [&] {
        return launch_coarsest_gmres<float, __half2>(rr, ee, L.B16, L.Bs, L.off, L.Nt, L.Nx, Rc, GMRES_RESTART,
                                                     GMRES_TOL, GMRES_MAX_CYCLES, V, h->gm_part, h->gm_st,
                                                     h->d_sync, h->gm_done, h->gm_blocks32, st);
      }));
  }
  return AMAMG_OK;
}

template <typename Cv>
int op_coarsest(amamg_ctx* h, const Cv* r, Cv* e, int R, cudaStream_t st) {
  const double bytes = (double)h->nd * h->nd * 16.0 + (double)R * 2 * h->nd * sizeof(Cv);
  return launch(h, "coarsest_gemv_f64", bytes, st,
                [&] { return launch_dense_gemv<Cv>(h->Ainv, r, e, h->nd, R, st); },
                (double)h->nd * h->nd * 8.0 * R);
}

// coarsest level inside a V-cycle: FP64 inverse for FP64 vectors, its FP32
// rounding for the FP32 (mixed-precision) V-cycle; or GMRES in the vectors'
// precision (FP16 + scale blocks for FP32)
int vcycle_coarsest(amamg_ctx* h, const double2* r, double2* e, int R, cudaStream_t st) {
  if (h->prm.coarsest == AMAMG_COARSEST_GMRES) return op_coarsest_gmres<double>(h, r, e, R, st);
  return op_coarsest<double2>(h, r, e, R, st);
}
int vcycle_coarsest(amamg_ctx* h, const float2* r, float2* e, int R, cudaStream_t st) {
  if (h->prm.coarsest == AMAMG_COARSEST_GMRES) return op_coarsest_gmres<float>(h, r, e, R, st);
  const double bytes = (double)h->nd * h->nd * 8.0 + (double)R * 2 * h->nd * 8.0;
  if (h->tc_ok && coarsest_tc_possible(h->nd, R))
    // many right-hand sides: a dense contraction, on the tensor cores (TF32 in, FP32 accumulate)
    return launch(h, "coarsest_mma_tf32", bytes, st, [&] {
      return launch_coarsest_tc(h->Ainv32, r, e, h->nd, R, h->tc_bop, reinterpret_cast<int*>(h->d_sync + 2), st);
    }, (double)h->nd * h->nd * 8.0 * R);
  return launch(h, "coarsest_gemv_f32", bytes, st,
                [&] { return launch_dense_gemv32(h->Ainv32, r, e, h->nd, R, st); },
                (double)h->nd * h->nd * 8.0 * R);
}

// V-cycle of Algorithm 1 (start vector 0, no pre-smoothing) from level l:
// e = P M_{l+1}(P^H r), then post-smoothing sweeps on A_l e = r.  The coarse
// levels' r and e come from w (the handle's own vectors, or caller scratch).
template <typename T>
int vcycle_from(amamg_ctx* h, int l, const typename cplx<T>::type* r, typename cplx<T>::type* e,
                const VcycleVecs<T>& w, int R, cudaStream_t st) {
  const int Lc = (int)h->lv.size() - 1;
  if (l == Lc) return vcycle_coarsest(h, r, e, R, st);
  typename cplx<T>::type* rc = w.r[l + 1];
  typename cplx<T>::type* ec = w.e[l + 1];
  CKS(op_restrict<T>(h, l, r, rc, R, st));
  CKS(vcycle_from<T>(h, l + 1, rc, ec, w, R, st));
  if (l == 0 && h->prm.post_smooth > 0 && fine_post_possible<T>(h, R))
    return op_fine_post<T>(h, ec, e, r, R, st);
  CKS(op_prolong<T>(h, l, ec, e, R, st));
  return smooth_impl<T>(h, l, e, r, R, h->prm.post_smooth, st);
}

// the handle's own coarse work vectors (ensure_vcycle_ws sizes them)
template <typename T>
VcycleVecs<T> handle_vecs(const amamg_ctx* h) {
  VcycleVecs<T> w;
  for (size_t l = 1; l < h->lv.size(); ++l) {
    if constexpr (sizeof(T) == 8) { w.r[l] = h->lv[l].r64; w.e[l] = h->lv[l].e64; }
    else { w.r[l] = h->lv[l].r32; w.e[l] = h->lv[l].e32; }
  }
  return w;
}

// ----------------------------------------------------------------- FGMRES
int norms(amamg_ctx* h, const double2* X, size_t xr, long len, int R, double2* out, int ldo, int off, double* inv,
          cudaStream_t st) {
  const int nb = dot_blocks(len);
  CKS(launch(h, "gs_dots", (double)R * len * 16.0, st,
             [&] { return launch_dots(X, 0, xr, X, xr, len, 1, R, h->partial, st); }));
  return launch(h, "gs_reduce", (double)R * nb * 16.0, st,
                [&] { return launch_reduce(h->partial, nb, 1, R, out, ldo, off, 1, inv, st); });
}

// The least-squares update of Arnoldi step j on the device (the rotation of
// the new Hessenberg column, g, the residual estimate and the stopping test per
// right-hand side, in FP64) and the copy of the per-RHS progress to pinned
// host memory, on the side stream ws2 once the step's norms are in d_h, so
// that it overlaps the normalisation of v_{j+1}; ls_join makes st wait for it.
int ls_fork(amamg_ctx* h, int j, int R, cudaStream_t st) {
  const int m = h->prm.restart;
  CK(cudaEventRecord(h->ev_fork, st));
  CK(cudaStreamWaitEvent(h->ws2, h->ev_fork, 0));
  CKS(launch(h, "ls_update", (double)R * (2.0 * (j + 2) * 16.0 * 3 + 64.0), h->ws2, [&] {
    return launch_ls_step(h->ls(), h->d_h, 3 * (m + 2), 2 * (m + 2), j, R, m, h->prm.tol, h->prm.max_iter, h->d_lsout,
                          h->ws2);
  }));
  CK(cudaMemcpyAsync(h->h_lsout, h->d_lsout, sizeof(LsOut) * R, cudaMemcpyDeviceToHost, h->ws2));
  CK(cudaEventRecord(h->ev_join, h->ws2));
  return AMAMG_OK;
}
int ls_join(amamg_ctx* h, cudaStream_t st) {
  CK(cudaStreamWaitEvent(st, h->ev_join, 0));
  return AMAMG_OK;
}

// One Arnoldi step j for all R right-hand sides, entirely on the device:
// z_j = M(v_j), w = D z_j, two classical Gram-Schmidt passes against v_0..v_j,
// ||w||, v_{j+1} = w / ||w||, and the copy of the new Hessenberg column and norm
// to pinned host memory.  Capturable as one CUDA graph.
int arnoldi_step(amamg_ctx* h, int j, int R, cudaStream_t st) {
  const int m = h->prm.restart;
  const long len = 2L * h->lv[0].n;
  const size_t vr = (size_t)len, vi = (size_t)R * len;
  const int ldh = 3 * (m + 2);
  double2* d_h1 = h->d_h;
  const double2* vj = h->V + (size_t)j * vi;
  const bool mixed = h->prm.precision == AMAMG_SOLVE_MIXED;
  if (mixed) {
    float2* zj = h->Z32 + (size_t)j * vi;
    // v_j in FP32: cast here for j = 0; for j >= 1 the previous step's
    // normalisation wrote it
    if (j == 0 && h->prm.gs_arith != AMAMG_GS_DF64)   // (double-float: the cycle start wrote it)
      CKS(launch(h, "cast_f64_f32", (double)R * len * 24.0, st,
                 [&] { return launch_cast<double2, float2>(vj, h->v32, (long)R * len, st); }));
    CKS(vcycle_from<float>(h, 0, h->v32, zj, handle_vecs<float>(h), R, st));
    const Level& L = h->lv[0];
    CKS(launch(h, "dslash_mixed", (double)L.n * (R * (16.0 + 32.0) + 32.0), st, [&] {
      return launch_dslash<float2, double2, double>(zj, h->w, nullptr, h->U64s, h->m0 + 2.0, L.Nt, L.Nx, R, st,
                                                    h->cur_diag64);
    }));
  } else {
    double2* zj = h->Z64 + (size_t)j * vi;
    CKS(vcycle_from<double>(h, 0, vj, zj, handle_vecs<double>(h), R, st));
    CKS(op_dslash<double>(h, zj, h->w, nullptr, R, st));
  }
  // Classical Gram-Schmidt with the DGKS criterion: one pass, and a second
  // pass only for right-hand sides whose norm dropped below 1/sqrt(2) of its
  // value before orthogonalisation (the second-pass kernels are gated per RHS).
  // Each pass is two kernels with their reductions fused in: the inner
  // products (pass 1 also ||w||^2), then the update with the new norm.
  const int J = j + 1;
  const int nrm_off = 2 * (m + 2);
  unsigned* tk_dots = h->d_tickets;
  unsigned* tk_norm = h->d_tickets + (size_t)R * (m + 2);
  if (h->prm.gs_arith == AMAMG_GS_DF64) {
    // the same four Gram-Schmidt steps in double-float arithmetic on the
    // double-float basis, then v_{j+1} = w / ||w|| and its FP32 rounding
    const double dfb = (double)R * len * 16.0;
    CKS(launch(h, "to_df", (double)R * len * 32.0, st, [&] { return launch_to_df(h->w, h->wdf, (long)R * len, st); }));
    double* dpart = h->df_part;
    double* npart = h->df_part + (size_t)R * 2 * (m + 2) * df_partial_blocks(len);
    CKS(launch(h, "gs_dots_df", dfb * (J + 1), st, [&] {
      return launch_dots_df(h->V, vi, vr, h->wdf, vr, len, J, R, true, nullptr, dpart, 2 * (m + 2), tk_dots, d_h1,
                            ldh, 0, st);
    }, (double)R * len * 8.0 * (J + 1)));
    CKS(launch(h, "gs_update_norm_df", dfb * (J + 2), st, [&] {
      return launch_axpy_norm_df(h->wdf, vr, h->V, vi, vr, d_h1, ldh, J, len, R, nullptr, npart, tk_norm, d_h1, ldh,
                                 nrm_off, h->d_inv, h->d_flag, J, 0.5, 2, st);
    }, (double)R * len * 8.0 * (J + 1)));
    CKS(launch(h, "gs2_dots_gated_df", dfb * (J + 1), st, [&] {
      return launch_dots_df(h->V, vi, vr, h->wdf, vr, len, J, R, false, h->d_flag, dpart, 2 * (m + 2), tk_dots, d_h1,
                            ldh, m + 2, st);
    }, (double)R * len * 8.0 * J));
    CKS(launch(h, "gs2_update_norm_gated_df", dfb * (J + 2), st, [&] {
      return launch_axpy_norm_df(h->wdf, vr, h->V, vi, vr, d_h1 + (m + 2), ldh, J, len, R, h->d_flag, npart, tk_norm,
                                 d_h1, ldh, nrm_off, h->d_inv, nullptr, 0, 0.0, 1, st);
    }, (double)R * len * 8.0 * (J + 1)));
    CKS(ls_fork(h, j, R, st));
    CKS(launch(h, "scale_copy", (double)R * len * 40.0, st, [&] {
      return launch_scale_copy_df(h->V + (size_t)(j + 1) * vi, h->v32, vr, h->wdf, nullptr, vr, h->d_inv, len, R, st);
    }));
    return ls_join(h, st);
  }
  if (h->prm.gs_method == AMAMG_GS_MGS) {
    // modified Gram-Schmidt: stage i subtracts the projection on v_{i-1} and
    // forms the inner product with v_i (the last stage the norm); J + 1 stages
    for (int i = 0; i <= J; ++i) {
      const double nvec = i == 0 ? 2.0 : (i < J ? 4.0 : 3.0);      // w, v_{i-1}, v_i read; w written
      const double fl = (i >= 1 ? 8.0 : 0.0) + (i < J ? 8.0 : 4.0);
      CKS(launch(h, i < J ? "mgs_stage" : "mgs_norm", (double)R * len * 16.0 * nvec, st, [&] {
        return launch_mgs_stage(h->w, vr, h->V, vi, vr, len, i, J, R, h->partial, m + 2, tk_dots, d_h1, ldh, m + 2,
                                nrm_off, h->d_inv, st);
      }, (double)R * len * fl));
    }
  } else {
  CKS(launch(h, "gs_dots", (double)R * len * 16.0 * (J + 1), st, [&] {
    return launch_dots_fused(h->V, vi, vr, h->w, vr, len, J, R, h->partial, true, nullptr, tk_dots, d_h1, ldh, 0, st);
  }, (double)R * len * 8.0 * (J + 1)));
  CKS(launch(h, "gs_update_norm", (double)R * len * 16.0 * (J + 2), st, [&] {
    return launch_axpy_norm(h->w, vr, h->V, vi, vr, d_h1, ldh, J, len, R, nullptr, h->d_npart, tk_norm, d_h1, ldh,
                            nrm_off, h->d_inv, h->d_flag, J, 0.5, 2, st);
  }, (double)R * len * 8.0 * (J + 1)));
  // second pass, gated by the DGKS flag (h2 = 0 where it is not needed); the
  // byte counts of these categories assume the pass runs (upper bounds)
  CKS(launch(h, "gs2_dots_gated", (double)R * len * 16.0 * (J + 1), st, [&] {
    return launch_dots_fused(h->V, vi, vr, h->w, vr, len, J, R, h->partial, false, h->d_flag, tk_dots, d_h1, ldh,
                             m + 2, st);
  }, (double)R * len * 8.0 * J));
  CKS(launch(h, "gs2_update_norm_gated", (double)R * len * 16.0 * (J + 2), st, [&] {
    return launch_axpy_norm(h->w, vr, h->V, vi, vr, d_h1 + (m + 2), ldh, J, len, R, h->d_flag, h->d_npart, tk_norm,
                            d_h1, ldh, nrm_off, h->d_inv, nullptr, 0, 0.0, 1, st);
  }, (double)R * len * 8.0 * (J + 1)));
  }
  CKS(ls_fork(h, j, R, st));
  if (mixed)
    CKS(launch(h, "scale_copy", (double)R * len * 40.0, st, [&] {
      return launch_scale_copy_dual(h->V + (size_t)(j + 1) * vi, h->v32, vr, h->w, vr, h->d_inv, len, R, st);
    }));
  else
    CKS(launch(h, "scale_copy", (double)R * len * 32.0, st, [&] {
      return launch_scale_copy<double2>(h->V + (size_t)(j + 1) * vi, vr, h->w, vr, h->d_inv, len, R, st);
    }));
  return ls_join(h, st);
}

// Runs Arnoldi step j: replays its captured graph (capturing it on first use),
// or launches eagerly when kernel profiling is on.
int run_step(amamg_ctx* h, int j, int R, cudaStream_t st) {
  if (h->prof || !h->use_graphs) return arnoldi_step(h, j, R, st);
  if (h->graph_R != R) {
    clear_graphs(h);
    h->graph_R = R;
  }
  if ((int)h->step_graphs.size() <= j) {
    h->step_graphs.resize(j + 1, nullptr);
    h->step_graph_kernels.resize(j + 1, 0);
  }
  if (!h->step_graphs[j]) {
    const long long l0 = h->launches;
    CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    const int rc = arnoldi_step(h, j, R, st);
    cudaGraph_t g = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(st, &g);
    if (rc != AMAMG_OK || ec != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      if (h->err.empty()) h->err = std::string("graph capture: ") + cudaGetErrorString(ec);
      return rc != AMAMG_OK ? rc : AMAMG_ERR_CUDA;
    }
    cudaGraphExec_t ex = nullptr;
    const cudaError_t ei = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    if (ei != cudaSuccess) {
      h->err = std::string("cudaGraphInstantiate: ") + cudaGetErrorString(ei);
      return AMAMG_ERR_CUDA;
    }
    h->step_graphs[j] = ex;
    h->step_graph_kernels[j] = h->launches - l0;
    h->launches = l0;
  }
  CK(cudaGraphLaunch(h->step_graphs[j], st));
  h->launches += h->step_graph_kernels[j];
  return AMAMG_OK;
}

// One restart cycle of the FP64 flexible GMRES for R right-hand sides b_r with
// iterates x_r (both [R][len] on the device), using the per-RHS host state st_.
// Recomputes the true residual r = b - D x, marks converged right-hand sides,
// runs Arnoldi steps (one captured graph each) until every still-active
// right-hand side meets its residual estimate or m steps are done, and adds
// Z y to x.  Returns AMAMG_OK; *any_left tells whether some right-hand side is
// still unconverged and within its iteration budget.
int fgmres_cycle(amamg_ctx* h, const double2* b, double2* x, int R, cudaStream_t st, std::vector<SlotState>& sl,
                 bool* any_left) {
  const int m = h->prm.restart;
  const long len = 2L * h->lv[0].n;
  const size_t vr = (size_t)len, vi = (size_t)R * len;
  const bool mixed = h->prm.precision == AMAMG_SOLVE_MIXED;
  const int ldh = 3 * (m + 2);
  const int nrm_off = 2 * (m + 2);
  double2* d_h1 = h->d_h;
  const double tol = h->prm.tol;
  OuterState& o = h->outer;
  o.resize(R, m);
  // true residual and the norms of r and b
  CKS(op_dslash<double>(h, x, h->res, b, R, st));
  CKS(norms(h, h->res, vr, len, R, d_h1, ldh, nrm_off, h->d_inv, st));
  CKS(norms(h, b, vr, len, R, d_h1, ldh, nrm_off + 1, nullptr, st));
  CK(cudaMemcpyAsync(h->h_h, h->d_h, sizeof(double2) * R * ldh, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  bool left = false;
  for (int r = 0; r < R; ++r) {
    SlotState& q = sl[r];
    o.k[r] = 0;
    o.building[r] = 0;
    if (!q.active || q.done) continue;
    if (q.fresh) {
      q.bnorm = h->h_h[(size_t)r * ldh + nrm_off + 1].x;
      q.fresh = 0;
      if (!std::isfinite(q.bnorm)) { q.status = AMAMG_ERR_NONFINITE; q.done = 1; continue; }
    }
    const double beta = h->h_h[(size_t)r * ldh + nrm_off].x;
    if (!std::isfinite(beta)) { q.status = AMAMG_ERR_NONFINITE; q.done = 1; continue; }
    q.relres = q.bnorm > 0 ? beta / q.bnorm : 0.0;
    if (q.relres <= tol) { q.done = 1; q.status = AMAMG_OK; continue; }
    if (q.iters >= h->prm.max_iter) { q.done = 1; q.status = AMAMG_NOT_CONVERGED; continue; }
    o.building[r] = 1;
    left = true;
  }
  *any_left = left;
  if (!left) return AMAMG_OK;
  // the device least-squares state: g = beta e_1, Q^H = I, progress counters
  for (int r = 0; r < R; ++r) {
    const SlotState& q = sl[r];
    h->h_lsinit[r] = LsInit{o.building[r] ? h->h_h[(size_t)r * ldh + nrm_off].x : 0.0, q.bnorm, o.building[r],
                            q.iters};
  }
  CK(cudaMemcpyAsync(h->d_lsinit, h->h_lsinit, sizeof(LsInit) * R, cudaMemcpyHostToDevice, st));
  CKS(launch(h, "ls_update", (double)R * (m + 1) * (m + 2) * 16.0, st,
             [&] { return launch_ls_init(h->ls(), h->d_lsinit, R, m, st); }));
  // V[0] = r / beta (zero for right-hand sides that are not building: their inv is
  // set by the norm of a zero or converged residual and they are ignored below)
  if (h->prm.gs_arith == AMAMG_GS_DF64)
    CKS(launch(h, "scale_copy", (double)R * len * 40.0, st, [&] {
      return launch_scale_copy_df(h->V, h->v32, vr, nullptr, h->res, vr, h->d_inv, len, R, st);
    }));
  else
    CKS(launch(h, "scale_copy", (double)R * len * 32.0, st, [&] {
      return launch_scale_copy<double2>(h->V, vr, h->res, vr, h->d_inv, len, R, st);
    }));
  int j = 0;
  for (; j < m; ++j) {
    CKS(run_step(h, j, R, st));
    CK(cudaStreamSynchronize(st));
    bool any = false;
    for (int r = 0; r < R; ++r) {
      if (!o.building[r]) continue;
      SlotState& q = sl[r];
      const LsOut& u = h->h_lsout[r];
      q.iters = u.iters;
      o.k[r] = u.k;
      if (u.nonfinite) { q.status = AMAMG_ERR_NONFINITE; q.done = 1; o.building[r] = 0; o.k[r] = 0; continue; }
      o.building[r] = u.building;
      if (o.building[r]) any = true;
    }
    if (!any) { ++j; break; }
  }
  // x += Z y  (per right-hand side k[r] columns; the rest zero), y from the
  // triangular factor and solve on the device
  const int jmax = j < m ? j : m;
  CKS(launch(h, "ls_update", (double)R * m * (m + 1) * 16.0 * 2, st,
             [&] { return launch_ls_solve(h->ls(), h->d_y, R, m, st); }));
  if (mixed)
    CKS(launch(h, "x_update", (double)R * len * (8.0 * jmax + 32.0), st, [&] {
      return launch_multi_axpy<float2>(x, vr, h->Z32, vi, vr, h->d_y, m, jmax, 1.0, len, R, st);
    }));
  else
    CKS(launch(h, "x_update", (double)R * len * (16.0 * jmax + 32.0), st, [&] {
      return launch_multi_axpy<double2>(x, vr, h->Z64, vi, vr, h->d_y, m, jmax, 1.0, len, R, st);
    }));
  return AMAMG_OK;
}

// Per-RHS masses of the fine operator for the next cycles: diag = m0_r + 2 and
// its inverse in FP64 and FP32, copied to the solver's device arrays.
int set_masses(amamg_ctx* h, const double* m0, int R, cudaStream_t st) {
  std::vector<double> d(R), i64(R);
  std::vector<float> i32(R);
  for (int r = 0; r < R; ++r) {
    d[r] = m0[r] + 2.0;
    i64[r] = 1.0 / d[r];
    i32[r] = (float)i64[r];
  }
  CK(cudaMemcpyAsync(h->d_diag64, d.data(), sizeof(double) * R, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(h->d_inv64, i64.data(), sizeof(double) * R, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(h->d_inv32, i32.data(), sizeof(float) * R, cudaMemcpyHostToDevice, st));
  CK(cudaStreamSynchronize(st));   // the host vectors go out of scope
  return AMAMG_OK;
}

// A grid or owner Gauss-Seidel sweep whose wait timed out left its flag set:
// report it and re-arm the counters (cooperative launches keep all blocks resident, so
// this does not happen in a correct run).
int check_grid_sync(amamg_ctx* h, cudaStream_t st) {
  unsigned flag[3] = {0, 0, 0};
  CK(cudaMemcpyAsync(flag, h->d_sync, sizeof(flag), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (!flag[2]) return AMAMG_OK;
  CK(cudaMemsetAsync(h->d_sync, 0, 8 * sizeof(unsigned), st));
  CK(cudaMemsetAsync(h->d_owner_flags, 0, OWNER_MAX_BLOCKS * sizeof(unsigned), st));
  h->err = "coarse Gauss-Seidel synchronisation timed out";
  return AMAMG_ERR_TIMEOUT;
}

// ----------------------------------------------------------------- autotuner
// With amamg_params.autotune, the first V-cycle of each right-hand-side count R
// (outside graph capture) times the coarse Gauss-Seidel candidates of every
// smoothed coarse level in the precision the V-cycle runs in -- the owner sweep
// in its shape variants (early-sum lanes 8 or 16, the fewest or twice the
// fewest sites per block), the grid sweep and the distributed-shared-memory
// cluster sweep, where each fits -- with CUDA events on the level's own work
// vectors (2 warm-up and 5 timed launches each), and keeps the fastest for
// that R.  The candidates compute the same sweeps; they differ only in the
// rounding order of the owner sweep's split sums.
template <typename T>
int tune_level(amamg_ctx* h, int l, int R, cudaStream_t st) {
  Level& L = h->lv[l];
  constexpr bool f64 = sizeof(T) == 8;
  using BT = typename std::conditional<f64, double2, __half2>::type;
  auto& tm = f64 ? L.tune64 : L.tune32;
  if (tm.count(R)) return AMAMG_OK;
  std::vector<std::pair<int, int>> cand;
  std::vector<OwnerConfig> seen;
  for (const int v : {0, 1, 2, 4, 5, 6}) {
    OwnerConfig oc;
    if (!owner_sweep_config<T, BT>(L.Nt, L.Nx, L.off.K, L.ncol, L.off, R, &oc, v)) continue;
    bool dup = false;
    for (const auto& o : seen) dup |= o.cnt == oc.cnt && o.early_lanes == oc.early_lanes && o.slots == oc.slots;
    if (dup) continue;
    seen.push_back(oc);
    cand.push_back({GS_OWNER, v});
  }
  if (grid_sweep_blocks<T, BT>(L.n, L.ncol, R) > 0) cand.push_back({GS_GRID, 0});
  if (dsmem_sweeps_possible<T, BT>(L.n, L.off.K, L.ncol, dsmem_blocks_in_smem<T>(L.n, L.off.K)))
    cand.push_back({GS_DSMEM, 0});
  if (cand.size() < 2) return AMAMG_OK;                      // nothing to choose: the fixed rule stands
  typename cplx<T>::type* e = f64 ? (typename cplx<T>::type*)L.e64 : (typename cplx<T>::type*)L.e32;
  typename cplx<T>::type* r = f64 ? (typename cplx<T>::type*)L.r64 : (typename cplx<T>::type*)L.r32;
  const size_t nb = sizeof(typename cplx<T>::type) * (size_t)R * 2 * L.n;
  CK(cudaMemsetAsync(r, 0, nb, st));
  CK(cudaMemsetAsync(e, 0, nb, st));
  cudaEvent_t a = nullptr, b = nullptr;
  CK(cudaEventCreate(&a));
  if (cudaEventCreate(&b) != cudaSuccess) { cudaEventDestroy(a); h->err = "cudaEventCreate"; return AMAMG_ERR_CUDA; }
  const bool prof = h->prof;
  h->prof = false;
  const int sweeps = h->prm.post_smooth > 0 ? h->prm.post_smooth : 2;
  float best = 1e30f;
  std::pair<int, int> pick = cand[0];
  int rc = AMAMG_OK;
  const bool log = getenv("AMAMG_TUNE_LOG") != nullptr;
  bool any = false, sticky = false;
  for (const auto& c : cand) {
    tm[R] = c;
    rc = AMAMG_OK;
    for (int w = 0; w < 2 && rc == AMAMG_OK; ++w) rc = smooth_impl<T>(h, l, e, r, R, sweeps, st);
    if (rc == AMAMG_OK && cudaEventRecord(a, st) != cudaSuccess) rc = AMAMG_ERR_CUDA;
    for (int w = 0; w < 5 && rc == AMAMG_OK; ++w) rc = smooth_impl<T>(h, l, e, r, R, sweeps, st);
    if (rc == AMAMG_OK && (cudaEventRecord(b, st) != cudaSuccess || cudaEventSynchronize(b) != cudaSuccess))
      rc = AMAMG_ERR_CUDA;
    if (rc != AMAMG_OK) {
      // a candidate the driver refuses at launch (a configuration error, not a
      // fault) is dropped; a sticky error ends the tuning
      const cudaError_t le = cudaGetLastError();
      if (log) fprintf(stderr, "amamg autotune: level %d R %d kernel %d variant %d refused: %s\n", l, R, c.first,
                       c.second, h->err.c_str());
      if (cudaStreamSynchronize(st) != cudaSuccess) { (void)le; sticky = true; break; }
      h->err.clear();
      continue;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    if (log) fprintf(stderr, "amamg autotune: level %d %s R %d kernel %d variant %d: %.1f us\n", l, f64 ? "f64" : "f32",
                     R, c.first, c.second, 1e3 * ms / 5);
    any = true;
    if (ms < best) { best = ms; pick = c; }
  }
  h->prof = prof;
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (sticky) {
    tm.erase(R);
    if (h->err.empty()) h->err = "autotune: the stream failed";
    return AMAMG_ERR_CUDA;
  }
  if (!any) {
    tm.erase(R);                                             // nothing ran: the fixed rule stands
    return AMAMG_OK;
  }
  tm[R] = pick;
  return check_grid_sync(h, st);
}

// Tunes every smoothed coarse level for R right-hand sides in precision prec
// (AMAMG_F64 or AMAMG_F32) when the handle asks for it.
int tune_smoothers(amamg_ctx* h, int R, int prec, cudaStream_t st) {
  if (!h->prm.autotune) return AMAMG_OK;
  for (int l = 1; l + 1 < (int)h->lv.size(); ++l)
    CKS(prec == AMAMG_F64 ? tune_level<double>(h, l, R, st) : tune_level<float>(h, l, R, st));
  return AMAMG_OK;
}

// Solver kernels read the per-RHS mass arrays while this guard is alive.
struct MassGuard {
  amamg_ctx* h;
  explicit MassGuard(amamg_ctx* hh) : h(hh) {
    h->cur_diag64 = h->d_diag64;
    h->cur_inv64 = h->d_inv64;
    h->cur_inv32 = h->d_inv32;
  }
  ~MassGuard() { h->cur_diag64 = nullptr; h->cur_inv64 = nullptr; h->cur_inv32 = nullptr; }
};

int fgmres_on(amamg_ctx* h, const double2* psi, double2* x, int R, cudaStream_t st, amamg_solve_info* info) {
  const long len = 2L * h->lv[0].n;
  CKS(ensure_vcycle_ws(h, R));
  CKS(ensure_solver_ws(h, R));
  CKS(tune_smoothers(h, R, h->prm.precision == AMAMG_SOLVE_MIXED ? AMAMG_F32 : AMAMG_F64, st));
  std::vector<double> masses(R, h->m0);
  CKS(set_masses(h, masses.data(), R, st));
  MassGuard guard(h);
  std::vector<SlotState> sl(R);
  for (auto& q : sl) { q.active = 1; q.fresh = 1; q.done = 0; }
  CK(cudaMemsetAsync(x, 0, sizeof(double2) * R * len, st));
  int cycles = 0;
  while (true) {
    bool left = false;
    CKS(fgmres_cycle(h, psi, x, R, st, sl, &left));
    if (!left) break;
    if (++cycles > h->prm.max_iter + 1) break;   // every cycle takes at least one step
  }
  int rc = AMAMG_OK;
  bool nonfinite = false;
  for (int r = 0; r < R; ++r) {
    if (info) { info[r].iterations = sl[r].iters; info[r].status = sl[r].status; info[r].true_relres = sl[r].relres; }
    if (sl[r].status == AMAMG_NOT_CONVERGED && rc == AMAMG_OK) rc = AMAMG_NOT_CONVERGED;
    if (sl[r].status == AMAMG_ERR_NONFINITE) nonfinite = true;
  }
  if (nonfinite) { h->err = "non-finite value in a right-hand side or residual"; rc = AMAMG_ERR_NONFINITE; }
  CKS(check_grid_sync(h, st));
  return rc;
}

// The solve runs on the handle's own stream, ordered after the caller's stream
// and before anything the caller enqueues afterwards.
int fgmres(amamg_ctx* h, const double2* psi, double2* x, int R, cudaStream_t st, amamg_solve_info* info) {
  CK(cudaEventRecord(h->ev_in, st));
  CK(cudaStreamWaitEvent(h->ws, h->ev_in, 0));
  const int rc = fgmres_on(h, psi, x, R, h->ws, info);
  CK(cudaEventRecord(h->ev_out, h->ws));
  CK(cudaStreamWaitEvent(st, h->ev_out, 0));
  return rc;
}

// ----------------------------------------------------------------- setup
int check_params(const amamg_params* p, int Nt, int Nx, std::string* why) {
  if (!p) { *why = "params is NULL"; return AMAMG_ERR_INVALID_ARG; }
  if (p->nlevels < 2 || p->nlevels > AMAMG_MAX_LEVELS) { *why = "nlevels must be 2..4"; return AMAMG_ERR_INVALID_ARG; }
  if (p->precision != AMAMG_SOLVE_FP64 && p->precision != AMAMG_SOLVE_MIXED) { *why = "bad precision"; return AMAMG_ERR_INVALID_ARG; }
  if (p->restart < 1 || p->restart > 64) { *why = "restart must be 1..64"; return AMAMG_ERR_INVALID_ARG; }
  if (p->autotune != 0 && p->autotune != 1) { *why = "autotune must be 0 or 1"; return AMAMG_ERR_INVALID_ARG; }
  if (p->max_iter < 1 || p->post_smooth < 0 || !(p->tol > 0.0)) { *why = "bad max_iter/post_smooth/tol"; return AMAMG_ERR_INVALID_ARG; }
  if (p->spin_split != 0 && p->spin_split != 1) { *why = "spin_split must be 0 or 1"; return AMAMG_ERR_INVALID_ARG; }
  if (p->normalization != AMAMG_NORM_NONE && p->normalization != AMAMG_NORM_ROWSUM) {
    *why = "normalization must be AMAMG_NORM_NONE or AMAMG_NORM_ROWSUM";
    return AMAMG_ERR_INVALID_ARG;
  }
  if (p->edge_owner != AMAMG_OWNER_TILE && p->edge_owner != AMAMG_OWNER_FIRST_LEX) {
    *why = "edge_owner must be AMAMG_OWNER_TILE or AMAMG_OWNER_FIRST_LEX";
    return AMAMG_ERR_INVALID_ARG;
  }
  if (Nt < 4 || Nx < 4 || (Nt & 1) || (Nx & 1)) { *why = "Nt, Nx must be even and >= 4"; return AMAMG_ERR_INVALID_ARG; }
  int nt = Nt, nx = Nx;
  for (int l = 0; l + 1 < p->nlevels; ++l) {
    const int a = p->agg[l];
    if (a != 2 && a != 4) { *why = "tile sides must be 2 or 4"; return AMAMG_ERR_INVALID_ARG; }
    if (nt % a || nx % a || nt / a < 2 || nx / a < 2) { *why = "tile side does not divide the level extents"; return AMAMG_ERR_INVALID_ARG; }
    if (l >= 1 && (nt % 4 || nx % 4)) { *why = "smoothed coarse levels need extents divisible by 4"; return AMAMG_ERR_INVALID_ARG; }
    nt /= a; nx /= a;
  }
  if (p->gs_arith != AMAMG_GS_FP64 && p->gs_arith != AMAMG_GS_DF64) {
    *why = "gs_arith must be AMAMG_GS_FP64 or AMAMG_GS_DF64";
    return AMAMG_ERR_INVALID_ARG;
  }
  if (p->gs_arith == AMAMG_GS_DF64 && p->precision != AMAMG_SOLVE_MIXED) {
    *why = "AMAMG_GS_DF64 needs AMAMG_SOLVE_MIXED";
    return AMAMG_ERR_INVALID_ARG;
  }
  if (p->gs_method != AMAMG_GS_CGS2 && p->gs_method != AMAMG_GS_MGS) {
    *why = "gs_method must be AMAMG_GS_CGS2 or AMAMG_GS_MGS";
    return AMAMG_ERR_INVALID_ARG;
  }
  if (p->gs_method == AMAMG_GS_MGS && p->gs_arith != AMAMG_GS_FP64) {
    *why = "AMAMG_GS_MGS runs in FP64 arithmetic (gs_arith AMAMG_GS_FP64)";
    return AMAMG_ERR_INVALID_ARG;
  }
  if (p->coarsest != AMAMG_COARSEST_DIRECT && p->coarsest != AMAMG_COARSEST_GMRES) {
    *why = "coarsest must be AMAMG_COARSEST_DIRECT or AMAMG_COARSEST_GMRES";
    return AMAMG_ERR_INVALID_ARG;
  }
  const double nd = 2.0 * nt * nx;
  if (p->coarsest == AMAMG_COARSEST_DIRECT && nd > 16384) {
    *why = "coarsest level too large for the dense inverse (2 Nt_L Nx_L > 16384)";
    return AMAMG_ERR_INVALID_ARG;
  }
  return AMAMG_OK;
}

void free_all(amamg_ctx* h) {
  for (auto& L : h->lv) {
    dfree(L.B64); dfree(L.B16); dfree(L.Bs); dfree(L.Dinv64); dfree(L.Dinv32);
    dfree(L.Bc64); dfree(L.Bc16); dfree(L.Bcs); dfree(L.Dc64); dfree(L.Dc32);
    dfree(L.P64); dfree(L.P16); dfree(L.Ps);
    dfree(L.r64); dfree(L.e64); dfree(L.r32); dfree(L.e32);
    dfree(L.ctW); dfree(L.ctWs);
  }
  dfree(h->ct_stage); dfree(h->ct_amax);
  clear_graphs(h);
  if (h->ws) cudaStreamDestroy(h->ws);
  if (h->ev_in) cudaEventDestroy(h->ev_in);
  if (h->ev_out) cudaEventDestroy(h->ev_out);
  h->ws = nullptr; h->ev_in = h->ev_out = nullptr;
  if (h->ws2) cudaStreamDestroy(h->ws2);
  if (h->ev_fork) cudaEventDestroy(h->ev_fork);
  if (h->ev_join) cudaEventDestroy(h->ev_join);
  h->ws2 = nullptr; h->ev_fork = h->ev_join = nullptr;
  dfree(h->U64); dfree(h->U64s); dfree(h->U32); dfree(h->Ainv); dfree(h->Ainv32); dfree(h->d_err); dfree(h->d_sync); dfree(h->d_owner_flags);
  dfree(h->d_smax); dfree(h->d_rowsum_skipped);
  dfree(h->gm_V); dfree(h->gm_part); dfree(h->gm_st); dfree(h->gm_done); dfree(h->tc_bop);
  dfree(h->V); dfree(h->Z64); dfree(h->Z32); dfree(h->v32); dfree(h->w); dfree(h->res); dfree(h->wdf); dfree(h->df_part);
  dfree(h->partial); dfree(h->d_h); dfree(h->d_inv); dfree(h->d_flag); dfree(h->d_y); dfree(h->d_tickets); dfree(h->d_npart);
  dfree(h->d_diag64); dfree(h->d_inv64); dfree(h->d_inv32);
  dfree(h->ls_H); dfree(h->ls_Q); dfree(h->ls_R); dfree(h->ls_g); dfree(h->ls_bnorm); dfree(h->ls_st);
  dfree(h->d_lsout); dfree(h->d_lsinit);
  if (h->h_h) cudaFreeHost(h->h_h);
  if (h->h_lsout) cudaFreeHost(h->h_lsout);
  if (h->h_lsinit) cudaFreeHost(h->h_lsinit);
  h->h_h = nullptr;
  h->h_lsout = nullptr;
  h->h_lsinit = nullptr;
  for (auto e : h->ev_pool) cudaEventDestroy(e);
  h->ev_pool.clear();
}

int do_setup(amamg_ctx* h, const void* Uin, cudaStream_t st) {
  const int L = h->prm.nlevels;
  h->lv.resize(L);
  {
    Level& F = h->lv[0];
    F.Nt = h->Nt; F.Nx = h->Nx; F.n = h->Nt * h->Nx;
  }
  const size_t nl = 2 * (size_t)h->lv[0].n;
  CK(cudaStreamCreateWithFlags(&h->ws, cudaStreamNonBlocking));
  CK(cudaEventCreateWithFlags(&h->ev_in, cudaEventDisableTiming));
  CK(cudaEventCreateWithFlags(&h->ev_out, cudaEventDisableTiming));
  CK(cudaStreamCreateWithFlags(&h->ws2, cudaStreamNonBlocking));
  CK(cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming));
  CK(cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming));
  CKS(dalloc(h, &h->U64, nl));
  CKS(dalloc(h, &h->U64s, nl));
  CKS(dalloc(h, &h->U32, nl));
  CKS(dalloc(h, &h->d_err, 1));
  CK(cudaMemsetAsync(h->d_err, 0, sizeof(int), st));
  CKS(dalloc(h, &h->d_sync, 8));
  CK(cudaMemsetAsync(h->d_sync, 0, 8 * sizeof(unsigned), st));
  CKS(dalloc(h, &h->d_owner_flags, OWNER_MAX_BLOCKS));
  CK(cudaMemsetAsync(h->d_owner_flags, 0, OWNER_MAX_BLOCKS * sizeof(unsigned), st));
  CKS(dalloc(h, &h->d_smax, 1));
  CKS(dalloc(h, &h->d_rowsum_skipped, AMAMG_MAX_LEVELS));
  CK(cudaMemsetAsync(h->d_rowsum_skipped, 0, AMAMG_MAX_LEVELS * sizeof(unsigned), st));
  CK(cudaMemcpyAsync(h->U64, Uin, nl * sizeof(double2), cudaMemcpyDeviceToDevice, st));
  CK(cudaMemcpyAsync(h->U64s, Uin, nl * sizeof(double2), cudaMemcpyDeviceToDevice, st));
  CKS(launch(h, "setup_cast_links", nl * 24.0, st, [&] {
    const cudaError_t e = launch_fold_boundary_sign(h->U64s, h->Nt, h->Nx, st);
    return e != cudaSuccess ? e : launch_cast<double2, float2>(h->U64s, h->U32, (long)nl, st);
  }));
  Offsets fine_off = wilson_offsets(h->Nt, h->Nx);
  for (int l = 0; l + 1 < L; ++l) {
    Level& F = h->lv[l];
    Level& C = h->lv[l + 1];
    F.a = h->prm.agg[l];
    F.Np = F.Nt / F.a; F.Nq = F.Nx / F.a; F.nT = F.Np * F.Nq; F.nrows = 2 * (F.a * F.a - 1);
    C.Nt = F.Np; C.Nx = F.Nq; C.n = F.nT;
    CKS(dalloc(h, &F.P64, (size_t)F.nT * 8 * F.nrows));
    CKS(dalloc(h, &F.P16, (size_t)F.nT * 8 * F.nrows));
    CKS(dalloc(h, &F.Ps, (size_t)F.nT));
    const Offsets& fo = (l == 0) ? fine_off : F.off;
    if (coarse_offsets(fo, F.Nt, F.Nx, F.a, h->prm.edge_owner, &C.off) != AMAMG_OK) {
      h->err = "coarse operator has more block offsets than the library stores (48)";
      return AMAMG_ERR_INVALID_ARG;
    }
    if (l + 2 < L && C.off.K - 1 > GS_MAX_OFFDIAG) {   // a smoothed coarse level
      h->err = "smoothed coarse level has more block offsets than the Gauss-Seidel kernels support (25)";
      return AMAMG_ERR_INVALID_ARG;
    }
    CKS(dalloc(h, &C.B64, (size_t)C.off.K * 4 * C.n));
    const int own = h->prm.edge_owner;
    // local interpolation, then Eq. (16)'s normalisation (row sums) and the
    // optional spin split, then the Galerkin product with the final P
    auto build_level = [&](const auto& op) -> int {
      CKS(launch(h, "setup_local_solve", 0.0, st,
                 [&] { return launch_local_solve(op, F.a, F.Np, F.Nq, F.P64, h->d_err, own, st); }));
      if (h->prm.normalization == AMAMG_NORM_ROWSUM)
        CKS(launch(h, "setup_rowsum", 0.0, st, [&] {
          return launch_rowsum_normalize(F.P64, F.nrows, F.nT, h->d_smax, h->d_rowsum_skipped + l, st);
        }));
      if (h->prm.spin_split)
        CKS(launch(h, "setup_spin_split", 0.0, st, [&] { return launch_spin_split_P(F.P64, F.nrows, F.nT, st); }));
      return launch(h, "setup_galerkin", 0.0, st,
                    [&] { return launch_galerkin(op, F.P64, F.a, F.Np, F.Nq, C.off, C.B64, own, st); });
    };
    if (l == 0) CKS(build_level(WilsonOp{h->U64, h->m0 + 2.0, F.Nt, F.Nx}));
    else CKS(build_level(StencilOp{F.B64, F.off, F.Nt, F.Nx}));
    CKS(launch(h, "setup_pack", 0.0, st, [&] { return launch_pack_P16(F.P64, 8 * F.nrows, F.nT, F.P16, F.Ps, st); }));
  }
  for (int l = 1; l < L; ++l) {
    Level& C = h->lv[l];
    CKS(dalloc(h, &C.B16, (size_t)C.off.K * 4 * C.n));
    CKS(dalloc(h, &C.Bs, (size_t)C.off.K * C.n));
    CKS(launch(h, "setup_pack", 0.0, st, [&] { return launch_pack_B16(C.B64, C.off.K, C.n, C.B16, C.Bs, st); }));
    if (l + 1 < L) {
      CKS(dalloc(h, &C.Dinv64, 4 * (size_t)C.n));
      CKS(dalloc(h, &C.Dinv32, 4 * (size_t)C.n));
      CKS(launch(h, "setup_diag_inv", 0.0, st, [&] { return launch_diag_inv(C.B64, C.n, C.Dinv64, C.Dinv32, h->d_err, st); }));
      C.ncol = gs_colours(C);
      const size_t nb = (size_t)(C.off.K - 1) * C.n;      // ncol colours x (K-1) offsets x n/ncol sites
      CKS(dalloc(h, &C.Bc64, 4 * nb));
      CKS(dalloc(h, &C.Bc16, 4 * nb));
      CKS(dalloc(h, &C.Bcs, nb));
      CKS(dalloc(h, &C.Dc64, 4 * (size_t)C.n));
      CKS(dalloc(h, &C.Dc32, 4 * (size_t)C.n));
      CKS(launch(h, "setup_pack", 0.0, st, [&] {
        return launch_pack_colour_major(C.B64, C.B16, C.Bs, C.Dinv64, C.Dinv32, C.off.K, C.Nt, C.Nx, C.ncol, C.Bc64,
                                        C.Bc16, C.Bcs, C.Dc64, C.Dc32, st);
      }));
      choose_gs_kernels(C);
    }
  }
  // coarsest: GMRES workspace, or the dense matrix and its Gauss-Jordan inverse
  Level& Cl = h->lv[L - 1];
  h->nd = 2 * Cl.n;
  const size_t nd = (size_t)h->nd;
  if (h->prm.coarsest == AMAMG_COARSEST_GMRES) {
    h->gm_blocks64 = coarsest_gmres_blocks<double, double2>(GMRES_RESTART);
    h->gm_blocks32 = coarsest_gmres_blocks<float, __half2>(GMRES_RESTART);
    const int gb = std::max(h->gm_blocks64, h->gm_blocks32);
    if (h->gm_blocks64 <= 0 || h->gm_blocks32 <= 0) {
      h->err = "cooperative launches are unavailable for the coarsest GMRES";
      return AMAMG_ERR_CUDA;
    }
    CKS(dalloc(h, &h->gm_V, (size_t)(GMRES_RESTART + 1) * GMRES_MAX_R * nd));
    CKS(dalloc(h, &h->gm_part, (size_t)gb * GMRES_MAX_R * (GMRES_RESTART + 2)));
    CKS(dalloc(h, &h->gm_st, (size_t)GMRES_MAX_R));
    CKS(dalloc(h, &h->gm_done, 1));
    int herr = 0;
    CK(cudaMemcpyAsync(&herr, h->d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (herr) {
      h->err = (herr & 1) ? "vanishing pivot in a local basket solve" : "singular 2x2 diagonal block on a coarse level";
      return AMAMG_ERR_SINGULAR;
    }
    return AMAMG_OK;
  }
  double2* X = nullptr;
  double2* colk = nullptr;
  int* perm = nullptr;
  CKS(dalloc(h, &X, nd * nd));
  int rc = dalloc(h, &h->Ainv, nd * nd);
  if (rc == AMAMG_OK) rc = dalloc(h, &colk, nd);
  if (rc == AMAMG_OK) rc = dalloc(h, &perm, nd);
  if (rc == AMAMG_OK && cudaMemsetAsync(X, 0, nd * nd * sizeof(double2), st) != cudaSuccess) rc = AMAMG_ERR_CUDA;
  if (rc == AMAMG_OK)
    rc = launch(h, "setup_coarsest", 0.0, st, [&] { return launch_dense_from_blocks(Cl.B64, Cl.off, Cl.Nt, Cl.Nx, X, st); });
  for (int k = 0; rc == AMAMG_OK && k < h->nd; ++k)
    rc = launch(h, "setup_coarsest", 0.0, st, [&] { return launch_gj_step(X, h->nd, k, colk, perm, h->d_err, 1e-300, st); });
  std::vector<int> hperm(nd), cols(nd);
  if (rc == AMAMG_OK && cudaMemcpyAsync(hperm.data(), perm, nd * sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess) rc = AMAMG_ERR_CUDA;
  if (rc == AMAMG_OK && cudaStreamSynchronize(st) != cudaSuccess) rc = AMAMG_ERR_CUDA;
  if (rc == AMAMG_OK) {
    for (size_t i = 0; i < nd; ++i) cols[i] = (int)i;
    for (int k = h->nd - 1; k >= 0; --k) std::swap(cols[k], cols[hperm[k]]);
    if (cudaMemcpyAsync(perm, cols.data(), nd * sizeof(int), cudaMemcpyHostToDevice, st) != cudaSuccess) rc = AMAMG_ERR_CUDA;
  }
  if (rc == AMAMG_OK)
    rc = launch(h, "setup_coarsest", 0.0, st, [&] { return launch_gather_cols(X, h->Ainv, perm, h->nd, st); });
  if (rc == AMAMG_OK) rc = dalloc(h, &h->Ainv32, nd * nd);
  if (rc == AMAMG_OK)
    rc = launch(h, "setup_cast", 0.0, st, [&] { return launch_cast<double2, float2>(h->Ainv, h->Ainv32, (long)(nd * nd), st); });
  // tensor-core apply of Ainv32 to many right-hand sides (mixed V-cycle)
  const char* tc_env = std::getenv("AMAMG_COARSEST_TC");
  if (rc == AMAMG_OK && coarsest_tc_possible(h->nd, 8) && !(tc_env && std::strcmp(tc_env, "0") == 0) &&
      coarsest_tc_init() == cudaSuccess) {
    rc = dalloc(h, &h->tc_bop, coarsest_tc_scratch_elems(h->nd));
    h->tc_ok = rc == AMAMG_OK;
  }
  cudaGetLastError();
  int herr = 0;
  if (rc == AMAMG_OK && cudaMemcpyAsync(&herr, h->d_err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess) rc = AMAMG_ERR_CUDA;
  if (rc == AMAMG_OK && cudaStreamSynchronize(st) != cudaSuccess) rc = AMAMG_ERR_CUDA;
  dfree(X); dfree(colk); dfree(perm);
  if (rc == AMAMG_ERR_CUDA && h->err.empty()) h->err = cudaGetErrorString(cudaGetLastError());
  if (rc != AMAMG_OK) return rc;
  if (herr) {
    h->err = (herr & 1) ? "vanishing pivot in a local basket solve"
           : (herr & 2) ? "singular 2x2 diagonal block on a coarse level"
                        : "vanishing pivot in the coarsest inverse";
    return AMAMG_ERR_SINGULAR;
  }
  return AMAMG_OK;
}

bool valid_level(amamg_ctx* h, int level, bool need_next) {
  if (level < 0 || level >= (int)h->lv.size()) return false;
  if (need_next && level + 1 >= (int)h->lv.size()) return false;
  return true;
}

}  // namespace

template <typename T>
int engine_vcycle(amamg_ctx* h, const typename cplx<T>::type* r, typename cplx<T>::type* e, const VcycleVecs<T>& w,
                  int R, cudaStream_t st) {
  return vcycle_from<T>(h, 0, r, e, w, R, st);
}
template int engine_vcycle<double>(amamg_ctx*, const double2*, double2*, const VcycleVecs<double>&, int, cudaStream_t);
template int engine_vcycle<float>(amamg_ctx*, const float2*, float2*, const VcycleVecs<float>&, int, cudaStream_t);

// =================================================================== C ABI
extern "C" {

int amamg_default_params(amamg_params* p) {
  if (!p) return AMAMG_ERR_INVALID_ARG;
  std::memset(p, 0, sizeof(*p));
  p->nlevels = 2;
  p->agg[0] = 4; p->agg[1] = 2; p->agg[2] = 2; p->agg[3] = 2;
  p->precision = AMAMG_SOLVE_FP64;
  p->restart = 30;
  p->max_iter = 3000;
  p->post_smooth = 2;
  p->tol = 1e-10;
  return AMAMG_OK;
}

int amamg_query_bytes(const amamg_params* p, int Nt, int Nx, int max_rhs, size_t* setup_bytes, size_t* per_rhs_bytes) {
  std::string why;
  int rc = check_params(p, Nt, Nx, &why);
  if (rc != AMAMG_OK) return rc;
  if (max_rhs < 1) return AMAMG_ERR_INVALID_ARG;
  size_t sb = 2 * (size_t)Nt * Nx * (16 + 16 + 8);   // links FP64 (as given, sign-folded) + FP32
  size_t vb = 0;                                 // V-cycle vectors per RHS
  int nt = Nt, nx = Nx;
  Offsets off = wilson_offsets(Nt, Nx);
  for (int l = 0; l + 1 < p->nlevels; ++l) {
    const int a = p->agg[l];
    const size_t nT = (size_t)(nt / a) * (nx / a), nrows = 2 * (a * a - 1);
    sb += nT * 8 * nrows * (16 + 4) + nT * 4;
    Offsets c;
    if (coarse_offsets(off, nt, nx, a, p->edge_owner, &c) != AMAMG_OK) return AMAMG_ERR_INVALID_ARG;
    nt /= a; nx /= a;
    const size_t n = (size_t)nt * nx;
    sb += (size_t)c.K * n * (4 * 16 + 4 * 4 + 4) + 4 * n * (16 + 8);
    vb += 2 * n * 2 * (16 + 8);
    off = c;
  }
  const size_t nd = 2 * (size_t)nt * nx;
  if (p->coarsest == AMAMG_COARSEST_GMRES)
    sb += (size_t)(30 + 1) * 32 * nd * 16 + 32 * sizeof(GmresRhs) + (size_t)2 * 148 * 32 * 32 * 16;
  else
    sb += 2 * nd * nd * 16 + nd * nd * 8;        // inverse, its work copy during setup, its FP32 rounding
  const size_t len = 2 * (size_t)Nt * Nx;
  const int m = p->restart;
  size_t rb = vb + (size_t)(m + 1) * len * 16 + 2 * len * 16 +
              (p->precision == AMAMG_SOLVE_MIXED ? (size_t)(m + 1) * len * 8 : (size_t)m * len * 16);
  if (setup_bytes) *setup_bytes = sb;
  if (per_rhs_bytes) *per_rhs_bytes = rb;
  return AMAMG_OK;
}

int amamg_setup(const amamg_params* p, const void* U, int Nt, int Nx, double m0, void* stream, amamg_handle* out) {
  if (!out) return AMAMG_ERR_INVALID_ARG;
  *out = nullptr;
  std::string why;
  int rc = check_params(p, Nt, Nx, &why);
  if (rc != AMAMG_OK) return rc;
  if (!U || !std::isfinite(m0)) return AMAMG_ERR_INVALID_ARG;
  amamg_ctx* h = new amamg_ctx();
  h->prm = *p;
  // AMAMG_GRAPHS=0 runs the Arnoldi steps as plain launches instead of CUDA
  // graphs (same kernels; for profilers that handle graph nodes slowly)
  if (const char* g = std::getenv("AMAMG_GRAPHS")) h->use_graphs = std::strcmp(g, "0") != 0;
  // AMAMG_FINE_FUSED=1 runs the fine-level prolongation and red-black sweeps as
  // one cooperative launch (same arithmetic; measured no faster than the
  // separate launches on the 256^2 workload, so off by default)
  if (const char* g = std::getenv("AMAMG_FINE_FUSED")) h->fine_fused = std::atoi(g) != 0;
  if (const char* g = std::getenv("AMAMG_FAIL_ALLOC_AFTER")) h->fail_alloc_after = std::atoi(g);
  h->Nt = Nt; h->Nx = Nx; h->m0 = m0;
  cudaStream_t st = S(stream);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0, st);
  rc = do_setup(h, U, st);
  if (rc == AMAMG_OK) {
    cudaEventRecord(e1, st);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    h->setup_s = ms * 1e-3;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != AMAMG_OK) {
    fprintf(stderr, "amamg_setup: %s\n", h->err.c_str());
    free_all(h);
    delete h;
    return rc;
  }
  h->recs.clear();
  h->ev_used = 0;
  *out = h;
  return AMAMG_OK;
}

int amamg_solve(amamg_handle h, const void* psi, void* x, int R, void* stream, amamg_solve_info* info) {
  if (!h || !psi || !x || R < 1) return AMAMG_ERR_INVALID_ARG;
  return fgmres(h, (const double2*)psi, (double2*)x, R, S(stream), info);
}

int amamg_batch_create(amamg_handle h, int slots, amamg_batch_handle* out) {
  if (!h || !out || slots < 1) return AMAMG_ERR_INVALID_ARG;
  *out = nullptr;
  int rc = ensure_vcycle_ws(h, slots);
  if (rc == AMAMG_OK) rc = ensure_solver_ws(h, slots);
  if (rc != AMAMG_OK) return rc;
  amamg_batch* b = new amamg_batch();
  b->h = h;
  b->S = slots;
  const size_t n = (size_t)slots * 2 * (size_t)h->lv[0].n;   // slots x len complex elements
  if (cudaMalloc((void**)&b->B, n * sizeof(double2)) != cudaSuccess ||
      cudaMalloc((void**)&b->X, n * sizeof(double2)) != cudaSuccess) {
    cudaGetLastError();
    if (b->B) cudaFree(b->B);
    if (b->X) cudaFree(b->X);
    delete b;
    h->err = "amamg_batch_create: out of device memory";
    return AMAMG_ERR_OOM;
  }
  cudaMemset(b->B, 0, n * sizeof(double2));
  cudaMemset(b->X, 0, n * sizeof(double2));
  b->sl.assign(slots, SlotState());
  b->mass.assign(slots, h->m0);
  *out = b;
  return AMAMG_OK;
}

int amamg_batch_admit(amamg_batch_handle b, int slot, const void* psi, double m0, void* stream) {
  if (!b || !psi || slot < 0 || slot >= b->S || !std::isfinite(m0)) return AMAMG_ERR_INVALID_ARG;
  amamg_ctx* h = b->h;
  if (b->sl[slot].active) { h->err = "amamg_batch_admit: slot is occupied"; return AMAMG_ERR_INVALID_ARG; }
  const size_t len = 2 * (size_t)h->lv[0].n;
  cudaStream_t st = S(stream);
  CK(cudaMemcpyAsync(b->B + slot * len, psi, len * sizeof(double2), cudaMemcpyDeviceToDevice, st));
  CK(cudaMemsetAsync(b->X + slot * len, 0, len * sizeof(double2), st));
  SlotState q;
  q.active = 1; q.fresh = 1; q.done = 0;
  b->sl[slot] = q;
  b->mass[slot] = m0;
  return AMAMG_OK;
}

int amamg_batch_cycle(amamg_batch_handle b, void* stream, amamg_slot_info* info) {
  if (!b) return AMAMG_ERR_INVALID_ARG;
  amamg_ctx* h = b->h;
  cudaStream_t st = S(stream);
  const int R = b->S;
  int rc = ensure_vcycle_ws(h, R);
  if (rc == AMAMG_OK) rc = ensure_solver_ws(h, R);
  if (rc != AMAMG_OK) return rc;
  CK(cudaEventRecord(h->ev_in, st));
  CK(cudaStreamWaitEvent(h->ws, h->ev_in, 0));
  rc = tune_smoothers(h, R, h->prm.precision == AMAMG_SOLVE_MIXED ? AMAMG_F32 : AMAMG_F64, h->ws);
  if (rc == AMAMG_OK) rc = set_masses(h, b->mass.data(), R, h->ws);
  bool left = false;
  if (rc == AMAMG_OK) {
    MassGuard guard(h);
    rc = fgmres_cycle(h, b->B, b->X, R, h->ws, b->sl, &left);
  }
  if (rc == AMAMG_OK) rc = check_grid_sync(h, h->ws);
  CK(cudaEventRecord(h->ev_out, h->ws));
  CK(cudaStreamWaitEvent(st, h->ev_out, 0));
  CK(cudaStreamSynchronize(st));
  if (info)
    for (int r = 0; r < R; ++r) {
      const SlotState& q = b->sl[r];
      info[r].active = q.active;
      info[r].done = q.active ? q.done : 1;
      info[r].status = q.status;
      info[r].iterations = q.iters;
      info[r].true_relres = q.relres;
    }
  return rc;
}

int amamg_batch_retire(amamg_batch_handle b, int slot, void* x, void* stream) {
  if (!b || slot < 0 || slot >= b->S) return AMAMG_ERR_INVALID_ARG;
  amamg_ctx* h = b->h;
  const size_t len = 2 * (size_t)h->lv[0].n;
  cudaStream_t st = S(stream);
  if (x) CK(cudaMemcpyAsync(x, b->X + slot * len, len * sizeof(double2), cudaMemcpyDeviceToDevice, st));
  CK(cudaMemsetAsync(b->B + slot * len, 0, len * sizeof(double2), st));
  CK(cudaMemsetAsync(b->X + slot * len, 0, len * sizeof(double2), st));
  b->sl[slot] = SlotState();
  b->mass[slot] = h->m0;
  return AMAMG_OK;
}

int amamg_batch_destroy(amamg_batch_handle b) {
  if (!b) return AMAMG_ERR_INVALID_ARG;
  cudaDeviceSynchronize();
  if (b->B) cudaFree(b->B);
  if (b->X) cudaFree(b->X);
  delete b;
  return AMAMG_OK;
}

int amamg_apply_D(amamg_handle h, const void* in, void* out, int R, int precision, void* stream) {
  if (!h || !in || !out || R < 1) return AMAMG_ERR_INVALID_ARG;
  if (precision == AMAMG_F64) return op_dslash<double>(h, (const double2*)in, (double2*)out, nullptr, R, S(stream));
  if (precision == AMAMG_F32) return op_dslash<float>(h, (const float2*)in, (float2*)out, nullptr, R, S(stream));
  if (precision == AMAMG_F32_F64) {
    const Level& L = h->lv[0];
    cudaStream_t st = S(stream);
    return launch(h, "dslash_mixed", (double)L.n * (R * (16.0 + 32.0) + 32.0), st, [&] {
      return launch_dslash<float2, double2, double>((const float2*)in, (double2*)out, nullptr, h->U64s, h->m0 + 2.0,
                                                    L.Nt, L.Nx, R, st);
    }, (double)L.n * R * 56.0);
  }
  return AMAMG_ERR_INVALID_ARG;
}

int amamg_apply_P(amamg_handle h, int level, const void* ci, void* fo, int R, int precision, void* stream) {
  if (!h || !ci || !fo || R < 1 || !valid_level(h, level, true)) return AMAMG_ERR_INVALID_ARG;
  if (precision == AMAMG_F64) return op_prolong<double>(h, level, (const double2*)ci, (double2*)fo, R, S(stream));
  if (precision == AMAMG_F32) return op_prolong<float>(h, level, (const float2*)ci, (float2*)fo, R, S(stream));
  return AMAMG_ERR_INVALID_ARG;
}

int amamg_apply_PH(amamg_handle h, int level, const void* fi, void* co, int R, int precision, void* stream) {
  if (!h || !fi || !co || R < 1 || !valid_level(h, level, true)) return AMAMG_ERR_INVALID_ARG;
  if (precision == AMAMG_F64) return op_restrict<double>(h, level, (const double2*)fi, (double2*)co, R, S(stream));
  if (precision == AMAMG_F32) return op_restrict<float>(h, level, (const float2*)fi, (float2*)co, R, S(stream));
  return AMAMG_ERR_INVALID_ARG;
}

int amamg_apply_coarse(amamg_handle h, int level, const void* in, void* out, int R, int precision, void* stream) {
  if (!h || !in || !out || R < 1 || level < 1 || !valid_level(h, level, false)) return AMAMG_ERR_INVALID_ARG;
  if (precision == AMAMG_F64)
    return op_coarse<double>(h, level, (const double2*)in, (double2*)out, nullptr, R, S(stream));
  if (precision == AMAMG_F32)
    return op_coarse<float>(h, level, (const float2*)in, (float2*)out, nullptr, R, S(stream));
  return AMAMG_ERR_INVALID_ARG;
}

int amamg_smooth(amamg_handle h, int level, const void* r, void* e, int R, int sweeps, int precision, void* stream) {
  if (!h || !r || !e || R < 1 || sweeps < 0 || !valid_level(h, level, true)) return AMAMG_ERR_INVALID_ARG;
  if (precision == AMAMG_F64) return smooth_impl<double>(h, level, (double2*)e, (const double2*)r, R, sweeps, S(stream));
  if (precision == AMAMG_F32) return smooth_impl<float>(h, level, (float2*)e, (const float2*)r, R, sweeps, S(stream));
  return AMAMG_ERR_INVALID_ARG;
}

int amamg_selftest_sync_timeout(amamg_handle h, int level, int precision, void* stream) {
  if (!h || level < 1 || level + 1 >= (int)h->lv.size()) return AMAMG_ERR_INVALID_ARG;
  if (precision != AMAMG_F64 && precision != AMAMG_F32) return AMAMG_ERR_INVALID_ARG;
  cudaStream_t st = S(stream);
  CKS(ensure_vcycle_ws(h, 1));
  Level& L = h->lv[level];
  OwnerConfig oc;
  const bool f64 = precision == AMAMG_F64;
  const bool ok = f64 ? owner_sweep_config<double, double2>(L.Nt, L.Nx, L.off.K, L.ncol, L.off, 1, &oc)
                      : owner_sweep_config<float, __half2>(L.Nt, L.Nx, L.off.K, L.ncol, L.off, 1, &oc);
  if (!ok || oc.blocks < 2) {
    h->err = "level has no owner sweep with two or more blocks";
    return AMAMG_ERR_INVALID_ARG;
  }
  cudaError_t e;
  if (f64) {
    CK(cudaMemsetAsync(L.r64, 0, sizeof(double2) * 2 * L.n, st));
    CK(cudaMemsetAsync(L.e64, 0, sizeof(double2) * 2 * L.n, st));
    e = launch_coarse_sweeps_owner<double, double2>(L.e64, L.r64, L.Bc64, nullptr, L.Dc64, L.off, L.Nt, L.Nx, L.ncol,
                                                    2, 1, h->d_owner_flags, h->d_sync, st, 0);
  } else {
    CK(cudaMemsetAsync(L.r32, 0, sizeof(float2) * 2 * L.n, st));
    CK(cudaMemsetAsync(L.e32, 0, sizeof(float2) * 2 * L.n, st));
    e = launch_coarse_sweeps_owner<float, __half2>(L.e32, L.r32, L.Bc16, L.Bcs, L.Dc32, L.off, L.Nt, L.Nx, L.ncol,
                                                   2, 1, h->d_owner_flags, h->d_sync, st, 0);
  }
  CK(e);
  h->launches++;
  return AMAMG_OK;
}

int amamg_sync_status(amamg_handle h, void* stream) {
  if (!h) return AMAMG_ERR_INVALID_ARG;
  return check_grid_sync(h, S(stream));
}

int amamg_coarsest_solve(amamg_handle h, const void* r, void* e, int R, void* stream) {
  if (!h || !r || !e || R < 1) return AMAMG_ERR_INVALID_ARG;
  return vcycle_coarsest(h, (const double2*)r, (double2*)e, R, S(stream));
}

int amamg_coarsest_apply(amamg_handle h, const void* r, void* e, int R, int precision, void* stream) {
  if (!h || !r || !e || R < 1) return AMAMG_ERR_INVALID_ARG;
  if (precision == AMAMG_F64) return vcycle_coarsest(h, (const double2*)r, (double2*)e, R, S(stream));
  if (precision == AMAMG_F32) return vcycle_coarsest(h, (const float2*)r, (float2*)e, R, S(stream));
  return AMAMG_ERR_INVALID_ARG;
}

int amamg_query_smoother(amamg_handle h, int level, int precision, int R, int* kernel, int* variant) {
  if (!h || !kernel || !variant || level < 1 || level + 1 >= (int)h->lv.size() || R < 1) return AMAMG_ERR_INVALID_ARG;
  std::pair<int, int> c;
  if (precision == AMAMG_F64) c = gs_choice<double>(h->lv[level], R);
  else if (precision == AMAMG_F32) c = gs_choice<float>(h->lv[level], R);
  else return AMAMG_ERR_INVALID_ARG;
  *kernel = c.first;
  *variant = c.second;
  return AMAMG_OK;
}

int amamg_vcycle(amamg_handle h, const void* r, void* e, int R, int precision, void* stream) {
  if (!h || !r || !e || R < 1) return AMAMG_ERR_INVALID_ARG;
  if (precision != AMAMG_F64 && precision != AMAMG_F32) return AMAMG_ERR_INVALID_ARG;
  int rc = ensure_vcycle_ws(h, R);
  if (rc == AMAMG_OK) rc = tune_smoothers(h, R, precision, S(stream));
  if (rc != AMAMG_OK) return rc;
  if (precision == AMAMG_F64)
    return vcycle_from<double>(h, 0, (const double2*)r, (double2*)e, handle_vecs<double>(h), R, S(stream));
  if (precision == AMAMG_F32)
    return vcycle_from<float>(h, 0, (const float2*)r, (float2*)e, handle_vecs<float>(h), R, S(stream));
  return AMAMG_ERR_INVALID_ARG;
}

int amamg_export_structure(amamg_handle h, int level, int32_t* role, int32_t* owner_tile, int32_t* nbr_offsets,
                           int32_t* nbr_count) {
  if (!h || !valid_level(h, level, true)) return AMAMG_ERR_INVALID_ARG;
  const Level& L = h->lv[level];
  const Level& C = h->lv[level + 1];
  if (role || owner_tile) {
    // computed on the device by the ownership rule the transfer kernels use
    int* d = nullptr;
    CKS(dalloc(h, &d, 2 * (size_t)L.n));
    cudaError_t e = launch_structure(L.Nt, L.Nx, L.a, h->prm.edge_owner, d, d + L.n, 0);
    std::vector<int> tmp(2 * (size_t)L.n);
    if (e == cudaSuccess) e = cudaMemcpy(tmp.data(), d, sizeof(int) * 2 * L.n, cudaMemcpyDeviceToHost);
    dfree(d);
    CK(e);
    for (int s = 0; s < L.n; ++s) {
      if (role) role[s] = tmp[s];
      if (owner_tile) owner_tile[s] = tmp[L.n + s];
    }
  }
  if (nbr_offsets)
    for (int k = 0; k < C.off.K; ++k) { nbr_offsets[2 * k] = C.off.dt[k]; nbr_offsets[2 * k + 1] = C.off.dx[k]; }
  if (nbr_count) *nbr_count = C.off.K;
  return AMAMG_OK;
}

int amamg_level_info(amamg_handle h, int level, int* Nt_l, int* Nx_l, int* n_offsets) {
  if (!h || !valid_level(h, level, false)) return AMAMG_ERR_INVALID_ARG;
  const Level& L = h->lv[level];
  if (Nt_l) *Nt_l = L.Nt;
  if (Nx_l) *Nx_l = L.Nx;
  if (n_offsets) *n_offsets = level == 0 ? 5 : L.off.K;
  return AMAMG_OK;
}

int amamg_export_P(amamg_handle h, int level, void* out, void* stream) {
  if (!h || !out || !valid_level(h, level, true)) return AMAMG_ERR_INVALID_ARG;
  const Level& L = h->lv[level];
  CK(cudaMemcpyAsync(out, L.P64, sizeof(double2) * L.nT * 8 * L.nrows, cudaMemcpyDeviceToDevice, S(stream)));
  return AMAMG_OK;
}

int amamg_export_coarse(amamg_handle h, int level, void* out, void* stream) {
  if (!h || !out || level < 1 || !valid_level(h, level, false)) return AMAMG_ERR_INVALID_ARG;
  const Level& L = h->lv[level];
  CK(cudaMemcpyAsync(out, L.B64, sizeof(double2) * L.off.K * 4 * L.n, cudaMemcpyDeviceToDevice, S(stream)));
  return AMAMG_OK;
}

int amamg_profile_enable(amamg_handle h, int on) {
  if (!h) return AMAMG_ERR_INVALID_ARG;
  if (!on && h->prof) {
    int rc = collect_profile(h);
    if (rc != AMAMG_OK) return rc;
  }
  h->prof = on != 0;
  return AMAMG_OK;
}

int amamg_profile_reset(amamg_handle h) {
  if (!h) return AMAMG_ERR_INVALID_ARG;
  int rc = collect_profile(h);
  h->cats.clear();
  return rc;
}

int amamg_profile_get(amamg_handle h, int idx, const char** name, long long* launches, double* total_ms, double* bytes,
                      double* flops) {
  if (!h) return AMAMG_ERR_INVALID_ARG;
  int rc = collect_profile(h);
  if (rc != AMAMG_OK) return rc;
  if (idx < 0 || idx >= (int)h->cats.size()) return AMAMG_ERR_INVALID_ARG;
  const ProfCat& c = h->cats[idx];
  if (name) *name = c.name.c_str();
  if (launches) *launches = c.launches;
  if (total_ms) *total_ms = c.ms;
  if (bytes) *bytes = c.bytes;
  if (flops) *flops = c.flops;
  return AMAMG_OK;
}

long long amamg_launch_count(amamg_handle h) { return h ? h->launches : -1; }

double amamg_setup_seconds(amamg_handle h) { return h ? h->setup_s : -1.0; }

int amamg_destroy(amamg_handle h) {
  if (!h) return AMAMG_ERR_INVALID_ARG;
  cudaDeviceSynchronize();
  free_all(h);
  delete h;
  return AMAMG_OK;
}

const char* amamg_status_string(int s) {
  switch (s) {
    case AMAMG_OK: return "ok";
    case AMAMG_NOT_CONVERGED: return "not converged (max_iter reached)";
    case AMAMG_ERR_INVALID_ARG: return "invalid argument";
    case AMAMG_ERR_OOM: return "out of device memory";
    case AMAMG_ERR_CUDA: return "CUDA error";
    case AMAMG_ERR_SINGULAR: return "singular pivot in setup";
    case AMAMG_ERR_NONFINITE: return "non-finite value";
    case AMAMG_ERR_TIMEOUT: return "timeout";
    default: return "unknown status";
  }
}

const char* amamg_last_error(amamg_handle h) { return h ? h->err.c_str() : "null handle"; }

}  // extern "C"
