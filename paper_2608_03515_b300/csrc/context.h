// Host-side state of one hierarchy (the object behind amamg_handle).
#pragma once
#include <map>
#include <string>
#include <vector>

#include "../../include/amamg.h"
#include "kernels.h"

struct Level {
  int Nt = 0, Nx = 0, n = 0;            // sites of this level
  // coarsening to the next level (unused on the coarsest)
  int a = 0, Np = 0, Nq = 0, nT = 0, nrows = 0;
  // this level's operator for l >= 1: canonical offsets and blocks
  Offsets off{};
  double2* B64 = nullptr;
  __half2* B16 = nullptr;
  float* Bs = nullptr;
  double2* Dinv64 = nullptr;
  float2* Dinv32 = nullptr;
  // Gauss-Seidel colours of a smoothed coarse level: 8 ((t + 3x) mod 8) where no
  // coupling joins two sites of one such colour, else 16 ((t mod 4, x mod 4))
  int ncol = 16;
  // coarse Gauss-Seidel kernel of this level in FP64 and in FP32 (GsKernel),
  // chosen in setup
  int gs64 = 0, gs32 = 0;
  int gs32_multi = 0;        // FP32 with R >= 2 right-hand sides
  // the autotuner's (kernel, owner variant) per right-hand-side count
  std::map<int, std::pair<int, int>> tune64, tune32;
  // colour-major copies for the Gauss-Seidel kernels (smoothed coarse levels)
  double2* Bc64 = nullptr;
  __half2* Bc16 = nullptr;
  float* Bcs = nullptr;
  double2* Dc64 = nullptr;
  float2* Dc32 = nullptr;
  // tensor-core apply of this level's operator to many right-hand sides:
  // FP16 super-block images with per-row scales (built at the first use);
  // ct_state 0: not yet tried, 1: built, -1: not available for this level
  __half* ctW = nullptr;
  float* ctWs = nullptr;
  int ct_state = 0;
  // interpolation to the next level
  double2* P64 = nullptr;
  __half2* P16 = nullptr;
  float* Ps = nullptr;
  // V-cycle work vectors (capacity Rcap right-hand sides)
  double2* r64 = nullptr;
  double2* e64 = nullptr;
  float2* r32 = nullptr;
  float2* e32 = nullptr;
};

struct ProfCat {
  std::string name;
  long long launches = 0;
  double ms = 0.0;
  double bytes = 0.0;
  double flops = 0.0;
};

struct ProfRec {
  int cat;
  cudaEvent_t a, b;
  double bytes;
  double flops;
};

// per right-hand side state of the outer FGMRES (host side)
struct SlotState {
  double bnorm = 0.0, relres = 0.0;
  int iters = 0;
  int status = AMAMG_OK;
  int active = 0;   // slot holds a right-hand side
  int fresh = 0;    // ||b|| not yet measured
  int done = 1;     // converged, out of iterations, or failed
};

// Arnoldi scratch of one restart cycle (host side), R right-hand sides x m steps
// host mirror of the per-RHS progress of a restart cycle (the least-squares
// state itself lives on the device, LsView)
struct OuterState {
  int R = 0, m = 0;
  std::vector<int> k, building;
  void resize(int R_, int m_) {
    if (R_ == R && m_ == m) return;
    R = R_; m = m_;
    k.assign(R, 0);
    building.assign(R, 0);
  }
};

// Coarse Gauss-Seidel kernels (identical arithmetic per site): one launch per
// colour; all phases on an 8-block cluster with e in L2; all phases on a
// 16-block cluster with the level in distributed shared memory; all phases in
// one cooperative launch over the whole GPU with a software grid barrier; all
// phases in one cooperative launch of site-owning blocks that wait only for
// the owners of their sites' neighbours.
enum GsKernel : int { GS_COLOUR = 0, GS_CLUSTER = 1, GS_DSMEM = 2, GS_GRID = 3, GS_OWNER = 4 };

// The kernel a smoothing launch of R right-hand sides uses on level L: the one
// chosen in setup (FP32: one for R = 1, one for R >= 2), or the whole-GPU grid
// sweep when the owner sweep has no resident shape for this R.
template <typename T>
inline int gs_kind_for(const Level& L, int R) {
  constexpr bool f64 = sizeof(T) == 8;
  const int kind = f64 ? L.gs64 : (R == 1 ? L.gs32 : L.gs32_multi);
  if (kind != GS_OWNER || R == 1) return kind;
  OwnerConfig rc;
  const bool ok = f64 ? owner_sweep_config<double, double2>(L.Nt, L.Nx, L.off.K, L.ncol, L.off, R, &rc)
                      : owner_sweep_config<float, __half2>(L.Nt, L.Nx, L.off.K, L.ncol, L.off, R, &rc);
  return ok ? GS_OWNER : GS_GRID;
}

// (kernel, owner-sweep variant) of a smoothing launch: the autotuner's pick
// for this R where it ran (amamg_params.autotune), else the fixed rule above
template <typename T>
inline std::pair<int, int> gs_choice(const Level& L, int R) {
  const auto& tm = sizeof(T) == 8 ? L.tune64 : L.tune32;
  const auto it = tm.find(R);
  if (it != tm.end()) return it->second;
  return {gs_kind_for<T>(L, R), 0};
}

// Coarse-level work vectors of one V-cycle: r_l and e_l of level l >= 1
// (entry 0 unused), R right-hand sides each, [R][2][n_l] complex.
template <typename T>
struct VcycleVecs {
  typename cplx<T>::type* r[AMAMG_MAX_LEVELS] = {};
  typename cplx<T>::type* e[AMAMG_MAX_LEVELS] = {};
};

struct amamg_ctx {
  amamg_params prm{};
  int Nt = 0, Nx = 0;
  double m0 = 0.0;
  std::vector<Level> lv;
  double2* U64 = nullptr;    // links as given (setup's local operators)
  double2* U64s = nullptr;   // with the t-boundary sign folded in (stencil kernels)
  float2* U32 = nullptr;     // FP32 rounding of U64s
  // coarsest solve by GMRES (AMAMG_COARSEST_GMRES): basis, partial sums,
  // per-RHS least-squares state, "all done" word (GMRES_MAX_R right-hand sides
  // per launch)
  double2* gm_V = nullptr;
  double2* gm_part = nullptr;
  GmresRhs* gm_st = nullptr;
  int* gm_done = nullptr;
  int gm_blocks64 = 0, gm_blocks32 = 0;   // co-resident blocks of the GMRES kernel per precision
  double2* Ainv = nullptr;   // coarsest inverse, nd x nd row-major
  float2* Ainv32 = nullptr;  // its FP32 rounding, applied by the mixed-precision V-cycle
  float* tc_bop = nullptr;   // tensor-core coarsest apply: its right-hand-side operand (scratch)
  bool tc_ok = false;        // the tensor-core coarsest apply is available (AMAMG_COARSEST_TC=0: off)
  __half* ct_stage = nullptr;  // tensor-core coarse apply: FP16 staging of the right-hand sides
  size_t ct_stage_cap = 0;     // (halves)
  unsigned* ct_amax = nullptr; // their largest components (FP32 bits)
  int ct_amax_cap = 0;
  int nd = 0;
  int* d_err = nullptr;
  // coarse Gauss-Seidel synchronisation: [0] grid-barrier count, [1] its
  // generation, [2] time-out flag, [3] owner-sweep epoch base, [4] its end ticket
  unsigned* d_sync = nullptr;
  unsigned* d_owner_flags = nullptr;   // [OWNER_MAX_BLOCKS] owner-sweep phase counters
  unsigned long long* d_smax = nullptr;     // row-sum normalisation: largest |row sum| of a level (setup)
  unsigned* d_rowsum_skipped = nullptr;     // [AMAMG_MAX_LEVELS] rows left unnormalised per level

  // solver workspace
  int Rcap = 0;              // V-cycle work vectors
  int Rsolve = 0;            // FGMRES basis capacity
  int mcap = 0;
  double2* V = nullptr;      // [m+1][R][len]
  double2* Z64 = nullptr;    // [m][R][len]
  float2* Z32 = nullptr;     // [m][R][len]
  float2* v32 = nullptr;     // [R][len]
  double2* w = nullptr;      // [R][len]
  double2* res = nullptr;    // [R][len]
  double2* wdf = nullptr;    // [R][len] w in double-float form (AMAMG_GS_DF64; 16 bytes per entry)
  double* df_part = nullptr; // its inner-product and norm partial sums (pairs of floats, 8 bytes each)
  double2* partial = nullptr;
  size_t partial_elems = 0;
  double2* d_h = nullptr;    // [R][3 (m+2)] device: h1 | h2 | norms
  double* d_inv = nullptr;   // [R]
  int* d_flag = nullptr;     // [R] second Gram-Schmidt pass needed (DGKS)
  unsigned* d_tickets = nullptr;   // [R (m+2)] dots + [R] norms: last-block tickets (kept zero between uses)
  double* d_npart = nullptr;       // [R][blocks] partial squared norms
  double* d_diag64 = nullptr;  // [R] m0_r + 2 of each right-hand side
  double* d_inv64 = nullptr;   // [R] 1 / (m0_r + 2)
  float* d_inv32 = nullptr;    // [R] its FP32 rounding
  // the arrays above while a solve or batch cycle runs (nullptr: the handle's m0)
  const double* cur_diag64 = nullptr;
  const double* cur_inv64 = nullptr;
  const float* cur_inv32 = nullptr;
  OuterState outer;
  double2* d_y = nullptr;    // [R][m]
  double2* h_h = nullptr;    // pinned host mirror of d_h (norms at the start of a cycle)
  // device least-squares state of the outer FGMRES and its host exchange
  double2* ls_H = nullptr;   // [R][m + 1][m] raw Hessenberg columns
  double2* ls_Q = nullptr;   // [R][m + 1][m + 1] accumulated rotations
  double2* ls_R = nullptr;   // [R][m][m] triangular factor
  double2* ls_g = nullptr;   // [R][m + 1]
  double* ls_bnorm = nullptr;  // [R]
  int* ls_st = nullptr;      // [R][4]
  LsOut* d_lsout = nullptr;  // [R] per-step progress, copied to h_lsout
  LsOut* h_lsout = nullptr;  // pinned
  LsInit* d_lsinit = nullptr;  // [R] cycle start, copied from h_lsinit
  LsInit* h_lsinit = nullptr;  // pinned
  LsView ls() const { return LsView{ls_H, ls_Q, ls_R, ls_g, ls_bnorm, ls_st}; }

  // work stream of the solver (graph capture needs a non-default stream) and the
  // per-step CUDA graphs of one Arnoldi step j (captured once, replayed)
  cudaStream_t ws = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  // side branch of an Arnoldi step: the least-squares update runs on ws2 beside
  // the normalisation of the new basis vector
  cudaStream_t ws2 = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  std::vector<cudaGraphExec_t> step_graphs;
  std::vector<long long> step_graph_kernels;
  int graph_R = 0;
  bool use_graphs = true;
  bool fine_fused = false;   // fine-level prolongation + red-black sweeps in one launch (AMAMG_FINE_FUSED=1: on)

  std::string err;
  long long launches = 0;
  int fail_alloc_after = -1;   // allocation-failure injection (AMAMG_FAIL_ALLOC_AFTER); -1: off
  int allocs = 0;              // device allocations made through dalloc
  bool prof = false;
  std::vector<ProfCat> cats;
  std::vector<ProfRec> recs;
  std::vector<cudaEvent_t> ev_pool;
  size_t ev_used = 0;
  double setup_s = 0.0;
};

// a batch of right-hand-side slots on one hierarchy (continuous batching)
struct amamg_batch {
  amamg_ctx* h = nullptr;
  int S = 0;
  double2* B = nullptr;   // [S][len] right-hand sides
  double2* X = nullptr;   // [S][len] iterates
  std::vector<SlotState> sl;
  std::vector<double> mass;
};

// One V-cycle of Algorithm 1 on the fine level (start vector 0, no
// pre-smoothing, post_smooth sweeps per level) with the coarse work vectors w:
// the kernels and kernel choice of amamg_vcycle (amamg.cu).
template <typename T>
int engine_vcycle(amamg_ctx* h, const typename cplx<T>::type* r, typename cplx<T>::type* e, const VcycleVecs<T>& w,
                  int R, cudaStream_t st);
