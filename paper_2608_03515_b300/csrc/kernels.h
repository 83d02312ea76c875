// Kernel launchers of the library (one declaration per kernel family).
// Every launcher enqueues on the given stream and returns cudaGetLastError().
#pragma once
#include "common.cuh"

// level operators as seen by the setup kernels
struct WilsonOp {          // fine level, Eq. (3)
  const double2* U;        // [2][Nt][Nx]
  double diag;             // m0 + 2
  int Nt, Nx;
};
struct StencilOp {         // Galerkin level, [K][4][n] blocks
  const double2* B;
  Offsets off;
  int Nt, Nx;
};

// dslash.cu
// diag = m0 + 2 (inv_diag = its inverse) for every right-hand side, or per
// right-hand side from a device array when diag_r / inv_diag_r is given
template <typename Cin, typename Cout, typename T>
cudaError_t launch_dslash(const Cin* in, Cout* out, const Cout* b, const typename cplx<T>::type* U, T diag, int Nt,
                          int Nx, int R, cudaStream_t st, const T* diag_r = nullptr);
// out = sigma_3 D sigma_3 in = D^H in (Eq. (6)), FP64, diag = m0 + 2
cudaError_t launch_dslash_dag(const double2* in, double2* out, const double2* U, double diag, int Nt, int Nx, int R,
                              cudaStream_t st);
template <typename T>
cudaError_t launch_rb_half(typename cplx<T>::type* e, const typename cplx<T>::type* r, const typename cplx<T>::type* U,
                           T inv_diag, int Nt, int Nx, int colour, int R, cudaStream_t st,
                           const T* inv_diag_r = nullptr);

// transfer.cu (own: edge-ownership rule, OwnerRule)
template <typename T, typename PT>
cudaError_t launch_prolong(const typename cplx<T>::type* ec, typename cplx<T>::type* ef, const PT* P,
                           const float* Pscale, int Nxf, int a, int Np, int Nq, int R, cudaStream_t st,
                           int own = OWN_TILE);
template <typename T, typename PT>
cudaError_t launch_restrict(const typename cplx<T>::type* ef, typename cplx<T>::type* ec, const PT* P,
                            const float* Pscale, int Nxf, int a, int Np, int Nq, int R, cudaStream_t st,
                            int own = OWN_TILE);

// role (0 vertex, 1 edge, 2 interior) and owner basket of every site of a
// level, as the transfer kernels index them (device int arrays of Nt Nx)
cudaError_t launch_structure(int Nt, int Nx, int a, int own, int* role, int* owner, cudaStream_t st);

// links with the t-boundary sign folded into U_0(Nt-1, x) (what the stencil
// kernels take)
cudaError_t launch_fold_boundary_sign(double2* U, int Nt, int Nx, cudaStream_t st);

// Fine-level end of the V-cycle (e = P e_c, then `sweeps` red-black sweeps on
// D e = r) in one cooperative launch of row-owning blocks with neighbour waits
// (flags / sync as the owner sweep); the same arithmetic per site as
// launch_prolong followed by the launch_rb_half sequence.  fine_post_rows = 0:
// no resident shape for R (the separate kernels run).
constexpr int FINE_MAX_BLOCKS = 4096;
template <typename T, typename PT>
int fine_post_rows(int Nt, int Nx, int a, int R);
template <typename T, typename PT>
cudaError_t launch_fine_post(const typename cplx<T>::type* ec, typename cplx<T>::type* e,
                             const typename cplx<T>::type* r, const PT* P, const float* Pscale,
                             const typename cplx<T>::type* U, T inv_diag, const T* inv_diag_r, int Nt, int Nx, int a,
                             int sweeps, int R, unsigned* flags, unsigned* sync, cudaStream_t st);

// coarse.cu
template <typename T, typename BT>
cudaError_t launch_coarse_apply(const typename cplx<T>::type* in, typename cplx<T>::type* out,
                                const typename cplx<T>::type* b, const BT* B, const float* Bs, const Offsets& off,
                                int Nt, int Nx, int R, cudaStream_t st);
template <typename T, typename BT>
cudaError_t launch_coarse_colour(typename cplx<T>::type* e, const typename cplx<T>::type* r, const BT* B,
                                 const float* Bs, const typename cplx<T>::type* Dinv, const Offsets& off, int Nt,
                                 int Nx, int ncol, int colour, int R, cudaStream_t st);
// all colours of `sweeps` sweeps in one launch, one 8-block cluster per RHS;
// usable while n / ncol <= 8 * 1024 sites per colour
constexpr int CLUSTER_BLOCKS = 8;
int cluster_sweep_threads(int n, int ncol);
template <typename T, typename BT>
cudaError_t launch_coarse_sweeps_cluster(typename cplx<T>::type* e, const typename cplx<T>::type* r, const BT* B,
                                         const float* Bs, const typename cplx<T>::type* Dinv, const Offsets& off,
                                         int Nt, int Nx, int ncol, int sweeps, int R, cudaStream_t st);
// all colours of `sweeps` sweeps in one cooperative launch over the whole GPU,
// colour phases separated by a bounded software grid barrier on
// sync[0..2] = {count, generation, error} (zeroed before first use; a time-out
// sets sync[2]); grid_sweep_blocks = 0 when cooperative launches are unavailable
template <typename T, typename BT>
int grid_sweep_blocks(int n, int ncol, int R);
template <typename T, typename BT>
cudaError_t launch_coarse_sweeps_grid(typename cplx<T>::type* e, const typename cplx<T>::type* r, const BT* B,
                                      const float* Bs, const typename cplx<T>::type* Dinv, const Offsets& off,
                                      int Nt, int Nx, int ncol, int sweeps, int R, unsigned* sync, cudaStream_t st);
// all colours of `sweeps` sweeps in one cooperative launch, each block owning
// cnt sites of every colour and waiting only for the blocks that own its
// sites' neighbours (per-block phase flags, no grid barrier); flags:
// OWNER_MAX_BLOCKS counters, sync[3] epoch base, sync[4] end ticket, sync[2]
// time-out flag
constexpr int OWNER_MAX_BLOCKS = 4096;
constexpr int OWNER_MAX_WAIT = 256;
struct OwnerConfig {
  int cnt = 0, threads = 0, blocks = 0, late_half = 0, slots = 4, nearly = 1, early_lanes = 8;
  size_t smem = 0;
  bool bsmem = false;
};
// variant: the autotuner's shape candidates (0: the fixed rule; see coarse.cu)
template <typename T, typename BT>
bool owner_sweep_config(int Nt, int Nx, int K, int ncol, const Offsets& off, int R, OwnerConfig* cfg,
                        int variant = 0);
template <typename T, typename BT>
cudaError_t launch_coarse_sweeps_owner(typename cplx<T>::type* e, const typename cplx<T>::type* r, const BT* Bc,
                                       const float* Sc, const typename cplx<T>::type* Dc, const Offsets& off,
                                       int Nt, int Nx, int ncol, int sweeps, int R, unsigned* flags, unsigned* sync,
                                       cudaStream_t st, int withhold = -1, int variant = 0);
// Coarse Gauss-Seidel kernel choice.  Levels with n = 16 ncol per sites (per <= 64)
// run all colours on one 16-block cluster with the level in distributed shared
// memory; in FP32 also the off-diagonal blocks live in shared memory when they
// fit (n <= 8192).  Other FP32 levels use the L2-based clustered sweep, other
// FP64 levels one launch per colour spread over all SMs.
constexpr int DSMEM_CLUSTER = 16;
size_t dsmem_sweep_bytes(int n, int K, size_t cbytes, bool bsmem, size_t bt_bytes);
template <typename T, typename BT>
bool dsmem_sweeps_possible(int n, int K, int ncol, bool bsmem);
template <typename T>
inline bool dsmem_blocks_in_smem(int n, int K) {
  return sizeof(T) == 4 && dsmem_sweep_bytes(n, K, 8, true, 4) <= 200 * 1024;
}
template <typename T>
inline bool use_cluster_sweeps(int n, int ncol) {
  return sizeof(T) == 4 && cluster_sweep_threads(n, ncol) <= 1024;
}
template <typename T, typename BT>
cudaError_t launch_coarse_sweeps_dsmem(typename cplx<T>::type* e, const typename cplx<T>::type* r, const BT* Bc,
                                       const float* Sc, const typename cplx<T>::type* Dc, const Offsets& off,
                                       int Nt, int Nx, int ncol, int sweeps, int R, bool bsmem, cudaStream_t st);
template <typename Cv>
cudaError_t launch_dense_gemv(const double2* A, const Cv* x, Cv* y, int nd, int R, cudaStream_t st);
cudaError_t launch_dense_gemv32(const float2* A, const float2* x, float2* y, int nd, int R, cudaStream_t st);

// blas.cu
int dot_blocks(long len);
// dots of w with V_0..V_{J-1} (and with itself when with_self); blocks of a
// right-hand side whose gate flag is 0 do nothing
cudaError_t launch_dots(const double2* V, size_t vi, size_t vr, const double2* w, size_t wr, long len, int J, int R,
                        double2* partial, cudaStream_t st, bool with_self = false, const int* gate = nullptr);
cudaError_t launch_reduce(const double2* partial, int nb, int J, int R, double2* out, int ldo, int off, int mode,
                          double* inv, cudaStream_t st, int* flag = nullptr, int ref_off = 0, double eta2 = 0.5);
// Gram-Schmidt kernels with the reductions fused in (last-block tickets)
cudaError_t launch_dots_fused(const double2* V, size_t vi, size_t vr, const double2* w, size_t wr, long len, int J,
                              int R, double2* partial, bool with_self, const int* gate, unsigned* tickets,
                              double2* out, int ldo, int off, cudaStream_t st);
// stage i of modified Gram-Schmidt (w -= h_{i-1} v_{i-1}, then h_i = v_i^H w,
// or ||w|| at i = J); partial: pslots x dot_blocks(len) double2 per RHS
cudaError_t launch_mgs_stage(double2* w, size_t wr, const double2* V, size_t vi, size_t vr, long len, int i, int J,
                             int R, double2* partial, int pslots, unsigned* tickets, double2* out, int ldo, int off2,
                             int nrm_off, double* inv, cudaStream_t st);
int axpy_norm_blocks(long len);
cudaError_t launch_axpy_norm(double2* y, size_t yr, const double2* X, size_t xi, size_t xr, const double2* coef,
                             int ldc, int J, long len, int R, const int* gate, double* partial, unsigned* tickets,
                             double2* out, int ldo, int nrm_off, double* inv, int* flag, int ref_off, double eta2,
                             int mode, cudaStream_t st);
template <typename Cx>
cudaError_t launch_multi_axpy(double2* y, size_t yr, const Cx* X, size_t xi, size_t xr, const double2* coef, int ldc,
                              int J, double sign, long len, int R, cudaStream_t st, const int* gate = nullptr);
template <typename Cd>
cudaError_t launch_scale_copy(Cd* dst, size_t dr, const double2* src, size_t sr, const double* scale, long len, int R,
                              cudaStream_t st);
// dst_r = scale[r] src_r and dst32_r = its FP32 rounding (same strides)
cudaError_t launch_scale_copy_dual(double2* dst, float2* dst32, size_t dr, const double2* src, size_t sr,
                                   const double* scale, long len, int R, cudaStream_t st);
template <typename Cs, typename Cd>
cudaError_t launch_cast(const Cs* src, Cd* dst, long len, cudaStream_t st);
// Least-squares part of the outer FGMRES on the device, per right-hand side:
// the raw Hessenberg columns, the accumulated rotations Q^H (the product of
// the Givens rotations so far, (m + 1) x (m + 1), identity beyond the current
// step), the rotated right-hand side g = Q^H beta e_1 and st = {building, k,
// iters, nonfinite}.
struct LsView {
  double2* Hraw;    // [R][m + 1][m]: column j = (h_0j .. h_jj, h_{j+1,j})
  double2* Q;       // [R][m + 1][m + 1] accumulated Q^H (row i, column c at i (m + 1) + c)
  double2* Rm;      // [R][m][m] triangular factor Q^H H at the end of a cycle
  double2* g;       // [R][m + 1]
  double* bnorm;    // [R]
  int* st;          // [R][4]
};
struct LsOut { double est2; int building, k, iters, nonfinite; };  // per RHS (est2 = |g_{j+1}|^2), read each step
struct LsInit { double beta, bnorm; int building, iters; };        // per RHS, written by the host each cycle
cudaError_t launch_ls_init(LsView v, const LsInit* init, int R, int m, cudaStream_t st);
// Arnoldi step j: column j = h1 + h2 (the two Gram-Schmidt passes, rows 0..j of
// hcol[r]) and h_{j+1,j} = ||w|| (hcol[r][nrm_off].x); the rotation that
// annihilates h_{j+1,j} after the earlier ones, Q^H and g updated; the RHS
// stops building when |g_{j+1}| <= tol ||b||, on breakdown or after max_iter
// steps in total
cudaError_t launch_ls_step(LsView v, const double2* hcol, int ldh, int nrm_off, int j, int R, int m, double tol,
                           int max_iter, LsOut* out, cudaStream_t st);
// end of a cycle: R = Q^H H (k_r x k_r upper triangle), y_r = R^-1 g_r,
// zero-padded to m
cudaError_t launch_ls_solve(LsView v, double2* y, int R, int m, cudaStream_t st);

// setup.cu
// own: edge-ownership rule (OwnerRule, row_basket)
template <typename Op>
cudaError_t launch_local_solve(const Op& op, int a, int Np, int Nq, double2* P, int* err, int own, cudaStream_t st);
template <typename Op>
cudaError_t launch_galerkin(const Op& op, const double2* P, int a, int Np, int Nq, const Offsets& offc, double2* Bc,
                            int own, cudaStream_t st);
// Eq. (16) with N = diag(1 / row sum): every stored row divided by the sum of
// its 8 weights, except rows whose |sum| is below 1e-12 x the level's largest
// (their number is added to *skipped); smax: one device word of scratch
cudaError_t launch_rowsum_normalize(double2* P, int nrows, int ntiles, unsigned long long* smax, unsigned* skipped,
                                    cudaStream_t st);
cudaError_t launch_diag_inv(const double2* B, int n, double2* D64, float2* D32, int* err, cudaStream_t st);
cudaError_t launch_dense_from_blocks(const double2* B, const Offsets& off, int Nt, int Nx, double2* Ad,
                                     cudaStream_t st);
cudaError_t launch_gj_step(double2* A, int nd, int k, double2* colk, int* perm, int* err, double tol2,
                           cudaStream_t st);
cudaError_t launch_gather_cols(const double2* X, double2* Y, const int* cols, int nd, cudaStream_t st);
cudaError_t launch_pack_P16(const double2* P, int per_tile, int ntiles, __half2* P16, float* scale, cudaStream_t st);
// zero the cross-spin weights of every P tile ([ntiles][8][nrows])
cudaError_t launch_spin_split_P(double2* P, int nrows, int ntiles, cudaStream_t st);
cudaError_t launch_pack_B16(const double2* B, int K, int n, __half2* B16, float* scale, cudaStream_t st);
cudaError_t launch_pack_colour_major(const double2* B64, const __half2* B16, const float* Bs, const double2* D64,
                                     const float2* D32, int K, int Nt, int Nx, int ncol, double2* Bc64, __half2* Bc16,
                                     float* Bcs, double2* Dc64, float2* Dc32, cudaStream_t st);

// coarsest_gmres.cu: the coarsest level by unpreconditioned restarted GMRES to
// relative residual tol from a zero start (Sec. 5), one cooperative launch per
// at most GMRES_MAX_R right-hand sides; restart length m <= GMRES_MAX_M.
constexpr int GMRES_MAX_M = 32;
constexpr int GMRES_MAX_R = 32;
struct GmresRhs {                    // the small least-squares problem of one right-hand side (FP64)
  double2 H[(GMRES_MAX_M + 1) * GMRES_MAX_M];   // Hessenberg matrix, rotated in place, H[i * GMRES_MAX_M + j]
  double2 H2[GMRES_MAX_M];           // second-pass Gram-Schmidt coefficients of the current column
  double2 g[GMRES_MAX_M + 1];        // rotated right-hand side beta e_1
  double2 sn[GMRES_MAX_M];
  double2 y[GMRES_MAX_M];
  double cs[GMRES_MAX_M];
  double s[GMRES_MAX_M + 1];         // inverse norms of the stored (unnormalised) basis vectors
  double bnorm;
  int k, done, cdone, iters;         // steps this cycle, solved, cycle ended, total steps
};
size_t coarsest_gmres_smem(int R, int m);
// co-resident blocks of the kernel (cap of max_blocks), 0 without cooperative launches
template <typename T, typename BT>
int coarsest_gmres_blocks(int m);
// r, e: [R][2][Nt][Nx] (R <= GMRES_MAX_R); V: (m + 1) R 2 Nt Nx elements;
// part: max_blocks R (m + 2) double2; st: R records; sync: grid-barrier words
// {count (0 between launches), generation, time-out}
template <typename T, typename BT>
cudaError_t launch_coarsest_gmres(const typename cplx<T>::type* r, typename cplx<T>::type* e, const BT* B,
                                  const float* Bs, const Offsets& off, int Nt, int Nx, int R, int m, double tol,
                                  int max_cycles, typename cplx<T>::type* V, double2* part, GmresRhs* st,
                                  unsigned* sync, int* all_done, int max_blocks, cudaStream_t s);

// coarsest_tc.cu: y_r = Ainv32 x_r for R >= 8 right-hand sides on the tensor
// cores (tcgen05.mma kind::tf32 fed by TMA, FP32 accumulation in tensor
// memory, K split over CTAs for small levels); nd a multiple of 128.  scratch:
// coarsest_tc_scratch_elems(nd) floats; err: a word set when a bounded wait ran
// out.  coarsest_tc_init: once per process (opts the kernel in to its
// shared-memory size), outside stream capture.
bool coarsest_tc_possible(int nd, int R);
size_t coarsest_tc_scratch_elems(int nd);
cudaError_t coarsest_tc_init();
cudaError_t launch_coarsest_tc(const float2* A, const float2* x, float2* y, int nd, int R, float* scratch, int* err,
                               cudaStream_t st);

// coarse_tc.cu: y_r = A_l x_r for many right-hand sides on the tensor cores
// (tcgen05.mma kind::f16 over 2 x 4-site super-blocks, FP32 accumulation in
// tensor memory).  Operator images (coarse_tc_image_halves FP16 + scale floats)
// from the FP64 blocks by launch_coarse_tc_pack_w; per call the right-hand
// sides are staged in FP16 (stage: coarse_tc_stage_halves, amax: R words).
// coarse_tc_possible: even Nt >= 8, Nx >= 8 a multiple of 4, offsets within
// |dt|, |dx| <= 2.  coarse_tc_init: once per process, outside stream capture.
bool coarse_tc_possible(int Nt, int Nx, const Offsets& off);
size_t coarse_tc_image_halves(int Nt, int Nx);
size_t coarse_tc_scale_floats(int Nt, int Nx);
size_t coarse_tc_stage_halves(int Nt, int Nx, int R);
cudaError_t coarse_tc_init();
cudaError_t launch_coarse_tc_pack_w(const double2* B, const Offsets& off, int Nt, int Nx, __half* W, float* Ws,
                                    cudaStream_t st);
cudaError_t launch_coarse_tc(const float2* x, float2* y, const __half* W, const float* Ws, int Nt, int Nx, int R,
                             __half* stage, unsigned* amax, int* err, cudaStream_t st);

// gs_df.cu: the outer solver's Gram-Schmidt in double-float arithmetic (basis
// stored as double-float complex entries, 16 bytes each; see the file header)
cudaError_t launch_to_df(const double2* w, void* wd, long n, cudaStream_t st);
int df_partial_blocks(long len);   // inner-product partial sums: R (2 (m + 2)) df_partial_blocks(len) pairs
int df_norm_blocks(long len);      // norm partial sums: R df_norm_blocks(len) pairs
cudaError_t launch_dots_df(const void* V, size_t vi, size_t vr, const void* w, size_t wr, long len, int J, int R,
                           bool with_self, const int* gate, void* partial, int ps, unsigned* tickets, double2* out,
                           int ldo, int off, cudaStream_t st);
cudaError_t launch_axpy_norm_df(void* w, size_t wr, const void* V, size_t vi, size_t vr, const double2* coef, int ldc,
                                int J, long len, int R, const int* gate, void* partial, unsigned* tickets,
                                double2* out, int ldo, int nrm_off, double* inv, int* flag, int ref_off, double eta2,
                                int mode, cudaStream_t st);
cudaError_t launch_scale_copy_df(void* dst, float2* dst32, size_t dr, const void* src_df, const double2* src_d,
                                 size_t sr, const double* scale, long len, int R, cudaStream_t st);
