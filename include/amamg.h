/*
 * amamg.h - C ABI of the B300 library for the SM-AMG preconditioned
 * Wilson-Dirac solve of the two-dimensional (Schwinger-model) Wilson operator.
 *
 * Problem statement (paper: "A first look at Structured-Multiscale Algebraic
 * Multigrid for Lattice Field Theory"):
 *   solve D x = psi (Eq. (1)) with the Wilson-Dirac operator D of Eq. (3)
 *   (Pauli basis of Eq. (4), periodic in x, antiperiodic in t, Eq. (7)), using
 *   FGMRES preconditioned by an SM-AMG V-cycle (Algorithm 1, Sec. 4): compact
 *   wirebasket aggregates with overlapping borders, ideal local interpolation
 *   (Eqs. (14)-(16)), Galerkin coarse operators A_H = P^H A P (Sec. 2).
 *
 * Conventions shared by every call
 *   - Lattice sites n = (t, x), 0 <= t < Nt, 0 <= x < Nx, site index t*Nx + x.
 *   - Gauge links U: device array of complex128 (two doubles re, im) laid out
 *     [mu][t][x], mu = 0 the t direction, mu = 1 the x direction.
 *   - Fine vectors: device arrays [R][spin 2][Nt][Nx] of complex128
 *     (AMAMG_F64) or complex64 (AMAMG_F32); R right-hand sides back to back.
 *   - Level-l vectors (l >= 1): [R][2][Nt_l][Nx_l], Nt_l = Nt / (a_0 ... a_{l-1}).
 *     The coarse variable of vertex (p, q), spin alpha is element
 *     [alpha][p][q]; vertex (p, q) is fine site (p*a, q*a) of the level below.
 *   - All device pointers are caller-owned (e.g. allocated by PyTorch); the
 *     library never frees them and keeps no pointer to them after a call
 *     returns.  The hierarchy (interpolators, coarse operators, coarsest
 *     inverse, solver workspace) is owned by the handle and freed by
 *     amamg_destroy.
 *   - Every call is ordered on the caller's stream (a cudaStream_t passed as
 *     void*, NULL = legacy default stream).  A handle is used by one stream at
 *     a time.  Calls that return data to the host (amamg_solve's info, the
 *     export functions) synchronise that stream.
 *   - Errors: every call returns an int status, AMAMG_OK (0) on success, a
 *     negative AMAMG_ERR_* on failure (no exception or abort crosses the ABI,
 *     no device assert or trap is used).  amamg_last_error(handle) gives a
 *     message for the last failure on that handle.
 */
#ifndef AMAMG_H
#define AMAMG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct amamg_ctx* amamg_handle;

/* status codes */
#define AMAMG_OK                 0
#define AMAMG_NOT_CONVERGED      1   /* max_iter reached; x holds the last iterate */
#define AMAMG_ERR_INVALID_ARG   -1
#define AMAMG_ERR_OOM           -2
#define AMAMG_ERR_CUDA          -3
#define AMAMG_ERR_SINGULAR      -4   /* a local or coarsest pivot vanished in setup */
#define AMAMG_ERR_NONFINITE     -5   /* NaN/Inf in a right-hand side or a residual */
#define AMAMG_ERR_TIMEOUT       -6   /* a bounded device wait of a coarse smoother ran out (reported by
                                        amamg_solve, amamg_batch_cycle and amamg_sync_status; the
                                        handle stays usable) */

/* vector precision of apply-style calls */
#define AMAMG_F64 0                  /* complex128 vectors, FP64 operators */
#define AMAMG_F32 1                  /* complex64 vectors, FP32 links, FP16+scale P and coarse blocks */
#define AMAMG_F32_F64 2              /* amamg_apply_D only: complex64 input, complex128 output, FP64 links
                                        and arithmetic (the product w = D z of the mixed solve, z from the
                                        FP32 V-cycle); equal to the FP64 stencil of the input widened to
                                        complex128 */

/* solve precision */
#define AMAMG_SOLVE_FP64  0          /* every step in FP64 */
#define AMAMG_SOLVE_MIXED 1          /* FP64 outer FGMRES, FP32 V-cycle, FP64 coarsest solve */

#define AMAMG_MAX_LEVELS 4

/* normalisation N of the local interpolation, Eq. (16) */
#define AMAMG_NORM_NONE   0          /* N = identity: the exact ideal interpolation (default) */
#define AMAMG_NORM_ROWSUM 1          /* every non-vertex scalar row of P divided by its complex row sum;
                                        rows whose |sum| is below 1e-12 x the level's largest |sum| stay */

/* coarsest-level solver inside the V-cycle */
#define AMAMG_COARSEST_DIRECT 0      /* exact: the FP64 inverse from setup (default) */
#define AMAMG_COARSEST_GMRES  1      /* the paper's setting (Sec. 5): unpreconditioned GMRES(30) from a
                                        zero start to relative residual 0.1, on the device */

/* arithmetic of the outer solver's Gram-Schmidt (inner products, updates, norms) */
#define AMAMG_GS_FP64 0              /* FP64 (default) */
#define AMAMG_GS_DF64 1              /* double-float: pairs of floats with about 48 significant bits, formed
                                        with error-free transformations on the FP32 pipe; the basis is kept
                                        in that form; mixed precision only.  A faster alternative on GPUs
                                        with a narrow FP64 pipe; the true residual stays FP64 */

/* variant of the outer solver's Gram-Schmidt (FP64 arithmetic) */
#define AMAMG_GS_CGS2 0              /* classical, with a second pass wherever the DGKS test asks for it
                                        (default): four kernels per Arnoldi step */
#define AMAMG_GS_MGS  1              /* modified (the oracle's variant): one stage per basis vector, each
                                        a fused update and inner product, half the FP64 work of CGS2 */

/* which basket a border site takes its formula from ("the first aggregate it
 * was assigned to", Sec. 4.1) */
#define AMAMG_OWNER_TILE      0      /* the basket of the tile containing the site, W(t/a, x/a) (default) */
#define AMAMG_OWNER_FIRST_LEX 1      /* of the baskets containing the site, the one of smallest index
                                        p (Nx/a) + q */

typedef struct {
    int    nlevels;                  /* 2..4 levels including the fine one */
    int    agg[AMAMG_MAX_LEVELS];    /* tile side a per coarsening step, 2 or 4; a | N_l, N_l/a >= 2 */
    int    precision;                /* AMAMG_SOLVE_FP64 or AMAMG_SOLVE_MIXED */
    int    restart;                  /* FGMRES restart length m, 1..64 */
    int    max_iter;                 /* total Arnoldi steps before AMAMG_NOT_CONVERGED */
    int    post_smooth;              /* post-smoothing sweeps per level (paper: 2); no pre-smoothing */
    double tol;                      /* relative residual ||psi - D x|| / ||psi|| */
    int    spin_split;               /* 0 (default): the ideal interpolation of Eq. (16), spins mixed;
                                        1: only its spin-diagonal weights, (P + s3 P s3) / 2, so the
                                        coarse operators keep sigma_3-hermiticity (the direction
                                        Sec. 6 proposes; a comparison hierarchy, not the method as read) */
    int    normalization;            /* AMAMG_NORM_NONE (default) or AMAMG_NORM_ROWSUM, every level */
    int    edge_owner;               /* AMAMG_OWNER_TILE (default) or AMAMG_OWNER_FIRST_LEX, every level */
    int    coarsest;                 /* AMAMG_COARSEST_DIRECT (default) or AMAMG_COARSEST_GMRES; with
                                        GMRES no dense inverse is formed (no size limit on the coarsest
                                        level) and the V-cycle is no longer a fixed linear map (the
                                        outer FGMRES is flexible) */
    int    gs_arith;                 /* AMAMG_GS_FP64 (default) or AMAMG_GS_DF64 (with AMAMG_SOLVE_MIXED) */
    int    autotune;                 /* 0 (default): fixed rules pick each coarse level's Gauss-Seidel
                                        kernel and its shape; 1: the first solve, batch cycle or
                                        amamg_vcycle of each right-hand-side count times the
                                        candidates on the handle's work vectors (CUDA events, before
                                        any graph capture) and keeps the fastest; the candidates
                                        compute the same sweeps up to rounding order.  Not part of
                                        the paper's method. */
    int    gs_method;                /* AMAMG_GS_CGS2 (default) or AMAMG_GS_MGS (with AMAMG_GS_FP64) */
} amamg_params;

typedef struct {
    int    iterations;               /* Arnoldi steps taken for this right-hand side */
    int    status;                   /* AMAMG_OK, AMAMG_NOT_CONVERGED or AMAMG_ERR_NONFINITE */
    double true_relres;              /* ||psi - D x|| / ||psi|| recomputed in FP64 at the end */
} amamg_solve_info;

/* Fills *p with the defaults: 2 levels, agg {4}, FP64, restart 30,
 * max_iter 3000, 2 post-smoothing sweeps, tol 1e-10. */
int amamg_default_params(amamg_params* p);

/* Device bytes the hierarchy of a Nt x Nx lattice needs (setup_bytes) and the
 * solver workspace per right-hand side (per_rhs_bytes); no GPU work, no
 * allocation.  Used for admission control. */
int amamg_query_bytes(const amamg_params* p, int Nt, int Nx, int max_rhs,
                      size_t* setup_bytes, size_t* per_rhs_bytes);

/* Setup phase (Sec. 2; SM-AMG interpolation Sec. 4.1, Eqs. (14)-(16)).
 * U: device complex128 [2][Nt][Nx] gauge links (read during the call only).
 * m0: bare mass.  Builds, on the device: wirebasket structure per level, the
 * local ideal interpolation of every basket (batched dense solves
 * -A_FF^{-1} A_FV in FP64), the Galerkin coarse operators P^H A P in
 * block-stencil form, their FP16+scale copies, the coarse smoother's 2x2
 * diagonal inverses and the coarsest level's inverse (FP64 LU with partial
 * pivoting carried to the inverse).  Requires Nt, Nx even and divisible by
 * every tile side, smoothed coarse levels with extents divisible by 4.
 * *out receives the handle; AMAMG_ERR_SINGULAR if a pivot vanishes. */
int amamg_setup(const amamg_params* p, const void* U, int Nt, int Nx, double m0,
                void* stream, amamg_handle* out);

/* Solve D x_r = psi_r for R right-hand sides (FGMRES(m), right-preconditioned
 * by one V-cycle per step; Sec. 1 and Sec. 5).  psi, x: device complex128
 * [R][2][Nt][Nx]; x is overwritten with the solution (start vector 0).
 * info: host array of R records.  Returns AMAMG_OK when every right-hand side
 * converged, AMAMG_NOT_CONVERGED if some stopped at max_iter, or an error. */
int amamg_solve(amamg_handle h, const void* psi, void* x, int R, void* stream,
                amamg_solve_info* info);

/* ---- Slot batches: continuous batching of solves on one hierarchy ----------
 * A batch owns S right-hand-side slots (device buffers for b and x).  Callers
 * admit a right-hand side into a free slot at any time between cycles, run
 * restart cycles of the outer FGMRES (Sec. 1 and Sec. 5) over every occupied
 * slot at once, and retire slots whose right-hand side is done, so that new
 * requests join while others are in flight.  Each slot carries its own bare
 * mass m0: the fine operator is D(m0_slot) = D(m0_setup) + (m0_slot - m0_setup) I
 * (Eq. (3)); the interpolators and coarse operators stay those of the setup
 * mass (the flexible outer solver tolerates the preconditioner's mass offset).
 * One batch per handle at a time (it uses the handle's solver workspace). */
typedef struct amamg_batch* amamg_batch_handle;

typedef struct {
    int    active;                   /* slot holds a right-hand side */
    int    done;                     /* converged, out of iterations, or failed */
    int    status;                   /* AMAMG_OK, AMAMG_NOT_CONVERGED or AMAMG_ERR_NONFINITE */
    int    iterations;               /* Arnoldi steps taken since admission */
    double true_relres;              /* ||b - D(m0) x|| / ||b|| at the start of the last cycle */
} amamg_slot_info;

/* Creates a batch of `slots` slots on hierarchy h (allocates its buffers). */
int amamg_batch_create(amamg_handle h, int slots, amamg_batch_handle* out);
/* Copies psi (device complex128 [2][Nt][Nx]) into free slot `slot` with mass m0,
 * on the caller's stream; AMAMG_ERR_INVALID_ARG if the slot is occupied. */
int amamg_batch_admit(amamg_batch_handle b, int slot, const void* psi, double m0, void* stream);
/* One restart cycle (at most `restart` Arnoldi steps) over every occupied,
 * unfinished slot; fills info[0..slots-1] (host) and synchronises the stream. */
int amamg_batch_cycle(amamg_batch_handle b, void* stream, amamg_slot_info* info);
/* Copies the slot's iterate to x (device complex128 [2][Nt][Nx]) and frees it. */
int amamg_batch_retire(amamg_batch_handle b, int slot, void* x, void* stream);
/* Synchronises the device and frees the batch's buffers (slots not retired
 * are dropped); the hierarchy stays.  AMAMG_ERR_INVALID_ARG for NULL. */
int amamg_batch_destroy(amamg_batch_handle b);

/* out = D in on the fine lattice, Eq. (3).  precision AMAMG_F64 (complex128 in
 * and out), AMAMG_F32 (complex64 in and out, FP32 links) or AMAMG_F32_F64
 * (complex64 in, complex128 out, FP64 links and arithmetic). */
int amamg_apply_D(amamg_handle h, const void* in, void* out, int R, int precision, void* stream);

/* out = D^H in = sigma_3 D sigma_3 in (sigma_3-hermiticity, Eq. (6)) on the
 * fine lattice at the setup mass; in, out: device complex128 [R][2][Nt][Nx]. */
int amamg_apply_Ddag(amamg_handle h, const void* in, void* out, int R, void* stream);

/* The paper's unpreconditioned comparison solver (Sec. 5): conjugate
 * gradients on the normal equations D^H D x = D^H psi (CGNR, x0 = 0) with
 * D^H = sigma_3 D sigma_3 (Eq. (6)), in FP64 on the device, at the setup mass.
 * psi, x: device complex128 [R][2][Nt][Nx] (x overwritten).  One iteration
 * applies D and D^H once; iterations stop for a right-hand side when the
 * recursive ||psi - D x|| / ||psi|| reaches tol, and the solve ends when the
 * true residual is below tol for every right-hand side (the recurrence restarts
 * from the true residual where it is not) or max_iter iterations are spent.
 * info: host array of R records (iterations, status, true relative residual).
 * Returns AMAMG_OK, AMAMG_NOT_CONVERGED (x holds the last iterate),
 * AMAMG_ERR_NONFINITE or an error; allocates its work vectors (4 R vectors). */
int amamg_cgnr(amamg_handle h, const void* psi, void* x, int R, int max_iter, double tol, void* stream,
               amamg_solve_info* info);

/* fine_out = P_l coarse_in: interpolation from level l+1 to level l
 * (Eq. (16) rows for owned edge/interior sites, identity on vertices).
 * coarse_in: level-(l+1) vectors, fine_out: level-l vectors ([R][2][Nt][Nx]
 * of that level), complex128 with AMAMG_F64 (FP64 P) or complex64 with
 * AMAMG_F32 (P in FP16 with one FP32 scale per tile); caller-owned, not
 * aliased.  AMAMG_ERR_INVALID_ARG for a level without a coarser one. */
int amamg_apply_P(amamg_handle h, int level, const void* coarse_in, void* fine_out,
                  int R, int precision, void* stream);

/* coarse_out = P_l^H fine_in: restriction from level l to level l+1 (Sec. 2);
 * layouts, precisions and errors as amamg_apply_P. */
int amamg_apply_PH(amamg_handle h, int level, const void* fine_in, void* coarse_out,
                   int R, int precision, void* stream);

/* out = A_l in with the Galerkin operator of level l >= 1 (A_l = P^H A_{l-1} P,
 * Sec. 2), a block stencil of 2x2 complex blocks.  in, out: level-l vectors
 * [R][2][Nt_l][Nx_l], complex128 (AMAMG_F64: FP64 blocks) or complex64
 * (AMAMG_F32).  With AMAMG_F32 and R >= 32 on a level with even Nt_l >= 8,
 * Nx_l >= 8 a multiple of 4 and block offsets within 2 sites, the product runs
 * on the tensor cores: 2 x 4-site super-blocks of the operator as dense
 * 16 x 96 complex tiles in FP16 with one FP32 scale per operator row, the
 * right-hand sides in FP16 with one power-of-two scale each, FP32 accumulation
 * (relative error about 5e-4 against the FP64 product, like the FP16 block
 * storage of the CUDA-core FP32 kernel, whose scale is per 2x2 block).  Its
 * first use on a level builds that level's FP16 images (6 KB per 8 coarse
 * sites) and a staging buffer of 2 bytes per complex entry of in, owned by the
 * handle; AMAMG_COARSE_TC=0 in the environment keeps the CUDA-core kernel.
 * A bounded wait of the tensor-core kernel that runs out is reported by
 * amamg_sync_status. */
int amamg_apply_coarse(amamg_handle h, int level, const void* in, void* out,
                       int R, int precision, void* stream);

/* Time-outs of apply-style calls.  The coarse smoothers of amamg_smooth,
 * amamg_vcycle and amamg_vcycle_noalloc wait on other thread blocks with
 * bounded polls; these calls only enqueue work and do not report a wait that
 * ran out (their e is then not the smoothed result).  Such a time-out stays
 * recorded on the handle until amamg_sync_status (or the next amamg_solve /
 * amamg_batch_cycle, which check at their end) reports it and re-arms the
 * counters. */

/* sweeps block Gauss-Seidel sweeps on A_l e = r, starting from the e passed in
 * (red-black on the fine level; on coarse levels 8 colours (t + 3x) mod 8
 * when both extents are multiples of 8 and no coupling (dt, dx) of the level
 * has dt + 3dx = 0 mod 8, else 16 colours (t mod 4, x mod 4); colours in
 * increasing order; "block solver as smoother", Sec. 5). */
int amamg_smooth(amamg_handle h, int level, const void* r, void* e, int R,
                 int sweeps, int precision, void* stream);

/* e = A_L^{-1} r on the coarsest level, in FP64 (complex128 vectors): the dense
 * inverse, or with AMAMG_COARSEST_GMRES the GMRES solve to relative residual 0.1. */
int amamg_coarsest_solve(amamg_handle h, const void* r, void* e, int R, void* stream);

/* The coarsest step of the V-cycle in the given precision: AMAMG_F64 as
 * amamg_coarsest_solve; AMAMG_F32 (complex64 vectors) the FP32 rounding of the
 * FP64 inverse, applied on the tensor cores (TF32 inputs, FP32 accumulation)
 * when R >= 8 and 2 Nt_L Nx_L is a multiple of 128, or GMRES in FP32 with
 * AMAMG_COARSEST_GMRES. */
int amamg_coarsest_apply(amamg_handle h, const void* r, void* e, int R, int precision, void* stream);

/* coarse Gauss-Seidel kernels (amamg_query_smoother) */
#define AMAMG_SMOOTHER_COLOUR  0     /* one launch per colour */
#define AMAMG_SMOOTHER_CLUSTER 1     /* all phases on an 8-block cluster, e in L2 (FP32) */
#define AMAMG_SMOOTHER_DSMEM   2     /* all phases on a 16-block cluster, the level in distributed shared memory */
#define AMAMG_SMOOTHER_GRID    3     /* all phases in one cooperative launch, a grid barrier per phase */
#define AMAMG_SMOOTHER_OWNER   4     /* all phases in one cooperative launch of site-owning blocks */

/* The coarse Gauss-Seidel kernel (AMAMG_SMOOTHER_*) and owner-sweep shape
 * variant (0: the fixed rule; bits 0-1: early-sum lanes 8 (1) or 16 (2); bit
 * 2: twice the fewest sites per block) that a smoothing of level `level`
 * (1 .. nlevels-2, the smoothed coarse levels) with R right-hand sides in
 * `precision` (AMAMG_F64 / AMAMG_F32) uses now: the autotuner's pick where it
 * ran for that R, else the fixed rule.  Host-only; no GPU work. */
int amamg_query_smoother(amamg_handle h, int level, int precision, int R, int* kernel, int* variant);

/* e = M(r): one V-cycle of Algorithm 1 on the fine level with start vector 0,
 * no pre-smoothing and post_smooth sweeps per level. */
int amamg_vcycle(amamg_handle h, const void* r, void* e, int R, int precision, void* stream);

/* Size of the fixed device array behind amamg_vcycle_noalloc (8 MiB). */
#define AMAMG_NOALLOC_SCRATCH_BYTES (8u << 20)

/* amamg_vcycle without any device allocation.  The paper has no counterpart:
 * this exists for callers that cannot call cudaMalloc while they run (a host
 * callback, a region recorded for replay with fixed addresses, an application
 * whose memory pool forbids allocations after start-up).  Same arguments and
 * the same result as amamg_vcycle; the coarse-level work vectors live in one
 * file-scope __device__ array of AMAMG_NOALLOC_SCRATCH_BYTES that every GPU
 * loading the library holds until the process exits.
 *   - Needs 2 * R * 2 * (n_1 + ... + n_L) complex elements (r and e of every
 *     coarse level l >= 1, two spins per site, R right-hand sides; each level's
 *     vectors rounded up to 256 bytes); larger requests return
 *     AMAMG_ERR_INVALID_ARG with the sizes in amamg_last_error.
 *   - Like amamg_vcycle it does not report a time-out of a coarse smoother's
 *     bounded wait: follow it with amamg_sync_status where that matters (that
 *     call synchronises the stream and allocates nothing).
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress, with that device current); make that first call
 *     before any stream capture.
 *   - Every call on a device shares the one array and leaves its contents
 *     behind; nothing in it has to start at zero (each level's vectors are
 *     written before they are read).  Calls that overlap on the GPU (other
 *     streams, other handles) race on it: serialise them. */
int amamg_vcycle_noalloc(amamg_handle h, const void* r, void* e, int R, int precision, void* stream);

/* Reports (and clears) a time-out of a coarse smoother's bounded wait left by
 * any earlier call on this handle: synchronises the stream, reads the
 * handle's time-out flag, and when it is set re-arms the synchronisation
 * counters and returns AMAMG_ERR_TIMEOUT; else AMAMG_OK.  Allocates nothing. */
int amamg_sync_status(amamg_handle h, void* stream);

/* Self-test of the bounded waits of the coarse Gauss-Seidel owner sweep (the
 * kernel that runs coarse smoothing on most levels; its blocks wait only for
 * the blocks owning their sites' neighbours, each wait limited to about half a
 * second of polling).  Enqueues one two-sweep smoothing of coarse level l
 * (1 <= l < nlevels - 1) in `precision` on the handle's own zero work vectors
 * with one block that never publishes its phase counter, so its neighbours'
 * waits run out; like the other apply-style calls it does not report the
 * time-out itself: amamg_sync_status then returns AMAMG_ERR_TIMEOUT (the
 * expected outcome; the counters are re-armed and the handle stays usable).
 * Returns AMAMG_OK once enqueued, or AMAMG_ERR_INVALID_ARG when level l has no
 * owner sweep with two or more blocks.  Nothing else in the library uses this
 * path. */
int amamg_selftest_sync_timeout(amamg_handle h, int level, int precision, void* stream);

/* Integer structure of level l (host arrays; bit-exact tests):
 * role[Nt_l*Nx_l] (0 vertex, 1 edge, 2 interior), owner_tile[Nt_l*Nx_l]
 * (index p*(Nx_l/a)+q of the basket a site takes its formula from under the
 * handle's edge_owner rule; both computed on the device by the rule the
 * transfer kernels index with),
 * nbr_offsets[2*K] canonical (dt mod Nt_{l+1}, dx mod Nx_{l+1}) block offsets of
 * the level-(l+1) operator, lexicographically sorted, *nbr_count = K.
 * Arrays may be NULL to skip them; nbr_offsets must hold 2*48 ints. */
int amamg_export_structure(amamg_handle h, int level, int32_t* role, int32_t* owner_tile,
                           int32_t* nbr_offsets, int32_t* nbr_count);

/* Lattice extents and block-offset count of level l. */
int amamg_level_info(amamg_handle h, int level, int* Nt_l, int* Nx_l, int* n_offsets);

/* Copies level-l data to caller device buffers (complex128):
 * amamg_export_P: P_l tiles [nT][8][2(a^2-1)] (column 2c+beta = corner c of
 *   the tile's basket, c = 2 di + dj for corner (p+di, q+dj); row 2(l-1)+alpha
 *   for in-tile site l = i*a + j, l >= 1);
 * amamg_export_coarse: A_l blocks [K][4][n_l] (entry 2 alpha + beta) for l >= 1. */
int amamg_export_P(amamg_handle h, int level, void* out, void* stream);
int amamg_export_coarse(amamg_handle h, int level, void* out, void* stream);

/* Kernel timing for measurement: when enabled, every kernel the handle
 * launches is bracketed by CUDA events on its stream (and the solver's
 * Arnoldi steps run eagerly instead of as graphs).  amamg_profile_get
 * synchronises, then reports for kernel category idx (0..count-1) its name,
 * launches, summed device time, and the algorithmic bytes moved and
 * floating-point operations done (each input read once, each output written
 * once).  Returns AMAMG_ERR_INVALID_ARG past the last category. */
int amamg_profile_enable(amamg_handle h, int on);
/* Collects outstanding records and forgets every category. */
int amamg_profile_reset(amamg_handle h);
int amamg_profile_get(amamg_handle h, int idx, const char** name, long long* launches,
                      double* total_ms, double* bytes, double* flops);

/* Number of kernels the handle has launched since setup (all categories). */
long long amamg_launch_count(amamg_handle h);

/* Seconds of device time of the last amamg_setup (measured with events). */
double amamg_setup_seconds(amamg_handle h);

/* Synchronises the device and frees everything the handle owns (hierarchy,
 * solver workspace, graphs, streams); caller buffers are untouched.
 * AMAMG_ERR_INVALID_ARG for NULL. */
int amamg_destroy(amamg_handle h);
/* A static string naming an AMAMG_* status code. */
const char* amamg_status_string(int status);
/* The message of the last failure on h (empty when none), valid until the
 * next call on h; "null handle" for NULL. */
const char* amamg_last_error(amamg_handle h);

#ifdef __cplusplus
}
#endif
#endif /* AMAMG_H */
