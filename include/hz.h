/*
 * hz.h -- C ABI of the GB300 polarized-traces Helmholtz solver (online phase).
 *
 * Problem (paper's Formulation section, Eqs. 1 and 3-7): on an nx*ny*nz grid of
 * spacing h, solve  (Delta_h + omega^2 m) u = f  with absorbing PML pads obtained
 * by complex coordinate stretching d/dx -> beta(x) d/dx, beta = 1/(1 + i sigma/omega),
 * sigma quadratic in the pad (Eq. 5).  The discrete operator is used in its
 * complex-symmetric form A = S (Delta_h^stretched + omega^2 m), S = s_x s_y s_z,
 * s = 1/beta, and the system solved is  A u = S f.
 *
 * Method (SIE and polarized-traces sections, Algorithms 1-9): the domain is cut
 * into n_layers slabs along z, each padded with its own PML at internal faces;
 * every slab's local operator is factored once (Algorithm 1) by a multifrontal
 * nested-dissection LDL^T on the GPU; a solve (Algorithm 2) runs local solves,
 * forms the polarized trace right-hand side, runs GMRES on P M_pol (Eqs. 14-16)
 * whose every matrix-vector product is a set of multi-RHS local solves, and
 * rebuilds the volume with the Green's representation formula.
 *
 * Conventions for every entry point:
 *  - Grids are stored z-slowest, x-fastest: index (z*ny + y)*nx + x.
 *  - Complex arrays are interleaved (re, im) pairs of double (C99 double _Complex
 *    layout); a "complex array of length n" is 2n doubles.
 *  - Pointers documented "device" must be CUDA device (or managed) memory of the
 *    current device; "host" pointers are ordinary host memory (pinned memory is
 *    faster for the copies but not required).
 *  - Every call returns a status and never aborts, traps or exits; on failure
 *    hz_last_error() returns a one-line reason.  The handle owns every buffer it
 *    allocates; the caller owns every buffer it passes in.
 *  - All work is queued on the stream given to hz_create (0 = legacy default
 *    stream); calls are synchronous with respect to the host on return unless
 *    stated otherwise.  A handle must not be used from two host threads at once.
 */
#ifndef HZ_H
#define HZ_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    HZ_OK = 0,
    HZ_ERR_ARG = 1,            /* invalid argument (sizes, null pointers, omega <= 0, ...) */
    HZ_ERR_OOM = 2,            /* device memory exhausted (other allocation failures are HZ_ERR_CUDA) */
    HZ_ERR_ADMISSION = 3,      /* request does not fit in the free device memory */
    HZ_ERR_STATE = 4,          /* call out of order (e.g. solve before factor) */
    HZ_ERR_NONFINITE = 5,      /* NaN/Inf in m, rhs or a result */
    HZ_ERR_PIVOT = 6,          /* a pivot of the unpivoted LDL^T was tiny or non-finite */
    HZ_ERR_NO_CONVERGENCE = 7, /* GMRES / refinement hit its iteration cap; u and info still written */
    HZ_ERR_TIMEOUT = 8,        /* a bounded device-side wait gave up */
    HZ_ERR_CUDA = 9            /* a CUDA runtime call failed */
} hz_status;

typedef enum {
    HZ_PREC_FP64 = 0,  /* complex128 factors and local solves, FP64 GMRES */
    HZ_PREC_MIXED = 1, /* complex64 factors and local solves (FP64 pivot blocks), FP64 GMRES
                          on the traces, FP64 volume residual + defect correction */
    HZ_PREC_MIXED_FP64_FACTOR = 2  /* as HZ_PREC_MIXED online, but the offline factorization runs in
                          FP64 and its factors are rounded to complex64 (slower factorization,
                          more accurate local solves) */
} hz_precision;

typedef struct { int32_t nx, ny, nz; double h; } hz_grid;

/* npml: global pad thickness in nodes on every face (sigma measured from the first
 * physical node, delta = npml*h); C: profile strength of Eq. 5; npml_local: pad
 * thickness added at internal layer interfaces (<0 means npml). */
typedef struct { int32_t npml; double C; int32_t npml_local; } hz_pml;

typedef struct {
    double gmres_tol;    /* stop when ||P(f - M u)|| <= tol ||P f|| per column (default 1e-10 FP64, 1e-7 mixed);
                            in mixed mode this is the first pass's tolerance: each defect-correction
                            pass solves to 0.1 refine_tol / (its starting volume residual), capped at 0.1 */
    int32_t restart;     /* Krylov dimension before restart (default 12) */
    int32_t max_iter;    /* total GMRES iterations cap (default 100) */
    double refine_tol;   /* mixed mode: stop refining when ||S f - A u|| <= refine_tol ||S f|| (default 1e-9) */
    int32_t max_refine;  /* mixed mode: maximum defect-correction passes (default 3) */
    int32_t krylov;      /* Krylov solver on the trace system: 0 GMRES(restart) (default), 1 Bi-CGSTAB
                            (two products P M_pol per iteration, six trace vectors per column instead
                            of restart + 1; gmres_tol and max_iter apply to it as well) */
} hz_solve_opts;

typedef struct {
    int32_t iters;         /* GMRES iterations of the last pass */
    int32_t refinements;   /* defect-correction passes done (mixed mode) */
    double trace_relres;   /* final preconditioned relative residual estimate of GMRES */
    double volume_relres;  /* ||S f - A u|| / ||S f|| in FP64 (computed when refining or requested) */
    float ms_total;        /* device time of the whole call for this batch, milliseconds */
    int32_t iters_total;   /* Krylov iterations of all passes (the first solve and every correction) */
} hz_solve_info;

typedef struct hz_handle hz_handle;

/* Fills *opts with the defaults listed above for the given precision (the Krylov solve of Eq. 15;
 * the paper's experiments stop GMRES at a relative residual of 1e-7, Numerical Experiments section). */
void hz_default_opts(hz_precision prec, hz_solve_opts* opts);

/*
 * hz_create -- set up a problem (layered decomposition of the Formulation section,
 * Fig. 1 and Eq. 6; symbolic nested dissection of every distinct slab shape).
 *   grid      grid sizes (each >= 3) and spacing h > 0
 *   m         squared slowness, real, nz*ny*nx doubles, host or device (or managed) memory; copied
 *   omega     angular frequency > 0
 *   pml       PML parameters (see hz_pml)
 *   n_layers  number of slabs L, 1 <= L <= number of physical z planes
 *   prec      HZ_PREC_FP64, HZ_PREC_MIXED or HZ_PREC_MIXED_FP64_FACTOR
 *   stream    cudaStream_t to queue work on (0 for the default stream)
 *   out       receives the new handle (NULL on failure)
 * Errors: HZ_ERR_ARG, HZ_ERR_NONFINITE (m), HZ_ERR_OOM, HZ_ERR_CUDA.
 * Environment variables read here (they change speed, never the solution beyond rounding):
 *   HZ_SUBST_TC       complex64 substitutions on the tcgen05 kernel: 0 never, 1 always (for
 *                     column blocks of >= 64), 2 (default) when the autotuner times it faster
 *   HZ_TC_MIN_TILES   default minimum output tiles of a tensor-core product (8)
 *   HZ_PRECOND_SPLIT  1: single-term TF32 tensor-core products inside the preconditioner
 *                     (default 3 terms, FP32-level)
 *   HZ_TC_CFG=1       with HZ_AUTOTUNE=0: the persistent tensor-core kernel (one block per SM
 *                     walking the work items) instead of one block per work item (0)
 *   HZ_AUTOTUNE=0     keep the fixed defaults; HZ_GRAPHS=0 no CUDA-graph replay;
 *   HZ_LEAF           nested-dissection leaf size (cells, default 256)
 *   HZ_SPARSE         substitutions inside M_pol, the preconditioner and the polarized right-hand
 *                     side skip the products of subtrees that hold none of a layer's interface
 *                     planes (3, default: forward and backward; 2: backward only; 0: never)
 *   HZ_FACTOR_PROFILE=1  time every factorization launch by kernel kind (hz_factor_report)
 *   HZ_TC_WAIT_POLLS  poll limit of the tensor-core kernels' pipeline waits (default 2^26, and
 *                     2 s of wall time); a tiny value makes them give up at once, which a solve
 *                     reports as HZ_ERR_TIMEOUT (the blocks still drain their own copies and MMAs)
 *   HZ_FACTOR_TC_MIN  complex64 fronts with at least this many update unknowns (default 128)
 *                     compute L21 and their Schur complement on the tensor cores; 0: never
 */
hz_status hz_create(const hz_grid* grid, const double* m, double omega, const hz_pml* pml,
                    int32_t n_layers, hz_precision prec, void* stream, hz_handle** out);

/*
 * hz_create_ex -- hz_create for a heterogeneous density (the extension the paper's Introduction
 * names): the operator is div(b grad u) + omega^2 m u with b = 1/rho, discretized in the same
 * symmetric 7-point form with b at the half nodes (the average of the two nodes; the node itself
 * beyond the grid), so the structure, the method and the boundary are unchanged.
 *   b   1/rho, nz*ny*nx doubles, host or device memory, every entry finite and > 0; copied.  NULL gives
 *       b = 1 (exactly hz_create)
 * Other arguments and errors as hz_create, plus HZ_ERR_ARG for b <= 0 and HZ_ERR_NONFINITE for
 * a non-finite b.
 */
hz_status hz_create_ex(const hz_grid* grid, const double* m, const double* b, double omega, const hz_pml* pml,
                       int32_t n_layers, hz_precision prec, void* stream, hz_handle** out);

/*
 * hz_factor -- offline phase (Algorithm 1): assemble and factor every layer's
 * local operator H^l = L D L^T (complex symmetric, unpivoted, nested dissection,
 * FP64 diagonal pivot blocks), keeping the factors resident in device memory.  In mixed
 * precision the L21 and Schur-complement products of large fronts run on the tensor cores
 * (split-TF32, FP32 accumulation).
 * Errors: HZ_ERR_OOM, HZ_ERR_PIVOT, HZ_ERR_CUDA, HZ_ERR_TIMEOUT.
 */
hz_status hz_factor(hz_handle* h);

/*
 * hz_solve -- online phase (Algorithm 2) for R right-hand sides.
 *   rhs   device, complex array of R*nz*ny*nx: f for each right-hand side
 *   R     number of right-hand sides, >= 1
 *   u     device, complex array of R*nz*ny*nx, caller-owned, receives u
 *   opts  NULL for the defaults
 *   info  NULL or array of R entries, one per right-hand side (iters etc. of its column)
 * Errors: HZ_ERR_STATE (not factored), HZ_ERR_ARG, HZ_ERR_ADMISSION (workspace for R
 * does not fit), HZ_ERR_OOM, HZ_ERR_NONFINITE, HZ_ERR_NO_CONVERGENCE (u and info still written),
 * HZ_ERR_TIMEOUT (a tensor-core kernel's bounded wait gave up), HZ_ERR_CUDA.
 */
hz_status hz_solve(hz_handle* h, const double* rhs, int32_t R, double* u,
                   const hz_solve_opts* opts, hz_solve_info* info);

/*
 * hz_solve_group -- batched online phase for n independent problems of different sizes and
 * right-hand-side counts (one handle each, all factored).  Every member is solved as by
 * hz_solve on its own handle's stream, all members at once (one host thread per member), so
 * the device overlaps their launches; each member's GMRES matrix-vector product is replayed
 * as a CUDA graph.  Give every handle its own stream, otherwise the members serialise.
 *   hs        n distinct handles (a handle may appear once)
 *   rhs, u    per member: device complex [R[i]][nz][ny][nx] of that member's grid
 *   R         per member right-hand-side counts
 *   opts      NULL for each member's defaults
 *   info      NULL, or n pointers to arrays of R[i] entries (each may be NULL)
 *   statuses  NULL or n statuses
 * No counterpart in the paper's algorithms (it solves one problem at a time on a cluster): the
 * batching of uneven problems the single-GPU design adds.  Returns HZ_OK or the first member's
 * failure status.
 */
hz_status hz_solve_group(hz_handle* const* hs, int32_t n, const double* const* rhs, const int32_t* R,
                         double* const* u, const hz_solve_opts* opts, hz_solve_info* const* info,
                         hz_status* statuses);

/*
 * hz_solve_host -- as hz_solve (Algorithm 2) with HOST rhs and u: copies rhs to the device, solves,
 * copies u back (end-to-end entry point).  Same errors as hz_solve.  The device copies of the two
 * volumes (2 x R x nx*ny*nz complex128) are kept by the handle for later calls and released by
 * hz_destroy (or replaced when a later call has more right-hand sides); pinned host buffers
 * give the fastest copies.
 */
hz_status hz_solve_host(hz_handle* h, const double* rhs_host, int32_t R, double* u_host,
                        const hz_solve_opts* opts, hz_solve_info* info);

/*
 * hz_create_shared -- a second handle on an already factored problem: it borrows src's
 * resident factors and problem data (read-only) and gets its own solve workspaces, error flags
 * and stream, so that several solves of the same (model, omega) can run at once (one host
 * thread per handle).  src must stay alive until every handle created from it is destroyed.
 * No counterpart in the paper: the factors of Algorithm 1 shared by the serving workers.
 * Errors: HZ_ERR_ARG, HZ_ERR_STATE (src not factored), HZ_ERR_OOM, HZ_ERR_CUDA.
 */
hz_status hz_create_shared(hz_handle* src, void* stream, hz_handle** out);

/* hz_destroy -- frees every device and host buffer the handle owns (NULL is allowed).  No
 * counterpart in the paper (resource management). */
hz_status hz_destroy(hz_handle* h);

/* One-line description of the last failure on this handle ("" if none); the string
 * stays valid until the next call on the handle.  h may be NULL (reports failures of
 * hz_create and hz_symbolic_shape).  No counterpart in the paper (error reporting). */
const char* hz_last_error(const hz_handle* h);

/* ------------------------------------------------------------------------------------
 * Introspection and stage-level entry points.  Each runs one step of the online path
 * on the device so that it can be checked on its own; none is needed for a solve.
 * ------------------------------------------------------------------------------------ */

/* Layer geometry of the layered decomposition (Formulation section, Fig. 1 and Eq. 6): owned
 * global planes [lo, hi] and extended local grid [zlo, zhi] of layer ell (0-based). */
hz_status hz_layer_info(const hz_handle* h, int32_t ell, int32_t* lo, int32_t* hi,
                        int32_t* zlo, int32_t* zhi);

/* Statistics of the factorization of Algorithm 1 (the multifrontal solver of the Local Solves
 * section; its cost model is in the Complexity of Polarized Traces section): number of tree nodes, stored
 * factor entries (padded tiles, summed over layers), factorization flops (real),
 * front workspace bytes, and the time hz_factor took in milliseconds. */
hz_status hz_factor_stats(const hz_handle* h, int64_t* nodes, int64_t* factor_entries,
                          double* factor_flops, int64_t* workspace_bytes, float* factor_ms);

/* Cost of one local solve (the substitutions of the Local Solves section): bytes of packed
 * factors streamed by one forward+backward substitution of layer ell
 * (each factor tile read once forward, once backward), and its real flop count per
 * right-hand-side column. */
hz_status hz_layer_solve_cost(const hz_handle* h, int32_t ell, double* bytes, double* flops_per_col);

/*
 * Local solve (Algorithm 2, its local solves): w = (H^ell)^{-1} g for ncols
 * columns on layer ell's extended local grid of nzl = zhi-zlo+1 planes.
 *   g, w  device, complex arrays [ncols][nzl][ny][nx] (natural local order)
 */
hz_status hz_layer_solve(hz_handle* h, int32_t ell, const double* g, int32_t ncols, double* w);

/*
 * Polarized right-hand side (Algorithm 2, local solves + forming the trace rhs):
 *   rhs   device complex [R][nz][ny][nx], f (scaled by S inside)
 *   fpol  device complex [R][2][K][2][ny][nx]: (down, up) x interface j x (P_j, Q_j) planes
 * K = n_layers - 1.
 */
hz_status hz_polarized_rhs(hz_handle* h, const double* rhs, int32_t R, double* fpol);

/* y = M_pol x (appendix, Application Polarized: Algorithms 6-9), x and y device
 * complex [R][2][K][2][ny][nx]. */
hz_status hz_apply_mpol(hz_handle* h, const double* x, int32_t R, double* y);

/* y = P x, the Gauss-Seidel preconditioner of Eq. 16 (Algorithms 4-6), same layout. */
hz_status hz_apply_precond(hz_handle* h, const double* x, int32_t R, double* y);

/*
 * hz_symbolic_shape -- the symbolic phase that hz_create runs for every distinct slab shape,
 * on its own: the nested-dissection reordering of the Local Solves section, here geometric
 * (recursive bisection of the box by one-cell planes down to leaf boxes of at most `leaf`
 * cells), with every tree node's own unknowns and update set.  Host code only: needs no GPU.
 *   nx, ny, nz  box sizes (>= 1, at most 2^30 cells); leaf: largest leaf box in cells (>= 1)
 *   n_nodes, n_upd   receive the node count and the total length of the update sets
 *   perm        int32[nx*ny*nz] or NULL: elimination index -> natural cell (z*ny + y)*nx + x
 *   own0, nown, parent   int32[n_nodes] or NULL: node k owns elimination indices
 *               [own0[k], own0[k] + nown[k]); parent[k] = -1 at the root; nodes are in
 *               post-order (children before parents), so a subtree's unknowns are contiguous
 *   upd_off     int64[n_nodes] or NULL, upd_idx int32[n_upd] or NULL: node k's update set is
 *               upd_idx[upd_off[k] .. upd_off[k] + (its length)), sorted elimination indices;
 *               lengths follow from upd_off and n_upd in node order
 * Call once with NULL arrays for the counts, then with caller-owned arrays of those sizes.
 * Errors: HZ_ERR_ARG (sizes), HZ_ERR_OOM (host memory); hz_last_error(NULL) explains.
 */
hz_status hz_symbolic_shape(int32_t nx, int32_t ny, int32_t nz, int32_t leaf, int64_t* n_nodes, int64_t* n_upd,
                            int32_t* perm, int32_t* own0, int32_t* nown, int32_t* parent, int64_t* upd_off,
                            int32_t* upd_idx);

/*
 * hz_trace_blocks -- explicit trace-to-trace Green's blocks.  The paper applies the blocks of the SIE
 * and polarized matrices only matrix-free, by local solves with interface sources (Reduction to a
 * surface integral equation section, Algorithms 4-9: in 3D the matrix is never formed), and cites
 * selective inversion (Local Solves section) for trading factor storage for dense products; this
 * entry point takes that trade one step further on problems small enough for it.  For every
 * layer it computes the dense 2P x 2P blocks E_rs (P = nx*ny) taking a trace pair on the layer's
 * top or bottom interface s, through that interface's source, to the layer's top or bottom
 * read-out pair r: 4L - 6 blocks, one local solve per unit source trace, in the precision of the
 * handle's local solves (complex64 in the mixed modes, complex128 in FP64).  M_pol and the
 * preconditioner (hz_apply_mpol, hz_apply_precond and every Krylov iteration of hz_solve) then
 * apply block products instead of local solves whenever the call has at most max_cols columns;
 * the right-hand side preparation and the reconstruction keep their local solves.
 *   max_cols  > 0: build the blocks (once per factorization) and use them up to this many
 *             columns; 0: release them and return to the local solves everywhere
 *   bytes     may be NULL; receives the device bytes the blocks hold
 * The blocks are owned by the handle (released by hz_destroy, by hz_trace_blocks(h, 0, ...), and by
 * hz_factor, after which they must be built again); handles from hz_create_shared have their own.
 * Memory: (4L - 6) * 4 P^2 complex elements, 14.0 GB at 64^3 with 8 layers in complex64 -- the
 * blocks pay where layers are thin and right-hand sides few; at 128^3 they do not fit.
 * Errors: HZ_ERR_ARG (max_cols < 0), HZ_ERR_STATE (not factored), HZ_ERR_OOM / HZ_ERR_ADMISSION
 * (blocks or the build's workspace do not fit; the handle is left without blocks), HZ_ERR_CUDA.
 */
hz_status hz_trace_blocks(hz_handle* h, int32_t max_cols, int64_t* bytes);

/* Reconstruction (Algorithm 2, inner solves): u from f and the traces t = u_down + u_up,
 * t device complex [R][K][2][ny][nx]; u device complex [R][nz][ny][nx]. */
hz_status hz_reconstruct(hz_handle* h, const double* rhs, const double* t, int32_t R, double* u);

/* FP64 volume residual r = S f - A u of the global discrete system (Formulation section: the
 * 7-point stencil with the stretched PML) and its per-column relative norms ||r|| / ||S f||; r may
 * be NULL.  The mixed precision's defect correction uses it; the paper (FP64 throughout) has none. */
hz_status hz_volume_residual(hz_handle* h, const double* rhs, const double* u, int32_t R,
                             double* r, double* relres_host);

/* ------------------------------------------------------------------------------------
 * Measurement (no counterpart in the paper, which reports wall-clock times per stage in the
 * tables of its Numerical Experiments section).  hz_profile_begin starts recording CUDA events around every batched
 * forward+backward substitution (the kernel family that dominates the online phase);
 * hz_profile_end synchronizes the handle's stream and returns the number of recorded
 * substitution calls, their summed device time in ms, and the summed algorithmic factor
 * bytes (each stored factor entry read once forward and once backward) and real flops.
 * hz_profile_begin_detail does the same and also records events around every kernel launch
 * of those substitutions; hz_profile_kernel then returns, per kernel kind, the launches, their
 * summed device time in ms and their algorithmic factor bytes and real flops over the interval
 * closed by the last hz_profile_end (kind 0: CUDA-core substitution kernels, 1: tensor-core
 * kernel, 2: the explicit trace-block products of hz_trace_blocks, whose bytes are the block
 * entries each launch reads and whose flops are 8 per entry and column; any other kind is
 * HZ_ERR_ARG).  Detail mode adds an event pair per launch and
 * replaces CUDA-graph replay by direct launches: profile an interval apart from timed runs.
 * hz_kernel_launches returns the number of kernels the library has launched in this
 * process (all handles).
 * ------------------------------------------------------------------------------------ */
/*
 * hz_volume_residual_noalloc -- the FP64 volume residual of hz_volume_residual computed
 * without allocating any memory during the call.  It has no counterpart in the paper.  It is
 * for callers that cannot allocate device memory where they need the residual: a process whose
 * device memory is all held by a caching allocator (a cudaMalloc there fails, or forces the
 * allocator to release its cache with a device-wide synchronisation), or a serving loop that
 * must keep a fixed memory footprint per request.  The per-column sums the kernel needs live
 * in a fixed device array inside the library instead of a buffer allocated per call; only
 * buffers the handle already owns and the caller's arrays are used.
 *   rhs, u     device complex [R][nz][ny][nx] (f, unscaled; and the candidate solution)
 *   R          1 <= R <= 1024 (the fixed scratch holds 1024 columns, 16 KiB per device); larger R
 *              returns HZ_ERR_ARG with a message saying so
 *   r          device complex [R][nz][ny][nx] receiving S f - A u, or NULL
 *   relres_host  host double[R] receiving ||S f - A u|| / ||S f||
 * The call runs on the handle's device and stream, copies the sums to the host and
 * synchronizes that stream before it returns.  The first call on a device looks up the device
 * address of the fixed array (set-up); make that first call before any stream capture.  All
 * calls in the process share the array, which keeps the last call's sums (each call clears the
 * columns it uses): calls that overlap on the GPU (different streams or threads at once) race
 * on it.
 */
hz_status hz_volume_residual_noalloc(hz_handle* h, const double* rhs, const double* u, int32_t R, double* r,
                                     double* relres_host);

/*
 * hz_tensor_peak -- measures the tensor pipe's dense MMA rate on the current device (no
 * counterpart in the paper; it is the denominator of the tensor-core kernels' roofline).
 * One block per SM issues tcgen05 MMAs (M = 128, N = n, one instruction's K) from operands
 * resident in shared memory, with no global-memory traffic, for about `seconds` seconds.
 *   kind     0: kind::tf32 (tf32 x tf32 -> f32, K = 8); 1: kind::f16 with bf16 operands (K = 16);
 *            2: kind::tf32 with the A operand read from tensor memory instead of shared memory
 *   n        64, 128 or 256
 *   seconds  0 < seconds <= 30
 *   tflops   receives 2*128*n*K flops per MMA x MMAs / time, in TFLOP/s
 *   ms       NULL or receives the measured run's device time
 * Errors: HZ_ERR_ARG, HZ_ERR_OOM, HZ_ERR_CUDA, HZ_ERR_TIMEOUT (the bounded completion wait gave up).
 */
hz_status hz_tensor_peak(int32_t kind, int32_t n, double seconds, double* tflops, double* ms);

hz_status hz_profile_begin(hz_handle* h);
hz_status hz_profile_begin_detail(hz_handle* h);
hz_status hz_profile_end(hz_handle* h, int64_t* calls, double* total_ms, double* alg_bytes, double* alg_flops);
hz_status hz_profile_kernel(hz_handle* h, int32_t kind, int64_t* launches, double* total_ms, double* alg_bytes,
                            double* alg_flops);
int64_t hz_kernel_launches(void);

/* Text table of the last detail-profiled interval (hz_profile_begin_detail .. hz_profile_end):
 * one line per kernel kind, substitution phase (FA, FB, BA, BB) and tree level with its launches,
 * work items (tasks, before the split into column chunks), summed device ms and algorithmic
 * TFLOP/s.  The string stays valid until the next call on the handle.  No counterpart in the paper. */
const char* hz_profile_report(hz_handle* h);

/* Per-kernel-kind device time of the last hz_factor on this handle (one line per kind: launch
 * groups timed and summed ms), recorded only when the environment variable HZ_FACTOR_PROFILE=1
 * was set at hz_create ("" otherwise; the event pairs serialise nothing but add host work).  The
 * string stays valid until the next hz_factor on the handle.  No counterpart in the paper. */
const char* hz_factor_report(hz_handle* h);

/* The substitution autotuner's record for this handle: one line per tuned batch signature
 * (layer shapes and column width) with the time of every candidate split-K depth and column
 * chunk and the choice made.  The autotuner runs the first time a signature is solved (set the
 * environment variable HZ_AUTOTUNE=0 before hz_create to keep the fixed defaults).  The string
 * stays valid until the next call on the handle.  No counterpart in the paper. */
const char* hz_tuning_report(hz_handle* h);

#ifdef __cplusplus
}
#endif
#endif /* HZ_H */
