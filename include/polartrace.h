/*
 * polartrace.h - C ABI of the GB300 (sm_103a) implementation of the method of
 * polarized traces for the 2D Helmholtz equation (Zepeda-Nunez & Demanet,
 * "The method of polarized traces for the 2D Helmholtz equation", 2014).
 *
 * Problem statement (Section 2.1): find u on the extended grid
 * (n_x + 2 n_pml) x (n_z + 2 n_pml) with
 *     -alpha_x d_x(alpha_x d_x u) - alpha_z d_z(alpha_z d_z u) - omega^2 u / c^2 = f,
 * 5-point finite differences of step h, PML profile sigma = (C/delta)(d/delta)^2
 * (delta = n_pml h) and homogeneous Dirichlet data one node outside the grid.
 * The z axis is split into L layers (Section 2.2); the online solve
 * (Algorithm 2) forms the interface right-hand side by local solves, solves
 * the polarized jump system (Definition 9) by GMRES preconditioned with
 * Algorithm 4, and rebuilds the volume field by local solves.
 *
 * Conventions for every entry point:
 *  - Every function returns pt_status; none aborts, throws or exits.
 *  - "device" pointers are CUDA global-memory addresses on the current
 *    device; "host" pointers are ordinary CPU memory.  The caller owns every
 *    buffer; the library keeps device pointers only between pt_create and
 *    pt_destroy and never allocates device memory (scratch comes from the
 *    caller through the workspace arguments).
 *  - Complex numbers are pt_c128 {re, im} (16 bytes, interleaved).
 *  - Volume arrays are row-major [z][x] on the extended grid (x fastest):
 *    element (p, q) of the paper (p, q = -n_pml+1 .. n+n_pml) sits at index
 *    (q + n_pml - 1) * n_t + (p + n_pml - 1), n_t = n_x + 2 n_pml,
 *    N_z = n_z + 2 n_pml.  Several sources are stacked as [source][z][x].
 *  - Interface traces are laid out [source][dir][interface][trace][x]:
 *    dir 0 = down-going, 1 = up-going (Section 3.2); interface i = 0..L-2
 *    lies between layers i and i+1 (0-based); trace 0 is the last row of
 *    layer i (u^i_n = u^{i+1}_0), trace 1 the first row of layer i+1
 *    (u^i_{n+1} = u^{i+1}_1); x runs over n_t columns.
 *  - All device work is ordered on the stream given to pt_create.
 *    pt_solve and pt_solve_host synchronise that stream once per GMRES
 *    iteration to read the residual estimate and return only when done.
 */
#ifndef POLARTRACE_H
#define POLARTRACE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pt_ctx pt_ctx;

typedef struct {
  double re, im;
} pt_c128;

typedef enum {
  PT_OK = 0,
  PT_ERR_ARG = 1,           /* invalid argument; nothing was launched          */
  PT_ERR_WORKSPACE = 2,     /* a workspace / scratch buffer is too small        */
  PT_ERR_CUDA = 3,          /* a CUDA runtime call failed                       */
  PT_ERR_SINGULAR = 4,      /* zero pivot in a local factorization              */
  PT_ERR_NOT_CONVERGED = 5, /* GMRES hit max_it; outputs hold the best iterate  */
  PT_ERR_TIMEOUT = 6,       /* a bounded device-side wait gave up               */
  PT_ERR_NUMERIC = 7        /* NaN/Inf met in the data                          */
} pt_status;

typedef enum {
  PT_FP64 = 0,       /* every block product in FP64                                  */
  PT_MIXED_FP32 = 1, /* preconditioner (Algorithm 4) applies FP32 copies of the
                        blocks (FP16 ones by option); the GMRES
                        matvec runs in double-float (FP32 pairs, ~1e-14); local
                        solves (right-hand side, reconstruction) in
                        FP32 with the FP64 factors rounded to complex64, chunked
                        along x (~1e-6 on the field; PT_OPT_LOCAL_SOLVE = 1
                        selects double-float);
                        the explicit residual between restart cycles in double-float;
                        Arnoldi and least squares in FP64 (flexible GMRES).  With
                        compressed blocks (plr) the products are FP64 instead of
                        double-float.                                               */
  PT_MIXED_TC = 2    /* for batches of sources: the block products run on the tensor
                        cores with FP16 operands (power-of-two scales) and FP32
                        accumulation - one pass in the preconditioner, the three-pass
                        hi/lo split (~1e-5) in the GMRES matvec; the explicit residual
                        between restart cycles is double-float (iterative refinement);
                        local solves (right-hand side, reconstruction) in FP32 with
                        the FP64 factors rounded to complex64, batched over groups
                        of sources; Arnoldi and least squares in FP64.
                        pt_volume_residual gives an FP64 check.                   */
} pt_precision;

typedef struct {
  int32_t nx, nz;   /* interior grid points (Section 2.1)                          */
  int32_t npml;     /* PML points on each side, n_pml = delta / h                   */
  int32_t L;        /* number of layers (Section 2.2)                               */
  double h;         /* grid step                                                    */
  double omega;     /* angular frequency                                            */
  double pml_C;     /* PML strength C of sigma = (C/delta)(d/delta)^2               */
  int32_t precision;  /* pt_precision                                               */
  int32_t gs_iters;   /* n_it of Algorithm 4 (the paper uses 2)                      */
  int32_t max_sources;/* largest nsrc a pt_solve call may use                       */
  int32_t max_krylov; /* largest GMRES iteration count a pt_solve call may use      */
  int32_t plr;        /* 1: compress the interface blocks to partitioned low rank
                         (Section 5.1, Algorithm 5) and apply them in the GMRES matvec
                         and the preconditioner; 0: dense blocks                     */
  double plr_eps;     /* relative threshold: a node is a leaf when sigma_{r_max+1}
                         < plr_eps * sigma_1 of its whole block                      */
  int32_t plr_rmax;   /* r_max, 1 .. 31                                              */
  int32_t learned;    /* 1: reserve the solve-scratch buffers of the learned
                         preconditioner correction (pt_set_correction,
                         PT_OPT_LEARNED); 0: none                                    */
  const int32_t* layer_rows; /* host, L ints or NULL.  The rows n^l of each layer (Section
                         2.2 allows any increasing sequence of interfaces): layer l
                         covers the extended-grid rows row_start[l] ..
                         row_start[l] + n^l - 1, the sum must be N_z = nz + 2 npml,
                         every n^l >= 3, and no interface may lie in or next to the
                         PML (npml + 1 <= row_start[l] <= N_z - npml - 1 for l >= 1).
                         NULL: the near-equal split of pt_layer_partition.  Read
                         only during the call it is passed to (pt_create copies
                         the partition).                                             */
} pt_params;

/* Layer partition used by the library (Section 2.2): layer_rows when given,
 * otherwise the near-equal split in which the first (N_z mod L) layers get
 * one extra row.  row_start must hold L+1 ints (host); on return
 * row_start[l] is the first extended-grid row of layer l and row_start[L] = N_z.
 * Fails with PT_ERR_ARG when an interface would lie within one row of the
 * PML or a layer would have fewer than 3 rows. */
pt_status pt_layer_partition(const pt_params* prm, int32_t* row_start);

/* Device memory the caller must provide (bytes, host outputs):
 *   persistent_bytes : kept from pt_create to pt_destroy (local factors,
 *                      interface Green's matrices, tables);
 *   setup_bytes      : temporary, used only inside pt_create;
 *   solve_bytes      : scratch for one pt_solve call with max_sources sources
 *                      and max_krylov iterations.
 * Any output pointer may be NULL. */
pt_status pt_workspace_size(const pt_params* prm, size_t* persistent_bytes, size_t* setup_bytes,
                            size_t* solve_bytes);

/* Offline phase (Algorithm 1) on the GPU, in FP64: assembles every local
 * problem H^l (Section 2.2, padded PML, normal extension of m = 1/c^2),
 * factors it along x by block elimination with pivoted Gauss-Jordan
 * inversion of the Schur complements, and extracts the interface Green's
 * matrices G^l(z_j, z_k), j, k in {0, 1, n, n+1} (Definition 1) by solves
 * with identity columns.
 *   c_ext      device, N_z * n_t doubles, wave speed c > 0 on the extended grid
 *   persistent device, >= persistent_bytes, 256-byte aligned
 *   setup      device, >= setup_bytes, 256-byte aligned (free after return)
 *   stream     cudaStream_t (may be NULL for the legacy default stream)
 *   out        host, receives the context
 * Errors: PT_ERR_ARG (sizes, partition, h/omega/C not positive, alignment),
 * PT_ERR_WORKSPACE, PT_ERR_NUMERIC (c not finite or not positive),
 * PT_ERR_SINGULAR (zero pivot), PT_ERR_CUDA.  Blocks until done. */
pt_status pt_create(const pt_params* prm, const double* c_ext, void* persistent, size_t persistent_bytes,
                    void* setup, size_t setup_bytes, void* stream, pt_ctx** out);

/* Online phase (Algorithm 2) for nsrc right-hand sides, all device pointers:
 *   f        device, nsrc * N_z * n_t pt_c128 sources
 *   u        device, nsrc * N_z * n_t pt_c128 volume field out (NULL: skip
 *            the reconstruction step)
 *   traces   device, nsrc * 4 (L-1) n_t pt_c128 polarized traces out (NULL: skip)
 *   rel_tol  GMRES stops when the flexible GMRES least-squares estimate is
 *            <= rel_tol * ||P b|| and the explicit FP64 residual confirms it
 *   max_it   <= max_krylov
 *   scratch  device, >= solve_bytes
 *   iters    host, nsrc ints: GMRES iterations per source (may be NULL)
 *   relres   host, nsrc doubles: true relative residual of the polarized
 *            system per source (may be NULL)
 * Returns PT_ERR_NOT_CONVERGED (with outputs written) when some source did
 * not reach rel_tol within max_it iterations. */
pt_status pt_solve(pt_ctx* ctx, int32_t nsrc, const pt_c128* f, pt_c128* u, pt_c128* traces, double rel_tol,
                   int32_t max_it, void* scratch, size_t scratch_bytes, int32_t* iters, double* relres);

/* Gauss-Seidel iteration used as a solver (Algorithm 3, Section 4.1) on the
 * permuted polarized jump system:  u^0 = 0,
 *     u^{k+1} = D^{-1} (P b - R u^k),
 * stopping when ||u^{k+1} - u^k|| / ||u^k|| <= rel_tol for every source (the
 * test of Algorithm 3, per source) or after max_it iterations; then the
 * volume field is reconstructed as in pt_solve (Algorithm 2).  The sweeps
 * D^{-1} and the coupling R use the exact FP64 blocks in every precision
 * form.  Arguments and layouts are those of pt_solve; iters[s] counts the
 * iterations, relres[s] is the FP64 true relative residual
 * ||P b - P M u|| / ||P b||.  max_it is not limited by max_krylov.
 * Returns PT_ERR_NOT_CONVERGED (outputs written) when some source did not
 * meet the test within max_it iterations; the iteration's convergence
 * depends on the spectral radius of D^{-1} R (Section 4.2), which exceeds 1
 * in some media, where only preconditioned GMRES (pt_solve) converges. */
pt_status pt_solve_gs(pt_ctx* ctx, int32_t nsrc, const pt_c128* f, pt_c128* u, pt_c128* traces, double rel_tol,
                      int32_t max_it, void* scratch, size_t scratch_bytes, int32_t* iters, double* relres);

/* Same as pt_solve with f and u in HOST memory (pinned memory gives the best
 * copy rate); the library copies them through the scratch buffer, whose size
 * must be >= solve_bytes + 2 * nsrc * N_z * n_t * 16 bytes. */
pt_status pt_solve_host(pt_ctx* ctx, int32_t nsrc, const pt_c128* f_host, pt_c128* u_host, double rel_tol,
                        int32_t max_it, void* scratch, size_t scratch_bytes, int32_t* iters, double* relres);

/* Building blocks of the online phase, exposed for testing and composition.
 * All pointers device; x, y hold nsrc polarized-trace vectors in the layout
 * above.  Each applies the FP64 blocks.
 *   pt_apply_matvec       y = P M x  (Definition 9, permuted: D + R)
 *   pt_apply_precond      y = Algorithm 4 applied to the permuted residual x
 *                         (n_it = gs_iters; uses the context's precision)
 *   pt_apply_D_inverse    y = D^{-1} x (the two sweeps of Section 4.1)
 *   pt_apply_R            y = R x
 *   pt_rhs                y = P b, b = (-f, -f_0) from the local Newton
 *                         potentials of f (device, nsrc * N_z * n_t)
 * scratch >= solve_bytes. */
pt_status pt_apply_matvec(pt_ctx* ctx, int32_t nsrc, const pt_c128* x, pt_c128* y);
pt_status pt_apply_precond(pt_ctx* ctx, int32_t nsrc, const pt_c128* x, pt_c128* y, void* scratch,
                           size_t scratch_bytes);
pt_status pt_apply_D_inverse(pt_ctx* ctx, int32_t nsrc, const pt_c128* x, pt_c128* y);
pt_status pt_apply_R(pt_ctx* ctx, int32_t nsrc, const pt_c128* x, pt_c128* y);
pt_status pt_rhs(pt_ctx* ctx, int32_t nsrc, const pt_c128* f, pt_c128* y, void* scratch, size_t scratch_bytes);

/* pt_rhs_noalloc: the same result as pt_rhs (y = P b for nsrc sources; f and
 * y device, same layouts) for callers that cannot allocate device memory at
 * all, not even the scratch buffer that pt_rhs takes as an argument.  Such
 * callers are, for example, code running inside a host framework whose pool
 * owns every device allocation and hands out none, or a serving loop that
 * must not call cudaMalloc after start-up because the call can synchronise
 * the device and stall work on other streams.  The paper has no counterpart:
 * this is an interface convenience, not part of the method.
 *   Scratch: the local-solve storage lives in one 16 MiB array in the
 *   library's own device memory (loaded with the library, held by every GPU
 *   that loads it until the process exits).  A call needs
 *   nsrc * L * n_t * nloc_max * 16 bytes (rounded up to 256) plus
 *   nsrc * L * 4 bytes, nloc_max = the largest layer height + 2 n_pml;
 *   larger requests fail with PT_ERR_WORKSPACE and nothing is launched
 *   (use pt_rhs then).  No call allocates (no cudaMalloc, cudaFree or any
 *   allocating library routine).
 *   Set-up: the first call on a device, with that device current, looks up
 *   the array's device address once (cudaGetSymbolAddress) and caches it;
 *   make that first call before any stream capture.  The device current at
 *   every call must be the one the context was created on; otherwise the
 *   call returns PT_ERR_ARG before any lookup or launch.
 *   Sharing: every call uses the same array and leaves its contents behind;
 *   a call writes every byte it reads, so nothing needs clearing, but calls
 *   that overlap on the GPU (other streams, other threads) race on the array.
 *   The call returns after its work on the context's stream has finished. */
pt_status pt_rhs_noalloc(pt_ctx* ctx, int32_t nsrc, const pt_c128* f, pt_c128* y);

/* One operator of the permuted polarized jump system in the representation
 * the solver works with.  which: 0 = P M (Definition 9), 1 = R, 2 = D^{-1}
 * (the sweeps of Section 4.1).  working = 0: dense FP64 blocks (the exact
 * operator, as pt_apply_matvec / pt_apply_R / pt_apply_D_inverse);
 * working = 1: what pt_solve uses for it - the partitioned low-rank blocks
 * when the context compresses (plr = 1), FP32 blocks for R and D^{-1} in the
 * mixed precision, double-float for P M in the mixed precision.  which = 3:
 * P M in the arithmetic of the explicit residual that pt_solve forms between
 * restart cycles (double-float in the mixed forms with dense blocks, FP64
 * otherwise; working is ignored).  x and y are device trace vectors (nsrc of
 * them), scratch >= solve_bytes. */
pt_status pt_apply(pt_ctx* ctx, int32_t which, int32_t working, int32_t nsrc, const pt_c128* x, pt_c128* y,
                   void* scratch, size_t scratch_bytes);

/* FP64 residual of the discrete Helmholtz equation of Section 2.1 on the
 * whole extended grid: relres[s] = ||f_s - H u_s||_2 / ||f_s||_2 for nsrc
 * volume fields u (device, layout of pt_solve's u) and sources f (device);
 * relres host, nsrc doubles; scratch >= solve_bytes.  This is the check that
 * does not depend on how the interface system was solved. */
pt_status pt_volume_residual(pt_ctx* ctx, int32_t nsrc, const pt_c128* f, const pt_c128* u, double* relres,
                             void* scratch, size_t scratch_bytes);

/* Size of the partitioned low-rank representation built by pt_create with
 * plr = 1 (Algorithm 5): complex entries stored (dense leaves count m n,
 * low-rank leaves r (m + n)) and number of leaves, both host outputs (NULL
 * allowed).  Zero when the context keeps dense blocks. */
pt_status pt_plr_stats(const pt_ctx* ctx, int64_t* stored_entries, int32_t* leaves);

/* Tuning options of a context (they change speed, not results beyond
 * rounding).  PT_OPT_LAYER_GROUP: sources per CTA of the source-batched
 * local solves of PT_MIXED_TC (Algorithm 2 and the reconstruction of
 * Section 2.3): 0 = chosen from L and nsrc (default), or 8, 16, 32.
 * PT_OPT_LEARNED: 1 = flexible GMRES adds the learned correction to the
 * preconditioner (needs learned = 1 at pt_create and weights, see below),
 * 0 = plain Algorithm 4 (default).
 * PT_OPT_LOCAL_SOLVE: local solves of PT_MIXED_FP32 - 4 = FP32, each layer's
 * columns cut into chunks solved in parallel, one CTA per (layer, chunk,
 * source): every chunk from zero boundary values, then the boundary values
 * from chunk-transfer matrices formed at pt_create (FP64, kept in complex64),
 * then every chunk again from its boundary values (default, ~1e-6 on the
 * field); 0 = FP32 on a cluster of 4 CTAs per (layer, source), each CTA
 * holding a quarter of the rows of the next column's factors in shared
 * memory; 3 = the same on 8 CTAs; 2 = FP32 on one CTA; 1 = double-float on
 * clusters of 4 CTAs (~1e-13, slower).
 * PT_OPT_SWEEP: the sweeps D^{-1} of the PT_MIXED_FP32 preconditioner -
 * 0 = all L-1 steps of a sweep in one cooperative launch with a grid barrier
 * between steps (default; used when the shape fits its register and shared-
 * memory bounds, and never inside pt_solve_many, whose contexts share the
 * GPU); 1 = one launch per step.  Both give the same products.
 * PT_OPT_RELAX: GMRES matvecs of PT_MIXED_FP32 - 1 = inexact Krylov
 * relaxation (default): once the residual estimate of every active source
 * is below 1e4 rel_tol ||b||, the matvec uses the FP32 blocks instead of the
 * double-float ones (the residual gap this opens stays about 1e-2 rel_tol
 * ||b||; the restart residual is always double-float); 0 = double-float
 * matvecs throughout.
 * PT_OPT_PRECOND_FP16: block products of the PT_MIXED_FP32 preconditioner
 * (Algorithm 4: the sweeps D^{-1} and R) - 0 = the complex64 copies (default,
 * about 1e-7); 1 = FP16 copies of the blocks, each block row scaled by a
 * power of two into FP16 range (plr = 0 only; about 5e-4 relative on the
 * preconditioner's output: half the bytes of every sweep step and R apply,
 * sometimes one more GMRES iteration).
 * PT_OPT_RESTART: the explicit residual P b - P M x that PT_MIXED_TC forms
 * between restart cycles (iterative refinement) - 1 = split products on the
 * tensor cores (default): blocks and inputs cut into five 7-bit integer
 * slices held exactly in FP16 (Ozaki et al.'s error-free splitting), the 15
 * slice pairs of weight >= 2^-42 accumulated exactly in FP32 over K segments
 * of 512 and summed in double-float, ~1e-10 relative to the largest block
 * entry of a row times the largest input entry of a source; 0 = the
 * double-float product on the FP32 pipes (~1e-14).
 * PT_ERR_ARG for an unknown option or value. */
enum {
  PT_OPT_LAYER_GROUP = 1,
  PT_OPT_LEARNED = 2,
  PT_OPT_LOCAL_SOLVE = 3,
  PT_OPT_SWEEP = 4,
  PT_OPT_RELAX = 5,
  PT_OPT_PRECOND_FP16 = 6,
  PT_OPT_RESTART = 7
};
pt_status pt_set_option(pt_ctx* ctx, int32_t option, int32_t value);

/* ---- learned preconditioner correction (not in the paper) ------------------
 * A network N_theta on interface traces corrects the Gauss-Seidel
 * preconditioner K^{-1} of Algorithm 4 inside flexible GMRES (Section 4.2):
 * z = K^{-1} v + N_theta(v).  For one source, v (a permuted residual, the
 * vectors GMRES preconditions) is divided by its RMS s; each interface i
 * gives one sequence of n_t positions with 8 channels, Re/Im of the rows
 * 2i, 2i+1, T+2i, T+2i+1 (T = 2(L-1)); the network is
 *   h1 = b1 + W1 * x   (1D cross-correlation over x, kernel 7, zero padding, 8 -> 256)
 *   h2 = b2 + W2 g(h1), h3 = b3 + W3 g(h2), y = b4 + W4 g(h3)
 * with g(x) = x/2 (1 + tanh(sqrt(2/pi)(x + 0.044715 x^3))); y (8 channels)
 * times s is added to the same slots of z.  Weights are used in BF16,
 * activations and accumulation in FP32; training keeps an FP32 master copy
 * and Adam moments.  Flat FP32 parameter order:
 *   W1 (256, 8, 7) | b1 (256) | W2 (256, 256) | b2 | W3 (256, 256) | b3 | W4 (8, 256) | b4 (8).
 * Features and outputs in the calls below are channel-major float arrays
 * x[c * P + pos], pos = seq * n_t + position, P = nseq * n_t (device). */
pt_status pt_correction_nparams(int64_t* nparams);
/* Weights from / to host memory (nparams floats).  Setting resets Adam. */
pt_status pt_set_correction(pt_ctx* ctx, const float* params, int64_t nparams);
pt_status pt_get_correction(const pt_ctx* ctx, float* params, int64_t nparams);
/* Device scratch for pt_correction_forward / pt_correction_grad on nseq sequences. */
pt_status pt_correction_scratch_bytes(const pt_ctx* ctx, int32_t nseq, size_t* bytes);
/* y = N_theta(x) on raw features (no RMS scaling): x, y device, 8 x P floats. */
pt_status pt_correction_forward(pt_ctx* ctx, int32_t nseq, const float* x, float* y, void* scratch,
                                size_t scratch_bytes);
/* Loss 0.5 mean (N_theta(x) - t)^2 (host double) and its gradient with respect
 * to the parameters (device, nparams floats, overwritten), at the BF16 weights. */
pt_status pt_correction_grad(pt_ctx* ctx, int32_t nseq, const float* x, const float* t, double* loss, float* grad,
                             void* scratch, size_t scratch_bytes);
/* Scratch for pt_train_correction with npairs pairs and minibatches of batch pairs. */
pt_status pt_train_bytes(const pt_ctx* ctx, int32_t npairs, int32_t batch, size_t* bytes);
/* Train on solver-generated pairs: r[p] a permuted residual and e[p] the error
 * it belongs to ((P M) e = r, e.g. e = x* - x_k and r = P b - P M x_k of a
 * GMRES iterate), both device, npairs x 4(L-1) x n_t complex.  Targets are
 * (e - K^{-1} r) / RMS(r) with K^{-1} at the context's precision; Adam with
 * learning rate lr for `steps` minibatches of `batch` pairs drawn with `seed`.
 * Starts from the current weights (a seeded default initialisation when none
 * were set).  loss_first / loss_last (host, NULL allowed): loss of the first
 * and the last minibatch.  scratch >= pt_train_bytes. */
pt_status pt_train_correction(pt_ctx* ctx, int32_t npairs, const pt_c128* r, const pt_c128* e, int32_t steps,
                              int32_t batch, double lr, uint64_t seed, double* loss_first, double* loss_last,
                              void* scratch, size_t scratch_bytes);
/* z = N_theta(v) for nsrc permuted residuals (device); needs learned = 1 and
 * weights; scratch >= solve_bytes. */
pt_status pt_apply_correction(pt_ctx* ctx, int32_t nsrc, const pt_c128* v, pt_c128* z, void* scratch,
                              size_t scratch_bytes);

/* Copy the interface Green's matrix G^l(z_j, z_k) / h (the block that the
 * incomplete Green's integrals of Definition 2 multiply) to dst (device,
 * n_t * n_t pt_c128, row-major, row = target node, column = source node).
 * j, k are the paper's local row indices and must be among {0, 1, n^l, n^l+1}
 * of the layer's interfaces.  Fails with PT_ERR_ARG otherwise. */
pt_status pt_get_block(pt_ctx* ctx, int32_t layer, int32_t j, int32_t k, pt_c128* dst);

/* Uneven batch: independent contexts (different media, grids, layer counts
 * and source counts), each solved as by pt_solve, concurrently - one host
 * thread per context, each context on its own stream (contexts created on
 * the same stream serialise).  Arrays of length nctx: ctxs (distinct),
 * nsrc, f (device), u (device, or u = NULL for no volume output), scratch,
 * scratch_bytes.  iters and relres (host, NULL allowed) hold sum(nsrc)
 * entries, context after context; status (host, NULL allowed) nctx.
 * Returns the first failing context's status (its index in the error text). */
pt_status pt_solve_many(int32_t nctx, pt_ctx* const* ctxs, const int32_t* nsrc, const pt_c128* const* f,
                        pt_c128* const* u, double rel_tol, int32_t max_it, void* const* scratch,
                        const size_t* scratch_bytes, int32_t* iters, double* relres, int32_t* status);

/* Statistics of the last pt_solve: number of kernel launches it issued and
 * the GMRES iteration count of the slowest source. */
pt_status pt_last_solve_stats(const pt_ctx* ctx, int64_t* kernel_launches, int32_t* max_iterations);

/* Restart cycles of the last pt_solve (each ends with an explicit residual) and
 * how many of them applied the learned correction (host outputs, NULL allowed). */
pt_status pt_last_solve_cycles(const pt_ctx* ctx, int32_t* cycles, int32_t* learned_cycles);

/* Matvecs of the last pt_solve that ran in FP32 under PT_OPT_RELAX.
 * PT_ERR_ARG for a NULL argument. */
pt_status pt_last_solve_relaxed(const pt_ctx* ctx, int32_t* relaxed_matvecs);

void pt_destroy(pt_ctx* ctx);
const char* pt_status_string(pt_status s);
/* Text of the last error recorded on this thread (empty when none). */
const char* pt_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* POLARTRACE_H */
