/*
 * sea.h -- C ABI of the GB300 exact-exchange engine for SCDM+exx+ACE
 * (arXiv 2208.06097).
 *
 * The library applies the exact-exchange operator V_xx to a set of localized,
 * orthonormal, real (Gamma-point) occupied orbitals on the real-space grid of
 * an orthorhombic periodic cell, and builds and applies the adaptively
 * compressed exchange (ACE) operator from the result:
 *
 *   sea_apply_vxx   Sec. II B: domain truncation (Eq. oii), pair selection
 *                   (Eq. sij), per-pair Poisson problem (Eq. pe) with
 *                   multipole boundary values (Eqs. me, mepole), local
 *                   D^i (Eq. tDxx) and E_xx (Eq. exxGen_mlwf);
 *                   V_xx phi_i = -D^i (Eq. DxxVxx).
 *   sea_build_ace   Sec. II C, Eq. Vace, App. A: M = Phi^T W dV with
 *                   W = V_xx Phi, Mbar = (M + M^T)/2, -Mbar = L L^T,
 *                   Xi = W L^-T.
 *   sea_apply_ace   V^ACE psi = -Xi (Xi^T psi dV) (Eq. Vace).
 *
 * Units: bohr and hartree.  Grid functions are float64 arrays laid out
 * [n][nz][ny][nx] (x fastest); point (x, y, z) sits at (x hx, y hy, z hz)
 * with h = cell / grid, and every inner product carries dV = hx hy hz.
 *
 * Ownership: the caller owns every buffer it passes and every buffer the
 * library writes into; the library keeps its own device copy of the
 * orbitals and its own workspace, released by sea_destroy.  Pointers marked
 * "host or device" are device pointers when on_device != 0, else pageable or
 * pinned host pointers.
 *
 * Errors: every call returns a sea_status; nothing is thrown across the ABI.
 * A CUDA error poisons the context: later calls return SEA_ERR_STATE.
 * sea_last_error gives a one-line message for the last failure.
 *
 * Streams: all work is ordered on the stream given to sea_create (NULL: the
 * legacy default stream).  Calls that return numbers to the host
 * (sea_apply_vxx's E_xx, status words) synchronize that stream.
 */
#ifndef SEA_H
#define SEA_H

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  SEA_OK = 0,
  SEA_ERR_ARG = 1,              /* bad argument (NULL, size, unsupported option) */
  SEA_ERR_STATE = 2,            /* call order violated, or context poisoned      */
  SEA_ERR_CUDA = 3,             /* a CUDA runtime call failed                    */
  SEA_ERR_OOM = 4,              /* device allocation failed                      */
  SEA_ERR_CG_NOT_CONVERGED = 5, /* a pair's CG hit cg_max_iter (result kept)     */
  SEA_ERR_NOT_PD = 6,           /* -Mbar not positive definite (Cholesky pivot)  */
  SEA_ERR_TIMEOUT = 7,          /* the CG's time budget (timeout_ms) was spent   */
  SEA_ERR_INPUT = 8,            /* orbitals not finite, or not unit norm         */
  SEA_ERR_LIMIT = 9             /* request above a fixed capacity (see below)    */
} sea_status;

/* Method knobs.  Defaults (sea_default_params): eps = 10^-3.5 (Eq. oii),
 * delta = 1e-3 (Eq. sij), cg_tol = 1e-8, cg_tol_mode = 0 (stop when
 * ||r||_2 <= cg_tol ||b||_2; 1: stop when rms(r)/(4 pi) <= cg_tol, a
 * residual density in bohr^-3 as App. C states it), cg_max_iter = 5000,
 * lmax = 6 (App. C), fd_order = 12 (App. C, O(h^12) Laplacian; the only
 * supported value), self_scale = 2 (Omega^D_ii = scale_2x Omega_ii, the only
 * supported value), ace_decomp = 0 (Cholesky of -Mbar, with the eigen
 * decomposition of App. A -- -Mbar = Q Lambda Q^T, operator
 * -W Q |Lambda|^-1 Q^T W^T (the complex zeta of App. A under a Hermitian
 * inner product), eigenvalues within 1e-13 max|lambda| of zero dropped --
 * when a Cholesky pivot is not positive), precision = 0 (FP64 everywhere; 1: the mixed form --
 * FP32 stencil sweeps and CG vectors inside an iterative refinement of
 * each pair's solve, whose true residual and solution are FP64 for
 * cg_tol < 1e-10 and double-float (pairs of FP32 values, about 48 bits)
 * from 1e-10 up, the stopping rule on that true residual; E_xx FP64; the
 * inner FP32 CG uses compensated FP32 dot products and FP32 step lengths;
 * the multipole moments, boundary values and far-field products in
 * double-float arithmetic; the two contractions with W (M = Phi^T W dV,
 * W^T psi, W H) on the tensor cores from exact digit splits of FP64 values
 * (FP16 digits in both, the contraction and the expansion), truncated
 * at 2^-47 of each 64-point segment's largest value; the Cholesky of -Mbar,
 * L^-1, E_xx^ACE and the products with L^-1 in double-float),
 * warm_start = 0
 * (1: every pair's CG starts from the attached learned model's guess and
 * runs to the same tolerance; the batched form always starts from zero). */
typedef struct {
  double eps;
  double delta;
  double cg_tol;
  int cg_tol_mode;
  int cg_max_iter;
  int lmax;       /* 0..6 */
  int fd_order;   /* 12 */
  double self_scale;
  int precision;  /* 0: FP64, 1: mixed (FP32 CG inside FP64 refinement) */
  int warm_start; /* 0: none; 1: the attached sea_unet's guesses (sea_unet_attach) */
  double timeout_ms; /* time budget of sea_apply_vxx's persistent CG launch
                        (0: none).  Once it is spent no CTA takes another
                        pair; the call then returns SEA_ERR_TIMEOUT and its
                        results are not valid (the context stays usable). */
  int ace_decomp; /* 0: Cholesky, eigen form of App. A if a pivot fails;
                     1: Cholesky only (SEA_ERR_NOT_PD on failure); 2: eigen form */
  double orth_tol; /* sea_set_orbitals returns SEA_ERR_INPUT when some
                      |<phi_i|phi_i> - 1| exceeds it (default 1e-6; 0: no
                      norm check).  Mutual orthogonality is not checked: that
                      needs the dense Gram matrix Phi^T Phi dV. */
} sea_params;

/* Per-call statistics of the last sea_apply_vxx / sea_build_ace /
 * sea_apply_ace on a context (device times from CUDA events on the context
 * stream; the sea_apply_ace times are filled once its work has finished). */
typedef struct {
  int n_orb;
  int n_pairs;        /* selected pairs <ij>, i <= j                       */
  int n_proto_pairs;  /* pairs with Omega_ij non-empty before screening    */
  long long n_unknowns; /* sum over pairs of |Omega_ij| (CG unknowns)      */
  long long n_window_points; /* sum over accumulation windows (Eq. tDxx)   */
  int cg_iters_min, cg_iters_max;
  double cg_iters_mean;
  long long cg_unknown_iters; /* sum over pairs of |Omega_ij| x iterations */
  double exx;         /* last E_xx from sea_apply_vxx                      */
  double ms_plan, ms_setup, ms_cg, ms_accumulate; /* device time, last apply_vxx */
  double ms_ace_build, ms_ace_apply;
  long long ace_support_points; /* sum over orbitals of tile-rounded support */
  long long n_launches;  /* kernels this context has launched since creation */
  double ms_gram_build;  /* M = Phi^T W dV contraction, last sea_build_ace       */
  double ms_gram_apply, ms_expand_apply; /* W^T psi and W H, last sea_apply_ace */
  int ace_eigen;                /* 1 if the last build used the eigen form      */
  int ace_eigen_sweeps;         /* Jacobi sweeps of that build                  */
  int ace_negative_eigenvalues; /* eigenvalues of -Mbar below zero              */
  int ace_dropped_eigenvalues;  /* eigenvalues treated as zero                  */
  int batch_graph;  /* last sea_apply_vxx_batch led by this context: 0 direct
                       launches, 1 graph captured, 2 graph replayed            */
  int ace_max_tile_list; /* longest W list of a tile, last sea_build_ace (the
                            mixed form expands lists up to 32 on the tensor
                            cores, longer ones in FP32 error-free arithmetic) */
  int batch_order;       /* last sea_apply_vxx_batch led by this context: the
                            autotuned order of the CG's work items (0 ranks
                            round-robin over configurations, 1 all pairs
                            longest first, 2 configuration-major)          */
  int batch_ctas_per_sm, batch_ctas_per_sm_fp64; /* its autotuned persistent
                            grids (CTAs per SM) of the mixed-form and FP64 CG */
  double batch_tune_ms;  /* device time spent tuning in that call (0: the
                            workload's choice was already known)           */
  double exx_ace; /* E_xx^ACE = sum_i <phi_i|V^ACE|phi_i> = -sum_ik <phi_i|xi_k>^2
                     (Eq. exx_ace), last sea_build_ace: -tr(M K M^T) with
                     K = (-Mbar)^-1 = L^-T L^-1 (Cholesky form) or
                     Q |Lambda|^-1 Q^T (eigen form, kept eigenvalues) */
} sea_stats;

typedef struct sea_ctx sea_ctx;

/* Fill *p with the defaults listed above. */
void sea_default_params(sea_params* p);

/* Create a context for an orthorhombic cell.  cell[3]: edge lengths (bohr,
 * > 0); grid[3]: points per axis (nx, ny, nz), each in [8, 1024];
 * p: NULL for defaults; cuda_stream: a cudaStream_t or NULL.  The context
 * selects no device: the current device at creation is used for its life. */
sea_status sea_create(const double cell[3], const int grid[3], const sea_params* p,
                      void* cuda_stream, sea_ctx** out);

/* Copy n_orb orbitals ([n_orb][nz][ny][nx], host or device) into the
 * context.  Any earlier exchange/ACE result is invalidated.  Returns
 * SEA_ERR_INPUT if a value is not finite or, with orth_tol > 0, if some
 * orbital's norm <phi_i|phi_i> = dV sum phi_i^2 (FP64) differs from 1 by
 * more than orth_tol.  Host orbitals are copied in orbital ranges, each
 * range checked while the next one is in flight. */
sea_status sea_set_orbitals(sea_ctx* ctx, const double* phi, int n_orb, int on_device);

/* SCDM localization (Sec. II A): from n_orb orthonormal orbitals phi
 * (canonical or any other basis of the occupied space; [n_orb][nz][ny][nx],
 * host or device, orthonormal with the grid weight) the context's orbitals
 * become Phi~ = Phi U with
 *   Phi^T Pi = Q R (column-pivoted QR, Eq. phi_qr), C = first n_orb pivots,
 *   B = (Phi^T)_{:,C}, P_CC = B^T B, U = B P_CC^{-1/2} (Eqs. nonortho_scdm,
 *   ortho_scdm, unitary_scdm).
 * U[n_orb][n_orb] (row-major, host, may be NULL) receives U and cols[n_orb]
 * (host, may be NULL) the selected grid points (flat index z ny nx + y nx
 * + x) in pivot order.  Pivots: at each step the grid point whose column
 * of Phi^T has the longest component orthogonal to those already chosen
 * (ties: smallest index).  Any earlier exchange/ACE result is invalidated.
 * SEA_ERR_INPUT if a value is not finite or the orbitals are rank
 * deficient.  Synchronizes the context stream. */
sea_status sea_scdm(sea_ctx* ctx, const double* phi, int n_orb, int on_device, double* U,
                    int* cols);

/* Apply V_xx to every orbital: vxx_phi[n_orb][nz][ny][nx] (host or device,
 * caller-owned) receives V_xx phi_i = -D^i; *exx (may be NULL) receives E_xx.
 * Synchronizes the context stream after the plan (sizes) and at the end (E_xx
 * and the status word).  With a host vxx_phi (page-locked for full speed)
 * the last stage runs by orbital ranges and each range's copy out overlaps
 * the kernels of the next.
 * Returns SEA_ERR_CG_NOT_CONVERGED (results still written) if any pair's CG
 * reached cg_max_iter. */
sea_status sea_apply_vxx(sea_ctx* ctx, double* vxx_phi, int on_device, double* exx);

/* Batched form: apply V_xx for n independent configurations (each its own
 * context, orbitals already set) in one pass -- all their pairs' Poisson
 * problems in one persistent launch.  The launch's pair order and grid are
 * autotuned per workload (pair counts, unknowns, grids and forms of the
 * configurations): the first call for a workload times each candidate on
 * the batch and keeps the fastest for the process (sea_stats.batch_*);
 * every candidate gives the same results bit for bit.  All contexts must use the same device
 * and the same stream; vxx_phi[k] (host or device per on_device) receives
 * configuration k's V_xx phi, exx[k] (may be NULL) its E_xx.  The phase
 * after the plan (pair setup, CG, far field, accumulation) is captured in a
 * CUDA graph on the first call and replayed while the plan's sizes and the
 * buffers stay the same (not on the legacy NULL stream, which cannot be
 * captured).  Per-context results and statistics as for sea_apply_vxx;
 * returns SEA_ERR_CG_NOT_CONVERGED if any configuration hit the cap. */
sea_status sea_apply_vxx_batch(sea_ctx* const* ctxs, int n, double* const* vxx_phi,
                               int on_device, double* exx);

/* Build the ACE operator from the orbitals and the last sea_apply_vxx
 * result, and E_xx^ACE (Eq. exx_ace, the energy the paper's SeA reports;
 * in sea_stats.exx_ace).  Returns SEA_ERR_STATE if no sea_apply_vxx result
 * is current and SEA_ERR_NOT_PD when -Mbar has a non-positive Cholesky
 * pivot and ace_decomp = 1 (with ace_decomp = 0 the eigen form takes
 * over). */
sea_status sea_build_ace(sea_ctx* ctx);

/* Same, from a caller-supplied W = V_xx Phi ([n_orb][nz][ny][nx], host or
 * device; the decomposition step of Fig. 2(c) on its own).  W is treated
 * as dense (its support is not known), and it replaces any earlier
 * sea_apply_vxx result in the context. */
sea_status sea_build_ace_from(sea_ctx* ctx, const double* W, int on_device);

/* out[n_vec][nz][ny][nx] = V^ACE psi for psi[n_vec][nz][ny][nx] (host or
 * device, same flag for both).  Requires a successful sea_build_ace.
 * With host buffers (page-locked for full speed) the call works through
 * chunks of at least 32 vectors, overlapping the copy in of one chunk, the
 * kernels of the previous one and the copy out of the one before on
 * separate streams; it returns when out is written.  Stats of such a call:
 * ms_ace_apply spans the whole pipeline (copies included), ms_gram_apply
 * and ms_expand_apply the last chunk's kernels. */
sea_status sea_apply_ace(sea_ctx* ctx, const double* psi, int n_vec, double* out,
                         int on_device);

/* Optional exports of the last results (host or device destination).
 *   sea_get_ace_matrices: M[n][n] (M_ij = <phi_i|W_j>), L[n][n] (lower,
 *     zero above the diagonal; in the eigen form, the diagonalized -Mbar:
 *     eigenvalues on the diagonal); either pointer may be NULL.
 *   sea_get_ace_vectors: xi[n][nz][ny][nx], the ACE vectors Xi = W L^-T
 *     (materialized on demand; the operator itself is applied in the
 *     factored form W L^-T L^-1 W^T).  SEA_ERR_STATE in the eigen form,
 *     whose vectors may be complex.
 *   sea_get_plan: box[n][6] (start x,y,z then extent x,y,z of Omega_ii),
 *     pairs[P][2], lo[P][3], ext[P][3] (Omega_ij in i's unwrapped frame),
 *     S[P] (Eq. sij), iters[P] (CG iterations, negative if capped),
 *     epair[P] (sum over Omega_ij of rho v dV); host pointers, any may be
 *     NULL; *n_pairs receives P (required). */
sea_status sea_get_ace_matrices(sea_ctx* ctx, double* M, double* L, int on_device);
sea_status sea_get_ace_vectors(sea_ctx* ctx, double* xi, int on_device);
sea_status sea_get_plan(sea_ctx* ctx, int* box, int* n_pairs, int max_pairs, int* pairs,
                        int* lo, int* ext, double* S, int* iters, double* epair);

sea_status sea_get_stats(const sea_ctx* ctx, sea_stats* s);

/* The per-pair Poisson solver on its own (Eq. pe with the O(h^12)
 * Laplacian of App. C): solve -Lap_h x_b = rhs_b on each of n_box boxes with
 * zero values outside the box (boundary values, if any, already moved into
 * rhs), by CG from x = 0 with the stopping rule of sea_params (tol,
 * tol_mode, max_iter).  h[3]: grid spacing (bohr); ext[n_box][3] (host):
 * box extents (x, y, z), each in [1, 1024]; rhs, x (device): the boxes'
 * values concatenated in order, each box [ez][ey][ex]; iters (host, may be
 * NULL) receives the iteration counts (negative: capped).  Allocates and
 * frees its own device scratch (3 vectors of the total length) on every
 * call and synchronizes the stream.  Returns SEA_ERR_CG_NOT_CONVERGED if a
 * box reached max_iter (x still written). */
sea_status sea_poisson_batch(const double h[3], int n_box, const int* ext, const double* rhs,
                             double* x, double tol, int tol_mode, int max_iter, int* iters,
                             void* cuda_stream);

/* Same solve as sea_poisson_batch, for callers that cannot allocate device
 * memory: plugins whose host framework owns all device memory through its
 * own pool, and processes whose device footprint is fixed at start-up.  It
 * allocates nothing: its scratch is one fixed array of device memory inside
 * the library (about 25 MB, held on every GPU that loads the library until
 * the process exits).  The paper has no counterpart to this entry point.
 * Limits: n_box <= 4096 and sum of box sizes <= 1048576 unknowns, else
 * SEA_ERR_LIMIT before any GPU work.  The caller still provides rhs and x
 * (device) and ext, iters (host), as for sea_poisson_batch.  All calls share
 * the one array: calls that overlap on the GPU race, so order them; each
 * call clears what must start at zero.  The first call on a device looks up
 * the array's device address (once per device).  The call is synchronous
 * (pageable host copies and a stream synchronize), so it must not be made
 * while its stream is being captured into a CUDA graph: on a capturing
 * stream it returns SEA_ERR_ARG before queueing anything, and the capture
 * stays valid. */
sea_status sea_poisson_batch_noalloc(const double h[3], int n_box, const int* ext,
                                     const double* rhs, double* x, double tol, int tol_mode,
                                     int max_iter, int* iters, void* cuda_stream);

/* Learned warm start for the pair solves (the paper has no counterpart:
 * its CG starts from zero; this changes only the starting point).  A 3-level
 * 3D U-Net (width c: 16/32/64 channels for c = 16) maps a pair's
 * right-hand side b of -Lap_h v = b (Eq. pe with the ghost-shell boundary
 * terms of Eqs. me, mepole moved into b), divided by s = max|b| on the box,
 * together with the box mask -- both embedded at the centre of a 32^3
 * patch, layout [2][32][32][32] floats -- to v / s on the patch.  Pairs
 * whose box exceeds 32 points on an axis start from zero.  BF16 weights,
 * FP32 activations and accumulation, fixed-order reductions.
 *   sea_unet_create       seeded He-normal weights, zero biases; NULL stream
 *                         = legacy stream.  width 1..64.
 *   sea_unet_num_weights  length of the flat FP32 weight array: per layer
 *                         (conv3 2->c, c->c, c->2c, 2c->2c, 2c->4c, 4c->4c,
 *                         6c->2c, 2c->2c, 3c->c, c->c, conv1 c->1) W[cout][cin][k]
 *                         (k = 27 as z, y, x of the 3x3x3 stencil, or 1), then
 *                         b[cout].
 *   sea_unet_weights      host copy out (set = 0) or in (set = 1); the kernels
 *                         use the weights rounded to BF16, the biases as FP32.
 *   sea_unet_forward      out[B][32^3] for in[B][2][32^3] (host or device).
 *   sea_unet_loss_grad    masked mean squared error of forward(in) against
 *                         target[B][32^3] (mask = input channel 1) and its
 *                         gradient w.r.t. the flat weights (host, may be NULL);
 *                         B <= 32.
 *   sea_unet_collect      appends the context's last sea_apply_vxx pairs as
 *                         training samples (b / s and mask -> v / s).
 *   sea_unet_train        Adam (beta 0.9, 0.999) for `steps` batches drawn with
 *                         replacement (seeded); *last_loss = the last batch's.
 *   sea_unet_attach       the model warm-starts ctx's CG when
 *                         params.warm_start = 1 (NULL detaches; the context
 *                         does not own the model, keep it alive while attached).
 * All calls synchronize the model's stream (the warm start itself runs on the
 * context's stream inside sea_apply_vxx). */
typedef struct sea_unet sea_unet;
sea_status sea_unet_create(int width, int seed, void* cuda_stream, sea_unet** out);
long long sea_unet_num_weights(const sea_unet* net);
sea_status sea_unet_weights(sea_unet* net, float* w, int set);
sea_status sea_unet_forward(sea_unet* net, const float* in, int B, float* out, int on_device);
sea_status sea_unet_loss_grad(sea_unet* net, const float* in, const float* target, int B,
                              double* loss, float* grad, int on_device);
sea_status sea_unet_collect(sea_unet* net, sea_ctx* ctx);
long long sea_unet_num_samples(const sea_unet* net);
sea_status sea_unet_train(sea_unet* net, int steps, int batch, double lr, int seed,
                          double* last_loss);
sea_status sea_unet_attach(sea_ctx* ctx, sea_unet* net);
const char* sea_unet_last_error(const sea_unet* net);
void sea_unet_destroy(sea_unet* net);

/* Message for the last failing call on ctx (static text; never NULL). */
const char* sea_last_error(const sea_ctx* ctx);

/* Release everything the context owns.  NULL is ignored. */
void sea_destroy(sea_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* SEA_H */
