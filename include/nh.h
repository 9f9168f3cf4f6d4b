/*
 * nh.h -- C ABI of the GB300 (sm_103a) hybrid lattice-Boltzmann + finite-
 * difference nematohydrodynamics library.
 *
 * The method is the one of Amaral, Sedahmed, Telo da Gama and Coelho,
 * "Efficient single-precision simulations of nematohydrodynamics"
 * (arXiv:2503.06610):
 *   - flow: D3Q19 lattice Boltzmann with single relaxation time, Guo forcing
 *     and (optionally) shifted populations f_i - w_i (Sec. II.C, Eqs. feq-eq,
 *     shifted-feq, shifted-rho, shifeted-u, shifted-lbe), half-way bounce-back
 *     plates in z and periodic sides;
 *   - director: Ericksen-Leslie equation (Sec. II.A, Eq. director-time-eq)
 *     with a one-constant chiral Frank field, advanced by the predictor-
 *     corrector of Sec. II.B on its own time step dt_FD and renormalised;
 *   - coupling: the LC force of Eq. force-lc-eq, recomputed every dt_FD steps
 *     and held fixed in between (Sec. II.D).
 *
 * Conventions shared by every entry point
 *   - Site index s = x + nx*(y + ny*z), x fastest.  N = nx*ny*nz.
 *   - Vector fields are structure-of-arrays double[3][N]; scalars double[N];
 *     populations double[19][N] in the D3Q19 order
 *       0:(0,0,0) 1:(+x) 2:(-x) 3:(+y) 4:(-y) 5:(+z) 6:(-z)
 *       7:(+x+y) 8:(-x-y) 9:(+x-y) 10:(-x+y) 11:(+x+z) 12:(-x-z)
 *       13:(+x-z) 14:(-x+z) 15:(+y+z) 16:(-y-z) 17:(+y-z) 18:(-y+z).
 *   - With walls_z = 1 the plates are solid layers at z = -1 and z = nz; the
 *     no-slip walls sit half-way, at z = -1/2 and nz - 1/2.
 *   - All quantities are in lattice units (Delta x = Delta t = rho0 = 1).
 *   - Pointers flagged "on_device" are CUDA device pointers on the context's
 *     device; otherwise they are host pointers (pinned memory is faster, any
 *     host memory works).  The caller owns every buffer it passes.
 *   - Every function returns NH_OK (0) or a negative error code; no C++
 *     exception crosses this boundary and no device code traps.  The text of
 *     the last error of a context is available from nh_last_error().
 *   - Device memory: the library allocates none.  The caller obtains the
 *     size from nh_workspace_bytes(), allocates it (e.g. with PyTorch) and
 *     binds it with nh_bind_workspace(); it must stay alive until
 *     nh_destroy().
 */
#ifndef NH_H
#define NH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define NH_OK 0
#define NH_EINVAL (-1)    /* bad argument, dimensions or parameters */
#define NH_ECUDA (-2)     /* a CUDA runtime call failed */
#define NH_ENOMEM (-3)    /* workspace missing or too small */
#define NH_EUNSTABLE (-4) /* a NaN or Inf was found in the fields */
#define NH_ETIMEOUT (-5)  /* a bounded wait expired (nh_set_wait_limit) */

#define NH_FP64 0 /* arithmetic precision */
#define NH_FP32 1

#define NH_STORE_F64 0   /* population storage: double            (FP64 only) */
#define NH_STORE_F32 1   /* float                                 (FP32 only) */
#define NH_STORE_F16S 2  /* IEEE half of 2^k * f_shifted          (FP32, shifted) */
#define NH_STORE_BF16S 3 /* bfloat16 of 2^k * f_shifted           (FP32, shifted) */

#define NH_ANCHOR_NONE 0        /* ghost director = adjacent fluid layer */
#define NH_ANCHOR_HOMEOTROPIC 1 /* infinite homeotropic anchoring: ghost director = z_hat */

#define NH_MAX_TUBES 32

/* Parameters of one channel.  Table I of the paper lists a physical set; the
 * field names follow the paper's symbols. */
typedef struct nh_params {
    int32_t nx, ny, nz;   /* lattice size, each >= 1, 19*nx*ny*nz < 2^31 */
    int32_t walls_z;      /* 1: bounce-back plates in z; 0: periodic in z */
    int32_t anchoring;    /* NH_ANCHOR_* (used only with walls_z = 1) */
    int32_t precision;    /* NH_FP64 or NH_FP32 */
    int32_t storage;      /* NH_STORE_* */
    int32_t shifted;      /* 1: store f_i - w_i (Eq. shifted-feq); 0: plain f_i */
    int32_t dt_fd;        /* FD time step in LB steps, >= 1 (Sec. II.D) */
    int32_t check_stability; /* 1: reject dt_fd * 6 K / gamma1 > 1 (Heun limit of the 3D compact Laplacian) */
    int32_t paper_order;  /* 1: the loop order of Sec. II.D taken literally: on a step that completes an
                             FD interval the FD update runs between the macroscopic fields and the
                             collision, so that collision's Guo source carries the new force while its
                             u carries half of the old one (an extra LB launch per FD interval).
                             0 (default): the collision of that step keeps the old force and the new
                             force acts from the next step.  Not supported by nh_batch_step. */
    int32_t frank3;       /* 1: three-constant Frank energy (Eq. free-energy-eq with K11, K22, K33): the
                             one-constant lattice energy with K plus, per fluid site,
                             (K11-K)/2 (div n)^2 + (K22-K)/2 (n.curl n + q0)^2 + (K33-K)/2 |n x curl n|^2
                             with central differences; h is its exact variational derivative.  Runs on the
                             per-site FD kernels (nh_set_fd_variant 0), in batches too. */
    /* Reading flags.  The paper is silent on each choice below; 0 is the default reading.  Each
       flag is 0 or 1; any other value is NH_EINVAL. */
    int32_t renorm_predictor; /* 1: also renormalise the predictor n^P to |n^P| = 1 before the corrector
                             evaluates its rate (Sec. II.B lists no renormalisation; 0: only the corrected
                             director is renormalised).  All FD kernels and the batched calls. */
    int32_t lap_wide;     /* 1: the second derivatives of the molecular field are central differences of
                             central differences, (n(x+2e) - 2 n(x) + n(x-2e))/4 per axis (the first-
                             derivative stencil of Sec. II.B applied twice), reading the ghost rule at
                             distance 2 as at distance 1; 0: the compact 3-point Laplacian, which makes h
                             the exact derivative of the lattice energy.  Per-site FD kernels only. */
    int32_t n_from_rate;  /* 1: the kinematic transport N of the viscous stress (Sec. II.A, N = dn/dt +
                             u.grad n - W n) takes dn/dt from the corrector's averaged rate of the FD update
                             that produced n, and the sum is projected normal to n; 0: N from the director equation,
                             [h_perp - gamma2 (I - n n) D n]/gamma1.  A force computed without an FD update
                             (nh_set_fields, nh_restore) uses the 0 reading.  Per-site FD kernels only. */
    int32_t ghost_sigma;  /* stress at the plates' ghost layers in the force divergence (Sec. II.B computes
                             gradients at fluid nodes only): 0 = zero stress; 1 = mirror, the stress of the
                             adjacent fluid layer (zero normal gradient; the total force then equals the
                             stress difference across the channel).  All FD kernels. */
    double tau;           /* SRT relaxation time, > 1/2; nu = (tau - 1/2)/3 */
    double g[3];          /* body acceleration g of Eq. NS-eq; the LB force is F_lc + rho g */
    double K;             /* one-constant Frank elasticity */
    double q0;            /* cholesteric wavenumber 2 pi / P */
    double gamma1;        /* rotational viscosity alpha3 - alpha2, > 0 */
    double gamma2;        /* torsion coefficient alpha3 + alpha2 */
    double alpha1, alpha2, alpha3, alpha4p, alpha5, alpha6; /* Leslie viscosities; alpha4p = alpha_4' */
    double W0;            /* bulk effective anchoring: h += W0 n_z z_hat */
    double K11, K22, K33; /* splay, twist, bend constants, used when frank3 = 1 (each > 0) */
} nh_params;

/* Result of nh_diagnostics.  Reductions are accumulated in FP64. */
typedef struct nh_diag {
    int64_t step;          /* completed LB steps */
    double mass;           /* sum over sites and populations of f_i */
    double energy;         /* lattice Frank energy E_d of the director (see nh_diagnostics) */
    double max_u;          /* max |u| over sites */
    double min_norm, max_norm; /* extrema of |n| */
    int32_t nonfinite;     /* sites with a NaN/Inf in n, plus sites with one in u, rho or the sum of
                              their populations (a site bad in both counts twice): 0 iff all is finite */
    int32_t n_tubes;       /* number of tracked tubes */
    double centroid[NH_MAX_TUBES][2]; /* tube centroids (x, y) in [0, nx) x [0, ny) */
    double tube_weight[NH_MAX_TUBES]; /* sum of (1 - n_z)/2 over each tube's sites */
} nh_diag;

/* Per-kernel-class timing, collected when nh_set_timing(ctx, 1) is on. */
#define NH_KCLASS_LB 0
#define NH_KCLASS_FD_PREDICT 1
#define NH_KCLASS_FD_CORRECT 2
#define NH_KCLASS_STRESS 3
#define NH_KCLASS_FORCE 4
#define NH_KCLASS_COUNT 5
typedef struct nh_timing {
    int64_t launches[NH_KCLASS_COUNT];
    double ms[NH_KCLASS_COUNT];
} nh_timing;

typedef struct nh_ctx nh_ctx;

/* Text for an error code. */
const char* nh_error_string(int code);

/* Text of the last error recorded on ctx (empty if none); ctx may be NULL
 * for errors of nh_create and nh_batch_step. */
const char* nh_last_error(const nh_ctx* ctx);

/* Bytes of device workspace a context with parameters *p needs.
 * Returns NH_EINVAL for invalid parameters (same checks as nh_create). */
int nh_workspace_bytes(const nh_params* p, size_t* bytes);

/* Create a context for one channel on the current CUDA device.  cuda_stream
 * (a cudaStream_t, may be NULL for the legacy default stream) is the default
 * stream of later calls.  Validates the parameters: sizes >= 1, tau > 1/2,
 * gamma1 > 0, dt_fd >= 1, a storage that matches the precision, shifted = 1
 * for the 16-bit stores, and (if check_stability) the Heun limit.  The
 * context is not usable until a workspace is bound. */
int nh_create(const nh_params* p, void* cuda_stream, nh_ctx** out);

/* Bind the caller-owned device workspace (at least nh_workspace_bytes,
 * 256-byte aligned).  Rebinding discards the fields. */
int nh_bind_workspace(nh_ctx* ctx, void* dev_ptr, size_t bytes);

/* Initialise the state (Sec. II.D "Initialization"): director n [3][N]
 * (required; normalised on load), velocity u [3][N] (NULL = rest) and density
 * rho [N] (NULL = 1).  Populations are set to the equilibrium f^eq(rho, u)
 * (shifted if the context is shifted), the step counter to 0, and the LC force
 * is computed from n and u (Eq. force-lc-eq).  Enqueued on the context's
 * stream; host buffers are read before the call returns. */
int nh_set_fields(nh_ctx* ctx, const double* n, const double* u, const double* rho, int on_device);

/* Copy out the director n [3][N], and the velocity u [3][N] and density
 * rho [N] of the last completed LB step (Eqs. shifted-rho, shifeted-u).  Any
 * pointer may be NULL to skip that field.  Synchronises the context's stream. */
int nh_get_fields(nh_ctx* ctx, double* n, double* u, double* rho, int on_device);

/* Copy out the post-collision populations of the last step as double
 * [19][N], in the context's representation (f_i - w_i when shifted,
 * decoded from the 16-bit scale when stored in 16 bits).  Synchronises. */
int nh_get_populations(nh_ctx* ctx, double* f, int on_device);

/* Replace the populations (same representation as nh_get_populations); for
 * checkpoint / resume together with nh_set_director and nh_set_step. */
int nh_set_populations(nh_ctx* ctx, const double* f, int on_device);

/* Copy out the LC force F_lc [3][N] in effect (frozen between FD steps). */
int nh_get_force(nh_ctx* ctx, double* F, int on_device);

/* Restore a checkpoint: director n [3][N], force F_lc [3][N] (NULL:
 * recompute from n and the stored u), velocity u [3][N] and rho [N] of the
 * checkpointed step (NULL: leave), and the step counter. */
int nh_restore(nh_ctx* ctx, const double* n, const double* F, const double* u, const double* rho,
               int64_t step, int on_device);

/* Advance n_lb_steps LB steps (Sec. II.D): every step one fused LB
 * collide-and-stream launch; after each step whose count s is a multiple of
 * dt_fd, the FD predictor-corrector on n with that step's u, then the LC
 * stress and force.  Asynchronous on stream (NULL = the context's stream).
 * Whole dt_fd blocks run from a CUDA graph unless timing is on. */
int nh_step(nh_ctx* ctx, int64_t n_lb_steps, void* stream);

/* Run one FD update now (predictor, corrector + renormalisation, stress,
 * force) with the context's current u, without an LB step. */
int nh_fd_update(nh_ctx* ctx, void* stream);

/* Advance count independent channels (uneven sizes and parameters allowed)
 * by n_lb_steps each.  Every pass (LB sweep, FD predict, correct, stress,
 * force) is one persistent launch per group of up to 64 channels: the grid
 * walks a work list of (channel, tile) pairs, and the channel descriptors
 * travel as kernel parameters.  Whole dt_fd blocks are replayed from a CUDA
 * graph cached per list of contexts (dropped when a context is rebound,
 * re-tuned or destroyed).  All contexts must share precision, storage,
 * shifted and dt_fd, be on one device, have fields set and be at the same
 * step phase (step mod dt_fd and buffer parity), and not use paper_order,
 * lap_wide or n_from_rate; otherwise NH_EINVAL and nothing runs.  The FD
 * passes use the fused kernels when every channel does, else the per-site
 * kernels (with the three-constant P stages when a channel has frank3); with
 * obstacles in any channel the LB sweep runs one site per thread.  Launch
 * counts and timing are recorded on ctxs[0]; the launch shape is ctxs[0]'s LB
 * variant (see nh_batch_autotune).  Asynchronous on stream (NULL = ctxs[0]'s
 * stream). */
int nh_batch_step(nh_ctx* const* ctxs, int count, int64_t n_lb_steps, void* stream);

/* Autotuner of the batched LB launch: times every launch shape valid for all
 * channels on the batch itself (the state is not advanced), keeps the fastest
 * for this list of contexts and returns it in *chosen.  Synchronises. */
int nh_batch_autotune(nh_ctx* const* ctxs, int count, void* stream, int* chosen);

/* ------------------------------------------------------------------------
 * Slabs along y: one channel split over several contexts (the domain
 * decomposition of a channel across devices; here every slab sits on the one
 * device of the run and the halos move by device copies).
 *
 * Slab k of count (k = 0 lowest in y, periodic: the last is below the first)
 * holds ny_local[k] >= 1 interior rows of the global channel plus one ghost
 * row on each side: its context is created with ny = ny_local[k] + 2 and its
 * row r is global row y0_k + r - 1 (y0_k = sum of the ny_local below it).
 * Every kernel runs over the whole slab; the ghost rows are overwritten with
 * the neighbours' interior rows before anything reads them:
 *   - after every LB step, the populations the interior pulls across each
 *     face: the five with e_y = +1 (3, 7, 10, 15, 17) into the lower ghost
 *     row and the five with e_y = -1 (4, 8, 9, 16, 18) into the upper one
 *     (pull streaming, Sec. II.C);
 *   - in an FD update, u before the predictor, n^P before the corrector, n
 *     before the stress and the stress before its divergence (the radius-1
 *     central differences of Sec. II.B).
 * The interior rows then follow the single-channel run exactly (the same
 * kernels on the same operands).  Slabs use the per-site FD kernels. */
#define NH_HALO_POPULATIONS 0 /* populations after an LB step */
#define NH_HALO_VECTOR 1      /* n, n^P or u: three components */
#define NH_HALO_STRESS 2      /* sigma: nine components */
typedef struct nh_row_copy {
    int32_t src_slab, src_row; /* copy row src_row of slab src_slab ... */
    int32_t dst_slab, dst_row; /* ... into row dst_row of slab dst_slab (rows 0 and ny_local + 1 are ghosts) */
    uint32_t comp_mask;        /* bit c: component c (population plane, vector or stress component) */
} nh_row_copy;

/* The halo plan of count (1 .. 64) slabs for one kind of exchange: the row
 * copies, two per slab (its lower and its upper ghost row), written to out
 * (capacity entries; out may be NULL to ask for the count in *n_out).  Host
 * only: needs no device, so a multi-process transport can follow the same
 * plan.  NH_EINVAL for a bad count, kind or ny_local < 1. */
int nh_slab_plan(int count, const int32_t* ny_local, int kind, nh_row_copy* out, int capacity, int* n_out);

/* Make the slabs consistent after nh_set_fields on each: exchange the ghost
 * rows of the populations, n and u, then recompute every slab's stress,
 * exchange its ghost rows and recompute the force.  The slabs must share
 * every parameter but ny, be on one device at the same step, use F64 or F32
 * stores, and not use paper_order, frank3, lap_wide or obstacles (NH_EINVAL
 * otherwise).  Asynchronous on stream (NULL = slabs[0]'s stream). */
int nh_slab_init(nh_ctx* const* slabs, int count, void* stream);

/* Advance every slab by n_lb_steps hybrid steps (as nh_step) with the halo
 * exchanges above; direct launches on stream (NULL = slabs[0]'s stream).
 * Same requirements as nh_slab_init.  Launch counts go to each slab (row
 * copies to slabs[0]). */
int nh_slab_step(nh_ctx* const* slabs, int count, int64_t n_lb_steps, void* stream);

/* Director-only relaxation (the plain method that relaxes an ansatz, Sec. II.A
 * "minimizing its free energy"): sets u = 0 and runs n_fd_steps
 * predictor-corrector steps of length dt_fd of Eq. director-time-eq, which
 * at rest is the gradient flow dn/dt = h/gamma1 of the Frank energy, each
 * followed by |n| = 1.  No LB step, stress or force is computed: after it the
 * populations and F_lc are stale until nh_set_fields.  Asynchronous. */
int nh_relax(nh_ctx* ctx, int64_t n_fd_steps, void* stream);

/* nh_relax for count channels at once, one launch per pass per group of up to
 * 64 channels (same work-list kernels as nh_batch_step).  Channels must share
 * precision and device; sizes and parameters may differ.  Launches and timing
 * are recorded on ctxs[0]. */
int nh_batch_relax(nh_ctx* const* ctxs, int count, int64_t n_fd_steps, void* stream);

/* Largest change of the director since the previous call: *max_change =
 * max over sites of |n - n_snapshot| (INFINITY on the first call after
 * nh_set_fields), then the snapshot is replaced by the current n.  Used to
 * decide when a relaxation has converged.  Synchronises the stream. */
int nh_director_change(nh_ctx* ctx, double* max_change);

/* Project the director onto fields symmetric under rotations by 90 degrees
 * about the z axis through the site (nx/2, nx/2) (requires nx == ny): the
 * average of the four rotated images (site and vector rotated), normalised.
 * Rotations about z are symmetries of the chiral Frank energy, the plates and
 * the director equation at rest, so a tube centred on that axis stays
 * centred.  Populations and F_lc are not updated.  Asynchronous. */
int nh_symmetrize_c4(nh_ctx* ctx);

/* Obstacles (Sec. II.B: solid boundaries, obstacles included, carry infinite
 * homeotropic anchoring and no-slip by bounce-back): mask[N]
 * (host, or device when on_device = 1) with 1 at solid nodes, 0 at fluid
 * nodes, site index x + nx*(y + ny*z); NULL removes the obstacles.  A lattice
 * link from a fluid site to a solid node bounces back half-way, like the
 * plates; solid nodes keep the director they hold (store the surface normal
 * there, with nh_set_fields or nh_restore: infinite anchoring), their velocity
 * and stress are zero and their populations are carried over unchanged; the
 * diagnostics sum over fluid sites (links with at least one fluid end).
 * The mask is copied into the workspace; the force is recomputed if the
 * fields are set.  Obstacles run on the per-site FD kernels (the fused FD
 * variant is rejected); a batch with obstacles in any channel runs the
 * per-site FD kernels and a one-site-per-thread LB sweep for all.  With
 * walls_z = 1 the plates stay as they are.  Synchronises the context's stream
 * (the fluid sites are counted on the host). */
int nh_set_solid(nh_ctx* ctx, const uint8_t* mask, int on_device);

/* Set the tube centroids to track (count <= NH_MAX_TUBES, centres[2*count]
 * as (x, y) pairs); 0 disables tracking. */
int nh_set_tubes(nh_ctx* ctx, const double* centres, int count);

/* FP64 global diagnostics of the current state: mass, lattice Frank energy
 *   E_d = sum over nearest-neighbour links (x, x+e_b), including links to the
 *         wall ghost layers, of K/2 |n(x+e_b) - n(x)|^2
 *         + K q0 eps_abc n_a(x) n_c(x+e_b), plus sum over sites of
 *         K q0^2/2 - W0/2 n_z^2,
 * |u| and |n| extrema, a NaN/Inf count, and the tracked tube centroids
 * (circular means of the weight (1 - n_z)/2 over the sites nearest to each
 * previous centroid); the new centroids become the tracked ones.
 * Synchronises the stream; returns NH_EUNSTABLE if nonfinite > 0 (the struct
 * is still filled). */
int nh_diagnostics(nh_ctx* ctx, nh_diag* out);

/* Enqueue the diagnostics reductions of the current state on stream (NULL =
 * the context's stream) without waiting; nh_diagnostics_read() then waits for
 * the last enqueued result and decodes it like nh_diagnostics (which is
 * nh_diagnostics_enqueue followed by nh_diagnostics_read).  The tube
 * assignment uses the centroids known to the host at enqueue time. */
int nh_diagnostics_enqueue(nh_ctx* ctx, void* stream);
int nh_diagnostics_read(nh_ctx* ctx, nh_diag* out);

/* Per-kernel timing with CUDA events on the launching stream: 0 = off,
 * 1 = every kernel class, 2 = the LB class only.  Timing forces direct
 * launches (no graphs); consecutive launches of one class form one segment
 * bracketed by one pair of events, so nh_get_timing reports per class the
 * number of launches and their total time (gaps between back-to-back
 * launches of the class included).  nh_get_timing synchronises and resets. */
int nh_set_timing(nh_ctx* ctx, int on);
int nh_get_timing(nh_ctx* ctx, nh_timing* out);

/* Kernel launches this context has issued (graph nodes counted per replay). */
int64_t nh_launch_count(const nh_ctx* ctx);

/* Select the launch shape of the fused LB kernel: 0 = two sites per thread,
 * 256 threads (default; needs even nx), 1 = one site per thread, 256 threads,
 * 2 = two sites, 128 threads, 3 = one site, 128 threads, 4 = four sites,
 * 128 threads, 5 = four sites, 64 threads (4 and 5 need nx % 4 == 0),
 * 6 = 16-bit stores only (F16S, BF16S): whole x-rows of the 19 source planes
 * staged in shared memory by bulk asynchronous copies, the next row in flight
 * while a block collides the current one, four sites per thread (needs
 * nx % 128 == 0 and nx <= 256; with obstacles it runs as variant 0).  All variants compute the same arithmetic
 * and give bit-identical results.  Batches use variants 0 .. 5 (a batch of
 * channels set to 6 runs variant 0).  NH_EINVAL if the variant does not fit
 * the domain.  Variant 6 bounds its waits on the copies: an expired wait is
 * reported by the next nh_diagnostics / nh_diagnostics_read as NH_ETIMEOUT
 * (that launch's populations are incomplete). */
int nh_set_lb_variant(nh_ctx* ctx, int variant);

/* Select the FD kernels: 1 = fused (default): one 2.5D shared-memory kernel
 * for predictor + corrector + renormalisation and one for stress + force
 * (the stress never leaves the chip); 0 = one kernel per stage.  Same
 * arithmetic.  With the fused kernels the timing classes FD_PREDICT and
 * STRESS hold the two fused kernels. */
int nh_set_fd_variant(nh_ctx* ctx, int fused);

/* Autotuner: time every valid LB variant on the context's own domain (a few
 * launches each, CUDA events on stream; the state is not advanced), keep the
 * fastest and return its index in *chosen (may be NULL).  Synchronises. */
int nh_autotune(nh_ctx* ctx, void* stream, int* chosen);

/* Use CUDA graphs for whole dt_fd blocks (default on). */
int nh_set_graphs(nh_ctx* ctx, int on);

/* Diagnostics folded into the step (default on): every LB launch that
 * writes u and rho (the steps that feed an FD update or end a call) also
 * leaves per-block FP64 sums of the stored populations, max |u| and the
 * non-finite count, so that nh_diagnostics of that state reads only the
 * director (the energy, |n| and the tube sums) instead of every population,
 * u and rho again.  When that LB launch is followed by an FD update on the
 * fused kernels (nh_set_fd_variant 1), the stress kernel of the update also
 * leaves the director's partials (lattice Frank energy, |n| extrema and
 * non-finite count, tube sums about the previous centroids), so that
 * nh_diagnostics of the state right after the update runs only the final
 * reduction; a change of the centroids in between (nh_set_tubes, or the
 * tracking of an earlier nh_diagnostics) falls back to the director-only
 * pass.  Applies to F32 and F64 stores without obstacles and without
 * paper_order; the results equal the unfolded ones up to the summation
 * order.  0 turns it off (drops the cached graphs). */
int nh_set_diag_fold(nh_ctx* ctx, int on);

/* Bound the host-side waits of this context (nh_get_fields, nh_get_populations, nh_get_force,
 * nh_diagnostics, nh_diagnostics_read, nh_director_change): with seconds > 0 a wait that has
 * not seen the context's stream finish within that time returns NH_ETIMEOUT and leaves the
 * work running (the output buffers are then not written, and a later call waits again);
 * seconds <= 0 (the default) waits without a limit.  Failure detection for callers that must
 * not block on a GPU that stopped making progress; the paper has no counterpart. */
int nh_set_wait_limit(nh_ctx* ctx, double seconds);

/* Diagnostics for callers that cannot allocate device memory.
 *
 * nh_diagnostics needs a context, whose workspace the caller allocated in
 * advance.  Callers that have no such workspace and may not allocate one when
 * they need the numbers (a host application that hands over only its own
 * input and output buffers and forbids further device allocations, or a
 * time-critical loop that cannot afford cudaMalloc's implicit device
 * synchronisation) call this instead.  The paper has no counterpart: it is a
 * library convenience.
 *
 * Inputs are device pointers on the current device laid out as everywhere in
 * this header: populations f [19][N] (double for FP64/F64, float for FP32/F32;
 * the 16-bit stores are not accepted), director n [3][N], velocity u [3][N]
 * and density rho [N], in the precision of *p.  Output: out[6] on the device,
 *   out[0] = sum of the stored populations (the mass is out[0] + N when
 *            p->shifted, out[0] otherwise), out[1] = lattice Frank energy E_d
 *   (as in nh_diagnostics), out[2] = max |u|, out[3] = min |n|,
 *   out[4] = max |n|, out[5] = non-finite count (as nh_diag.nonfinite).
 * Asynchronous on stream (NULL = legacy default stream); no tube tracking.
 * The sums are deterministic for given inputs and pointer alignment: with
 * even nx and every field pointer aligned to two elements the reduction reads
 * x-pairs of sites (as nh_diagnostics does), otherwise single sites, so two
 * calls that differ only in alignment agree to rounding, not bit for bit.
 *
 * Scratch: a static device array inside the library (48 KiB per GPU that
 * loads it, held until the process exits); the call allocates nothing.  The
 * parameters get the checks of nh_create (NH_EINVAL otherwise).  Size limit, a
 * bound on the work of one call rather than on the scratch (at most 1024
 * reduction blocks stride over the domain): nx * ny * ceil(nz / 16) <=
 * NH_NOALLOC_MAX_ITEMS, else NH_EINVAL with a message in nh_last_error(NULL).  The first call on each device looks up
 * the array's device address with that device current; make that first call
 * before any stream capture.  All calls share the one array, which keeps the
 * last call's partial sums (each call overwrites what it reads, so nothing
 * needs clearing): calls that overlap on the GPU, from any thread or stream,
 * race on it and must be serialised by the caller. */
#define NH_NOALLOC_MAX_ITEMS (1024 * 256)
int nh_diagnostics_noalloc(const nh_params* p, const void* f, const void* n, const void* u, const void* rho,
                           double* out, void* stream);

/* ------------------------------------------------------------------------
 * Learned warm start (no counterpart in the paper): a 3D U-Net (4 levels, widths
 * 16/16/32/64, 394 419 parameters) that maps the extruded skyrmion ansatz and
 * the channel parameters (q0, Lz, W0) to the relaxed director; the plain
 * relaxation (nh_relax) continues from its prediction, which counts only if
 * that run ends where the relaxation from the ansatz ends.
 * Activations are BF16, accumulation FP32, convolutions run on the tensor
 * cores (the forward on the 5th-generation ones: tcgen05.mma with TMEM
 * accumulators); parameters, gradients and Adam moments are caller-owned FP32
 * device vectors in the layout: per conv layer W[tap][cout][cin] (tap = 9 kz + 3 ky
 * + kx, offsets -1..1) then bias[cout], layers enc1a enc1b enc2a enc2b enc3a
 * enc3b bota botb dec3a dec3b dec2a dec2b dec1a dec1b, then the head
 * W[3][16], bias[3].  Convolutions are periodic in x, y and zero-padded in z.
 * Fields are FP32 device arrays [batch][3][nx*ny*nz] (site order as above);
 * scalars [batch][3] = (q0, Lz, W0). */
typedef struct nh_unet nh_unet;
int64_t nh_unet_param_count(void);
/* A network instance for batch x nx x ny x nz inputs (nx, ny multiples of 8,
 * >= 16; nz a multiple of 8).  Its device workspace is caller-owned. */
int nh_unet_create(int batch, int nx, int ny, int nz, nh_unet** out);
int nh_unet_workspace_bytes(const nh_unet* net, size_t* bytes);
int nh_unet_bind(nh_unet* net, void* dev_ptr, size_t bytes);
/* Refresh the BF16 (and transposed BF16) weight copies from the FP32 params;
 * call after every parameter change. */
int nh_unet_set_params(nh_unet* net, const float* params, void* stream);
/* Forward pass; keeps the activations for nh_unet_backward.  n_out may be NULL. */
int nh_unet_forward(nh_unet* net, const float* params, const float* n_ansatz, const float* scalars, float* n_out,
                    void* stream);
/* Status of the network's tensor-core convolutions since the last call: the
 * forward convolutions bound every wait for their MMAs, and one that expired
 * leaves its output tile unwritten and raises a flag instead of hanging.
 * Synchronises stream; NH_ETIMEOUT (flag cleared) if a wait expired, else
 * NH_OK. */
int nh_unet_status(nh_unet* net, void* stream);
/* Loss mean |n - target|^2 over all sites into *loss (device float) and its
 * gradient with respect to the parameters into grad (overwritten), for the
 * activations of the last forward pass. */
int nh_unet_backward(nh_unet* net, const float* params, const float* n_ansatz, const float* target, float* grad,
                     float* loss, void* stream);
/* Copy the stored output of conv layer `layer` (0..13 in the order above) of
 * the last forward pass to out (FP32 device, channels-last [batch][z][y][x][c]). */
int nh_unet_activation(nh_unet* net, int layer, float* out, void* stream);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected, step >= 1). */
int nh_unet_adam(float* params, const float* grad, float* m, float* v, int64_t count, int step, float lr, void* stream);
void nh_unet_destroy(nh_unet* net);

/* Release the context (NULL-safe).  Does not free the caller's workspace. */
void nh_destroy(nh_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* NH_H */
