/*
 * rt.h -- C ABI of the GB300 long-characteristics radiative-transfer library.
 *
 * The library solves the scattering problem of Hauschildt & Baron, "A 3D
 * radiative transfer framework IV: spherical & cylindrical coordinate
 * systems": a formal solution along full (long) characteristics through a
 * spherical (r, theta_c, phi_c) or cylindrical (R, phi_c, z) voxel grid
 * (Sect. 2 "Method"), driven by an operator-splitting (ALI) iteration with a
 * diagonal approximate Lambda operator and Ng acceleration (Sect. 3.2.1), for
 * a grey continuum with coherent isotropic scattering
 * S = (1 - eps) J + eps B (Sect. 3.1, item 6).
 *
 * Conventions
 *  - Every call returns an int status (RT_OK = 0 on success).  On failure the
 *    grid is left unchanged unless stated otherwise, and rt_last_error()
 *    returns a message for the calling thread.
 *  - Voxel index v = (i*n2 + j)*n3 + k with (i, j, k) = (r, theta_c, phi_c) on
 *    the spherical grid and (R, phi_c, z) on the cylindrical grid.  Per-voxel
 *    arrays are contiguous doubles of length n_vox = n1*n2*n3.
 *  - `where` says whether a data pointer is host memory (RT_HOST, any pageable
 *    or pinned buffer) or device memory of the grid's GPU (RT_DEVICE, e.g. the
 *    data pointer of a CUDA tensor); device copies are ordered on the grid's
 *    stream.  Host pointers are only read or written during the call.
 *  - The library owns all device memory it allocates; the caller owns every
 *    buffer it passes.  A grid is not thread-safe: serialise calls on one grid.
 */
#ifndef RT_H
#define RT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define RT_OK 0
#define RT_EINVAL 1         /* invalid argument; nothing changed */
#define RT_ENOMEM 2         /* device or host allocation failed */
#define RT_ECUDA 3          /* a CUDA runtime call failed */
#define RT_ENOTCONVERGED 4  /* rt_solve reached max_iter */
#define RT_ETIMEOUT 5       /* a bounded device wait gave up (results of that call invalid) */
#define RT_EDEVICE 6        /* a kernel raised its error flag (e.g. a lost characteristic) */

/* coordinate systems (Sect. 3 and 4) */
#define RT_SPHERICAL 0
#define RT_CYLINDRICAL 1
/* inner boundary: I = B of the innermost voxel on characteristics leaving the
 * core (Sect. 3.1, spherical tests), or a transparent hole crossed without
 * opacity */
#define RT_CORE_B 0
#define RT_TRANSPARENT 1
/* precision of the formal solution: all FP64, or FP32 ray march with FP64
 * accumulation, ALI/Ng and FP64 iterative refinement */
#define RT_FP64 0
#define RT_MIXED 1
/* source-function interpolation along a characteristic */
#define RT_PARABOLIC 0
#define RT_LINEAR 1
/* approximate Lambda operator of the ALI iteration (Sect. 2, 3.2.1): none
 * (Lambda iteration), the diagonal, or the 3^3 nearest neighbours built
 * exactly (needs n_phi >= 3) */
#define RT_LSTAR_NONE 0
#define RT_LSTAR_DIAG 1
#define RT_LSTAR_NN 2
/* memory spaces */
#define RT_HOST 0
#define RT_DEVICE 1

typedef struct rt_grid rt_grid;

/* Problem description for rt_grid_create.  All arrays are copied. */
typedef struct rt_grid_desc {
    int coord;              /* RT_SPHERICAL or RT_CYLINDRICAL */
    int n[3];               /* voxels per axis, each >= 1 */
    const double *edges[3]; /* n[a]+1 strictly increasing edges per axis.
                             * spherical: r (r_0 > 0), theta_c in [0, pi] (first 0,
                             * last pi), phi_c with last - first = 2 pi.
                             * cylindrical: R (R_0 >= 0), phi_c (2 pi span), z. */
    int n_angles;           /* solid angles, >= 1 (Sect. 2: prescribed set) */
    const double *dirs;     /* n_angles x 3 unit direction vectors (p_x, p_y, p_z) */
    const double *weights;  /* n_angles quadrature weights, positive, sum 1 */
    int inner_bc;           /* RT_CORE_B or RT_TRANSPARENT */
    int interp;             /* RT_PARABOLIC (default) or RT_LINEAR */
    double I_outer;         /* incident intensity at the outer boundary (paper: 0) */
    int precision;          /* RT_FP64 or RT_MIXED */
    int use_lstar;          /* RT_LSTAR_DIAG (1): diagonal Lambda* ALI; RT_LSTAR_NN (2): nearest-neighbour
                               Lambda*; RT_LSTAR_NONE (0): plain Lambda iteration */
    int ng;                 /* 1: order-2 Ng acceleration every 4 ALI iterates */
    int refine_every;       /* RT_MIXED: maximum FP32 correction sweeps per FP64
                             * refinement (0 = default 32; the fixed point is the
                             * FP64 one whatever the value, which sets only how often
                             * an FP64 formal solution is paid for) */
    int angle_block;        /* solid angles per formal-solution block (0 = auto) */
    int device;             /* CUDA device ordinal */
    void *stream;           /* cudaStream_t for all work (NULL = legacy default) */
} rt_grid_desc;

/* Sizes and diagnostics of a grid (rt_get_info). */
typedef struct rt_info {
    int64_t n_vox;
    int64_t n_angles;
    int64_t n_rays;         /* characteristics over all solid angles */
    int64_t n_segments;     /* voxel crossings over all solid angles */
    int64_t device_bytes;   /* device memory held by the grid */
    int32_t n_blocks;       /* formal-solution angle blocks */
    int32_t angle_block;
    int32_t lost_rays;      /* characteristics that could not be tracked (0 expected) */
    int32_t precision;
    double geometry_ms;     /* wall time of the characteristic geometry at create */
    double geometry_trace_ms; /* of which: coverage, characteristics and crossing lists */
    double geometry_lists_ms; /* of which: ownership lists, inverse path lengths, gather units */
} rt_info;

/* Thread-local message for the last failed call (never NULL). */
const char *rt_last_error(void);

/* Build a grid: copies the description, computes on the GPU, for every solid
 * angle, the characteristics (one through each boundary voxel the direction
 * enters, one leaving each core voxel, then one through every voxel not yet
 * hit, Sect. 2) and their voxel crossing lists (exact shell / cone /
 * half-plane / cylinder / z-plane crossings), and the per-voxel ownership
 * lists used to gather J and Lambda* without atomics.  Fields start as
 * chi = 1, eps = 1, B = 0, S = 0.  *out is set only on RT_OK. */
int rt_grid_create(rt_grid **out, const rt_grid_desc *d);

/* Release every resource of the grid (NULL is accepted). */
int rt_grid_destroy(rt_grid *g);

int rt_get_info(const rt_grid *g, rt_info *info);

/* Set extinction chi (> 0, finite), thermalisation eps (in (0, 1]) and Planck
 * function B (>= 0, finite) per voxel (Sect. 3.1 items 5-6).  Every call
 * resets S := B, the start of the ALI iteration, and clears the Ng history; a
 * warm restart from an earlier S calls rt_set_S after it.  Input out of range
 * (NaN and infinities included) gives RT_EINVAL with the first offending
 * voxel in rt_last_error() and nothing changed: host arrays are checked on the
 * host, device arrays by a kernel on the grid's stream, which this call then
 * waits for. */
int rt_set_opacity(rt_grid *g, const double *chi, const double *eps, const double *B, int where);

/* Replace the source function S (warm restart). */
int rt_set_S(rt_grid *g, const double *S, int where);

/* Switch the grid between RT_FP64 and RT_MIXED (affects rt_formal_solution,
 * rt_ali_step and rt_solve; the crossing lists serve both). */
int rt_set_precision(rt_grid *g, int precision);

/* Runtime tuning knobs (rt_tune).  RT_TUNE_MARCH_CHUNK: crossing segments per
 * warp bundle in the ray march, 64..16384 (default 512); a bundle always holds
 * whole characteristics, so results do not depend on it beyond rounding. */
#define RT_TUNE_MARCH_CHUNK 1
/* RT_TUNE_STREAMED_WEIGHTS (default 1): the J-only march of the ALI iteration
 * streams per-segment weights (E, alpha, beta, gamma) evaluated once per chi
 * in FP64 and the gather weight w l / L: as FP32 for RT_MIXED (16 extra bytes
 * per segment of device memory with the gather weight folded in, see
 * RT_TUNE_FOLD_WEIGHT; 20 without), as FP64 for RT_FP64 (40 bytes), each
 * allocated at its first use; 0, or when that memory is not available: the
 * march evaluates the weights itself from chi and l.
 * RT_TUNE_MARCH_COARSEN: segments per lane of the streamed-weight march, 1
 * (default), 2 or 4.  RT_TUNE_OVERLAP (default 1): the J gather of angle block b
 * runs on a second stream of the library while block b + 1 is marched (the
 * grid's stream waits for it before the call returns its work); 0: both on
 * the grid's stream.  RT_TUNE_SCATTER (default 1): the streamed-weight march
 * stores each segment's value at its place in the voxel-ordered ownership
 * lists (4 more bytes of device memory per segment), so the J gather reads
 * contiguous rows; 0: the gather reads the values through the lists.  None of
 * these changes results beyond FP32 rounding. */
#define RT_TUNE_STREAMED_WEIGHTS 2
#define RT_TUNE_MARCH_COARSEN 3
#define RT_TUNE_OVERLAP 4
#define RT_TUNE_SCATTER 5
/* RT_TUNE_MARCH_STAGES: depth of a per-warp shared-memory ring of segment
 * tiles in the streamed-weight march, 2..4 (the ring holds the tile being
 * processed and the ones in flight); 0 (default): one tile prefetched in
 * registers.  RT_TUNE_MARCH_BULK: fill the ring with bulk copies and mbarrier
 * completion (1) or 16-byte cp.async copies spread over the lanes (0,
 * default).  A bounded mbarrier wait that gives up makes the calling
 * rt_ali_step / rt_solve return RT_ETIMEOUT. */
#define RT_TUNE_MARCH_STAGES 6
#define RT_TUNE_MARCH_BULK 7
/* RT_TUNE_NN_JTOL: the OS step of the nearest-neighbour Lambda* stops its
 * Jacobi sweeps when a sweep changes dS by at most 10^-value max |dS|,
 * value 1..15 (default 14: the step solved to FP64 rounding).  A looser step
 * changes the iterates, not the fixed point.  Inside the FP32 correction
 * sweeps of an RT_MIXED rt_solve, whose right-hand sides carry FP32 rounding,
 * the bound is max(10^-value, 1e-8); its FP64 residual steps use 10^-value. */
#define RT_TUNE_NN_JTOL 8
/* RT_TUNE_MARCH64_COARSEN: segments per lane of the FP64 streamed-weight
 * march, 1 or 2 (default). */
#define RT_TUNE_MARCH64_COARSEN 9
/* RT_TUNE_MARCH_LOOKAHEAD (default 1): the register-prefetch FP32 march loads
 * the voxel words two tiles ahead and issues the S lookups of the next tile
 * while it marches the current one; 0 looks S up at the start of each tile.
 * Both give bit-identical results. */
#define RT_TUNE_MARCH_LOOKAHEAD 10
/* RT_TUNE_S_BLOCKED (default 1): the FP32 streamed-weight march looks S up in
 * a copy ordered by 4 x 2 x 4 blocks of (i, j, k) voxels (one 128-byte line
 * each) through words that carry the blocked slot; 0 uses the grid's voxel
 * order.  Both give bit-identical results. */
#define RT_TUNE_S_BLOCKED 11
/* RT_TUNE_NN_KRYLOV (default 1): the OS step of the nearest-neighbour Lambda*
 * first runs BiCGSTAB on the Jacobi-preconditioned system until its
 * preconditioned residual (the change a Jacobi sweep would make) is below the
 * RT_TUNE_NN_JTOL bound, then Jacobi sweeps confirm that bound; 0 runs the
 * Jacobi sweeps alone.  Both stop on the same criterion, tested after every
 * iteration and sweep.  The whole OS step is one cooperative launch whose
 * blocks meet at grid barriers; a barrier wait that gives up after a second
 * makes the calling rt_ali_step / rt_solve / rt_adjoint return RT_ETIMEOUT
 * with S not updated by that step. */
#define RT_TUNE_NN_KRYLOV 12
/* RT_TUNE_MARCH_STREAMS (default 3): with RT_TUNE_OVERLAP, the marches of
 * consecutive angle blocks alternate between 1, 2 or 3 streams (the FP64 march
 * uses at most 2), so that the next block's march can start while the last CTAs
 * of the previous one finish; with 3 the FP32 per-segment values are triple
 * buffered.  The gathers still run in block order on their own stream: all give
 * bit-identical J. */
#define RT_TUNE_MARCH_STREAMS 13
/* RT_TUNE_GRAPH (default 1): the overlapped J-only formal solution of the
 * iteration is captured as one CUDA graph at its second call with the same
 * precision, S and J, and replayed from then on (any rt_tune or
 * rt_set_opacity drops it; not used while rt_set_timing is on).  Bit-identical
 * J. */
#define RT_TUNE_GRAPH 15
/* RT_TUNE_GEOM_PREDICT (default 0), set with g = NULL for the grids created
 * afterwards: the coverage completion of the launch set walks each candidate
 * voxel's characteristic in float first and traces exactly (FP64) only
 * candidates that no earlier chosen candidate's guessed line crosses; the
 * decisions stay the exact serial ones, so the launch set and the crossing
 * lists are the same as with 0.  Other knobs need a grid. */
#define RT_TUNE_GEOM_PREDICT 16
/* RT_TUNE_FOLD_WEIGHT (default 1): the FP32 streamed-weight march carries the
 * gather weight c = w_Omega l / L of each segment inside its four weights
 * (it marches c_k I_k: E c_k / c_{k-1}, c alpha, c beta, c gamma, formed once per
 * chi: optical depths and c in FP64, the weights in FP32 on the FP32 pipe), so
 * the per-segment c stream is not read: 24 instead of 28 bytes per segment.
 * Register-prefetch march only (RT_TUNE_MARCH_STAGES 0); agrees with 0 (whose
 * weights are evaluated in FP64 and rounded) to FP32 rounding. */
#define RT_TUNE_FOLD_WEIGHT 17
/* RT_TUNE_NN_TEST_STALL (test hook, default 0): 1 makes one block of the next
 * nearest-neighbour OS step leave out its first barrier arrival, so every
 * bounded wait of that launch runs out: the call returns RT_ETIMEOUT, S is
 * not updated and the knob is 0 again.  It tests the bounded waits without a
 * device fault. */
#define RT_TUNE_NN_TEST_STALL 18
int rt_tune(rt_grid *g, int knob, int value);

/* Formal solution from the current S with the grid's precision: J, the
 * diagonal Lambda* and the flux vector per voxel (Sect. 2, 3.2). */
int rt_formal_solution(rt_grid *g);

/* Formal solution with an explicit precision (RT_FP64 or RT_MIXED, i.e. the
 * FP32 march) and optionally homogeneous boundaries (homog = 1: every incoming
 * intensity zero, so J = Lambda S). */
int rt_formal_solution_ex(rt_grid *g, int precision, int homog);

/* One ALI iteration: formal solution, S <- S + [(1-eps) J + eps B - S] /
 * (1 - (1-eps) Lambda*), and Ng extrapolation when four iterates have
 * accumulated (if enabled).  *max_rel_dS (may be NULL) receives
 * max_v |dS| / |S_new| of the update.  Lambda* depends on chi and the path
 * lengths only, so it is computed by the first iteration after rt_set_opacity
 * (or taken from an earlier rt_formal_solution of the same or higher
 * precision) and reused; later iterations compute J alone and leave the flux
 * of rt_get_flux unchanged (call rt_formal_solution for the flux of S). */
int rt_ali_step(rt_grid *g, double *max_rel_dS);

/* Iterate to max rel dS < tol.  RT_FP64: plain ALI(+Ng) with the FP64 formal
 * solution.  RT_MIXED: FP64 formal solutions give the exact residual
 * r = (1-eps) J + eps B - S, FP32 correction sweeps (ALI + Ng on the
 * homogeneous problem; at most refine_every of them, default 32) solve for
 * the update, repeated until the residual meets tol.  *iters (may be NULL) receives the number of formal solutions
 * of the precision that drives convergence (FP64 ones for RT_FP64 and the
 * total for RT_MIXED).  Returns RT_ENOTCONVERGED at max_iter. */
int rt_solve(rt_grid *g, double tol, int max_iter, int *iters);

/* Per-voxel results (n_vox doubles; flux: n_vox x 3 in the local basis
 * (r, theta, phi) or (R, phi, z) at the voxel centre). */
int rt_get_J(const rt_grid *g, double *out, int where);
int rt_get_S(const rt_grid *g, double *out, int where);
int rt_get_Lstar(const rt_grid *g, double *out, int where);
/* Nearest-neighbour Lambda* of the current chi (grid created with
 * use_lstar = RT_LSTAR_NN; built on demand, in FP64, and reused until
 * rt_set_opacity): out27[27 v + q] = dJ_v/dS_u for the voxel u at offset
 * (q/9 - 1, (q/3)%3 - 1, q%3 - 1) of v in (i, j, k), the phi index periodic;
 * 0 where that offset leaves the grid.  n_vox x 27 doubles, caller-owned.
 * With RT_LSTAR_NN the ALI step solves (I - (1-eps) L*) dS = (1-eps) J +
 * eps B - S until a Jacobi sweep would change dS by at most 1e-14 max |dS|
 * (BiCGSTAB on the Jacobi-preconditioned system, then confirming sweeps; see
 * RT_TUNE_NN_KRYLOV and RT_TUNE_NN_JTOL), and rt_get_Lstar returns the
 * diagonal. */
int rt_get_Lstar_nn(rt_grid *g, double *out27, int where);
int rt_get_flux(const rt_grid *g, double *out3, int where);

/* Convergence history of the last rt_solve / rt_ali_step sequence: up to max
 * values of max rel dS, *n receives the count stored. */
int rt_get_history(const rt_grid *g, double *hist, int max, int *n);

/* Gradients of a loss L(S, J, F) evaluated at the converged source function,
 * with respect to the per-voxel chi, eps and B that rt_set_opacity set.  The
 * fixed point S = (1 - eps) J(S; chi, B) + eps B of the ALI iteration (Sect.
 * 3.2.1, with J from the formal solution of Sect. 2) is differentiated
 * implicitly: the adjoint source function lam solves
 *   lam = gS + Lambda^T gJ + Lambda_F^T gF + Lambda^T ((1 - eps) lam)
 * by the same preconditioned iteration as the forward ALI (run to
 * max|d lam| <= tol max|lam|, at most max_iter sweeps), where Lambda^T is the
 * ray march run backwards along every characteristic: with the diagonal
 * Lambda* (use_lstar = RT_LSTAR_DIAG) each sweep divides the residual by
 * 1 - (1-eps) Lambda*; with RT_LSTAR_NN it solves (I - Lambda*_NN^T diag(1-eps)) x
 * = residual, the transpose of the forward OS step, by the same BiCGSTAB and
 * Jacobi sweeps (the NN operator is built for the grid's chi if it is not yet),
 * which keeps the sweep count small at eps << 1; then
 *   dL/dchi = (dJ/dchi)^T (gJ + (1-eps) lam) + (dF/dchi)^T gF,
 *   dL/dB   = eps lam + (dJ/dB)^T (gJ + (1-eps) lam) + (dF/dB)^T gF,
 *   dL/deps = lam (B - J).
 * The paper computes no gradients; this operation is an extension of it.
 * Inputs: dL_dS, dL_dJ (n_vox doubles) and dL_dF (n_vox x 3, the local basis
 * of rt_get_flux); any may be NULL (zero).  Outputs dchi, deps, dB: n_vox
 * doubles each, caller-owned, all in the memory space `where`.  The
 * derivatives hold at the grid's current S (call rt_solve first), in FP64
 * whatever the grid's precision; the parabola-or-linear choice of every
 * segment is held fixed.  Side effect: J, Lambda* and the flux of the grid
 * are recomputed in FP64 from the current S.  *iters (may be NULL) receives
 * the adjoint sweeps taken.  Returns RT_ENOTCONVERGED (outputs written from
 * the last iterate) when max_iter is reached, RT_EINVAL for a NULL grid or
 * output, bad `where`, tol <= 0, max_iter < 1 or use_lstar = 0, RT_ENOMEM when
 * its work arrays (about 6 n_vox + 3 segments-per-block doubles) cannot be
 * allocated. */
int rt_adjoint(rt_grid *g, const double *dL_dS, const double *dL_dJ, const double *dL_dF, double tol, int max_iter,
               double *dchi, double *deps, double *dB, int where, int *iters);

/* Crossing lists of solid angle omega (host buffers).  Call with NULL arrays
 * to get *n_rays and *n_seg, then with buffers of those sizes:
 * ray_off[n_rays+1] (segment offsets), ray_origin[n_rays] (voxel whose centre
 * the characteristic passes), ray_core[n_rays] (1: starts on the core),
 * vox[n_seg], len[n_seg] (FP64 path lengths), restart[n_seg] (1: first
 * segment after a transparent hole).  Rays are listed boundary voxels first,
 * then core voxels, then coverage completions, each in voxel order. */
int rt_get_crossings(const rt_grid *g, int omega, int64_t *n_rays, int64_t *n_seg, int32_t *ray_off,
                     int32_t *ray_origin, int32_t *ray_core, int32_t *vox, double *len, uint8_t *restart);

/* Path-length averaged intensity Ibar and Lambda* element of each voxel for
 * the n listed solid angles (out arrays n x n_vox), from the current S, with
 * the given precision.  Used to compare single solid angles. */
int rt_fs_angles(rt_grid *g, const int32_t *omegas, int n, int precision, double *Ibar, double *Lbar,
                 int where);

/* Formal solution of one solid angle for callers that cannot allocate device
 * memory at call time: code running inside another framework's memory pool or
 * under a device-memory budget that is already fully handed out, or a thread
 * that must not take the CUDA allocator's locks.  The paper has no counterpart;
 * this is a library service.  The call allocates nothing: its per-segment
 * scratch is a static device array of 16 MiB inside the library, so the solid
 * angle must have at most 1 Mi crossing segments in RT_FP64 or 2 Mi in
 * RT_MIXED (else RT_EINVAL with the counts in rt_last_error()).  The grid must
 * exist: rt_grid_create (which allocates anyway) looks up the array's device
 * address on its device, which is when the array is placed there (the
 * library's code loads lazily) and held until the process exits, and loads the
 * kernels this call launches; the call itself only reads that cached address.
 * Ibar and Lbar are caller-owned DEVICE buffers of n_vox doubles that receive
 * what rt_fs_angles returns for this angle, from the current S (the same
 * kernels on this angle's segments alone, so the two agree to rounding, not bit
 * for bit: rt_fs_angles marches the angle's whole block, which groups the
 * characteristics into warp bundles differently).  Work is queued on the
 * grid's stream and not waited for.  All calls share the one scratch array,
 * which keeps the last call's contents (nothing in it needs clearing: every
 * entry read is written first); calls whose GPU work overlaps (other streams,
 * other threads) race.  Not async-signal-safe: never call it from a signal
 * handler. */
int rt_fs_angle_noalloc(rt_grid *g, int omega, int precision, double *Ibar, double *Lbar);

/* FP64 fused multiply-add throughput of a device in flop/s (2 per FMA), the
 * denominator of the FP64 path's roofline (measurement service; the paper
 * has no counterpart): a grid that fills every SM runs independent FMA
 * chains, timed with CUDA events; *ms_per_launch is one launch's mean time.
 * Takes the device briefly (about a tenth of a second) on a stream of its own. */
int rt_measure_fp64_rate(int device, double *flops_per_s, double *ms_per_launch);

/* ---- batches: many opacity fields solved together ----------------------
 * A batch holds n_members problems (wavelengths of a line profile or
 * separate models, cf. the paper's wavelength "clusters", Sect. 3.2.2), each
 * on one of n_grids existing grids of possibly different sizes (member_grid[m]
 * gives its grid).  Members share their grid's characteristics but have their
 * own chi, eps, B, S, J and Lambda*.  One batch iteration applies, to every
 * member at once, the diagonal-Lambda* ALI update after an FP32 J-only formal
 * solution (no Ng); it runs as a single CUDA graph of persistent march and
 * gather launches that mix all members and grids.  The batch uses `stream` (or
 * a stream of its own when NULL); its grids must not be used on other streams
 * while the batch works, and must outlive it. */
typedef struct rt_batch rt_batch;

int rt_batch_create(rt_batch **out, rt_grid *const *grids, int n_grids, int n_members, const int32_t *member_grid,
                    void *stream);
int rt_batch_destroy(rt_batch *b);

/* Opacity of member m (n_vox of its grid each; validated like rt_set_opacity);
 * sets its S to B and computes its parabola choices and Lambda* (one full FP32
 * formal solution).  Every member must be set before the first iteration. */
int rt_batch_set_member(rt_batch *b, int m, const double *chi, const double *eps, const double *B, int where);

/* One iteration of every member; max_rel_dS (may be NULL) gets n_members values. */
int rt_batch_ali_step(rt_batch *b, double *max_rel_dS);

/* Solve every member to its fixed point in mixed precision with FP64
 * refinement (as rt_solve does with RT_MIXED for one grid): an FP64 formal
 * solution of each member still iterating gives its exact residual
 * r = (1-eps) J + eps B - S; up to 16 batched FP32 J-only sweeps (one CUDA
 * graph, no incoming radiation) then solve for the correction D of S with the
 * diagonal Lambda* (D <- D + [(1-eps) J(D) + r - D] / (1 - (1-eps) Lambda*)),
 * stopping early once a sweep changes D by < tol/100 relative, and S += D.  A
 * member is done when the ALI update its FP64 residual asks for is below tol
 * (max |dS| / |S + dS|); its S is then left alone.  The fixed point is the
 * FP64 one.  max_iter bounds the formal solutions (FP64 and FP32 alike); iters
 * (may be NULL) gets, per member, the formal-solution count at which it was
 * found done (0 if never).  RT_ENOTCONVERGED when some member is not done. */
int rt_batch_solve(rt_batch *b, double tol, int max_iter, int32_t *iters);

/* Member m's S (what = 0), J (1) or Lambda* (2). */
int rt_batch_get(const rt_batch *b, int m, int what, double *out, int where);

/* Times one batch iteration for several bundle sizes (rays per warp) and
 * persistent grid sizes, keeps the fastest and reports it (any output may be
 * NULL).  Member S is restored afterwards. */
int rt_batch_autotune(rt_batch *b, int32_t *chunk_out, int32_t *grid_out, double *ms_out);

/* ---- Two-level-atom line transfer (Sect. 3.1, 3.2.2) ----
 *
 * A line sampled at n_freq frequencies on one grid: profile phi[k] >= 0 and
 * quadrature weights wq[k] >= 0 with sum_k wq[k] phi[k] = 1 (checked to 1e-10,
 * else RT_EINVAL).  At frequency k the opacity is chi_k = chi_c + chi_l phi_k
 * and the source function mixes a thermal continuum (S_c = B) and the line,
 *     S_k = (chi_c B + chi_l phi_k S_l) / chi_k,
 *     S_l = (1 - eps_l) Jbar + eps_l B,   Jbar = sum_k wq_k phi_k J_k.
 * The problem is an rt_batch whose member k is frequency k (rt_batch_get
 * reads S_k, J_k and Lambda*_k; rt_batch_autotune tunes it and restores S_l;
 * rt_batch_set_member, rt_batch_ali_step and rt_batch_solve are RT_EINVAL on
 * it).  One iteration, a single CUDA graph: S_k from S_l for every k, the
 * n_freq FP32 J-only formal solutions, then Jbar (frequencies summed in
 * ascending order, FP64) and the ALI update of S_l with the frequency-averaged
 * diagonal operator Lbar* = sum_k wq_k phi_k (chi_l phi_k / chi_k) Lambda*_k:
 *     S_l <- S_l + [(1 - eps_l) Jbar + eps_l B - S_l] / (1 - (1 - eps_l) Lbar*).
 * Lambda*_k comes from one full FP32 formal solution per frequency.
 * use_lstar = RT_LSTAR_NN (needs n_phi >= 3) replaces the diagonal operator by
 * the exact dJbar_v / dS_l,u on the 3 x 3 x 3 index neighbourhood of v,
 *     Lbar*_vu = sum_k wq_k phi_k Lambda*_NN,k,vu (chi_l phi_k / chi_k)_u,
 * built once per rt_line_set from each frequency's exact nearest-neighbour
 * Lambda* (as rt_get_Lstar_nn), and each iteration solves
 * (I - (1 - eps_l) Lbar*) dS_l = (1 - eps_l) Jbar + eps_l B - S_l after the
 * graph, until a Jacobi sweep would change dS_l by at most 1e-14 max |dS_l|
 * (BiCGSTAB, then confirming sweeps, as rt_ali_step).  use_lstar
 * other than RT_LSTAR_DIAG / RT_LSTAR_NN is RT_EINVAL.  ng = 1 applies order-2
 * Ng extrapolation to S_l whenever four iterates have accumulated since the
 * last one (as rt_ali_step; rt_line_solve skips it once tol is met); ng other
 * than 0 / 1 is RT_EINVAL.
 * The grid must outlive the problem; it is used on the problem's stream. */
int rt_line_create(rt_batch **out, rt_grid *g, int n_freq, const double *phi, const double *wq, int use_lstar, int ng,
                   void *stream);

/* chi_c, chi_l (>= 0, with chi_c + chi_l phi_k > 0 for every k), eps_l in
 * (0, 1] and B >= 0, n_vox each (host arrays validated, device arrays not);
 * computes every frequency's parabola choices, Lambda*_k and Lbar*, and sets
 * S_l = B.  Required before the first step. */
int rt_line_set(rt_batch *b, const double *chi_c, const double *chi_l, const double *eps_l, const double *B,
                int where);

/* One iteration (then Ng, if enabled and due); max_rel_dSl (may be NULL) gets
 * max_v |dS_l| / |S_l| of the ALI update. */
int rt_line_step(rt_batch *b, double *max_rel_dSl);

/* Iterate until max rel dS_l < tol (RT_ENOTCONVERGED after max_iter);
 * iters (may be NULL) gets the iterations done. */
int rt_line_solve(rt_batch *b, double tol, int max_iter, int32_t *iters);

/* S_l (what = 0), Jbar of the last iteration (1) or the diagonal Lbar* (2),
 * n_vox values; of a nearest-neighbour line also its Lbar* (3), 27 n_vox values
 * in the slot order of rt_get_Lstar_nn (RT_EINVAL on a diagonal line). */
int rt_line_get(const rt_batch *b, int what, double *out, int where);

/* ---- Formal solution over a large solid-angle set (angle-resolution study) ----
 *
 * J and the flux (local basis, as rt_get_flux) of the field (chi, S, B) for the
 * grid and solid-angle set of d, processed angles_per_chunk solid angles at a
 * time so that only one chunk's characteristics are held (Sect. 3.1-3.2: the
 * flux vectors of the outermost voxels with up to 512^2 solid angles).  Each
 * chunk is a temporary grid built from d (its weights renormalised to 1),
 * solved with `precision` (RT_FP64: FP64 march and gather; RT_MIXED: FP32),
 * and its J and flux are added with the chunk's share of the total weight;
 * d->use_lstar, d->ng and d->refine_every are ignored.  chi, S, B: n_vox each
 * (host arrays validated as by rt_set_opacity); J: n_vox, F: 3 n_vox, all on
 * `where`.  Uses d->device and d->stream.  Chunk geometry dominates the time
 * (larger chunks amortise it better, within device memory).  Errors of a
 * chunk's grid are returned as they are; the outputs are written only on RT_OK. */
int rt_fs_sweep(const rt_grid_desc *d, int angles_per_chunk, const double *chi, const double *S, const double *B,
                int precision, double *J, double *F, int where);

/* Device timing of the hot kernels.  rt_set_timing(g, 1) resets the counters
 * and brackets every ray-march and gather launch of later calls with CUDA
 * events on the stream each runs on; rt_set_timing(g, N) with N > 1 brackets
 * only every N-th ray-march launch (less event overhead; the march sums then
 * cover that sample, the gather sums stay 0); rt_set_timing(g, 0) stops
 * recording (counters are kept).  N < 0 is RT_EINVAL.  rt_get_timing
 * synchronises the stream and returns the sums. */
typedef struct rt_timing {
    double march_ms;          /* summed event time of ray-march launches */
    double gather_ms;         /* summed event time of ownership-gather launches */
    int64_t march_launches;
    int64_t gather_launches;
    int64_t march_segments;   /* crossing segments processed by the timed march launches */
    int64_t kernel_launches;  /* every kernel this library launched on the grid since the reset */
    int64_t march_bytes;      /* DRAM bytes the timed march launches stream by design (per segment:
                                 8 FP32, 12 FP64; streamed-weight FP32 24, or 20 without RT_TUNE_SCATTER,
                                 4 more without RT_TUNE_FOLD_WEIGHT; streamed-weight FP64 48 / 44) */
    double os_ms;             /* summed event time of the nearest-neighbour OS-step solves (timing 1 only) */
    int64_t os_solves;        /* OS-step solves since the reset (counted at any timing setting) */
    int64_t os_krylov_its;    /* their BiCGSTAB iterations */
    int64_t os_sweeps;        /* their Jacobi sweeps */
} rt_timing;

int rt_set_timing(rt_grid *g, int enable);
int rt_get_timing(rt_grid *g, rt_timing *t);

#ifdef __cplusplus
}
#endif
#endif /* RT_H */
