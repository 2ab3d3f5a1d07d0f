// rt_internal.h -- device data layout and kernel entry points shared by the
// translation units of the GB300 radiative-transfer library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "rt.h"

// Segment word: voxel id in the low 28 bits plus four flags.
#define RTK_RAYSTART 0x80000000u  // first segment of a characteristic
#define RTK_CORE 0x40000000u      // the characteristic starts on the core (I_in = B of this voxel)
#define RTK_RESTART 0x20000000u   // first segment after a transparent hole (I carries over)
#define RTK_PARA 0x10000000u      // parabolic weights for this segment (decided in FP64 from chi)
#define RTK_VOXMASK 0x0FFFFFFFu

// Long ownership lists are cut into chunks of this many entries (J-only gathers).
#define RTK_JCHUNK 1024
// Lists of at most this many entries are summed by one thread (J-only gathers).
#define RTK_JSHORT 64
// Upstream voxels whose derivative a characteristic carries while building the NN Lambda*.
#define RTK_NNW 16

#define RTK_END_EXIT 1
#define RTK_END_CORE 2
#define RTK_END_LOST 3

namespace rtk {

// Message returned by rt_last_error() on this thread (for other translation units).
void set_last_error(const char *msg);

// Grid geometry as seen by the geometry kernels (device pointers).
struct GeomDev {
    int coord, n1, n2, n3, nphi, inner_bc, nvox;
    const double *e1, *e2, *e3;
    const double *ct;          // cos(theta_j), j = 0..n2 (spherical)
    const double *ctm, *stm;   // cos/sin of theta mid-points (spherical)
    const double *cp, *sp;     // cos/sin of phi_k, k = 0..nphi-1
    const double *cpm, *spm;   // cos/sin of phi mid-points
};

// ---- geometry (geom.cu, compiled without FMA contraction) ----
// Marks every voxel hit by the characteristics of the boundary and core voxels.
cudaError_t geom_mark_boundary(const GeomDev &G, const double *dirs, int w0, int nw, uint32_t *hit, int words,
                               int *lost, uint32_t *cnt, cudaStream_t st);
// Coverage completion in increasing voxel order, one warp per solid angle.
cudaError_t geom_complete(const GeomDev &G, const double *dirs, int w0, int nw, uint32_t *hit, uint32_t *comp,
                          int words, int32_t *scratch, int cap, int *lost, uint32_t *cnt, cudaStream_t st);
// cnt[w n_vox + v]: cells of the backward (high 16 bits) and forward walk of the
// characteristic launched at voxel v for solid angle w, recorded by the two
// launch-set passes; the segment counts then need no walk of their own.
cudaError_t geom_gather_counts(int nvox, int64_t n_rays, const int32_t *ray_origin, const int32_t *ray_angle,
                               const uint32_t *cnt, int32_t *nseg, int32_t *nback, cudaStream_t st);
cudaError_t geom_count_rays(const GeomDev &G, const double *dirs, int n_ang, const uint32_t *comp, int words,
                            int32_t *counts, cudaStream_t st);
cudaError_t geom_list_rays(const GeomDev &G, const double *dirs, int n_ang, const uint32_t *comp, int words,
                           const int64_t *ang_ray_off, int32_t *ray_origin, int32_t *ray_angle, cudaStream_t st);
cudaError_t geom_write_segs(const GeomDev &G, const double *dirs, int64_t n_rays, const int32_t *ray_origin,
                            const int32_t *ray_angle, const int64_t *ray_off, const int32_t *nback, uint32_t *vox,
                            double *len64, float *len32, int *lost, cudaStream_t st);
int geom_scratch_cap(const GeomDev &G);
struct GeomF;
// Coverage completion guided by a float guess of each candidate's line (same
// launch set as geom_complete); pscr: 32 lists of cap per solid angle, stamp:
// n_vox per solid angle, zeroed before the call.
cudaError_t geom_complete_pred(const GeomDev &G, const GeomF &F, const double *dirs, int w0, int nw, uint32_t *hit,
                               uint32_t *comp, int words, int32_t *scratch, int32_t *pscr, int32_t *stamp, int cap,
                               int *lost, uint32_t *cnt, cudaStream_t st);

// ---- scans and small helpers (scan.cu) ----
// out[0] = 0, out[i+1] = out[i] + in[i]  (n + 1 outputs); tmp holds >= scan_tmp_elems(n) int64.
int64_t scan_tmp_elems(int64_t n);
cudaError_t scan_i32(const int32_t *in, int64_t *out, int64_t n, int64_t *tmp, cudaStream_t st);
cudaError_t gather_i64(const int64_t *src, const int64_t *idx, int64_t *dst, int n, cudaStream_t st);

// ---- ownership lists and gather (gather.cu) ----
// Scratch of the stable radix sort that builds the ownership lists: keys and
// values twice (cap entries each), digit histograms and their scan
// (256 * radix_tiles(cap) entries, plus scan_tmp_elems of that for tmp).
struct RadixScratch {
    uint32_t *kA, *kB;
    int32_t *vA, *vB;
    int32_t *hist;
    int64_t *off, *tmp;
    int64_t cap;
};
int64_t radix_tiles(int64_t n);
// Ownership (CSR) lists of one angle block: csr_off (nvox + 1) and perm_blk, every
// voxel's segment indices in increasing order.
cudaError_t csr_build(int nvox, const uint32_t *vox_blk, int64_t nseg_blk, int32_t *counts, int32_t *csr_off,
                      int32_t *perm_blk, int64_t *tmp, const RadixScratch &rs, cudaStream_t st);
cudaError_t csr_invL(int nvox, const int32_t *csr_off, const int32_t *perm_blk, const double *len64_blk,
                     const int64_t *ang_seg_off, int w0, int nw, int64_t seg_lo, double *invL, cudaStream_t st);
// Work units of one block's ownership lists (pieces of at most 32 entries):
// nu[v] units per voxel, ufirst = exclusive scan (nvox + 1), then per unit its voxel and first entry.
cudaError_t gather_units_build(int nvox, const int32_t *csr_off, int32_t *nu, int64_t *ufirst, int64_t *tmp,
                               cudaStream_t st);
cudaError_t gather_units_fill(int nvox, const int32_t *csr_off, const int64_t *ufirst, int32_t *urow, int32_t *ubeg,
                              cudaStream_t st);
// FP32 gather weights wt_w / L_wv per (solid angle, voxel).
cudaError_t make_wL32(int n_ang, int nvox, const double *invL, const double *wt, float *wL, cudaStream_t st);
// J, Lambda*, flux (Cartesian) of one block from the per-segment (l I, l lambda); first = 1 overwrites.
template <typename P>
cudaError_t gather_block(int nvox, const int32_t *csr_off, const int32_t *perm_blk, const P *buf,
                         const int64_t *ang_seg_off, int w0, int nw, int64_t seg_lo, const double *invL,
                         const float *wL32, const double *wt, const double *dirs, const int32_t *urow,
                         const int32_t *ubeg, const int64_t *ufirst, int64_t nunits, const int32_t *multi,
                         int nmulti, const int32_t *order, const int32_t *ulen, const int64_t *gbase,
                         const int32_t *sell, double *part, double *J, double *Lst, double *Fc, int first,
                         cudaStream_t st);
// Sliced-ELL layout of one block's work units: unit lengths, order (longest
// first), per-group width 32*max length (gw, to be scanned into gbase), fill.
cudaError_t sell_order(int64_t nunits, const int32_t *urow, const int32_t *ubeg, const int32_t *csr_off, int32_t *ulen,
                       int32_t *hist, int32_t *order, int32_t *gw, cudaStream_t st);
cudaError_t sell_fill(int64_t nunits, const int32_t *order, const int32_t *ulen, const int32_t *ubeg,
                      const int32_t *perm_blk, const int64_t *gbase, int32_t *sell, cudaStream_t st);
// Voxels of a block whose ownership list spans more than one unit: pos[nvox+1] = scan of the flags.
cudaError_t gather_multi_rows(int nvox, const int64_t *ufirst, int32_t *flag, int64_t *pos, int64_t *tmp,
                              int32_t *multi, cudaStream_t st);
// J-only gather tables of one block (see gather.cu): short lists in a
// sliced-ELL copy, long lists cut into chunks finished by their last warp.
struct GatherJTables {
    int64_t nshort = 0;            // voxels with short lists
    const int32_t *jorder = nullptr;  // short voxels, longest list first
    const int64_t *jgbase = nullptr;  // sliced-ELL group offsets (ceil(nshort/32)+1)
    const int32_t *jsell = nullptr;   // interleaved list entries
    int64_t nchunks = 0;
    const int32_t *crow = nullptr, *cbeg = nullptr, *clr = nullptr;  // per chunk: voxel, first entry, long-voxel index
    int nlong = 0;
    const int32_t *lfirst = nullptr;  // per long voxel: first chunk
    int *cnt = nullptr;               // per long voxel: chunks finished (returns to 0)
};
cudaError_t gatherJ_classify(int nvox, const int32_t *csr_off, int32_t *hist, int32_t *longflag, int32_t *nch,
                             cudaStream_t st);
cudaError_t gatherJ_short(int nvox, const int32_t *csr_off, int32_t *hist, int32_t *jorder, int64_t nshort, int32_t *gw,
                          cudaStream_t st);
cudaError_t gatherJ_sell(int64_t nshort, const int32_t *csr_off, const int32_t *jorder, const int32_t *perm_blk,
                         const int64_t *gbase, int32_t *sell, cudaStream_t st);
cudaError_t gatherJ_long(int nvox, const int32_t *csr_off, const int32_t *longflag, const int64_t *lpos,
                         const int64_t *cpos, int32_t *lrows, int32_t *lfirst, int32_t *crow, int32_t *cbeg,
                         int32_t *clr, cudaStream_t st);
template <typename T>
cudaError_t gather_J(int nvox, const int32_t *csr_off, const GatherJTables &t, const int32_t *perm_blk, const T *buf,
                     const int64_t *ang_seg_off, int w0, int nw, int64_t seg_lo, const float *wL32,
                     const double *invL, const double *wt, double *part, double *J, int first, cudaStream_t st);

// One batched J-gather work item: an angle block of one member (FP32 buffer).
// nbs = blocks of short lists, nbc = blocks of long-list chunks (8 chunks each).
struct GatherItem {
    GatherJTables t;        // tables of the grid's block, with this member's cnt slice
    const int32_t *off, *perm;
    const float *buf;
    const int64_t *ang_seg_off;
    const float *wL;
    const double *invL, *wt;
    double *part;           // this member's chunk sums
    double *J;              // this member's J
    int64_t seg_lo;
    int w0, nw, nvox, first;
    int64_t nbs, nbc;
};
cudaError_t gather_J_batch(const GatherItem *items, const int64_t *wpfx, int n_items, int64_t total,
                           unsigned long long *counter, int grid_blocks, cudaStream_t st);

// Ibar, Lbar of one solid angle whose segments are [s_lo, s_hi) of the block;
// the value of block segment s is buf[s - buf_base].
cudaError_t gather_angle_range(int nvox, const int32_t *csr_off, const int32_t *perm_blk, const void *buf,
                               int64_t buf_base, int fp32, int64_t s_lo, int64_t s_hi, const double *invL_w,
                               double *Ibar, double *Lbar, cudaStream_t st);
// Loads the kernels of gather_angle_range and march_block on the current device
// (modules load lazily otherwise, on their first launch).
cudaError_t gather_angle_preload();
cudaError_t march_block_preload();
cudaError_t pack_preload();
// *first_bad = min over bad voxels v of 4 v + c (c: 0 chi, 1 eps, 2 B), all ones if none (ali.cu).
cudaError_t check_opacity(int nvox, const double *chi, const double *eps, const double *B,
                          unsigned long long *first_bad, cudaStream_t st);
// Resolves the device address of the allocation-free path's static scratch on
// device dev (current) and loads the kernels that path launches (noalloc.cu).
int noalloc_prepare(int dev);
cudaError_t flux_local(const GeomDev &G, const double *Fc, double *F, cudaStream_t st);

// ---- ray march (march.cu) ----
// The same march writing only l I_k per segment (J without Lambda*: the ALI
// iteration reuses Lambda*, which depends on chi but not on S).
template <typename T, typename P>
cudaError_t march_block_J(const uint32_t *vox, const T *len, const int64_t *ray_off, int64_t r_lo, int64_t r_hi,
                          int64_t seg_lo, int64_t nseg, const P *chiS, const T *B, T I_outer, int homog, T *out,
                          int chunk, cudaStream_t st);
// FP64 march writing I_k (not l I_k) per segment: forward intensities for the adjoint.
cudaError_t march_block_I(const uint32_t *vox, const double *len, const int64_t *ray_off, int64_t r_lo, int64_t r_hi,
                          int64_t seg_lo, int64_t nseg, const double2 *chiS, const double *B, double I_outer, int homog,
                          double *out, int chunk, cudaStream_t st);
// FP64 weights of every segment for the chi given, as FP32 (E, alpha, beta + [run start] alpha, gamma).
cudaError_t coef_stream(const uint32_t *vox, const double *len64, const double *chi, int64_t nseg, float4 *cw,
                        cudaStream_t st);
// The same weights with the gather weight c_s = w_Omega l_s / L_{Omega v_s}
// folded in: (E c_s / c_{s-1} (c_s E at a characteristic start), c alpha,
// c beta, c gamma), so the march yields c_s I_s directly.
cudaError_t coef_stream_fold(const uint32_t *vox, const double *len64, const double *chi, const int64_t *ang_seg_off,
                             int n_ang, const double *wt, const double *invL, int nvox, int64_t nseg, float4 *cw,
                             cudaStream_t st);
// w_Omega l_s / L_{Omega v_s} of every segment (geometry only).
cudaError_t seg_weight(const uint32_t *vox, const double *len64, const int64_t *ang_seg_off, int n_ang,
                       const double *wt, const double *invL, int nvox, int64_t nseg, float *cg, cudaStream_t st);
// Streamed-weight J-only formal solution (fs_sw.cu): march of one angle block,
// J gather of one block.
struct SwMarch {
    using T = float;
    using W = float4;
    const uint32_t *vox;
    const float4 *cw;      // (E, alpha, beta, gamma) per segment (coef_stream)
    const float *cg;       // w_Omega l / L per segment (seg_weight)
    const int2 *bnd;       // bundle bounds of the block (sw_bundles), relative to seg_lo
    const int32_t *pos;    // NULL: out[s] in segment order; else out[pos[s]] (ownership-list order)
    int stages;            // 0: register prefetch of one tile; 2..4: shared-memory ring of that many tiles per warp
    int bulk;              // ring filled by bulk copies (1) or by per-lane 16-byte cp.async (0)
    int lookahead;         // register prefetch: S lookups of the next tile issued during this one (1)
    int fold;              // cw carries c = w l / L (c E_k / c_{k-1}, c alpha, c beta, c gamma); cg unused
    int *err;              // raised when a bounded wait of the staged march gives up
    int64_t seg_lo, nbundles;
    const float *S;        // S per voxel, FP32
    const float *B;
    float I_outer;
    int homog;
    float *out;            // c_s I_s per segment of the block
};
// FP64 weights of one segment (E, alpha, beta + [run start] alpha, gamma).
struct alignas(32) Wd4 {
    double x, y, z, w;
};
// The same march in FP64 (streamed FP64 weights and w l / L).
struct SwMarch64 {
    using T = double;
    using W = Wd4;
    const uint32_t *vox;
    const Wd4 *cw;
    const double *cg;
    const int2 *bnd;
    const int32_t *pos;
    int64_t seg_lo, nbundles;
    const double *S;
    const double *B;
    double I_outer;
    int homog;
    double *out;
};
struct SwGather {
    const int32_t *off, *jorder, *jsell, *crow, *cbeg, *clr, *lfirst, *perm;
    const int64_t *jgbase;
    int *cnt;
    double *part;
    const float *buf;      // c_s I_s of the block (FP32 march)
    const double *buf64;   // c_s I_s of the block (FP64 march); used when not NULL
    double *J;
    int64_t nshort, nchunks, nbs;
    int nlong, first;
};
// Blocked voxel order of the FP32 march's S lookups: words with the voxel field
// replaced by its blocked slot vblk[v] (flags RAYSTART, CORE, RESTART kept),
// and S, B scattered to their slots.
cudaError_t make_voxb(const uint32_t *vox, int64_t nseg, const int32_t *vblk, uint32_t *voxb, cudaStream_t st);
cudaError_t blk_scatter(int nvox, const int32_t *vblk, const float *S, const float *B, float *Sb, float *Bb,
                        cudaStream_t st);
cudaError_t sw_bundles(const int64_t *ray_off, int64_t r_lo, int64_t r_hi, int64_t seg_lo, int64_t nseg, int chunk,
                       int2 *bnd, cudaStream_t st);
cudaError_t march_sw_launch(const SwMarch &m, int coarsen, cudaStream_t st);
// coarsen: segments per lane, 1 or 2.
cudaError_t march_sw64_launch(const SwMarch64 &m, int coarsen, cudaStream_t st);
// FP64 weights and w l / L per segment for the FP64 streamed march.
cudaError_t coef_stream64(const uint32_t *vox, const double *len64, const double *chi, int64_t nseg, Wd4 *cw,
                          cudaStream_t st);
cudaError_t seg_weight64(const uint32_t *vox, const double *len64, const int64_t *ang_seg_off, int n_ang,
                         const double *wt, const double *invL, int nvox, int64_t nseg, double *cg, cudaStream_t st);
cudaError_t gather_sw_launch(const SwGather &t, cudaStream_t st);
// J from values in ownership-list order (march with pos): contiguous rows.
cudaError_t gather_rows_sw_launch(const SwGather &t, int nvox, cudaStream_t st);
// pos_blk[perm_blk[e]] = e for the n segments of a block.
cudaError_t inv_perm(const int32_t *perm_blk, int64_t n, int32_t *pos_blk, cudaStream_t st);
// One batched march work item: an angle block of one member (FP32, J only).
struct MarchItem {
    const uint32_t *vox;
    const float *len;
    const int64_t *ray_off;
    int64_t r_lo, r_hi, seg_lo, nseg;
    const float2 *cs;      // member (chi, S) per voxel
    const float *B;        // member B (FP32) for characteristics leaving the core
    const uint32_t *pbits; // member parabola choices, bit per segment of the grid
    float I_outer;
    float *out;            // l I per segment of the block (wave scratch)
};
// bpfx[i] = first bundle of item i (n_items + 1 entries); counter starts at 0.
cudaError_t march_batch(const MarchItem *items, const int64_t *bpfx, int n_items, int64_t total, int chunk, int homog,
                        unsigned long long *counter, int grid_blocks, cudaStream_t st);
cudaError_t march_block_bits(const uint32_t *vox, const float *len, const int64_t *ray_off, int64_t r_lo, int64_t r_hi,
                             int64_t seg_lo, int64_t nseg, const float2 *chiS, const float *B, float I_outer,
                             float2 *out, int chunk, const uint32_t *pbits, cudaStream_t st);
// FP64 march writing l I per segment with the parabola choices of a bitmask.
cudaError_t march_block_bits64J(const uint32_t *vox, const double *len, const int64_t *ray_off, int64_t r_lo,
                                int64_t r_hi, int64_t seg_lo, int64_t nseg, const double2 *chiS, const double *B,
                                double I_outer, int homog, double *out, int chunk, const uint32_t *pbits,
                                cudaStream_t st);
cudaError_t para_bits(const uint32_t *vox, const double *len64, const double *chi, int64_t nseg, int parabolic,
                      uint32_t *bits, cudaStream_t st);
// Parabola-guard decision per segment, taken once in FP64 from chi and the FP64
// lengths (dtau_{k+1} >= dtau_k / 2 and not the last node of a run), stored in
// the RTK_PARA bit so the FP32 and FP64 marches use identical interpolants.
cudaError_t mark_parabola(uint32_t *vox, const double *len64, const double *chi, int64_t nseg, int parabolic,
                          cudaStream_t st);
// One warp per bundle of whole characteristics holding about `chunk` segments.
template <typename T, typename P>
cudaError_t march_block(const uint32_t *vox, const T *len, const int64_t *ray_off, int64_t r_lo, int64_t r_hi,
                        int64_t seg_lo, int64_t nseg, const P *chiS, const T *B, T I_outer, int homog,
                        int parabolic, P *out, int chunk, cudaStream_t st);

// ---- nearest-neighbour Lambda* (nn.cu) ----
struct NnWalk {
    const uint32_t *vox;
    const double *len64;
    const int64_t *ray_off;
    const int32_t *ray_angle;
    int64_t r_lo, r_hi, seg_lo;  // characteristics of one angle block; segments relative to seg_lo
    const double *chi, *wt, *invL;
    const uint32_t *pbits;       // parabola choices of chi, bit per segment; NULL: the RTK_PARA bits of vox
    int nvox, n2, n3, sph;
    int8_t *slot;                // RTK_NNW per segment: neighbour slot of v_s or -1
    double *val;                 // RTK_NNW per segment: w l / L times dI_s/dS_u
};
cudaError_t nn_walk(const NnWalk &a, cudaStream_t st);
// An angle block's gather work units (its ownership lists cut into pieces of
// at most a fixed number of entries): unit voxel and first entry, per-voxel
// unit offsets, and the voxels with more than one unit.
struct NnUnits {
    const int32_t *urow, *ubeg;
    const int64_t *ufirst;
    int64_t nunits;
    const int32_t *multi;
    int64_t nmulti;
};
// L27 (+)= the block's per-segment (slot, value) records gathered per voxel;
// part: 27 doubles per unit.
cudaError_t nn_gather(int nvox, const int32_t *off, const int32_t *perm, const int8_t *slot, const double *val,
                      const NnUnits &un, double *part, double *L27, int first, cudaStream_t st);
cudaError_t nn_diag(int nvox, const double *L27, double *L, cudaStream_t st);
// Operator-splitting step (I - (1-eps) L*) x = y of the nearest-neighbour
// Lambda* (slot planes): BiCGSTAB on the Jacobi-preconditioned system (krylov
// != 0, at most kmax iterations) to a preconditioned residual <= jtol max |x|,
// then Jacobi sweeps until one changes x by <= jtol max |x| (at most jmax), all
// in one cooperative launch; synchronises st.  work: nn_os_work_elems(nvox)
// doubles.  *status: 0 converged, 1 not within jmax sweeps, 2 non-finite, 3 a
// grid-barrier wait gave up (x invalid); *x_out: the solution's buffer (in work).
// stall != 0 (test hook): one block skips its first barrier arrival, so every
// wait of the launch runs out and the status is 3.
struct NnOs {
    int nvox, sph, n1, n2, n3;
    const double *L27, *eps, *y;
    double *work;
    double jtol;
    int jmax, krylov, kmax;
    int stall;
};
int64_t nn_os_work_elems(int nvox);
cudaError_t nn_os_solve(const NnOs &o, cudaStream_t st, double **x_out, int *krylov_its, int *sweeps, int *status);
// The operator's 27 slot planes (L27[q nvox + v]) as rows: rows[27 v + q].
cudaError_t nn_rows(int nvox, const double *planes, double *rows, cudaStream_t st);
cudaError_t nn_rhs(int n, const double *S, const double *J, const double *eps, const double *B, double *y,
                   cudaStream_t st);
cudaError_t nn_rhs_corr(int n, const double *d, const double *Jd, const double *r, const double *eps, double *y,
                        cudaStream_t st);
cudaError_t nn_apply(int n, double *target, const double *x, const double *ref, double *slot,
                     unsigned long long *maxrel, cudaStream_t st);

// ---- ALI, Ng, refinement (ali.cu) ----
cudaError_t pack_chiS64(int nvox, const double *chi, const double *S, double2 *cs, cudaStream_t st);
// (chi, S) and B in FP32; S alone into S32 as well when S32 is not NULL.
cudaError_t pack_chiS32(int nvox, const double *chi, const double *S, const double *B, float2 *cs, float *B32, float *S32,
                        cudaStream_t st);
cudaError_t ali_update(int nvox, double *S, const double *J, const double *Lst, const double *eps, const double *B,
                       int use_lstar, double *hist_slot, unsigned long long *maxrel, cudaStream_t st);
// Order-2 Ng from four iterates (y0 newest), weights 1/wref^2 (wref = y0 when null);
// writes the extrapolation to out only when the 2x2 system is regular (coef[2] = 1).
cudaError_t ng_extrapolate(int nvox, const double *y0, const double *y1, const double *y2, const double *y3,
                           const double *wref, double *partial, double *coef, double *out, cudaStream_t st);
int ng_partial_elems(int nvox);
cudaError_t residual(int nvox, const double *S, const double *J, const double *Lst, const double *eps,
                     const double *B, int use_lstar, double *r, unsigned long long *maxrel, cudaStream_t st);
cudaError_t ali_correction(int nvox, double *delta, const double *Jd, const double *r, const double *Lst,
                           const double *eps, const double *S, int use_lstar, double *hist_slot,
                           unsigned long long *maxrel, cudaStream_t st);
cudaError_t add_inplace(int nvox, double *S, const double *delta, cudaStream_t st);
cudaError_t fill_const(int n, double *x, double v, cudaStream_t st);

}  // namespace rtk
