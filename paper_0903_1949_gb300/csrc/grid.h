// grid.h -- host-side state of one rt_grid (internal to the library).
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "rt_internal.h"

struct rt_grid {
    int device = 0;
    cudaStream_t st = nullptr;
    int coord = 0, n1 = 0, n2 = 0, n3 = 0, nvox = 0, n_ang = 0, nphi = 0;
    int inner_bc = 0, interp = 0, precision = 0, use_lstar = 1, ng = 1, refine_every = 32;
    double I_outer = 0.0;
    std::vector<double> h_e[3], h_dirs, h_wt;
    std::vector<void *> allocs;
    int64_t bytes = 0;
    rtk::GeomDev G{};
    double *d_dirs = nullptr, *d_wt = nullptr;
    int64_t n_rays = 0, n_seg = 0;
    std::vector<int64_t> h_ang_ray_off, h_ang_seg_off;
    int64_t *d_ang_seg_off = nullptr, *d_ray_off = nullptr;
    int32_t *d_ray_origin = nullptr, *d_ray_angle = nullptr;
    uint32_t *d_vox = nullptr;
    double *d_len64 = nullptr;
    float *d_len32 = nullptr;
    int ablk = 1, nblk = 0;
    std::vector<int> blk_w0, blk_nw;
    int64_t max_blk_seg = 0;
    int32_t *d_csr_off = nullptr, *d_perm = nullptr;
    double *d_invL = nullptr;
    // gather work units per block: unit voxel / first entry (concatenated), per-voxel unit offsets
    std::vector<int64_t> h_ubase, h_nunits;
    int32_t *d_urow = nullptr, *d_ubeg = nullptr;
    int64_t *d_ufirst = nullptr;
    double *d_part = nullptr;
    float *d_wL32 = nullptr;  // FP32 gather weights wt_w / L_wv
    std::vector<int64_t> h_mbase;     // per block: offset of its multi-unit voxel list
    int32_t *d_multi = nullptr;       // voxels whose list needs several units, per block
    // sliced-ELL copy of the ownership lists (coalesced gather reads), per block
    int32_t *d_ulen = nullptr, *d_order = nullptr, *d_sell = nullptr;
    int64_t *d_gbase = nullptr;
    std::vector<int64_t> h_goff, h_soff;  // per block offsets into d_gbase / d_sell
    std::vector<rtk::GatherJTables> jt;  // J-only gather tables per block
    double *d_partJ = nullptr;           // chunk sums of long lists (J-only gather)
    int lstar_prec = -1;                 // precision of the FS that computed d_L (-1: none since the last chi)
    void *d_segbuf = nullptr;
    double *d_chi = nullptr, *d_eps = nullptr, *d_B = nullptr, *d_S = nullptr;
    double *d_J = nullptr, *d_L = nullptr, *d_Fc = nullptr, *d_F = nullptr;
    double2 *d_cs64 = nullptr;
    float2 *d_cs32 = nullptr;
    float *d_B32 = nullptr;
    float *d_S32 = nullptr;  // S alone in FP32 (streamed-weight march)
    double *d_H = nullptr, *d_ng_part = nullptr, *d_ng_coef = nullptr;
    unsigned long long *d_maxrel = nullptr;
    double *d_r = nullptr, *d_delta = nullptr, *d_Jd = nullptr, *d_Ld = nullptr, *d_Fcd = nullptr, *d_Lkeep = nullptr;
    double *h_pin = nullptr;  // pinned scalars read back by the iteration control
    int *d_lost = nullptr;
    int lost = 0;
    double geom_ms = 0.0, geom_trace_ms = 0.0, geom_lists_ms = 0.0;
    int hs[4] = {0, 1, 2, 3};
    int nh = 0;
    std::vector<double> history;
    // kernel timing (rt_set_timing) and launch accounting
    bool timing = false;
    int timing_every = 1;             // 1: every march and gather launch; N > 1: every N-th march launch
    int64_t timing_count = 0;
    std::vector<cudaEvent_t> ev;      // event pool, two per timed launch
    size_t ev_used = 0;
    std::vector<int> ev_kind;         // 0 march, 1 gather, 2 NN OS-step solve
    std::vector<int64_t> ev_segs;
    int64_t launches = 0;
    int march_chunk = 512;  // segments per warp bundle (RT_TUNE_MARCH_CHUNK)
    std::vector<int64_t> ev_bytes;  // streamed DRAM bytes of each timed march launch
    // streamed-weight FP32 march (RT_TUNE_STREAMED_WEIGHTS)
    float4 *d_cw4 = nullptr;  // (E, alpha, beta, gamma) per segment for the current chi
    float *d_cg = nullptr;    // w_Omega l / L per segment
    int sw_enabled = 1;
    int sw_state = 0;         // 0 not allocated yet, 1 allocated, -1 allocation failed
    rtk::Wd4 *d_cw64 = nullptr;  // FP64 weights per segment (FP64 streamed march)
    double *d_cg64 = nullptr;    // FP64 w l / L per segment
    int sw64_state = 0;
    int sw64_coarsen = 2;     // segments per lane of the FP64 streamed march (RT_TUNE_MARCH64_COARSEN)
    bool cw64_ok = false;
    int pos_state = 0;        // list positions: 0 not tried, 1 allocated, -1 not available
    bool cw_ok = false;       // d_cw4 matches the current chi
    int sw_coarsen = 1;       // segments per lane (RT_TUNE_MARCH_COARSEN)
    int sw_overlap = 1;       // gather of block b on st2 while block b + 1 is marched (RT_TUNE_OVERLAP)
    int sw_scatter = 1;       // march stores in ownership-list order (RT_TUNE_SCATTER)
    int sw_stages = 0;        // shared-memory ring depth of the streamed-weight march (RT_TUNE_MARCH_STAGES)
    int sw_bulk = 0;          // ring filled by bulk copies instead of cp.async (RT_TUNE_MARCH_BULK)
    int sw_lookahead = 1;
    int sw_fold = 1;          // gather weight folded into the streamed weights (RT_TUNE_FOLD_WEIGHT)
    int cw_fold = -1;         // the fold state the current d_cw4 was built with
    // blocked voxel order of the FP32 streamed-weight march's S lookups (RT_TUNE_S_BLOCKED)
    int sblk = 1, sblk_state = 0;
    int32_t *d_vblk = nullptr;
    uint32_t *d_voxb = nullptr;
    float *d_S32b = nullptr, *d_B32b = nullptr;  // S lookups of the next tile issued during this one (register prefetch path)
    int *d_err = nullptr;     // raised by a bounded device wait that gave up
    int32_t *d_pos = nullptr; // list position of every segment within its block (NULL: not available)
    cudaStream_t st2 = nullptr;  // second stream of the overlapped gather (created on first use)
    cudaStream_t st3 = nullptr;  // second and third march streams (RT_TUNE_MARCH_STREAMS; created on first use)
    cudaStream_t st4 = nullptr;
    int sw_mstreams = 3;         // march streams of the overlapped J-only formal solution (RT_TUNE_MARCH_STREAMS)
    // the overlapped J-only formal solution as one CUDA graph (RT_TUNE_GRAPH): captured on
    // a private stream at the second call with the same arguments, replayed on st; two
    // argument sets are kept (the FP64 residual and the FP32 corrections of rt_solve)
    struct FsGraph {
        cudaGraphExec_t exec = nullptr;
        int prec = -1, homog = -1, calls = 0;
        const void *S = nullptr, *J = nullptr;
        int64_t launches = 0;    // kernel launches of one replay
        uint64_t used = 0;
    };
    int sw_graph = 1;
    cudaStream_t stc = nullptr;
    FsGraph fsg[2];
    uint64_t fsg_tick = 0;
    cudaEvent_t sev[10] = {};    // fork, join, march done x3, gather done x3, joins of st3 and st4
    int2 *d_bnd = nullptr;    // bundle bounds of every block for bnd_chunk
    // nearest-neighbour Lambda* (use_lstar = 2)
    double *d_L27 = nullptr;            // 27 per voxel
    double *d_nnx = nullptr, *d_nny = nullptr;  // Jacobi iterates (2 n) and right-hand side (n)
    unsigned long long *d_nnmx = nullptr;
    bool nn_ok = false;                 // d_L27 matches the current chi
    int nn_sweeps = 0;                  // Jacobi sweeps of the last OS step
    double nn_jtol = 1e-14;
    int nn_jmax = 100000;
    int nn_krylov = 1, nn_krylov_its = 0;  // BiCGSTAB before the Jacobi sweeps of the OS step
    int nn_stall = 0;                   // RT_TUNE_NN_TEST_STALL
    int64_t os_solves = 0, os_its = 0, os_sweeps = 0;  // OS-step counters since the timing reset
    std::vector<int64_t> h_bnd_off;
    int bnd_chunk = 0;
};

// FP32 formal solution of another opacity field on this grid's geometry (a
// batch member): (chi, S) packed in cs, B in B32, parabola choices in pbits.
// Writes J, Lambda* and the Cartesian flux sums Fc; returns an RT_ status.
int rt_grid_member_fs(rt_grid *g, const float2 *cs, const float *B32, const uint32_t *pbits, double *J, double *L,
                      double *Fc, cudaStream_t st);

// The grid's exact nearest-neighbour Lambda* (d_L27) for its current chi, built
// on first use after rt_set_opacity; returns an RT_ status.
int rt_grid_build_nn(rt_grid *g);

// FP64 J of another opacity field on this grid's geometry (a batch member):
// (chi, S) packed in cs64, B, parabola choices in pbits.  Runs on st.
int rt_grid_member_fs64J(rt_grid *g, const double2 *cs64, const double *B64, const uint32_t *pbits, double *J,
                         cudaStream_t st);

// The exact nearest-neighbour Lambda* (27 entries per voxel, slot q = 9 (di+1) +
// 3 (dj+1) + (dk+1), phi periodic) of another opacity field chi, with its
// parabola choices pbits (bit per segment, as para_bits), on this grid's
// geometry, into L27; runs on st and returns after it has drained.
int rt_grid_nn_lstar(rt_grid *g, const double *chi, const uint32_t *pbits, double *L27, cudaStream_t st);
