/*
 * rt_oracle.c -- serial FP64 CPU oracle for the long-characteristics formal
 * solution and the diagonal-Lambda* operator-splitting (ALI) iteration with
 * Ng acceleration on spherical (r, theta_c, phi_c) and cylindrical
 * (R, phi_c, z) voxel grids (Hauschildt & Baron, "A 3D radiative transfer
 * framework IV", Sect. 2 "Method", Sect. 3.1 "Testing environment").
 *
 * TEST INFRASTRUCTURE.  This file is the slow, obviously-correct reference the
 * CUDA path is checked against.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark load it; the product library never does, and
 * the two share no code.  Everything is plain double precision, one voxel,
 * one ray, one segment at a time, in the order the method states.  It must be
 * compiled with floating-point contraction disabled (-ffp-contract=off) so
 * that every + - * / sqrt is a single IEEE-rounded operation.
 *
 * Where the paper defers to Papers I-II or is silent, this file states the
 * reading it takes beside the code that takes it: the geometry rules at
 * voxel_centre, quad_roots, the crossing functions and trace; the
 * formal-solution weights and their series at orc_coeffs; the parabola guard
 * at use_parabola; the launch set at orc_angle_geometry; the ALI update at
 * orc_ali_update; Ng at orc_ng.
 *
 * Voxel index: v = (i*n2 + j)*n3 + k, with (i,j,k) = (r,theta,phi) on the
 * spherical grid and (R,phi,z) on the cylindrical grid.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_SPH 0
#define ORC_CYL 1
#define ORC_CORE_B 0
#define ORC_TRANSPARENT 1
#define ORC_PARABOLIC 0
#define ORC_LINEAR 1

#define END_EXIT 1
#define END_CORE 2
#define END_LOST 3

static const double INF = 1.0 / 0.0;
static const double FOUR_PI = 12.566370614359172953850573533118;

typedef struct {
    int vox;
    double t_in, t_out;
    int after_hole; /* a transparent hole lies between this cell and the previous cell of the trace */
} cell_t;

typedef struct {
    int ready;
    int n_rays, n_seg, n_lost;
    int *ray_off;    /* n_rays + 1 */
    int *ray_origin; /* voxel through whose centre the characteristic runs */
    int *ray_kind;   /* 0 outer-boundary voxel, 1 inner-boundary voxel, 2 coverage completion */
    int *ray_core;   /* 1: the characteristic starts on the core (I_in = B of its first voxel) */
    int *vox;
    double *len;
    unsigned char *restart; /* 1: first segment after a transparent hole */
} angle_t;

typedef struct {
    int coord, n1, n2, n3, nvox, nphi;
    double *e1, *e2, *e3;
    int inner_bc, interp;
    double I_outer;
    int n_ang;
    double *dir, *wt;
    double *ct;        /* cos(theta_j), j = 0..n2 (spherical only) */
    double *ctm, *stm; /* cos, sin of theta mid-points (spherical only) */
    double *cp, *sp;   /* cos, sin of phi_k, k = 0..nphi-1 */
    double *cpm, *spm; /* cos, sin of phi mid-points */
    angle_t *ang;
} orc_grid;

/* ------------------------------------------------------------------ grid -- */

static int vox_id(const orc_grid *g, int i, int j, int k) { return (i * g->n2 + j) * g->n3 + k; }

static void vox_ijk(const orc_grid *g, int v, int *i, int *j, int *k)
{
    *k = v % g->n3;
    *j = (v / g->n3) % g->n2;
    *i = v / (g->n3 * g->n2);
}

static double *dup_array(const double *a, int n)
{
    double *b = (double *)malloc(sizeof(double) * (size_t)n);
    memcpy(b, a, sizeof(double) * (size_t)n);
    return b;
}

static void free_angle(angle_t *A)
{
    free(A->ray_off); free(A->ray_origin); free(A->ray_kind); free(A->ray_core);
    free(A->vox); free(A->len); free(A->restart);
    memset(A, 0, sizeof(*A));
}

void orc_destroy(orc_grid *g)
{
    if (!g) return;
    for (int w = 0; w < g->n_ang; ++w) free_angle(&g->ang[w]);
    free(g->ang);
    free(g->e1); free(g->e2); free(g->e3); free(g->dir); free(g->wt);
    free(g->ct); free(g->ctm); free(g->stm); free(g->cp); free(g->sp); free(g->cpm); free(g->spm);
    free(g);
}

/* Grid edges: n1+1, n2+1, n3+1 values per axis; directions: n_ang unit
 * vectors (x,y,z); weights: n_ang quadrature weights (sum 1).  Returns NULL
 * on invalid input. */
orc_grid *orc_create(int coord, int n1, int n2, int n3, const double *e1, const double *e2,
                     const double *e3, int n_ang, const double *dir, const double *wt,
                     int inner_bc, double I_outer, int interp)
{
    if (n1 < 1 || n2 < 1 || n3 < 1 || n_ang < 1) return NULL;
    orc_grid *g = (orc_grid *)calloc(1, sizeof(orc_grid));
    g->coord = coord; g->n1 = n1; g->n2 = n2; g->n3 = n3;
    g->nvox = n1 * n2 * n3;
    g->e1 = dup_array(e1, n1 + 1); g->e2 = dup_array(e2, n2 + 1); g->e3 = dup_array(e3, n3 + 1);
    g->inner_bc = inner_bc; g->I_outer = I_outer; g->interp = interp;
    g->n_ang = n_ang; g->dir = dup_array(dir, 3 * n_ang); g->wt = dup_array(wt, n_ang);
    g->ang = (angle_t *)calloc((size_t)n_ang, sizeof(angle_t));
    /* trigonometric tables of the angular edges and mid-points (G0) */
    const double *pe = (coord == ORC_SPH) ? e3 : e2;
    int nphi = (coord == ORC_SPH) ? n3 : n2;
    g->nphi = nphi;
    g->cp = (double *)malloc(sizeof(double) * nphi); g->sp = (double *)malloc(sizeof(double) * nphi);
    g->cpm = (double *)malloc(sizeof(double) * nphi); g->spm = (double *)malloc(sizeof(double) * nphi);
    for (int k = 0; k < nphi; ++k) {
        double pm = 0.5 * (pe[k] + pe[k + 1]);
        g->cp[k] = cos(pe[k]); g->sp[k] = sin(pe[k]);
        g->cpm[k] = cos(pm); g->spm[k] = sin(pm);
    }
    if (coord == ORC_SPH) {
        g->ct = (double *)malloc(sizeof(double) * (n2 + 1));
        g->ctm = (double *)malloc(sizeof(double) * n2); g->stm = (double *)malloc(sizeof(double) * n2);
        for (int j = 0; j <= n2; ++j) g->ct[j] = cos(e2[j]);
        for (int j = 0; j < n2; ++j) {
            double tm = 0.5 * (e2[j] + e2[j + 1]);
            g->ctm[j] = cos(tm); g->stm[j] = sin(tm);
        }
    }
    return g;
}

/* Voxel centre: mid-points of the edges in each coordinate (G1). */
static void voxel_centre(const orc_grid *g, int i, int j, int k, double x[3])
{
    if (g->coord == ORC_SPH) {
        double rm = 0.5 * (g->e1[i] + g->e1[i + 1]);
        double w = rm * g->stm[j];
        x[0] = w * g->cpm[k];
        x[1] = w * g->spm[k];
        x[2] = rm * g->ctm[j];
    } else {
        double Rm = 0.5 * (g->e1[i] + g->e1[i + 1]);
        x[0] = Rm * g->cpm[j];
        x[1] = Rm * g->spm[j];
        x[2] = 0.5 * (g->e3[k] + g->e3[k + 1]);
    }
}

/* -------------------------------------------------------------- geometry -- */

typedef struct {
    double x, y, z, dx, dy, dz;
    double a, b, p2, zd, z2; /* invariants of the line x(t) = x0 + t d (G2) */
} line_t;

static void line_init(const orc_grid *g, line_t *L, const double x0[3], const double d[3])
{
    L->x = x0[0]; L->y = x0[1]; L->z = x0[2];
    L->dx = d[0]; L->dy = d[1]; L->dz = d[2];
    if (g->coord == ORC_SPH) {
        L->a = (d[0] * d[0] + d[1] * d[1]) + d[2] * d[2];
        L->b = (x0[0] * d[0] + x0[1] * d[1]) + x0[2] * d[2];
        L->p2 = (x0[0] * x0[0] + x0[1] * x0[1]) + x0[2] * x0[2];
    } else {
        L->a = d[0] * d[0] + d[1] * d[1];
        L->b = x0[0] * d[0] + x0[1] * d[1];
        L->p2 = x0[0] * x0[0] + x0[1] * x0[1];
    }
    L->zd = x0[2] * d[2];
    L->z2 = x0[2] * x0[2];
}

/* Roots of A t^2 + 2 B t + C = 0 (A != 0) in the cancellation-free form
 * q = -(B + sign(B) sqrt(B^2 - A C)), t = q/A and C/q (G3). */
static int quad_roots(double A, double B, double C, double *lo, double *hi)
{
    double disc = B * B - A * C;
    if (!(disc > 0.0)) return 0;
    double s = sqrt(disc);
    double q = (B >= 0.0) ? -(B + s) : (s - B);
    double r1 = q / A;
    double r2 = C / q;
    if (r1 <= r2) { *lo = r1; *hi = r2; } else { *lo = r2; *hi = r1; }
    return 1;
}

/* Sphere (spherical grid) or infinite cylinder (cylindrical grid) of radius e1[m] (G4). */
static int shell_roots(const orc_grid *g, const line_t *L, int m, double *lo, double *hi)
{
    if (!(L->a > 0.0)) return 0;
    double rm = g->e1[m];
    double C = L->p2 - rm * rm;
    return quad_roots(L->a, L->b, C, lo, hi);
}

/* Next crossing of the cone theta = e2[jc] after t (G5). */
static double cone_next(const orc_grid *g, const line_t *L, int jc, double t)
{
    double c = g->ct[jc];
    if (fabs(c) < 1e-12) { /* the equatorial cone is the plane z = 0 */
        if (L->dz == 0.0) return INF;
        double r = -(L->z / L->dz);
        return (r > t) ? r : INF;
    }
    double cc = c * c;
    double A = L->dz * L->dz - cc * L->a;
    double B = L->zd - cc * L->b;
    double C = L->z2 - cc * L->p2;
    double roots[2];
    int nr;
    if (A == 0.0) {
        if (B == 0.0) return INF;
        roots[0] = -(C / (2.0 * B));
        nr = 1;
    } else {
        double lo, hi;
        if (!quad_roots(A, B, C, &lo, &hi)) return INF;
        if (lo == hi) return INF; /* touching the cone does not change the cell */
        roots[0] = lo; roots[1] = hi;
        nr = 2;
    }
    for (int q = 0; q < nr; ++q) {
        double r = roots[q];
        if (!(r > t)) continue;
        double zz = L->z + r * L->dz; /* the root must lie on the nappe with sign(z) = sign(cos theta) */
        if ((c > 0.0) ? (zz > 0.0) : (zz < 0.0)) return r;
    }
    return INF;
}

/* Next crossing of the half-plane phi = phi_kp (through the z axis) after t (G6). */
static double halfplane_next(const orc_grid *g, const line_t *L, int kp, double t)
{
    double c = g->cp[kp], s = g->sp[kp];
    double den = c * L->dy - s * L->dx;
    if (den == 0.0) return INF;
    double num = c * L->y - s * L->x;
    double r = -(num / den);
    if (!(r > t)) return INF;
    double xx = L->x + r * L->dx;
    double yy = L->y + r * L->dy;
    double h = c * xx + s * yy;
    return (h > 0.0) ? r : INF;
}

/* Next crossing of the plane z = e3[m] (cylindrical grid) after t (G7). */
static double zplane_next(const orc_grid *g, const line_t *L, int m, double t)
{
    if (L->dz == 0.0) return INF;
    double r = (g->e3[m] - L->z) / L->dz;
    return (r > t) ? r : INF;
}

/* Cell of the angular coordinates at parameter t (G10); used after a hole. */
static void locate_angles(const orc_grid *g, const line_t *L, double t, int *jo, int *ko)
{
    double x = L->x + t * L->dx;
    double y = L->y + t * L->dy;
    double z = L->z + t * L->dz;
    int nphi = g->nphi, kphi = 0;
    if (nphi > 1) {
        for (int kk = 0; kk < nphi; ++kk) {
            int k1 = (kk + 1) % nphi;
            double g0 = g->cp[kk] * y - g->sp[kk] * x;
            double g1 = g->cp[k1] * y - g->sp[k1] * x;
            if (g0 >= 0.0 && g1 < 0.0) { kphi = kk; break; }
        }
    }
    if (g->coord == ORC_SPH) {
        double r = sqrt((x * x + y * y) + z * z);
        int jt = g->n2 - 1;
        for (int jj = 0; jj < g->n2 - 1; ++jj)
            if (z > g->ct[jj + 1] * r) { jt = jj; break; }
        *jo = jt; *ko = kphi;
    } else {
        int kz = g->n3 - 1;
        for (int kk = 0; kk < g->n3; ++kk)
            if (z < g->e3[kk + 1]) { kz = kk; break; }
        *jo = kphi; *ko = kz;
    }
}

/* Track a characteristic from the centre x0 of voxel (i,j,k) along d until it
 * leaves the domain (END_EXIT) or meets the opaque core (END_CORE).  Every
 * step goes from a voxel to its neighbour across the nearest bounding
 * surface (G8).  rec[q] holds the q-th cell and its entry/exit parameters. */
static int trace(const orc_grid *g, const double x0[3], const double d[3], int i, int j, int k,
                 cell_t *rec, int cap, int *nrec)
{
    line_t L;
    line_init(g, &L, x0, d);
    double t = 0.0;
    int n = 0;
    int maxsteps = 4 * (g->n1 + g->n2 + g->n3) + 16;
    rec[0].vox = vox_id(g, i, j, k); rec[0].t_in = 0.0; rec[0].after_hole = 0;
    n = 1;
    for (int step = 0; step < maxsteps; ++step) {
        double cand[6] = {INF, INF, INF, INF, INF, INF};
        double lo, hi;
        /* axis 1: inner bounding shell e1[i] (we are outside it) and outer e1[i+1] (inside it) */
        if (!(i == 0 && g->e1[0] == 0.0))
            if (shell_roots(g, &L, i, &lo, &hi) && lo < hi && lo > t) cand[0] = lo;
        if (shell_roots(g, &L, i + 1, &lo, &hi) && hi > t) cand[1] = hi;
        if (g->coord == ORC_SPH) {
            if (j >= 1) cand[2] = cone_next(g, &L, j, t);
            if (j + 1 <= g->n2 - 1) cand[3] = cone_next(g, &L, j + 1, t);
            if (g->n3 > 1) {
                cand[4] = halfplane_next(g, &L, k, t);
                cand[5] = halfplane_next(g, &L, (k + 1) % g->n3, t);
            }
        } else {
            if (g->n2 > 1) {
                cand[2] = halfplane_next(g, &L, j, t);
                cand[3] = halfplane_next(g, &L, (j + 1) % g->n2, t);
            }
            if (L.dz < 0.0) cand[4] = zplane_next(g, &L, k, t);
            if (L.dz > 0.0) cand[5] = zplane_next(g, &L, k + 1, t);
        }
        double best = INF;
        for (int q = 0; q < 6; ++q)
            if (cand[q] < best) best = cand[q];
        if (best == INF) { *nrec = n; return END_LOST; }
        rec[n - 1].t_out = best;
        /* every surface crossed at exactly this parameter moves its own axis */
        int ni = i, nj = j, nk = k, ex = 0, core = 0;
        if (cand[0] == best) { if (i == 0) core = 1; else ni = i - 1; }
        if (cand[1] == best) { if (i == g->n1 - 1) ex = 1; else ni = i + 1; }
        if (g->coord == ORC_SPH) {
            if (cand[2] == best) nj = nj - 1;
            if (cand[3] == best) nj = nj + 1;
            if (cand[4] == best) nk = (nk + g->n3 - 1) % g->n3;
            if (cand[5] == best) nk = (nk + 1) % g->n3;
        } else {
            if (cand[2] == best) nj = (nj + g->n2 - 1) % g->n2;
            if (cand[3] == best) nj = (nj + 1) % g->n2;
            if (cand[4] == best) { if (k == 0) ex = 1; else nk = k - 1; }
            if (cand[5] == best) { if (k == g->n3 - 1) ex = 1; else nk = k + 1; }
        }
        if (ex) { *nrec = n; return END_EXIT; }
        double t_new = best;
        int hole = 0;
        if (core) {
            if (g->inner_bc == ORC_CORE_B) { *nrec = n; return END_CORE; }
            /* transparent inner boundary: cross the hole without opacity (G9) */
            shell_roots(g, &L, 0, &lo, &hi);
            double tout = hi;
            if (g->coord == ORC_CYL) {
                double tz = INF;
                if (L.dz > 0.0) tz = (g->e3[g->n3] - L.z) / L.dz;
                if (L.dz < 0.0) tz = (g->e3[0] - L.z) / L.dz;
                if (tz <= tout) { *nrec = n; return END_EXIT; }
            }
            locate_angles(g, &L, tout, &nj, &nk);
            ni = 0;
            t_new = tout;
            hole = 1;
        }
        if (n >= cap) { *nrec = n; return END_LOST; }
        i = ni; j = nj; k = nk; t = t_new;
        rec[n].vox = vox_id(g, i, j, k); rec[n].t_in = t; rec[n].after_hole = hole;
        n++;
    }
    *nrec = n;
    return END_LOST;
}

/* The characteristic through the centre of voxel o: trace back along -d to
 * where it enters the domain, forward along d to where it leaves, and list
 * its segments in the direction of propagation (G11). */
static int build_ray(const orc_grid *g, int o, const double d[3], cell_t *bw, cell_t *fw, int cap,
                     int *vox, double *len, unsigned char *restart, int *nseg, int *starts_on_core)
{
    int i, j, k;
    vox_ijk(g, o, &i, &j, &k);
    double x0[3];
    voxel_centre(g, i, j, k, x0);
    double db[3] = {-d[0], -d[1], -d[2]};
    int nb = 0, nf = 0;
    int eb = trace(g, x0, db, i, j, k, bw, cap, &nb);
    int ef = trace(g, x0, d, i, j, k, fw, cap, &nf);
    if (eb == END_LOST || ef == END_LOST) return -1;
    int n = 0;
    for (int q = nb - 1; q >= 1; --q) {
        vox[n] = bw[q].vox;
        len[n] = bw[q].t_out - bw[q].t_in;
        restart[n] = (q + 1 < nb) ? (unsigned char)bw[q + 1].after_hole : 0;
        n++;
    }
    vox[n] = bw[0].vox;
    len[n] = bw[0].t_out + fw[0].t_out;
    restart[n] = (nb > 1) ? (unsigned char)bw[1].after_hole : 0;
    n++;
    for (int p = 1; p < nf; ++p) {
        vox[n] = fw[p].vox;
        len[n] = fw[p].t_out - fw[p].t_in;
        restart[n] = (unsigned char)fw[p].after_hole;
        n++;
    }
    *nseg = n;
    *starts_on_core = (eb == END_CORE);
    return 0;
}

/* Launch rule (G12): a boundary voxel starts a characteristic when the
 * direction enters the domain through its boundary face. */
static int is_outer_launch(const orc_grid *g, int i, int j, int k, const double d[3])
{
    if (g->coord == ORC_SPH) {
        if (i != g->n1 - 1) return 0;
        double c0 = g->stm[j] * g->cpm[k], c1 = g->stm[j] * g->spm[k], c2 = g->ctm[j];
        double dot = (d[0] * c0 + d[1] * c1) + d[2] * c2;
        return dot < 0.0;
    }
    int side = (i == g->n1 - 1) && ((d[0] * g->cpm[j] + d[1] * g->spm[j]) < 0.0);
    int bot = (k == 0) && (d[2] > 0.0);
    int top = (k == g->n3 - 1) && (d[2] < 0.0);
    return side || bot || top;
}

static int is_core_launch(const orc_grid *g, int i, int j, int k, const double d[3])
{
    if (g->inner_bc != ORC_CORE_B || i != 0) return 0;
    if (g->coord == ORC_SPH) {
        double c0 = g->stm[j] * g->cpm[k], c1 = g->stm[j] * g->spm[k], c2 = g->ctm[j];
        double dot = (d[0] * c0 + d[1] * c1) + d[2] * c2;
        return dot > 0.0;
    }
    return (d[0] * g->cpm[j] + d[1] * g->spm[j]) > 0.0;
}

/* Characteristics of solid angle w: one per entering boundary voxel, one per
 * core voxel it leaves from, then one through every voxel that no earlier
 * characteristic of this angle has hit, in increasing voxel index (G12). */
int orc_angle_geometry(orc_grid *g, int w)
{
    if (w < 0 || w >= g->n_ang) return -1;
    angle_t *A = &g->ang[w];
    if (A->ready) return 0;
    const double *d = &g->dir[3 * w];
    int nvox = g->nvox;
    int cap = 4 * (g->n1 + g->n2 + g->n3) + 32;
    cell_t *bw = (cell_t *)malloc(sizeof(cell_t) * cap);
    cell_t *fw = (cell_t *)malloc(sizeof(cell_t) * cap);
    int *rv = (int *)malloc(sizeof(int) * 2 * cap);
    double *rl = (double *)malloc(sizeof(double) * 2 * cap);
    unsigned char *rr = (unsigned char *)malloc(2 * cap);
    unsigned char *hit = (unsigned char *)calloc((size_t)nvox, 1);
    int rays_cap = 1024, seg_cap = 16384;
    A->ray_off = (int *)malloc(sizeof(int) * (rays_cap + 1));
    A->ray_origin = (int *)malloc(sizeof(int) * rays_cap);
    A->ray_kind = (int *)malloc(sizeof(int) * rays_cap);
    A->ray_core = (int *)malloc(sizeof(int) * rays_cap);
    A->vox = (int *)malloc(sizeof(int) * seg_cap);
    A->len = (double *)malloc(sizeof(double) * seg_cap);
    A->restart = (unsigned char *)malloc(seg_cap);
    A->n_rays = 0; A->n_seg = 0; A->n_lost = 0;
    A->ray_off[0] = 0;
    for (int pass = 0; pass < 3; ++pass) {
        for (int v = 0; v < nvox; ++v) {
            int i, j, k;
            vox_ijk(g, v, &i, &j, &k);
            int launch;
            if (pass == 0) launch = is_outer_launch(g, i, j, k, d);
            else if (pass == 1) launch = is_core_launch(g, i, j, k, d);
            else launch = !hit[v];
            if (!launch) continue;
            int ns = 0, oncore = 0;
            if (build_ray(g, v, d, bw, fw, cap, rv, rl, rr, &ns, &oncore) != 0) {
                A->n_lost++;
                hit[v] = 1;
                continue;
            }
            if (A->n_rays + 1 > rays_cap) {
                rays_cap *= 2;
                A->ray_off = (int *)realloc(A->ray_off, sizeof(int) * (rays_cap + 1));
                A->ray_origin = (int *)realloc(A->ray_origin, sizeof(int) * rays_cap);
                A->ray_kind = (int *)realloc(A->ray_kind, sizeof(int) * rays_cap);
                A->ray_core = (int *)realloc(A->ray_core, sizeof(int) * rays_cap);
            }
            while (A->n_seg + ns > seg_cap) {
                seg_cap *= 2;
                A->vox = (int *)realloc(A->vox, sizeof(int) * seg_cap);
                A->len = (double *)realloc(A->len, sizeof(double) * seg_cap);
                A->restart = (unsigned char *)realloc(A->restart, seg_cap);
            }
            int r = A->n_rays;
            A->ray_origin[r] = v; A->ray_kind[r] = pass; A->ray_core[r] = oncore;
            for (int s = 0; s < ns; ++s) {
                A->vox[A->n_seg + s] = rv[s];
                A->len[A->n_seg + s] = rl[s];
                A->restart[A->n_seg + s] = rr[s];
                hit[rv[s]] = 1;
            }
            A->n_seg += ns;
            A->n_rays = r + 1;
            A->ray_off[r + 1] = A->n_seg;
        }
    }
    free(bw); free(fw); free(rv); free(rl); free(rr); free(hit);
    A->ready = 1;
    return A->n_lost;
}

void orc_angle_free(orc_grid *g, int w)
{
    if (w >= 0 && w < g->n_ang) free_angle(&g->ang[w]);
}

/* Sizes of the crossing lists of angle w (computed on demand). */
int orc_angle_counts(orc_grid *g, int w, int *n_rays, int *n_seg, int *n_lost)
{
    int rc = orc_angle_geometry(g, w);
    if (rc < 0) return rc;
    *n_rays = g->ang[w].n_rays; *n_seg = g->ang[w].n_seg; *n_lost = g->ang[w].n_lost;
    return 0;
}

int orc_angle_copy(orc_grid *g, int w, int *ray_off, int *ray_origin, int *ray_kind, int *ray_core,
                   int *vox, double *len, unsigned char *restart)
{
    int rc = orc_angle_geometry(g, w);
    if (rc < 0) return rc;
    angle_t *A = &g->ang[w];
    memcpy(ray_off, A->ray_off, sizeof(int) * (A->n_rays + 1));
    memcpy(ray_origin, A->ray_origin, sizeof(int) * A->n_rays);
    memcpy(ray_kind, A->ray_kind, sizeof(int) * A->n_rays);
    memcpy(ray_core, A->ray_core, sizeof(int) * A->n_rays);
    memcpy(vox, A->vox, sizeof(int) * A->n_seg);
    memcpy(len, A->len, sizeof(double) * A->n_seg);
    memcpy(restart, A->restart, A->n_seg);
    return 0;
}

/* ------------------------------------------------------- formal solution -- */

/* Interpolation weights of one segment of optical depth dm = dtau_k followed
 * by dp = dtau_{k+1}:  I_k = I_{k-1} e^{-dm} + alpha S_{k-1} + beta S_k +
 * gamma S_{k+1}, the exact integral of the parabola through the three nodes
 * against e^{-(dm - u)} (R6).  e0 = 1 - e^{-dm}, e1 = dm - e0,
 * e2 = dm^2 - 2 e1; below dm = 0.1 e1 and e2 come from their Taylor series
 * (R7).  parabolic = 0 gives the linear (last-node) weights. */
void orc_coeffs(double dm, double dp, int parabolic, double *alpha, double *beta, double *gamma)
{
    double e0 = -expm1(-dm);
    double e1, e2;
    if (dm < 0.1) {
        double term = dm; /* dm^n / n! */
        e1 = 0.0;
        e2 = 0.0;
        for (int n = 2; n <= 18; ++n) {
            term = term * dm / (double)n;
            double sgn = (n % 2 == 0) ? 1.0 : -1.0;
            e1 += sgn * term;
            if (n >= 3) e2 += -2.0 * sgn * term;
        }
    } else {
        e1 = dm - e0;
        e2 = dm * dm - 2.0 * e1;
    }
    if (parabolic) {
        double D = dm + dp;
        *alpha = e0 + (e2 - (dp + 2.0 * dm) * e1) / (dm * D);
        *beta = (D * e1 - e2) / (dm * dp);
        *gamma = (e2 - dm * e1) / (dp * D);
    } else {
        *alpha = e0 - e1 / dm;
        *beta = e1 / dm;
        *gamma = 0.0;
    }
}

/* The parabola through S_{k-1}, S_k, S_{k+1} is used when segment k is not
 * the last of its run and the next node is at least half as far in optical
 * depth as the previous one; otherwise the linear weights are used. */
static int use_parabola(const orc_grid *g, double dm, double dp)
{
    return g->interp == ORC_PARABOLIC && dp >= 0.5 * dm;
}

/* Formal solution of one solid angle: march every characteristic of angle w
 * and accumulate, per voxel, sum l*I, sum l*lambda and sum l over all visits.
 * homog = 1 sets every incoming intensity to zero (the pure Lambda operator).
 * Iexit (optional) receives the emergent intensity of each characteristic. */
static int fs_angle_sums(orc_grid *g, int w, const double *S, const double *chi, const double *B,
                         int homog, double *sumI, double *sumL, double *sumLen, double *Iexit)
{
    int rc = orc_angle_geometry(g, w);
    if (rc < 0) return rc;
    angle_t *A = &g->ang[w];
    for (int r = 0; r < A->n_rays; ++r) {
        int s0 = A->ray_off[r], s1 = A->ray_off[r + 1];
        double I;
        if (homog) I = 0.0;
        else I = A->ray_core[r] ? B[A->vox[s0]] : g->I_outer;
        double gamma_prev = 0.0;
        int run_start = s0;
        for (int s = s0; s < s1; ++s) {
            if (s > s0 && A->restart[s]) { run_start = s; gamma_prev = 0.0; }
            int last = (s + 1 == s1) || A->restart[s + 1];
            int v = A->vox[s];
            double dm = chi[v] * A->len[s];
            double Sk = S[v];
            double Skm = (s == run_start) ? Sk : S[A->vox[s - 1]];
            double alpha, beta, gamma, Skp = 0.0;
            double dp = 0.0;
            if (!last) dp = chi[A->vox[s + 1]] * A->len[s + 1];
            if (!last && use_parabola(g, dm, dp)) {
                orc_coeffs(dm, dp, 1, &alpha, &beta, &gamma);
                Skp = S[A->vox[s + 1]];
            } else {
                orc_coeffs(dm, 0.0, 0, &alpha, &beta, &gamma);
            }
            double E = exp(-dm);
            I = I * E + alpha * Skm + beta * Sk + gamma * Skp;
            /* dI_k / dS_k through this segment and the previous one; at the start
             * of a run the boundary node carries S_k as well (S_0 := S_1) */
            double lam = beta + gamma_prev * E;
            if (s == run_start) lam += alpha;
            sumI[v] += A->len[s] * I;
            sumL[v] += A->len[s] * lam;
            sumLen[v] += A->len[s];
            gamma_prev = gamma;
        }
        if (Iexit) Iexit[r] = I;
    }
    return 0;
}

/* Per-voxel path-length averaged intensity and Lambda* element for one
 * angle: Ibar_v = sum l I / sum l over all visits of voxel v (R8, R9). */
int orc_fs_angle(orc_grid *g, int w, const double *S, const double *chi, const double *B, int homog,
                 double *Ibar, double *Lbar, double *Iexit)
{
    int nvox = g->nvox;
    double *sI = (double *)calloc(nvox, sizeof(double));
    double *sL = (double *)calloc(nvox, sizeof(double));
    double *sl = (double *)calloc(nvox, sizeof(double));
    int rc = fs_angle_sums(g, w, S, chi, B, homog, sI, sL, sl, Iexit);
    int missing = 0;
    if (rc == 0) {
        for (int v = 0; v < nvox; ++v) {
            if (sl[v] > 0.0) { Ibar[v] = sI[v] / sl[v]; Lbar[v] = sL[v] / sl[v]; }
            else { Ibar[v] = 0.0; Lbar[v] = 0.0; missing++; }
        }
    }
    free(sI); free(sL); free(sl);
    if (rc < 0) return rc;
    return missing;
}

/* Local orthonormal basis at the voxel centre: (r, theta, phi) on the
 * spherical grid, (R, phi, z) on the cylindrical grid. */
static void local_basis(const orc_grid *g, int i, int j, int k, double e[3][3])
{
    (void)i;
    if (g->coord == ORC_SPH) {
        double st = g->stm[j], ctt = g->ctm[j], c = g->cpm[k], s = g->spm[k];
        e[0][0] = st * c;  e[0][1] = st * s;  e[0][2] = ctt;
        e[1][0] = ctt * c; e[1][1] = ctt * s; e[1][2] = -st;
        e[2][0] = -s;      e[2][1] = c;       e[2][2] = 0.0;
    } else {
        double c = g->cpm[j], s = g->spm[j];
        e[0][0] = c;  e[0][1] = s; e[0][2] = 0.0;
        e[1][0] = -s; e[1][1] = c; e[1][2] = 0.0;
        e[2][0] = 0.0; e[2][1] = 0.0; e[2][2] = 1.0;
    }
}

/* Full formal solution: J_v = sum_w wt_w Ibar_v(w), Lambda*_v likewise,
 * flux F_v = 4 pi sum_w wt_w n_w Ibar_v(w) in the local basis (R8, R9).
 * F may be NULL.  Returns the number of (voxel, angle) pairs no
 * characteristic hit (0 when the coverage guarantee holds), or < 0. */
int orc_formal_solution(orc_grid *g, const double *S, const double *chi, const double *B, int homog,
                        double *J, double *Lstar, double *F)
{
    int nvox = g->nvox, missing = 0;
    double *Ib = (double *)malloc(sizeof(double) * nvox);
    double *Lb = (double *)malloc(sizeof(double) * nvox);
    double *Fc = (double *)calloc(3 * (size_t)nvox, sizeof(double));
    for (int v = 0; v < nvox; ++v) { J[v] = 0.0; Lstar[v] = 0.0; }
    for (int w = 0; w < g->n_ang; ++w) {
        int rc = orc_fs_angle(g, w, S, chi, B, homog, Ib, Lb, NULL);
        if (rc < 0) { missing = rc; break; }
        missing += rc;
        double wt = g->wt[w];
        const double *d = &g->dir[3 * w];
        for (int v = 0; v < nvox; ++v) {
            J[v] += wt * Ib[v];
            Lstar[v] += wt * Lb[v];
            Fc[3 * v + 0] += FOUR_PI * wt * d[0] * Ib[v];
            Fc[3 * v + 1] += FOUR_PI * wt * d[1] * Ib[v];
            Fc[3 * v + 2] += FOUR_PI * wt * d[2] * Ib[v];
        }
    }
    if (F) {
        for (int v = 0; v < nvox; ++v) {
            int i, j, k;
            vox_ijk(g, v, &i, &j, &k);
            double e[3][3];
            local_basis(g, i, j, k, e);
            for (int c = 0; c < 3; ++c)
                F[3 * v + c] = e[c][0] * Fc[3 * v + 0] + e[c][1] * Fc[3 * v + 1] + e[c][2] * Fc[3 * v + 2];
        }
    }
    free(Ib); free(Lb); free(Fc);
    return missing;
}

/* The same formal solution with the angle loop spread over nthreads host
 * threads (OpenMP when the oracle is compiled with it; one thread
 * otherwise).  Thread t takes the solid angles w = t, t + nthreads, ... in
 * increasing order and adds their terms into its own partial sums, exactly
 * as the serial loop does; the partial sums are then added in thread order.
 * The result is reproducible for a given thread count and equals the serial
 * one up to the association of the angle sum.  Returns the number of
 * (voxel, angle) pairs no characteristic hit, or < 0; *used receives the
 * thread count that ran. */
int orc_formal_solution_par(orc_grid *g, const double *S, const double *chi, const double *B, int homog,
                            double *J, double *Lstar, double *F, int nthreads, int *used)
{
    int nvox = g->nvox;
    if (nthreads < 1) nthreads = 1;
#ifndef _OPENMP
    nthreads = 1;
#endif
    size_t stride = 5 * (size_t)nvox; /* per thread: J, Lambda*, three flux components */
    double *part = (double *)calloc((size_t)nthreads * stride, sizeof(double));
    int *miss = (int *)calloc((size_t)nthreads, sizeof(int));
    if (!part || !miss) { free(part); free(miss); return -2; }
    int ran = 1;
#ifdef _OPENMP
#pragma omp parallel num_threads(nthreads)
#endif
    {
        int t = 0;
#ifdef _OPENMP
        t = omp_get_thread_num();
#pragma omp single
        ran = omp_get_num_threads();
#endif
        double *Ib = (double *)malloc(sizeof(double) * nvox);
        double *Lb = (double *)malloc(sizeof(double) * nvox);
        double *P = part + (size_t)t * stride;
        for (int w = t; w < g->n_ang && Ib && Lb; w += nthreads) {
            int rc = orc_fs_angle(g, w, S, chi, B, homog, Ib, Lb, NULL);
            if (rc < 0) { miss[t] = rc; break; }
            miss[t] += rc;
            double wt = g->wt[w];
            const double *d = &g->dir[3 * w];
            for (int v = 0; v < nvox; ++v) {
                P[v] += wt * Ib[v];
                P[nvox + v] += wt * Lb[v];
                P[2 * (size_t)nvox + v] += FOUR_PI * wt * d[0] * Ib[v];
                P[3 * (size_t)nvox + v] += FOUR_PI * wt * d[1] * Ib[v];
                P[4 * (size_t)nvox + v] += FOUR_PI * wt * d[2] * Ib[v];
            }
        }
        if (!Ib || !Lb) miss[t] = -2;
        free(Ib); free(Lb);
    }
    int missing = 0;
    for (int t = 0; t < nthreads; ++t) {
        if (miss[t] < 0) { missing = miss[t]; break; }
        missing += miss[t];
    }
    for (int v = 0; v < nvox; ++v) {
        double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
        for (int t = 0; t < nthreads; ++t)
            for (int c = 0; c < 5; ++c) acc[c] += part[(size_t)t * stride + (size_t)c * nvox + v];
        J[v] = acc[0];
        Lstar[v] = acc[1];
        if (F) {
            int i, j, k;
            vox_ijk(g, v, &i, &j, &k);
            double e[3][3];
            local_basis(g, i, j, k, e);
            for (int c = 0; c < 3; ++c) F[3 * v + c] = e[c][0] * acc[2] + e[c][1] * acc[3] + e[c][2] * acc[4];
        }
    }
    free(part); free(miss);
    if (used) *used = ran;
    return missing;
}

/* ---------------------------------------------------------- ALI and Ng -- */

/* Operator-splitting update with the diagonal Lambda* (R10):
 * S_new = S + [(1-eps) J + eps B - S] / (1 - (1-eps) Lambda*).
 * use_lstar = 0 is the plain Lambda iteration.  Returns max |dS| / |S_new|. */
double orc_ali_update(int nvox, double *S, const double *J, const double *Lstar, const double *eps,
                      const double *B, int use_lstar)
{
    double maxrel = 0.0;
    for (int v = 0; v < nvox; ++v) {
        double e = eps[v];
        double L = use_lstar ? Lstar[v] : 0.0;
        double Snew = S[v] + ((1.0 - e) * J[v] + e * B[v] - S[v]) / (1.0 - (1.0 - e) * L);
        double rel = fabs(Snew - S[v]) / fabs(Snew);
        if (rel > maxrel) maxrel = rel;
        S[v] = Snew;
    }
    return maxrel;
}

/* Ng acceleration of order 2 (R11): y0 newest .. y3 oldest of four
 * successive iterates.  Minimises the 1/y0^2-weighted norm of the residual
 * combination and writes (1-a-b) y0 + a y1 + b y2 to out.  Returns 1 when
 * applied, 0 when the 2x2 system is singular (out untouched). */
int orc_ng(int nvox, const double *y0, const double *y1, const double *y2, const double *y3, double *out)
{
    double A11 = 0, A12 = 0, A22 = 0, b1 = 0, b2 = 0;
    for (int v = 0; v < nvox; ++v) {
        double W = 1.0 / (y0[v] * y0[v]);
        double r1 = y0[v] - y1[v], r2 = y1[v] - y2[v], r3 = y2[v] - y3[v];
        double d1 = r1 - r2, d2 = r1 - r3;
        A11 += W * d1 * d1;
        A12 += W * d1 * d2;
        A22 += W * d2 * d2;
        b1 += W * d1 * r1;
        b2 += W * d2 * r1;
    }
    double det = A11 * A22 - A12 * A12;
    if (!(fabs(det) > 1e-14 * (A11 * A22)) || !(det == det)) return 0;
    double a = (b1 * A22 - b2 * A12) / det;
    double b = (A11 * b2 - A12 * b1) / det;
    for (int v = 0; v < nvox; ++v) out[v] = (1.0 - a - b) * y0[v] + a * y1[v] + b * y2[v];
    return 1;
}

/* ------------------------------------------- nearest-neighbour Lambda* -- */

/* Slot of voxel u in the 3x3x3 index neighbourhood of voxel v:
 * (di+1)*9 + (dj+1)*3 + (dk+1) for the offset (di, dj, dk) in {-1,0,1}^3 that
 * reaches u, the phi index (axis 3 spherical, axis 2 cylindrical) taken modulo
 * n_phi; -1 when u is not a neighbour.  Needs n_phi >= 3 (one offset per
 * neighbour); slot 13 is v itself. */
static int nn_slot(const orc_grid *g, int v, int u)
{
    int i, j, k, a, b, c;
    vox_ijk(g, v, &i, &j, &k);
    vox_ijk(g, u, &a, &b, &c);
    int d[3] = {a - i, b - j, c - k};
    int per = (g->coord == ORC_SPH) ? 2 : 1, nper = (g->coord == ORC_SPH) ? g->n3 : g->n2;
    if (d[per] == nper - 1) d[per] = -1;
    else if (d[per] == 1 - nper) d[per] = 1;
    for (int q = 0; q < 3; ++q)
        if (d[q] < -1 || d[q] > 1) return -1;
    return (d[0] + 1) * 9 + (d[1] + 1) * 3 + (d[2] + 1);
}

/* Voxel in slot q of v's neighbourhood, or -1 outside the grid. */
static int nn_voxel(const orc_grid *g, int v, int q)
{
    int i, j, k;
    vox_ijk(g, v, &i, &j, &k);
    i += q / 9 - 1;
    j += (q / 3) % 3 - 1;
    k += q % 3 - 1;
    if (g->coord == ORC_SPH) k = (k + g->n3) % g->n3;
    else j = (j + g->n2) % g->n2;
    if (i < 0 || i >= g->n1 || j < 0 || j >= g->n2 || k < 0 || k >= g->n3) return -1;
    return vox_id(g, i, j, k);
}

/* Nearest-neighbour approximate Lambda operator, built exactly (Sect. 2: 3^3
 * neighbour voxels, Paper I): L27[27 v + q] = dJ_v / dS_u for the voxel u in
 * slot q of v's neighbourhood.  J_v = sum_w wt_w sum_{visits s of v} (l_s /
 * L_wv) I_s and I_s = sum over the segments j <= s of its characteristic of
 * (alpha_j S_prev(j) + beta_j S_{v_j} + gamma_j S_{v_{j+1}}) times the
 * attenuation exp(-(tau_{j+1} + ... + tau_s)), where prev(j) is the previous
 * node's voxel, or v_j at the start of a run; every upstream segment is
 * visited for every s (brute force).  Returns 0, or < 0 on a geometry error
 * (-2: n_phi < 3). */
int orc_nn_lstar(orc_grid *g, const double *chi, double *L27)
{
    const int nvox = g->nvox;
    if ((g->coord == ORC_SPH ? g->n3 : g->n2) < 3) return -2;
    double *acc = (double *)calloc(27 * (size_t)nvox, sizeof(double));
    double *sl = (double *)calloc(nvox, sizeof(double));
    for (size_t q = 0; q < 27 * (size_t)nvox; ++q) L27[q] = 0.0;
    int rc = 0;
    for (int w = 0; w < g->n_ang && rc == 0; ++w) {
        rc = orc_angle_geometry(g, w);
        if (rc < 0) break;
        angle_t *A = &g->ang[w];
        memset(acc, 0, sizeof(double) * 27 * (size_t)nvox);
        memset(sl, 0, sizeof(double) * nvox);
        int nmax = 0;
        for (int r = 0; r < A->n_rays; ++r)
            if (A->ray_off[r + 1] - A->ray_off[r] > nmax) nmax = A->ray_off[r + 1] - A->ray_off[r];
        double *E = (double *)malloc(sizeof(double) * (nmax + 1));
        double *al = (double *)malloc(sizeof(double) * (nmax + 1));
        double *be = (double *)malloc(sizeof(double) * (nmax + 1));
        double *ga = (double *)malloc(sizeof(double) * (nmax + 1));
        int *vm = (int *)malloc(sizeof(int) * (nmax + 1));
        int *vp = (int *)malloc(sizeof(int) * (nmax + 1));
        for (int r = 0; r < A->n_rays; ++r) {
            const int s0 = A->ray_off[r], s1 = A->ray_off[r + 1];
            int run_start = s0;
            for (int s = s0; s < s1; ++s) { /* weights of every segment of the characteristic */
                if (s > s0 && A->restart[s]) run_start = s;
                const int last = (s + 1 == s1) || A->restart[s + 1];
                const int v = A->vox[s];
                const double dm = chi[v] * A->len[s];
                const double dp = last ? 0.0 : chi[A->vox[s + 1]] * A->len[s + 1];
                double a, b, c;
                if (!last && use_parabola(g, dm, dp)) {
                    orc_coeffs(dm, dp, 1, &a, &b, &c);
                    vp[s - s0] = A->vox[s + 1];
                } else {
                    orc_coeffs(dm, 0.0, 0, &a, &b, &c);
                    vp[s - s0] = -1;
                }
                E[s - s0] = exp(-dm);
                al[s - s0] = a;
                be[s - s0] = b;
                ga[s - s0] = c;
                vm[s - s0] = (s == run_start) ? v : A->vox[s - 1];
            }
            for (int s = s0; s < s1; ++s) {
                const int v = A->vox[s];
                double *row = acc + 27 * (size_t)v;
                double P = A->len[s]; /* l_s times the attenuation from segment j to s */
                for (int j = s; j >= s0; --j) {
                    const int jj = j - s0;
                    int q = nn_slot(g, v, A->vox[j]);
                    if (q >= 0) row[q] += P * be[jj];
                    q = nn_slot(g, v, vm[jj]);
                    if (q >= 0) row[q] += P * al[jj];
                    if (vp[jj] >= 0) {
                        q = nn_slot(g, v, vp[jj]);
                        if (q >= 0) row[q] += P * ga[jj];
                    }
                    P *= E[jj];
                }
                sl[v] += A->len[s];
            }
        }
        free(E); free(al); free(be); free(ga); free(vm); free(vp);
        const double wt = g->wt[w];
        for (int v = 0; v < nvox; ++v)
            if (sl[v] > 0.0)
                for (int q = 0; q < 27; ++q) L27[27 * (size_t)v + q] += wt * acc[27 * (size_t)v + q] / sl[v];
    }
    free(acc);
    free(sl);
    return rc < 0 ? rc : 0;
}

/* Operator-splitting update with the nearest-neighbour Lambda*: the change dS
 * solves (I - (1-eps) L*) dS = (1-eps) J + eps B - S with L* restricted to the
 * 27-voxel neighbourhoods; Jacobi sweeps
 *   dS_v <- [r_v + (1-eps_v) sum_{u != v} L*_vu dS_u] / (1 - (1-eps_v) L*_vv)
 * from dS = 0 until max |sweep change| <= jtol max |dS| (at most jmax sweeps;
 * *sweeps receives the count).  S <- S + dS; returns max |dS| / |S_new|, or NaN
 * with S unchanged when a sweep leaves a non-finite iterate (the sweeps do not
 * contract when (1-eps) times a row's off-diagonal weight outgrows its diagonal
 * term; the system itself may still be regular). */
double orc_nn_ali_update(const orc_grid *g, double *S, const double *J, const double *L27, const double *eps,
                         const double *B, double jtol, int jmax, int *sweeps)
{
    const int nvox = g->nvox;
    double *r = (double *)malloc(sizeof(double) * nvox);
    double *x = (double *)calloc(nvox, sizeof(double));
    double *y = (double *)malloc(sizeof(double) * nvox);
    for (int v = 0; v < nvox; ++v) r[v] = (1.0 - eps[v]) * J[v] + eps[v] * B[v] - S[v];
    int m;
    for (m = 1; m <= jmax; ++m) {
        double dmax = 0.0, xmax = 0.0;
        for (int v = 0; v < nvox; ++v) {
            const double *L = L27 + 27 * (size_t)v;
            double off = 0.0;
            for (int q = 0; q < 27; ++q) {
                if (q == 13) continue;
                const int u = nn_voxel(g, v, q);
                if (u >= 0) off += L[q] * x[u];
            }
            y[v] = (r[v] + (1.0 - eps[v]) * off) / (1.0 - (1.0 - eps[v]) * L[13]);
        }
        int finite = 1;
        for (int v = 0; v < nvox; ++v) {
            if (!isfinite(y[v])) finite = 0;
            if (fabs(y[v] - x[v]) > dmax) dmax = fabs(y[v] - x[v]);
            if (fabs(y[v]) > xmax) xmax = fabs(y[v]);
            x[v] = y[v];
        }
        /* a sweep that leaves a non-finite iterate has not solved the OS system
         * (the sweeps do not contract there): S stays as it was, the result is NaN */
        if (!finite) {
            if (sweeps) *sweeps = m;
            free(r); free(x); free(y);
            return NAN;
        }
        if (!(dmax > jtol * xmax)) break;
    }
    if (sweeps) *sweeps = m > jmax ? jmax : m;
    double maxrel = 0.0;
    for (int v = 0; v < nvox; ++v) {
        const double Snew = S[v] + x[v];
        const double rel = fabs(x[v]) / fabs(Snew);
        if (rel > maxrel) maxrel = rel;
        S[v] = Snew;
    }
    free(r); free(x); free(y);
    return maxrel;
}

/* ALI iteration to max rel dS < tol (R10, R11).  S holds the start value on
 * entry (the caller passes B) and the result on exit.  use_lstar: 0 Lambda
 * iteration, 1 diagonal Lambda*, 2 nearest-neighbour Lambda* (built once,
 * OS step solved by Jacobi sweeps to 1e-14).  ng = 1 applies Ng whenever four
 * ALI iterates have accumulated since the last extrapolation.  hist
 * (optional, max_iter entries) receives max rel dS of every step.  With
 * nthreads > 1 each formal solution runs its angle loop over that many host
 * threads (orc_formal_solution_par).  Returns the number of steps taken
 * (negative: not converged). */
int orc_solve(orc_grid *g, double *S, const double *chi, const double *eps, const double *B, double tol,
              int max_iter, int use_lstar, int ng, double *hist, int nthreads)
{
    int nvox = g->nvox;
    double *J = (double *)malloc(sizeof(double) * nvox);
    double *L = (double *)malloc(sizeof(double) * nvox);
    double *H = (double *)malloc(sizeof(double) * 4 * (size_t)nvox);
    double *L27 = NULL;
    if (use_lstar == 2) {
        L27 = (double *)malloc(sizeof(double) * 27 * (size_t)nvox);
        if (orc_nn_lstar(g, chi, L27) < 0) {
            free(J); free(L); free(H); free(L27);
            return -max_iter;
        }
    }
    int nh = 0, it, done = 0;
    for (it = 1; it <= max_iter; ++it) {
        if (nthreads > 1) orc_formal_solution_par(g, S, chi, B, 0, J, L, NULL, nthreads, NULL);
        else orc_formal_solution(g, S, chi, B, 0, J, L, NULL);
        double rel;
        if (use_lstar == 2) rel = orc_nn_ali_update(g, S, J, L27, eps, B, 1e-14, 100000, NULL);
        else rel = orc_ali_update(nvox, S, J, L, eps, B, use_lstar);
        if (hist) hist[it - 1] = rel;
        if (isnan(rel)) break; /* the OS step failed: not converged */
        if (rel < tol) { done = 1; break; }
        if (ng) {
            /* history slots: H[3] newest */
            if (nh == 4) { memmove(H, H + nvox, sizeof(double) * 3 * nvox); nh = 3; }
            memcpy(H + (size_t)nh * nvox, S, sizeof(double) * nvox);
            nh++;
            if (nh == 4) {
                if (orc_ng(nvox, H + 3 * (size_t)nvox, H + 2 * (size_t)nvox, H + (size_t)nvox, H, S)) nh = 0;
            }
        }
    }
    free(J); free(L); free(H); free(L27);
    return done ? it : -max_iter;
}

/* ----------------------------------------------- 1D spherical comparison -- */

/* Exact intensity of the 1D spherically symmetric problem with shell-constant
 * S and chi (shells r_0 < ... < r_n, core r < r_0 emitting I_core, or
 * transparent when core_b = 0) at radius r along direction mu = cos angle to
 * the outward radial direction: the characteristic with impact parameter
 * p = r sqrt(1 - mu^2) is integrated exactly segment by segment, I <- I e^-dtau
 * + S (1 - e^-dtau), from where it enters the atmosphere. */
double orc_pz_intensity(int n, const double *rs, const double *Sh, const double *chih, int core_b,
                        double I_core, double r, double mu)
{
    double p2 = r * r * (1.0 - mu * mu);
    if (p2 < 0.0) p2 = 0.0;
    double zq = r * mu;
    /* breakpoints along the line z (position along the ray) */
    int nb = 0;
    double *zb = (double *)malloc(sizeof(double) * (2 * (n + 1) + 2));
    for (int m = 0; m <= n; ++m) {
        double rm2 = rs[m] * rs[m];
        if (rm2 > p2) {
            double h = sqrt(rm2 - p2);
            zb[nb++] = -h;
            zb[nb++] = h;
        }
    }
    /* sort breakpoints */
    for (int a = 1; a < nb; ++a) {
        double x = zb[a];
        int c = a - 1;
        while (c >= 0 && zb[c] > x) { zb[c + 1] = zb[c]; c--; }
        zb[c + 1] = x;
    }
    double zout = sqrt(rs[n] * rs[n] - p2);
    double zstart = -zout, I = 0.0;
    double r02 = rs[0] * rs[0];
    if (core_b && p2 < r02) {
        double zc = sqrt(r02 - p2);
        if (zq >= zc) { zstart = zc; I = I_core; }
    }
    double zcur = zstart;
    for (int a = 0; a <= nb; ++a) {
        double znext = (a < nb) ? zb[a] : zq;
        if (znext > zq) znext = zq;
        if (znext <= zcur) continue;
        double zmid = 0.5 * (zcur + znext);
        double rmid = sqrt(p2 + zmid * zmid);
        int sh = -1;
        for (int m = 0; m < n; ++m)
            if (rmid >= rs[m] && rmid < rs[m + 1]) { sh = m; break; }
        if (sh >= 0) {
            double dt = chih[sh] * (znext - zcur);
            double E = exp(-dt);
            I = I * E + Sh[sh] * (1.0 - E);
        }
        zcur = znext;
        if (zcur >= zq) break;
    }
    free(zb);
    return I;
}
