// geom.cu -- characteristic geometry on the GPU: launch set and exact voxel
// crossing lists for every solid angle (Hauschildt & Baron IV, Sect. 2:
// full characteristics from the boundary, stepping voxel to neighbour, every
// voxel hit at least once per solid angle).
//
// This translation unit is compiled with -fmad=false: every +, -, *, / and
// sqrt below is one IEEE double rounding, in the order written, so crossing
// parameters are reproducible bit for bit by any implementation of the same
// geometry rules:
//  * voxel centre = mid-points of the edges, x = (r_m sin th_m) cos ph_m,
//    y = (r_m sin th_m) sin ph_m, z = r_m cos th_m (cylinder: R_m cos ph_m,
//    R_m sin ph_m, z_m), with cos/sin of edges and mid-points from host libm;
//  * line invariants a = n.n, b = x0.n, p2 = x0.x0 (cylinder: x, y only);
//  * roots of A t^2 + 2 B t + C: disc = B B - A C > 0, q = -(B + sign(B) sqrt),
//    roots q/A and C/q; inner shell = smaller root, outer = larger;
//  * cones: |cos th_j| < 1e-12 is the plane z = 0, else the quadratic with
//    the nappe test sign(z(t)) = sign(cos th_j); a double root is no crossing;
//  * half-planes: t = -(c y - s x)/(c n_y - s n_x), valid if c x(t) + s y(t) > 0;
//  * z-planes only in the direction of n_z;
//  * step to the smallest candidate > t; tied surfaces move all their axes in
//    one step; leaving the domain takes precedence;
//  * a transparent hole is crossed to the larger root of the inner surface;
//  * a characteristic = the backward walk reversed + the forward walk, the
//    origin's length the sum of both first steps;
//  * launch order: outer-boundary voxels, core voxels, then completions, each
//    in increasing voxel index.
#include <cuda_runtime.h>
#include <stdint.h>

#include "geom_pred.cuh"
#include "rt_internal.h"

namespace rtk {
namespace {

__device__ __forceinline__ double dinf() { return __longlong_as_double(0x7ff0000000000000LL); }

struct Line {
    double x, y, z, dx, dy, dz;
    double a, b, p2, zd, z2;
};

__device__ __forceinline__ int vid(const GeomDev &G, int i, int j, int k) { return (i * G.n2 + j) * G.n3 + k; }

__device__ __forceinline__ void centre_of(const GeomDev &G, int i, int j, int k, double &x, double &y, double &z)
{
    if (G.coord == RT_SPHERICAL) {
        double rm = 0.5 * (G.e1[i] + G.e1[i + 1]);
        double w = rm * G.stm[j];
        x = w * G.cpm[k];
        y = w * G.spm[k];
        z = rm * G.ctm[j];
    } else {
        double Rm = 0.5 * (G.e1[i] + G.e1[i + 1]);
        x = Rm * G.cpm[j];
        y = Rm * G.spm[j];
        z = 0.5 * (G.e3[k] + G.e3[k + 1]);
    }
}

__device__ __forceinline__ Line make_line(const GeomDev &G, double x, double y, double z, double dx, double dy,
                                          double dz)
{
    Line L;
    L.x = x; L.y = y; L.z = z;
    L.dx = dx; L.dy = dy; L.dz = dz;
    if (G.coord == RT_SPHERICAL) {
        L.a = (dx * dx + dy * dy) + dz * dz;
        L.b = (x * dx + y * dy) + z * dz;
        L.p2 = (x * x + y * y) + z * z;
    } else {
        L.a = dx * dx + dy * dy;
        L.b = x * dx + y * dy;
        L.p2 = x * x + y * y;
    }
    L.zd = z * dz;
    L.z2 = z * z;
    return L;
}

// A t^2 + 2 B t + C = 0, A != 0: ordered roots when the discriminant is positive.
__device__ __forceinline__ bool roots2(double A, double B, double C, double &lo, double &hi)
{
    double disc = B * B - A * C;
    if (!(disc > 0.0)) return false;
    double s = sqrt(disc);
    double q = (B >= 0.0) ? -(B + s) : (s - B);
    double r1 = q / A;
    double r2 = C / q;
    lo = (r1 <= r2) ? r1 : r2;
    hi = (r1 <= r2) ? r2 : r1;
    return true;
}

// Sphere (spherical) or cylinder (cylindrical) of radius e1[m].
__device__ __forceinline__ bool shell(const GeomDev &G, const Line &L, int m, double &lo, double &hi)
{
    if (!(L.a > 0.0)) return false;
    double rm = G.e1[m];
    return roots2(L.a, L.b, L.p2 - rm * rm, lo, hi);
}

// Angular cell at parameter t (after crossing a transparent hole).
__device__ void locate(const GeomDev &G, const Line &L, double t, int &jo, int &ko)
{
    double x = L.x + t * L.dx;
    double y = L.y + t * L.dy;
    double z = L.z + t * L.dz;
    int kphi = 0;
    if (G.nphi > 1) {
        for (int kk = 0; kk < G.nphi; ++kk) {
            int k1 = (kk + 1 == G.nphi) ? 0 : kk + 1;
            double g0 = G.cp[kk] * y - G.sp[kk] * x;
            double g1 = G.cp[k1] * y - G.sp[k1] * x;
            if (g0 >= 0.0 && g1 < 0.0) { kphi = kk; break; }
        }
    }
    if (G.coord == RT_SPHERICAL) {
        double r = sqrt((x * x + y * y) + z * z);
        int jt = G.n2 - 1;
        for (int jj = 0; jj + 1 < G.n2; ++jj) {
            if (z > G.ct[jj + 1] * r) { jt = jj; break; }
        }
        jo = jt;
        ko = kphi;
    } else {
        int kz = G.n3 - 1;
        for (int kk = 0; kk < G.n3; ++kk) {
            if (z < G.e3[kk + 1]) { kz = kk; break; }
        }
        jo = kphi;
        ko = kz;
    }
}

__device__ __forceinline__ int max_steps(const GeomDev &G) { return 4 * (G.n1 + G.n2 + G.n3) + 16; }

// Where a line crosses a given surface does not depend on the cell the walk is
// in, so each surface's candidate parameters are evaluated once per walk (by
// the same operations, in the same order, as a per-step evaluation) and kept
// for the three most recently used surfaces of each axis.  Invalid candidates
// are stored as +inf.

// Shell m: ordered roots (lo, hi), NaN when the line misses it.
__device__ __forceinline__ void shell_roots(const GeomDev &G, const Line &L, int m, double &lo, double &hi)
{
    if (!shell(G, L, m, lo, hi)) {  // no crossing: neither candidate is taken
        lo = dinf();
        hi = dinf();
    }
}

// Cone jc: the roots on its own nappe, smaller first (+inf where none).
__device__ void cone_roots(const GeomDev &G, const Line &L, int jc, double &ra, double &rb)
{
    const double INF = dinf();
    ra = INF;
    rb = INF;
    double c = G.ct[jc];
    if (fabs(c) < 1e-12) {  // the cone at theta = pi/2 is the plane z = 0
        if (L.dz != 0.0) ra = -(L.z / L.dz);
        return;
    }
    double cc = c * c;
    double A = L.dz * L.dz - cc * L.a;
    double B = L.zd - cc * L.b;
    double C = L.z2 - cc * L.p2;
    double r0, r1;
    int nr;
    if (A == 0.0) {
        if (B == 0.0) return;
        r0 = -(C / (2.0 * B));
        r1 = r0;
        nr = 1;
    } else {
        if (!roots2(A, B, C, r0, r1)) return;
        if (r0 == r1) return;  // a tangent line stays in its cell
        nr = 2;
    }
    for (int q = 0; q < nr; ++q) {
        double r = (q == 0) ? r0 : r1;
        double zz = L.z + r * L.dz;
        bool nappe = (c > 0.0) ? (zz > 0.0) : (zz < 0.0);
        if (nappe) {
            if (q == 0) ra = r;
            else rb = r;
        }
    }
}

// Half-plane phi = phi_kp bounded by the z axis: its crossing, +inf if none.
__device__ __forceinline__ double halfplane_root(const GeomDev &G, const Line &L, int kp)
{
    double c = G.cp[kp], s = G.sp[kp];
    double den = c * L.dy - s * L.dx;
    if (den == 0.0) return dinf();
    double num = c * L.y - s * L.x;
    double r = -(num / den);
    double xx = L.x + r * L.dx;
    double yy = L.y + r * L.dy;
    double h = c * xx + s * yy;
    return (h > 0.0) ? r : dinf();
}

__device__ __forceinline__ double zplane_root(const GeomDev &G, const Line &L, int m)
{
    if (L.dz == 0.0) return dinf();
    return (G.e3[m] - L.z) / L.dz;
}

// kind: 0 shell, 1 cone, 2 half-plane, 3 z-plane; three entries in scalars
// (kept in registers), replaced in turn
template <int KIND>
struct SurfCache {
    int i0, i1, i2, rr;
    double a0, a1, a2, b0, b1, b2;
    __device__ __forceinline__ void init()
    {
        i0 = i1 = i2 = -1;
        rr = 0;
        a0 = a1 = a2 = b0 = b1 = b2 = 0.0;
    }
    __device__ __forceinline__ void get(const GeomDev &G, const Line &L, int m, double &ra, double &rb)
    {
        if (i0 == m) { ra = a0; rb = b0; return; }
        if (i1 == m) { ra = a1; rb = b1; return; }
        if (i2 == m) { ra = a2; rb = b2; return; }
        if (KIND == 0) shell_roots(G, L, m, ra, rb);
        else if (KIND == 1) cone_roots(G, L, m, ra, rb);
        else if (KIND == 2) { ra = halfplane_root(G, L, m); rb = ra; }
        else { ra = zplane_root(G, L, m); rb = ra; }
        if (rr == 0) { i0 = m; a0 = ra; b0 = rb; }
        else if (rr == 1) { i1 = m; a1 = ra; b1 = rb; }
        else { i2 = m; a2 = ra; b2 = rb; }
        rr = (rr == 2) ? 0 : rr + 1;
    }
};

// the first crossing after t among one or two candidates (+inf: none)
// The step rule compares crossing parameters only with t >= 0 and among
// candidates greater than t, i.e. among positive doubles (or +inf), whose order
// is that of their bit patterns as signed 64-bit integers: the selection runs on
// the integer pipe, the values are the doubles themselves.
__device__ __forceinline__ long long bits(double x) { return __double_as_longlong(x); }

// the first crossing after t among one or two candidates (+inf: none), as bits
__device__ __forceinline__ long long after(double ra, double rb, long long tb, long long infb)
{
    const long long a = bits(ra), b = bits(rb);
    return min(a > tb ? a : infb, b > tb ? b : infb);
}

// Walk from the centre of voxel (i,j,k) along (dx,dy,dz), reporting each
// traversed cell to vis.cell(vox, t_in, t_out, after_hole).  Returns how the
// characteristic ended: left the domain, met the opaque core, or lost.
template <class Visit>
__device__ int walk(const GeomDev &G, double x0, double y0, double z0, double dx, double dy, double dz, int i,
                    int j, int k, Visit &vis)
{
    const Line L = make_line(G, x0, y0, z0, dx, dy, dz);
    const double INF = dinf();
    const bool sph = (G.coord == RT_SPHERICAL);
    SurfCache<0> csh;
    SurfCache<1> ccone;
    SurfCache<2> chp;
    SurfCache<3> czp;
    csh.init();
    ccone.init();
    chp.init();
    czp.init();
    double t = 0.0;
    int hole = 0;
    const int nsteps = max_steps(G);
    const long long INFB = bits(INF);
    for (int step = 0; step < nsteps; ++step) {
        const long long tb = bits(t);
        long long c0 = INFB, c1 = INFB, c2 = INFB, c3 = INFB, c4 = INFB, c5 = INFB;
        double lo, hi;
        if (!(i == 0 && G.e1[0] == 0.0)) {
            csh.get(G, L, i, lo, hi);
            // lo > t >= 0 makes lo and hi >= lo positive, so the bit order is theirs
            if (bits(lo) > tb && bits(lo) < bits(hi)) c0 = bits(lo);
        }
        csh.get(G, L, i + 1, lo, hi);
        if (bits(hi) > tb) c1 = bits(hi);
        double ra, rb;
        if (sph) {
            if (j >= 1) {
                ccone.get(G, L, j, ra, rb);
                c2 = after(ra, rb, tb, INFB);
            }
            if (j + 1 <= G.n2 - 1) {
                ccone.get(G, L, j + 1, ra, rb);
                c3 = after(ra, rb, tb, INFB);
            }
            if (G.n3 > 1) {
                chp.get(G, L, k, ra, rb);
                c4 = bits(ra) > tb ? bits(ra) : INFB;
                chp.get(G, L, (k + 1 == G.n3) ? 0 : k + 1, ra, rb);
                c5 = bits(ra) > tb ? bits(ra) : INFB;
            }
        } else {
            if (G.n2 > 1) {
                chp.get(G, L, j, ra, rb);
                c2 = bits(ra) > tb ? bits(ra) : INFB;
                chp.get(G, L, (j + 1 == G.n2) ? 0 : j + 1, ra, rb);
                c3 = bits(ra) > tb ? bits(ra) : INFB;
            }
            if (L.dz < 0.0) {
                czp.get(G, L, k, ra, rb);
                c4 = bits(ra) > tb ? bits(ra) : INFB;
            }
            if (L.dz > 0.0) {
                czp.get(G, L, k + 1, ra, rb);
                c5 = bits(ra) > tb ? bits(ra) : INFB;
            }
        }
        const long long best = min(min(min(c0, c1), min(c2, c3)), min(c4, c5));
        if (best == INFB) return RTK_END_LOST;
        const double bestd = __longlong_as_double(best);
        vis.cell(vid(G, i, j, k), t, bestd, hole);
        int ni = i, nj = j, nk = k;
        bool ex = false, core = false;
        if (c0 == best) { if (i == 0) core = true; else ni = i - 1; }
        if (c1 == best) { if (i == G.n1 - 1) ex = true; else ni = i + 1; }
        if (sph) {
            if (c2 == best) nj = nj - 1;
            if (c3 == best) nj = nj + 1;
            if (c4 == best) nk = (nk == 0) ? G.n3 - 1 : nk - 1;
            if (c5 == best) nk = (nk + 1 == G.n3) ? 0 : nk + 1;
        } else {
            if (c2 == best) nj = (nj == 0) ? G.n2 - 1 : nj - 1;
            if (c3 == best) nj = (nj + 1 == G.n2) ? 0 : nj + 1;
            if (c4 == best) { if (k == 0) ex = true; else nk = k - 1; }
            if (c5 == best) { if (k == G.n3 - 1) ex = true; else nk = k + 1; }
        }
        if (ex) return RTK_END_EXIT;
        double tn = bestd;
        hole = 0;
        if (core) {
            if (G.inner_bc == RT_CORE_B) return RTK_END_CORE;
            shell(G, L, 0, lo, hi);
            double tout = hi;
            if (!sph) {
                double tz = INF;
                if (L.dz > 0.0) tz = (G.e3[G.n3] - L.z) / L.dz;
                if (L.dz < 0.0) tz = (G.e3[0] - L.z) / L.dz;
                if (tz <= tout) return RTK_END_EXIT;
            }
            locate(G, L, tout, nj, nk);
            ni = 0;
            tn = tout;
            hole = 1;
        }
        i = ni; j = nj; k = nk;
        t = tn;
    }
    return RTK_END_LOST;
}

__device__ __forceinline__ void ijk_of(const GeomDev &G, int v, int &i, int &j, int &k)
{
    k = v % G.n3;
    j = (v / G.n3) % G.n2;
    i = v / (G.n3 * G.n2);
}

__device__ __forceinline__ bool outer_launch(const GeomDev &G, int i, int j, int k, double dx, double dy, double dz)
{
    if (G.coord == RT_SPHERICAL) {
        if (i != G.n1 - 1) return false;
        double c0 = G.stm[j] * G.cpm[k], c1 = G.stm[j] * G.spm[k], c2 = G.ctm[j];
        double dot = (dx * c0 + dy * c1) + dz * c2;
        return dot < 0.0;
    }
    bool side = (i == G.n1 - 1) && ((dx * G.cpm[j] + dy * G.spm[j]) < 0.0);
    bool bot = (k == 0) && (dz > 0.0);
    bool top = (k == G.n3 - 1) && (dz < 0.0);
    return side || bot || top;
}

__device__ __forceinline__ bool core_launch(const GeomDev &G, int i, int j, int k, double dx, double dy, double dz)
{
    if (G.inner_bc != RT_CORE_B || i != 0) return false;
    if (G.coord == RT_SPHERICAL) {
        double c0 = G.stm[j] * G.cpm[k], c1 = G.stm[j] * G.spm[k], c2 = G.ctm[j];
        double dot = (dx * c0 + dy * c1) + dz * c2;
        return dot > 0.0;
    }
    return (dx * G.cpm[j] + dy * G.spm[j]) > 0.0;
}

struct MarkVisit {
    uint32_t *H;
    int n;
    __device__ void cell(int v, double, double, int)
    {
        atomicOr(H + (v >> 5), 1u << (v & 31));
        n++;
    }
};

// cells of the backward and forward walk of a launched characteristic, packed
// for the segment counts (1 and 1 when a walk was lost, as the counting rule)
__device__ __forceinline__ uint32_t pack_counts(int nb, int nf, bool lost)
{
    if (lost) nb = nf = 1;
    return ((uint32_t)nb << 16) | (uint32_t)nf;
}

struct ListVisit {
    int32_t *list;
    int cap, n;
    __device__ void cell(int v, double, double, int)
    {
        if (n < cap) list[n] = v;
        n++;
    }
};

// Writes the upstream half in reverse: cell q of the backward walk goes to
// position base - q; the hole flag of cell q belongs to the cell written
// just before it (the next one downstream).
struct BackWrite {
    uint32_t *vox;
    double *l64;
    float *l32;
    int64_t base;  // position of the origin cell
    int nb;        // cells counted for this half by the counting pass
    int q;
    double t_first;  // exit parameter of the origin cell along -d
    __device__ void cell(int v, double tin, double tout, int hole)
    {
        int64_t pos = base - q;
        if (q >= nb) {  // never written outside this characteristic's range
            q++;
            return;
        }
        if (q == 0) {
            t_first = tout;
            vox[pos] = (uint32_t)v;
        } else {
            double l = tout - tin;
            vox[pos] = (uint32_t)v;
            l64[pos] = l;
            l32[pos] = (float)l;
            if (hole) vox[pos + 1] |= RTK_RESTART;
        }
        q++;
    }
};

struct FwdWrite {
    uint32_t *vox;
    double *l64;
    float *l32;
    int64_t base;
    int nf;  // cells of this half that fit the characteristic's range
    int p;
    double t_back;
    __device__ void cell(int v, double tin, double tout, int hole)
    {
        int64_t pos = base + p;
        if (p >= nf) {
            p++;
            return;
        }
        if (p == 0) {
            double l = t_back + tout;
            l64[pos] = l;
            l32[pos] = (float)l;
        } else {
            double l = tout - tin;
            vox[pos] = (uint32_t)v | (hole ? RTK_RESTART : 0u);
            l64[pos] = l;
            l32[pos] = (float)l;
        }
        p++;
    }
};

__global__ void k_mark_boundary(GeomDev G, const double *dirs, int w0, int nw, uint32_t *hit, int words, int *lost,
                                uint32_t *cnt)
{
    int64_t total = (int64_t)nw * G.nvox;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        int wl = (int)(idx / G.nvox);
        int v = (int)(idx - (int64_t)wl * G.nvox);
        int w = w0 + wl;
        int i, j, k;
        ijk_of(G, v, i, j, k);
        double dx = dirs[3 * w], dy = dirs[3 * w + 1], dz = dirs[3 * w + 2];
        if (!outer_launch(G, i, j, k, dx, dy, dz) && !core_launch(G, i, j, k, dx, dy, dz)) continue;
        double x, y, z;
        centre_of(G, i, j, k, x, y, z);
        MarkVisit mv{hit + (int64_t)wl * words, 0};
        int eb = walk(G, x, y, z, -dx, -dy, -dz, i, j, k, mv);
        const int nb = mv.n;
        int ef = walk(G, x, y, z, dx, dy, dz, i, j, k, mv);
        const bool bad = eb == RTK_END_LOST || ef == RTK_END_LOST;
        if (bad) atomicAdd(lost, 1);
        cnt[(int64_t)w * G.nvox + v] = pack_counts(nb, mv.n - nb, bad);
    }
}

__device__ __forceinline__ uint32_t read_word(uint32_t *p) { return atomicOr(p, 0u); }

// One warp per solid angle.  The warp takes the next (up to) 32 voxels that
// are not yet hit, traces the 32 characteristics through their centres in
// parallel, then accepts them in voxel order: candidate m is kept only if no
// accepted characteristic of a lower voxel has hit it, exactly as a serial
// pass in increasing voxel index would decide.
// One warp per CTA: the CTAs, one per solid angle, spread over every SM (the
// walks are FP64-bound, so SMs with more solid angles than others finish last).
constexpr int CPL_WARPS = 1;

__global__ void __launch_bounds__(32 * CPL_WARPS) k_complete(GeomDev G, const double *dirs, int w0, int nw, uint32_t *hit,
                                                  uint32_t *comp, int words, int32_t *scratch, int cap, int *lost,
                                                  uint32_t *cnt)
{
    __shared__ int cand_s[CPL_WARPS][32];
    const int wib = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int wl = blockIdx.x * CPL_WARPS + wib;
    if (wl >= nw) return;
    const int w = w0 + wl;
    const double dx = dirs[3 * w], dy = dirs[3 * w + 1], dz = dirs[3 * w + 2];
    uint32_t *H = hit + (int64_t)wl * words;
    uint32_t *C = comp + (int64_t)wl * words;
    int32_t *mylist = scratch + ((int64_t)wl * 32 + lane) * cap;
    int *cand = cand_s[wib];
    int pos = 0;
    while (pos < G.nvox) {
        // collect up to 32 unhit voxels in increasing order
        int ncand = 0;
        int scan = pos;
        while (ncand < 32 && scan < G.nvox) {
            uint32_t w0w = 0, w1w = 0;
            if (lane == 0) {
                w0w = read_word(H + (scan >> 5));
                if ((scan >> 5) + 1 < words) w1w = read_word(H + (scan >> 5) + 1);
            }
            w0w = __shfl_sync(0xffffffffu, w0w, 0);
            w1w = __shfl_sync(0xffffffffu, w1w, 0);
            int v = scan + lane;
            uint32_t word = ((v >> 5) == (scan >> 5)) ? w0w : w1w;
            bool unhit = (v < G.nvox) && !((word >> (v & 31)) & 1u);
            uint32_t m = __ballot_sync(0xffffffffu, unhit);
            int need = 32 - ncand;
            int cnt = __popc(m);
            int last_taken_lane = 31;
            if (cnt > need) {
                // keep the first `need` set bits
                uint32_t mm = m;
                for (int q = 0; q < need; ++q) mm &= mm - 1;
                m &= ~mm;
                last_taken_lane = 31 - __clz(m);
            }
            if (unhit && ((m >> lane) & 1u)) {
                int rank = __popc(m & ((1u << lane) - 1u));
                cand[ncand + rank] = v;
            }
            ncand += __popc(m);
            scan += (cnt > need) ? last_taken_lane + 1 : 32;
            __syncwarp();
        }
        pos = scan;
        // trace the candidates
        int nl = 0, bad = 0;
        uint32_t pc = 0;  // packed walk counts of this lane's candidate
        if (lane < ncand) {
            int v = cand[lane];
            int i, j, k;
            ijk_of(G, v, i, j, k);
            double x, y, z;
            centre_of(G, i, j, k, x, y, z);
            ListVisit lv{mylist, cap, 0};
            int eb = walk(G, x, y, z, -dx, -dy, -dz, i, j, k, lv);
            const int nbk = lv.n;
            int ef = walk(G, x, y, z, dx, dy, dz, i, j, k, lv);
            nl = lv.n < cap ? lv.n : cap;
            bad = (eb == RTK_END_LOST || ef == RTK_END_LOST || lv.n > cap) ? 1 : 0;
            pc = pack_counts(nbk, lv.n - nbk, eb == RTK_END_LOST || ef == RTK_END_LOST);
        }
        __syncwarp();
        // accept in voxel order
        for (int m = 0; m < ncand; ++m) {
            int v = cand[m];
            int n_m = __shfl_sync(0xffffffffu, nl, m);
            int bad_m = __shfl_sync(0xffffffffu, bad, m);
            const uint32_t pc_m = __shfl_sync(0xffffffffu, pc, m);
            uint32_t word = 0;
            if (lane == 0) word = read_word(H + (v >> 5));
            word = __shfl_sync(0xffffffffu, word, 0);
            if (!((word >> (v & 31)) & 1u)) {
                if (bad_m) {
                    if (lane == 0) {
                        atomicOr(H + (v >> 5), 1u << (v & 31));
                        atomicAdd(lost, 1);
                    }
                } else {
                    if (lane == 0) {
                        atomicOr(C + (v >> 5), 1u << (v & 31));
                        cnt[(int64_t)w * G.nvox + v] = pc_m;
                    }
                    const int32_t *lst = scratch + ((int64_t)wl * 32 + m) * cap;
                    for (int e = lane; e < n_m; e += 32) {
                        int u = lst[e];
                        atomicOr(H + (u >> 5), 1u << (u & 31));
                    }
                }
            }
            __syncwarp();
        }
    }
}

// Candidates the predictor may hold back in one round of k_complete_pred.
constexpr int PRED_PREFIX = 256;

struct PredVisit {
    int32_t *list;
    int cap, n;
    __device__ void cell(int v)
    {
        if (n < cap) list[n] = v;
        n++;
    }
};

// The coverage completion of k_complete with a guess of which candidates will
// be hit.  A round looks at the unhit voxels in increasing order, 32 at a time:
// each is walked in float (pwalk) and, in voxel order, either held back (an
// earlier chosen candidate's guessed line crosses it: stamp[v] == round) or
// chosen, up to 32 chosen; the chosen ones are traced exactly (FP64 walk) and
// then every voxel of the round is decided in voxel order as the serial rule
// does: a voxel hit by then is skipped, a chosen unhit one is launched, and a
// held-back unhit one ends the round (it is the next round's first candidate,
// which is always chosen, so every round launches at least one characteristic).
__global__ void __launch_bounds__(32) k_complete_pred(GeomDev G, GeomF F, const double *dirs, int w0, int nw,
                                                      uint32_t *hit, uint32_t *comp, int words, int32_t *scratch,
                                                      int32_t *pscr, int32_t *stamp, int cap, int *lost,
                                                      uint32_t *cnt)
{
    __shared__ int cand[32];
    __shared__ int prefv[PRED_PREFIX];
    __shared__ uint32_t prefsel[PRED_PREFIX / 32];
    __shared__ int selv[32];
    const int lane = threadIdx.x & 31;
    const int wl = blockIdx.x;
    if (wl >= nw) return;
    const int w = w0 + wl;
    const double dx = dirs[3 * w], dy = dirs[3 * w + 1], dz = dirs[3 * w + 2];
    const float fdx = (float)dx, fdy = (float)dy, fdz = (float)dz;
    uint32_t *H = hit + (int64_t)wl * words;
    uint32_t *C = comp + (int64_t)wl * words;
    int32_t *mylist = scratch + ((int64_t)wl * 32 + lane) * cap;
    int32_t *myplist = pscr + ((int64_t)wl * 32 + lane) * cap;
    volatile int32_t *ST = stamp + (int64_t)wl * G.nvox;
    int pos = 0, round = 0;
    while (pos < G.nvox) {
        ++round;
        if (lane < PRED_PREFIX / 32) prefsel[lane] = 0u;
        int npref = 0, nsel = 0, scan = pos;
        bool full = false;
        __syncwarp();
        while (!full && npref < PRED_PREFIX && scan < G.nvox) {
            // the next unhit voxels, in increasing order
            const int want = min(32, PRED_PREFIX - npref);
            int ncand = 0, cscan = scan;
            while (ncand < want && cscan < G.nvox) {
                uint32_t w0w = 0, w1w = 0;
                if (lane == 0) {
                    w0w = read_word(H + (cscan >> 5));
                    if ((cscan >> 5) + 1 < words) w1w = read_word(H + (cscan >> 5) + 1);
                }
                w0w = __shfl_sync(0xffffffffu, w0w, 0);
                w1w = __shfl_sync(0xffffffffu, w1w, 0);
                const int v = cscan + lane;
                const uint32_t word = ((v >> 5) == (cscan >> 5)) ? w0w : w1w;
                const bool unhit = (v < G.nvox) && !((word >> (v & 31)) & 1u);
                uint32_t m = __ballot_sync(0xffffffffu, unhit);
                const int need = want - ncand;
                const int cntm = __popc(m);
                int last_taken_lane = 31;
                if (cntm > need) {
                    uint32_t mm = m;
                    for (int q = 0; q < need; ++q) mm &= mm - 1;
                    m &= ~mm;
                    last_taken_lane = 31 - __clz(m);
                }
                if (unhit && ((m >> lane) & 1u)) cand[ncand + __popc(m & ((1u << lane) - 1u))] = v;
                ncand += __popc(m);
                cscan += (cntm > need) ? last_taken_lane + 1 : 32;
                __syncwarp();
            }
            // guessed lines of this batch
            int pn = 0;
            if (lane < ncand) {
                const int v = cand[lane];
                int i, j, k;
                ijk_of(G, v, i, j, k);
                float x, y, z;
                pcentre(F, i, j, k, x, y, z);
                PredVisit pv{myplist, cap, 0};
                pwalk(F, x, y, z, -fdx, -fdy, -fdz, i, j, k, pv);
                pwalk(F, x, y, z, fdx, fdy, fdz, i, j, k, pv);
                pn = pv.n < cap ? pv.n : cap;
            }
            __syncwarp();
            // choose in voxel order
            int m = 0;
            for (; m < ncand; ++m) {
                const int v = cand[m];
                int sv = 0;
                if (lane == 0) sv = ST[v];
                sv = __shfl_sync(0xffffffffu, sv, 0);
                if (sv == round && nsel > 0) {  // held back (the round's first candidate never is)
                    if (lane == 0) prefv[npref] = v;
                    npref++;
                    continue;
                }
                if (nsel == 32) break;  // round full: v starts the next one
                if (lane == 0) {
                    prefv[npref] = v;
                    prefsel[npref >> 5] |= 1u << (npref & 31);
                    selv[nsel] = v;
                }
                npref++;
                nsel++;
                const int n_m = __shfl_sync(0xffffffffu, pn, m);
                const int32_t *pl = pscr + ((int64_t)wl * 32 + m) * cap;
                for (int e = lane; e < n_m; e += 32) ST[pl[e]] = round;
                __syncwarp();
            }
            if (m < ncand) {
                scan = cand[m];
                full = true;
            } else {
                scan = cscan;
            }
            __syncwarp();
        }
        // exact traces of the chosen candidates
        int nl = 0, bad = 0;
        uint32_t pc = 0;
        if (lane < nsel) {
            const int v = selv[lane];
            int i, j, k;
            ijk_of(G, v, i, j, k);
            double x, y, z;
            centre_of(G, i, j, k, x, y, z);
            ListVisit lv{mylist, cap, 0};
            const int eb = walk(G, x, y, z, -dx, -dy, -dz, i, j, k, lv);
            const int nbk = lv.n;
            const int ef = walk(G, x, y, z, dx, dy, dz, i, j, k, lv);
            nl = lv.n < cap ? lv.n : cap;
            bad = (eb == RTK_END_LOST || ef == RTK_END_LOST || lv.n > cap) ? 1 : 0;
            pc = pack_counts(nbk, lv.n - nbk, eb == RTK_END_LOST || ef == RTK_END_LOST);
        }
        __syncwarp();
        // decide in voxel order
        int next = scan, si = 0;
        for (int e = 0; e < npref; ++e) {
            const int v = prefv[e];
            const bool sel = (prefsel[e >> 5] >> (e & 31)) & 1u;
            const int m = si;
            if (sel) si++;
            uint32_t word = 0;
            if (lane == 0) word = read_word(H + (v >> 5));
            word = __shfl_sync(0xffffffffu, word, 0);
            if ((word >> (v & 31)) & 1u) continue;  // hit by then: no launch, as in the serial rule
            if (!sel) {  // unhit but not traced: the next round starts here
                next = v;
                break;
            }
            const int n_m = __shfl_sync(0xffffffffu, nl, m);
            const int bad_m = __shfl_sync(0xffffffffu, bad, m);
            const uint32_t pc_m = __shfl_sync(0xffffffffu, pc, m);
            if (bad_m) {
                if (lane == 0) {
                    atomicOr(H + (v >> 5), 1u << (v & 31));
                    atomicAdd(lost, 1);
                }
            } else {
                if (lane == 0) {
                    atomicOr(C + (v >> 5), 1u << (v & 31));
                    cnt[(int64_t)w * G.nvox + v] = pc_m;
                }
                const int32_t *lst = scratch + ((int64_t)wl * 32 + m) * cap;
                for (int q = lane; q < n_m; q += 32) {
                    const int u = lst[q];
                    atomicOr(H + (u >> 5), 1u << (u & 31));
                }
            }
            __syncwarp();
        }
        pos = next;
    }
}

__device__ __forceinline__ int ray_kind(const GeomDev &G, int pass, int v, double dx, double dy, double dz,
                                        const uint32_t *C)
{
    int i, j, k;
    ijk_of(G, v, i, j, k);
    if (pass == 0) return outer_launch(G, i, j, k, dx, dy, dz);
    if (pass == 1) return core_launch(G, i, j, k, dx, dy, dz);
    return (C[v >> 5] >> (v & 31)) & 1u;
}

__global__ void __launch_bounds__(256) k_count_rays(GeomDev G, const double *dirs, const uint32_t *comp, int words,
                                                    int32_t *counts)
{
    const int w = blockIdx.x;
    const double dx = dirs[3 * w], dy = dirs[3 * w + 1], dz = dirs[3 * w + 2];
    const uint32_t *C = comp + (int64_t)w * words;
    int n = 0;
    for (int pass = 0; pass < 3; ++pass)
        for (int v = threadIdx.x; v < G.nvox; v += blockDim.x) n += ray_kind(G, pass, v, dx, dy, dz, C);
    __shared__ int red[256];
    red[threadIdx.x] = n;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) counts[w] = red[0];
}

__global__ void __launch_bounds__(256) k_list_rays(GeomDev G, const double *dirs, const uint32_t *comp, int words,
                                                   const int64_t *ang_ray_off, int32_t *ray_origin,
                                                   int32_t *ray_angle)
{
    __shared__ int wsum[8];
    const int w = blockIdx.x;
    const double dx = dirs[3 * w], dy = dirs[3 * w + 1], dz = dirs[3 * w + 2];
    const uint32_t *C = comp + (int64_t)w * words;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int64_t base = ang_ray_off[w];
    for (int pass = 0; pass < 3; ++pass) {
        for (int c0 = 0; c0 < G.nvox; c0 += 256) {
            int v = c0 + threadIdx.x;
            int f = (v < G.nvox) ? ray_kind(G, pass, v, dx, dy, dz, C) : 0;
            uint32_t m = __ballot_sync(0xffffffffu, f);
            int rank = __popc(m & ((1u << lane) - 1u));
            if (lane == 0) wsum[wid] = __popc(m);
            __syncthreads();
            int before = 0, total = 0;
            for (int q = 0; q < 8; ++q) {
                if (q < wid) before += wsum[q];
                total += wsum[q];
            }
            if (f) {
                ray_origin[base + before + rank] = v;
                ray_angle[base + before + rank] = w;
            }
            base += total;
            __syncthreads();
        }
    }
}

// Segment counts of every characteristic from the walks of the launch-set pass.
__global__ void k_gather_counts(int nvox, int64_t n_rays, const int32_t *ray_origin, const int32_t *ray_angle,
                                const uint32_t *cnt, int32_t *nseg, int32_t *nback)
{
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n_rays; r += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t c = cnt[(int64_t)ray_angle[r] * nvox + ray_origin[r]];
        const int nb = (int)(c >> 16), nf = (int)(c & 0xffffu);
        nseg[r] = nb + nf - 1;
        nback[r] = nb;
    }
}

__global__ void k_write_segs(GeomDev G, const double *dirs, int64_t n_rays, const int32_t *ray_origin,
                             const int32_t *ray_angle, const int64_t *ray_off, const int32_t *nback, uint32_t *vox,
                             double *len64, float *len32, int *lost)
{
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n_rays; r += (int64_t)gridDim.x * blockDim.x) {
        int v = ray_origin[r], w = ray_angle[r];
        double dx = dirs[3 * w], dy = dirs[3 * w + 1], dz = dirs[3 * w + 2];
        int i, j, k;
        ijk_of(G, v, i, j, k);
        double x, y, z;
        centre_of(G, i, j, k, x, y, z);
        int64_t off = ray_off[r];
        int nb = nback[r];
        int64_t expect = ray_off[r + 1] - off;
        BackWrite bw{vox, len64, len32, off + nb - 1, nb, 0, 0.0};
        int eb = walk(G, x, y, z, -dx, -dy, -dz, i, j, k, bw);
        FwdWrite fw{vox, len64, len32, off + nb - 1, (int)(expect - nb + 1), 0, bw.t_first};
        int ef = walk(G, x, y, z, dx, dy, dz, i, j, k, fw);
        if (eb == RTK_END_LOST || ef == RTK_END_LOST || bw.q != nb || (int64_t)(nb + fw.p - 1) != expect) {
            atomicAdd(lost, 1);
            continue;
        }
        vox[off] |= RTK_RAYSTART | ((eb == RTK_END_CORE) ? RTK_CORE : 0u);
    }
}

int blocks_for(int64_t n, int threads)
{
    int64_t b = (n + threads - 1) / threads;
    if (b > 152 * 64) b = 152 * 64;
    if (b < 1) b = 1;
    return (int)b;
}

}  // namespace

int geom_scratch_cap(const GeomDev &G) { return 2 * (4 * (G.n1 + G.n2 + G.n3) + 16) + 8; }

cudaError_t geom_mark_boundary(const GeomDev &G, const double *dirs, int w0, int nw, uint32_t *hit, int words,
                               int *lost, uint32_t *cnt, cudaStream_t st)
{
    int64_t total = (int64_t)nw * G.nvox;
    k_mark_boundary<<<blocks_for(total, 256), 256, 0, st>>>(G, dirs, w0, nw, hit, words, lost, cnt);
    return cudaGetLastError();
}

cudaError_t geom_complete(const GeomDev &G, const double *dirs, int w0, int nw, uint32_t *hit, uint32_t *comp,
                          int words, int32_t *scratch, int cap, int *lost, uint32_t *cnt, cudaStream_t st)
{
    k_complete<<<(nw + CPL_WARPS - 1) / CPL_WARPS, 32 * CPL_WARPS, 0, st>>>(G, dirs, w0, nw, hit, comp, words, scratch,
                                                                           cap, lost, cnt);
    return cudaGetLastError();
}

cudaError_t geom_complete_pred(const GeomDev &G, const GeomF &F, const double *dirs, int w0, int nw, uint32_t *hit,
                               uint32_t *comp, int words, int32_t *scratch, int32_t *pscr, int32_t *stamp, int cap,
                               int *lost, uint32_t *cnt, cudaStream_t st)
{
    k_complete_pred<<<nw, 32, 0, st>>>(G, F, dirs, w0, nw, hit, comp, words, scratch, pscr, stamp, cap, lost, cnt);
    return cudaGetLastError();
}

cudaError_t geom_count_rays(const GeomDev &G, const double *dirs, int n_ang, const uint32_t *comp, int words,
                            int32_t *counts, cudaStream_t st)
{
    k_count_rays<<<n_ang, 256, 0, st>>>(G, dirs, comp, words, counts);
    return cudaGetLastError();
}

cudaError_t geom_list_rays(const GeomDev &G, const double *dirs, int n_ang, const uint32_t *comp, int words,
                           const int64_t *ang_ray_off, int32_t *ray_origin, int32_t *ray_angle, cudaStream_t st)
{
    k_list_rays<<<n_ang, 256, 0, st>>>(G, dirs, comp, words, ang_ray_off, ray_origin, ray_angle);
    return cudaGetLastError();
}

cudaError_t geom_gather_counts(int nvox, int64_t n_rays, const int32_t *ray_origin, const int32_t *ray_angle,
                               const uint32_t *cnt, int32_t *nseg, int32_t *nback, cudaStream_t st)
{
    k_gather_counts<<<blocks_for(n_rays, 256), 256, 0, st>>>(nvox, n_rays, ray_origin, ray_angle, cnt, nseg, nback);
    return cudaGetLastError();
}

cudaError_t geom_write_segs(const GeomDev &G, const double *dirs, int64_t n_rays, const int32_t *ray_origin,
                            const int32_t *ray_angle, const int64_t *ray_off, const int32_t *nback, uint32_t *vox,
                            double *len64, float *len32, int *lost, cudaStream_t st)
{
    k_write_segs<<<blocks_for(n_rays, 128), 128, 0, st>>>(G, dirs, n_rays, ray_origin, ray_angle, ray_off, nback, vox,
                                                          len64, len32, lost);
    return cudaGetLastError();
}

}  // namespace rtk
