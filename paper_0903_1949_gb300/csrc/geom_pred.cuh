// geom_pred.cuh -- single-precision guess of the voxels a characteristic
// crosses, for the coverage completion of the launch set (Sect. 2: every
// voxel hit at least once per solid angle, characteristics launched in voxel
// order).  The completion traces candidate voxels speculatively and accepts
// them in voxel order; this walk predicts which later candidates an earlier
// candidate's characteristic will hit, so that fewer traced candidates turn out
// to be hit already.  Nothing it returns enters the crossing lists or decides
// a launch: the exact FP64 walk does both, and a wrong guess only ends a round
// of the completion early.
//
// The step rule is that of the FP64 walk (nearest bounding surface of the
// current cell after the current parameter; shells, cones and half-planes, or
// cylinders, half-planes and z-planes), evaluated per step in float without a
// cache.  Host and device compile the same code (the CPU tests run it against
// the oracle's launch sets).
#pragma once

#include <math.h>
#include <stdint.h>

#include "rt.h"

#ifdef __CUDACC__
#define RTK_HD __host__ __device__
#else
#define RTK_HD
#endif

namespace rtk {

// Float copies of the geometry tables (same meaning as GeomDev's).
struct GeomF {
    int coord, n1, n2, n3, nphi, inner_bc, nvox;
    const float *e1, *e3;     // radial (or R) edges; z edges (cylindrical)
    const float *ct;          // cos(theta_j), j = 0..n2 (spherical)
    const float *ctm, *stm;   // cos/sin of theta mid-points (spherical)
    const float *cp, *sp;     // cos/sin of phi_k
    const float *cpm, *spm;   // cos/sin of phi mid-points
};

enum { PRED_EXIT = 0, PRED_CORE = 1, PRED_LOST = 2 };

struct PLine {
    float x, y, z, dx, dy, dz, a, b, p2, zd, z2;
};

RTK_HD inline float pinf() { return HUGE_VALF; }

RTK_HD inline int pvid(const GeomF &G, int i, int j, int k) { return (i * G.n2 + j) * G.n3 + k; }

RTK_HD inline void pcentre(const GeomF &G, int i, int j, int k, float &x, float &y, float &z)
{
    if (G.coord == RT_SPHERICAL) {
        float rm = 0.5f * (G.e1[i] + G.e1[i + 1]);
        float w = rm * G.stm[j];
        x = w * G.cpm[k];
        y = w * G.spm[k];
        z = rm * G.ctm[j];
    } else {
        float Rm = 0.5f * (G.e1[i] + G.e1[i + 1]);
        x = Rm * G.cpm[j];
        y = Rm * G.spm[j];
        z = 0.5f * (G.e3[k] + G.e3[k + 1]);
    }
}

RTK_HD inline bool proots(float A, float B, float C, float &lo, float &hi)
{
    float disc = B * B - A * C;
    if (!(disc > 0.0f)) return false;
    float s = sqrtf(disc);
    float q = (B >= 0.0f) ? -(B + s) : (s - B);
    float r1 = q / A, r2 = C / q;
    lo = r1 <= r2 ? r1 : r2;
    hi = r1 <= r2 ? r2 : r1;
    return true;
}

RTK_HD inline bool pshell(const GeomF &G, const PLine &L, int m, float &lo, float &hi)
{
    if (!(L.a > 0.0f)) return false;
    float rm = G.e1[m];
    return proots(L.a, L.b, L.p2 - rm * rm, lo, hi);
}

// first crossing after t of the cone theta = theta_jc on its own nappe
RTK_HD inline float pcone(const GeomF &G, const PLine &L, int jc, float t)
{
    const float INF = pinf();
    float c = G.ct[jc];
    if (fabsf(c) < 1e-12f) {  // the plane z = 0
        if (L.dz == 0.0f) return INF;
        float r = -(L.z / L.dz);
        return r > t ? r : INF;
    }
    float cc = c * c;
    float A = L.dz * L.dz - cc * L.a;
    float B = L.zd - cc * L.b;
    float C = L.z2 - cc * L.p2;
    float r0, r1;
    int nr;
    if (A == 0.0f) {
        if (B == 0.0f) return INF;
        r0 = -(C / (2.0f * B));
        r1 = r0;
        nr = 1;
    } else {
        if (!proots(A, B, C, r0, r1)) return INF;
        if (r0 == r1) return INF;
        nr = 2;
    }
    float best = INF;
    for (int q = 0; q < nr; ++q) {
        float r = q == 0 ? r0 : r1;
        float zz = L.z + r * L.dz;
        bool nappe = c > 0.0f ? zz > 0.0f : zz < 0.0f;
        if (nappe && r > t && r < best) best = r;
    }
    return best;
}

// crossing after t of the half-plane phi = phi_kp bounded by the z axis
RTK_HD inline float phalf(const GeomF &G, const PLine &L, int kp, float t)
{
    float c = G.cp[kp], s = G.sp[kp];
    float den = c * L.dy - s * L.dx;
    if (den == 0.0f) return pinf();
    float r = -((c * L.y - s * L.x) / den);
    float h = c * (L.x + r * L.dx) + s * (L.y + r * L.dy);
    return (h > 0.0f && r > t) ? r : pinf();
}

// angular cell at parameter t (after crossing a transparent hole)
RTK_HD inline void plocate(const GeomF &G, const PLine &L, float t, int &jo, int &ko)
{
    float x = L.x + t * L.dx, y = L.y + t * L.dy, z = L.z + t * L.dz;
    int kphi = 0;
    if (G.nphi > 1) {
        for (int kk = 0; kk < G.nphi; ++kk) {
            int k1 = (kk + 1 == G.nphi) ? 0 : kk + 1;
            if (G.cp[kk] * y - G.sp[kk] * x >= 0.0f && G.cp[k1] * y - G.sp[k1] * x < 0.0f) {
                kphi = kk;
                break;
            }
        }
    }
    if (G.coord == RT_SPHERICAL) {
        float r = sqrtf(x * x + y * y + z * z);
        int jt = G.n2 - 1;
        for (int jj = 0; jj + 1 < G.n2; ++jj)
            if (z > G.ct[jj + 1] * r) {
                jt = jj;
                break;
            }
        jo = jt;
        ko = kphi;
    } else {
        int kz = G.n3 - 1;
        for (int kk = 0; kk < G.n3; ++kk)
            if (z < G.e3[kk + 1]) {
                kz = kk;
                break;
            }
        jo = kphi;
        ko = kz;
    }
}

// Walk from (x0, y0, z0) in cell (i, j, k) along (dx, dy, dz), reporting each
// cell to vis.cell(voxel); at most 4 (n1 + n2 + n3) + 16 steps.
template <class Visit>
RTK_HD int pwalk(const GeomF &G, float x0, float y0, float z0, float dx, float dy, float dz, int i, int j, int k,
                 Visit &vis)
{
    const bool sph = G.coord == RT_SPHERICAL;
    PLine L;
    L.x = x0; L.y = y0; L.z = z0;
    L.dx = dx; L.dy = dy; L.dz = dz;
    if (sph) {
        L.a = dx * dx + dy * dy + dz * dz;
        L.b = x0 * dx + y0 * dy + z0 * dz;
        L.p2 = x0 * x0 + y0 * y0 + z0 * z0;
    } else {
        L.a = dx * dx + dy * dy;
        L.b = x0 * dx + y0 * dy;
        L.p2 = x0 * x0 + y0 * y0;
    }
    L.zd = z0 * dz;
    L.z2 = z0 * z0;
    const float INF = pinf();
    const int nsteps = 4 * (G.n1 + G.n2 + G.n3) + 16;
    float t = 0.0f;
    for (int step = 0; step < nsteps; ++step) {
        float c0 = INF, c1 = INF, c2 = INF, c3 = INF, c4 = INF, c5 = INF, lo, hi;
        if (!(i == 0 && G.e1[0] == 0.0f))
            if (pshell(G, L, i, lo, hi) && lo > t && lo < hi) c0 = lo;
        if (pshell(G, L, i + 1, lo, hi) && hi > t) c1 = hi;
        if (sph) {
            if (j >= 1) c2 = pcone(G, L, j, t);
            if (j + 1 <= G.n2 - 1) c3 = pcone(G, L, j + 1, t);
            if (G.n3 > 1) {
                c4 = phalf(G, L, k, t);
                c5 = phalf(G, L, k + 1 == G.n3 ? 0 : k + 1, t);
            }
        } else {
            if (G.n2 > 1) {
                c2 = phalf(G, L, j, t);
                c3 = phalf(G, L, j + 1 == G.n2 ? 0 : j + 1, t);
            }
            if (L.dz < 0.0f) {
                float r = (G.e3[k] - L.z) / L.dz;
                if (r > t) c4 = r;
            }
            if (L.dz > 0.0f) {
                float r = (G.e3[k + 1] - L.z) / L.dz;
                if (r > t) c5 = r;
            }
        }
        float best = fminf(fminf(fminf(c0, c1), fminf(c2, c3)), fminf(c4, c5));
        if (!(best < INF)) return PRED_LOST;
        vis.cell(pvid(G, i, j, k));
        int ni = i, nj = j, nk = k;
        bool ex = false, core = false;
        if (c0 == best) {
            if (i == 0) core = true;
            else ni = i - 1;
        }
        if (c1 == best) {
            if (i == G.n1 - 1) ex = true;
            else ni = i + 1;
        }
        if (sph) {
            if (c2 == best) nj = nj - 1;
            if (c3 == best) nj = nj + 1;
            if (c4 == best) nk = nk == 0 ? G.n3 - 1 : nk - 1;
            if (c5 == best) nk = nk + 1 == G.n3 ? 0 : nk + 1;
        } else {
            if (c2 == best) nj = nj == 0 ? G.n2 - 1 : nj - 1;
            if (c3 == best) nj = nj + 1 == G.n2 ? 0 : nj + 1;
            if (c4 == best) {
                if (k == 0) ex = true;
                else nk = k - 1;
            }
            if (c5 == best) {
                if (k == G.n3 - 1) ex = true;
                else nk = k + 1;
            }
        }
        if (ex) return PRED_EXIT;
        float tn = best;
        if (core) {
            if (G.inner_bc == RT_CORE_B) return PRED_CORE;
            if (!pshell(G, L, 0, lo, hi)) return PRED_LOST;
            float tout = hi;
            if (!sph) {
                float tz = INF;
                if (L.dz > 0.0f) tz = (G.e3[G.n3] - L.z) / L.dz;
                if (L.dz < 0.0f) tz = (G.e3[0] - L.z) / L.dz;
                if (tz <= tout) return PRED_EXIT;
            }
            plocate(G, L, tout, nj, nk);
            ni = 0;
            tn = tout;
        }
        if (!(tn > t)) return PRED_LOST;  // no progress at float resolution: the guess ends here
        if (nj < 0 || nj >= G.n2 || nk < 0 || nk >= G.n3) return PRED_LOST;
        i = ni;
        j = nj;
        k = nk;
        t = tn;
    }
    return PRED_LOST;
}

}  // namespace rtk
