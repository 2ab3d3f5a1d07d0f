// Host build of the library's float predictor walk (csrc/geom_pred.cuh) for
// the CPU tests: the guided coverage completion is replayed in Python against
// the oracle's launch sets with exactly the guesses the GPU kernel makes (the
// header is plain IEEE float arithmetic, compiled here without contraction).
#include <cmath>
#include <cstdint>
#include <vector>

#include "geom_pred.cuh"

namespace {

struct Pred {
    std::vector<float> e1, e3, ct, ctm, stm, cp, sp, cpm, spm;
    rtk::GeomF F{};
};

struct ListOut {
    int32_t *out;
    int cap, n;
    void cell(int v)
    {
        if (n < cap) out[n] = v;
        n++;
    }
};

}  // namespace

extern "C" {

// Tables as the library uploads them for the guided completion: cos/sin in
// double of the edges and edge mid-points, rounded to float.
void *pred_create(int coord, int n1, int n2, int n3, int inner_bc, const double *e1, const double *e2,
                  const double *e3)
{
    Pred *p = new Pred;
    const bool sph = coord == RT_SPHERICAL;
    const int nphi = sph ? n3 : n2;
    const double *pe = sph ? e3 : e2;
    for (int k = 0; k < nphi; ++k) {
        const double pm = 0.5 * (pe[k] + pe[k + 1]);
        p->cp.push_back((float)std::cos(pe[k]));
        p->sp.push_back((float)std::sin(pe[k]));
        p->cpm.push_back((float)std::cos(pm));
        p->spm.push_back((float)std::sin(pm));
    }
    if (sph) {
        for (int j = 0; j <= n2; ++j) p->ct.push_back((float)std::cos(e2[j]));
        for (int j = 0; j < n2; ++j) {
            const double tm = 0.5 * (e2[j] + e2[j + 1]);
            p->ctm.push_back((float)std::cos(tm));
            p->stm.push_back((float)std::sin(tm));
        }
    } else {
        p->ct.assign(1, 0.0f);
        p->ctm.assign(1, 0.0f);
        p->stm.assign(1, 0.0f);
    }
    for (int i = 0; i <= n1; ++i) p->e1.push_back((float)e1[i]);
    for (int k = 0; k <= n3; ++k) p->e3.push_back((float)e3[k]);
    rtk::GeomF &F = p->F;
    F.coord = coord;
    F.n1 = n1;
    F.n2 = n2;
    F.n3 = n3;
    F.nphi = nphi;
    F.inner_bc = inner_bc;
    F.nvox = n1 * n2 * n3;
    F.e1 = p->e1.data();
    F.e3 = p->e3.data();
    F.ct = p->ct.data();
    F.ctm = p->ctm.data();
    F.stm = p->stm.data();
    F.cp = p->cp.data();
    F.sp = p->sp.data();
    F.cpm = p->cpm.data();
    F.spm = p->spm.data();
    return p;
}

void pred_destroy(void *h) { delete (Pred *)h; }

// Guessed cells of the characteristic through the centre of voxel v along
// (dx, dy, dz): the backward walk, then the forward walk (the origin twice),
// as the completion kernel records them; returns the count (entries beyond cap
// are not written).
int pred_line(void *h, double dx, double dy, double dz, int v, int32_t *out, int cap)
{
    const rtk::GeomF &F = ((Pred *)h)->F;
    const int k = v % F.n3, j = (v / F.n3) % F.n2, i = v / (F.n3 * F.n2);
    float x, y, z;
    rtk::pcentre(F, i, j, k, x, y, z);
    const float fx = (float)dx, fy = (float)dy, fz = (float)dz;
    ListOut lo{out, cap, 0};
    rtk::pwalk(F, x, y, z, -fx, -fy, -fz, i, j, k, lo);
    rtk::pwalk(F, x, y, z, fx, fy, fz, i, j, k, lo);
    return lo.n;
}

}  // extern "C"
