// coef.cuh -- interpolation weights of one segment of the long-characteristic
// formal solution (voxel-node parabolic scheme R6 with series-stable
// evaluation R7), shared by the forward march and the adjoint march.
#pragma once

#include <cuda_runtime.h>

namespace rtk {

// 1/n! for n = 0..20
__device__ __forceinline__ double inv_fact(int n)
{
    const double f[21] = {1.0,
                          1.0,
                          1.0 / 2.0,
                          1.0 / 6.0,
                          1.0 / 24.0,
                          1.0 / 120.0,
                          1.0 / 720.0,
                          1.0 / 5040.0,
                          1.0 / 40320.0,
                          1.0 / 362880.0,
                          1.0 / 3628800.0,
                          1.0 / 39916800.0,
                          1.0 / 479001600.0,
                          1.0 / 6227020800.0,
                          1.0 / 87178291200.0,
                          1.0 / 1307674368000.0,
                          1.0 / 20922789888000.0,
                          1.0 / 355687428096000.0,
                          1.0 / 6402373705728000.0,
                          1.0 / 121645100408832000.0,
                          1.0 / 2432902008176640000.0};
    return f[n];
}

// Weights of one segment of optical depth x followed by p.
//   e0 = 1 - e^{-x},  f1 = (x - e0)/x,  f2 = (x(2 - e0) - 2 e0)/x
//   parabolic: alpha = e0 - f1 - f2/(x+p), beta = f1 + f2/p, gamma = -x f2/(p (x+p))
//   linear:    alpha = e0 - f1,           beta = f1,         gamma = 0
// f1 and f2 are odd/even power series in x that cancel catastrophically when
// evaluated from e0 at small x; below the threshold they are summed directly
// (Horner), above it they come from expm1.
struct Coef64 {
    static constexpr int NS = 19;  // series terms for x < 0.5
    __device__ __forceinline__ static void eval(double x, double p, bool para, double &E, double &al, double &be,
                                                double &ga)
    {
        double e0, f1, f2;
        if (x < 0.5) {
            double h1 = 0.0, h2 = 0.0;
#pragma unroll
            for (int n = NS + 1; n >= 2; --n) h1 = inv_fact(n) - x * h1;        // sum (-x)^(n-2)/n!
#pragma unroll
            for (int m = NS + 1; m >= 3; --m) h2 = (double)(m - 2) * inv_fact(m) - x * h2;
            f1 = x * h1;
            f2 = (x * x) * h2;
            e0 = x - x * f1;
            E = 1.0 - e0;
        } else {
            double em = expm1(-x);
            e0 = -em;
            E = 1.0 + em;
            f1 = (x - e0) / x;
            f2 = (x * (2.0 - e0) - 2.0 * e0) / x;
        }
        if (para) {
            double iD = 1.0 / (x + p), ip = 1.0 / p;
            al = (e0 - f1) - f2 * iD;
            be = f1 + f2 * ip;
            ga = -(x * f2) * (ip * iD);
        } else {
            al = e0 - f1;
            be = f1;
            ga = 0.0;
        }
    }
};

// FP32 weights for the marches that evaluate them per segment (batch members,
// the full FP32 formal solution, chunked sweeps).  Below x = 1, f1 = x h1(x)
// and f2 = x^2 h2(x) with h1(x) = (e^{-x} - 1 + x)/x^2 = 1/2 - x/6 + x^2/24 - ...
// and h2(x) = f2(x)/x^2 = 1/6 - x/12 + x^2/40 - ... taken from degree-6
// polynomials fitted to those definitions on [0, 1] in the minimax sense of
// relative error (fit error 5e-10 for h1, 1.4e-9 for h2, under FP32 rounding);
// above, from the exponential as in Coef64.  Reciprocals are the hardware
// approximation (about one ulp), ample for FP32 weights.
struct Coef32 {
    __device__ __forceinline__ static float h1(float x)
    {
        float h = 1.687989424681291e-05f;
        h = fmaf(h, x, -1.8817881937138736e-04f);
        h = fmaf(h, x, 1.3820757158100605e-03f);
        h = fmaf(h, x, -8.330963551998138e-03f);
        h = fmaf(h, x, 4.1666269302368164e-02f);
        h = fmaf(h, x, -1.66666641831398e-01f);
        return fmaf(h, x, 0.5f);
    }
    __device__ __forceinline__ static float h2(float x)
    {
        float h = 1.2951083590451162e-05f;
        h = fmaf(h, x, -1.4058091619517654e-04f);
        h = fmaf(h, x, 9.86545579507947e-04f);
        h = fmaf(h, x, -5.553617607802153e-03f);
        h = fmaf(h, x, 2.4999670684337616e-02f);
        h = fmaf(h, x, -8.333331346511841e-02f);
        return fmaf(h, x, 1.666666716337204e-01f);
    }
    __device__ __forceinline__ static float rcp(float v) { return __fdividef(1.0f, v); }
    __device__ __forceinline__ static void eval(float x, float p, bool para, float &E, float &al, float &be, float &ga)
    {
        float e0, f1, f2;
        if (x < 1.0f) {
            f1 = x * h1(x);
            f2 = (x * x) * h2(x);
            e0 = x - x * f1;
            E = 1.0f - e0;
        } else {
            E = __expf(-x);
            e0 = 1.0f - E;
            const float ix = rcp(x);
            f1 = (x - e0) * ix;
            f2 = (x * (2.0f - e0) - 2.0f * e0) * ix;
        }
        if (para) {
            const float iD = rcp(x + p), ip = rcp(p);
            al = (e0 - f1) - f2 * iD;
            be = f1 + f2 * ip;
            ga = -(x * f2) * (ip * iD);
        } else {
            al = e0 - f1;
            be = f1;
            ga = 0.0f;
        }
    }
};

// Derivatives of (E, alpha, beta, gamma) with respect to x = dtau_k and
// p = dtau_{k+1}, from  e0' = E, f1' = (e0 - f1)/x = g1, f2' = e0 - f1 - f2/x = g2
// (g1, g2 summed as series below the threshold):
//   parabolic: alpha = e0 - f1 - f2/(x+p), beta = f1 + f2/p, gamma = -x f2/(p (x+p))
//   linear:    alpha = e0 - f1,           beta = f1
struct Coef64D {
    static constexpr int NS = 19;
    __device__ __forceinline__ static void eval(double x, double p, bool para, double &E, double &al, double &be,
                                                double &ga, double &dE, double &dal_x, double &dbe_x, double &dga_x,
                                                double &dal_p, double &dbe_p, double &dga_p)
    {
        double e0, f1, f2, g1, g2;
        if (x < 0.5) {
            double h1 = 0.0, h2 = 0.0, k1 = 0.0, k2 = 0.0;
#pragma unroll
            for (int n = NS + 1; n >= 2; --n) h1 = inv_fact(n) - x * h1;
#pragma unroll
            for (int m = NS + 1; m >= 3; --m) h2 = (double)(m - 2) * inv_fact(m) - x * h2;
            // g1 = sum_{n>=2} (-1)^n (n-1) x^(n-2) / n!,  g2 = sum_{m>=3} (-1)^(m+1) (m-2)(m-1) x^(m-2) / m!
#pragma unroll
            for (int n = NS + 1; n >= 2; --n) k1 = (double)(n - 1) * inv_fact(n) - x * k1;
#pragma unroll
            for (int m = NS + 1; m >= 3; --m) k2 = (double)((m - 2) * (m - 1)) * inv_fact(m) - x * k2;
            f1 = x * h1;
            f2 = (x * x) * h2;
            g1 = k1;
            g2 = x * k2;
            e0 = x - x * f1;
            E = 1.0 - e0;
        } else {
            double em = expm1(-x);
            e0 = -em;
            E = 1.0 + em;
            f1 = (x - e0) / x;
            f2 = (x * (2.0 - e0) - 2.0 * e0) / x;
            g1 = (e0 - f1) / x;
            g2 = e0 - f1 - f2 / x;
        }
        dE = -E;
        if (para) {
            const double D = x + p, iD = 1.0 / D, ip = 1.0 / p;
            al = (e0 - f1) - f2 * iD;
            be = f1 + f2 * ip;
            ga = -(x * f2) * (ip * iD);
            dal_x = E - g1 - g2 * iD + f2 * iD * iD;
            dal_p = f2 * iD * iD;
            dbe_x = g1 + g2 * ip;
            dbe_p = -f2 * ip * ip;
            dga_x = -(f2 * p + x * g2 * D) * (ip * iD * iD);
            dga_p = x * f2 * (x + 2.0 * p) * (ip * ip * iD * iD);
        } else {
            al = e0 - f1;
            be = f1;
            ga = 0.0;
            dal_x = E - g1;
            dbe_x = g1;
            dga_x = 0.0;
            dal_p = dbe_p = dga_p = 0.0;
        }
    }
};

}  // namespace rtk
