// tts_fastmath.cuh -- per-spin update of the fast engines (checkerboard and
// resident), shared by both.
//
// The sub-step map is the exact LLG flow (paper Eq. 1) under a field B held
// fixed for time h, written without tan(theta/2):  with b = B/|B|, c = s.b,
// s_perp = s - c b, q = b x s, phi = gamma'|B| h, x = alpha phi, E = e^{-2x},
//   D   = (1 + c) + (1 - c) E
//   c'  = ((1 + c) - (1 - c) E) / D          (= tanh(x + atanh c))
//   rho = 2 e^{-x} / D                       (= sin(theta') / sin(theta))
//   s'  = c' b + rho (cos(phi) s_perp + sin(phi) q)
// which follows from tan(theta'/2) = tan(theta/2) e^{-x} and precession by phi
// about +B; it needs no square root of |s_perp| and no branch at s_perp = 0.
#pragma once
#include <cuda_runtime.h>

#include "tts_philox.cuh"

namespace tts {

// sin and cos of a non-negative angle.  Below 0.25 rad (the usual sub-step
// angle is ~0.01-0.1 rad) Taylor polynomials through phi^7 / phi^8, whose
// truncation error is below 1e-10; above it the library sincosf.
__device__ __forceinline__ void small_sincos(float phi, float &s, float &c)
{
    if (phi < 0.25f) {
        const float p2 = phi * phi;
        s = phi * fmaf(p2, fmaf(p2, fmaf(p2, -1.0f / 5040.0f, 1.0f / 120.0f), -1.0f / 6.0f), 1.0f);
        c = fmaf(p2, fmaf(p2, fmaf(p2, fmaf(p2, 1.0f / 40320.0f, -1.0f / 720.0f), 1.0f / 24.0f), -0.5f), 1.0f);
    } else {
        sincosf(phi, &s, &c);
    }
}

template <typename R>
struct Fast;

template <>
struct Fast<float> {
    __device__ static float rsqrt_(float x) { return rsqrtf(x); }
    __device__ static float exp_(float x) { return __expf(x); }
    __device__ static float rcp_(float x) { return __fdividef(1.0f, x); }
    __device__ static void sincos_small(float x, float *s, float *c) { small_sincos(x, *s, *c); }
    // Box-Muller from one Philox block: (g1, g2) = sqrt(-2 ln u0) (cos, sin)(2 pi u1),
    // g3 = sqrt(-2 ln u2) cos(2 pi u3), with the angles shifted by pi into
    // (-pi, pi) for the hardware sine/cosine (cos(2 pi u) = -cos(2 pi (u - 1/2))).
    __device__ static void gauss3(const u32x4 &w, float &g1, float &g2, float &g3)
    {
        const float u0 = uniform_f(w.x), u1 = uniform_f(w.y), u2 = uniform_f(w.z), u3 = uniform_f(w.w);
        const float l0 = -2.0f * __logf(u0), l2 = -2.0f * __logf(u2);
        const float r01 = l0 * rsqrtf(l0), r23 = l2 * rsqrtf(l2);
        float s1, c1;
        __sincosf(6.28318530717958648f * (u1 - 0.5f), &s1, &c1);
        const float c3 = __cosf(6.28318530717958648f * (u3 - 0.5f));
        g1 = -r01 * c1;
        g2 = -r01 * s1;
        g3 = -r23 * c3;
    }
};

template <>
struct Fast<double> {
    __device__ static double rsqrt_(double x) { return 1.0 / sqrt(x); }
    __device__ static double exp_(double x) { return exp(x); }
    __device__ static double rcp_(double x) { return 1.0 / x; }
    __device__ static void sincos_small(double x, double *s, double *c) { sincos(x, s, c); }
    __device__ static void gauss3(const u32x4 &w, double &g1, double &g2, double &g3)
    {
        const double u0 = uniform_d(w.x), u1 = uniform_d(w.y), u2 = uniform_d(w.z), u3 = uniform_d(w.w);
        const double r01 = sqrt(-2.0 * log(u0)), r23 = sqrt(-2.0 * log(u2));
        double s1, c1, s3, c3;
        sincospi(2.0 * u1, &s1, &c1);
        sincospi(2.0 * u3, &s3, &c3);
        g1 = r01 * c1;
        g2 = r01 * s1;
        g3 = r23 * c3;
    }
};

// Constants of one species for the fast update (field already divided by mu).
template <typename R>
struct FastSpecies {
    R J0, J1;      // J(t_i, species 0) / mu_i, J(t_i, species 1) / mu_i   (tesla)
    R kappa;       // 2 K / mu_i (tesla)
    R alpha;
    R gprime;      // gamma / (1 + alpha^2)
};

// One sub-step of one spin: field from the neighbour sums (htot = sum of
// neighbour spins, h1 = sum over species-1 neighbours), anisotropy, Zeeman,
// noise sig * g, the midpoint anisotropy correction, the exact flow and
// renormalisation.  Returns the new spin in (sx, sy, sz).
// AXZ: the anisotropy axis is +z (n = (0, 0, 1)), which removes the
// general projections.
template <typename R, bool AXZ = false>
__device__ __forceinline__ void fast_update(R &sx, R &sy, R &sz, R htx, R hty, R htz, R h1x, R h1y, R h1z,
                                            const FastSpecies<R> &sp, R nx, R ny, R nz, R Bex, R Bey, R Bez,
                                            R sig, const u32x4 *noise, R h)
{
    using F = Fast<R>;
    if (AXZ) {
        nx = R(0);
        ny = R(0);
        nz = R(1);
    }
    const R dJ = sp.J1 - sp.J0;
    const R cn0 = AXZ ? sz : sx * nx + sy * ny + sz * nz;
    const R ka = sp.kappa * cn0;
    R Bx = AXZ ? sp.J0 * htx + dJ * h1x + Bex : sp.J0 * htx + dJ * h1x + ka * nx + Bex;
    R By = AXZ ? sp.J0 * hty + dJ * h1y + Bey : sp.J0 * hty + dJ * h1y + ka * ny + Bey;
    R Bz = AXZ ? sp.J0 * htz + dJ * h1z + ka + Bez : sp.J0 * htz + dJ * h1z + ka * nz + Bez;
    if (noise) {
        R g1, g2, g3;
        F::gauss3(*noise, g1, g2, g3);
        Bx += sig * g1;
        By += sig * g2;
        Bz += sig * g3;
    }
    // on-site anisotropy taken at the predicted sub-step midpoint
    if (AXZ) {
        const R n_sxB = sx * By - sy * Bx;
        const R sB = sx * Bx + sy * By + sz * Bz;
        Bz += sp.kappa * R(0.5) * h * (-sp.gprime * (n_sxB + sp.alpha * (cn0 * sB - Bz)));
    } else if (sp.kappa != R(0)) {
        const R cx = sy * Bz - sz * By, cy = sz * Bx - sx * Bz, cz = sx * By - sy * Bx;
        const R n_sxB = nx * cx + ny * cy + nz * cz;
        const R sB = sx * Bx + sy * By + sz * Bz;
        const R nB = nx * Bx + ny * By + nz * Bz;
        const R corr = sp.kappa * R(0.5) * h * (-sp.gprime * (n_sxB + sp.alpha * (cn0 * sB - nB)));
        Bx += corr * nx;
        By += corr * ny;
        Bz += corr * nz;
    }
    const R B2 = Bx * Bx + By * By + Bz * Bz;
    if (!(B2 > R(0))) return;
    const R rb = F::rsqrt_(B2);
    const R bx = Bx * rb, by = By * rb, bz = Bz * rb;
    const R Bm = B2 * rb;
    const R c = sx * bx + sy * by + sz * bz;
    const R px = sx - c * bx, py = sy - c * by, pz = sz - c * bz;
    const R qx = by * sz - bz * sy, qy = bz * sx - bx * sz, qz = bx * sy - by * sx;
    const R phi = sp.gprime * Bm * h;
    const R em = F::exp_(-sp.alpha * phi);
    const R E = em * em;
    const R opc = R(1) + c, omc = R(1) - c;
    const R iD = F::rcp_(opc + omc * E);
    const R cp = (opc - omc * E) * iD;
    const R rho = R(2) * em * iD;
    R sn, cs;
    F::sincos_small(phi, &sn, &cs);
    const R a = rho * cs, b = rho * sn;
    R ox = cp * bx + a * px + b * qx;
    R oy = cp * by + a * py + b * qy;
    R oz = cp * bz + a * pz + b * qz;
    const R on = F::rsqrt_(ox * ox + oy * oy + oz * oz);
    sx = ox * on;
    sy = oy * on;
    sz = oz * on;
}

}  // namespace tts
